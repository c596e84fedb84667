// C ABI of the D2V16-FFT-TLB library: simulation contexts, host-side tables and the
// orchestration of the four kernel passes of each Runge-Kutta stage (Sec. 2.3).
//
// A context holds nb >= 1 independent simulations of one grid size stacked along y: the row
// passes are row-local and treat them as one nx x (nb ny) grid, the column passes take the
// instance from grid.z. A batch (lbm_batch_*) groups instances of different sizes into
// contexts, one per size, whose steps run as parallel branches of one CUDA graph.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "lbm_internal.cuh"

using namespace lbm;

namespace {

thread_local std::string g_last_error;

int fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

#define CU_TRY(expr)                                                                                   \
    do {                                                                                               \
        cudaError_t e_ = (expr);                                                                       \
        if (e_ != cudaSuccess) return fail(LBM_ERR_CUDA, "%s: %s", #expr, cudaGetErrorString(e_));      \
    } while (0)

bool is_pow2(int n) { return n >= 2 && (n & (n - 1)) == 0; }

// Rows of the 16x16 matrix of moment functionals
// 1; v_x, v_y; psi; v_x v_x, v_x v_y, v_y v_y; psi v_x, psi v_y; v_x^3, v_x^2 v_y, v_x v_y^2, v_y^3;
// psi v_x^2, psi v_x v_y, psi v_y^2 (psi = v^2 + eta^2) evaluated on the 16 velocities.
void moment_rows(double eta0, double rows[16][16]) {
    for (int i = 0; i < 16; ++i) {
        const double vx = vel_x(i), vy = vel_y(i);
        const double psi = vel_sq(i) + (i < 4 ? eta0 * eta0 : 0.0);
        const double row[16] = {1.0,         vx,          vy,          psi,         vx * vx,     vx * vy,
                                vy * vy,     psi * vx,    psi * vy,    vx * vx * vx, vx * vx * vy, vx * vy * vy,
                                vy * vy * vy, psi * vx * vx, psi * vx * vy, psi * vy * vy};
        for (int r = 0; r < 16; ++r) rows[r][i] = row[r];
    }
}

// its inverse, by Gauss-Jordan elimination with partial pivoting
bool moment_inverse(double eta0, double out[256]) {
    double a[16][32], rows[16][16];
    moment_rows(eta0, rows);
    for (int r = 0; r < 16; ++r)
        for (int i = 0; i < 16; ++i) a[r][i] = rows[r][i];
    for (int r = 0; r < 16; ++r)
        for (int j = 0; j < 16; ++j) a[r][16 + j] = (r == j) ? 1.0 : 0.0;
    for (int col = 0; col < 16; ++col) {
        int piv = col;
        for (int r = col + 1; r < 16; ++r)
            if (std::fabs(a[r][col]) > std::fabs(a[piv][col])) piv = r;
        if (std::fabs(a[piv][col]) < 1e-12) return false;
        if (piv != col)
            for (int j = 0; j < 32; ++j) std::swap(a[piv][j], a[col][j]);
        const double inv = 1.0 / a[col][col];
        for (int j = 0; j < 32; ++j) a[col][j] *= inv;
        for (int r = 0; r < 16; ++r)
            if (r != col && a[r][col] != 0.0) {
                const double f = a[r][col];
                for (int j = 0; j < 32; ++j) a[r][j] -= f * a[col][j];
            }
    }
    for (int r = 0; r < 16; ++r)
        for (int j = 0; j < 16; ++j) out[r * 16 + j] = a[r][16 + j];
    return true;
}

}  // namespace

struct lbm_ctx {
    int nx = 0, ny = 0, lx = 0, ly = 0;  // ny: rows of one instance
    int nb = 1;                          // instances stacked along y
    long long n = 0;                     // nodes of one instance
    lbm_params p{};
    cudaStream_t stream = nullptr;
    int device = 0;
    bool mixed = false;
    bool rho64 = false;  // LBM_MIXED_RHO64: the density chain in float64 (r64, geo64)
    size_t fsize = 8;

    char *slab = nullptr;
    size_t slab_bytes = 0;
    // state and stage scratch in row-interleaved blocks (lbm_internal.cuh) over nb * ny rows;
    // element type double (LBM_FP64) or float (LBM_MIXED)
    void *f0 = nullptr, *f1 = nullptr;  // [nb ny][16][nx]: f^n (then f^{n+1}) and f^{n+1/2}
    void *Ay = nullptr;                 // [nb ny][12][nx]
    void *m = nullptr;                  // [nb ny][NF_M][nx]
    void *Ax = nullptr;                 // [nb ny][16][nx]: d_x f_i, only when geo.upd_ax
    double *r64 = nullptr;              // [nb ny][NR64][nx]: the float64 density chain (rho64 only)
    double *partial = nullptr;
    int diag_blocks = 0;
    // pipelined diagnostics (lbm_diagnostics_begin / _end): two pinned host slots, each the
    // per-block partial sums and the error word of one request, and a ring of pending requests
    double *hpart = nullptr;
    size_t dslot = 0;                 // doubles per slot: partial values, then the error word
    int dnparts[2] = {0, 0};          // partial values (blocks) in each slot
    cudaEvent_t dev_ev[2] = {nullptr, nullptr};
    long long dsteps[2] = {0, 0};
    int dhead = 0, dcount = 0;
    // a request fused into the next step: that step's first macro pass (which has the moments and
    // the density derivatives of the requested state at hand) writes the partial values to fpart,
    // one block per macro CTA; graph_diag is the step graph with that pass
    int fuse_slot = -1;
    int fuse_capture = -1;             // slot whose buffer the launches being issued write, or -1
    double *fpart[2] = {nullptr, nullptr};            // per slot: the fused partial values
    cudaGraphExec_t graph_diag[2] = {nullptr, nullptr};  // per slot: the step graph writing fpart[slot]
    cudaStream_t dstream = nullptr;   // copies of fused partial values, off the stepping stream
    cudaEvent_t fev[2] = {nullptr, nullptr};           // per slot: the fused step has written fpart
    int *err = nullptr;               // device error word of the bounded waits (tma::kErrTimeout)
    unsigned long long *bad = nullptr;  // lowest failing node of the last initial-field check
    long long wait_cycles = 1LL << 31;  // budget of one device-side wait (about a second)
    int starve = 0;                   // fault-injection hook (lbm_fault_inject)
    // per-axis tables
    double2 *tw64x = nullptr, *tw64y = nullptr;
    float2 *tw32x = nullptr, *tw32y = nullptr;
    double *k1x = nullptr, *k2x = nullptr, *k1y = nullptr, *k2y = nullptr;
    float *k1x32 = nullptr, *k2x32 = nullptr, *k1y32 = nullptr, *k2y32 = nullptr;
    double *kfx = nullptr, *kfy = nullptr;  // solution filter W(m) / N per axis (params filter_alpha > 0)
    float *kfx32 = nullptr, *kfy32 = nullptr;
    double minv[256];

    Geometry geo;    // launch geometry
    Geometry geo64;  // float64 launch geometry of the density chain's transforms (rho64 only)

    std::vector<char> initialized;  // per instance
    long long steps = 0;

    // one captured step (both stages) for lbm_step when timing is off
    cudaStream_t cap = nullptr;
    cudaGraphExec_t graph = nullptr;

    // per-launch timing
    bool timing = false;
    std::vector<cudaEvent_t> ev;
    std::vector<int> ev_cls;
    size_t ev_used = 0;

    bool all_initialized() const {
        for (char v : initialized)
            if (!v) return false;
        return true;
    }
    size_t row0(int k) const { return (size_t)k * ny; }  // first row of instance k
};

struct lbm_batch_ctx {
    std::vector<lbm_ctx *> groups;              // one context per grid size
    std::vector<std::pair<int, int>> where;      // instance -> (group, index in group)
    cudaStream_t stream = nullptr;
    cudaStream_t cap = nullptr;
    std::vector<cudaStream_t> branch;            // one capture stream per group
    std::vector<cudaEvent_t> join;
    cudaEvent_t fork = nullptr;
    cudaGraphExec_t graph = nullptr;
    std::vector<long long> steps;                // per instance, since its lbm_batch_init
    // persistent form (kernels_batch.cu): one launch per step over all instances
    int form = LBM_BATCH_GRAPH;
    cudaGraphExec_t pgraph = nullptr;            // memset of the control words + the persistent kernel
    int *bctrl = nullptr;                        // queue counter, abort flag, completion counters; then
    size_t bctrl_ints = 0;                       // the error word at bctrl[bctrl_ints]
    long long wait_cycles = 1LL << 31;
    int withhold = 0;
    int ptpb = 512;                              // threads per CTA of the persistent kernel (256 or 512)
};

namespace {

struct LaunchTimer {
    lbm_ctx *c;
    size_t slot = (size_t)-1;
    LaunchTimer(lbm_ctx *cc, int cls) : c(cc) {
        if (!c->timing) return;
        if (c->ev_used + 2 > c->ev.size()) {
            if (c->ev.size() >= (1u << 20)) return;
            for (int k = 0; k < 256; ++k) {
                cudaEvent_t e;
                if (cudaEventCreate(&e) != cudaSuccess) return;
                c->ev.push_back(e);
                c->ev_cls.push_back(0);
            }
        }
        slot = c->ev_used;
        c->ev_used += 2;
        c->ev_cls[slot] = cls;
        cudaEventRecord(c->ev[slot], c->stream);
    }
    ~LaunchTimer() {
        if (slot != (size_t)-1) cudaEventRecord(c->ev[slot + 1], c->stream);
    }
};

template <typename R> Axis<R> axis(const lbm_ctx *c, bool xdir);
template <> Axis<double> axis<double>(const lbm_ctx *c, bool xdir) {
    return xdir ? Axis<double>{c->tw64x, c->k1x, c->k2x, c->lx} : Axis<double>{c->tw64y, c->k1y, c->k2y, c->ly};
}
template <> Axis<float> axis<float>(const lbm_ctx *c, bool xdir) {
    return xdir ? Axis<float>{c->tw32x, c->k1x32, c->k2x32, c->lx}
                : Axis<float>{c->tw32y, c->k1y32, c->k2y32, c->ly};
}

template <typename R> ColArgs<R> col_args(const lbm_ctx *c, int nb, int W) {
    ColArgs<R> a{};
    a.nx = c->nx;
    a.ny = c->ny;
    a.W = W;
    a.log2W = log2_int(W);
    a.nb = nb;
    a.ay = axis<R>(c, false);
    return a;
}

// One stage of all instances: K_COL, K_MACRO, K_FLUX, K_UPDATE. stage 0 / 1: the two
// Runge-Kutta stages (f^{n+1/2} = f^n + dt/2 R(f^n) into f1; f^{n+1} = f^n + dt R(f^{n+1/2})
// into f0); stage 2: a forward Euler step f^{n+1} = f^n + dt R(f^n) in place in f0.
// pass selection for run_stage (all by default; the autotuner times them one at a time)
enum { PASS_COL = 1, PASS_MACRO = 2, PASS_FLUX = 4, PASS_UPDATE = 8, PASS_ALL = 15 };

// A column pass in the chosen form: the TMA-fed kernel, or direct loads (also where TMA cannot
// serve the shape: rows narrower than 16 bytes, misaligned fields)
template <typename R>
cudaError_t launch_col_pass(const lbm_ctx *c, const ColArgs<R> &a, int nj, int kind, size_t direct_smem) {
    if (kind == LBM_COL_TMA || kind == LBM_COL_TMA1) {
        const cudaError_t e =
            launch_col_tma<R>(a, nj, c->err, c->wait_cycles, c->starve, c->stream, kind == LBM_COL_TMA1 ? 1 : 2);
        if (e != cudaErrorNotSupported) return e;
        cudaGetLastError();
    }
    if (kind == LBM_COL_LOOKAHEAD && col_cluster(a.W, a.ay.log2n, sizeof(R)) == 1) {
        ColArgs<R> b = a;
        b.pf = 1;  // the launcher sets the distance
        return launch_col<R>(b, nj, direct_smem, c->stream);
    }
    return launch_col<R>(a, nj, direct_smem, c->stream);
}

// Arguments of the passes of one stage (stage 0 / 1: the two Runge-Kutta stages; 2: a forward
// Euler step in place), shared by the per-pass launches and the persistent batch kernel.
template <typename R> int column_jobs(const lbm_ctx *c, int stage, ColArgs<R> &a) {
    const lbm_params &p = c->p;
    const int nx = c->nx, ldf = NF_F * nx, lda = NF_A * nx, ldm = NF_M * nx;
    R *m = static_cast<R *>(c->m), *Ay = static_cast<R *>(c->Ay);
    const R *fs = static_cast<const R *>(stage == 1 ? c->f1 : c->f0);
    auto M = [m, nx](int k) { return m + (size_t)k * nx; };  // first row of macro field k
    int nj = 0;
    // Ay = -h v_iy d_y f_i: the stage's time step and the velocity folded into the multiplier
    const double hs = stage == 0 ? 0.5 * p.dt : p.dt;
    if (!(p.flags & LBM_FLAG_NO_ADVECTION))
        for (int k = 0; k < 12; ++k) {
            const int i = yfield(k);
            a.jobs[nj++] = ColJob<R>{fs + (size_t)i * nx, Ay + (size_t)k * nx, ldf, lda, 1, (R)(-hs * vel_y(i))};
        }
    if (!(p.flags & LBM_FLAG_NO_FORCE)) {
        if (!c->rho64) {  // (LBM_MIXED_RHO64: the float64 density chain instead)
            a.jobs[nj++] = ColJob<R>{M(M_RHO), M(M_RY), ldm, ldm, 1, R(1)};
            a.jobs[nj++] = ColJob<R>{M(M_RHO), M(M_RYY), ldm, ldm, 2, R(1)};
        }
        a.jobs[nj++] = ColJob<R>{M(M_UX), M(M_UXY), ldm, ldm, 1, R(1)};
        a.jobs[nj++] = ColJob<R>{M(M_UY), M(M_UYY), ldm, ldm, 1, R(1)};
        a.jobs[nj++] = ColJob<R>{M(M_T), M(M_TY), ldm, ldm, 1, R(1)};
    }
    return nj;
}

template <typename R> void flux_jobs(const lbm_ctx *c, ColArgs<R> &a) {
    const int nx = c->nx, ldm = NF_M * nx;
    R *m = static_cast<R *>(c->m);
    auto M = [m, nx](int k) { return m + (size_t)k * nx; };
    a.jobs[0] = ColJob<R>{M(M_QY), M(M_DQY), ldm, ldm, 1, R(1)};
    a.jobs[1] = ColJob<R>{M(M_SXY), M(M_DSXYY), ldm, ldm, 1, R(1)};
    a.jobs[2] = ColJob<R>{M(M_SYY), M(M_DSYY), ldm, ldm, 1, R(1)};
    a.jobs[3] = ColJob<R>{M(M_DIVU), M(M_DDIVUY), ldm, ldm, 1, R(1)};
}

template <typename R> MacroArgs<R> macro_args(const lbm_ctx *c, int rows_per_cta) {
    const lbm_params &p = c->p;
    MacroArgs<R> a{};
    a.m = static_cast<R *>(c->m);
    a.nx = c->nx;
    a.ny = c->nb * c->ny;
    a.rows = rows_per_cta;
    a.serial = c->geo.macro_serial ? 1 : 0;
    a.ax = axis<R>(c, true);
    a.K = (R)p.K; a.H = (R)p.H; a.q = (R)p.q; a.zeta = (R)p.zeta;
    a.K64 = p.K; a.H64 = p.H; a.q64 = p.q; a.zeta64 = p.zeta;
    a.r64 = c->rho64 ? c->r64 : nullptr;
    return a;
}

// LBM_MIXED_RHO64: rho of the stage's f as a float64 sum, then its derivatives by float64
// transforms: d_y rho, d_yy rho (one column launch) and d_x rho, d_xx rho (two row launches).
int run_rho64_chain(lbm_ctx *c, const float *fs) {
    const int nx = c->nx, rows = c->nb * c->ny, ld = NR64 * nx;
    double *r = c->r64;
    auto F = [r, nx](int k) { return r + (size_t)k * nx; };
    LaunchTimer t(c, LBM_K_RHO64);
    CU_TRY(launch_rho64(fs, r, nx, rows, c->stream));
    ColArgs<double> ca = col_args<double>(c, c->nb, c->geo64.colW);
    ca.jobs[0] = ColJob<double>{F(R64_RHO), F(R64_RY), ld, ld, 1, 1.0};
    ca.jobs[1] = ColJob<double>{F(R64_RHO), F(R64_RYY), ld, ld, 2, 1.0};
    CU_TRY(launch_col<double>(ca, 2, c->geo64.col_smem, c->stream));
    for (int order = 1; order <= 2; ++order) {
        RowDerivArgs<double> ra{};
        ra.in[0] = F(R64_RHO);
        ra.out[0] = F(order == 1 ? R64_RX : R64_RXX);
        ra.ld = ld;
        ra.nin = 1;
        ra.nx = nx;
        ra.ny = rows;
        ra.rows = c->geo64.rows_rowd;
        ra.order = order;
        ra.ax = axis<double>(c, true);
        CU_TRY(launch_row_deriv<double>(ra, c->geo64.rowd_smem, c->stream));
    }
    return LBM_OK;
}

template <typename R> UpdateArgs<R> update_args(const lbm_ctx *c, int stage, int rows_per_cta) {
    const lbm_params &p = c->p;
    const bool adv = !(p.flags & LBM_FLAG_NO_ADVECTION);
    R *f0 = static_cast<R *>(c->f0), *f1 = static_cast<R *>(c->f1);
    UpdateArgs<R> a{};
    a.fs = stage == 1 ? f1 : f0;
    a.Ax = (adv && c->geo.upd_ax) ? static_cast<const R *>(c->Ax) : nullptr;
    a.fbase = f0;
    a.fout = stage == 0 ? f1 : f0;  // stage 2 (Euler): in place, same node, same thread
    a.Ay = static_cast<const R *>(c->Ay);
    a.m = static_cast<R *>(c->m);
    a.nx = c->nx; a.ny = c->nb * c->ny; a.rows = rows_per_cta;
    a.cs = c->geo.upd_cs;
    a.ax = axis<R>(c, true);
    a.tau_inv = (R)(1.0 / p.tau);
    a.h = (R)(stage == 0 ? 0.5 * p.dt : p.dt);
    for (int q = 0; q < 6; ++q) a.cx[q] = (R)(-(stage == 0 ? 0.5 * p.dt : p.dt) * vel_x(xfield(2 * q)));
    a.T_iso = (R)p.T_iso;
    a.K = (R)p.K;
    a.b = (R)p.b;
    a.eta2 = (R)(p.eta0 * p.eta0);
    for (int i = 0; i < 16; ++i) {
        const double psi = vel_sq(i) + (i < 4 ? p.eta0 * p.eta0 : 0.0);
        a.k.psi_hi[i] = (R)psi;
        a.k.psi_lo[i] = (R)(psi - (double)a.k.psi_hi[i]);
    }
    a.flags = p.flags;
    for (int k = 0; k < 256; ++k) a.k.minv[k] = (R)c->minv[k];
    return a;
}

template <typename R>
int run_stage(lbm_ctx *c, int stage, int passes = PASS_ALL) {
    const lbm_params &p = c->p;
    const bool adv = !(p.flags & LBM_FLAG_NO_ADVECTION);
    const bool frc = !(p.flags & LBM_FLAG_NO_FORCE);
    const int nx = c->nx, rows = c->nb * c->ny;
    const R *fs = static_cast<const R *>(stage == 1 ? c->f1 : c->f0);
    const int ldf = NF_F * nx;
    {
        ColArgs<R> a = col_args<R>(c, c->nb, c->geo.colW);
        const int nj = column_jobs<R>(c, stage, a);
        if (nj && (passes & PASS_COL)) {
            LaunchTimer t(c, LBM_K_COL);
            CU_TRY(launch_col_pass<R>(c, a, nj, c->geo.col_kind, c->geo.col_smem));
        }
    }
    if constexpr (sizeof(R) == 4) {
        if (c->rho64 && frc && (passes & PASS_COL)) {
            const int rc = run_rho64_chain(c, reinterpret_cast<const float *>(fs));
            if (rc) return rc;
        }
    }
    if (frc && (passes & PASS_MACRO)) {
        MacroArgs<R> a = macro_args<R>(c, c->geo.rows_macro);
        const bool fused = c->fuse_capture >= 0 && stage != 1;
        if (fused) {  // the step's first macro pass: the state's diagnostics
            a.diag_partial = c->fpart[c->fuse_capture];
            a.diag_hK = (float)(0.5 * c->p.K);
        }
        {
            LaunchTimer t(c, LBM_K_MACRO);
            CU_TRY(launch_macro<R>(a, c->geo.macro_smem, c->stream));
        }
        // the partial values are ready here: their copy can start while the step goes on (in a
        // captured step an external event-record node, which streams outside the graph can wait on)
        if (fused) {
            cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
            CU_TRY(cudaStreamIsCapturing(c->stream, &cs));
            CU_TRY(cs == cudaStreamCaptureStatusActive
                       ? cudaEventRecordWithFlags(c->fev[c->fuse_capture], c->stream, cudaEventRecordExternal)
                       : cudaEventRecord(c->fev[c->fuse_capture], c->stream));
        }
    }
    if (frc && (passes & PASS_FLUX)) {
        ColArgs<R> a = col_args<R>(c, c->nb, c->geo.fluxW);
        flux_jobs<R>(c, a);
        LaunchTimer t(c, LBM_K_FLUX);
        CU_TRY(launch_col_pass<R>(c, a, 4, c->geo.flux_kind, c->geo.flux_smem));
    }
    if ((passes & PASS_UPDATE) && adv && c->geo.upd_ax) {
        // d_x f_i of the 12 fields with v_x != 0 into Ax, two fields per complex line
        for (int k = 0; k < 12; k += 2) {
            RowDerivArgs<R> ra{};
            ra.in[0] = fs + (size_t)xfield(k) * nx;
            ra.in[1] = fs + (size_t)xfield(k + 1) * nx;
            ra.out[0] = static_cast<R *>(c->Ax) + (size_t)xfield(k) * nx;
            ra.out[1] = static_cast<R *>(c->Ax) + (size_t)xfield(k + 1) * nx;
            ra.ld = ldf;
            ra.nin = 2;
            ra.nx = nx;
            ra.ny = rows;
            ra.rows = c->geo.rows_rowd;
            ra.order = 1;
            ra.ax = axis<R>(c, true);
            LaunchTimer t(c, LBM_K_UPDATE);
            CU_TRY(launch_row_deriv<R>(ra, c->geo.rowd_smem, c->stream));
        }
    }
    if (passes & PASS_UPDATE) {
        const UpdateArgs<R> a = update_args<R>(c, stage, c->geo.rows_upd);
        LaunchTimer t(c, LBM_K_UPDATE);
        CU_TRY(launch_update<R>(a, c->geo.upd_smem, c->stream));
    }
    return LBM_OK;
}

// The solution filter (params filter_alpha > 0): f_i <- the inverse transform of W(m_x) W(m_y)
// times the spectrum of f_i for all 16 fields in place, as a row pass (launches of four or two
// fields) and a column pass (16 jobs), each adding the transform of the correction W - 1 to the
// field, then the moments of the filtered f for the next step.
template <typename R> Axis<R> filter_axis(const lbm_ctx *c, bool xdir);
template <> Axis<double> filter_axis<double>(const lbm_ctx *c, bool xdir) {
    return xdir ? Axis<double>{c->tw64x, c->k1x, c->kfx, c->lx} : Axis<double>{c->tw64y, c->k1y, c->kfy, c->ly};
}
template <> Axis<float> filter_axis<float>(const lbm_ctx *c, bool xdir) {
    return xdir ? Axis<float>{c->tw32x, c->k1x32, c->kfx32, c->lx} : Axis<float>{c->tw32y, c->k1y32, c->kfy32, c->ly};
}

template <typename R> int run_filter(lbm_ctx *c) {
    const int nx = c->nx, rows = c->nb * c->ny, ldf = NF_F * nx;
    R *f = static_cast<R *>(c->f0);
    // four fields (two lines per row) per launch where the threads allow it, else two
    const int per = 2 * c->geo.rows_rowd * line_G(c->lx) <= max_threads(c->fsize) ? 4 : 2;
    for (int k = 0; k < 16; k += per) {
        RowDerivArgs<R> ra{};
        for (int j = 0; j < per; ++j) {
            ra.in[j] = f + (size_t)(k + j) * nx;
            ra.out[j] = f + (size_t)(k + j) * nx;
        }
        ra.ld = ldf;
        ra.nin = per;
        ra.nx = nx;
        ra.ny = rows;
        ra.rows = c->geo.rows_rowd;
        ra.order = 2;
        ra.acc = 1;
        ra.ax = filter_axis<R>(c, true);
        LaunchTimer t(c, LBM_K_UPDATE);
        CU_TRY(launch_row_deriv<R>(ra, (per / 2) * c->geo.rowd_smem, c->stream));
    }
    ColArgs<R> a = col_args<R>(c, c->nb, c->geo.colW);
    a.ay = filter_axis<R>(c, false);
    for (int i = 0; i < 16; ++i) a.jobs[i] = ColJob<R>{f + (size_t)i * nx, f + (size_t)i * nx, ldf, ldf, 2, R(1), 1};
    {
        LaunchTimer t(c, LBM_K_COL);
        CU_TRY(launch_col<R>(a, 16, c->geo.col_smem, c->stream));
    }
    MomArgs ma{};
    ma.f = f;
    ma.m = c->m;
    ma.nx = nx;
    ma.ny = rows;
    ma.b = c->p.b;
    ma.T_iso = (c->p.flags & LBM_FLAG_ISOTHERMAL) ? c->p.T_iso : 0.0;
    for (int i = 0; i < 16; ++i) ma.psi[i] = vel_sq(i) + (i < 4 ? c->p.eta0 * c->p.eta0 : 0.0);
    LaunchTimer t(c, LBM_K_UPDATE);
    CU_TRY(launch_moments<R>(ma, c->stream));
    return LBM_OK;
}

int run_step_launches(lbm_ctx *c) {
    int rc = LBM_OK;
    if (c->p.flags & LBM_FLAG_EULER) {
        rc = c->mixed ? run_stage<float>(c, 2) : run_stage<double>(c, 2);
    } else {
        for (int st = 0; st < 2 && rc == LBM_OK; ++st) rc = c->mixed ? run_stage<float>(c, st) : run_stage<double>(c, st);
    }
    if (rc == LBM_OK && c->p.filter_alpha > 0) rc = c->mixed ? run_filter<float>(c) : run_filter<double>(c);
    return rc;
}

// Captures one step of the context (launches on `s`, then restores its stream) into a graph.
int capture_into(lbm_ctx *c, cudaStream_t s) {
    cudaStream_t saved = c->stream;
    c->stream = s;
    const int rc = run_step_launches(c);
    c->stream = saved;
    return rc;
}

// One step's launches as a CUDA graph: c->graph, or for a fused diagnostics request in slot
// `slot` (>= 0) c->graph_diag[slot], whose first macro pass also writes the diagnostics partial
// values into fpart[slot].
int build_step_graph(lbm_ctx *c, int slot = -1) {
    if (!c->cap) CU_TRY(cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking));
    CU_TRY(cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeRelaxed));
    c->fuse_capture = slot;
    const int rc = capture_into(c, c->cap);
    c->fuse_capture = -1;
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(c->cap, &g);
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    CU_TRY(e);
    const cudaError_t ei = cudaGraphInstantiate(slot >= 0 ? &c->graph_diag[slot] : &c->graph, g, 0);
    cudaGraphDestroy(g);
    CU_TRY(ei);
    return LBM_OK;
}

// Drops the step graphs (recaptured at the next step, e.g. with new launch shapes).
void drop_graphs(lbm_ctx *c) {
    if (c->graph) cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
    for (cudaGraphExec_t &g : c->graph_diag) {
        if (g) cudaGraphExecDestroy(g);
        g = nullptr;
    }
}

// ---- autotuner: tile and CTA shapes by measurement ------------------------------------

// Candidate column tile widths: W columns (W/2 complex lines of G threads) with at most
// pass_threads threads per CTA, lines split over a cluster of 2 or 4 CTAs where they need more
// (col_cluster), and at most 100 KB of line buffers per CTA.
std::vector<int> col_candidates(const lbm_ctx *c) {
    std::vector<int> out;
    for (int W = 2; W <= c->nx && W * (int)c->fsize <= 256; W *= 2)
        if (col_cluster(W, c->ly, c->fsize) > 0 && col_smem(W, c->ly, c->fsize) <= 100 * 1024) out.push_back(W);
    return out;
}
// Whether the TMA-fed column kernel can take tiles of W columns with `kind`'s staging buffers
// (LBM_COL_TMA: two, LBM_COL_TMA1: one): rows of at least 16 bytes, aligned field rows, the
// buffers within a CTA's shared memory.
bool col_tma_ok(const lbm_ctx *c, int W, int kind) {
    const size_t sm = col_tma_smem(c->nx, c->ny, W, c->fsize, kind == LBM_COL_TMA1 ? 1 : 2);
    return col_cluster(W, c->ly, c->fsize) == 1 && sm > 0 && sm <= kMaxCtaSmem && (c->nx * c->fsize) % 16 == 0;
}
// Whether the direct column kernel can prefetch tiles of W columns row by row: rows of at least
// 16 bytes (the bulk prefetch granule), whole lines in one CTA.
bool col_lookahead_ok(const lbm_ctx *c, int W) {
    return col_cluster(W, c->ly, c->fsize) == 1 && W * c->fsize >= 16 && (c->nx * c->fsize) % 16 == 0;
}
// Whether a cluster of cs CTAs may split the update pass's rows: float32 rows of 2048 or more
// in two, of 4096 in four.
bool upd_split_ok(const lbm_ctx *c, int cs) {
    return c->fsize == 4 && !c->geo.upd_ax && ((cs == 2 && c->lx >= 11) || (cs == 4 && c->lx >= 12));
}
// Candidate rows per CTA of the update pass (6 line buffers per row within a CTA's shared memory).
std::vector<int> upd_candidates(const lbm_ctx *c) {
    std::vector<int> out;
    const size_t SM = (size_t)line_smem(c->lx) * 2 * c->fsize;
    for (int r = 1; r <= c->ny && r * c->nx <= 4096; r *= 2)
        if (6 * r * SM <= kMaxCtaSmem) out.push_back(r);
    return out;
}
// Candidate rows per CTA of the macro pass (two lines per row within its thread bound).
std::vector<int> macro_candidates(const lbm_ctx *c) {
    std::vector<int> out;
    for (int r = 1; r <= c->ny && r * c->nx <= 4096; r *= 2)
        if (2 * r * line_G(c->lx) <= macro_threads(c->fsize, c->lx) && macro_smem(r, c->lx, c->fsize) <= kMaxCtaSmem)
            out.push_back(r);
    return out;
}

template <typename R> int run_stage(lbm_ctx *c, int stage, int passes);

// Times one whole step as lbm_step runs it (the step's launches captured into a CUDA graph):
// one untimed launch, then the mean of three, each after a write of `flush_bytes` to `flush`
// (larger than L2, so every step starts from a cold cache, as in a long run of steps whose
// working set exceeds L2; a working set that fits L2 would otherwise favour shapes that only
// win when their inputs are already cached). The whole step is timed because a pass's shape
// also changes what it leaves in L2 for the next pass. The steps advance the state, which the
// caller saves and restores.
int time_step(lbm_ctx *c, void *flush, size_t flush_bytes, cudaEvent_t e0, cudaEvent_t e1, float *ms) {
    drop_graphs(c);
    int rc = build_step_graph(c);
    if (rc) return rc;
    CU_TRY(cudaGraphLaunch(c->graph, c->stream));
    float sum = 0.0f;
    for (int k = 0; k < 3; ++k) {
        if (flush) CU_TRY(cudaMemsetAsync(flush, k, flush_bytes, c->stream));
        CU_TRY(cudaEventRecord(e0, c->stream));
        CU_TRY(cudaGraphLaunch(c->graph, c->stream));
        CU_TRY(cudaEventRecord(e1, c->stream));
        CU_TRY(cudaEventSynchronize(e1));
        float t = 0.0f;
        CU_TRY(cudaEventElapsedTime(&t, e0, e1));
        sum += t;
    }
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
    *ms = sum / 3.0f;
    return LBM_OK;
}

// Chooses the column pass forms and tile widths, the macro pass's rows per CTA and the update
// pass's split and rows per CTA by timing whole steps with every candidate, one pass's shape at
// a time (the others at their current choice). The distributions f^n and the moment fields
// are saved first and restored at the end, so the state is unchanged; the other buffers are
// scratch of a step. Per-row and per-column work does not depend on these shapes, so results
// stay bit for bit the same.
template <typename R> int autotune_impl(lbm_ctx *c, float best_ms[4]) {
    const bool timing = c->timing;
    c->timing = false;
    const size_t es = c->fsize, rows = (size_t)c->nb * c->ny, fbytes = rows * NF_F * c->nx * es;
    void *save = nullptr, *save_f = nullptr, *flush = nullptr;
    size_t flush_bytes = 0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = LBM_OK;
    const Geometry geo0 = c->geo;
    bool saved = false;
    auto restore = [&]() {
        cudaError_t e = cudaMemcpy2DAsync(c->m, NF_M * c->nx * es, save, 4 * c->nx * es, 4 * c->nx * es, rows,
                                          cudaMemcpyDeviceToDevice, c->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(c->f0, save_f, fbytes, cudaMemcpyDeviceToDevice, c->stream);
        return e;
    };
    auto done = [&](int code) {
        if (code != LBM_OK) {  // failed midway: the previous shapes and, if possible, the state
            c->geo = geo0;
            if (saved) restore();
            cudaStreamSynchronize(c->stream);
        }
        drop_graphs(c);  // recaptured with the chosen shapes at the next step
        if (save) cudaFree(save);
        if (save_f) cudaFree(save_f);
        if (flush) cudaFree(flush);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        c->timing = timing;
        return code;
    };
    if (cudaMalloc(&save, 4 * c->nx * es * rows) != cudaSuccess || cudaMalloc(&save_f, fbytes) != cudaSuccess) {
        cudaGetLastError();
        return done(fail(LBM_ERR_NOMEM, "autotune: no scratch for the state"));
    }
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return done(fail(LBM_ERR_CUDA, "autotune: cudaEventCreate failed"));
    {  // L2 flush buffer: twice the L2 size (without it, the timings are taken warm)
        int dev = 0, l2 = 0;
        if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) == cudaSuccess &&
            l2 > 0 && cudaMalloc(&flush, 2 * (size_t)l2) == cudaSuccess)
            flush_bytes = 2 * (size_t)l2;
        else
            flush = nullptr, cudaGetLastError();
    }
    // moment fields M_RHO..M_T: 4 nx contiguous elements per row of the macroscopic block
    if (cudaMemcpy2DAsync(save, 4 * c->nx * es, c->m, NF_M * c->nx * es, 4 * c->nx * es, rows,
                          cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess ||
        cudaMemcpyAsync(save_f, c->f0, fbytes, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess)
        return done(fail(LBM_ERR_CUDA, "autotune: saving the state failed"));
    saved = true;
    const bool frc = !(c->p.flags & LBM_FLAG_NO_FORCE);

    float t = 0;
    // column tile widths and forms of the column pass and of the flux column pass
    for (int pass : {PASS_COL, PASS_FLUX}) {
        if (pass == PASS_FLUX && !frc) continue;
        int &Wg = pass == PASS_COL ? c->geo.colW : c->geo.fluxW;
        size_t &Sg = pass == PASS_COL ? c->geo.col_smem : c->geo.flux_smem;
        int &Kg = pass == PASS_COL ? c->geo.col_kind : c->geo.flux_kind;
        int bestW = Wg, bestK = Kg;
        float bt = 1e30f;
        for (int kind : {LBM_COL_DIRECT, LBM_COL_TMA, LBM_COL_LOOKAHEAD, LBM_COL_TMA1}) {
            for (int W : col_candidates(c)) {
                if ((kind == LBM_COL_TMA || kind == LBM_COL_TMA1) && !col_tma_ok(c, W, kind)) continue;
                if (kind == LBM_COL_LOOKAHEAD && !col_lookahead_ok(c, W)) continue;
                Wg = W;
                Kg = kind;
                Sg = col_smem(W, c->ly, es);
                if ((rc = time_step(c, flush, flush_bytes, e0, e1, &t))) return done(rc);
                if (t < bt) bt = t, bestW = W, bestK = kind;
            }
        }
        Wg = bestW;
        Kg = bestK;
        Sg = col_smem(bestW, c->ly, es);
        best_ms[pass == PASS_COL ? 0 : 3] = bt;
    }
    best_ms[1] = 0;
    if (frc && !c->geo.macro_serial) {
        int bestr = c->geo.rows_macro;
        float bt = 1e30f;
        for (int r : macro_candidates(c)) {
            c->geo.rows_macro = r;
            c->geo.macro_smem = macro_smem(r, c->lx, es);
            if ((rc = time_step(c, flush, flush_bytes, e0, e1, &t))) return done(rc);
            if (t < bt) bt = t, bestr = r;
        }
        c->geo.rows_macro = bestr;
        c->geo.macro_smem = macro_smem(bestr, c->lx, es);
        best_ms[1] = bt < 1e30f ? bt : 0.0f;
    }
    best_ms[2] = 0;
    if (!c->geo.upd_ax) {
        int bestr = c->geo.rows_upd, bestcs = c->geo.upd_cs;
        float bt = 1e30f;
        for (int cs : {1, 2, 4}) {
            if (cs > 1 && !upd_split_ok(c, cs)) continue;
            for (int r : upd_candidates(c)) {
                if (cs > 1 && r != 1) continue;
                c->geo.rows_upd = r;
                c->geo.upd_cs = cs;
                c->geo.upd_smem = upd_smem(r, c->lx, es, cs);
                if ((rc = time_step(c, flush, flush_bytes, e0, e1, &t))) return done(rc);
                if (t < bt) bt = t, bestr = r, bestcs = cs;
            }
        }
        c->geo.rows_upd = bestr;
        c->geo.upd_cs = bestcs;
        c->geo.upd_smem = upd_smem(bestr, c->lx, es, bestcs);
        best_ms[2] = bt < 1e30f ? bt : 0.0f;
    }
    saved = false;  // restored here, on success as on failure
    if (restore() != cudaSuccess) return done(fail(LBM_ERR_CUDA, "autotune: restoring the state failed"));
    if (cudaStreamSynchronize(c->stream) != cudaSuccess)
        return done(fail(LBM_ERR_CUDA, "autotune: %s", cudaGetErrorString(cudaGetLastError())));
    return done(LBM_OK);
}

int autotune_ctx(lbm_ctx *c, float best_ms[4]) {
    if (!c->all_initialized()) return fail(LBM_ERR_STATE, "autotune needs an initialised state");
    return c->mixed ? autotune_impl<float>(c, best_ms) : autotune_impl<double>(c, best_ms);
}

int check_params(const lbm_params *p) {
    if (!p) return fail(LBM_ERR_ARG, "params is NULL");
    const double v[] = {p->tau, p->dt, p->dx, p->dy, p->K, p->H, p->q, p->zeta, p->b, p->eta0,
                        p->win_alpha, p->win_p};
    for (double x : v)
        if (!std::isfinite(x)) return fail(LBM_ERR_ARG, "non-finite parameter");
    if (p->tau <= 0 || p->dt <= 0 || p->dx <= 0 || p->dy <= 0 || p->b <= 0)
        return fail(LBM_ERR_ARG, "tau, dt, dx, dy and b must be positive");
    if (p->win_alpha < 0 || p->win_p <= 0) return fail(LBM_ERR_ARG, "need win_alpha >= 0 and win_p > 0");
    if (!std::isfinite(p->filter_alpha) || !std::isfinite(p->filter_p) || p->filter_alpha < 0 || p->filter_p <= 0)
        return fail(LBM_ERR_ARG, "need finite filter_alpha >= 0 and filter_p > 0");
    if (p->precision != LBM_FP64 && p->precision != LBM_MIXED && p->precision != LBM_MIXED_RHO64)
        return fail(LBM_ERR_ARG, "precision must be LBM_FP64, LBM_MIXED or LBM_MIXED_RHO64");
    if (p->flags & ~(LBM_FLAG_NO_ADVECTION | LBM_FLAG_NO_COLLISION | LBM_FLAG_NO_FORCE | LBM_FLAG_EULER |
                     LBM_FLAG_ISOTHERMAL))
        return fail(LBM_ERR_ARG, "unknown flag bits");
    if (p->keff_terms < 1 || p->keff_terms > 8) return fail(LBM_ERR_ARG, "keff_terms must be in [1, 8]");
    if ((p->flags & LBM_FLAG_ISOTHERMAL) && !(std::isfinite(p->T_iso) && p->T_iso > 0))
        return fail(LBM_ERR_ARG, "LBM_FLAG_ISOTHERMAL needs a finite T_iso > 0");
    return LBM_OK;
}

void free_ctx(lbm_ctx *c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    else cudaDeviceSynchronize();
    if (c->dstream) cudaStreamSynchronize(c->dstream);
    if (c->graph) cudaGraphExecDestroy(c->graph);
    for (int k = 0; k < 2; ++k) {
        if (c->graph_diag[k]) cudaGraphExecDestroy(c->graph_diag[k]);
        if (c->fpart[k]) cudaFree(c->fpart[k]);
        if (c->fev[k]) cudaEventDestroy(c->fev[k]);
    }
    if (c->dstream) cudaStreamDestroy(c->dstream);
    if (c->cap) cudaStreamDestroy(c->cap);
    for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
    for (cudaEvent_t e : c->dev_ev)
        if (e) cudaEventDestroy(e);
    if (c->hpart) cudaFreeHost(c->hpart);
    cudaFree(c->slab);
    delete c;
}

// nb instances of nx x ny, all device memory in one slab
int create_ctx(int nx, int ny, int nb, const lbm_params *params, cudaStream_t stream, lbm_ctx **out) {
    *out = nullptr;
    if (!is_pow2(nx) || !is_pow2(ny) || nx > 4096 || ny > 4096)
        return fail(LBM_ERR_ARG, "nx=%d, ny=%d: each must be a power of two in [2, 4096]", nx, ny);
    // instances: grid.z of the column passes (<= 65535), rows of the row passes (< 2^31 CTAs)
    if (nb < 1 || nb > 65535 || (long long)nb * ny > (1LL << 24))
        return fail(LBM_ERR_ARG, "%d instances of %d x %d: need 1 <= count <= 65535 and count * ny <= 2^24", nb, nx,
                    ny);
    int rc = check_params(params);
    if (rc) return rc;

    lbm_ctx *c = new (std::nothrow) lbm_ctx();
    if (!c) return fail(LBM_ERR_NOMEM, "host allocation failed");
    c->nx = nx;
    c->ny = ny;
    c->nb = nb;
    c->lx = log2_int(nx);
    c->ly = log2_int(ny);
    c->n = (long long)nx * ny;
    c->p = *params;
    c->stream = stream;
    c->mixed = params->precision != LBM_FP64;
    c->rho64 = params->precision == LBM_MIXED_RHO64;
    c->fsize = c->mixed ? 4 : 8;
    c->initialized.assign(nb, 0);
    if (cudaGetDevice(&c->device) != cudaSuccess) {
        delete c;
        return fail(LBM_ERR_CUDA, "no CUDA device");
    }
    if (!moment_inverse(params->eta0, c->minv)) {
        delete c;
        return fail(LBM_ERR_ARG, "moment matrix is singular for eta0=%g", params->eta0);
    }

    // launch geometry
    int smem_optin = 0;
    cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device);
    pass_geometry(nx, ny, c->fsize, &c->geo);
    size_t need =
        std::max(std::max(c->geo.upd_smem, c->geo.macro_smem), std::max(c->geo.col_smem, c->geo.rowd_smem));  // flux = col
    if (c->rho64) {  // the density chain's float64 column and row transforms
        pass_geometry(nx, ny, 8, &c->geo64);
        need = std::max(need, std::max(c->geo64.col_smem, c->geo64.rowd_smem));
    }
    if (need > (size_t)smem_optin) {
        delete c;
        return fail(LBM_ERR_UNSUPPORTED, "nx=%d ny=%d needs %zu B of shared memory per block (device: %d)", nx,
                    ny, need, smem_optin);
    }

    // device memory: one slab, 256-byte aligned pieces
    const size_t plane_f = (size_t)c->n * nb * c->fsize;
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    c->diag_blocks = (int)std::min<long long>(1024, (c->n + 255) / 256);
    size_t off = 0;
    std::vector<std::pair<void **, size_t>> parts;
    parts.push_back({&c->f0, 16 * plane_f});
    parts.push_back({&c->f1, 16 * plane_f});
    parts.push_back({&c->Ay, 12 * plane_f});
    parts.push_back({&c->m, (size_t)NF_M * plane_f});
    if (c->geo.upd_ax) parts.push_back({&c->Ax, 16 * plane_f});
    if (c->rho64) parts.push_back({reinterpret_cast<void **>(&c->r64), (size_t)NR64 * c->n * nb * sizeof(double)});
    parts.push_back({reinterpret_cast<void **>(&c->partial), (size_t)c->diag_blocks * 5 * 8});
    parts.push_back({reinterpret_cast<void **>(&c->err), sizeof(int)});
    parts.push_back({reinterpret_cast<void **>(&c->bad), sizeof(unsigned long long)});
    parts.push_back({reinterpret_cast<void **>(&c->tw64x), (size_t)nx * 16});
    parts.push_back({reinterpret_cast<void **>(&c->tw64y), (size_t)ny * 16});
    parts.push_back({reinterpret_cast<void **>(&c->tw32x), (size_t)nx * 8});
    parts.push_back({reinterpret_cast<void **>(&c->tw32y), (size_t)ny * 8});
    parts.push_back({reinterpret_cast<void **>(&c->k1x), (size_t)nx * 8});
    parts.push_back({reinterpret_cast<void **>(&c->k2x), (size_t)nx * 8});
    parts.push_back({reinterpret_cast<void **>(&c->k1y), (size_t)ny * 8});
    parts.push_back({reinterpret_cast<void **>(&c->k2y), (size_t)ny * 8});
    parts.push_back({reinterpret_cast<void **>(&c->k1x32), (size_t)nx * 4});
    parts.push_back({reinterpret_cast<void **>(&c->k2x32), (size_t)nx * 4});
    parts.push_back({reinterpret_cast<void **>(&c->k1y32), (size_t)ny * 4});
    parts.push_back({reinterpret_cast<void **>(&c->k2y32), (size_t)ny * 4});
    parts.push_back({reinterpret_cast<void **>(&c->kfx), (size_t)nx * 8});
    parts.push_back({reinterpret_cast<void **>(&c->kfy), (size_t)ny * 8});
    parts.push_back({reinterpret_cast<void **>(&c->kfx32), (size_t)nx * 4});
    parts.push_back({reinterpret_cast<void **>(&c->kfy32), (size_t)ny * 4});
    for (auto &pp : parts) off += al(pp.second);
    if (cudaMalloc(&c->slab, off) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return fail(LBM_ERR_NOMEM, "cudaMalloc of %zu bytes failed", off);
    }
    c->slab_bytes = off;
    off = 0;
    for (auto &pp : parts) {
        *pp.first = c->slab + off;
        off += al(pp.second);
    }

    // tables: twiddles on the device (sincospi), multipliers on the host (Eq. (3))
    cudaError_t e = cudaMemsetAsync(c->err, 0, sizeof(int), c->stream);
    if (e == cudaSuccess) e = launch_twiddles(c->tw64x, c->tw32x, nx, c->stream);
    if (e == cudaSuccess) e = launch_twiddles(c->tw64y, c->tw32y, ny, c->stream);
    for (int ax = 0; ax < 2 && e == cudaSuccess; ++ax) {
        const int N = ax == 0 ? nx : ny;
        const double d = ax == 0 ? params->dx : params->dy;
        std::vector<double> k1(N), k2(N);
        std::vector<float> k1f(N), k2f(N);
        derivative_tables(N, d, params->win_alpha, params->win_p, k1.data(), k2.data(), params->keff_terms);
        for (int pos = 0; pos < N; ++pos) {
            k1f[pos] = (float)k1[pos];
            k2f[pos] = (float)k2[pos];
        }
        double *dk1 = ax == 0 ? c->k1x : c->k1y, *dk2 = ax == 0 ? c->k2x : c->k2y;
        float *fk1 = ax == 0 ? c->k1x32 : c->k1y32, *fk2 = ax == 0 ? c->k2x32 : c->k2y32;
        e = cudaMemcpy(dk1, k1.data(), N * 8, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(dk2, k2.data(), N * 8, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(fk1, k1f.data(), N * 4, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(fk2, k2f.data(), N * 4, cudaMemcpyHostToDevice);
        // the solution filter's table (unused while filter_alpha = 0)
        std::vector<double> kf(N);
        std::vector<float> kff(N);
        filter_table(N, params->filter_alpha, params->filter_p, kf.data());
        for (int pos = 0; pos < N; ++pos) kff[pos] = (float)kf[pos];
        if (e == cudaSuccess) e = cudaMemcpy(ax == 0 ? c->kfx : c->kfy, kf.data(), N * 8, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(ax == 0 ? c->kfx32 : c->kfy32, kff.data(), N * 4, cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        cudaFree(c->slab);
        delete c;
        return fail(LBM_ERR_CUDA, "table setup: %s", cudaGetErrorString(e));
    }
    *out = c;
    return LBM_OK;
}

// After a synchronisation of the context's stream: the error word of the bounded device
// waits. A set word is reported once (and cleared) as LBM_ERR_TIMEOUT.
int check_device_error(lbm_ctx *c) {
    int v = 0;
    CU_TRY(cudaMemcpyAsync(&v, c->err, sizeof v, cudaMemcpyDeviceToHost, c->stream));
    CU_TRY(cudaStreamSynchronize(c->stream));
    if (v == 0) return LBM_OK;
    CU_TRY(cudaMemsetAsync(c->err, 0, sizeof v, c->stream));
    CU_TRY(cudaStreamSynchronize(c->stream));
    return fail(LBM_ERR_TIMEOUT, "a bounded device-side wait gave up (error word %d): the steps since the last "
                "check did not complete and the state is not valid",
                v);
}

// f_i := f_i^eq(rho, u, T) for instance k from device arrays [ny][nx]
int init_instance(lbm_ctx *c, int k, const double *rho, const double *ux, const double *uy, const double *T) {
    InitArgs a{};
    a.rho = rho; a.ux = ux; a.uy = uy; a.T = T;
    a.f = static_cast<char *>(c->f0) + c->row0(k) * NF_F * c->nx * c->fsize;
    a.m = static_cast<char *>(c->m) + c->row0(k) * NF_M * c->nx * c->fsize;
    a.nx = c->nx;
    a.ny = c->ny;
    a.b = c->p.b;
    a.T_iso = (c->p.flags & LBM_FLAG_ISOTHERMAL) ? c->p.T_iso : 0.0;
    for (int j = 0; j < 256; ++j) a.minv[j] = c->minv[j];
    for (int i = 0; i < 16; ++i) a.psi[i] = vel_sq(i) + (i < 4 ? c->p.eta0 * c->p.eta0 : 0.0);
    CU_TRY(c->mixed ? launch_init<float>(a, c->stream) : launch_init<double>(a, c->stream));
    c->initialized[k] = 1;
    c->steps = 0;
    return LBM_OK;
}

int init_instance_host(lbm_ctx *c, int k, const double *rho, const double *ux, const double *uy, const double *T) {
    if (!rho || !ux || !uy || !T) return fail(LBM_ERR_ARG, "NULL argument");
    // stage the four float64 fields in the half-step buffer f1 (free outside a step;
    // it holds at least 16 * 4 bytes per node >= 4 * 8), check them there, and only then
    // replace the state
    const size_t bytes = (size_t)c->n * 8;
    double *st = static_cast<double *>(c->f1);
    CU_TRY(cudaMemcpyAsync(st, rho, bytes, cudaMemcpyHostToDevice, c->stream));
    CU_TRY(cudaMemcpyAsync(st + c->n, ux, bytes, cudaMemcpyHostToDevice, c->stream));
    CU_TRY(cudaMemcpyAsync(st + 2 * c->n, uy, bytes, cudaMemcpyHostToDevice, c->stream));
    CU_TRY(cudaMemcpyAsync(st + 3 * c->n, T, bytes, cudaMemcpyHostToDevice, c->stream));
    CU_TRY(cudaMemsetAsync(c->bad, 0xff, sizeof(unsigned long long), c->stream));
    CU_TRY(launch_check_init(st, st + c->n, st + 2 * c->n, st + 3 * c->n, c->n, c->bad, c->stream));
    unsigned long long bad = 0;
    CU_TRY(cudaMemcpyAsync(&bad, c->bad, sizeof bad, cudaMemcpyDeviceToHost, c->stream));
    CU_TRY(cudaStreamSynchronize(c->stream));  // the host buffers are free from here on
    if (bad != ~0ULL) return fail(LBM_ERR_ARG, "node %llu: need 0 < rho < 3, T > 0 and finite u", bad);
    return init_instance(c, k, st, st + c->n, st + 2 * c->n, st + 3 * c->n);
}

// rho, u_x, u_y, T (macro fields 0..3) of instance k as dense float64 [ny][nx] device arrays
int moments_to_device(lbm_ctx *c, int k, double *const out[4]) {
    const int ld = NF_M * c->nx;
    for (int j = 0; j < 4; ++j) {
        if (!out[j]) continue;
        const size_t off = c->row0(k) * ld + (size_t)j * c->nx;
        if (c->mixed)
            CU_TRY(launch_field_out<float>(static_cast<const float *>(c->m) + off, ld, out[j], c->nx, c->ny,
                                           c->stream));
        else
            CU_TRY(launch_field_out<double>(static_cast<const double *>(c->m) + off, ld, out[j], c->nx, c->ny,
                                            c->stream));
    }
    return LBM_OK;
}

int moments_host(lbm_ctx *c, int k, double *rho, double *ux, double *uy, double *T) {
    // gather through the half-step buffer (free outside a step), 4 x n doubles <= its size
    double *st = static_cast<double *>(c->f1);
    double *const dev[4] = {rho ? st : nullptr, ux ? st + c->n : nullptr, uy ? st + 2 * c->n : nullptr,
                            T ? st + 3 * c->n : nullptr};
    int rc = moments_to_device(c, k, dev);
    if (rc) return rc;
    double *const host[4] = {rho, ux, uy, T};
    for (int j = 0; j < 4; ++j)
        if (host[j]) CU_TRY(cudaMemcpyAsync(host[j], dev[j], (size_t)c->n * 8, cudaMemcpyDeviceToHost, c->stream));
    CU_TRY(cudaStreamSynchronize(c->stream));
    return check_device_error(c);
}

// the API's [16][ny][nx] float64 layout <-> the device block [ny][16][nx] of instance k
int get_f_host(lbm_ctx *c, int k, double *f16) {
    const size_t cnt = (size_t)16 * c->n, nx = c->nx, ny = c->ny;
    std::vector<unsigned char> tmp(cnt * c->fsize);
    const char *src0 = static_cast<const char *>(c->f0) + c->row0(k) * NF_F * nx * c->fsize;
    CU_TRY(cudaMemcpyAsync(tmp.data(), src0, tmp.size(), cudaMemcpyDeviceToHost, c->stream));
    CU_TRY(cudaStreamSynchronize(c->stream));
    if (int rc = check_device_error(c)) return rc;
    for (size_t y = 0; y < ny; ++y)
        for (size_t i = 0; i < 16; ++i) {
            const size_t src = (y * 16 + i) * nx, dst = (i * ny + y) * nx;
            if (c->mixed) {
                const float *sp = reinterpret_cast<const float *>(tmp.data()) + src;
                for (size_t x = 0; x < nx; ++x) f16[dst + x] = (double)sp[x];
            } else {
                std::memcpy(f16 + dst, reinterpret_cast<const double *>(tmp.data()) + src, nx * 8);
            }
        }
    return LBM_OK;
}

int set_f_host(lbm_ctx *c, int k, const double *f16) {
    const size_t cnt = (size_t)16 * c->n, nx = c->nx, ny = c->ny;
    for (size_t j = 0; j < cnt; ++j)
        if (!std::isfinite(f16[j])) return fail(LBM_ERR_NONFINITE, "f16[%zu] is not finite", j);
    std::vector<unsigned char> tmp(cnt * c->fsize);
    for (size_t y = 0; y < ny; ++y)
        for (size_t i = 0; i < 16; ++i) {
            const size_t src = (i * ny + y) * nx, dst = (y * 16 + i) * nx;
            if (c->mixed) {
                float *dp = reinterpret_cast<float *>(tmp.data()) + dst;
                for (size_t x = 0; x < nx; ++x) dp[x] = (float)f16[src + x];
            } else {
                std::memcpy(reinterpret_cast<double *>(tmp.data()) + dst, f16 + src, nx * 8);
            }
        }
    char *f = static_cast<char *>(c->f0) + c->row0(k) * NF_F * nx * c->fsize;
    CU_TRY(cudaMemcpyAsync(f, tmp.data(), tmp.size(), cudaMemcpyHostToDevice, c->stream));
    CU_TRY(cudaStreamSynchronize(c->stream));
    MomArgs a{};
    a.f = f;
    a.m = static_cast<char *>(c->m) + c->row0(k) * NF_M * nx * c->fsize;
    a.nx = c->nx;
    a.ny = c->ny;
    a.b = c->p.b;
    a.T_iso = (c->p.flags & LBM_FLAG_ISOTHERMAL) ? c->p.T_iso : 0.0;
    for (int i = 0; i < 16; ++i) a.psi[i] = vel_sq(i) + (i < 4 ? c->p.eta0 * c->p.eta0 : 0.0);
    CU_TRY(c->mixed ? launch_moments<float>(a, c->stream) : launch_moments<double>(a, c->stream));
    c->initialized[k] = 1;
    return LBM_OK;
}

// ---- checkpoint blobs: header, then per row the 16 distributions and the 4 moments --------
struct StateHeader {
    char magic[8];
    uint32_t version;
    int32_t nx, ny, precision;
    int64_t steps;
    uint64_t params_hash;
    uint64_t payload_bytes;
    uint32_t element_size;
    uint32_t reserved[3];
};
static_assert(sizeof(StateHeader) == 64, "state header is 64 bytes");
constexpr char kStateMagic[8] = {'L', 'B', 'M', 'S', 'T', 'A', 'T', 'E'};

// FNV-1a (64-bit) over the parameter fields in declaration order, each value's bytes taken
// least significant first (the same on every host)
uint64_t hash_params(const lbm_params &p) {
    uint64_t h = 1469598103934665603ULL;
    auto bytes = [&h](uint64_t v, int n) {
        for (int k = 0; k < n; ++k) {
            h ^= (v >> (8 * k)) & 0xffu;
            h *= 1099511628211ULL;
        }
    };
    auto dbl = [&bytes](double d) {
        uint64_t u;
        std::memcpy(&u, &d, 8);
        bytes(u, 8);
    };
    auto i32 = [&bytes](int v) { bytes((uint32_t)v, 4); };
    for (double d : {p.tau, p.dt, p.dx, p.dy, p.K, p.H, p.q, p.zeta, p.b, p.eta0, p.win_alpha, p.win_p}) dbl(d);
    i32(p.precision);
    i32(p.flags);
    dbl(p.T_iso);
    i32(p.keff_terms);
    i32(p.reserved);
    dbl(p.filter_alpha);
    dbl(p.filter_p);
    return h;
}

size_t state_payload(int nx, int ny, size_t es) { return (size_t)ny * (NF_F + 4) * nx * es; }

int get_state_host(lbm_ctx *c, int k, long long steps, void *blob, size_t bytes) {
    const size_t es = c->fsize, nx = c->nx, ny = c->ny, pay = state_payload(c->nx, c->ny, es);
    if (!blob) return fail(LBM_ERR_ARG, "NULL blob");
    if (bytes < sizeof(StateHeader) + pay)
        return fail(LBM_ERR_ARG, "blob of %zu bytes, the state needs %zu", bytes, sizeof(StateHeader) + pay);
    StateHeader hd{};
    std::memcpy(hd.magic, kStateMagic, 8);
    hd.version = 1;
    hd.nx = c->nx;
    hd.ny = c->ny;
    hd.precision = c->p.precision;
    hd.steps = steps;
    hd.params_hash = hash_params(c->p);
    hd.payload_bytes = pay;
    hd.element_size = (uint32_t)es;
    std::memcpy(blob, &hd, sizeof hd);
    char *dst = static_cast<char *>(blob) + sizeof hd;
    const size_t row = (NF_F + 4) * nx * es;
    const char *f = static_cast<const char *>(c->f0) + c->row0(k) * NF_F * nx * es;
    const char *m = static_cast<const char *>(c->m) + c->row0(k) * NF_M * nx * es;
    CU_TRY(cudaMemcpy2DAsync(dst, row, f, NF_F * nx * es, NF_F * nx * es, ny, cudaMemcpyDeviceToHost, c->stream));
    CU_TRY(cudaMemcpy2DAsync(dst + NF_F * nx * es, row, m, NF_M * nx * es, 4 * nx * es, ny, cudaMemcpyDeviceToHost,
                             c->stream));
    CU_TRY(cudaStreamSynchronize(c->stream));
    return check_device_error(c);
}

// validates a blob against context c; on success *steps is its step counter
int check_state(const lbm_ctx *c, const void *blob, size_t bytes, long long *steps) {
    const size_t es = c->fsize, pay = state_payload(c->nx, c->ny, es);
    if (!blob) return fail(LBM_ERR_ARG, "NULL blob");
    if (bytes < sizeof(StateHeader)) return fail(LBM_ERR_ARG, "blob of %zu bytes has no header", bytes);
    StateHeader hd;
    std::memcpy(&hd, blob, sizeof hd);
    if (std::memcmp(hd.magic, kStateMagic, 8) != 0 || hd.version != 1)
        return fail(LBM_ERR_ARG, "not a version-1 state blob");
    if (hd.nx != c->nx || hd.ny != c->ny || hd.precision != c->p.precision || hd.element_size != es ||
        hd.payload_bytes != pay)
        return fail(LBM_ERR_ARG, "blob of a %d x %d state in precision %d, the handle is %d x %d in %d", hd.nx, hd.ny,
                    hd.precision, c->nx, c->ny, c->p.precision);
    if (hd.params_hash != hash_params(c->p))
        return fail(LBM_ERR_ARG, "blob was written with other parameters (hash %016llx, handle %016llx)",
                    (unsigned long long)hd.params_hash, (unsigned long long)hash_params(c->p));
    if (bytes < sizeof hd + pay) return fail(LBM_ERR_ARG, "blob of %zu bytes is truncated", bytes);
    if (hd.steps < 0) return fail(LBM_ERR_ARG, "negative step count in the blob");
    const char *src = static_cast<const char *>(blob) + sizeof hd;
    const size_t vals = pay / es;
    for (size_t j = 0; j < vals; ++j) {
        double v;
        if (es == 4) {
            float x;
            std::memcpy(&x, src + j * 4, 4);
            v = x;
        } else {
            std::memcpy(&v, src + j * 8, 8);
        }
        if (!std::isfinite(v)) return fail(LBM_ERR_NONFINITE, "blob value %zu is not finite", j);
    }
    *steps = hd.steps;
    return LBM_OK;
}

int set_state_host(lbm_ctx *c, int k, const void *blob) {
    const size_t es = c->fsize, nx = c->nx, ny = c->ny;
    const size_t row = (NF_F + 4) * nx * es;
    const char *src = static_cast<const char *>(blob) + sizeof(StateHeader);
    char *f = static_cast<char *>(c->f0) + c->row0(k) * NF_F * nx * es;
    char *m = static_cast<char *>(c->m) + c->row0(k) * NF_M * nx * es;
    CU_TRY(cudaMemcpy2DAsync(f, NF_F * nx * es, src, row, NF_F * nx * es, ny, cudaMemcpyHostToDevice, c->stream));
    CU_TRY(cudaMemcpy2DAsync(m, NF_M * nx * es, src + NF_F * nx * es, row, 4 * nx * es, ny, cudaMemcpyHostToDevice,
                             c->stream));
    CU_TRY(cudaStreamSynchronize(c->stream));
    c->initialized[k] = 1;
    return LBM_OK;
}

template <typename R> int diag_launch(lbm_ctx *c, int k) {
    // d_y rho into M_RY, d_x rho into M_DQX of instance k (stage scratch, rebuilt by the next stage)
    const int nx = c->nx, ldm = NF_M * nx;
    R *m = static_cast<R *>(c->m) + c->row0(k) * ldm;
    // one job: the narrowest tiles with 16-byte rows, so that its CTAs spread over the SMs
    const int W = std::min(nx, std::max(2, 16 / (int)sizeof(R)));
    const int Wd = col_cluster(W, c->ly, sizeof(R)) == 1 ? W : c->geo.colW;
    ColArgs<R> ca = col_args<R>(c, 1, Wd);
    ca.jobs[0] = ColJob<R>{m + (size_t)M_RHO * nx, m + (size_t)M_RY * nx, ldm, ldm, 1, R(1)};
    CU_TRY(launch_col<R>(ca, 1, Wd == c->geo.colW ? c->geo.col_smem : col_smem(Wd, c->ly, sizeof(R)), c->stream));
    RowDerivArgs<R> ra{};
    ra.in[0] = m + (size_t)M_RHO * nx;
    ra.out[0] = m + (size_t)M_DQX * nx;
    ra.ld = ldm;
    ra.nin = 1;
    ra.nx = c->nx;
    ra.ny = c->ny;
    ra.rows = c->geo.rows_rowd;
    ra.order = 1;
    ra.ax = axis<R>(c, true);
    CU_TRY(launch_row_deriv<R>(ra, c->geo.rowd_smem, c->stream));
    DiagArgs da{};
    da.rho = m + (size_t)M_RHO * nx;
    da.ux = m + (size_t)M_UX * nx;
    da.uy = m + (size_t)M_UY * nx;
    da.T = m + (size_t)M_T * nx;
    da.rx = m + (size_t)M_DQX * nx;
    da.ry = m + (size_t)M_RY * nx;
    da.ld = ldm;
    da.partial = c->partial;
    da.nx = c->nx;
    da.ny = c->ny;
    da.K = c->p.K;
    da.cell = c->p.dx * c->p.dy;
    CU_TRY(launch_diag<R>(da, c->diag_blocks, c->stream));
    return LBM_OK;
}

int diagnostics_instance(lbm_ctx *c, int k, long long steps, double out[6]) {
    int rc = c->mixed ? diag_launch<float>(c, k) : diag_launch<double>(c, k);
    if (rc) return rc;
    std::vector<double> part((size_t)c->diag_blocks * 5);
    CU_TRY(cudaMemcpyAsync(part.data(), c->partial, part.size() * 8, cudaMemcpyDeviceToHost, c->stream));
    CU_TRY(cudaStreamSynchronize(c->stream));
    if ((rc = check_device_error(c))) return rc;
    double s[4] = {0, 0, 0, 0}, mx = 0;
    for (int b = 0; b < c->diag_blocks; ++b) {
        for (int j = 0; j < 4; ++j) s[j] += part[b * 5 + j];
        mx = std::max(mx, part[b * 5 + 4]);
    }
    const double cell = c->p.dx * c->p.dy;
    for (int j = 0; j < 4; ++j) out[j] = s[j] * cell;
    out[4] = std::sqrt(mx);
    out[5] = (double)steps;
    for (int j = 0; j < 5; ++j)
        if (!std::isfinite(out[j])) return fail(LBM_ERR_NONFINITE, "diagnostic %d is not finite", j);
    return LBM_OK;
}

// host reduction of one slot of per-block partial sums into out[0..4]
int reduce_partials(const lbm_ctx *c, const double *part, int nparts, double out[6]) {
    double s[4] = {0, 0, 0, 0}, mx = 0;
    for (int b = 0; b < nparts; ++b) {
        for (int j = 0; j < 4; ++j) s[j] += part[b * 5 + j];
        mx = std::max(mx, part[b * 5 + 4]);
    }
    const double cell = c->p.dx * c->p.dy;
    for (int j = 0; j < 4; ++j) out[j] = s[j] * cell;
    out[4] = std::sqrt(mx);
    for (int j = 0; j < 5; ++j)
        if (!std::isfinite(out[j])) return fail(LBM_ERR_NONFINITE, "diagnostic %d is not finite", j);
    return LBM_OK;
}

// Circularly averaged structure factor of instance k's density (kernels_sf.cu): the spectra
// go to the half-step buffer f1 (16 bytes per node, free outside a step); the frequency
// tables and shell sums to a temporary device buffer.
int structure_factor_instance(lbm_ctx *c, int k, int nbins, double *S, double *count) {
    if (nbins < 1 || nbins > 8192) return fail(LBM_ERR_ARG, "nbins must be in [1, 8192]");
    const int nx = c->nx, ny = c->ny, N = std::max(nx, ny);
    const size_t ldm = (size_t)NF_M * nx;
    SfArgs a{};
    a.rho = static_cast<const char *>(c->m) + c->row0(k) * ldm * c->fsize;  // M_RHO is field 0
    a.ld = (int)ldm;
    a.nx = nx; a.ny = ny; a.lx = c->lx; a.ly = c->ly;
    a.rows = std::max(1, std::min(ny, 256 / line_G(c->lx)));
    a.cols = std::max(1, std::min(nx, 256 / line_G(c->ly)));
    a.Z = static_cast<double2 *>(c->f1);
    a.twx = c->tw64x; a.twy = c->tw64y;
    const size_t tab_bytes = ((size_t)(nx + ny) * sizeof(int) + 255) & ~(size_t)255;
    char *tmp = nullptr;
    if (cudaMalloc(&tmp, tab_bytes + (size_t)nbins * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return fail(LBM_ERR_NOMEM, "structure factor: no device scratch");
    }
    struct Free {
        char *p;
        ~Free() { cudaFree(p); }
    } free_tmp{tmp};
    int *fx = reinterpret_cast<int *>(tmp), *fy = fx + nx;
    double *dS = reinterpret_cast<double *>(tmp + tab_bytes);
    a.fx = fx; a.fy = fy;
    a.sx = (double)N / nx; a.sy = (double)N / ny;
    a.nbins = nbins;
    a.S = dS;
    std::vector<int> hx(nx), hy(ny);
    position_frequencies(nx, hx.data());
    position_frequencies(ny, hy.data());
    CU_TRY(cudaMemcpyAsync(fx, hx.data(), nx * sizeof(int), cudaMemcpyHostToDevice, c->stream));
    CU_TRY(cudaMemcpyAsync(fy, hy.data(), ny * sizeof(int), cudaMemcpyHostToDevice, c->stream));
    CU_TRY(cudaMemsetAsync(dS, 0, nbins * sizeof(double), c->stream));
    CU_TRY(c->mixed ? launch_structure_factor<float>(a, c->stream) : launch_structure_factor<double>(a, c->stream));
    std::vector<double> tot(nbins);
    CU_TRY(cudaMemcpyAsync(tot.data(), dS, nbins * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CU_TRY(cudaStreamSynchronize(c->stream));
    // shell populations from the same index geometry; shell 0 (the mean) reported as 0
    std::vector<double> cnt(nbins, 0.0);
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            const double qx = hx[x] * a.sx, qy = hy[y] * a.sy;
            const int b = (int)std::rint(std::sqrt(qx * qx + qy * qy));
            if (b < nbins) cnt[b] += 1.0;
        }
    for (int b = 0; b < nbins; ++b) {
        S[b] = (b == 0 || cnt[b] == 0) ? 0.0 : tot[b] / cnt[b];
        if (count) count[b] = cnt[b];
        if (!std::isfinite(S[b])) return fail(LBM_ERR_NONFINITE, "structure factor bin %d is not finite", b);
    }
    return LBM_OK;
}

}  // namespace

extern "C" {

int lbm_structure_factor(lbm_handle c, int nbins, double *S, double *count) {
    if (!c || !S) return fail(LBM_ERR_ARG, "NULL argument");
    if (!c->all_initialized()) return fail(LBM_ERR_STATE, "no state yet");
    return structure_factor_instance(c, 0, nbins, S, count);
}

int lbm_batch_structure_factor(lbm_batch b, int k, int nbins, double *S, double *count) {
    if (!b || !S || k < 0 || k >= (int)b->where.size()) return fail(LBM_ERR_ARG, "bad batch or instance");
    lbm_ctx *c = b->groups[b->where[k].first];
    if (!c->initialized[b->where[k].second]) return fail(LBM_ERR_STATE, "instance %d has no state yet", k);
    CU_TRY(cudaStreamSynchronize(b->stream));
    return structure_factor_instance(c, b->where[k].second, nbins, S, count);
}

void lbm_default_params(lbm_params *p) {
    if (!p) return;
    std::memset(p, 0, sizeof *p);
    p->tau = 1e-4;
    p->dt = 1e-4;
    p->dx = 1.0 / 256.0;
    p->dy = 1.0 / 256.0;
    p->K = 5e-6;
    p->H = 0.0;
    p->q = -0.004;
    p->zeta = 0.0;
    p->b = 2.0;
    p->eta0 = 2.5;
    p->win_alpha = 0.0;
    p->win_p = 36.0;
    p->precision = LBM_FP64;
    p->flags = 0;
    p->T_iso = 0.0;
    p->keff_terms = 8;
    p->reserved = 0;
    p->filter_alpha = 0.0;
    p->filter_p = 36.0;
}

const char *lbm_strerror(int code) {
    switch (code) {
        case LBM_OK: return "ok";
        case LBM_ERR_ARG: return "invalid argument";
        case LBM_ERR_NOMEM: return "device allocation failed";
        case LBM_ERR_CUDA: return "CUDA error";
        case LBM_ERR_NONFINITE: return "non-finite value in the state";
        case LBM_ERR_TIMEOUT: return "device wait timed out";
        case LBM_ERR_STATE: return "call out of order";
        case LBM_ERR_UNSUPPORTED: return "unsupported size or precision";
        default: return "unknown error";
    }
}

const char *lbm_last_error(void) { return g_last_error.c_str(); }

int lbm_create(int nx, int ny, const lbm_params *params, void *stream, lbm_handle *out) {
    if (!out) return fail(LBM_ERR_ARG, "out is NULL");
    return create_ctx(nx, ny, 1, params, static_cast<cudaStream_t>(stream), out);
}

void lbm_destroy(lbm_handle c) { free_ctx(c); }

int diag_flush(lbm_ctx *c);
int step_with_diag(lbm_ctx *c);

int lbm_init(lbm_handle c, const double *rho, const double *ux, const double *uy, const double *T) {
    if (!c) return fail(LBM_ERR_ARG, "NULL handle");
    const int rc = diag_flush(c);
    return rc ? rc : init_instance_host(c, 0, rho, ux, uy, T);
}

int lbm_init_device(lbm_handle c, const double *rho, const double *ux, const double *uy, const double *T) {
    if (!c || !rho || !ux || !uy || !T) return fail(LBM_ERR_ARG, "NULL argument");
    const int rc = diag_flush(c);
    return rc ? rc : init_instance(c, 0, rho, ux, uy, T);
}

int lbm_step(lbm_handle c, int n) {
    if (!c || n < 0) return fail(LBM_ERR_ARG, "bad handle or n < 0");
    if (!c->all_initialized()) return fail(LBM_ERR_STATE, "lbm_step before lbm_init / lbm_set_f");
    if (n == 0) return LBM_OK;
    if (c->fuse_slot >= 0) {  // a diagnostics request of the current state rides on this step
        const int rc = step_with_diag(c);
        if (rc) return rc;
        ++c->steps;
        if (--n == 0) return LBM_OK;
    }
    if (c->timing) {  // direct launches, each between the timing events
        for (int s = 0; s < n; ++s) {
            int rc = run_step_launches(c);
            if (rc) return rc;
            ++c->steps;
        }
        return LBM_OK;
    }
    if (!c->graph) {
        int rc = build_step_graph(c);
        if (rc) return rc;
    }
    for (int s = 0; s < n; ++s) {
        CU_TRY(cudaGraphLaunch(c->graph, c->stream));
        ++c->steps;
    }
    return LBM_OK;
}

int lbm_moments_device(lbm_handle c, double *rho, double *ux, double *uy, double *T) {
    if (!c) return fail(LBM_ERR_ARG, "NULL handle");
    if (!c->all_initialized()) return fail(LBM_ERR_STATE, "no state yet");
    double *const out[4] = {rho, ux, uy, T};
    return moments_to_device(c, 0, out);
}

int lbm_moments(lbm_handle c, double *rho, double *ux, double *uy, double *T) {
    if (!c) return fail(LBM_ERR_ARG, "NULL handle");
    if (!c->all_initialized()) return fail(LBM_ERR_STATE, "no state yet");
    return moments_host(c, 0, rho, ux, uy, T);
}

int lbm_get_f(lbm_handle c, double *f16) {
    if (!c || !f16) return fail(LBM_ERR_ARG, "NULL argument");
    if (!c->all_initialized()) return fail(LBM_ERR_STATE, "no state yet");
    return get_f_host(c, 0, f16);
}

int lbm_set_f(lbm_handle c, const double *f16) {
    if (!c || !f16) return fail(LBM_ERR_ARG, "NULL argument");
    const int rc = diag_flush(c);
    return rc ? rc : set_f_host(c, 0, f16);
}

size_t lbm_state_bytes(int nx, int ny, int precision) {
    if (!is_pow2(nx) || !is_pow2(ny) || nx > 4096 || ny > 4096) return 0;
    if (precision != LBM_FP64 && precision != LBM_MIXED && precision != LBM_MIXED_RHO64) return 0;
    return sizeof(StateHeader) + state_payload(nx, ny, precision == LBM_FP64 ? 8 : 4);
}

unsigned long long lbm_params_hash(const lbm_params *params) { return params ? hash_params(*params) : 0ULL; }

int lbm_get_state(lbm_handle c, void *blob, size_t bytes) {
    if (!c) return fail(LBM_ERR_ARG, "NULL handle");
    if (!c->all_initialized()) return fail(LBM_ERR_STATE, "no state yet");
    return get_state_host(c, 0, c->steps, blob, bytes);
}

int lbm_set_state(lbm_handle c, const void *blob, size_t bytes) {
    if (!c) return fail(LBM_ERR_ARG, "NULL handle");
    long long steps = 0;
    int rc = check_state(c, blob, bytes, &steps);
    if (rc) return rc;
    if ((rc = diag_flush(c))) return rc;
    rc = set_state_host(c, 0, blob);
    if (rc) return rc;
    c->steps = steps;
    return LBM_OK;
}

int lbm_diagnostics(lbm_handle c, double out[6]) {
    if (!c || !out) return fail(LBM_ERR_ARG, "NULL argument");
    if (!c->all_initialized()) return fail(LBM_ERR_STATE, "no state yet");
    return diagnostics_instance(c, 0, c->steps, out);
}

// A diagnostics request can be fused into the next step when that step's first macro pass
// computes it: float32 passes (LBM_MIXED), the forcing chain on, one instance.
static bool diag_fusable(const lbm_ctx *c) {
    return c->mixed && !c->rho64 && !(c->p.flags & LBM_FLAG_NO_FORCE) && !c->geo.macro_serial && c->nb == 1;
}

// Queues the copy of `nparts` partial values from `dev` and the error word into slot `slot`, and
// the slot's event.
static int diag_copy_out(lbm_ctx *c, int slot, const double *dev, int nparts) {
    double *h = c->hpart + slot * c->dslot;
    CU_TRY(cudaMemcpyAsync(h, dev, (size_t)nparts * 5 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CU_TRY(cudaMemcpyAsync(h + c->dslot - 1, c->err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CU_TRY(cudaEventRecord(c->dev_ev[slot], c->stream));
    c->dnparts[slot] = nparts;
    return LBM_OK;
}

// The standalone form of a request: the diagnostics of the current state into slot `slot`.
static int diag_standalone(lbm_ctx *c, int slot) {
    int rc = c->mixed ? diag_launch<float>(c, 0) : diag_launch<double>(c, 0);
    if (rc) return rc;
    return diag_copy_out(c, slot, c->partial, c->diag_blocks);
}

// A request still waiting for a step is computed now, before the state changes other than by
// a step (init, set_f, set_state, autotune).
int diag_flush(lbm_ctx *c) {
    if (c->fuse_slot < 0) return LBM_OK;
    const int slot = c->fuse_slot;
    c->fuse_slot = -1;
    return diag_standalone(c, slot);
}

// The fused request's step: the step graph whose first macro pass writes the partial values
// into the slot's buffer and then records the slot's event; their copy to the host slot runs on
// a side stream from that event, while the rest of the step runs, so lbm_diagnostics_end
// returns before the step ends and the caller can queue the next step in time. The slot's
// previous copy has been waited for by the lbm_diagnostics_end that freed the slot.
int step_with_diag(lbm_ctx *c) {
    const int slot = c->fuse_slot;
    if (c->timing) {
        c->fuse_capture = slot;
        const int rc = run_step_launches(c);
        c->fuse_capture = -1;
        if (rc) return rc;
    } else {
        if (!c->graph_diag[slot]) {
            const int rc = build_step_graph(c, slot);
            if (rc) return rc;  // nothing launched: the request stays pending (computed on its own at the end)
        }
        CU_TRY(cudaGraphLaunch(c->graph_diag[slot], c->stream));
    }
    c->fuse_slot = -1;
    CU_TRY(cudaStreamWaitEvent(c->dstream, c->fev[slot], 0));
    double *h = c->hpart + slot * c->dslot;
    const int nparts = (c->nb * c->ny) / c->geo.rows_macro;
    CU_TRY(cudaMemcpyAsync(h, c->fpart[slot], (size_t)nparts * 5 * sizeof(double), cudaMemcpyDeviceToHost, c->dstream));
    CU_TRY(cudaMemcpyAsync(h + c->dslot - 1, c->err, sizeof(int), cudaMemcpyDeviceToHost, c->dstream));
    CU_TRY(cudaEventRecord(c->dev_ev[slot], c->dstream));
    c->dnparts[slot] = nparts;
    return LBM_OK;
}

int lbm_diagnostics_begin(lbm_handle c) {
    if (!c) return fail(LBM_ERR_ARG, "NULL handle");
    if (!c->all_initialized()) return fail(LBM_ERR_STATE, "no state yet");
    if (c->dcount == 2) return fail(LBM_ERR_STATE, "two requests pending: call lbm_diagnostics_end first");
    if (!c->hpart) {
        // per slot: the partial values of the larger of the diagnostics kernel's blocks and the
        // macro pass's CTAs (one row each at most), then the error word
        c->dslot = (size_t)std::max(c->diag_blocks, c->nb * c->ny) * 5 + 1;
        if (cudaHostAlloc(&c->hpart, 2 * c->dslot * sizeof(double), cudaHostAllocDefault) != cudaSuccess) {
            cudaGetLastError();
            c->hpart = nullptr;
            return fail(LBM_ERR_NOMEM, "no pinned host memory for the diagnostics slots");
        }
        for (cudaEvent_t &e : c->dev_ev) CU_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    const int slot = (c->dhead + c->dcount) & 1;
    c->dsteps[slot] = c->steps;
    if (diag_fusable(c) && c->fuse_slot < 0) {  // computed by the next step (or at lbm_diagnostics_end)
        if (!c->dstream) {
            bool ok = cudaStreamCreateWithFlags(&c->dstream, cudaStreamNonBlocking) == cudaSuccess;
            for (int k = 0; k < 2 && ok; ++k)
                ok = cudaMalloc(&c->fpart[k], (size_t)c->nb * c->ny * 5 * sizeof(double)) == cudaSuccess &&
                     cudaEventCreateWithFlags(&c->fev[k], cudaEventDisableTiming) == cudaSuccess;
            if (!ok) return fail(LBM_ERR_NOMEM, "no device memory or stream for the fused diagnostics");
        }
        c->fuse_slot = slot;
        ++c->dcount;
        return LBM_OK;
    }
    const int rc = diag_standalone(c, slot);
    if (rc) return rc;
    ++c->dcount;
    return LBM_OK;
}

int lbm_diagnostics_end(lbm_handle c, double out[6]) {
    if (!c || !out) return fail(LBM_ERR_ARG, "NULL argument");
    if (c->dcount == 0) return fail(LBM_ERR_STATE, "no diagnostics request pending");
    const int slot = c->dhead;
    if (slot == c->fuse_slot) {  // no step since the request: computed on its own now
        const int rc = diag_flush(c);
        if (rc) return rc;
    }
    c->dhead ^= 1;
    --c->dcount;
    CU_TRY(cudaEventSynchronize(c->dev_ev[slot]));
    const double *h = c->hpart + slot * c->dslot;
    int err = 0;
    std::memcpy(&err, h + c->dslot - 1, sizeof err);
    if (err) {
        CU_TRY(cudaMemsetAsync(c->err, 0, sizeof(int), c->stream));
        return fail(LBM_ERR_TIMEOUT, "a bounded device-side wait gave up (error word %d) before this request", err);
    }
    out[5] = (double)c->dsteps[slot];
    return reduce_partials(c, h, c->dnparts[slot], out);
}

int lbm_synchronize(lbm_handle c) {
    if (!c) return fail(LBM_ERR_ARG, "NULL handle");
    CU_TRY(cudaStreamSynchronize(c->stream));
    return check_device_error(c);
}

int lbm_pass_kinds(lbm_handle c, int kinds[3]) {
    if (!c || !kinds) return fail(LBM_ERR_ARG, "NULL argument");
    kinds[0] = c->geo.col_kind;
    kinds[1] = c->geo.flux_kind;
    kinds[2] = c->geo.upd_cs;
    return LBM_OK;
}

int lbm_set_pass_kinds(lbm_handle c, const int kinds[3]) {
    if (!c || !kinds) return fail(LBM_ERR_ARG, "NULL argument");
    for (int j = 0; j < 2; ++j) {
        if (kinds[j] != LBM_COL_DIRECT && kinds[j] != LBM_COL_TMA && kinds[j] != LBM_COL_LOOKAHEAD &&
            kinds[j] != LBM_COL_TMA1)
            return fail(LBM_ERR_ARG, "unknown pass kind");
        const int W = j == 0 ? c->geo.colW : c->geo.fluxW;
        if ((kinds[j] == LBM_COL_TMA || kinds[j] == LBM_COL_TMA1) && !col_tma_ok(c, W, kinds[j]))
            return fail(LBM_ERR_ARG, "the TMA column pass cannot take %d-column tiles of %d x %d", W, c->nx, c->ny);
        if (kinds[j] == LBM_COL_LOOKAHEAD && !col_lookahead_ok(c, W))
            return fail(LBM_ERR_ARG, "the lookahead column pass cannot take %d-column tiles of %d x %d", W, c->nx, c->ny);
    }
    if (kinds[2] != 1 && kinds[2] != 2 && kinds[2] != 4) return fail(LBM_ERR_ARG, "update CTAs per row must be 1, 2 or 4");
    if (kinds[2] > 1 && !(upd_split_ok(c, kinds[2]) && c->geo.rows_upd == 1))
        return fail(LBM_ERR_ARG,
                    "the update pass splits only float32 rows, of 2048 or more in two and of 4096 in four, one "
                    "row per cluster");
    CU_TRY(cudaStreamSynchronize(c->stream));
    c->geo.col_kind = kinds[0];
    c->geo.flux_kind = kinds[1];
    c->geo.upd_cs = kinds[2];
    c->geo.upd_smem = upd_smem(c->geo.rows_upd, c->lx, c->fsize, c->geo.upd_cs);
    drop_graphs(c);
    return LBM_OK;
}

int lbm_fault_inject(lbm_handle c, int what, long long wait_cycles) {
    if (!c || (what != LBM_FAULT_NONE && what != LBM_FAULT_STARVE_COPIES)) return fail(LBM_ERR_ARG, "bad argument");
    CU_TRY(cudaStreamSynchronize(c->stream));
    c->starve = what == LBM_FAULT_STARVE_COPIES ? 1 : 0;
    c->wait_cycles = wait_cycles > 0 ? wait_cycles : (1LL << 31);
    drop_graphs(c);
    return LBM_OK;
}

int lbm_timing(lbm_handle c, int enable) {
    if (!c) return fail(LBM_ERR_ARG, "NULL handle");
    CU_TRY(cudaStreamSynchronize(c->stream));
    c->timing = enable != 0;
    c->ev_used = 0;
    return LBM_OK;
}

int lbm_timing_read(lbm_handle c, int kernel, double *ms, long long *launches) {
    if (!c || !ms || !launches || kernel < 0 || kernel >= LBM_K_COUNT) return fail(LBM_ERR_ARG, "bad argument");
    CU_TRY(cudaStreamSynchronize(c->stream));
    double tot = 0;
    long long cnt = 0;
    for (size_t s = 0; s + 1 < c->ev_used; s += 2) {
        if (c->ev_cls[s] != kernel) continue;
        float t = 0;
        CU_TRY(cudaEventElapsedTime(&t, c->ev[s], c->ev[s + 1]));
        tot += t;
        ++cnt;
    }
    *ms = tot;
    *launches = cnt;
    return LBM_OK;
}

size_t lbm_device_bytes(lbm_handle c) { return c ? c->slab_bytes : 0; }

int lbm_launch_plan(int nx, int ny, int precision, int out[18]) {
    if (!out) return fail(LBM_ERR_ARG, "NULL argument");
    if (!is_pow2(nx) || !is_pow2(ny) || nx > 4096 || ny > 4096)
        return fail(LBM_ERR_ARG, "nx=%d, ny=%d: each must be a power of two in [2, 4096]", nx, ny);
    if (precision != LBM_FP64 && precision != LBM_MIXED && precision != LBM_MIXED_RHO64)
        return fail(LBM_ERR_ARG, "precision must be LBM_FP64, LBM_MIXED or LBM_MIXED_RHO64");
    const size_t es = precision == LBM_FP64 ? 8 : 4;
    const int lx = log2_int(nx), ly = log2_int(ny);
    Geometry g;
    pass_geometry(nx, ny, es, &g);
    const int v[18] = {g.colW, (g.colW / 2) * line_G(ly) / std::max(1, col_cluster(g.colW, ly, es)), (int)g.col_smem,
                       g.rows_macro, g.rows_macro * line_G(lx) * (g.macro_serial ? 1 : 2), (int)g.macro_smem,
                       g.macro_serial ? 1 : 0,
                       g.rows_upd, (int)g.upd_smem, g.upd_ax ? 1 : 0,
                       g.rows_rowd, g.rows_rowd * line_G(lx), (int)g.rowd_smem,
                       pass_threads(es), macro_threads(es, lx), (int)kMaxCtaSmem,
                       g.upd_cs, std::max(1, col_cluster(g.colW, ly, es))};
    for (int k = 0; k < 18; ++k) out[k] = v[k];
    const size_t need = std::max(std::max(g.upd_smem, g.macro_smem), std::max(g.col_smem, g.rowd_smem));
    if (need > kMaxCtaSmem)
        return fail(LBM_ERR_UNSUPPORTED, "nx=%d ny=%d needs %zu B of shared memory per block", nx, ny, need);
    return LBM_OK;
}

int lbm_geometry(lbm_handle c, int geometry[4]) {
    if (!c || !geometry) return fail(LBM_ERR_ARG, "NULL argument");
    geometry[0] = c->geo.colW;
    geometry[1] = c->geo.rows_macro;
    geometry[2] = c->geo.rows_upd;
    geometry[3] = c->geo.fluxW;
    return LBM_OK;
}

int lbm_set_geometry(lbm_handle c, const int geometry[4]) {
    if (!c || !geometry) return fail(LBM_ERR_ARG, "NULL argument");
    auto has = [](const std::vector<int> &v, int x) { return std::find(v.begin(), v.end(), x) != v.end(); };
    const std::vector<int> cw = col_candidates(c);
    if (!has(cw, geometry[0]) || !has(cw, geometry[3]))
        return fail(LBM_ERR_ARG, "column tile widths %d, %d are not valid for %d x %d", geometry[0], geometry[3], c->nx,
                    c->ny);
    // the macro and update shapes are fixed where their serial / separate-row-pass forms run
    if (c->geo.macro_serial ? geometry[1] != c->geo.rows_macro : !has(macro_candidates(c), geometry[1]))
        return fail(LBM_ERR_ARG, "macro rows per CTA %d not valid", geometry[1]);
    if (c->geo.upd_ax ? geometry[2] != c->geo.rows_upd : !has(upd_candidates(c), geometry[2]))
        return fail(LBM_ERR_ARG, "update rows per CTA %d not valid", geometry[2]);
    CU_TRY(cudaStreamSynchronize(c->stream));
    const size_t es = c->fsize;
    c->geo.colW = geometry[0];
    c->geo.col_smem = col_smem(geometry[0], c->ly, es);
    c->geo.fluxW = geometry[3];
    c->geo.flux_smem = col_smem(geometry[3], c->ly, es);
    // a pass kind the new widths cannot take falls back to the direct form
    auto kind_ok = [c](int kind, int W) {
        return kind == LBM_COL_TMA || kind == LBM_COL_TMA1 ? col_tma_ok(c, W, kind)
               : kind == LBM_COL_LOOKAHEAD                ? col_lookahead_ok(c, W)
                                                          : true;
    };
    if (!kind_ok(c->geo.col_kind, c->geo.colW)) c->geo.col_kind = LBM_COL_DIRECT;
    if (!kind_ok(c->geo.flux_kind, c->geo.fluxW)) c->geo.flux_kind = LBM_COL_DIRECT;
    if (!c->geo.macro_serial) {
        c->geo.rows_macro = geometry[1];
        c->geo.macro_smem = macro_smem(geometry[1], c->lx, es);
    }
    if (!c->geo.upd_ax) {
        c->geo.rows_upd = geometry[2];
        if (geometry[2] != 1) c->geo.upd_cs = 1;
        c->geo.upd_smem = upd_smem(geometry[2], c->lx, es, c->geo.upd_cs);
    }
    drop_graphs(c);  // recaptured with the new shapes at the next step
    return LBM_OK;
}

int lbm_autotune(lbm_handle c, int geometry[4], double ms[4]) {
    if (!c) return fail(LBM_ERR_ARG, "NULL handle");
    float t[4] = {0, 0, 0, 0};
    int rc = diag_flush(c);
    if (rc) return rc;
    rc = autotune_ctx(c, t);
    if (rc) return rc;
    if (ms)
        for (int k = 0; k < 4; ++k) ms[k] = t[k];
    return geometry ? lbm_geometry(c, geometry) : LBM_OK;
}

// Maxwell construction (Sec. 3.1) in chemical-potential form: equal pressure and equal
// mu(rho) = T ln(rho/(3 - rho)) + 3T/(3 - rho) - 9 rho/4 on the two outer branches of the
// van der Waals isotherm, by nested bisection on the saturation pressure.
int lbm_maxwell(double T, double *rho_l, double *rho_v) {
    if (!rho_l || !rho_v) return fail(LBM_ERR_ARG, "NULL output");
    if (!(T > 0.0 && T < 1.0)) return fail(LBM_ERR_ARG, "need 0 < T < 1 (T=%g)", T);
    auto P = [T](double r) { return 3.0 * r * T / (3.0 - r) - 1.125 * r * r; };
    auto mu = [T](double r) { return T * std::log(r / (3.0 - r)) + 3.0 * T / (3.0 - r) - 2.25 * r; };
    // spinodals: dP/drho = 0 <=> 4T = rho (3 - rho)^2, one root in (0,1), one in (1,3)
    auto sp = [T](double lo, double hi, bool rising) {
        for (int it = 0; it < 200; ++it) {
            const double m = 0.5 * (lo + hi);
            const double g = m * (3.0 - m) * (3.0 - m) - 4.0 * T;
            if ((g < 0) == rising) lo = m; else hi = m;
        }
        return 0.5 * (lo + hi);
    };
    const double sv = sp(0.0, 1.0, true), sl = sp(1.0, 3.0, false);
    // root of P(rho) = Ps on a monotone branch
    auto branch = [&](double lo, double hi, double Ps, bool increasing) {
        for (int it = 0; it < 200; ++it) {
            const double m = 0.5 * (lo + hi);
            if ((P(m) < Ps) == increasing) lo = m; else hi = m;
        }
        return 0.5 * (lo + hi);
    };
    double plo = std::max(P(sl), 0.0), phi = P(sv);
    double rl = 0, rv = 0;
    for (int it = 0; it < 200; ++it) {
        const double Ps = 0.5 * (plo + phi);
        rv = branch(1e-300, sv, Ps, true);
        rl = branch(sl, 3.0 - 1e-15, Ps, true);
        // d(mu_l - mu_v)/dPs = 1/rho_l - 1/rho_v < 0: a positive difference means Ps is too low
        if (mu(rl) - mu(rv) > 0) plo = Ps; else phi = Ps;
    }
    *rho_l = rl;
    *rho_v = rv;
    return LBM_OK;
}

// ---- batches of independent simulations ---------------------------------------------------

int lbm_batch_create(int count, const int *nx, const int *ny, const lbm_params *params, void *stream,
                     lbm_batch *out) {
    if (!out) return fail(LBM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (count < 1 || !nx || !ny) return fail(LBM_ERR_ARG, "need count >= 1 and size arrays");
    int rc = check_params(params);
    if (rc) return rc;
    // group the instances by grid size, keeping the order of first appearance
    std::vector<std::pair<int, int>> sizes;
    std::vector<int> group_of(count), index_in(count);
    std::vector<int> counts;
    for (int k = 0; k < count; ++k) {
        if (!is_pow2(nx[k]) || !is_pow2(ny[k]) || nx[k] > 4096 || ny[k] > 4096)
            return fail(LBM_ERR_ARG, "instance %d: nx=%d, ny=%d must be powers of two in [2, 4096]", k, nx[k], ny[k]);
        int g = -1;
        for (size_t j = 0; j < sizes.size(); ++j)
            if (sizes[j] == std::make_pair(nx[k], ny[k])) g = (int)j;
        if (g < 0) {
            g = (int)sizes.size();
            sizes.push_back({nx[k], ny[k]});
            counts.push_back(0);
        }
        group_of[k] = g;
        index_in[k] = counts[g]++;
    }
    lbm_batch_ctx *b = new (std::nothrow) lbm_batch_ctx();
    if (!b) return fail(LBM_ERR_NOMEM, "host allocation failed");
    b->stream = static_cast<cudaStream_t>(stream);
    for (size_t g = 0; g < sizes.size(); ++g) {
        lbm_ctx *c = nullptr;
        rc = create_ctx(sizes[g].first, sizes[g].second, counts[g], params, b->stream, &c);
        if (rc) {
            lbm_batch_destroy(b);
            return rc;
        }
        b->groups.push_back(c);
    }
    for (int k = 0; k < count; ++k) b->where.push_back({group_of[k], index_in[k]});
    b->steps.assign(count, 0);
    *out = b;
    return LBM_OK;
}

void lbm_batch_destroy(lbm_batch b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    else cudaDeviceSynchronize();
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->pgraph) cudaGraphExecDestroy(b->pgraph);
    if (b->bctrl) cudaFree(b->bctrl);
    for (cudaStream_t s : b->branch) cudaStreamDestroy(s);
    for (cudaEvent_t e : b->join) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->cap) cudaStreamDestroy(b->cap);
    for (lbm_ctx *c : b->groups) free_ctx(c);
    delete b;
}

int lbm_batch_count(lbm_batch b) { return b ? (int)b->where.size() : 0; }

static int build_batch_persistent_graph(lbm_batch b);
static int check_batch_error(lbm_batch b);

// The persistent form's CTA size (256 or 512 threads), by timing whole steps of each: the
// distributions and the macroscopic block of every group (all a step reads from the one
// before) are saved to a temporary device buffer first and put back afterwards, so the state
// and every later result are unchanged.
static int autotune_persistent(lbm_batch b) {
    std::vector<size_t> fb, mb;
    size_t total = 0;
    for (lbm_ctx *c : b->groups) {
        fb.push_back((size_t)c->n * c->nb * NF_F * c->fsize);
        mb.push_back((size_t)c->n * c->nb * NF_M * c->fsize);
        total += fb.back() + mb.back();
    }
    char *save = nullptr;
    if (cudaMalloc(&save, total) != cudaSuccess) {
        cudaGetLastError();
        return fail(LBM_ERR_NOMEM, "batch autotune: no device memory to save the states");
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = LBM_OK;
    auto copy_all = [&](bool to_save) {
        size_t off = 0;
        for (size_t g = 0; g < b->groups.size(); ++g) {
            lbm_ctx *c = b->groups[g];
            void *f = c->f0, *m = c->m;
            cudaError_t e = to_save ? cudaMemcpyAsync(save + off, f, fb[g], cudaMemcpyDeviceToDevice, b->stream)
                                    : cudaMemcpyAsync(f, save + off, fb[g], cudaMemcpyDeviceToDevice, b->stream);
            off += fb[g];
            if (e == cudaSuccess)
                e = to_save ? cudaMemcpyAsync(save + off, m, mb[g], cudaMemcpyDeviceToDevice, b->stream)
                            : cudaMemcpyAsync(m, save + off, mb[g], cudaMemcpyDeviceToDevice, b->stream);
            off += mb[g];
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    };
    const int tpb0 = b->ptpb;
    int best = tpb0;
    float bt = 1e30f;
    if (copy_all(true) != cudaSuccess) rc = fail(LBM_ERR_CUDA, "batch autotune: saving the states failed");
    if (rc == LBM_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
        rc = fail(LBM_ERR_CUDA, "batch autotune: cudaEventCreate failed");
    for (int tpb : {512, 256}) {
        if (rc) break;
        b->ptpb = tpb;
        if (b->pgraph) {
            cudaGraphExecDestroy(b->pgraph);
            b->pgraph = nullptr;
        }
        if ((rc = build_batch_persistent_graph(b))) break;
        float t = 0;
        cudaError_t e = cudaGraphLaunch(b->pgraph, b->stream);
        if (e == cudaSuccess) e = cudaEventRecord(e0, b->stream);
        for (int k = 0; k < 3 && e == cudaSuccess; ++k) e = cudaGraphLaunch(b->pgraph, b->stream);
        if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
        if (e != cudaSuccess) {
            rc = fail(LBM_ERR_CUDA, "batch autotune: %s", cudaGetErrorString(e));
            break;
        }
        if (t < bt) bt = t, best = tpb;
    }
    b->ptpb = rc ? tpb0 : best;
    if (b->pgraph) {
        cudaGraphExecDestroy(b->pgraph);
        b->pgraph = nullptr;
    }
    if (copy_all(false) != cudaSuccess && rc == LBM_OK) rc = fail(LBM_ERR_CUDA, "batch autotune: restoring the states failed");
    cudaStreamSynchronize(b->stream);
    if (rc == LBM_OK) rc = check_batch_error(b);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(save);
    return rc;
}

int lbm_batch_autotune(lbm_batch b) {
    if (!b) return fail(LBM_ERR_ARG, "NULL batch");
    CU_TRY(cudaStreamSynchronize(b->stream));
    for (lbm_ctx *c : b->groups) {
        float t[4];
        const int rc = autotune_ctx(c, t);
        if (rc) return rc;
    }
    if (b->graph) {  // recaptured with the new shapes at the next step
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    if (b->form == LBM_BATCH_PERSISTENT) return autotune_persistent(b);
    return LBM_OK;
}

int lbm_batch_geometry(lbm_batch b, int k, int geometry[4]) {
    if (!b || k < 0 || k >= (int)b->where.size()) return fail(LBM_ERR_ARG, "bad batch or instance");
    return lbm_geometry(b->groups[b->where[k].first], geometry);
}

int lbm_batch_init(lbm_batch b, int k, const double *rho, const double *ux, const double *uy, const double *T) {
    if (!b || k < 0 || k >= (int)b->where.size()) return fail(LBM_ERR_ARG, "bad batch or instance");
    lbm_ctx *c = b->groups[b->where[k].first];
    CU_TRY(cudaStreamSynchronize(b->stream));
    const int rc = init_instance_host(c, b->where[k].second, rho, ux, uy, T);
    if (rc == LBM_OK) b->steps[k] = 0;
    return rc;
}

// One graph per step: the groups' launches are parallel branches forked from and joined back
// into the capture stream.
static int build_batch_graph(lbm_batch b) {
    const size_t G = b->groups.size();
    if (!b->cap) CU_TRY(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
    if (!b->fork) CU_TRY(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming));
    while (b->branch.size() < G) {  // a branch stream and its join event, both or neither
        cudaStream_t s;
        cudaEvent_t e;
        CU_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
        const cudaError_t ee = cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
        if (ee != cudaSuccess) {
            cudaStreamDestroy(s);
            return fail(LBM_ERR_CUDA, "batch graph: cudaEventCreateWithFlags: %s", cudaGetErrorString(ee));
        }
        b->branch.push_back(s);
        b->join.push_back(e);
    }
    CU_TRY(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeRelaxed));
    int rc = LBM_OK;
    cudaError_t e = cudaEventRecord(b->fork, b->cap);
    for (size_t g = 0; g < G && rc == LBM_OK && e == cudaSuccess; ++g) {
        e = cudaStreamWaitEvent(b->branch[g], b->fork, 0);
        if (e == cudaSuccess) rc = capture_into(b->groups[g], b->branch[g]);
        if (rc == LBM_OK && e == cudaSuccess) e = cudaEventRecord(b->join[g], b->branch[g]);
        if (rc == LBM_OK && e == cudaSuccess) e = cudaStreamWaitEvent(b->cap, b->join[g], 0);
    }
    cudaGraph_t graph = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(b->cap, &graph);
    if (rc || e != cudaSuccess || ee != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        if (rc) return rc;
        return fail(LBM_ERR_CUDA, "batch graph capture: %s",
                    cudaGetErrorString(e != cudaSuccess ? e : ee));
    }
    const cudaError_t ei = cudaGraphInstantiate(&b->graph, graph, 0);
    cudaGraphDestroy(graph);
    CU_TRY(ei);
    return LBM_OK;
}

// Whether the persistent kernel can take the batch: float32, the full two-stage model (or the
// thermostat), at most kBatchGroups sizes, lines of 128 to 1024 points.
static bool batch_persistent_ok(lbm_batch b) {
    if (b->groups.empty() || (int)b->groups.size() > kBatchGroups) return false;
    for (lbm_ctx *c : b->groups)
        if (!c->mixed || c->rho64 || (c->p.flags & ~LBM_FLAG_ISOTHERMAL) || c->p.filter_alpha > 0 || c->lx < 7 || c->lx > 10 ||
            c->ly < 7 || c->ly > 10)
            return false;
    return true;
}

// Work items and tile shapes of the persistent kernel (CTAs of T = 512 or 256 threads): column
// tiles of W = min(nx, 2T / G) columns (W/2 lines of G threads fill the CTA), macro and update
// row blocks as large as T threads and the shared memory of two (T = 512) or three (T = 256)
// CTAs per SM allow.
static int batch_args(lbm_batch b, BatchArgs<float> &A, size_t &smem) {
    const int T = b->ptpb;
    constexpr size_t es = 4;
    const size_t cap = T == 512 ? 100 * 1024 : 72 * 1024;
    A.ngroups = (int)b->groups.size();
    smem = 0;
    int inst = 0;
    for (int gi = 0; gi < A.ngroups; ++gi) {
        lbm_ctx *c = b->groups[gi];
        BatchGroup<float> &G = A.g[gi];
        const int Gy = line_G(c->ly), Gx = line_G(c->lx);
        const int W = std::min(c->nx, 2 * T / Gy);
        int nrm = 1;
        while (2 * nrm <= c->ny && 2 * (2 * nrm) * Gx <= T &&
               macro_smem(2 * nrm, c->lx, es) <= cap)
            nrm *= 2;
        int nru = 1;
        while (2 * nru <= c->ny && 2 * nru * c->nx <= 8 * T && upd_smem(2 * nru, c->lx, es, 1) <= cap) nru *= 2;
        int nj = 0;
        for (int st = 0; st < 2; ++st) {
            G.col[st] = col_args<float>(c, c->nb, W);
            nj = column_jobs<float>(c, st, G.col[st]);
            G.flux[st] = col_args<float>(c, c->nb, W);
            flux_jobs<float>(c, G.flux[st]);
            G.upd[st] = update_args<float>(c, st, nru);
            G.upd[st].cs = 1;
            G.upd[st].lines_per_batch = update_lines_per_batch(6 * nru, Gx, T);
        }
        G.macro = macro_args<float>(c, nrm);
        G.tiles_x[0] = G.tiles_x[1] = c->nx / W;
        G.ntile[0] = nj * (c->nx / W);
        G.ntile[1] = c->ny / nrm;
        G.ntile[2] = 4 * (c->nx / W);
        G.ntile[3] = c->ny / nru;
        G.inst0 = inst;
        inst += c->nb;
        smem = std::max(smem, col_smem(W, c->ly, es));
        smem = std::max(smem, macro_smem(nrm, c->lx, es));
        smem = std::max(smem, upd_smem(nru, c->lx, es, 1));
    }
    int q = 0;
    for (int chain = 0; chain < kBatchPasses; ++chain)
        for (int gi = 0; gi < A.ngroups; ++gi) {
            A.seg[chain * A.ngroups + gi] = q;
            q += b->groups[gi]->nb * A.g[gi].ntile[chain & 3];
        }
    A.seg[kBatchPasses * A.ngroups] = q;
    const size_t ints = 2 + (size_t)inst * kBatchPasses;
    if (!b->bctrl || b->bctrl_ints != ints) {
        if (b->bctrl) cudaFree(b->bctrl);
        b->bctrl = nullptr;
        if (cudaMalloc(&b->bctrl, (ints + 1) * sizeof(int)) != cudaSuccess) {
            cudaGetLastError();
            return fail(LBM_ERR_NOMEM, "persistent batch: no device memory for its control words");
        }
        b->bctrl_ints = ints;
        CU_TRY(cudaMemset(b->bctrl, 0, (ints + 1) * sizeof(int)));
    }
    A.ctrl = b->bctrl;
    A.err = b->bctrl + ints;
    A.wait_cycles = b->wait_cycles;
    A.withhold = b->withhold;
    return LBM_OK;
}

static int build_batch_persistent_graph(lbm_batch b) {
    BatchArgs<float> *A = new (std::nothrow) BatchArgs<float>();
    if (!A) return fail(LBM_ERR_NOMEM, "host allocation failed");
    struct Del {
        BatchArgs<float> *p;
        ~Del() { delete p; }
    } del{A};
    size_t smem = 0;
    int rc = batch_args(b, *A, smem);
    if (rc) return rc;
    int dev = 0, sms = 0;
    CU_TRY(cudaGetDevice(&dev));
    CU_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    int per_sm = 0;
    const cudaError_t eo = batch_step_ctas_per_sm<float>(smem, b->ptpb, &per_sm);
    if (eo != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        return fail(LBM_ERR_UNSUPPORTED, "persistent batch: no CTA fits an SM (%zu B of shared memory; %s)", smem,
                    cudaGetErrorString(eo));
    }
    if (!b->cap) CU_TRY(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
    CU_TRY(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeRelaxed));
    cudaError_t e = cudaMemsetAsync(b->bctrl, 0, b->bctrl_ints * sizeof(int), b->cap);  // not the error word
    if (e == cudaSuccess) e = launch_batch_step<float>(*A, smem, per_sm * sms, b->ptpb, b->cap);
    cudaGraph_t graph = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(b->cap, &graph);
    if (e != cudaSuccess || ee != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return fail(LBM_ERR_CUDA, "persistent batch graph: %s", cudaGetErrorString(e != cudaSuccess ? e : ee));
    }
    const cudaError_t ei = cudaGraphInstantiate(&b->pgraph, graph, 0);
    cudaGraphDestroy(graph);
    CU_TRY(ei);
    return LBM_OK;
}

// After a synchronisation of the batch's stream: the persistent kernel's error word and every
// size group's own (TMA) error word; a set word is reported once as LBM_ERR_TIMEOUT.
static int check_batch_error(lbm_batch b) {
    if (b->bctrl) {
        int v = 0;
        CU_TRY(cudaMemcpy(&v, b->bctrl + b->bctrl_ints, sizeof v, cudaMemcpyDeviceToHost));
        if (v) {
            CU_TRY(cudaMemset(b->bctrl + b->bctrl_ints, 0, sizeof v));
            return fail(LBM_ERR_TIMEOUT, "a bounded wait of the persistent batch kernel gave up (error word %d): the "
                        "steps since the last check did not complete and the states are not valid",
                        v);
        }
    }
    for (lbm_ctx *c : b->groups) {
        const int rc = check_device_error(c);
        if (rc) return rc;
    }
    return LBM_OK;
}

int lbm_batch_synchronize(lbm_batch b) {
    if (!b) return fail(LBM_ERR_ARG, "NULL batch");
    CU_TRY(cudaStreamSynchronize(b->stream));
    return check_batch_error(b);
}

int lbm_batch_form(lbm_batch b) { return b ? b->form : -1; }

int lbm_batch_set_form(lbm_batch b, int form) {
    if (!b || (form != LBM_BATCH_GRAPH && form != LBM_BATCH_PERSISTENT)) return fail(LBM_ERR_ARG, "bad argument");
    if (form == LBM_BATCH_PERSISTENT && !batch_persistent_ok(b))
        return fail(LBM_ERR_UNSUPPORTED, "the persistent form takes float32 batches of at most %d sizes with lines "
                    "of 128 to 1024 points and no test flags",
                    kBatchGroups);
    CU_TRY(cudaStreamSynchronize(b->stream));
    b->form = form;
    return LBM_OK;
}

int lbm_batch_fault_inject(lbm_batch b, int what, long long wait_cycles) {
    if (!b || (what != LBM_FAULT_NONE && what != LBM_FAULT_WITHHOLD_COMPLETION)) return fail(LBM_ERR_ARG, "bad argument");
    CU_TRY(cudaStreamSynchronize(b->stream));
    b->withhold = what == LBM_FAULT_WITHHOLD_COMPLETION ? 1 : 0;
    b->wait_cycles = wait_cycles > 0 ? wait_cycles : (1LL << 31);
    if (b->pgraph) {
        cudaGraphExecDestroy(b->pgraph);
        b->pgraph = nullptr;
    }
    return LBM_OK;
}

int lbm_batch_step(lbm_batch b, int n) {
    if (!b || n < 0) return fail(LBM_ERR_ARG, "bad batch or n < 0");
    for (lbm_ctx *c : b->groups)
        if (!c->all_initialized()) return fail(LBM_ERR_STATE, "lbm_batch_step before every instance is initialised");
    if (n == 0) return LBM_OK;
    if (b->form == LBM_BATCH_PERSISTENT) {
        if (!b->pgraph) {
            int rc = build_batch_persistent_graph(b);
            if (rc) return rc;
        }
        for (int s = 0; s < n; ++s) CU_TRY(cudaGraphLaunch(b->pgraph, b->stream));
        for (long long &s : b->steps) s += n;
        return LBM_OK;
    }
    if (!b->graph) {
        int rc = build_batch_graph(b);
        if (rc) return rc;
    }
    for (int s = 0; s < n; ++s) CU_TRY(cudaGraphLaunch(b->graph, b->stream));
    for (long long &s : b->steps) s += n;
    return LBM_OK;
}

int lbm_batch_moments(lbm_batch b, int k, double *rho, double *ux, double *uy, double *T) {
    if (!b || k < 0 || k >= (int)b->where.size()) return fail(LBM_ERR_ARG, "bad batch or instance");
    lbm_ctx *c = b->groups[b->where[k].first];
    if (!c->initialized[b->where[k].second]) return fail(LBM_ERR_STATE, "instance %d has no state yet", k);
    CU_TRY(cudaStreamSynchronize(b->stream));
    if (int rc = check_batch_error(b)) return rc;
    return moments_host(c, b->where[k].second, rho, ux, uy, T);
}

int lbm_batch_get_f(lbm_batch b, int k, double *f16) {
    if (!b || !f16 || k < 0 || k >= (int)b->where.size()) return fail(LBM_ERR_ARG, "bad batch or instance");
    lbm_ctx *c = b->groups[b->where[k].first];
    if (!c->initialized[b->where[k].second]) return fail(LBM_ERR_STATE, "instance %d has no state yet", k);
    CU_TRY(cudaStreamSynchronize(b->stream));
    if (int rc = check_batch_error(b)) return rc;
    return get_f_host(c, b->where[k].second, f16);
}

int lbm_batch_get_state(lbm_batch b, int k, void *blob, size_t bytes) {
    if (!b || k < 0 || k >= (int)b->where.size()) return fail(LBM_ERR_ARG, "bad batch or instance");
    lbm_ctx *c = b->groups[b->where[k].first];
    if (!c->initialized[b->where[k].second]) return fail(LBM_ERR_STATE, "instance %d has no state yet", k);
    CU_TRY(cudaStreamSynchronize(b->stream));
    if (int rc = check_batch_error(b)) return rc;
    return get_state_host(c, b->where[k].second, b->steps[k], blob, bytes);
}

int lbm_batch_set_state(lbm_batch b, int k, const void *blob, size_t bytes) {
    if (!b || k < 0 || k >= (int)b->where.size()) return fail(LBM_ERR_ARG, "bad batch or instance");
    lbm_ctx *c = b->groups[b->where[k].first];
    long long steps = 0;
    int rc = check_state(c, blob, bytes, &steps);
    if (rc) return rc;
    CU_TRY(cudaStreamSynchronize(b->stream));
    rc = set_state_host(c, b->where[k].second, blob);
    if (rc) return rc;
    b->steps[k] = steps;
    return LBM_OK;
}

int lbm_batch_diagnostics(lbm_batch b, int k, double out[6]) {
    if (!b || !out || k < 0 || k >= (int)b->where.size()) return fail(LBM_ERR_ARG, "bad batch or instance");
    lbm_ctx *c = b->groups[b->where[k].first];
    if (!c->initialized[b->where[k].second]) return fail(LBM_ERR_STATE, "instance %d has no state yet", k);
    CU_TRY(cudaStreamSynchronize(b->stream));
    if (int rc = check_batch_error(b)) return rc;
    return diagnostics_instance(c, b->where[k].second, b->steps[k], out);
}

}  // extern "C"

// Lets other translation units report a detailed message through lbm_last_error().
namespace lbm {
void set_last_error(const char *msg) { g_last_error = msg; }

// DFT index held at position p after the forward passes of fft_reg.cuh: radix-16 passes
// from the full length down, then one radix-RL pass (mixed-radix digit reversal).
static int freq_at(int p, int n, int radix_first) {
    if (n == 1) return 0;
    const int r = radix_first;
    const int S = n / r;
    const int next = S >= 16 ? 16 : S;
    return p / S + r * freq_at(p % S, S, next);
}

void position_frequencies(int N, int *out) {
    int l2 = 0;
    while ((1 << l2) < N) ++l2;
    const int first = l2 >= 4 ? 16 : N;
    for (int p = 0; p < N; ++p) {
        const int k = freq_at(p, N, first);
        out[p] = k < N / 2 ? k : k - N;
    }
}

void derivative_tables(int N, double d, double win_alpha, double win_p, double *k1, double *k2, int terms) {
    static const double c[8] = {1.0, 1.0 / 6.0, 3.0 / 40.0, 5.0 / 112.0, 35.0 / 1152.0,
                                63.0 / 2816.0, 231.0 / 13312.0, 143.0 / 10240.0};
    int l2 = 0;
    while ((1 << l2) < N) ++l2;
    const int first = l2 >= 4 ? 16 : N;
    const int E = N < 16 ? N : 16, G = N / E;  // stored at G e + t for position E t + e
    for (int pos = 0; pos < N; ++pos) {
        const int k = freq_at(pos, N, first);
        const int m = k < N / 2 ? k : k - N;
        double ke = 0.0;
        if (2 * m != -N) {
            // Eq. (3): k_eff = (2/d) sum_{n=0}^{terms-1} c_n phi^(2n+1), phi = sin(pi m / N)
            const double phi = std::sin(M_PI * (double)m / (double)N);
            double s = 0.0, pw = phi;
            for (int n = 0; n < terms; ++n) {
                s += c[n] * pw;
                pw *= phi * phi;
            }
            const double w = win_alpha > 0
                                 ? std::exp(-win_alpha * std::pow(std::fabs((double)m) / (0.5 * N), win_p))
                                 : 1.0;
            ke = w * 2.0 / d * s;
        }
        const int at = G * (pos % E) + pos / E;
        k1[at] = ke / N;
        k2[at] = -ke * ke / N;
    }
}

void filter_table(int N, double alpha, double p, double *kf) {
    int l2 = 0;
    while ((1 << l2) < N) ++l2;
    const int first = l2 >= 4 ? 16 : N;
    const int E = N < 16 ? N : 16, G = N / E;  // stored at G e + t for position E t + e
    for (int pos = 0; pos < N; ++pos) {
        const int k = freq_at(pos, N, first);
        const int m = k < N / 2 ? k : k - N;
        const double w = alpha > 0 ? std::exp(-alpha * std::pow(std::fabs((double)m) / (0.5 * N), p)) : 1.0;
        kf[G * (pos % E) + pos / E] = (w - 1.0) / N;
    }
}

void pass_geometry(int nx, int ny, size_t esize, Geometry *g) {
    int lx = 0, ly = 0;
    while ((1 << lx) < nx) ++lx;
    while ((1 << ly) < ny) ++ly;
    const size_t cs = 2 * esize;  // complex element
    // column tiles: W columns = W/2 lines of G threads; at most pass_threads and 100 KB
    int W = (int)(128 / esize);
    if (W > nx) W = nx;
    const int maxt = max_threads(esize), colt = pass_threads(esize);
    while (W > 2 && ((W / 2) * line_G(ly) > colt || col_smem(W, ly, esize) > 100 * 1024)) W >>= 1;
    g->colW = g->fluxW = W;
    g->col_smem = g->flux_smem = col_smem(W, ly, esize);
    // float32 columns of 2048+ points: the TMA form with one staging buffer (measured against the
    // direct form: 2048^2 step 1.80 -> 1.70 ms, 4096^2 8.44 -> 8.29 ms); elsewhere the direct form
    g->col_kind = g->flux_kind = LBM_COL_DIRECT;
    if (esize == 4 && ly >= 11 && ((size_t)nx * esize) % 16 == 0) {
        const size_t sm = col_tma_smem(nx, ny, W, esize, 1);
        if (sm > 0 && sm <= kMaxCtaSmem) g->col_kind = g->flux_kind = LBM_COL_TMA1;
    }
    // row kernels: rows per CTA, starting from about 512 nodes per CTA
    const int G = line_G(lx);
    const size_t SM = (size_t)line_smem(lx) * cs;
    int r0 = 512 / nx;
    if (r0 < 1) r0 = 1;
    if (r0 > ny) r0 = ny;
    int r = r0;
    while (r > 1 && 6 * r * SM > 200 * 1024) r >>= 1;  // update: 6 line buffers per row
    g->rows_upd = r;
    g->upd_smem = 6 * (size_t)r * SM;
    // a row whose 6 line buffers exceed a CTA's shared memory (float64, nx = 4096: 418 KB) takes
    // its x-derivatives from a separate row pass instead (float32 at 4096 needs 209 KB and fits)
    g->upd_ax = g->upd_smem > kMaxCtaSmem;
    if (g->upd_ax) g->upd_smem = 0;
    // float32 rows of 4096: a cluster of four CTAs splits each row (two CTAs per SM instead of
    // the one that a whole row's 209 KB of line buffers leaves, and the six line transforms in
    // one batch; update pass per 4096^2 step: 3.37 ms over four CTAs, 3.55 over two)
    g->upd_cs = 1;
    if (esize == 4 && lx >= 12 && r == 1) {
        g->upd_cs = 4;
        g->upd_smem = upd_smem(1, lx, esize, 4);
    }
    r = r0;
    // macro: 2 lines per row with 3 buffers
    auto macro_bytes = [&](int rr) { return macro_smem(rr, lx, esize); };
    const int mact = macro_threads(esize, lx);
    while (r > 1 && (2 * r * G > mact || macro_bytes(r) > 200 * 1024)) r >>= 1;
    g->rows_macro = r;
    g->macro_smem = macro_bytes(r);
    // one row's two thread groups do not fit (float64, nx = 4096): one group, lines in turn,
    // and K rho d_x rho in a global slot instead of shared memory
    g->macro_serial = 2 * G > mact || g->macro_smem > kMaxCtaSmem;
    if (g->macro_serial) g->macro_smem = 3 * (size_t)SM;
    r = r0;
    while (r > 1 && r * G > maxt) r >>= 1;  // one line per row (diagnostics)
    g->rows_rowd = r;
    g->rowd_smem = (size_t)r * SM;
}
}  // namespace lbm
