// Internal declarations of the D2V16-FFT-TLB CUDA library (sm_103a).
//
// One Runge-Kutta stage (Sec. 2.3) is four kernel passes over HBM-resident fields:
//   K_COL     column pass: y-derivatives of 12 f_i (those with v_iy != 0) and of the
//             moments rho, u_x, u_y, T (d_y rho, d_yy rho, d_y u_x, d_y u_y, d_y T)
//   K_MACRO   row pass: x-derivatives of the moments, van der Waals pressure, stress
//             Lambda, the fluxes S and Q, the x-halves of div S and div Q, and the part
//             of C known at this point
//   K_FLUX    column pass: y-halves of div S, div Q and d_y(div u)
//   K_UPDATE  row pass: x-derivatives of 12 f_i, f^eq, I_i (Eq. (2)), BGK, the stage
//             combination, and the moments of the new f for the next stage
// With no spectral window the 2D derivative multiplier i (v_x k_x + v_y k_y) splits
// exactly into a row operator and a column operator, so every derivative is one line
// transform pair along one axis.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "fft_reg.cuh"
#include "lbm_d2v16.h"
#include "tma.cuh"

namespace lbm {

// D2V16 velocities (0-based), Sec. 2.1 (values: see the header comment of lbm_d2v16.h): the
// Kataoka-Tsutahara speeds 1 and 6 along the axes, sqrt2 and 3/sqrt2 along the diagonals.
__host__ __device__ constexpr double vel_x(int i) {
    switch (i) {
        case 0: return 1.0;  case 2: return -1.0;
        case 4: return 6.0;  case 6: return -6.0;
        case 8: return 1.0;  case 9: return -1.0;  case 10: return -1.0;  case 11: return 1.0;
        case 12: return 1.5; case 13: return -1.5; case 14: return -1.5; case 15: return 1.5;
        default: return 0.0;
    }
}
__host__ __device__ constexpr double vel_y(int i) {
    switch (i) {
        case 1: return 1.0;  case 3: return -1.0;
        case 5: return 6.0;  case 7: return -6.0;
        case 8: return 1.0;  case 9: return 1.0;  case 10: return -1.0;  case 11: return -1.0;
        case 12: return 1.5; case 13: return 1.5; case 14: return -1.5; case 15: return -1.5;
        default: return 0.0;
    }
}
// |v_i|^2 (without eta)
__host__ __device__ constexpr double vel_sq(int i) {
    return i < 4 ? 1.0 : (i < 8 ? 36.0 : (i < 12 ? 2.0 : 4.5));
}
// fields with v_x != 0, in the order of the 12 real rows of the update kernel's shared tile:
// row k holds field XF(k); complex line p packs rows 2p (real part) and 2p+1 (imag part)
__host__ __device__ constexpr int xfield(int k) { return k < 4 ? 2 * k : k + 4; }
__host__ __device__ constexpr int xslot(int i) { return i < 8 ? ((i & 1) ? -1 : i / 2) : i - 4; }
// fields with v_y != 0 and their slot in the 12-field column-pass output Ay
__host__ __device__ constexpr int yfield(int k) { return k < 4 ? 2 * k + 1 : k + 4; }
__host__ __device__ constexpr int yslot(int i) { return i < 8 ? ((i & 1) ? i / 2 : -1) : i - 4; }

// Line-transform geometry (fft_reg.cuh): points per thread, threads per line, and the stride
// between padded shared-memory line buffers in complex elements, for a line of 2^log2n points.
__host__ __device__ constexpr int line_E(int log2n) { return log2n < 4 ? (1 << log2n) : 16; }
__host__ __device__ constexpr int line_G(int log2n) { return (1 << log2n) / line_E(log2n); }
__host__ __device__ constexpr int line_smem(int log2n) { return (1 << log2n) + ((1 << log2n) >> 4) + 2; }
// threads per CTA of the line-transform kernels: float32 768 (<= 85 registers per thread),
// float64 384 (<= 170): one line's 16 complex points live in registers
template <typename R> struct MaxThreads {
    static constexpr int value = sizeof(R) == 8 ? 384 : 768;
};
__host__ __device__ constexpr int max_threads(size_t esize) { return esize == 8 ? 384 : 768; }
// column and update kernels: float32 CTAs of at most 512 threads, two resident per SM
// (<= 64 registers per thread); float64 as above
template <typename R> struct PassThreads {
    static constexpr int value = sizeof(R) == 8 ? 384 : 512;
    static constexpr int min_blocks = sizeof(R) == 8 ? 1 : 2;
};
__host__ __device__ constexpr int pass_threads(size_t esize) { return esize == 8 ? 384 : 512; }
// CTAs per cluster for a column tile of W columns of lines of 2^log2n points: 1 when the tile's
// W/2 lines fit one CTA's threads, else the split (2 or 4, lines of 512+ points) that makes
// them fit; 0 when no split serves the width
__host__ __device__ constexpr int col_cluster(int W, int log2n, size_t esize) {
    return (W / 2) * line_G(log2n) <= pass_threads(esize) ? 1
           : (log2n < 9)                                 ? 0
           : (W / 2) * line_G(log2n) <= 2 * pass_threads(esize) ? 2
           : (W / 2) * line_G(log2n) <= 4 * pass_threads(esize) ? 4
                                                                 : 0;
}
// shared memory of an update-pass CTA: 6 line buffers per row of its share (1 / cs) of the row
__host__ __device__ constexpr size_t upd_smem(int rows, int log2n, size_t esize, int cs) {
    return (size_t)6 * rows * (((1 << log2n) / cs) + (((1 << log2n) / cs) >> 4) + 2) * 2 * esize;
}
// Distance, in complex elements, between the line buffers of a column tile. The tile's L = W/2
// lines share warps (line index fastest), and shared memory serves an 8-byte access per
// half-warp and a 16-byte one per quarter-warp, in which each line's points cover 128/L
// contiguous bytes (or a stride-17 pattern over as many banks). So each padded buffer (nl +
// nl/16 elements for nl positions) is rounded up to 128 bytes and consecutive buffers start
// 128/L bytes apart in bank space (one element at least): the lines of a half- or quarter-warp
// take disjoint banks. The distance is a compile-time constant of each kernel (a run-time one
// costs the transforms registers), set for the kernel's default tile: 128 bytes of a row,
// halved until the tile's lines fit the CTAs of a cluster of cs; other widths stay correct.
__host__ __device__ constexpr int log2_int(int v) { return v > 1 ? 1 + log2_int(v >> 1) : 0; }
__host__ __device__ constexpr int col_tile_log2W(int log2n, size_t esize, int cs) {
    int lw = log2_int((int)(128 / esize));
    while (lw > 1 && (1 << (lw - 1)) * line_G(log2n) > cs * pass_threads(esize)) --lw;
    return lw;
}
__host__ __device__ constexpr int col_line_stride(int log2n, size_t esize, int cs) {
    const int nl = (1 << log2n) / cs, per128 = (int)(128 / (2 * esize));
    const int base = (int)((((size_t)(nl + (nl >> 4)) * 2 * esize + 127) / 128) * per128);
    const int off = per128 >> (col_tile_log2W(log2n, esize, cs) - 1);
    return base + (off > 0 ? off : 1);
}
// shared memory of a macroscopic row-pass CTA: three line buffers per row
__host__ __device__ constexpr size_t macro_smem(int rows, int log2n, size_t esize) {
    return (size_t)3 * rows * line_smem(log2n) * 2 * esize;
}
// shared memory of a direct column-pass CTA: W/2 line buffers of its share of each line
__host__ __device__ constexpr size_t col_smem(int W, int log2n, size_t esize) {
    return col_cluster(W, log2n, esize) == 0
               ? 0
               : (size_t)(W / 2) * col_line_stride(log2n, esize, col_cluster(W, log2n, esize)) * 2 * esize;
}
// macroscopic row pass (two lines of G threads per row): float32 CTAs of max(128, 2 G)
// threads; at 128 (nx <= 1024) seven are resident per SM (<= 72 registers per thread), so
// that 1024 rows fit in one wave of 152 SMs; at 256 (nx = 2048) three (<= 85 registers: 2048^2
// step 1.70 -> 1.56 ms against one); at 512 (nx = 4096) one (two at 64 registers spill, and
// that macro pass took 620 instead of 535 us per launch at 4096^2)
__host__ __device__ constexpr int macro_threads(size_t esize, int log2n) {
    return esize == 8 ? 384 : (2 * line_G(log2n) > 128 ? 2 * line_G(log2n) : 128);
}
template <typename R, int LOG2N> struct MacroThreads {
    static constexpr int value = macro_threads(sizeof(R), LOG2N);
    static constexpr int min_blocks = sizeof(R) == 8 ? 1 : value == 128 ? 7 : value == 256 ? 3 : 1;
};
// every supported line length 2^1 .. 2^12
#define LBM_FOR_LOG2N(X) X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12)

// Derivative multiplier tables of one axis in the digit-reversed order left by the forward
// transforms: k1[p] = W(m) k_eff(m) / N and k2[p] = -(W(m) k_eff(m))^2 / N for the DFT index m
// held at position p (zero at the Nyquist index). Eq. (3) and the window W (lbm_api.cu).
void derivative_tables(int N, double d, double win_alpha, double win_p, double *k1, double *k2, int terms = 8);
// The correction of the solution filter, (W(m) - 1) / N, of one axis in the same order (W(m) =
// exp(-alpha (|m|/(N/2))^p), the Nyquist index included): filtered = f + the inverse transform
// of the correction times the spectrum, so the rounding of the transforms touches only the small
// removed part and the mean (W(0) = 1) is kept exactly (lbm_api.cu).
void filter_table(int N, double alpha, double p, double *kf);

// Launch geometry of the four passes for an nx x ny grid and an element size (lbm_api.cu):
// column tile width and shared memory, rows per CTA and shared memory of the row kernels.
// opt-in dynamic shared memory per CTA on sm_100 / sm_103 (227 KB)
constexpr size_t kMaxCtaSmem = 232448;

struct Geometry {
    int colW = 2;            // column pass of the f and macroscopic fields
    size_t col_smem = 0;
    int fluxW = 2;           // flux column pass (tuned apart: 4 jobs instead of 17)
    size_t flux_smem = 0;
    int rows_upd = 1, rows_macro = 1, rows_rowd = 1;
    size_t upd_smem = 0, macro_smem = 0, rowd_smem = 0;
    bool upd_ax = false;        // update pass takes d_x f from a separate row pass (Ax)
    bool macro_serial = false;  // macro pass transforms a row's two lines in turn
    int upd_cs = 1;             // update pass: CTAs per row (2: a cluster splits each row)
    int col_kind = 0;           // column pass: LBM_COL_DIRECT, LBM_COL_TMA, LBM_COL_LOOKAHEAD or LBM_COL_TMA1 (width colW)
    int flux_kind = 0;          // flux column pass: the same choice (width fluxW)
};
void pass_geometry(int nx, int ny, size_t esize, Geometry *g);

// twiddles and derivative multipliers of one axis (digit-reversed order, see fft_reg.cuh)
template <typename R> struct Axis {
    const typename cplx<R>::T *tw;  // exp(-2 pi i k/N), k < N
    const R *k1;                    // k_eff(m(p)) / N, 0 at Nyquist
    const R *k2;                    // -k_eff(m(p))^2 / N, 0 at Nyquist
    int log2n;
};

// ---- HBM layout ------------------------------------------------------------------------
// Row-interleaved field blocks: a group of NF fields over an nx x ny grid is stored as
// [ny][NF][nx], so that field k of row y starts at (y NF + k) nx. One row of one field is
// contiguous (row passes and column tiles stay coalesced), and the NF values of a node are
// nx apart: one base address per node, the fields at immediate offsets.
constexpr int NF_F = 16;  // distributions f_i
constexpr int NF_A = 12;  // y-advection partials v_iy d_y f_i of the fields with v_iy != 0
// macroscopic block: moments, then the stage intermediates
enum MacroField {
    M_RHO, M_UX, M_UY, M_T,                    // moments of the current f
    M_RY, M_RYY, M_UXY, M_UYY, M_TY,           // column pass: d_y rho, d_yy rho, d_y u_x, d_y u_y, d_y T
    M_QY, M_SXY, M_SYY, M_DIVU,                // macro row pass -> flux column pass
    M_DQX, M_DSXX, M_DSXY, M_CNUM,             // macro row pass -> update pass
    M_DQY, M_DSXYY, M_DSYY, M_DDIVUY,          // flux column pass -> update pass
    NF_M
};

// ---- column derivative pass -------------------------------------------------------
// job: out = c * d^order/dy^order (in), one field per job; in/out point at the field's first
// row, row y at + y * ld (elements)
template <typename R> struct ColJob {
    const R *in;
    R *out;
    int ld_in, ld_out;
    int order;
    R c;
    int acc;  // 1: out = in + the transform's result (in place: the solution filter's correction)
};
#define LBM_MAX_COLJOBS 20
template <typename R> struct ColArgs {
    ColJob<R> jobs[LBM_MAX_COLJOBS];
    int nx, ny, W, log2W;  // ny: rows of one instance
    int nb;                // instances stacked along y (grid.z); row k ny + y of a field = instance k, row y
    Axis<R> ay;
    int pf;                // L2 lookahead of the direct kernel: CTA b first prefetches the input rows of
                           // the tile of CTA b + pf (about one wave of resident CTAs later); 0: none
};

// TMA-fed column pass (kernels_col.cu): a persistent grid of CTAs walks the work items
// (job, tile of W columns, instance); each CTA stages its next item's whole column tile in
// shared memory with tiled bulk tensor copies while it transforms the current one, and the
// staging buffer of the current item doubles as its transforms' line buffers.
template <typename R> struct ColTmaArgs {
    CUtensorMap map[LBM_MAX_COLJOBS];  // per job: the input field as a 2D tensor (nx, nb ny), box (W, boxr)
    ColArgs<R> c;
    int boxr;             // rows per copy (<= 256)
    int items;            // jobs x tiles x instances
    unsigned stage_bytes; // one staging buffer (also the item's line buffers), multiple of 128
    int *err;             // device error word (tma::kErrTimeout when a bounded wait gives up)
    long long wait_cycles;  // budget of one wait
    int starve;           // fault-injection hook: arm the barriers but issue no copies
    int nstage;           // staging buffers: 2 (the next item's copies land during this one) or 1
};
// Shared memory of the TMA column pass for a tile of W columns of ny rows (nstage = 1 or 2
// staging buffers, and two barriers); 0 if TMA cannot serve the shape.
size_t col_tma_smem(int nx, int ny, int W, size_t esize, int nstage);
// Encodes the job tensor maps and launches on a persistent grid of as many CTAs as fit (one per
// item at most) with nstage (1 or 2) staging buffers each; cudaErrorNotSupported when the shape
// or the driver cannot use TMA.
template <typename R>
cudaError_t launch_col_tma(const ColArgs<R> &a, int njobs, int *err, long long wait_cycles, int starve,
                           cudaStream_t s, int nstage);

// ---- row pass of the macroscopic chain ---------------------------------------------
template <typename R> struct MacroArgs {
    R *m;  // macroscopic block [ny][NF_M][nx]
    int nx, ny, rows;
    int serial;  // one thread group transforms both lines of a row in turn (float64, nx = 4096)
    Axis<R> ax;
    R K, H, q, zeta;
    // LBM_MIXED_RHO64: the float64 density chain [ny][NR64][nx] (nullptr otherwise) and the
    // parameters in float64 for the terms evaluated in float64
    const double *r64;
    double K64, H64, q64, zeta64;
    // diagnostics of the stage's input state fused into the pass (float32, nullptr otherwise):
    // five float64 partial values per CTA (as the diagnostics kernel writes them), hK = K/2
    double *diag_partial;
    float diag_hK;
};
// fields of the float64 density chain (LBM_MIXED_RHO64): rho = the float64 sum of the stored f,
// d_x rho, d_xx rho (row derivatives), d_y rho, d_yy rho (column derivatives)
enum Rho64Field { R64_RHO, R64_RX, R64_RXX, R64_RY, R64_RYY, NR64 };
// rho in float64 as the sum of the 16 stored distributions of each node (f: [ny][16][nx])
cudaError_t launch_rho64(const float *f, double *r64, int nx, int ny, cudaStream_t s);
// initial-field validity: the lowest failing node index into *bad (untouched if none fails)
cudaError_t launch_check_init(const double *rho, const double *ux, const double *uy, const double *T, long long n,
                              unsigned long long *bad, cudaStream_t s);

// ---- fused update row pass -----------------------------------------------------------
// tables of the model read with compile-time indices by the node loop (kernel parameters, so
// they are operands from the constant bank)
template <typename R> struct UpdateConst {
    R psi_hi[16], psi_lo[16];  // psi_i = |v_i|^2 + eta_i^2 as a two-term sum (hi + lo)
    R minv[256];               // inverse of the 16x16 moment matrix, row-major
};
template <typename R> struct UpdateArgs {
    const R *fs;     // f of this stage (derivatives, BGK, f^eq moments), [ny][16][nx]
    const R *fbase;  // f^n (the stage starts from it)
    R *fout;         // f^{n+1/2} or f^{n+1}; may alias fbase (same node, same thread)
    const R *Ay;     // [ny][12][nx]: -h v_iy d_y f_i (the stage's h folded in by the column pass)
    const R *Ax;     // nullptr: the kernel transforms its rows; else [ny][16][nx]: d_x f_i from a
                     // separate row pass (rows too long for the kernel's shared memory)
    R *m;            // macroscopic block; moments of fs in, moments of fout out
    int nx, ny, rows;
    int lines_per_batch;  // line transforms in flight per batch (the other threads wait)
    int cs;               // CTAs per row: 1, or 2 / 4 (a cluster splits the row; float32 rows of 2048+ / 4096)
    Axis<R> ax;
    R tau_inv, h, K, b, eta2;  // eta2 = eta0^2
    R cx[6];  // multiplier of row-transform line q: -h v_x of its first field (the second has -v_x)
    R T_iso;                   // LBM_FLAG_ISOTHERMAL: T at every node
    int flags;
    UpdateConst<R> k;          // the model's tables (a batch kernel passes one copy for all groups)
};

// lines per batch of the update pass: the largest divisor of the CTA's lines with LB G <= maxt
inline int update_lines_per_batch(int nlines, int G, int maxt) {
    int best = 1;
    for (int d = 1; d <= nlines; ++d)
        if (nlines % d == 0 && d * G <= maxt) best = d;
    return best;
}

// ---- persistent batch kernel (kernels_batch.cu) ----------------------------------------
constexpr int kBatchGroups = 4;  // size groups one persistent launch takes
constexpr int kBatchPasses = 8;  // passes of a step per instance: (column, macro, flux, update) x 2 stages
template <typename R> struct BatchGroup {
    ColArgs<R> col[2], flux[2];  // per stage
    MacroArgs<R> macro;          // the same for both stages
    UpdateArgs<R> upd[2];        // per stage (lines_per_batch set for the batch kernel's CTA)
    int ntile[4];                // items per instance: column (jobs x column tiles), macro row blocks,
                                 // flux (4 jobs x column tiles), update row blocks
    int tiles_x[2];              // column tiles of the column and flux passes
    int inst0;                   // the group's first instance in the completion counters
};
template <typename R> struct BatchArgs {
    BatchGroup<R> g[kBatchGroups];
    int ngroups;
    int seg[kBatchPasses * kBatchGroups + 1];  // first queue index of each (pass of the chain, group)
    int *ctrl;              // [0] queue counter, [1] abort flag, then [instances][kBatchPasses]
                            // completed items (all zeroed before each launch)
    int *err;               // device error word (tma::kErrTimeout)
    long long wait_cycles;  // budget of one wait
    int withhold;           // fault-injection hook: item 0 never reports completion
};
// tpb: threads per CTA of the persistent kernel, 256 or 512
template <typename R>
cudaError_t launch_batch_step(const BatchArgs<R> &a, size_t smem, int grid, int tpb, cudaStream_t s);
template <typename R> cudaError_t batch_step_ctas_per_sm(size_t smem, int tpb, int *n);

struct InitArgs {
    const double *rho, *ux, *uy, *T;  // inputs, [ny][nx]
    void *f;                          // [ny][16][nx] R
    void *m;                          // macroscopic block: the moments of the stored f (R)
    int nx, ny;
    double b;
    double T_iso;  // > 0: isothermal (T_iso replaces the input T)
    double minv[256];
    double psi[16];
};

struct MomArgs {
    const void *f;  // [ny][16][nx]
    void *m;        // macroscopic block
    int nx, ny;
    double psi[16];
    double b;
    double T_iso;  // > 0: isothermal (stored as the temperature field)
};

// ---- diagnostics of float32 states: exact float-pair sums ----------------------------
// A float32 value pair hi + lo (about 48 significant bits) and its exact-sum update (Knuth's
// TwoSum for hi, the error into lo), for sums of float32 terms without float64 arithmetic
// (GB300's float64 rate is 1/64 of float32).
struct FPair {
    float hi = 0.f, lo = 0.f;
    __device__ __forceinline__ void add(float x) {
        const float t = __fadd_rn(hi, x);
        const float bp = __fsub_rn(t, hi);
        lo = __fadd_rn(lo, __fadd_rn(__fsub_rn(hi, __fsub_rn(t, bp)), __fsub_rn(x, bp)));
        hi = t;
    }
    // x y added exactly: the product's rounding error from fmaf
    __device__ __forceinline__ void add_prod(float x, float y) {
        const float p = __fmul_rn(x, y);
        add(p);
        lo = __fadd_rn(lo, fmaf(x, y, -p));
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
    __device__ __forceinline__ void merge(const FPair &o) {
        add(o.hi);
        lo = __fadd_rn(lo, o.lo);
    }
    // the larger of two non-negative pairs (by hi, then lo)
    __device__ __forceinline__ void take_max(const FPair &o) {
        if (o.hi > hi || (o.hi == hi && o.lo > lo)) hi = o.hi, lo = o.lo;
    }
};
// One node's share of the diagnostics (Sec. 2.2): mass rho, momentum rho u, the energy density
// e_T = rho T - 9/8 rho^2 + K/2 |grad rho|^2 + rho |u|^2 / 2, and |u|^2 for its maximum. The
// large terms (rho, rho u, rho T, 9/8 rho^2, |u|^2) enter exactly as float pairs, the small
// ones (the gradient and kinetic parts of e_T) in float32. hK = K/2.
__device__ __forceinline__ void diag_accumulate(FPair S[5], float rho, float ux, float uy, float T, float rx, float ry,
                                                float hK) {
    S[0].add(rho);
    S[1].add_prod(rho, ux);
    S[2].add_prod(rho, uy);
    FPair u2;  // |u|^2 exactly
    u2.add_prod(ux, ux);
    u2.add_prod(uy, uy);
    S[3].add_prod(rho, T);
    const float r2 = __fmul_rn(rho, rho), er2 = fmaf(rho, rho, -r2);  // rho^2 = r2 + er2
    S[3].add_prod(-1.125f, r2);
    S[3].lo = __fadd_rn(S[3].lo, fmaf(hK, fmaf(rx, rx, ry * ry), fmaf(-1.125f, er2, 0.5f * rho * u2.hi)));
    S[4].take_max(u2);
}
// Block reduction, part 1 (every thread): each warp's pairs by shuffles into wpart[warp].
__device__ __forceinline__ void diag_warp_reduce(FPair S[5], float (*wpart)[5][2]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        for (int d = 16; d > 0; d >>= 1) {
            FPair o;
            o.hi = __shfl_down_sync(0xffffffffu, S[k].hi, d);
            o.lo = __shfl_down_sync(0xffffffffu, S[k].lo, d);
            if (k < 4) S[k].merge(o);
            else S[k].take_max(o);
        }
        if (lane == 0) wpart[warp][k][0] = S[k].hi, wpart[warp][k][1] = S[k].lo;
    }
}
// Part 2 (after a CTA barrier; the first warp works): the warps' pairs into the block's five
// float64 partial values (sums of mass, x and y momentum, e_T; the max of |u|^2).
__device__ __forceinline__ void diag_block_write(const float (*wpart)[5][2], double *out) {
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    if (threadIdx.x >= 32) return;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        FPair v;
        if (lane < nw) v.hi = wpart[lane][k][0], v.lo = wpart[lane][k][1];
        for (int d = 16; d > 0; d >>= 1) {
            FPair o;
            o.hi = __shfl_down_sync(0xffffffffu, v.hi, d);
            o.lo = __shfl_down_sync(0xffffffffu, v.lo, d);
            if (k < 4) v.merge(o);
            else v.take_max(o);
        }
        if (lane == 0) out[k] = v.value();
    }
}

// rho, u, T, d_x rho, d_y rho: row y of each at p + y * ld
struct DiagArgs {
    const void *rho, *ux, *uy, *T, *rx, *ry;
    int ld;
    double *partial;  // [blocks][5]
    int nx, ny;
    double K, cell;
};

template <typename R> struct RowDerivArgs {
    const R *in[4];
    R *out[4];
    int ld;  // row stride of every in / out field (elements)
    int nin;  // 1..4 inputs (paired two per complex line)
    int nx, ny, rows;
    int order;  // 1: d_x (table k1); 2: the real multiplier of table k2 (a second derivative or a filter)
    int acc;    // 1: out = in + the result (in place: the solution filter's correction)
    Axis<R> ax;
};

// ---- structure factor (kernels_sf.cu) -------------------------------------------------
struct SfArgs {
    const void *rho;         // density field, row y at rho + y * ld (element type of the path)
    int ld;                  // row stride in elements
    int nx, ny, lx, ly;      // grid and log2 sizes
    int rows, cols;          // rows per CTA of the row pass, columns per CTA of the column pass
    double2 *Z;              // scratch [ny][nx]: row spectra (digit-reversed positions)
    const double2 *twx, *twy;  // float64 twiddle tables of the two axes
    const int *fx, *fy;      // signed DFT index at each position of the two axes
    double sx, sy;           // shell scaling N/nx, N/ny (N = max(nx, ny))
    int nbins;
    double *S;               // [nbins] sums of |rho_hat|^2 / (nx ny) per shell (zeroed by the caller)
};

// Lets kernel `kern` use the device's whole opt-in dynamic shared memory per CTA. The limit is
// a property of the kernel function, not of a launch: a captured CUDA graph launches its
// nodes later, when another launch of the same function (another simulation, another pass
// with a different tile shape) may have set a smaller limit, so it is raised to the maximum
// once and never lowered. The shared memory a launch actually uses (its occupancy) is its own
// dynamic size.
template <typename K> inline cudaError_t allow_smem(K kern) {
    int dev = 0, optin = 0;
    cudaFuncAttributes fa{};
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kern);  // static shared memory counts against the limit
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
    return e;
}

// launchers (kernels_*.cu); all return cudaGetLastError() of the launch
template <typename R> cudaError_t launch_col(const ColArgs<R> &a, int njobs, size_t smem, cudaStream_t s);
template <typename R> cudaError_t launch_macro(const MacroArgs<R> &a, size_t smem, cudaStream_t s);
template <typename R> cudaError_t launch_update(const UpdateArgs<R> &a, size_t smem, cudaStream_t s);
template <typename R> cudaError_t launch_row_deriv(const RowDerivArgs<R> &a, size_t smem, cudaStream_t s);
template <typename R> cudaError_t launch_init(const InitArgs &a, cudaStream_t s);
template <typename R> cudaError_t launch_moments(const MomArgs &a, cudaStream_t s);
template <typename R> cudaError_t launch_diag(const DiagArgs &a, int blocks, cudaStream_t s);
cudaError_t launch_twiddles(double2 *tw64, float2 *tw32, int n, cudaStream_t s);
// strided copies between a field of a block (row y at src + y ld) and a dense float64 array [ny][nx]
template <typename R>
cudaError_t launch_field_out(const R *src, int ld, double *out, int nx, int ny, cudaStream_t s);

template <typename R> cudaError_t launch_structure_factor(const SfArgs &a, cudaStream_t s);
// signed DFT index held at each position of a forward line transform of length N (lbm_api.cu)
void position_frequencies(int N, int *out);

// sets the calling thread's message returned by lbm_last_error() (lbm_api.cu)
void set_last_error(const char *msg);

}  // namespace lbm
