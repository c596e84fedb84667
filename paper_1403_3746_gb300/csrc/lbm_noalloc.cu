// Global diagnostics without any device allocation.
//
// Some callers cannot allocate device memory at the time they need a diagnostic: host
// applications or plugins whose GPU memory is owned by another allocator or budgeted up
// front, and long-running services that must not grow their footprint after start-up.
// lbm_diagnostics_noalloc serves them. Its scratch (the spectral d_x rho and d_y rho fields,
// the per-block partial sums and the derivative tables) lives in the file-scope array below,
// which every GPU that loads this library holds until the process exits. The caller still
// passes the inputs (device fields) and the output (host array). The call copies its tables
// from host memory and waits for its stream, so it cannot be recorded into a CUDA graph: on a
// stream that is being captured it returns LBM_ERR_STATE before issuing any work.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <string>
#include <vector>

#include "lbm_internal.cuh"

using namespace lbm;

namespace {

constexpr long long kMaxNodes = 1LL << 20;  // nx * ny <= 1048576 (e.g. 1024 x 1024)
constexpr int kMaxN = 4096;                 // nx, ny <= 4096
constexpr int kMaxBlocks = 1024;            // reduction blocks

// layout of the scratch array, in doubles
constexpr size_t kOffRx = 0;                             // d_x rho   [kMaxNodes]
constexpr size_t kOffRy = kOffRx + kMaxNodes;            // d_y rho   [kMaxNodes]
constexpr size_t kOffPart = kOffRy + kMaxNodes;          // partials  [kMaxBlocks * 5]
constexpr size_t kOffK = kOffPart + kMaxBlocks * 5;      // k1x, k2x, k1y, k2y [4 * kMaxN]
constexpr size_t kOffTw64 = kOffK + 4 * kMaxN;           // double2 twiddles x, y [2 * kMaxN * 2]
constexpr size_t kOffTw32 = kOffTw64 + 4 * kMaxN;        // float2 twiddles x, y [2 * kMaxN]
constexpr size_t kScratchDoubles = kOffTw32 + 2 * kMaxN;  // about 16.3 MiB in total

static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

// errors are reported through lbm_last_error(), like every other entry point
int fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    set_last_error(buf);
    return code;
}

// Device address of the scratch array in the current device's context. In host code the
// array's name stands for a host-side shadow, not a device address, so a kernel must be given
// this address instead. It is looked up on every call (a cheap runtime query that allocates
// nothing), so a context that was reset and recreated since an earlier call is never handed a
// stale address.
int scratch_address(double **out) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
        return fail(LBM_ERR_CUDA, "cudaGetSymbolAddress of the scratch array: %s", cudaGetErrorString(e));
    *out = static_cast<double *>(p);
    return LBM_OK;
}

bool pow2(int n) { return n >= 2 && (n & (n - 1)) == 0; }
int log2i(int n) {
    int l = 0;
    while ((1 << l) < n) ++l;
    return l;
}
#define NA_TRY(expr)                                                                                   \
    do {                                                                                               \
        cudaError_t e_ = (expr);                                                                       \
        if (e_ != cudaSuccess) return fail(LBM_ERR_CUDA, "%s: %s", #expr, cudaGetErrorString(e_));      \
    } while (0)

}  // namespace

extern "C" int lbm_diagnostics_noalloc(int nx, int ny, double dx, double dy, double K, double win_alpha,
                                       double win_p, int keff_terms, const double *rho, const double *ux,
                                       const double *uy, const double *T, void *stream, double out[5]) {
    if (!rho || !ux || !uy || !T || !out) return fail(LBM_ERR_ARG, "NULL argument");
    if (!pow2(nx) || !pow2(ny) || nx > kMaxN || ny > kMaxN)
        return fail(LBM_ERR_ARG, "nx=%d, ny=%d: each must be a power of two in [2, %d]", nx, ny, kMaxN);
    const long long n = (long long)nx * ny;
    if (n > kMaxNodes)
        return fail(LBM_ERR_ARG, "nx*ny=%lld exceeds the %lld nodes of the built-in scratch array", n, kMaxNodes);
    if (!(dx > 0) || !(dy > 0) || !std::isfinite(dx) || !std::isfinite(dy) || !std::isfinite(K) ||
        !(win_alpha >= 0) || !(win_p > 0))
        return fail(LBM_ERR_ARG, "bad dx, dy, K or window parameters");
    if (keff_terms < 1 || keff_terms > 8) return fail(LBM_ERR_ARG, "keff_terms must be in [1, 8]");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    NA_TRY(cudaStreamIsCapturing(s, &cs));
    if (cs != cudaStreamCaptureStatusNone)
        return fail(LBM_ERR_STATE, "lbm_diagnostics_noalloc cannot run on a stream that is being captured "
                                   "(it copies from host memory and synchronises); no work was issued");
    double *sc = nullptr;
    int rc = scratch_address(&sc);
    if (rc) return rc;

    // derivative tables of both axes, rebuilt by every call
    double *k1x = sc + kOffK, *k2x = k1x + kMaxN, *k1y = k2x + kMaxN, *k2y = k1y + kMaxN;
    double2 *twx = reinterpret_cast<double2 *>(sc + kOffTw64), *twy = twx + kMaxN;
    float2 *twx32 = reinterpret_cast<float2 *>(sc + kOffTw32), *twy32 = twx32 + kMaxN;
    NA_TRY(launch_twiddles(twx, twx32, nx, s));
    NA_TRY(launch_twiddles(twy, twy32, ny, s));
    std::vector<double> tab(4 * (size_t)kMaxN);
    derivative_tables(nx, dx, win_alpha, win_p, tab.data(), tab.data() + kMaxN, keff_terms);
    derivative_tables(ny, dy, win_alpha, win_p, tab.data() + 2 * kMaxN, tab.data() + 3 * kMaxN, keff_terms);
    NA_TRY(cudaMemcpyAsync(k1x, tab.data(), 4 * (size_t)kMaxN * sizeof(double), cudaMemcpyHostToDevice, s));

    // d_y rho (column pass) and d_x rho (row pass) into the scratch fields
    Geometry geo;
    pass_geometry(nx, ny, sizeof(double), &geo);
    const int W = geo.colW;
    ColArgs<double> ca{};
    ca.nx = nx;
    ca.ny = ny;
    ca.W = W;
    ca.log2W = log2i(W);
    ca.ay = Axis<double>{twy, k1y, k2y, log2i(ny)};
    ca.jobs[0] = ColJob<double>{rho, sc + kOffRy, nx, nx, 1, 1.0};
    NA_TRY(launch_col<double>(ca, 1, geo.col_smem, s));
    RowDerivArgs<double> ra{};
    ra.in[0] = rho;
    ra.out[0] = sc + kOffRx;
    ra.ld = nx;
    ra.nin = 1;
    ra.nx = nx;
    ra.ny = ny;
    ra.rows = geo.rows_rowd;
    ra.order = 1;
    ra.ax = Axis<double>{twx, k1x, k2x, log2i(nx)};
    NA_TRY(launch_row_deriv<double>(ra, geo.rowd_smem, s));

    // per-block partial sums, then the final reduction on the host
    const int blocks = (int)std::min<long long>(kMaxBlocks, (n + 255) / 256);
    DiagArgs da{};
    da.rho = rho;
    da.ux = ux;
    da.uy = uy;
    da.T = T;
    da.rx = sc + kOffRx;
    da.ry = sc + kOffRy;
    da.ld = nx;
    da.partial = sc + kOffPart;
    da.nx = nx;
    da.ny = ny;
    da.K = K;
    da.cell = dx * dy;
    NA_TRY(launch_diag<double>(da, blocks, s));
    std::vector<double> part((size_t)blocks * 5);
    NA_TRY(cudaMemcpyAsync(part.data(), sc + kOffPart, part.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    NA_TRY(cudaStreamSynchronize(s));
    double acc[4] = {0, 0, 0, 0}, mx = 0;
    for (int b = 0; b < blocks; ++b) {
        for (int k = 0; k < 4; ++k) acc[k] += part[(size_t)b * 5 + k];
        mx = std::max(mx, part[(size_t)b * 5 + 4]);
    }
    const double cell = dx * dy;
    for (int k = 0; k < 4; ++k) out[k] = acc[k] * cell;
    out[4] = std::sqrt(mx);
    for (int k = 0; k < 5; ++k)
        if (!std::isfinite(out[k])) return fail(LBM_ERR_NONFINITE, "diagnostic %d is not finite", k);
    return LBM_OK;
}
