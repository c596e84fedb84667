// Column pass: spectral y-derivatives of whole columns (Sec. 2.3, Eq. (3) along y).
//
// A CTA owns a tile of W adjacent columns of one input field over the full height ny (rows of
// the field are `ld` elements apart, see the block layout in lbm_internal.cuh). Column
// pairs (2l, 2l+1) are packed into complex lines (L = W/2 lines); thread (l, t), with l the
// fast index, reads the points t + G e of its line straight from global memory, so each row
// segment of W values is one coalesced access. Forward transform, derivative multiplier
// and inverse transform run in registers with shared-memory exchanges (fft_reg.cuh); the
// result is written back in the same layout. blockIdx.y selects the job (input, output).
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

#include "pass_bodies.cuh"

namespace lbm {

// L2 lookahead (a.pf > 0): CTAs start in linear block order, so the CTA a.pf blocks later
// runs about one wave of resident CTAs after this one; its input rows are prefetched into L2
// now, one bulk prefetch per row.
template <typename R> __device__ __forceinline__ void col_lookahead(const ColArgs<R> &a) {
    const long long per_z = (long long)gridDim.x * gridDim.y;
    const long long b = blockIdx.x + (long long)gridDim.x * blockIdx.y + per_z * blockIdx.z + a.pf;
    if (b >= per_z * gridDim.z) return;
    const int z = (int)(b / per_z), rem = (int)(b % per_z), jn = rem / gridDim.x, tn = rem % gridDim.x;
    const ColJob<R> &job = a.jobs[jn];
    const unsigned bytes = (unsigned)(a.W * sizeof(R));
    const R *in = job.in + (size_t)z * a.ny * job.ld_in + (size_t)tn * a.W;
    for (int r = threadIdx.x; r < a.ny; r += blockDim.x) prefetch_l2(in + (size_t)r * job.ld_in, bytes);
}

// ACC: every job accumulates (out = in + result; the solution filter), instantiated apart.
template <typename R, int LOG2N, bool ACC>
__global__ void __launch_bounds__(PassThreads<R>::value, PassThreads<R>::min_blocks) col_deriv_kernel(const __grid_constant__ ColArgs<R> a) {
    if (a.pf > 0) col_lookahead(a);
    col_tile<R, LOG2N, 1, false, ACC>(a, blockIdx.y, blockIdx.z, blockIdx.x, 0u);
}

// Column tiles wider than one CTA's threads can transform: each line is split over the CS CTAs
// of a cluster (consecutive blockIdx.x), which exchange points through distributed shared memory.
template <typename R, int LOG2N, int CS, bool ACC>
__global__ void __cluster_dims__(CS, 1, 1) __launch_bounds__(PassThreads<R>::value, PassThreads<R>::min_blocks)
    col_cluster_kernel(const __grid_constant__ ColArgs<R> a) {
    col_tile<R, LOG2N, CS, false, ACC>(a, blockIdx.y, blockIdx.z, blockIdx.x / CS, reg::cluster_rank());
}

// whether every job of a launch accumulates (1), none does (0), or they are mixed (-1: refused)
template <typename R> static int jobs_acc(const ColArgs<R> &a, int njobs) {
    for (int j = 1; j < njobs; ++j)
        if ((a.jobs[j].acc != 0) != (a.jobs[0].acc != 0)) return -1;
    return a.jobs[0].acc != 0 ? 1 : 0;
}

template <typename R, int LOG2N, int CS, bool ACC>
static cudaError_t launch_col_cs_t(const ColArgs<R> &a, int njobs, size_t smem, cudaStream_t s) {
    using F = reg::LineFFT<R, LOG2N, true, CS>;
    dim3 grid((a.nx / a.W) * CS, njobs, a.nb > 0 ? a.nb : 1);
    if constexpr (CS == 1) {
        cudaError_t e = allow_smem(col_deriv_kernel<R, LOG2N, ACC>);
        if (e != cudaSuccess) return e;
        const int threads = (a.W / 2) * F::GL;
        if (a.pf == 0) {
            col_deriv_kernel<R, LOG2N, ACC><<<grid, threads, smem, s>>>(a);
        } else {  // lookahead distance: the CTAs resident at once
            int dev = 0, sms = 0, per_sm = 0;
            if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
            if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
            if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, col_deriv_kernel<R, LOG2N, ACC>, threads,
                                                                    smem)) != cudaSuccess)
                return e;
            ColArgs<R> b = a;
            b.pf = std::max(1, sms * per_sm);
            col_deriv_kernel<R, LOG2N, ACC><<<grid, threads, smem, s>>>(b);
        }
    } else {
        cudaError_t e = allow_smem(col_cluster_kernel<R, LOG2N, CS, ACC>);
        if (e != cudaSuccess) return e;
        col_cluster_kernel<R, LOG2N, CS, ACC><<<grid, (a.W / 2) * F::GL, smem, s>>>(a);
    }
    return cudaGetLastError();
}

template <typename R, int LOG2N, int CS> static cudaError_t launch_col_cs(const ColArgs<R> &a, int njobs, size_t smem,
                                                                           cudaStream_t s) {
    using F = reg::LineFFT<R, LOG2N, true, CS>;
    if (smem < (size_t)(a.W / 2) * col_line_stride(LOG2N, sizeof(R), CS) * sizeof(typename F::CT))
        return cudaErrorInvalidValue;
    const int acc = jobs_acc(a, njobs);
    if (acc < 0) return cudaErrorInvalidValue;
    return acc ? launch_col_cs_t<R, LOG2N, CS, true>(a, njobs, smem, s)
               : launch_col_cs_t<R, LOG2N, CS, false>(a, njobs, smem, s);
}

template <typename R, int LOG2N> static cudaError_t launch_col_n(const ColArgs<R> &a, int njobs, size_t smem,
                                                                  cudaStream_t s) {
    const int cs = col_cluster(a.W, LOG2N, sizeof(R));
    if constexpr (LOG2N >= 9) {
        if (cs == 2) return launch_col_cs<R, LOG2N, 2>(a, njobs, smem, s);
        if (cs == 4) return launch_col_cs<R, LOG2N, 4>(a, njobs, smem, s);
    }
    if (cs != 1) return cudaErrorInvalidValue;
    return launch_col_cs<R, LOG2N, 1>(a, njobs, smem, s);
}

// ---------------------------------------------------------------------------------------
// TMA-fed column pass. A persistent CTA walks the work items it + k gridDim (item = tile of W
// columns of one job's field in one instance). With two staging buffers (a.nstage = 2) item k
// is staged in buffer k & 1: thread 0 arms that buffer's barrier with the tile's byte count and
// issues ny / boxr tiled copies of (W x boxr) boxes; the copies of item k + 1 land while item k
// is transformed. Once every thread has read its points of item k into registers, the same
// buffer serves as the line buffers of item k's transforms (it is at least as large as both);
// after the CTA barrier that ends item k it is handed back to the copy engine for item k + 2.
// With one buffer (a.nstage = 1: half the shared memory, so two CTAs per SM where two buffers
// leave one) item k + 1 is issued after item k, and the CTA's copy overlaps the transforms of
// the other CTAs on its SM instead of its own. Results are written from registers, as in
// col_deriv_kernel, so every output value is bit for bit the same.
// ---------------------------------------------------------------------------------------
template <typename R, int LOG2N, bool ACC>
__global__ void __launch_bounds__(PassThreads<R>::value, PassThreads<R>::min_blocks)
    col_tma_kernel(const __grid_constant__ ColTmaArgs<R> a) {
    using F = reg::LineFFT<R, LOG2N, true>;
    using CT = typename F::CT;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const ColArgs<R> &c = a.c;
    const int W = c.W, L = W >> 1;
    const int l = threadIdx.x & (L - 1), t = threadIdx.x >> (c.log2W - 1);
    const int ns = a.nstage;  // 1 or 2
    unsigned char *stage0 = smem_raw, *stage1 = smem_raw + (ns - 1) * (size_t)a.stage_bytes;
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw + ns * (size_t)a.stage_bytes);
    volatile int *flag = reinterpret_cast<volatile int *>(bar + 2);
    const int tiles = c.nx / W, nb = c.nb > 0 ? c.nb : 1;
    const unsigned tile_bytes = (unsigned)c.ny * (unsigned)W * (unsigned)sizeof(R);
    // item -> (job, instance, tile), tile fastest
    auto job_of = [&](int it) { return it / (tiles * nb); };
    auto z_of = [&](int it) { return (it % (tiles * nb)) / tiles; };
    auto tile_of = [&](int it) { return it % tiles; };
    auto issue = [&](int it, int b) {  // thread 0
        tma::bar_arrive_expect_tx(&bar[b], tile_bytes);
        if (a.starve) return;  // fault injection: the barrier is armed, no copy will complete it
        unsigned char *dst = b ? stage1 : stage0;
        const int job = job_of(it), y0 = z_of(it) * c.ny, x0 = tile_of(it) * W;
        for (int r0 = 0; r0 < c.ny; r0 += a.boxr)
            tma::load_2d(dst + (size_t)r0 * W * sizeof(R), &a.map[job], x0, y0 + r0, &bar[b]);
    };
    bool pend0 = false, pend1 = false;  // thread 0: copies in flight per buffer
    if (threadIdx.x == 0) {
        tma::bar_init(&bar[0], 1);
        tma::bar_init(&bar[1], 1);
        tma::fence_bar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (blockIdx.x < a.items) issue(blockIdx.x, 0), pend0 = true;
        if (ns == 2 && blockIdx.x + gridDim.x < a.items) issue(blockIdx.x + gridDim.x, 1), pend1 = true;
    }
    int k = 0;
    for (int it = blockIdx.x; it < a.items; it += gridDim.x, ++k) {
        const int b = ns == 2 ? k & 1 : 0;
        if (threadIdx.x == 0) {
            bool ok = tma::bar_wait_bounded(&bar[b], ns == 2 ? (k >> 1) & 1 : k & 1, a.wait_cycles);
            if (b) pend1 = false; else pend0 = false;
            if (!ok) {
                atomicOr(a.err, tma::kErrTimeout);
                // the other buffer's copies (item k + 1) may still land: wait for them, bounded
                if (b ? pend0 : pend1) tma::bar_wait_bounded(&bar[b ^ 1], ((k + 1) >> 1) & 1, a.wait_cycles);
            }
            *flag = ok ? 1 : 0;
        }
        __syncthreads();
        if (!*flag) return;  // uniform: every thread read the same flag
        const ColJob<R> &jb = c.jobs[job_of(it)];
        CT *st = reinterpret_cast<CT *>(b ? stage1 : stage0);
        CT v[F::E];
#pragma unroll
        for (int e = 0; e < F::E; ++e) v[e] = st[(size_t)(t + F::G * e) * L + l];  // row t + G e, columns 2l, 2l+1
        CT *buf = st + l * col_line_stride(LOG2N, sizeof(R), 1);
        F::template forward<reg::SyncCta>(v, buf, t, c.ay.tw);
        F::multiply(v, t, jb.order, jb.c, c.ay.k1, c.ay.k2);
        F::template inverse<reg::SyncCta>(v, buf, t, c.ay.tw);
        const size_t rso = (size_t)(jb.ld_out >> 1), rsi = (size_t)(jb.ld_in >> 1);
        CT *out = reinterpret_cast<CT *>(jb.out + (size_t)z_of(it) * c.ny * jb.ld_out + tile_of(it) * W + 2 * l);
        const CT *inp = reinterpret_cast<const CT *>(jb.in + (size_t)z_of(it) * c.ny * jb.ld_in + tile_of(it) * W + 2 * l);
#pragma unroll
        for (int e = 0; e < F::E; ++e) {
            CT r = v[e];
            if constexpr (ACC) {  // out = in + result (in place: this thread's own positions)
                const CT o = __ldcg(inp + (size_t)(t + F::G * e) * rsi);
                r = reg::mk<R>(o.x + r.x, o.y + r.y);
            }
            out[(size_t)(t + F::G * e) * rso] = r;
        }
        reg::cta_barrier();  // every thread is done with this buffer
        if (threadIdx.x == 0 && it + ns * (int)gridDim.x < a.items) {
            tma::fence_proxy_async_smem();
            issue(it + ns * gridDim.x, b);
            if (b) pend1 = true; else pend0 = true;
        }
    }
}

size_t col_tma_smem(int nx, int ny, int W, size_t esize, int nstage) {
    if (W < 2 || W > nx || (W * esize) % 16 != 0 || (W * esize) > 256) return 0;
    int l2 = 0;
    while ((1 << l2) < ny) ++l2;
    const size_t lines = (size_t)(W / 2) * col_line_stride(l2, esize, 1) * 2 * esize;
    const size_t tile = (size_t)ny * W * esize;
    const size_t sb = (std::max(lines, tile) + 127) & ~(size_t)127;
    return nstage == 1 || nstage == 2 ? (size_t)nstage * sb + 32 : 0;
}

namespace {
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    std::call_once(g_encode_once, [] {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
        else
            cudaGetLastError();
    });
    return g_encode;
}
}  // namespace

template <typename R, int LOG2N, bool ACC>
static cudaError_t launch_col_tma_t(const ColTmaArgs<R> &a, size_t smem, cudaStream_t s) {
    using F = reg::LineFFT<R, LOG2N>;
    const int threads = (a.c.W / 2) * F::G;
    if (threads > PassThreads<R>::value ||
        a.stage_bytes < (unsigned)((a.c.W / 2) * col_line_stride(LOG2N, sizeof(R), 1) * sizeof(typename F::CT)))
        return cudaErrorNotSupported;
    cudaError_t e = allow_smem(col_tma_kernel<R, LOG2N, ACC>);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, col_tma_kernel<R, LOG2N, ACC>, threads, smem)) !=
        cudaSuccess)
        return e;
    if (per_sm < 1) return cudaErrorNotSupported;
    const int grid = std::min(a.items, sms * per_sm);
    col_tma_kernel<R, LOG2N, ACC><<<grid, threads, smem, s>>>(a);
    return cudaGetLastError();
}

template <typename R, int LOG2N>
static cudaError_t launch_col_tma_n(const ColTmaArgs<R> &a, int njobs, size_t smem, cudaStream_t s) {
    const int acc = jobs_acc(a.c, njobs);
    if (acc < 0) return cudaErrorInvalidValue;
    return acc ? launch_col_tma_t<R, LOG2N, true>(a, smem, s) : launch_col_tma_t<R, LOG2N, false>(a, smem, s);
}

template <typename R>
cudaError_t launch_col_tma(const ColArgs<R> &c, int njobs, int *err, long long wait_cycles, int starve,
                           cudaStream_t s, int nstage) {
    if (njobs <= 0) return cudaSuccess;
    const size_t es = sizeof(R);
    const size_t smem = col_tma_smem(c.nx, c.ny, c.W, es, nstage);
    if (smem == 0 || smem > kMaxCtaSmem || !err) return cudaErrorNotSupported;
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return cudaErrorNotSupported;
    ColTmaArgs<R> a{};
    a.c = c;
    a.boxr = std::min(c.ny, 256);
    const int nb = c.nb > 0 ? c.nb : 1;
    a.items = njobs * (c.nx / c.W) * nb;
    a.nstage = nstage;
    a.stage_bytes = (unsigned)((smem - 32) / nstage);
    a.err = err;
    a.wait_cycles = wait_cycles;
    a.starve = starve;
    for (int j = 0; j < njobs; ++j) {
        const ColJob<R> &jb = c.jobs[j];
        const cuuint64_t dims[2] = {(cuuint64_t)c.nx, (cuuint64_t)c.ny * nb};
        const cuuint64_t strides[1] = {(cuuint64_t)jb.ld_in * es};
        const cuuint32_t box[2] = {(cuuint32_t)c.W, (cuuint32_t)a.boxr};
        const cuuint32_t estr[2] = {1, 1};
        if ((reinterpret_cast<uintptr_t>(jb.in) & 15) || (strides[0] & 15)) return cudaErrorNotSupported;
        const CUresult r = enc(&a.map[j], es == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                               2, const_cast<R *>(jb.in), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return cudaErrorNotSupported;
    }
    switch (c.ay.log2n) {
#define LBM_CASE(L2) \
    case L2: return launch_col_tma_n<R, L2>(a, njobs, smem, s);
        LBM_FOR_LOG2N(LBM_CASE)
#undef LBM_CASE
        default: return cudaErrorInvalidValue;
    }
}

template cudaError_t launch_col_tma<double>(const ColArgs<double> &, int, int *, long long, int, cudaStream_t, int);
template cudaError_t launch_col_tma<float>(const ColArgs<float> &, int, int *, long long, int, cudaStream_t, int);

template <typename R>
cudaError_t launch_col(const ColArgs<R> &a, int njobs, size_t smem, cudaStream_t s) {
    if (njobs <= 0) return cudaSuccess;
    switch (a.ay.log2n) {
#define LBM_CASE(L2) \
    case L2: return launch_col_n<R, L2>(a, njobs, smem, s);
        LBM_FOR_LOG2N(LBM_CASE)
#undef LBM_CASE
        default: return cudaErrorInvalidValue;
    }
}

template cudaError_t launch_col<double>(const ColArgs<double> &, int, size_t, cudaStream_t);
template cudaError_t launch_col<float>(const ColArgs<float> &, int, size_t, cudaStream_t);

}  // namespace lbm
