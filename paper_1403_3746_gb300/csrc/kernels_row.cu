// Row passes: spectral x-derivatives of whole rows fused with the node-local physics.
//
// A CTA owns `rows` consecutive rows. Each complex line (two real rows of different fields)
// is owned by G consecutive threads, which read it with coalesced accesses, transform it in
// registers (fft_reg.cuh) and leave the derivative in shared memory in natural order; the
// node loops then map threads to consecutive x. Fields live in row-interleaved blocks
// [ny][NF][nx] (lbm_internal.cuh): a node's fields are nx apart. Template parameter R is
// the arithmetic and storage type of the path (double for LBM_FP64, float for LBM_MIXED).
#include <type_traits>

#include "pass_bodies.cuh"

namespace lbm {

template <typename R, int LOG2N, bool SERIAL, bool RHO64, bool DIAG = false>
__global__ void __launch_bounds__(MacroThreads<R, LOG2N>::value, MacroThreads<R, LOG2N>::min_blocks) macro_row_kernel(const __grid_constant__ MacroArgs<R> a) {
    macro_rows<R, LOG2N, SERIAL, false, RHO64, DIAG>(a, blockIdx.x);
}

template <typename R, int LOG2N, bool MOMENT_SPACE>
__global__ void __launch_bounds__(PassThreads<R>::value, PassThreads<R>::min_blocks) update_row_kernel(const __grid_constant__ UpdateArgs<R> a) {
    update_rows<R, LOG2N, MOMENT_SPACE, 1>(a, a.k, blockIdx.x, 0u);
}

// one row per cluster of CS CTAs (consecutive blockIdx.x)
template <typename R, int LOG2N, bool MOMENT_SPACE, int CS>
__global__ void __cluster_dims__(CS, 1, 1) __launch_bounds__(PassThreads<R>::value, PassThreads<R>::min_blocks)
    update_cluster_kernel(const __grid_constant__ UpdateArgs<R> a) {
    update_rows<R, LOG2N, MOMENT_SPACE, CS>(a, a.k, blockIdx.x / CS, reg::cluster_rank());
}


template <typename R, int LOG2N, int CS> static cudaError_t launch_update_cs(const UpdateArgs<R> &a, size_t smem,
                                                                              cudaStream_t s) {
    using F = reg::LineFFT<R, LOG2N, true, CS>;
    constexpr bool MS = sizeof(R) == 4;  // float32: moment-space collision
    cudaError_t e;
    if constexpr (CS == 1) e = allow_smem(update_row_kernel<R, LOG2N, MS>);
    else e = allow_smem(update_cluster_kernel<R, LOG2N, MS, CS>);
    if (e != cudaSuccess) return e;
    // the in-kernel row transforms need 6 line buffers per row; refuse a launch without them
    const bool adv = !(a.flags & LBM_FLAG_NO_ADVECTION);
    if (adv && a.Ax == nullptr && smem < (size_t)6 * a.rows * F::STRIDE * sizeof(typename F::CT))
        return cudaErrorInvalidValue;
    if (a.Ax != nullptr && !(sizeof(R) == 8 && LOG2N == 12 && CS == 1)) return cudaErrorInvalidValue;
    if (CS > 1 && a.rows != 1) return cudaErrorInvalidValue;
    // LB line transforms at a time; at least one thread per node of the CTA's rows (up to the cap)
    constexpr int cap = PassThreads<R>::value;
    UpdateArgs<R> b = a;
    b.lines_per_batch = update_lines_per_batch(6 * a.rows, F::GL, cap);
    const int nodes = a.rows * F::NL;
    int threads = b.lines_per_batch * F::GL;
    if (threads < nodes) threads = nodes < cap ? ((nodes + 31) & ~31) : cap;
    if constexpr (CS == 1) {
        update_row_kernel<R, LOG2N, MS><<<a.ny / a.rows, threads, smem, s>>>(b);
    } else {
        if (threads < 2 * NF_F + NF_A + NF_M) threads = 2 * NF_F + NF_A + NF_M;  // one prefetching thread per field
        update_cluster_kernel<R, LOG2N, MS, CS><<<(a.ny / a.rows) * CS, threads, smem, s>>>(b);
    }
    return cudaGetLastError();
}

template <typename R, int LOG2N> static cudaError_t launch_update_n(const UpdateArgs<R> &a, size_t smem,
                                                                    cudaStream_t s) {
    if constexpr (sizeof(R) == 4 && LOG2N >= 11) {
        if (a.cs == 2) return launch_update_cs<R, LOG2N, 2>(a, smem, s);
    }
    if constexpr (sizeof(R) == 4 && LOG2N >= 12) {
        if (a.cs == 4) return launch_update_cs<R, LOG2N, 4>(a, smem, s);
    }
    if (a.cs != 1 && a.cs != 0) return cudaErrorInvalidValue;
    return launch_update_cs<R, LOG2N, 1>(a, smem, s);
}

template <typename R, int LOG2N> static cudaError_t launch_macro_n(const MacroArgs<R> &a, size_t smem,
                                                                   cudaStream_t s) {
    using F = reg::LineFFT<R, LOG2N>;
    // three line buffers per row; refuse less
    const size_t need = (size_t)3 * a.rows * F::STRIDE * sizeof(typename F::CT);
    if (smem < need) return cudaErrorInvalidValue;
    if constexpr (sizeof(R) == 8 && LOG2N == 12) {  // the only shape that needs the serial form
        if (a.serial) {
            if (a.r64) return cudaErrorInvalidValue;
            cudaError_t e = allow_smem(macro_row_kernel<R, LOG2N, true, false>);
            if (e != cudaSuccess) return e;
            macro_row_kernel<R, LOG2N, true, false><<<a.ny / a.rows, a.rows * F::G, smem, s>>>(a);
            return cudaGetLastError();
        }
    }
    if (a.serial) return cudaErrorInvalidValue;
    if (a.diag_partial && (sizeof(R) != 4 || a.r64)) return cudaErrorInvalidValue;
    if constexpr (sizeof(R) == 4) {
        if (a.diag_partial) {  // the diagnostics of the input state fused in
            cudaError_t e = allow_smem(macro_row_kernel<R, LOG2N, false, false, true>);
            if (e != cudaSuccess) return e;
            macro_row_kernel<R, LOG2N, false, false, true><<<a.ny / a.rows, 2 * a.rows * F::G, smem, s>>>(a);
            return cudaGetLastError();
        }
    }
    if constexpr (sizeof(R) == 4) {  // the float64 density chain (LBM_MIXED_RHO64)
        if (a.r64) {
            cudaError_t e = allow_smem(macro_row_kernel<R, LOG2N, false, true>);
            if (e != cudaSuccess) return e;
            macro_row_kernel<R, LOG2N, false, true><<<a.ny / a.rows, 2 * a.rows * F::G, smem, s>>>(a);
            return cudaGetLastError();
        }
    }
    if (a.r64) return cudaErrorInvalidValue;
    cudaError_t e = allow_smem(macro_row_kernel<R, LOG2N, false, false>);
    if (e != cudaSuccess) return e;
    macro_row_kernel<R, LOG2N, false, false><<<a.ny / a.rows, 2 * a.rows * F::G, smem, s>>>(a);
    return cudaGetLastError();
}

template <typename R> cudaError_t launch_update(const UpdateArgs<R> &a, size_t smem, cudaStream_t s) {
    switch (a.ax.log2n) {
#define LBM_CASE(L2) \
    case L2: return launch_update_n<R, L2>(a, smem, s);
        LBM_FOR_LOG2N(LBM_CASE)
#undef LBM_CASE
        default: return cudaErrorInvalidValue;
    }
}

template <typename R> cudaError_t launch_macro(const MacroArgs<R> &a, size_t smem, cudaStream_t s) {
    switch (a.ax.log2n) {
#define LBM_CASE(L2) \
    case L2: return launch_macro_n<R, L2>(a, smem, s);
        LBM_FOR_LOG2N(LBM_CASE)
#undef LBM_CASE
        default: return cudaErrorInvalidValue;
    }
}

template cudaError_t launch_update<double>(const UpdateArgs<double> &, size_t, cudaStream_t);
template cudaError_t launch_update<float>(const UpdateArgs<float> &, size_t, cudaStream_t);
template cudaError_t launch_macro<double>(const MacroArgs<double> &, size_t, cudaStream_t);
template cudaError_t launch_macro<float>(const MacroArgs<float> &, size_t, cudaStream_t);

}  // namespace lbm
