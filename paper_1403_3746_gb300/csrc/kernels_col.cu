// Column pass: spectral y-derivatives of whole columns (Sec. 2.3, Eq. (3) along y).
//
// A CTA owns a tile of W adjacent columns of one input field over the full height ny (rows of
// the field are `ld` elements apart, see the block layout in lbm_internal.cuh). Column
// pairs (2l, 2l+1) are packed into complex lines (L = W/2 lines); thread (l, t), with l the
// fast index, reads the points t + G e of its line straight from global memory, so each row
// segment of W values is one coalesced access. Forward transform, derivative multiplier
// and inverse transform run in registers with shared-memory exchanges (fft_reg.cuh); the
// result is written back in the same layout. blockIdx.y selects the job (input, output).
#include "lbm_internal.cuh"

namespace lbm {

template <typename R, int LOG2N>
__global__ void __launch_bounds__(PassThreads<R>::value, PassThreads<R>::min_blocks) col_deriv_kernel(const __grid_constant__ ColArgs<R> a) {
    using F = reg::LineFFT<R, LOG2N, true>;
    using CT = typename F::CT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    CT *sbuf = reinterpret_cast<CT *>(smem_raw);
    const ColJob<R> &job = a.jobs[blockIdx.y];
    const int L = a.W >> 1;
    const int l = threadIdx.x & (L - 1), t = threadIdx.x >> (a.log2W - 1);
    const size_t rsi = (size_t)(job.ld_in >> 1), rso = (size_t)(job.ld_out >> 1);  // row strides, complex units
    const int x = blockIdx.x * a.W + 2 * l;
    // blockIdx.z: instance of a batch stacked along y (ny rows each)
    const size_t z = blockIdx.z;
    const CT *in = reinterpret_cast<const CT *>(job.in + z * a.ny * job.ld_in + x);
    CT *out = reinterpret_cast<CT *>(job.out + z * a.ny * job.ld_out + x);

    CT v[F::E];
#pragma unroll
    for (int e = 0; e < F::E; ++e) v[e] = __ldcg(in + (size_t)(t + F::G * e) * rsi);  // L2 only: single use
    CT *buf = sbuf + l * F::STRIDE;
    F::template forward<reg::SyncCta>(v, buf, t, a.ay.tw);
    F::multiply(v, t, job.order, job.c, a.ay.k1, a.ay.k2);
    F::template inverse<reg::SyncCta>(v, buf, t, a.ay.tw);
#pragma unroll
    for (int e = 0; e < F::E; ++e) out[(size_t)(t + F::G * e) * rso] = v[e];
}

template <typename R, int LOG2N> static cudaError_t launch_col_n(const ColArgs<R> &a, int njobs, size_t smem,
                                                                  cudaStream_t s) {
    using F = reg::LineFFT<R, LOG2N>;
    if (smem < (size_t)(a.W / 2) * F::STRIDE * sizeof(typename F::CT)) return cudaErrorInvalidValue;
    cudaError_t e = allow_smem(col_deriv_kernel<R, LOG2N>);
    if (e != cudaSuccess) return e;
    dim3 grid(a.nx / a.W, njobs, a.nb > 0 ? a.nb : 1);
    col_deriv_kernel<R, LOG2N><<<grid, (a.W / 2) * F::G, smem, s>>>(a);
    return cudaGetLastError();
}

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
