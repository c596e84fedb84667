// Column pass: spectral y-derivatives of whole columns (Sec. 2.3, Eq. (3) along y).
//
// A CTA owns a tile of W adjacent columns of one input field over the full height ny,
// loaded with coalesced row segments of W values. Adjacent columns are packed in pairs
// into complex lines (W/2 lines of length ny), transformed forward, multiplied by the
// job's derivative multiplier and transformed back; the output is written with the same
// coalesced row segments. blockIdx.y selects the job (input field, output field).
#include "lbm_internal.cuh"

namespace lbm {

template <typename R>
__global__ void __launch_bounds__(256) col_deriv_kernel(const __grid_constant__ ColArgs<R> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R *s0 = reinterpret_cast<R *>(smem_raw);
    const ColJob<R> &job = a.jobs[blockIdx.y];
    const int W = a.W, nx = a.nx, ny = a.ny;
    const int x0 = blockIdx.x * W;
    const int tile = ny * W;

    for (int idx = threadIdx.x; idx < tile; idx += blockDim.x) {
        const int y = idx >> a.log2W, c = idx & (W - 1);
        s0[idx] = job.in[(size_t)y * nx + x0 + c];
    }
    __syncthreads();

    const int log2n = a.ay.log2n;
    const LineSet<R> A{s0, W / 2, 2, W, 1};
    fft_forward<R, true>(A, log2n, a.ay.tw);
    spec_mul<R, true>(A, A, log2n, job.order, job.c, a.ay.k1, a.ay.k2);
    __syncthreads();
    fft_inverse<R, true>(A, log2n, a.ay.tw);

    for (int idx = threadIdx.x; idx < tile; idx += blockDim.x) {
        const int y = idx >> a.log2W, c = idx & (W - 1);
        job.out[(size_t)y * nx + x0 + c] = s0[idx];
    }
}

template <typename R>
cudaError_t launch_col(const ColArgs<R> &a, int njobs, size_t smem, cudaStream_t s) {
    if (njobs <= 0) return cudaSuccess;
    cudaError_t e =
        cudaFuncSetAttribute(col_deriv_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid(a.nx / a.W, njobs);
    col_deriv_kernel<R><<<grid, 256, smem, s>>>(a);
    return cudaGetLastError();
}

template cudaError_t launch_col<double>(const ColArgs<double> &, int, size_t, cudaStream_t);
template cudaError_t launch_col<float>(const ColArgs<float> &, int, size_t, cudaStream_t);

}  // namespace lbm
