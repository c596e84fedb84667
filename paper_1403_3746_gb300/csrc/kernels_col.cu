// Column pass: spectral y-derivatives of whole columns (Sec. 2.3, Eq. (3) along y).
//
// A CTA owns a tile of W adjacent columns of one input field over the full height ny,
// loaded with coalesced row segments of W values. Adjacent columns are packed in pairs
// into complex lines (W/2 lines of length ny), transformed forward, multiplied by the
// requested derivative multiplier(s) and transformed back; each output is written with
// the same coalesced row segments. blockIdx.y selects the job (input field + outputs).
#include "lbm_internal.cuh"

namespace lbm {

template <typename F>
__global__ void __launch_bounds__(256) col_deriv_kernel(const __grid_constant__ ColArgs<F> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    F *s0 = reinterpret_cast<F *>(smem_raw);
    const ColJob<F> &job = a.jobs[blockIdx.y];
    const int W = a.W, nx = a.nx, ny = a.ny;
    const int x0 = blockIdx.x * W;
    const int tile = ny * W;
    F *s1 = s0 + tile;

    for (int idx = threadIdx.x; idx < tile; idx += blockDim.x) {
        const int y = idx >> a.log2W, c = idx & (W - 1);
        s0[idx] = job.in[(size_t)y * nx + x0 + c];
    }
    __syncthreads();

    const int log2n = a.ay.log2n;
    LineSet<F> A{s0, W / 2, 2, W, 1};
    fft_forward<F, true>(A, log2n, a.ay.tw);
    if (job.out1) {
        LineSet<F> B{s1, W / 2, 2, W, 1};
        spec_mul<F, true>(B, A, log2n, job.order1, job.c1, a.ay.k1, a.ay.k2);
    }
    spec_mul<F, true>(A, A, log2n, job.order0, job.c0, a.ay.k1, a.ay.k2);
    __syncthreads();
    fft_inverse<F, true>(A, log2n, a.ay.tw);
    if (job.out1) {
        LineSet<F> B{s1, W / 2, 2, W, 1};
        fft_inverse<F, true>(B, log2n, a.ay.tw);
    }

    for (int idx = threadIdx.x; idx < tile; idx += blockDim.x) {
        const int y = idx >> a.log2W, c = idx & (W - 1);
        job.out0[(size_t)y * nx + x0 + c] = s0[idx];
        if (job.out1) job.out1[(size_t)y * nx + x0 + c] = s1[idx];
    }
}

template <typename F>
cudaError_t launch_col(const ColArgs<F> &a, int njobs, int threads, size_t smem, cudaStream_t s) {
    if (njobs <= 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(col_deriv_kernel<F>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid(a.nx / a.W, njobs);
    col_deriv_kernel<F><<<grid, threads, smem, s>>>(a);
    return cudaGetLastError();
}

template cudaError_t launch_col<double>(const ColArgs<double> &, int, int, size_t, cudaStream_t);
template cudaError_t launch_col<float>(const ColArgs<float> &, int, int, size_t, cudaStream_t);

}  // namespace lbm
