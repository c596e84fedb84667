// Circularly averaged structure factor of the density (the domain-growth measure of the
// phase-separation runs, Sec. 3.2), in float64 from the stored moment field:
//   S(b) = mean over shell b of |rho_hat(m)|^2 / (nx ny),
// rho_hat the unnormalised 2D DFT of rho, shell b = round(|q|), q = (m_x N/nx, m_y N/ny),
// N = max(nx, ny). The mean of rho only enters m = 0 (shell 0), which the host sets to 0.
// Row pass: one forward line transform per row (imaginary part 0), the spectrum written in
// the engine's digit-reversed order. Column pass: one forward transform per spectrum column;
// each power goes to a per-CTA shared-memory histogram, flushed to global with atomics.
#include "lbm_internal.cuh"

namespace lbm {

template <typename R, int LOG2N>
__global__ void __launch_bounds__(256) sf_row_kernel(const __grid_constant__ SfArgs a) {
    using F = reg::LineFFT<double, LOG2N>;
    using CT = double2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    CT *sb = reinterpret_cast<CT *>(smem_raw);
    const int slot = threadIdx.x / F::G, t = threadIdx.x % F::G;
    const int y = blockIdx.x * a.rows + slot;
    const R *src = static_cast<const R *>(a.rho) + (size_t)y * a.ld;
    CT v[F::E];
#pragma unroll
    for (int e = 0; e < F::E; ++e) v[e] = make_double2((double)src[t + F::G * e], 0.0);
    F::template forward<reg::SyncCta>(v, sb + (size_t)slot * F::STRIDE, t, a.twx);
    CT *dst = a.Z + (size_t)y * a.nx;
#pragma unroll
    for (int e = 0; e < F::E; ++e) dst[F::E * t + e] = v[e];
}

template <int LOG2N>
__global__ void __launch_bounds__(256) sf_col_kernel(const __grid_constant__ SfArgs a) {
    using F = reg::LineFFT<double, LOG2N>;
    using CT = double2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double *hist = reinterpret_cast<double *>(smem_raw);                      // [nbins]
    CT *sb = reinterpret_cast<CT *>(smem_raw + ((a.nbins * 8 + 15) & ~15));  // line buffers
    for (int b = threadIdx.x; b < a.nbins; b += blockDim.x) hist[b] = 0.0;
    reg::cta_barrier();
    const int L = blockDim.x / F::G;
    const int l = threadIdx.x % L, t = threadIdx.x / L;  // L columns per CTA, column fastest
    const int p = blockIdx.x * L + l;                     // spectrum column (position along x)
    CT v[F::E];
#pragma unroll
    for (int e = 0; e < F::E; ++e) v[e] = a.Z[(size_t)(t + F::G * e) * a.nx + p];
    F::template forward<reg::SyncCta>(v, sb + (size_t)l * F::STRIDE, t, a.twy);
    const double qx = (double)a.fx[p] * a.sx, inv = 1.0 / ((double)a.nx * (double)a.ny);
#pragma unroll
    for (int e = 0; e < F::E; ++e) {
        const double qy = (double)a.fy[F::E * t + e] * a.sy;
        const int b = (int)rint(sqrt(qx * qx + qy * qy));
        if (b < a.nbins) atomicAdd(&hist[b], (v[e].x * v[e].x + v[e].y * v[e].y) * inv);
    }
    reg::cta_barrier();
    for (int b = threadIdx.x; b < a.nbins; b += blockDim.x)
        if (hist[b] != 0.0) atomicAdd(&a.S[b], hist[b]);
}

template <typename R, int LOG2N> static cudaError_t sf_rows(const SfArgs &a, cudaStream_t s) {
    using F = reg::LineFFT<double, LOG2N>;
    const size_t smem = (size_t)a.rows * F::STRIDE * sizeof(double2);
    cudaError_t e = allow_smem(sf_row_kernel<R, LOG2N>);
    if (e != cudaSuccess) return e;
    sf_row_kernel<R, LOG2N><<<a.ny / a.rows, a.rows * F::G, smem, s>>>(a);
    return cudaGetLastError();
}

template <int LOG2N> static cudaError_t sf_cols(const SfArgs &a, cudaStream_t s) {
    using F = reg::LineFFT<double, LOG2N>;
    const size_t smem = (size_t)((a.nbins * 8 + 15) & ~15) + (size_t)a.cols * F::STRIDE * sizeof(double2);
    cudaError_t e = allow_smem(sf_col_kernel<LOG2N>);
    if (e != cudaSuccess) return e;
    sf_col_kernel<LOG2N><<<a.nx / a.cols, a.cols * F::G, smem, s>>>(a);
    return cudaGetLastError();
}

template <typename R> cudaError_t launch_structure_factor(const SfArgs &a, cudaStream_t s) {
    cudaError_t e = cudaErrorInvalidValue;
    switch (a.lx) {
#define LBM_CASE(L2) \
    case L2: e = sf_rows<R, L2>(a, s); break;
        LBM_FOR_LOG2N(LBM_CASE)
#undef LBM_CASE
        default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    switch (a.ly) {
#define LBM_CASE(L2) \
    case L2: return sf_cols<L2>(a, s);
        LBM_FOR_LOG2N(LBM_CASE)
#undef LBM_CASE
        default: return cudaErrorInvalidValue;
    }
}

template cudaError_t launch_structure_factor<double>(const SfArgs &, cudaStream_t);
template cudaError_t launch_structure_factor<float>(const SfArgs &, cudaStream_t);

}  // namespace lbm
