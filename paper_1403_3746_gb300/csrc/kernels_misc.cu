// Setup, readout and diagnostic kernels (not on the per-step hot path). Fields use the
// row-interleaved block layout of lbm_internal.cuh.
#include "lbm_internal.cuh"

namespace lbm {

// f_i := f_i^eq(rho, u, T) at every node (the initial state of Sec. 3's runs), then the
// moments of the stored f (so that the first stage uses the moments of f itself).
template <typename F>
__global__ void init_feq_kernel(const __grid_constant__ InitArgs a) {
    F *f = reinterpret_cast<F *>(a.f);
    F *m = reinterpret_cast<F *>(a.m);
    const long long n = (long long)a.nx * a.ny;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < n;
         g += (long long)gridDim.x * blockDim.x) {
        const long long y = g / a.nx, x = g - y * a.nx;
        const double rho = a.rho[g], ux = a.ux[g], uy = a.uy[g], T = a.T_iso > 0.0 ? a.T_iso : a.T[g];
        const double u2 = ux * ux + uy * uy, b = a.b;
        const double e = (b + 2.0) * T + u2, gq = (b + 4.0) * T + u2;
        const double mq[16] = {rho,
                               rho * ux,
                               rho * uy,
                               rho * (b * T + u2),
                               rho * (T + ux * ux),
                               rho * ux * uy,
                               rho * (T + uy * uy),
                               rho * ux * e,
                               rho * uy * e,
                               rho * ux * (3.0 * T + ux * ux),
                               rho * uy * (T + ux * ux),
                               rho * ux * (T + uy * uy),
                               rho * uy * (3.0 * T + uy * uy),
                               rho * (T * e + gq * ux * ux),
                               rho * gq * ux * uy,
                               rho * (T * e + gq * uy * uy)};
        F *fn = f + y * NF_F * a.nx + x;
        double mr = 0, mjx = 0, mjy = 0, mE = 0;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            double fe = 0;
#pragma unroll
            for (int j = 0; j < 16; ++j) fe += a.minv[i * 16 + j] * mq[j];
            const F fs = (F)fe;
            fn[i * a.nx] = fs;
            const double fd = (double)fs;
            mr += fd;
            mjx += vel_x(i) * fd;
            mjy += vel_y(i) * fd;
            mE += a.psi[i] * fd;
        }
        const double ir = 1.0 / mr, nux = mjx * ir, nuy = mjy * ir;
        F *mn = m + y * NF_M * a.nx + x;
        mn[M_RHO * a.nx] = (F)mr;
        mn[M_UX * a.nx] = (F)nux;
        mn[M_UY * a.nx] = (F)nuy;
        mn[M_T * a.nx] = a.T_iso > 0.0 ? (F)a.T_iso : (F)((mE * ir - (nux * nux + nuy * nuy)) / b);
    }
}

// Sec. 2.1 moments of a stored f.
template <typename F>
__global__ void moments_kernel(const __grid_constant__ MomArgs a) {
    const F *f = reinterpret_cast<const F *>(a.f);
    F *m = reinterpret_cast<F *>(a.m);
    const long long n = (long long)a.nx * a.ny;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < n;
         g += (long long)gridDim.x * blockDim.x) {
        const long long y = g / a.nx, x = g - y * a.nx;
        const F *fn = f + y * NF_F * a.nx + x;
        double mr = 0, mjx = 0, mjy = 0, mE = 0;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const double fd = (double)fn[i * a.nx];
            mr += fd;
            mjx += vel_x(i) * fd;
            mjy += vel_y(i) * fd;
            mE += a.psi[i] * fd;
        }
        const double ir = 1.0 / mr, nux = mjx * ir, nuy = mjy * ir;
        F *mn = m + y * NF_M * a.nx + x;
        mn[M_RHO * a.nx] = (F)mr;
        mn[M_UX * a.nx] = (F)nux;
        mn[M_UY * a.nx] = (F)nuy;
        mn[M_T * a.nx] = a.T_iso > 0.0 ? (F)a.T_iso : (F)((mE * ir - (nux * nux + nuy * nuy)) / a.b);
    }
}

// LBM_MIXED_RHO64: rho of every node as the float64 sum of its 16 stored float32 values (exact:
// the values span far fewer than the 29 bits a float64 has beyond a float32's significand).
__global__ void rho64_kernel(const float *f, double *r64, int nx, int ny) {
    const long long n = (long long)nx * ny;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < n;
         g += (long long)gridDim.x * blockDim.x) {
        const long long y = g / nx, x = g - y * nx;
        const float *fn = f + y * NF_F * nx + x;
        double s = 0.0;
#pragma unroll
        for (int i = 0; i < 16; ++i) s += (double)__ldcg(fn + i * nx);
        r64[(y * NR64 + R64_RHO) * nx + x] = s;
    }
}

// Per-block partial sums of mass, x/y momentum, e_T (Sec. 2.2) and the max of |u|^2.
// float64 states: float64 arithmetic. float32 states: the large terms (rho, rho u, rho T,
// 9/8 rho^2, |u|^2) enter as exact products and sums in float pairs, the small ones (the
// gradient and kinetic parts of e_T) in float32, so the sums agree with a float64 evaluation of
// the same stored values to about 1e-14 of the large terms while the per-node work stays in the
// float32 pipe (GB300's float64 rate is 1/64 of float32); the block's sums become float64 once.
template <typename R>
__global__ void __launch_bounds__(256) diag_kernel(const __grid_constant__ DiagArgs a) {
    const R *prho = static_cast<const R *>(a.rho), *pux = static_cast<const R *>(a.ux);
    const R *puy = static_cast<const R *>(a.uy), *pT = static_cast<const R *>(a.T);
    const R *prx = static_cast<const R *>(a.rx), *pry = static_cast<const R *>(a.ry);
    if constexpr (sizeof(R) == 8) {
        __shared__ double red[5][256];
        double s0 = 0, s1 = 0, s2 = 0, s3 = 0, mx = 0;
        const long long n = (long long)a.nx * a.ny;
        for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < n;
             g += (long long)gridDim.x * blockDim.x) {
            const long long y = g / a.nx, x = g - y * a.nx;
            const long long o = y * a.ld + x;
            const double rho = prho[o], ux = pux[o], uy = puy[o], T = pT[o];
            const double rx = prx[o], ry = pry[o];
            const double u2 = ux * ux + uy * uy;
            s0 += rho;
            s1 += rho * ux;
            s2 += rho * uy;
            s3 += rho * T - 1.125 * rho * rho + 0.5 * a.K * (rx * rx + ry * ry) + 0.5 * rho * u2;
            mx = fmax(mx, u2);
        }
        const int t = threadIdx.x;
        red[0][t] = s0; red[1][t] = s1; red[2][t] = s2; red[3][t] = s3; red[4][t] = mx;
        __syncthreads();
        for (int w = blockDim.x / 2; w > 0; w >>= 1) {
            if (t < w) {
                red[0][t] += red[0][t + w];
                red[1][t] += red[1][t + w];
                red[2][t] += red[2][t + w];
                red[3][t] += red[3][t + w];
                red[4][t] = fmax(red[4][t], red[4][t + w]);
            }
            __syncthreads();
        }
        if (t == 0)
            for (int k = 0; k < 5; ++k) a.partial[blockIdx.x * 5 + k] = red[k][0];
    } else {
        // rows of the block (no 64-bit index division per node)
        FPair S[5];  // mass, x and y momentum, e_T, max |u|^2
        const float hK = (float)(0.5 * a.K);
        for (int y = blockIdx.x; y < a.ny; y += gridDim.x) {
            const long long ro = (long long)y * a.ld;
            for (int x = threadIdx.x; x < a.nx; x += blockDim.x) {
                const long long o = ro + x;
                diag_accumulate(S, prho[o], pux[o], puy[o], pT[o], prx[o], pry[o], hK);
            }
        }
        __shared__ float wpart[32][5][2];
        diag_warp_reduce(S, wpart);
        __syncthreads();
        diag_block_write(wpart, a.partial + blockIdx.x * 5);
    }
}

// Twiddle table in the per-pass layout of fft_reg.cuh: entry idx = exp(-2 pi i a / n) with
// a = twiddle_exponent(n, idx), evaluated in float64 with sincospi (exact argument scaling),
// rounded once for the float32 table.
__global__ void twiddle_kernel(double2 *tw64, float2 *tw32, int n) {
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += gridDim.x * blockDim.x) {
        const int a = reg::twiddle_exponent(n, idx);
        double s = 0.0, c = 1.0;
        if (a > 0) sincospi(-2.0 * (double)a / (double)n, &s, &c);
        tw64[idx] = make_double2(c, s);
        tw32[idx] = make_float2((float)c, (float)s);
    }
}

// out[y][x] = src[y ld + x] as float64
template <typename R>
__global__ void field_out_kernel(const R *src, int ld, double *out, int nx, int ny) {
    const long long n = (long long)nx * ny;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < n;
         g += (long long)gridDim.x * blockDim.x) {
        const long long y = g / nx, x = g - y * nx;
        out[g] = (double)src[y * ld + x];
    }
}

// Generic spectral x-derivative (or, order 2, the real multiplier of table k2: a second
// derivative or the solution filter) of up to 4 fields (paired into complex lines), `rows` rows
// per CTA, G threads per line (fft_reg.cuh); row y of every field at + y * ld. A field may be
// transformed in place (out = in): every thread reads its points before any is written back.
template <typename R, int LOG2N>
__global__ void __launch_bounds__(MaxThreads<R>::value) row_deriv_kernel(const __grid_constant__ RowDerivArgs<R> a) {
    using F = reg::LineFFT<R, LOG2N>;
    using CT = typename F::CT;
    constexpr int G = F::G, E = F::E;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    CT *sb = reinterpret_cast<CT *>(smem_raw);
    const int NR = a.rows;
    const int slot = threadIdx.x / G, t = threadIdx.x % G;
    const int p = slot / NR, r = slot % NR;
    const size_t row = (size_t)(blockIdx.x * NR + r) * a.ld;
    const int ka = 2 * p, kb = 2 * p + 1;
    CT v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const size_t g = row + t + G * e;
        v[e] = reg::mk<R>(a.in[ka][g], kb < a.nin ? a.in[kb][g] : R(0));
    }
    CT *buf = sb + (size_t)slot * F::STRIDE;
    F::template forward<reg::SyncCta>(v, buf, t, a.ax.tw);
    F::multiply(v, t, a.order == 2 ? 2 : 1, R(1), a.ax.k1, a.ax.k2);
    F::template inverse<reg::SyncCta>(v, buf, t, a.ax.tw);
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const size_t g = row + t + G * e;
        if (a.acc) {  // each position is read and written by this thread only, so in may alias out
            a.out[ka][g] = a.in[ka][g] + v[e].x;
            if (kb < a.nin) a.out[kb][g] = a.in[kb][g] + v[e].y;
        } else {
            a.out[ka][g] = v[e].x;
            if (kb < a.nin) a.out[kb][g] = v[e].y;
        }
    }
}

template <typename R, int LOG2N> static cudaError_t launch_row_deriv_n(const RowDerivArgs<R> &a, size_t smem,
                                                                       cudaStream_t s) {
    using F = reg::LineFFT<R, LOG2N>;
    if (smem < (size_t)((a.nin + 1) / 2) * a.rows * F::STRIDE * sizeof(typename F::CT)) return cudaErrorInvalidValue;
    cudaError_t e = allow_smem(row_deriv_kernel<R, LOG2N>);
    if (e != cudaSuccess) return e;
    row_deriv_kernel<R, LOG2N><<<a.ny / a.rows, ((a.nin + 1) / 2) * a.rows * F::G, smem, s>>>(a);
    return cudaGetLastError();
}

static inline int grid_for(long long n) {
    long long b = (n + 255) / 256;
    return (int)(b < 4096 ? (b > 0 ? b : 1) : 4096);
}

cudaError_t launch_rho64(const float *f, double *r64, int nx, int ny, cudaStream_t s) {
    rho64_kernel<<<grid_for((long long)nx * ny), 256, 0, s>>>(f, r64, nx, ny);
    return cudaGetLastError();
}

// Validity of initial fields (0 < rho < 3, T > 0 and finite, u finite): the lowest index of a
// node that fails, by atomicMin into *bad (left untouched when every node passes).
__global__ void check_init_kernel(const double *rho, const double *ux, const double *uy, const double *T,
                                  long long n, unsigned long long *bad) {
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < n;
         g += (long long)gridDim.x * blockDim.x) {
        const double r = rho[g], t = T[g];
        if (!(r > 0.0 && r < 3.0) || !(t > 0.0) || !isfinite(t) || !isfinite(ux[g]) || !isfinite(uy[g]))
            atomicMin(bad, (unsigned long long)g);
    }
}

cudaError_t launch_check_init(const double *rho, const double *ux, const double *uy, const double *T, long long n,
                              unsigned long long *bad, cudaStream_t s) {
    check_init_kernel<<<grid_for(n), 256, 0, s>>>(rho, ux, uy, T, n, bad);
    return cudaGetLastError();
}

template <typename F> cudaError_t launch_init(const InitArgs &a, cudaStream_t s) {
    init_feq_kernel<F><<<grid_for((long long)a.nx * a.ny), 256, 0, s>>>(a);
    return cudaGetLastError();
}
template <typename F> cudaError_t launch_moments(const MomArgs &a, cudaStream_t s) {
    moments_kernel<F><<<grid_for((long long)a.nx * a.ny), 256, 0, s>>>(a);
    return cudaGetLastError();
}
template <typename R> cudaError_t launch_diag(const DiagArgs &a, int blocks, cudaStream_t s) {
    diag_kernel<R><<<blocks, 256, 0, s>>>(a);
    return cudaGetLastError();
}
cudaError_t launch_twiddles(double2 *tw64, float2 *tw32, int n, cudaStream_t s) {
    twiddle_kernel<<<(n + 255) / 256, 256, 0, s>>>(tw64, tw32, n);
    return cudaGetLastError();
}
template <typename R>
cudaError_t launch_field_out(const R *src, int ld, double *out, int nx, int ny, cudaStream_t s) {
    field_out_kernel<R><<<grid_for((long long)nx * ny), 256, 0, s>>>(src, ld, out, nx, ny);
    return cudaGetLastError();
}
template <typename R>
cudaError_t launch_row_deriv(const RowDerivArgs<R> &a, size_t smem, cudaStream_t s) {
    switch (a.ax.log2n) {
#define LBM_CASE(L2) \
    case L2: return launch_row_deriv_n<R, L2>(a, smem, s);
        LBM_FOR_LOG2N(LBM_CASE)
#undef LBM_CASE
        default: return cudaErrorInvalidValue;
    }
}

template cudaError_t launch_init<double>(const InitArgs &, cudaStream_t);
template cudaError_t launch_init<float>(const InitArgs &, cudaStream_t);
template cudaError_t launch_moments<double>(const MomArgs &, cudaStream_t);
template cudaError_t launch_moments<float>(const MomArgs &, cudaStream_t);
template cudaError_t launch_field_out<double>(const double *, int, double *, int, int, cudaStream_t);
template cudaError_t launch_field_out<float>(const float *, int, double *, int, int, cudaStream_t);
template cudaError_t launch_row_deriv<double>(const RowDerivArgs<double> &, size_t, cudaStream_t);
template cudaError_t launch_row_deriv<float>(const RowDerivArgs<float> &, size_t, cudaStream_t);
template cudaError_t launch_diag<double>(const DiagArgs &, int, cudaStream_t);
template cudaError_t launch_diag<float>(const DiagArgs &, int, cudaStream_t);

}  // namespace lbm
