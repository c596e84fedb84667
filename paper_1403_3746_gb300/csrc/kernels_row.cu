// Row passes: spectral x-derivatives of whole rows fused with the node-local physics.
//
// A CTA owns `rows` consecutive rows (rows * nx nodes); each row segment is read and
// written with coalesced accesses, and threads map to consecutive x in the node loops.
#include "lbm_internal.cuh"

namespace lbm {

// ---------------------------------------------------------------------------------------
// Macroscopic chain, row pass (Sec. 2.2, the coefficients after Eq. (2)).
// In: rho, u, T and their y-derivatives from the column pass.
// Lines (kind-major, stride 2 nx):  A = rho + i T,  B = u_x + i d_y u_y,  C = u_y,
// A2 = d_xx A, B2 = d_xx B. After the inverse transforms:
//   A -> (d_x rho, d_x T),  A2 -> d_xx rho,  B -> (d_x u_x, d_x d_y u_y),
//   B2 -> d_xx u_x,  C -> d_x u_y.
// Then per node: P^w, Lambda, S, Q, div u, the partial numerator of C; and a second
// transform pair gives d_x Q_x, d_x S_xx (line A) and d_x S_xy (line B).
// ---------------------------------------------------------------------------------------
template <typename M>
__global__ void __launch_bounds__(256) macro_row_kernel(const __grid_constant__ MacroArgs<M> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    M *s = reinterpret_cast<M *>(smem_raw);
    const int nx = a.nx, R = a.rows, log2n = a.ax.log2n;
    const int L2 = 2 * nx;
    const int nodes = R * nx;
    const size_t g0 = (size_t)blockIdx.x * nodes;
    M *sA = s, *sB = s + R * L2, *sC = s + 2 * R * L2, *sA2 = s + 3 * R * L2, *sB2 = s + 4 * R * L2;

    for (int idx = threadIdx.x; idx < nodes; idx += blockDim.x) {
        const int r = idx >> log2n, x = idx & (nx - 1);
        const size_t g = g0 + idx;
        const int o = r * L2 + x;
        sA[o] = a.rho[g];
        sA[o + nx] = a.T[g];
        sB[o] = a.ux[g];
        sB[o + nx] = a.uyy[g];
        sC[o] = a.uy[g];
        sC[o + nx] = M(0);
    }
    __syncthreads();
    const LineSet<M> ABC{s, 3 * R, L2, 1, nx};
    fft_forward<M, false>(ABC, log2n, a.ax.tw);
    spec_mul<M, false>(LineSet<M>{sA2, R, L2, 1, nx}, LineSet<M>{sA, R, L2, 1, nx}, log2n, 2, M(1), a.ax.k1,
                       a.ax.k2);
    spec_mul<M, false>(LineSet<M>{sB2, R, L2, 1, nx}, LineSet<M>{sB, R, L2, 1, nx}, log2n, 2, M(1), a.ax.k1,
                       a.ax.k2);
    __syncthreads();
    spec_mul<M, false>(ABC, ABC, log2n, 1, M(1), a.ax.k1, a.ax.k2);
    __syncthreads();
    fft_inverse<M, false>(LineSet<M>{s, 5 * R, L2, 1, nx}, log2n, a.ax.tw);

    const double K = a.K, H = a.H, q = a.q, zeta = a.zeta;
    for (int idx = threadIdx.x; idx < nodes; idx += blockDim.x) {
        const int r = idx >> log2n, x = idx & (nx - 1);
        const size_t g = g0 + idx;
        const int o = r * L2 + x;
        const double rx = sA[o], Tx = sA[o + nx], rxx = sA2[o];
        const double dux_dx = sB[o], dxduyy = sB[o + nx], dxxux = sB2[o];
        const double duy_dx = sC[o];
        const double rho = a.rho[g], T = a.T[g];
        const double ry = a.ry[g], ryy = a.ryy[g], dux_dy = a.uxy[g], duy_dy = a.uyy[g], Ty = a.Ty[g];

        const double lap = rxx + ryy;
        const double divu = dux_dx + duy_dy;
        const double ddivu_x = dxxux + dxduyy;  // d_x (div u)
        // van der Waals EOS (Sec. 2.2)
        const double rT = rho * T;
        const double Pw = 3.0 * rT / (3.0 - rho) - 1.125 * rho * rho;
        // Lambda with M = K + H T and grad(M/T) = -K grad T / T^2
        const double Mc = K + H * T;
        const double iT2 = 1.0 / (T * T);
        const double gx = -K * Tx * iT2, gy = -K * Ty * iT2;
        const double grr = rx * rx + ry * ry;
        const double iso = Mc * (rho * lap + 0.5 * grr) + rT * (rx * gx + ry * gy);
        const double Lxx = Mc * rx * rx - iso, Lxy = Mc * rx * ry, Lyy = Mc * ry * ry - iso;
        const double Pn = Pw - rT - zeta * divu;
        const double Sxx = Pn + Lxx, Sxy = Lxy, Syy = Pn + Lyy;
        const double qrT = q * rT;
        const double Qx = qrT * Tx, Qy = qrT * Ty;
        // numerator of C without the -K rho d_y rho d_y(div u) term (needs the flux pass)
        const double L_gradu = Lxx * dux_dx + Lxy * (duy_dx + dux_dy) + Lyy * duy_dy;
        const double r_gradu_r = rx * (dux_dx * rx + duy_dx * ry) + ry * (dux_dy * rx + duy_dy * ry);
        const double Cnum = (Pw - rT) * divu + L_gradu - zeta * divu * divu + 1.125 * rho * rho * divu +
                            K * (-0.5 * grr * divu - rho * rx * ddivu_x - r_gradu_r);
        a.Qy[g] = (M)Qy;
        a.Sxy[g] = (M)Sxy;
        a.Syy[g] = (M)Syy;
        a.divu[g] = (M)divu;
        a.Cnum[g] = (M)Cnum;
        sA[o] = (M)Qx;
        sA[o + nx] = (M)Sxx;
        sB[o] = (M)Sxy;
        sB[o + nx] = M(0);
    }
    __syncthreads();
    const LineSet<M> AB{s, 2 * R, L2, 1, nx};
    fft_forward<M, false>(AB, log2n, a.ax.tw);
    spec_mul<M, false>(AB, AB, log2n, 1, M(1), a.ax.k1, a.ax.k2);
    __syncthreads();
    fft_inverse<M, false>(AB, log2n, a.ax.tw);
    for (int idx = threadIdx.x; idx < nodes; idx += blockDim.x) {
        const int r = idx >> log2n, x = idx & (nx - 1);
        const size_t g = g0 + idx;
        const int o = r * L2 + x;
        a.dQx[g] = sA[o];
        a.dSxx[g] = sA[o + nx];
        a.dSxy[g] = sB[o];
    }
}

// ---------------------------------------------------------------------------------------
// Fused update row pass: Eq. (1) right-hand side and one Runge-Kutta stage (Sec. 2.3).
//   R_i = -(v_ix d_x f_i + v_iy d_y f_i) - (f_i - f_i^eq)/tau + I_i
//   f_out = f_base + h R_i        (h = dt/2, f_base = f^n for stage 1; h = dt for stage 2)
// f^eq = M^{-1} m^eq(rho, u, T): the 16 targets are the moments of a Maxwellian with b
// degrees of freedom (Sec. 2.1, 2.2). I_i from Eq. (2) with B = div S/(rho T),
// C_q = div Q/(rho T^2), A = -2 (C + C_q) T. The moments of f_out are written for the
// next stage.
// ---------------------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ void equilibrium_moments(R rho, R ux, R uy, R T, R b, R m[16]) {
    const R u2 = ux * ux + uy * uy;
    const R e = (b + R(2)) * T + u2;
    const R gq = (b + R(4)) * T + u2;
    m[0] = rho;
    m[1] = rho * ux;
    m[2] = rho * uy;
    m[3] = rho * (b * T + u2);
    m[4] = rho * (T + ux * ux);
    m[5] = rho * ux * uy;
    m[6] = rho * (T + uy * uy);
    m[7] = rho * ux * e;
    m[8] = rho * uy * e;
    m[9] = rho * ux * (R(3) * T + ux * ux);
    m[10] = rho * uy * (T + ux * ux);
    m[11] = rho * ux * (T + uy * uy);
    m[12] = rho * uy * (R(3) * T + uy * uy);
    m[13] = rho * (T * e + gq * ux * ux);
    m[14] = rho * gq * ux * uy;
    m[15] = rho * (T * e + gq * uy * uy);
}

template <typename F, typename M>
__global__ void __launch_bounds__(256) update_row_kernel(const __grid_constant__ UpdateArgs<F, M> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    F *s = reinterpret_cast<F *>(smem_raw);
    const int nx = a.nx, R = a.rows, log2n = a.ax.log2n;
    const int L2 = 2 * nx;
    const int nodes = R * nx;
    const size_t plane = (size_t)nx * a.ny;
    const size_t g0 = (size_t)blockIdx.x * nodes;
    const bool adv = !(a.flags & LBM_FLAG_NO_ADVECTION);
    const bool col = !(a.flags & LBM_FLAG_NO_COLLISION);
    const bool frc = !(a.flags & LBM_FLAG_NO_FORCE);

    if (adv) {
        for (int idx = threadIdx.x; idx < 12 * nodes; idx += blockDim.x) {
            const int k = idx / nodes, rem = idx - k * nodes;
            const int r = rem >> log2n, x = rem & (nx - 1);
            s[((k >> 1) * R + r) * L2 + (k & 1) * nx + x] = a.fs[xfield(k) * plane + g0 + rem];
        }
        __syncthreads();
        const LineSet<F> X{s, 6 * R, L2, 1, nx};
        fft_forward<F, false>(X, log2n, a.ax.tw);
        spec_mul<F, false>(X, X, log2n, 1, F(1), a.ax.k1, a.ax.k2);
        __syncthreads();
        fft_inverse<F, false>(X, log2n, a.ax.tw);
    }

    const double b = a.b, K = a.K, tau_inv = a.tau_inv, h = a.h;
    for (int idx = threadIdx.x; idx < nodes; idx += blockDim.x) {
        const int r = idx >> log2n, x = idx & (nx - 1);
        const size_t g = g0 + idx;
        const double rho = a.rho[g], ux = a.ux[g], uy = a.uy[g], T = a.T[g];
        double Bx = 0, By = 0, CC = 0, A = 0;
        if (frc) {
            const double rT = rho * T;
            const double irT = 1.0 / rT;
            Bx = (a.dSxx[g] + a.dSxyy[g]) * irT;
            By = (a.dSxy[g] + a.dSyy[g]) * irT;
            const double C = (a.Cnum[g] - K * rho * a.ry[g] * a.ddivuy[g]) * (0.5 * irT / T);
            const double Cq = (a.dQx[g] + a.dQy[g]) * (irT / T);
            CC = C + Cq;
            A = -2.0 * CC * T;
        }
        double m[16];
        equilibrium_moments<double>(rho, ux, uy, T, b, m);
        double mr = 0, mjx = 0, mjy = 0, mE = 0;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            double fe = 0;
#pragma unroll
            for (int j = 0; j < 16; ++j) fe += (double)a.minv[i * 16 + j] * m[j];
            const double fsi = a.fs[i * plane + g];
            double Ri = 0;
            if (adv) {
                double ad = 0;
                const int xs = xslot(i), ys = yslot(i);
                if (xs >= 0) ad += vel_x(i) * (double)s[((xs >> 1) * R + r) * L2 + (xs & 1) * nx + x];
                if (ys >= 0) ad += (double)a.Ay[ys * plane + g];
                Ri -= ad;
            }
            if (col) Ri -= (fsi - fe) * tau_inv;
            if (frc) {
                const double cx = vel_x(i) - ux, cy = vel_y(i) - uy;
                Ri -= (A + Bx * cx + By * cy + CC * (cx * cx + cy * cy)) * fe;
            }
            const F fo = (F)((double)a.fbase[i * plane + g] + h * Ri);
            a.fout[i * plane + g] = fo;
            const double fd = (double)fo;
            mr += fd;
            mjx += vel_x(i) * fd;
            mjy += vel_y(i) * fd;
            mE += (vel_sq(i) + (i < 4 ? a.eta2 : 0.0)) * fd;
        }
        const double irho = 1.0 / mr;
        const double nux = mjx * irho, nuy = mjy * irho;
        a.rho[g] = (M)mr;
        a.ux[g] = (M)nux;
        a.uy[g] = (M)nuy;
        a.T[g] = (M)((mE * irho - (nux * nux + nuy * nuy)) / b);
    }
}

template <typename F, typename M>
cudaError_t launch_update(const UpdateArgs<F, M> &a, int threads, size_t smem, cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(update_row_kernel<F, M>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    update_row_kernel<F, M><<<a.ny / a.rows, threads, smem, s>>>(a);
    return cudaGetLastError();
}

template <typename M>
cudaError_t launch_macro(const MacroArgs<M> &a, int threads, size_t smem, cudaStream_t s) {
    cudaError_t e =
        cudaFuncSetAttribute(macro_row_kernel<M>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    macro_row_kernel<M><<<a.ny / a.rows, threads, smem, s>>>(a);
    return cudaGetLastError();
}

template cudaError_t launch_update<double, double>(const UpdateArgs<double, double> &, int, size_t, cudaStream_t);
template cudaError_t launch_update<float, double>(const UpdateArgs<float, double> &, int, size_t, cudaStream_t);
template cudaError_t launch_macro<double>(const MacroArgs<double> &, int, size_t, cudaStream_t);

}  // namespace lbm
