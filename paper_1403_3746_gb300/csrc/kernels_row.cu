// Row passes: spectral x-derivatives of whole rows fused with the node-local physics.
//
// A CTA owns `rows` consecutive rows (rows * nx nodes); each row segment is read and
// written with coalesced accesses, and threads map to consecutive x in the node loops.
// Template parameter R is the arithmetic and storage type of the path (double for
// LBM_FP64, float for LBM_MIXED).
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
template <typename R>
__global__ void __launch_bounds__(256) macro_row_kernel(const __grid_constant__ MacroArgs<R> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R *s = reinterpret_cast<R *>(smem_raw);
    const int nx = a.nx, NR = a.rows, log2n = a.ax.log2n;
    const int L2 = 2 * nx;
    const int nodes = NR * nx;
    const size_t g0 = (size_t)blockIdx.x * nodes;
    R *sA = s, *sB = s + NR * L2, *sC = s + 2 * NR * L2, *sA2 = s + 3 * NR * L2, *sB2 = s + 4 * NR * L2;

    for (int idx = threadIdx.x; idx < nodes; idx += blockDim.x) {
        const int r = idx >> log2n, x = idx & (nx - 1);
        const size_t g = g0 + idx;
        const int o = r * L2 + x;
        sA[o] = a.rho[g];
        sA[o + nx] = a.T[g];
        sB[o] = a.ux[g];
        sB[o + nx] = a.uyy[g];
        sC[o] = a.uy[g];
        sC[o + nx] = R(0);
    }
    __syncthreads();
    const LineSet<R> ABC{s, 3 * NR, L2, 1, nx};
    fft_forward<R, false>(ABC, log2n, a.ax.tw);
    spec_mul<R, false>(LineSet<R>{sA2, NR, L2, 1, nx}, LineSet<R>{sA, NR, L2, 1, nx}, log2n, 2, R(1), a.ax.k1,
                       a.ax.k2);
    spec_mul<R, false>(LineSet<R>{sB2, NR, L2, 1, nx}, LineSet<R>{sB, NR, L2, 1, nx}, log2n, 2, R(1), a.ax.k1,
                       a.ax.k2);
    __syncthreads();
    spec_mul<R, false>(ABC, ABC, log2n, 1, R(1), a.ax.k1, a.ax.k2);
    __syncthreads();
    fft_inverse<R, false>(LineSet<R>{s, 5 * NR, L2, 1, nx}, log2n, a.ax.tw);

    const R K = a.K, H = a.H, q = a.q, zeta = a.zeta;
    for (int idx = threadIdx.x; idx < nodes; idx += blockDim.x) {
        const int r = idx >> log2n, x = idx & (nx - 1);
        const size_t g = g0 + idx;
        const int o = r * L2 + x;
        const R rx = sA[o], Tx = sA[o + nx], rxx = sA2[o];
        const R dux_dx = sB[o], dxduyy = sB[o + nx], dxxux = sB2[o];
        const R duy_dx = sC[o];
        const R rho = a.rho[g], T = a.T[g];
        const R ry = a.ry[g], ryy = a.ryy[g], dux_dy = a.uxy[g], duy_dy = a.uyy[g], Ty = a.Ty[g];

        const R lap = rxx + ryy;
        const R divu = dux_dx + duy_dy;
        const R ddivu_x = dxxux + dxduyy;  // d_x (div u)
        // van der Waals EOS (Sec. 2.2)
        const R rT = rho * T;
        const R Pw = R(3) * rT / (R(3) - rho) - R(1.125) * rho * rho;
        // Lambda with M = K + H T and grad(M/T) = -K grad T / T^2
        const R Mc = K + H * T;
        const R iT2 = R(1) / (T * T);
        const R gx = -K * Tx * iT2, gy = -K * Ty * iT2;
        const R grr = rx * rx + ry * ry;
        const R iso = Mc * (rho * lap + R(0.5) * grr) + rT * (rx * gx + ry * gy);
        const R Lxx = Mc * rx * rx - iso, Lxy = Mc * rx * ry, Lyy = Mc * ry * ry - iso;
        const R Pn = Pw - rT - zeta * divu;
        const R Sxx = Pn + Lxx, Sxy = Lxy, Syy = Pn + Lyy;
        const R qrT = q * rT;
        const R Qx = qrT * Tx, Qy = qrT * Ty;
        // numerator of C without the -K rho d_y rho d_y(div u) term (needs the flux pass)
        const R L_gradu = Lxx * dux_dx + Lxy * (duy_dx + dux_dy) + Lyy * duy_dy;
        const R r_gradu_r = rx * (dux_dx * rx + duy_dx * ry) + ry * (dux_dy * rx + duy_dy * ry);
        const R Cnum = (Pw - rT) * divu + L_gradu - zeta * divu * divu + R(1.125) * rho * rho * divu +
                       K * (-R(0.5) * grr * divu - rho * rx * ddivu_x - r_gradu_r);
        a.Qy[g] = Qy;
        a.Sxy[g] = Sxy;
        a.Syy[g] = Syy;
        a.divu[g] = divu;
        a.Cnum[g] = Cnum;
        sA[o] = Qx;
        sA[o + nx] = Sxx;
        sB[o] = Sxy;
        sB[o + nx] = R(0);
    }
    __syncthreads();
    const LineSet<R> AB{s, 2 * NR, L2, 1, nx};
    fft_forward<R, false>(AB, log2n, a.ax.tw);
    spec_mul<R, false>(AB, AB, log2n, 1, R(1), a.ax.k1, a.ax.k2);
    __syncthreads();
    fft_inverse<R, false>(AB, log2n, a.ax.tw);
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
// Moment sums of the new f (Sec. 2.1): rho = sum f, j = sum f v, E = sum f psi.
// float64 path: plain sums. float32 path: each sum is accumulated with error-free
// transformations (Knuth's TwoSum and the FMA-based TwoProduct, as in the compensated
// dot product "Dot2" of Ogita, Rump and Oishi, SIAM J. Sci. Comput. 26 (2005)), so the
// sums of the stored float32 values are as accurate as in twice the working precision;
// the irrational weights sqrt2 and 3/sqrt2 enter as float32 pairs (hi + lo).
// ---------------------------------------------------------------------------------------
template <typename R> struct MomentSums;

template <> struct MomentSums<double> {
    double r = 0, jx = 0, jy = 0, E = 0;
    __device__ __forceinline__ void add(int i, double f, double psi_hi, double) {
        r += f;
        if (vel_x(i) != 0.0) jx += vel_x(i) * f;
        if (vel_y(i) != 0.0) jy += vel_y(i) * f;
        E += psi_hi * f;
    }
    __device__ __forceinline__ void finish(double b, double &rho, double &ux, double &uy, double &T) const {
        rho = r;
        const double ir = 1.0 / r;
        ux = jx * ir;
        uy = jy * ir;
        T = (E * ir - (ux * ux + uy * uy)) / b;
    }
};

__device__ __forceinline__ void two_sum_acc(float &s, float &c, float x) {
    const float t = s + x;
    const float bp = t - s;
    c += (s - (t - bp)) + (x - bp);
    s = t;
}
__device__ __forceinline__ void dot2_acc(float &s, float &c, float f, float wh, float wl) {
    const float p = f * wh;
    const float e = fmaf(f, wh, -p);  // exact: f*wh = p + e
    two_sum_acc(s, c, p);
    c += fmaf(f, wl, e);
}

template <> struct MomentSums<float> {
    float rs = 0, rc = 0, xs = 0, xc = 0, ys = 0, yc = 0, es = 0, ec = 0;
    __device__ __forceinline__ void add(int i, float f, float psi_hi, float psi_lo) {
        two_sum_acc(rs, rc, f);
        if (vel_x(i) != 0.0) {
            const float wh = (float)vel_x(i), wl = (float)(vel_x(i) - (double)(float)vel_x(i));
            dot2_acc(xs, xc, f, wh, wl);
        }
        if (vel_y(i) != 0.0) {
            const float wh = (float)vel_y(i), wl = (float)(vel_y(i) - (double)(float)vel_y(i));
            dot2_acc(ys, yc, f, wh, wl);
        }
        dot2_acc(es, ec, f, psi_hi, psi_lo);
    }
    __device__ __forceinline__ void finish(float b, float &rho, float &ux, float &uy, float &T) const {
        rho = rs + rc;
        const float jx = xs + xc, jy = ys + yc, E = es + ec;
        ux = jx / rho;
        uy = jy / rho;
        T = (E / rho - (ux * ux + uy * uy)) / b;
    }
};

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

template <typename R, bool MOMENT_SPACE>
__global__ void __launch_bounds__(256) update_row_kernel(const __grid_constant__ UpdateArgs<R> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R *s = reinterpret_cast<R *>(smem_raw);
    const int nx = a.nx, NR = a.rows, log2n = a.ax.log2n;
    const int L2 = 2 * nx;
    const int nodes = NR * nx;
    const size_t plane = (size_t)nx * a.ny;
    const size_t g0 = (size_t)blockIdx.x * nodes;
    const bool adv = !(a.flags & LBM_FLAG_NO_ADVECTION);
    const bool col = !(a.flags & LBM_FLAG_NO_COLLISION);
    const bool frc = !(a.flags & LBM_FLAG_NO_FORCE);

    if (adv) {
        for (int idx = threadIdx.x; idx < 12 * nodes; idx += blockDim.x) {
            const int k = idx / nodes, rem = idx - k * nodes;
            const int r = rem >> log2n, x = rem & (nx - 1);
            s[((k >> 1) * NR + r) * L2 + (k & 1) * nx + x] = a.fs[xfield(k) * plane + g0 + rem];
        }
        __syncthreads();
        const LineSet<R> X{s, 6 * NR, L2, 1, nx};
        fft_forward<R, false>(X, log2n, a.ax.tw);
        spec_mul<R, false>(X, X, log2n, 1, R(1), a.ax.k1, a.ax.k2);
        __syncthreads();
        fft_inverse<R, false>(X, log2n, a.ax.tw);
    }

    const R b = a.b, K = a.K, tau_inv = a.tau_inv, h = a.h;
    for (int idx = threadIdx.x; idx < nodes; idx += blockDim.x) {
        const int r = idx >> log2n, x = idx & (nx - 1);
        const size_t g = g0 + idx;
        const R rho = a.rho[g], ux = a.ux[g], uy = a.uy[g], T = a.T[g];
        R Bx = 0, By = 0, CC = 0, A = 0;
        if (frc) {
            const R rT = rho * T;
            const R irT = R(1) / rT;
            Bx = (a.dSxx[g] + a.dSxyy[g]) * irT;
            By = (a.dSxy[g] + a.dSyy[g]) * irT;
            const R C = (a.Cnum[g] - K * rho * a.ry[g] * a.ddivuy[g]) * (R(0.5) * irT / T);
            const R Cq = (a.dQx[g] + a.dQy[g]) * (irT / T);
            CC = C + Cq;
            A = R(-2) * CC * T;
        }
        R m[16];
        equilibrium_moments<R>(rho, ux, uy, T, b, m);
        // neq_i = f_i^eq - f_i. float64: f^eq = M^-1 m^eq directly. float32: in moment space,
        // neq = M^-1 (m^eq - M f) over the 12 non-conserved moments only (the 4 conserved
        // ones agree exactly), so the rounding of M^-1 to float32 cannot bias mass, momentum
        // or energy: its error scales with the non-equilibrium part instead of with rho.
        R fsv[16], neq[16], fev[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) fsv[i] = a.fs[i * plane + g];
        if (MOMENT_SPACE) {
            R dm[12];
#pragma unroll
            for (int j = 0; j < 12; ++j) {
                R mf = 0;
#pragma unroll
                for (int i = 0; i < 16; ++i) mf += a.mrow[j * 16 + i] * fsv[i];
                dm[j] = m[4 + j] - mf;
            }
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                R ne = 0;
#pragma unroll
                for (int j = 0; j < 12; ++j) ne += a.minv[i * 16 + 4 + j] * dm[j];
                neq[i] = ne;
                fev[i] = fsv[i] + ne;
            }
        } else {
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                R fe = 0;
#pragma unroll
                for (int j = 0; j < 16; ++j) fe += a.minv[i * 16 + j] * m[j];
                fev[i] = fe;
                neq[i] = fe - fsv[i];
            }
        }
        MomentSums<R> acc;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const R fsi = fsv[i];
            const R fe = fev[i];
            R Ri = 0;
            if (adv) {
                R ad = 0;
                const int xs = xslot(i), ys = yslot(i);
                if (xs >= 0) ad += R(vel_x(i)) * s[((xs >> 1) * NR + r) * L2 + (xs & 1) * nx + x];
                if (ys >= 0) ad += a.Ay[ys * plane + g];
                Ri -= ad;
            }
            if (col) Ri += neq[i] * tau_inv;
            if (frc) {
                const R cx = R(vel_x(i)) - ux, cy = R(vel_y(i)) - uy;
                Ri -= (A + Bx * cx + By * cy + CC * (cx * cx + cy * cy)) * fe;
            }
            const R fo = a.fbase[i * plane + g] + h * Ri;
            a.fout[i * plane + g] = fo;
            acc.add(i, fo, a.psi_hi[i], a.psi_lo[i]);
        }
        R nr, nux, nuy, nT;
        acc.finish(b, nr, nux, nuy, nT);
        a.rho[g] = nr;
        a.ux[g] = nux;
        a.uy[g] = nuy;
        a.T[g] = nT;
    }
}

// float64 (the plain method): f^eq = M^-1 m^eq; float32: the moment-space collision.
template <typename R> cudaError_t launch_update(const UpdateArgs<R> &a, size_t smem, cudaStream_t s) {
    constexpr bool MS = sizeof(R) == 4;
    cudaError_t e = cudaFuncSetAttribute(update_row_kernel<R, MS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    update_row_kernel<R, MS><<<a.ny / a.rows, 256, smem, s>>>(a);
    return cudaGetLastError();
}

template <typename R> cudaError_t launch_macro(const MacroArgs<R> &a, size_t smem, cudaStream_t s) {
    cudaError_t e =
        cudaFuncSetAttribute(macro_row_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    macro_row_kernel<R><<<a.ny / a.rows, 256, smem, s>>>(a);
    return cudaGetLastError();
}

template cudaError_t launch_update<double>(const UpdateArgs<double> &, size_t, cudaStream_t);
template cudaError_t launch_update<float>(const UpdateArgs<float> &, size_t, cudaStream_t);
template cudaError_t launch_macro<double>(const MacroArgs<double> &, size_t, cudaStream_t);
template cudaError_t launch_macro<float>(const MacroArgs<float> &, size_t, cudaStream_t);

}  // namespace lbm
