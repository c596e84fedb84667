// Device bodies of the pass kernels (Sec. 2.2, 2.3), shared by the per-pass kernels
// (kernels_col.cu, kernels_row.cu) and the persistent batch kernel (kernels_batch.cu): the
// column tile of y-derivatives, the macroscopic row pass, the moment sums and the fused update
// row pass. Fields use the row-interleaved block layout of lbm_internal.cuh.
#pragma once
#include <type_traits>

#include "lbm_internal.cuh"

namespace lbm {
// One CTA's share of a column tile: CS = 1 (whole lines in one CTA) or the CTA of rank `rank`
// in a cluster of CS that splits every line of the tile (fft_reg.cuh); tile = the tile index.
// job: index into a.jobs; z: instance of a batch stacked along y (ny rows each). Threads beyond
// the tile's lines (a CTA larger than the tile needs, as in the batch kernel) only keep the
// barrier count. ACC: every job of the launch accumulates (out = in + result, the solution
// filter's correction), a separate instantiation so that the plain passes keep their registers.
template <typename R, int LOG2N, int CS, bool EXTRA = false, bool ACC = false>
__device__ __forceinline__ void col_tile(const ColArgs<R> &a, int jobi, int z, int tile, unsigned rank) {
    using F = reg::LineFFT<R, LOG2N, true, CS>;
    using CT = typename F::CT;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    CT *sbuf = reinterpret_cast<CT *>(smem_raw);
    const ColJob<R> &job = a.jobs[jobi];
    const int L = a.W >> 1;
    if (EXTRA && (int)threadIdx.x >= L * F::GL) {
        if constexpr (CS == 1) {
            F::template idle<reg::SyncCta>();
            F::template idle<reg::SyncCta>();
        } else {
            F::template idle_forward<reg::SyncCta>();
            F::template idle_inverse<reg::SyncCta>();
        }
        return;
    }
    const int l = threadIdx.x & (L - 1);
    const int t = (int)rank * F::GL + (threadIdx.x >> (a.log2W - 1));  // thread of the line, across the cluster
    const size_t rsi = (size_t)(job.ld_in >> 1), rso = (size_t)(job.ld_out >> 1);  // row strides, complex units
    const int x = tile * a.W + 2 * l;
    const CT *in = reinterpret_cast<const CT *>(job.in + z * a.ny * job.ld_in + x);
    CT *out = reinterpret_cast<CT *>(job.out + z * a.ny * job.ld_out + x);

    CT v[F::E];
#pragma unroll
    for (int e = 0; e < F::E; ++e) v[e] = __ldcg(in + (size_t)(t + F::G * e) * rsi);  // L2 only: single use
    CT *buf = sbuf + l * col_line_stride(LOG2N, sizeof(R), CS);
    F::template forward<reg::SyncCta>(v, buf, t, a.ay.tw);
    F::multiply(v, t, job.order, job.c, a.ay.k1, a.ay.k2);
    F::template inverse<reg::SyncCta>(v, buf, t, a.ay.tw);
    if constexpr (ACC) {  // out = in + result; each position is read and written by this thread only
#pragma unroll
        for (int e = 0; e < F::E; ++e) {
            const CT o = __ldcg(in + (size_t)(t + F::G * e) * rsi);
            out[(size_t)(t + F::G * e) * rso] = reg::mk<R>(o.x + v[e].x, o.y + v[e].y);
        }
    } else {
#pragma unroll
        for (int e = 0; e < F::E; ++e) out[(size_t)(t + F::G * e) * rso] = v[e];
    }
}


// Streaming global load: cached in L2 only, so single-use data does not evict the line
// transforms' tables (and register spills) from L1.
template <typename T> __device__ __forceinline__ T ldcg(const T *p) { return __ldcg(p); }

// a / b in the path's precision: float64 divides exactly; float32 uses the reciprocal unit and
// one multiply (__fdividef, within 2 ulp for the O(1) physical operands here) instead of the
// IEEE division sequence.
template <typename R> __device__ __forceinline__ R quot(R a, R b);
template <> __device__ __forceinline__ double quot<double>(double a, double b) { return a / b; }
template <> __device__ __forceinline__ float quot<float>(float a, float b) { return __fdividef(a, b); }

// compile-time loop: f(std::integral_constant<int, I>) for I = B .. E-1
template <int B, int E, class Fn> __device__ __forceinline__ void static_for(Fn &&f) {
    if constexpr (B < E) {
        f(std::integral_constant<int, B>{});
        static_for<B + 1, E>(f);
    }
}

// Prefetch a contiguous span into L2 (bulk, asynchronous; no data returned). The bulk form
// needs a 16-byte aligned address and size; other spans (tiny grids) are skipped.
__device__ __forceinline__ void prefetch_l2(const void *p, unsigned bytes) {
    if (((reinterpret_cast<uintptr_t>(p) | bytes) & 15) != 0 || bytes == 0) return;
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// ---------------------------------------------------------------------------------------
// Macroscopic chain, row pass (Sec. 2.2, the coefficients after Eq. (2)).
// In: rho, u, T and their y-derivatives from the column pass. Per row two lines:
// A = rho + i T -> (d_x rho, d_x T) and, from the same spectrum, d_xx rho;
// B = u_x + i u_y -> (d_x u_x, d_x u_y).
// Then per node: P^w, Lambda, S, Q, div u and the numerator of C without its
// d_x(div u) term. A second round of lines, (Q_x + i S_xx) and (S_xy + i div u), gives
// d_x Q_x, d_x S_xx, d_x S_xy and d_x(div u), which completes that numerator.
// ---------------------------------------------------------------------------------------
// SERIAL = false: the two lines of a row are transformed side by side by two groups of G
// threads (the B group waits while A computes d_xx rho). SERIAL = true (rows too long for two
// groups, float64 at nx = 4096): one group transforms A, then B, and K rho d_x rho waits in the
// global slot of d_x S_xy (free until round 2 writes it) instead of shared memory.
// Threads beyond the row lines' groups (a CTA larger than the pass needs, as in the batch
// kernel) only keep the barrier count. Inputs written by other passes are read L2-only.
// RHO64 (LBM_MIXED_RHO64): rho and its derivatives come from the float64 density chain
// (a.r64) and the node loop's rho-dependent terms (P^w, Lambda, S, Q, the C numerator) are
// evaluated in float64, then rounded to the path's type; d_y rho is also written to M_RY for the
// update pass. DIAG (float32): the node loop also accumulates the diagnostics of the stage's
// input state (the nodes' rho, u, T and the d_x rho, d_y rho it has at hand) and the CTA writes
// its five partial values to a.diag_partial, as the diagnostics kernel would.
template <typename R, int LOG2N, bool SERIAL, bool EXTRA = false, bool RHO64 = false, bool DIAG = false>
__device__ __forceinline__ void macro_rows(const MacroArgs<R> &a, int blk) {
    using F = reg::LineFFT<R, LOG2N, true>;
    using CT = typename F::CT;
    constexpr int NX = F::N, G = F::G, E = F::E, SM = F::STRIDE;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    CT *sb = reinterpret_cast<CT *>(smem_raw);
    const int NR = a.rows, nodes = NR * NX;
    // per row three line buffers: A1, A2 (line A) and B1 (line B). K rho d_x rho of node x waits
    // in A2[x].y between the rounds (d_xx T, the other half of A2, is not needed), unless SERIAL.
    // The partial numerator of C waits in its own global slot (M_CNUM) between the rounds.
    CT *lines = sb;  // [NR][3 SM]
    const int y0 = blk * NR;
    const int slot = threadIdx.x / G, t = threadIdx.x % G;
    const bool active = !EXTRA || slot < (SERIAL ? NR : 2 * NR);
    const int my_kind = SERIAL ? 0 : (active ? slot / NR : 1), r = SERIAL ? (active ? slot : 0) : slot % NR;
    R *mrow = a.m + (size_t)(y0 + r) * NF_M * NX;  // this line's row of the macroscopic block
    auto buf1 = [&](int kind) { return lines + (size_t)r * 3 * SM + (kind == 0 ? 0 : 2 * SM); };
    CT *O2 = lines + (size_t)r * 3 * SM + SM;  // line A's second buffer

    if (threadIdx.x < NR) {  // the node loop's inputs from the column pass start moving into L2
        prefetch_l2(a.m + ((size_t)(y0 + threadIdx.x) * NF_M + M_RY) * NX, 5 * NX * sizeof(R));
        if constexpr (RHO64) prefetch_l2(a.r64 + (size_t)(y0 + threadIdx.x) * NR64 * NX, NR64 * NX * sizeof(double));
    }

    // round 1: derivatives of the moments along x
    CT v[E];
    for (int kind = my_kind; kind <= (SERIAL ? 1 : my_kind); ++kind) {
        if (!active) {  // the barriers of the line groups (A then B in turn when SERIAL, else B)
            for (int k = 0; k < (SERIAL ? 2 : 1); ++k) {
                F::template idle<reg::SyncCta>();
                F::template idle<reg::SyncCta>();
                reg::cta_barrier();
                if (!SERIAL || k == 0) F::template idle<reg::SyncCta>();
                reg::cta_barrier();
            }
            break;
        }
        CT *O1 = buf1(kind);
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int x = t + G * e;
            v[e] = kind == 0 ? reg::mk<R>(__ldcg(mrow + M_RHO * NX + x), __ldcg(mrow + M_T * NX + x))
                             : reg::mk<R>(__ldcg(mrow + M_UX * NX + x), __ldcg(mrow + M_UY * NX + x));
        }
        F::template forward<reg::SyncCta>(v, O1, t, a.ax.tw);
        if (kind == 0) F::storeF(v, O2, t);  // keep the spectrum of A for d_xx rho (thread-private slots)
        F::multiply(v, t, 1, R(1), a.ax.k1, a.ax.k2);
        F::template inverse<reg::SyncCta>(v, O1, t, a.ax.tw);
        reg::cta_barrier();
#pragma unroll
        for (int e = 0; e < E; ++e) O1[t + G * e] = v[e];
        if (kind == 0) {
            F::loadF(v, O2, t);
            F::multiply(v, t, 2, R(1), a.ax.k1, a.ax.k2);
            F::template inverse<reg::SyncCta>(v, O2, t, a.ax.tw);
        } else if (!SERIAL) {
            F::template idle<reg::SyncCta>();
        }
        reg::cta_barrier();
        if (kind == 0) {
#pragma unroll
            for (int e = 0; e < E; ++e) O2[t + G * e] = v[e];
        }
    }
    __syncthreads();

    using D = std::conditional_t<RHO64, double, R>;  // type of the rho-dependent terms
    const D K = RHO64 ? (D)a.K64 : (D)a.K, H = RHO64 ? (D)a.H64 : (D)a.H, q = RHO64 ? (D)a.q64 : (D)a.q,
            zeta = RHO64 ? (D)a.zeta64 : (D)a.zeta;
    static_assert(!DIAG || (sizeof(R) == 4 && !RHO64 && !SERIAL && !EXTRA), "fused diagnostics: float32 pass only");
    FPair dS[DIAG ? 5 : 1];
    for (int idx = threadIdx.x; idx < nodes; idx += blockDim.x) {
        const int rr = idx / NX, x = idx % NX;
        R *mn = a.m + (size_t)(y0 + rr) * NF_M * NX + x;  // this node: field k at mn[k * NX]
        CT *A1 = lines + (size_t)rr * 3 * SM, *A2 = A1 + SM, *B1 = A1 + 2 * SM;
        const D Tx = A1[x].y;
        const D dux_dx = B1[x].x, duy_dx = B1[x].y;
        const D T = __ldcg(mn + M_T * NX);
        const D dux_dy = __ldcg(mn + M_UXY * NX), duy_dy = __ldcg(mn + M_UYY * NX);
        const D Ty = __ldcg(mn + M_TY * NX);
        D rho, rx, rxx, ry, ryy;
        if constexpr (RHO64) {
            const double *rn = a.r64 + (size_t)(y0 + rr) * NR64 * NX + x;
            rho = __ldcg(rn + R64_RHO * NX);
            rx = __ldcg(rn + R64_RX * NX);
            rxx = __ldcg(rn + R64_RXX * NX);
            ry = __ldcg(rn + R64_RY * NX);
            ryy = __ldcg(rn + R64_RYY * NX);
            mn[M_RY * NX] = (R)ry;  // read by the update pass's C term
        } else {
            rho = __ldcg(mn + M_RHO * NX);
            rx = A1[x].x;
            rxx = A2[x].x;
            ry = __ldcg(mn + M_RY * NX);
            ryy = __ldcg(mn + M_RYY * NX);
        }

        if constexpr (DIAG)
            diag_accumulate(dS, (float)rho, __ldcg(mn + M_UX * NX), __ldcg(mn + M_UY * NX), (float)T, (float)rx,
                            (float)ry, a.diag_hK);

        const D lap = rxx + ryy;
        const D divu = dux_dx + duy_dy;
        // van der Waals EOS (Sec. 2.2)
        const D rT = rho * T;
        const D Pw = quot(D(3) * rT, D(3) - rho) - D(1.125) * rho * rho;
        // Lambda with M = K + H T and grad(M/T) = -K grad T / T^2
        const D Mc = K + H * T;
        const D iT2 = quot(D(1), T * T);
        const D gx = -K * Tx * iT2, gy = -K * Ty * iT2;
        const D grr = rx * rx + ry * ry;
        const D iso = Mc * (rho * lap + D(0.5) * grr) + rT * (rx * gx + ry * gy);
        const D Lxx = Mc * rx * rx - iso, Lxy = Mc * rx * ry, Lyy = Mc * ry * ry - iso;
        const D Pn = Pw - rT - zeta * divu;
        const D Sxx = Pn + Lxx, Sxy = Lxy, Syy = Pn + Lyy;
        const D qrT = q * rT;
        const D Qx = qrT * Tx, Qy = qrT * Ty;
        // numerator of C without -K rho (d_x rho d_x(div u) + d_y rho d_y(div u)): the x term is
        // added after round 2 below, the y term by the update pass (after the flux pass)
        const D L_gradu = Lxx * dux_dx + Lxy * (duy_dx + dux_dy) + Lyy * duy_dy;
        const D r_gradu_r = rx * (dux_dx * rx + duy_dx * ry) + ry * (dux_dy * rx + duy_dy * ry);
        mn[M_CNUM * NX] = (R)((Pw - rT) * divu + L_gradu - zeta * divu * divu + D(1.125) * rho * rho * divu +
                              K * (-D(0.5) * grr * divu - r_gradu_r));
        if constexpr (SERIAL) mn[M_DSXY * NX] = (R)(K * rho * rx);
        else A2[x].y = (R)(K * rho * rx);  // this thread read A2[x].x above
        mn[M_QY * NX] = (R)Qy;
        mn[M_SXY * NX] = (R)Sxy;
        mn[M_SYY * NX] = (R)Syy;
        mn[M_DIVU * NX] = (R)divu;
        A1[x] = reg::mk<R>((R)Qx, (R)Sxx);  // round-2 lines, same node and thread as the reads above
        B1[x] = reg::mk<R>((R)Sxy, (R)divu);
    }
    if constexpr (DIAG) {
        __shared__ float dwarp[32][5][2];
        diag_warp_reduce(dS, dwarp);
        __syncthreads();
        diag_block_write(dwarp, a.diag_partial + (size_t)blk * 5);
    }
    __syncthreads();

    // round 2: d_x of (Q_x, S_xx) on line A and of (S_xy, div u) on line B
    for (int kind = my_kind; kind <= (SERIAL ? 1 : my_kind); ++kind) {
        if (!active) {
            for (int k = 0; k < (SERIAL ? 4 : 2); ++k) F::template idle<reg::SyncCta>();
            break;
        }
        CT *O1 = buf1(kind);
#pragma unroll
        for (int e = 0; e < E; ++e) v[e] = O1[t + G * e];
        F::template forward<reg::SyncCta>(v, O1, t, a.ax.tw);
        F::multiply(v, t, 1, R(1), a.ax.k1, a.ax.k2);
        F::template inverse<reg::SyncCta>(v, O1, t, a.ax.tw);
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int x = t + G * e;
            if (kind == 0) {
                mrow[M_DQX * NX + x] = v[e].x;
                mrow[M_DSXX * NX + x] = v[e].y;
            } else {
                // - K rho d_x rho d_x(div u); the partial value was written by this CTA's node loop
                const R k = SERIAL ? mrow[M_DSXY * NX + x] : O2[x].y;
                mrow[M_DSXY * NX + x] = v[e].x;
                mrow[M_CNUM * NX + x] -= k * v[e].y;
            }
        }
    }
}

// ---------------------------------------------------------------------------------------
// Moment sums of the new f (Sec. 2.1): rho = sum f, j = sum f v, E = sum f psi.
// float64 path: plain sums. float32 path: a fixed-quantum split makes the sums of the stored
// float32 values exact up to one final rounding (as accurate as float64 sums, then rounded).
// Each value is split as f = h 2^-16 + l: t = f + 192 rounds f to a multiple of 2^-16 (t lies in
// [128, 256), whose float32 spacing is 2^-16, for |f| < 64), the bit pattern of t minus that of
// 192 is the integer h exactly (float32 bit patterns are linear in the value within a binade),
// and l = f - (t - 192) is exact with |l| <= 2^-17. The integer parts are summed exactly in
// 32-bit integers with the weights 2 v_i and 2 psi_i of velocities 4..15 (integers for this
// velocity set), the small parts in float32 (rounding below 2^-36 of the sum), and the two are
// combined once. psi of velocities 0..3 (1 + eta0^2, a parameter) enters as a float pair.
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

// Knuth's TwoSum: a + b = s + e exactly (no fused operations).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bp = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
}

// speed group of velocity i: 0 (speed 1, carries eta), 1 (6), 2 (sqrt2 diagonals), 3 (3/sqrt2)
__host__ __device__ constexpr int speed_group(int i) { return i >> 2; }
// twice a velocity component and twice |v|^2, as integers (exact for this velocity set)
__host__ __device__ constexpr int twice(double x) { return (int)(2.0 * x); }
static_assert(2.0 * vel_x(12) == (double)twice(vel_x(12)) && 2.0 * vel_sq(12) == (double)twice(vel_sq(12)),
              "the integer moment weights need 2 v and 2 |v|^2 integral");

template <> struct MomentSums<float> {
    static constexpr float kMagic = 192.0f;  // 1.5 2^7: f + 192 in [128, 256) for |f| < 64
    static constexpr float kQ = 1.0f / 65536.0f;
    unsigned sA = 0u, sB = 0u, sC = 0u, sD = 0u;  // per speed group: sum of bits(t) (offset bits(192) per value)
    int jx2 = 0, jy2 = 0;                // 2 v-weighted integer parts (pair differences: no offset)
    float lr = 0.f, le = 0.f, lx = 0.f, ly = 0.f;  // small parts
    float psiA_hi = 0.f, psiA_lo = 0.f;  // psi of group 0 (1 + eta0^2) as a float pair

    static __device__ __forceinline__ unsigned bits(float x) { return __float_as_uint(x); }

    // Velocities i and i + 2 are opposite: their contributions enter as the integer pair sum
    // (to rho and E) and difference (to j, weight v_i), and the same for the small parts.
    template <int I> __device__ __forceinline__ void add_pair(float fi, float fk, float psi_hi, float psi_lo) {
        constexpr int g = speed_group(I);
        const float ti = __fadd_rn(fi, kMagic), tk = __fadd_rn(fk, kMagic);
        const float li = __fsub_rn(fi, __fsub_rn(ti, kMagic)), lk = __fsub_rn(fk, __fsub_rn(tk, kMagic));
        const unsigned bi = bits(ti), bk = bits(tk), sp = bi + bk;
        if constexpr (g == 0) sA += sp;
        else if constexpr (g == 1) sB += sp;
        else if constexpr (g == 2) sC += sp;
        else sD += sp;
        const int d = (int)(bi - bk);
        const float ls = __fadd_rn(li, lk), ld = __fsub_rn(li, lk);
        lr = __fadd_rn(lr, ls);
        le = fmaf(psi_hi, ls, le);
        if constexpr (g == 0) {
            psiA_hi = psi_hi;
            psiA_lo = psi_lo;
        }
        if constexpr (vel_x(I) != 0.0) {
            jx2 += twice(vel_x(I)) * d;
            lx = fmaf((float)vel_x(I), ld, lx);
        }
        if constexpr (vel_y(I) != 0.0) {
            jy2 += twice(vel_y(I)) * d;
            ly = fmaf((float)vel_y(I), ld, ly);
        }
    }

    __device__ __forceinline__ void finish(float b, float &rho, float &ux, float &uy, float &T) const {
        const unsigned off = 4u * bits(kMagic);  // four values per group
        const int SA = (int)(sA - off), SB = (int)(sB - off), SC = (int)(sC - off), SD = (int)(sD - off);
        rho = fmaf((float)(SA + SB + SC + SD), kQ, lr);  // integer sum below 2^24: exact as float
        // E: 2 psi = 72, 4, 9 for groups 1..3, exact in int32, converted as an exact float pair
        const int Ei = twice(vel_sq(4)) * SB + twice(vel_sq(8)) * SC + twice(vel_sq(12)) * SD;
        const float e1 = __int2float_rz(Ei);
        const float e2v = (float)(Ei - __float2int_rz(e1));
        const float fa = (float)SA;
        const float pa = fa * psiA_hi, ea = fmaf(fa, psiA_hi, -pa);
        float s, t;
        two_sum(0.5f * e1, pa, s, t);  // 0.5 e1: exact (a power-of-two scaling)
        const float corr = fmaf(fa, psiA_lo, t + 0.5f * e2v + ea);
        const float E = fmaf(s, kQ, fmaf(corr, kQ, le));
        // j: 2 v-weighted integer sums below 2^24 (exact as floats), scaled by 2^-17
        const float jx = fmaf((float)jx2, 0.5f * kQ, lx), jy = fmaf((float)jy2, 0.5f * kQ, ly);
        const float ir = __fdividef(1.0f, rho);
        ux = jx * ir;
        uy = jy * ir;
        T = __fdividef(E * ir - (ux * ux + uy * uy), b);
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

// The 12 non-conserved moments 4..15 of the moment matrix as monomials v_x^px v_y^py, times
// psi = |v|^2 + eta^2 for the psi rows: all known at compile time except the eta^2 part of
// psi, which only velocities 0..3 carry.
__host__ __device__ constexpr int mom_px(int j) {
    constexpr int p[12] = {2, 1, 0, 1, 0, 3, 2, 1, 0, 2, 1, 0};
    return p[j];
}
__host__ __device__ constexpr int mom_py(int j) {
    constexpr int p[12] = {0, 1, 2, 0, 1, 0, 1, 2, 3, 0, 1, 2};
    return p[j];
}
__host__ __device__ constexpr bool mom_psi(int j) { return j == 3 || j == 4 || j >= 9; }
__host__ __device__ constexpr double ipow(double x, int n) { return n == 0 ? 1.0 : x * ipow(x, n - 1); }
__host__ __device__ constexpr double mom_mono(int j, int i) {
    return ipow(vel_x(i), mom_px(j)) * ipow(vel_y(i), mom_py(j));
}
// moment-matrix entry (4 + j, i) without the eta^2 part, and the coefficient of eta^2
__host__ __device__ constexpr double mom_entry(int j, int i) {
    return mom_mono(j, i) * (mom_psi(j) ? vel_sq(i) : 1.0);
}
__host__ __device__ constexpr double mom_entry_eta(int j, int i) {
    return (mom_psi(j) && i < 4) ? mom_mono(j, i) : 0.0;
}
// Reflection symmetry: for an axis velocity the inverse-matrix entry of a moment that is odd
// in the velocity's zero component vanishes identically (for every eta0).
__host__ __device__ constexpr bool minv_zero(int i, int j) {
    return i < 8 && ((vel_y(i) == 0.0 && (mom_py(j) & 1)) || (vel_x(i) == 0.0 && (mom_px(j) & 1)));
}
// Opposite velocities: v_{i+2} = -v_i for i in {0, 1, 4, 5, 8, 9, 12, 13} (pair p, i = pair_rep(p)).
// A moment of odd degree in v changes sign between the two, an even one does not; so does the
// matching column of M^-1: M^-1[i+2][4+j] = +-M^-1[i][4+j] (M P = S M for the swap P of the
// pairs and S = diag(+-1) of the moment parities).
__host__ __device__ constexpr int pair_rep(int p) { return 4 * (p >> 1) + (p & 1); }
__host__ __device__ constexpr bool mom_odd(int j) { return (mom_px(j) + mom_py(j)) & 1; }

// One node (y, x) of the fused update pass: the body of its node loop. dl: the node's row of
// d_x line buffers (line q at dl + q ls, natural order), xl: the node's index in them.
template <typename R, int LOG2N, bool MOMENT_SPACE, bool AX_POSSIBLE>
__device__ __forceinline__ void update_node(const UpdateArgs<R> &a, const UpdateConst<R> &kc, size_t y, int x,
                                            const reg::C<R> *dl, size_t ls, int xl) {
    using CT = reg::C<R>;
    constexpr int NX = 1 << LOG2N;
    const R b = a.b, K = a.K, tau_inv = a.tau_inv, h = a.h;
    const bool adv = !(a.flags & LBM_FLAG_NO_ADVECTION);
    const bool col = !(a.flags & LBM_FLAG_NO_COLLISION);
    const bool frc = !(a.flags & LBM_FLAG_NO_FORCE);
    const bool same_base = a.fbase == a.fs;
    const bool iso = a.flags & LBM_FLAG_ISOTHERMAL;
    const bool ax_mode = AX_POSSIBLE && a.Ax != nullptr;
    {
        const R *fn = a.fs + y * NF_F * NX + x;       // field i at fn[i * NX]
        const R *an = a.Ay + y * NF_A * NX + x;       // slot k at an[k * NX]
        R *mn = a.m + y * NF_M * NX + x;              // macro field k at mn[k * NX]
        const R rho = ldcg(mn + M_RHO * NX), ux = ldcg(mn + M_UX * NX), uy = ldcg(mn + M_UY * NX);
        const R T = ldcg(mn + M_T * NX);
        // I_i = -[A + B.(v_i - u) + (C + C_q)|v_i - u|^2] f_i^eq expands, per node, into
        // -(al + bx v_ix + by v_iy + cc |v_i|^2) f_i^eq; h (the stage's time step) is folded in.
        R hal = 0, hbx = 0, hby = 0, hcc = 0;
        if (frc) {
            const R rT = rho * T;
            const R irT = quot(R(1), rT), irTT = quot(irT, T);
            const R Bx = (ldcg(mn + M_DSXX * NX) + ldcg(mn + M_DSXYY * NX)) * irT;
            const R By = (ldcg(mn + M_DSXY * NX) + ldcg(mn + M_DSYY * NX)) * irT;
            const R C = (ldcg(mn + M_CNUM * NX) - K * rho * ldcg(mn + M_RY * NX) * ldcg(mn + M_DDIVUY * NX)) *
                        (R(0.5) * irTT);
            const R Cq = (ldcg(mn + M_DQX * NX) + ldcg(mn + M_DQY * NX)) * irTT;
            const R CC = C + Cq;
            const R A = R(-2) * CC * T;
            hal = h * (A - Bx * ux - By * uy + CC * (ux * ux + uy * uy));
            hbx = h * (Bx - R(2) * CC * ux);
            hby = h * (By - R(2) * CC * uy);
            hcc = h * CC;
        }
        const R htau = h * tau_inv;
        R m[16];
        equilibrium_moments<R>(rho, ux, uy, T, b, m);
        R fsv[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) fsv[i] = ldcg(fn + i * NX);
        const R *bn = a.fbase + y * NF_F * NX + x;
        R *on = a.fout + y * NF_F * NX + x;
        // f_out_i = f_base_i + h R_i with the non-equilibrium part ne_i = f_i^eq - f_i and the
        // forcing factor q_i = al + bx v_ix + by v_iy + cc |v_i|^2 (all with h folded in)
        auto out_value = [&](auto I, R ne, R q) -> R {
            constexpr int i = decltype(I)::value;
            R dfo = 0;  // h R_i
            if (adv) {
                // -h v_i . grad f_i: both parts come with -h v folded into their multipliers (the
                // row line's second field has the opposite v_x, hence the sign of its part)
                constexpr int xs = xslot(i), ys = yslot(i);
                if constexpr (xs >= 0) {
                    if (ax_mode) {
                        dfo = -h * (R(vel_x(i)) * ldcg(a.Ax + (y * NF_F + i) * NX + x));
                    } else {
                        const CT d = dl[(xs >> 1) * ls + xl];
                        dfo = (xs & 1) ? -d.y : d.x;
                    }
                }
                if constexpr (ys >= 0) dfo += ldcg(an + ys * NX);
            }
            if (col) dfo += htau * ne;
            if (frc) dfo -= q * (fsv[i] + ne);
            return (same_base ? fsv[i] : ldcg(bn + i * NX)) + dfo;
        };
        MomentSums<R> acc;
        if constexpr (MOMENT_SPACE) {
            // neq = M^-1 (m^eq - M f) over the 12 non-conserved moments only (the 4 conserved
            // ones agree exactly), so the rounding of M^-1 to float32 cannot bias mass, momentum
            // or energy: its error scales with the non-equilibrium part instead of with rho.
            // Opposite-velocity pairs: even moments see fi + fk, odd ones fi - fk, and
            // ne_i, ne_k = E +- O from the even and odd columns of M^-1.
            R sp[8], dp[8];
            static_for<0, 8>([&](auto P) {
                constexpr int p = decltype(P)::value, i = pair_rep(p);
                sp[p] = fsv[i] + fsv[i + 2];
                dp[p] = fsv[i] - fsv[i + 2];
            });
            const R eta2 = a.eta2;
            R dm[12];
            static_for<0, 12>([&](auto J) {
                constexpr int j = decltype(J)::value;
                R mf = 0, me = 0;
                static_for<0, 8>([&](auto P) {
                    constexpr int p = decltype(P)::value, i = pair_rep(p);
                    const R g = mom_odd(j) ? dp[p] : sp[p];
                    if constexpr (mom_entry(j, i) != 0.0) mf += R(mom_entry(j, i)) * g;
                    if constexpr (mom_entry_eta(j, i) != 0.0) me += R(mom_entry_eta(j, i)) * g;
                });
                dm[j] = m[4 + j] - (mf + eta2 * me);
            });
            // isothermal: the energy moment (row 3, even) is not conserved by the thermostat either
            R dE = 0;
            if (iso) {
                R me = 0;
                static_for<0, 8>([&](auto P) {
                    constexpr int p = decltype(P)::value;
                    me += kc.psi_hi[pair_rep(p)] * sp[p];
                });
                dE = m[3] - me;
            }
            static_for<0, 8>([&](auto P) {
                constexpr int p = decltype(P)::value, i = pair_rep(p);
                R ev = 0, od = 0;
                static_for<0, 12>([&](auto J) {
                    constexpr int j = decltype(J)::value;
                    if constexpr (!minv_zero(i, j)) {
                        if constexpr (mom_odd(j)) od += kc.minv[i * 16 + 4 + j] * dm[j];
                        else ev += kc.minv[i * 16 + 4 + j] * dm[j];
                    }
                });
                if (iso) ev += kc.minv[i * 16 + 3] * dE;
                R qe = 0, qo = 0;
                if (frc) {
                    qe = hal + hcc * R(vel_sq(i));
                    if constexpr (vel_x(i) != 0.0) qo += hbx * R(vel_x(i));
                    if constexpr (vel_y(i) != 0.0) qo += hby * R(vel_y(i));
                }
                const R fi = out_value(std::integral_constant<int, i>{}, ev + od, qe + qo);
                const R fk = out_value(std::integral_constant<int, i + 2>{}, ev - od, qe - qo);
                on[i * NX] = fi;
                on[(i + 2) * NX] = fk;
                acc.template add_pair<i>(fi, fk, kc.psi_hi[i], kc.psi_lo[i]);
            });
        } else {
            // float64: f^eq = M^-1 m^eq directly
            static_for<0, 16>([&](auto I) {
                constexpr int i = decltype(I)::value;
                R fe = 0;
#pragma unroll
                for (int j = 0; j < 16; ++j) fe += kc.minv[i * 16 + j] * m[j];
                R q = 0;
                if (frc) {
                    q = hal + hcc * R(vel_sq(i));
                    if constexpr (vel_x(i) != 0.0) q += hbx * R(vel_x(i));
                    if constexpr (vel_y(i) != 0.0) q += hby * R(vel_y(i));
                }
                const R fo = out_value(I, fe - fsv[i], q);
                on[i * NX] = fo;
                acc.add(i, fo, kc.psi_hi[i], kc.psi_lo[i]);
            });
        }
        R nr, nux, nuy, nT;
        acc.finish(b, nr, nux, nuy, nT);
        if (iso) nT = a.T_iso;
        mn[M_RHO * NX] = nr;
        mn[M_UX * NX] = nux;
        mn[M_UY * NX] = nuy;
        mn[M_T * NX] = nT;
    }
}

// CS = 1: a CTA owns `rows` whole rows. CS > 1 (float32 rows of 2048 or more, 4096 for CS = 4, one row per
// cluster): the CS CTAs of a cluster split the row's line transforms (fft_reg.cuh) and CTA
// `rank` runs the node loop over its x-range [rank N/CS, (rank + 1) N/CS), whose derivatives the
// transforms leave in its own shared memory.
template <typename R, int LOG2N, bool MOMENT_SPACE, int CS>
__device__ __forceinline__ void update_rows(const UpdateArgs<R> &a, const UpdateConst<R> &kc, int blk, unsigned rank) {
    using F = reg::LineFFT<R, LOG2N, true, CS>;
    using CT = typename F::CT;
    constexpr int NX = F::N, G = F::G, E = F::E, SM = F::STRIDE, NL = F::NL;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    CT *sb = reinterpret_cast<CT *>(smem_raw);
    const int NR = a.rows, nodes = NR * NL;  // nodes of this CTA
    const int y0 = blk * NR, x0 = (int)rank * NL;
    const bool adv = !(a.flags & LBM_FLAG_NO_ADVECTION);
    const bool frc = !(a.flags & LBM_FLAG_NO_FORCE);
    const bool same_base = a.fbase == a.fs;
    // d_x f_i from global memory instead of the row transforms: only float64 rows of 4096 need it
    constexpr bool AX_POSSIBLE = sizeof(R) == 8 && LOG2N == 12 && CS == 1;
    const bool ax_mode = AX_POSSIBLE && a.Ax != nullptr;

    // the node loop's other inputs start moving into L2 while the lines are transformed
    if constexpr (CS == 1) {
        if (threadIdx.x < NR) {
            const size_t y = y0 + threadIdx.x;
            prefetch_l2(a.fs + y * NF_F * NX, NF_F * NX * sizeof(R));
            if (adv) prefetch_l2(a.Ay + y * NF_A * NX, NF_A * NX * sizeof(R));
            if (!same_base) prefetch_l2(a.fbase + y * NF_F * NX, NF_F * NX * sizeof(R));
            if (adv && ax_mode) prefetch_l2(a.Ax + y * NF_F * NX, NF_F * NX * sizeof(R));
            prefetch_l2(a.m + y * NF_M * NX, (M_RY + 1) * NX * sizeof(R));
            if (frc) prefetch_l2(a.m + (y * NF_M + M_DQX) * NX, (NF_M - M_DQX) * NX * sizeof(R));
        }
    } else {  // this CTA's x-range of every field of the row (NR = 1)
        const int k = threadIdx.x;
        const size_t y = y0, bytes = NL * sizeof(R);
        if (k < NF_F) prefetch_l2(a.fs + (y * NF_F + k) * NX + x0, bytes);
        else if (k < NF_F + NF_A) { if (adv) prefetch_l2(a.Ay + (y * NF_A + k - NF_F) * NX + x0, bytes); }
        else if (k < 2 * NF_F + NF_A) { if (!same_base) prefetch_l2(a.fbase + (y * NF_F + k - NF_F - NF_A) * NX + x0, bytes); }
        else if (k < 2 * NF_F + NF_A + NF_M) {
            const int j = k - 2 * NF_F - NF_A;
            if (j <= M_RY || (frc && j >= M_DQX)) prefetch_l2(a.m + (y * NF_M + j) * NX + x0, bytes);
        }
    }

    if (adv && !ax_mode) {
        // 6 lines per row (the 12 fields with v_x != 0, paired); LB lines per batch (LB divides
        // 6 NR); threads past LB G/CS only take part in the barriers
        const int LB = a.lines_per_batch;
        const int ls = threadIdx.x / F::GL, t = (int)rank * F::GL + threadIdx.x % F::GL;
        for (int b0 = 0; b0 < 6 * NR; b0 += LB) {
            if (ls < LB) {
                const int line = b0 + ls;
                const int p = line / NR, r = line % NR;
                CT *buf = sb + (size_t)line * SM;
                const R *frow = a.fs + (size_t)(y0 + r) * NF_F * NX;
                const R *fa = frow + xfield(2 * p) * NX, *fb = frow + xfield(2 * p + 1) * NX;
                CT v[E];
#pragma unroll
                for (int e = 0; e < E; ++e) v[e] = reg::mk<R>(ldcg(fa + t + G * e), ldcg(fb + t + G * e));
                F::template forward<reg::SyncCta>(v, buf, t, a.ax.tw);
                F::multiply(v, t, 1, a.cx[p], a.ax.k1, a.ax.k2);  // -h v_x folded in
                F::template inverse<reg::SyncCta>(v, buf, t, a.ax.tw);
                if constexpr (CS == 1) reg::cta_barrier();  // (a split inverse ends with a cluster barrier)
                F::store_natural(v, buf, t);
            } else {
                F::template idle_forward<reg::SyncCta>();
                F::template idle_inverse<reg::SyncCta>();
                if constexpr (CS == 1) reg::cta_barrier();
            }
        }
        if constexpr (CS == 1) __syncthreads();
        else reg::cluster_barrier();  // every CTA's part of every line has landed
    }

    for (int idx = threadIdx.x; idx < nodes; idx += blockDim.x) {
        const int r = idx / NL, xl = idx % NL;  // xl: index in this CTA's line buffers
        update_node<R, LOG2N, MOMENT_SPACE, AX_POSSIBLE>(a, kc, (size_t)(y0 + r), x0 + xl, sb + (size_t)r * SM,
                                                         (size_t)NR * SM, xl);
    }
}

}  // namespace lbm
