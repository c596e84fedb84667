// Register-resident line FFTs for the spectral derivatives of Sec. 2.3 / Eq. (3).
//
// A "line" is a complex sequence of N = 2^LOG2N points that packs two real lines (real part
// = one field line, imaginary part = another). The derivative multiplier d(m) = i W(m)
// k_eff(m) satisfies d(-m) = conj(d(m)), so one complex transform pair differentiates two
// real lines at once.
//
// G = N/E threads own a line, E = min(16, N) points each. The forward transform is a
// decimation-in-frequency sequence of radix-16 passes (a 16-point DFT in registers, built as
// 4 x 4, then the outer twiddles) and one final radix-RL pass (RL = 2, 4 or 8) when log2 N
// is not a multiple of 4. Between passes the points are exchanged through a padded
// shared-memory line buffer (one pad slot per 16 points keeps every exchange free of bank
// conflicts, for 8- and 16-byte complex types). The forward output stays in digit-reversed
// order, thread t holding positions [E t, E t + E); the derivative multiplier table holds
// position E t + e at index G e + t (1/N folded in), so the G threads of a line read
// consecutive entries. The inverse is the same pass sequence in reverse, with
// conjugate roots: it takes the digit-reversed spectrum back to natural order, thread t
// holding points t + G e (e < E), the layout in which the forward transform reads its input.
// So rows are read and written with coalesced accesses straight from and to global memory.
#pragma once
#include <cuda_runtime.h>

namespace lbm {

template <typename R> struct cplx;
template <> struct cplx<double> { typedef double2 T; };
template <> struct cplx<float> { typedef float2 T; };

namespace reg {

template <typename R> using C = typename cplx<R>::T;

template <typename R> __device__ __forceinline__ C<R> mk(R x, R y) {
    C<R> c;
    c.x = x;
    c.y = y;
    return c;
}
// Complex addition and subtraction of the butterflies. PK = true: float32 pairs as one packed
// two-lane instruction (add.rn.f32x2, sm_100 and later), the same IEEE results with half
// the instructions; used by the kernels whose registers allow the pairing.
template <typename R, bool PK> struct Arith {
    static __device__ __forceinline__ C<R> add(C<R> a, C<R> b) { return mk<R>(a.x + b.x, a.y + b.y); }
    static __device__ __forceinline__ C<R> sub(C<R> a, C<R> b) { return mk<R>(a.x - b.x, a.y - b.y); }
};
template <> struct Arith<float, true> {
    static __device__ __forceinline__ float2 add(float2 a, float2 b) { return __fadd2_rn(a, b); }
    static __device__ __forceinline__ float2 sub(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
};
// a * w and a * conj(w)
template <typename R> __device__ __forceinline__ C<R> mul(C<R> a, C<R> w) {
    return mk<R>(a.x * w.x - a.y * w.y, a.x * w.y + a.y * w.x);
}
template <typename R> __device__ __forceinline__ C<R> mulc(C<R> a, C<R> w) {
    return mk<R>(a.x * w.x + a.y * w.y, a.y * w.x - a.x * w.y);
}
// multiplication by -i (forward) or +i (inverse)
template <typename R, bool INV> __device__ __forceinline__ C<R> rot(C<R> a) {
    return INV ? mk<R>(-a.y, a.x) : mk<R>(a.y, -a.x);
}

template <typename R, bool INV, bool PK> __device__ __forceinline__ void dft2(C<R> &x0, C<R> &x1) {
    const C<R> t = x0;
    x0 = Arith<R, PK>::add(t, x1);
    x1 = Arith<R, PK>::sub(t, x1);
}

// y_k = sum_q x_q w4^{qk}, w4 = exp(-+ 2 pi i / 4); in place, outputs in natural order
template <typename R, bool INV, bool PK> __device__ __forceinline__ void dft4(C<R> &x0, C<R> &x1, C<R> &x2, C<R> &x3) {
    const C<R> t0 = Arith<R, PK>::add(x0, x2), t1 = Arith<R, PK>::sub(x0, x2), t2 = Arith<R, PK>::add(x1, x3);
    const C<R> t3 = rot<R, INV>(Arith<R, PK>::sub(x1, x3));
    x0 = Arith<R, PK>::add(t0, t2);
    x1 = Arith<R, PK>::add(t1, t3);
    x2 = Arith<R, PK>::sub(t0, t2);
    x3 = Arith<R, PK>::sub(t1, t3);
}

// a * w16^M (forward: w16 = exp(-2 pi i/16); inverse: the conjugate), M a compile-time constant
template <typename R, bool INV, int M> __device__ __forceinline__ C<R> w16(C<R> a) {
    constexpr int m = M & 15;
    if (m == 0) return a;
    if (m == 4) return rot<R, INV>(a);
    if (m == 8) return mk<R>(-a.x, -a.y);
    if (m == 12) return rot<R, !INV>(a);
    // cos and sin of 2 pi m / 16
    constexpr double cs[16] = {1.0, 0.92387953251128675613, 0.70710678118654752440, 0.38268343236508977173,
                               0.0, -0.38268343236508977173, -0.70710678118654752440, -0.92387953251128675613,
                               -1.0, -0.92387953251128675613, -0.70710678118654752440, -0.38268343236508977173,
                               0.0, 0.38268343236508977173, 0.70710678118654752440, 0.92387953251128675613};
    constexpr double sn[16] = {0.0, 0.38268343236508977173, 0.70710678118654752440, 0.92387953251128675613,
                               1.0, 0.92387953251128675613, 0.70710678118654752440, 0.38268343236508977173,
                               0.0, -0.38268343236508977173, -0.70710678118654752440, -0.92387953251128675613,
                               -1.0, -0.92387953251128675613, -0.70710678118654752440, -0.38268343236508977173};
    const R c = (R)cs[m], s = (R)(INV ? sn[m] : -sn[m]);
    return mk<R>(a.x * c - a.y * s, a.x * s + a.y * c);
}

// 16-point DFT in registers (q = q1 + 4 q2, k = k2 + 4 k1); v[k] holds y_k on return
template <typename R, bool INV, bool PK> __device__ __forceinline__ void dft16(C<R> v[16]) {
#pragma unroll
    for (int q1 = 0; q1 < 4; ++q1) dft4<R, INV, PK>(v[q1], v[q1 + 4], v[q1 + 8], v[q1 + 12]);
    // v[q1 + 4 k2] = b(q1, k2); twiddle by w16^(q1 k2)
    v[5] = w16<R, INV, 1>(v[5]);
    v[6] = w16<R, INV, 2>(v[6]);
    v[7] = w16<R, INV, 3>(v[7]);
    v[9] = w16<R, INV, 2>(v[9]);
    v[10] = w16<R, INV, 4>(v[10]);
    v[11] = w16<R, INV, 6>(v[11]);
    v[13] = w16<R, INV, 3>(v[13]);
    v[14] = w16<R, INV, 6>(v[14]);
    v[15] = w16<R, INV, 9>(v[15]);
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) dft4<R, INV, PK>(v[4 * k2], v[4 * k2 + 1], v[4 * k2 + 2], v[4 * k2 + 3]);
    // v[4 k2 + k1] = y(k2 + 4 k1): transpose the 4 x 4 block (register renaming only)
    C<R> t[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) t[k] = v[4 * (k & 3) + (k >> 2)];
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = t[k];
}

// 8-point DFT (q = q1 + 2 q2, k = k2 + 4 k1)
template <typename R, bool INV, bool PK> __device__ __forceinline__ void dft8(C<R> v[8]) {
    dft4<R, INV, PK>(v[0], v[2], v[4], v[6]);
    dft4<R, INV, PK>(v[1], v[3], v[5], v[7]);
    // v[q1 + 2 k2] = b(q1, k2); twiddle q1 = 1 by w8^k2 = w16^(2 k2)
    v[3] = w16<R, INV, 2>(v[3]);
    v[5] = w16<R, INV, 4>(v[5]);
    v[7] = w16<R, INV, 6>(v[7]);
    dft2<R, INV, PK>(v[0], v[1]);
    dft2<R, INV, PK>(v[2], v[3]);
    dft2<R, INV, PK>(v[4], v[5]);
    dft2<R, INV, PK>(v[6], v[7]);
    // v[2 k2 + k1] = y(k2 + 4 k1)
    C<R> t[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) t[k] = v[2 * (k & 3) + (k >> 2)];
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = t[k];
}

template <typename R, bool INV, int RADIX, bool PK> __device__ __forceinline__ void dft_small(C<R> *v) {
    if (RADIX == 2) dft2<R, INV, PK>(v[0], v[1]);
    if (RADIX == 4) dft4<R, INV, PK>(v[0], v[1], v[2], v[3]);
    if (RADIX == 8) dft8<R, INV, PK>(v);
}

// CTA-wide barrier in its non-aligned form (PTX barrier.sync without .aligned): threads of one
// warp may reach it from different branches. Kernels give their threads different roles (a
// thread transforms a line, or only keeps the barrier count while others do), and the split
// between roles need not fall on a warp boundary; the aligned form (__syncthreads) would be
// undefined there. Same memory ordering among the CTA's threads as __syncthreads.
__device__ __forceinline__ void cta_barrier() { asm volatile("barrier.sync 0;" ::: "memory"); }
struct SyncCta {
    static __device__ __forceinline__ void run() { cta_barrier(); }
};
struct SyncWarp {
    static __device__ __forceinline__ void run() { __syncwarp(); }
};

// ---- thread-block clusters: a line split over CS CTAs of one cluster ----------------------
// rank of this CTA in its cluster
__device__ __forceinline__ unsigned cluster_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
// barrier over every thread of every CTA of the cluster, with release / acquire ordering of
// shared-memory accesses at cluster scope (non-aligned form: threads may arrive from different
// branches)
__device__ __forceinline__ void cluster_barrier() {
    asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}
// shared::cluster address of the same shared-memory offset as p in the CTA of the given rank
__device__ __forceinline__ uint32_t cluster_map(const void *p, unsigned rank) {
    const uint32_t a = static_cast<uint32_t>(__cvta_generic_to_shared(p));
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}
__device__ __forceinline__ void st_cluster(uint32_t a, float2 v) {
    asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(a), "f"(v.x), "f"(v.y) : "memory");
}
__device__ __forceinline__ void st_cluster(uint32_t a, double2 v) {
    asm volatile("st.shared::cluster.v2.f64 [%0], {%1, %2};" ::"r"(a), "d"(v.x), "d"(v.y) : "memory");
}
__device__ __forceinline__ void ld_cluster(uint32_t a, float2 &v) {
    asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a) : "memory");
}
__device__ __forceinline__ void ld_cluster(uint32_t a, double2 &v) {
    asm volatile("ld.shared::cluster.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "r"(a) : "memory");
}

// Twiddle table of a line length n = 2^log2n: for each radix-16 pass P (span S = n / 16^P,
// M = S / 16 sub-sequences, M > 1) the roots w_n^(16^P j k) for k = 1..15, j = 0..M-1 at
// index twiddle_offset(n, P) + (k - 1) M + j, so the threads of a pass (consecutive j)
// read consecutive entries. The table has fewer than n entries.
__host__ __device__ constexpr int twiddle_offset(int n, int P) {
    return P == 0 ? 0 : twiddle_offset(n, P - 1) + 15 * (n >> (4 * P));
}
// exponent a (root w_n^a) stored at table index idx; -1 for an unused slot
__host__ __device__ inline int twiddle_exponent(int n, int idx) {
    for (int P = 0, off = 0; (n >> (4 * (P + 1))) >= 1; ++P) {
        const int M = n >> (4 * (P + 1));
        if (idx < off + 15 * M) {
            const int k = (idx - off) / M + 1, j = (idx - off) % M;
            return (int)(((long long)j * k << (4 * P)) & (n - 1));
        }
        off += 15 * M;
    }
    return -1;
}

// CS > 1: the line is split over the CS CTAs of a thread-block cluster. Thread t of the line
// (0 <= t < G, numbered across the cluster) lives in the CTA of rank t / (G / CS), and each CTA's
// line buffer holds the positions [rank N/CS, (rank + 1) N/CS) (padded). Every exchange but one
// stays inside a CTA: the points of the first radix-16 pass (stride G) are spread over the whole
// line, so the forward transform writes them into the other CTAs' buffers (distributed shared
// memory) between two cluster barriers, and the inverse reads them back from there; an inverse
// ends with a cluster barrier so that no CTA reuses or releases a buffer another still reads.
template <typename R, int LOG2N, bool PK = false, int CS = 1> struct LineFFT {
    static constexpr int N = 1 << LOG2N;
    static constexpr int E = N < 16 ? N : 16;                // points per thread
    static constexpr int G = N / E;                          // threads per line
    static constexpr int NP16 = LOG2N >= 4 ? LOG2N / 4 : 0;  // radix-16 passes
    static constexpr int RL = LOG2N >= 4 ? (1 << (LOG2N & 3)) : N;  // final radix (1 = none)
    static_assert(CS == 1 || (NP16 >= 2 && CS <= 16 && G % CS == 0), "cluster split needs lines of 256+ points");
    static constexpr int NL = N / CS;                        // positions held by one CTA
    static constexpr int GL = G / CS;                        // threads of a line in one CTA
    static constexpr int SMEM = NL + (NL >> 4);              // padded line buffer, complex elements
    // distance between consecutive line buffers of the row passes: two extra elements shift each
    // buffer by 16 or 32 bytes (the column tiles, whose lines share warps, space their buffers by
    // their line count instead: col_line_stride in lbm_internal.cuh)
    static constexpr int STRIDE = SMEM + 2;
    typedef C<R> CT;

    static __device__ __forceinline__ int pad(int p) { return p + (p >> 4); }
    // padded index of this CTA's first position (0 without a cluster split)
    static __device__ __forceinline__ int pad_base() {
        if constexpr (CS == 1) return 0;
        else return pad((int)cluster_rank() * NL);
    }
    // position of point e of thread t in the input layout of radix-16 pass P
    template <int P> static __device__ __forceinline__ int pos16(int t, int e) {
        constexpr int S = N >> (4 * P), M = S >> 4;
        return (t / M) * S + (t & (M - 1)) + M * e;
    }

    template <int P, bool INV> static __device__ __forceinline__ void pass16(CT v[16], int t, const CT *__restrict__ tw) {
        constexpr int S = N >> (4 * P), M = S >> 4;
        const int j = t & (M - 1);
        const CT *twp = tw + twiddle_offset(N, P) + j;  // root of (j, k) at twp[(k - 1) M]
        if (INV) {
            if (M > 1 && j) {
#pragma unroll
                for (int k = 1; k < 16; ++k) v[k] = mulc<R>(v[k], twp[(k - 1) * M]);
            }
            dft16<R, true, PK>(v);
        } else {
            dft16<R, false, PK>(v);
            if (M > 1 && j) {
#pragma unroll
                for (int k = 1; k < 16; ++k) v[k] = mul<R>(v[k], twp[(k - 1) * M]);
            }
        }
    }

    template <int P> static __device__ __forceinline__ void store16(const CT v[E], CT *buf, int t, int pb = 0) {
#pragma unroll
        for (int e = 0; e < E; ++e) buf[pad(pos16<P>(t, e)) - pb] = v[e];
    }
    template <int P> static __device__ __forceinline__ void load16(CT v[E], const CT *buf, int t, int pb = 0) {
#pragma unroll
        for (int e = 0; e < E; ++e) v[e] = buf[pad(pos16<P>(t, e)) - pb];
    }
    static __device__ __forceinline__ void storeF(const CT v[E], CT *buf, int t, int pb = 0) {
#pragma unroll
        for (int e = 0; e < E; ++e) buf[pad(t * E + e) - pb] = v[e];
    }
    static __device__ __forceinline__ void loadF(CT v[E], const CT *buf, int t, int pb = 0) {
#pragma unroll
        for (int e = 0; e < E; ++e) v[e] = buf[pad(t * E + e) - pb];
    }
    // the layout of the first radix-16 pass across the cluster: position t + G e is held by the
    // CTA of rank e CS / 16 (a compile-time value per e once the loop is unrolled)
    // (the E / CS points bound for one rank are consecutive in e, so one mapped base at a time)
    static __device__ __forceinline__ void store0_remote(const CT v[E], CT *buf, int t) {
        const uint32_t off = (uint32_t)pad(t) * (uint32_t)sizeof(CT);
#pragma unroll
        for (int r = 0; r < CS; ++r) {
            const uint32_t base = cluster_map(buf, r) + off;
#pragma unroll
            for (int e = r * (E / CS); e < (r + 1) * (E / CS); ++e)
                st_cluster(base + (uint32_t)(pad(t + G * e) - pad(t) - pad(r * NL)) * (uint32_t)sizeof(CT), v[e]);
        }
    }
    static __device__ __forceinline__ void load0_remote(CT v[E], const CT *buf, int t) {
        const uint32_t off = (uint32_t)pad(t) * (uint32_t)sizeof(CT);
#pragma unroll
        for (int r = 0; r < CS; ++r) {
            const uint32_t base = cluster_map(buf, r) + off;
#pragma unroll
            for (int e = r * (E / CS); e < (r + 1) * (E / CS); ++e)
                ld_cluster(base + (uint32_t)(pad(t + G * e) - pad(t) - pad(r * NL)) * (uint32_t)sizeof(CT), v[e]);
        }
    }
    // results in natural order x = t + G e, unpadded, into the line buffer of the CTA that holds x
    // (a plain local store without a cluster split); the caller synchronises before reading
    static __device__ __forceinline__ void store_natural(const CT v[E], CT *buf, int t) {
        if constexpr (CS == 1) {
#pragma unroll
            for (int e = 0; e < E; ++e) buf[t + G * e] = v[e];
        } else {
#pragma unroll
            for (int r = 0; r < CS; ++r) {
                const uint32_t base = cluster_map(buf + t, r);
#pragma unroll
                for (int e = r * (E / CS); e < (r + 1) * (E / CS); ++e)
                    st_cluster(base + (uint32_t)(G * e - r * NL) * (uint32_t)sizeof(CT), v[e]);
            }
        }
    }

    template <int P, class SYNC> static __device__ __forceinline__ void fwd_from(CT v[E], CT *buf, int t,
                                                                                const CT *__restrict__ tw, int pb) {
        if constexpr (P < NP16) {
            pass16<P, false>(v, t, tw);
            if constexpr (P + 1 < NP16) {
                if constexpr (P == 0 && CS > 1) {  // the one exchange across the cluster
                    cluster_barrier();
                    store0_remote(v, buf, t);
                    cluster_barrier();
                } else {
                    SYNC::run();
                    store16<P>(v, buf, t, pb);
                    SYNC::run();
                }
                load16<P + 1>(v, buf, t, pb);
            } else if constexpr (RL > 1) {
                SYNC::run();
                store16<P>(v, buf, t, pb);
                SYNC::run();
                loadF(v, buf, t, pb);
            }
            fwd_from<P + 1, SYNC>(v, buf, t, tw, pb);
        } else if constexpr (RL > 1) {
#pragma unroll
            for (int kb = 0; kb < E / RL; ++kb) dft_small<R, false, RL, PK>(v + kb * RL);
        }
    }

    template <int P, class SYNC> static __device__ __forceinline__ void inv_from(CT v[E], CT *buf, int t,
                                                                                const CT *__restrict__ tw, int pb) {
        if constexpr (P >= 0) {
            pass16<P, true>(v, t, tw);
            if constexpr (P > 0) {
                SYNC::run();
                store16<P>(v, buf, t, pb);
                if constexpr (P == 1 && CS > 1) {  // read the first pass's layout across the cluster
                    cluster_barrier();
                    load0_remote(v, buf, t);
                } else {
                    SYNC::run();
                    load16<P - 1>(v, buf, t, pb);
                }
                inv_from<P - 1, SYNC>(v, buf, t, tw, pb);
            }
        }
    }

    // Forward DFT of a line held as v[e] = x[t + G e]; on return v[e] = X at digit-reversed
    // position E t + e. buf: this line's shared buffer of SMEM elements. Every thread of the
    // block (SyncCta) or warp (SyncWarp) must call it; with a cluster split, every thread of
    // the cluster.
    template <class SYNC> static __device__ __forceinline__ void forward(CT v[E], CT *buf, int t,
                                                                        const CT *__restrict__ tw) {
        fwd_from<0, SYNC>(v, buf, t, tw, pad_base());
    }

    // Inverse (N times the inverse DFT) of a spectrum held at positions E t + e; on return
    // v[e] = x[t + G e].
    template <class SYNC> static __device__ __forceinline__ void inverse(CT v[E], CT *buf, int t,
                                                                        const CT *__restrict__ tw) {
        const int pb = pad_base();
        if constexpr (RL > 1) {
#pragma unroll
            for (int kb = 0; kb < E / RL; ++kb) dft_small<R, true, RL, PK>(v + kb * RL);
            if constexpr (NP16 > 0) {
                SYNC::run();
                storeF(v, buf, t, pb);
                SYNC::run();
                load16<NP16 - 1>(v, buf, t, pb);
            }
        }
        inv_from<NP16 - 1, SYNC>(v, buf, t, tw, pb);
        if constexpr (CS > 1) cluster_barrier();
    }

    // Barriers only: a thread with no line in this transform calls it so that the block's
    // barrier count matches the threads that run forward() or inverse() (same count each).
    static constexpr int EXCHANGES = (NP16 > 1 ? NP16 - 1 : 0) + ((RL > 1 && NP16 > 0) ? 1 : 0);
    template <class SYNC> static __device__ __forceinline__ void idle() {
        static_assert(CS == 1, "with a cluster split use idle_forward / idle_inverse");
#pragma unroll
        for (int k = 0; k < 2 * EXCHANGES; ++k) SYNC::run();
    }
    // the barrier sequence of forward() / inverse() (CTA barriers and, with a cluster split,
    // cluster barriers in the same order)
    template <class SYNC> static __device__ __forceinline__ void idle_forward() {
        if constexpr (CS == 1) {
            idle<SYNC>();
        } else {
            cluster_barrier();
            cluster_barrier();
#pragma unroll
            for (int k = 0; k < 2 * (EXCHANGES - 1); ++k) SYNC::run();
        }
    }
    template <class SYNC> static __device__ __forceinline__ void idle_inverse() {
        if constexpr (CS == 1) {
            idle<SYNC>();
        } else {
#pragma unroll
            for (int k = 0; k < 2 * (EXCHANGES - 1); ++k) SYNC::run();
            SYNC::run();
            cluster_barrier();
            cluster_barrier();
        }
    }

    // v <- d^order * c * v at positions E t + e (tables k1 = W k_eff / N, k2 = -(W k_eff)^2 / N,
    // position E t + e at index G e + t)
    static __device__ __forceinline__ void multiply(CT v[E], int t, int order, R c, const R *__restrict__ k1,
                                                    const R *__restrict__ k2) {
#pragma unroll
        for (int e = 0; e < E; ++e) {
            if (order == 1) {
                const R w = c * k1[G * e + t];
                v[e] = mk<R>(-w * v[e].y, w * v[e].x);
            } else {
                const R w = c * k2[G * e + t];
                v[e] = mk<R>(w * v[e].x, w * v[e].y);
            }
        }
    }
};

}  // namespace reg
}  // namespace lbm
