// Shared-memory line FFTs for the spectral derivatives of Sec. 2.3 / Eq. (3).
//
// A "line" is a complex sequence of N = 2^log2n points that packs two real lines
// (real part = one real field line, imaginary part = another). The spatial derivative
// multiplier d(m) = i k_eff(m) (zero at the Nyquist index) satisfies d(-m) = conj(d(m)),
// so the operator maps real lines to real lines and one complex transform pair
// differentiates two real lines at once.
//
// Forward transforms are radix-4 decimation in frequency (plus one radix-2 stage when
// log2n is odd) and leave the spectrum in digit-reversed order; inverse transforms are the
// exact transpose (decimation in time, conjugate twiddles) and take digit-reversed input
// to natural order. No bit-reversal pass is ever needed: the derivative multiplier tables
// are stored in the same digit-reversed order, with the 1/N of the inverse folded in.
#pragma once
#include <cuda_runtime.h>

namespace lbm {

template <typename R> struct cplx;
template <> struct cplx<double> { typedef double2 T; };
template <> struct cplx<float> { typedef float2 T; };

// L complex lines in shared memory: element k of line l has its real part at
// s[l * ls + k * es] and its imaginary part at s[l * ls + k * es + ioff].
template <typename R> struct LineSet {
    R *s;
    int L, ls, es, ioff;
};

// Work item t -> (line l, butterfly u). LINES_FAST puts consecutive threads on consecutive
// lines (column tiles, where lines are adjacent in memory); otherwise on consecutive
// butterflies of one line (rows, where elements are adjacent).
template <bool LINES_FAST>
__device__ __forceinline__ void split_item(int t, int L, int log2q, int &l, int &u) {
    if (LINES_FAST) {
        l = t % L;
        u = t / L;
    } else {
        u = t & ((1 << log2q) - 1);
        l = t >> log2q;
    }
}

template <typename R>
__device__ __forceinline__ void cmul(R &xr, R &xi, R wr, R wi) {
    R t = xr * wr - xi * wi;
    xi = xr * wi + xi * wr;
    xr = t;
}

template <typename R>
__device__ __forceinline__ void radix2_pass(const LineSet<R> &ls, int log2n) {
    const int nb = ls.L << (log2n - 1);
    for (int t = threadIdx.x; t < nb; t += blockDim.x) {
        int l, u;
        split_item<false>(t, ls.L, log2n - 1, l, u);
        R *p0 = ls.s + l * ls.ls + (2 * u) * ls.es;
        R *p1 = p0 + ls.es;
        R ar = p0[0], ai = p0[ls.ioff], br = p1[0], bi = p1[ls.ioff];
        p0[0] = ar + br;
        p0[ls.ioff] = ai + bi;
        p1[0] = ar - br;
        p1[ls.ioff] = ai - bi;
    }
}

// Forward DFT X[k] = sum_j x[j] exp(-2 pi i j k / N) of every line, output digit-reversed.
// tw[k] = exp(-2 pi i k / N), k < N. Ends with __syncthreads().
template <typename R, bool LINES_FAST>
__device__ void fft_forward(const LineSet<R> ls, int log2n, const typename cplx<R>::T *__restrict__ tw) {
    const int nr4 = log2n >> 1;
    int l2sub = log2n;
    for (int st = 0; st < nr4; ++st) {
        const int l2S = l2sub - 2;
        const int S = 1 << l2S;
        const int tws = log2n - l2sub;
        const int nb = ls.L << (log2n - 2);
        for (int t = threadIdx.x; t < nb; t += blockDim.x) {
            int l, u;
            split_item<LINES_FAST>(t, ls.L, log2n - 2, l, u);
            const int j = u & (S - 1);
            const int base = ((u >> l2S) << l2sub) + j;
            R *p0 = ls.s + l * ls.ls + base * ls.es;
            const int d = S * ls.es, io = ls.ioff;
            R *p1 = p0 + d, *p2 = p1 + d, *p3 = p2 + d;
            R a0r = p0[0], a0i = p0[io], a1r = p1[0], a1i = p1[io];
            R a2r = p2[0], a2i = p2[io], a3r = p3[0], a3i = p3[io];
            R t0r = a0r + a2r, t0i = a0i + a2i;
            R t1r = a0r - a2r, t1i = a0i - a2i;
            R t2r = a1r + a3r, t2i = a1i + a3i;
            R t3r = a1i - a3i, t3i = a3r - a1r;  // -i (a1 - a3)
            R y0r = t0r + t2r, y0i = t0i + t2i;
            R y1r = t1r + t3r, y1i = t1i + t3i;
            R y2r = t0r - t2r, y2i = t0i - t2i;
            R y3r = t1r - t3r, y3i = t1i - t3i;
            if (j) {
                typename cplx<R>::T w1 = tw[j << tws], w2 = tw[(2 * j) << tws], w3 = tw[(3 * j) << tws];
                cmul(y1r, y1i, w1.x, w1.y);
                cmul(y2r, y2i, w2.x, w2.y);
                cmul(y3r, y3i, w3.x, w3.y);
            }
            p0[0] = y0r; p0[io] = y0i;
            p1[0] = y1r; p1[io] = y1i;
            p2[0] = y2r; p2[io] = y2i;
            p3[0] = y3r; p3[io] = y3i;
        }
        __syncthreads();
        l2sub -= 2;
    }
    if (log2n & 1) {
        radix2_pass(ls, log2n);
        __syncthreads();
    }
}

// Inverse (unnormalised: returns N times the inverse DFT) of a digit-reversed spectrum,
// natural-order output. Ends with __syncthreads().
template <typename R, bool LINES_FAST>
__device__ void fft_inverse(const LineSet<R> ls, int log2n, const typename cplx<R>::T *__restrict__ tw) {
    if (log2n & 1) {
        radix2_pass(ls, log2n);
        __syncthreads();
    }
    const int nr4 = log2n >> 1;
    int l2sub = log2n & 1;
    for (int st = 0; st < nr4; ++st) {
        l2sub += 2;
        const int l2S = l2sub - 2;
        const int S = 1 << l2S;
        const int tws = log2n - l2sub;
        const int nb = ls.L << (log2n - 2);
        for (int t = threadIdx.x; t < nb; t += blockDim.x) {
            int l, u;
            split_item<LINES_FAST>(t, ls.L, log2n - 2, l, u);
            const int j = u & (S - 1);
            const int base = ((u >> l2S) << l2sub) + j;
            R *p0 = ls.s + l * ls.ls + base * ls.es;
            const int d = S * ls.es, io = ls.ioff;
            R *p1 = p0 + d, *p2 = p1 + d, *p3 = p2 + d;
            R y0r = p0[0], y0i = p0[io], y1r = p1[0], y1i = p1[io];
            R y2r = p2[0], y2i = p2[io], y3r = p3[0], y3i = p3[io];
            if (j) {
                typename cplx<R>::T w1 = tw[j << tws], w2 = tw[(2 * j) << tws], w3 = tw[(3 * j) << tws];
                cmul(y1r, y1i, w1.x, -w1.y);
                cmul(y2r, y2i, w2.x, -w2.y);
                cmul(y3r, y3i, w3.x, -w3.y);
            }
            R u0r = y0r + y2r, u0i = y0i + y2i;
            R u1r = y0r - y2r, u1i = y0i - y2i;
            R u2r = y1r + y3r, u2i = y1i + y3i;
            R u3r = y3i - y1i, u3i = y1r - y3r;  // +i (y1 - y3)
            p0[0] = u0r + u2r; p0[io] = u0i + u2i;
            p1[0] = u1r + u3r; p1[io] = u1i + u3i;
            p2[0] = u0r - u2r; p2[io] = u0i - u2i;
            p3[0] = u1r - u3r; p3[io] = u1i - u3i;
        }
        __syncthreads();
    }
}

// dst <- M(p) * src for every line, where M is the derivative multiplier of the given
// order at digit-reversed position p, times c:
//   order 1: i c k1[p]   (k1 = k_eff / N, zero at Nyquist)
//   order 2: c k2[p]     (k2 = -k_eff^2 / N, zero at Nyquist)
// dst may equal src. No trailing barrier.
template <typename R, bool LINES_FAST>
__device__ void spec_mul(const LineSet<R> dst, const LineSet<R> src, int log2n, int order, R c,
                         const R *__restrict__ k1, const R *__restrict__ k2) {
    const int n = src.L << log2n;
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        int l, p;
        split_item<LINES_FAST>(t, src.L, log2n, l, p);
        const R *q = src.s + l * src.ls + p * src.es;
        R *o = dst.s + l * dst.ls + p * dst.es;
        R zr = q[0], zi = q[src.ioff];
        if (order == 1) {
            R w = c * k1[p];
            o[0] = -w * zi;
            o[dst.ioff] = w * zr;
        } else {
            R w = c * k2[p];
            o[0] = w * zr;
            o[dst.ioff] = w * zi;
        }
    }
}

}  // namespace lbm
