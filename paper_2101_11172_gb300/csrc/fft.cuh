// FFT engine for the w-plane transforms (Algorithm 5 step 3b, Algorithm 6
// step 3c).
//
// A CTA transforms one or two length-n sequences cooperatively with mixed-
// radix decimation in time, in place in shared memory.  The first stage reads
// its inputs straight from the caller (global memory, with zero padding and
// screens applied on the fly), transforms them in registers and scatters them
// to digit-reversed positions; every later stage reads, twiddles, transforms
// and writes back the same R positions, so a thread holds one butterfly at a
// time and a stage needs a single barrier; the last stage hands its outputs
// straight back (global stores, crops, accumulations).  Radices: 16, 8, 4
// (power-of-two part) and 7, 5, 3.  Twiddles come from a table of
// exp(-2 pi i m / n) computed in double precision on the host.
//
// Shared-memory addressing inserts one pad slot after every n / radix[0]
// elements (a power of two), which removes the bank conflicts of the
// digit-reversed scatter for the main sizes; two transforms of a CTA sit
// 8 (mod 16) slots apart so interleaved lanes use different banks.
#pragma once

#include <cuda_runtime.h>

#include "fft_plan.hpp"

namespace ws {

namespace fftdev {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// multiply by -i (forward) or +i (inverse)
__device__ __forceinline__ float2 rot_q(float2 a, bool inv) {
    return inv ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}
// exp(-+ 2 pi i m / n) from the forward table
__device__ __forceinline__ float2 twiddle(const float2 *__restrict__ tw, int m, bool inv) {
    float2 w = __ldg(tw + m);
    return inv ? make_float2(w.x, -w.y) : w;
}

__device__ __forceinline__ void dft4(float2 &a0, float2 &a1, float2 &a2, float2 &a3, bool inv) {
    const float2 t0 = cadd(a0, a2), t1 = csub(a0, a2), t2 = cadd(a1, a3), t3 = rot_q(csub(a1, a3), inv);
    a0 = cadd(t0, t2);
    a2 = csub(t0, t2);
    a1 = cadd(t1, t3);
    a3 = csub(t1, t3);
}

// cos and sin of 2 pi m / 16 for m = 1, 2, 3 (exact decimal expansions)
constexpr float kC1 = 0.92387953251128674f;   // cos(pi/8)
constexpr float kS1 = 0.38268343236508978f;   // sin(pi/8)
constexpr float kR2 = 0.70710678118654752f;   // sqrt(1/2)

// exp(-+ 2 pi i m / 16) for m in 0..9 (the products q*k1 of the 4x4 split)
__device__ __forceinline__ float2 w16(int m, bool inv) {
    float c, s;
    switch (m) {
        case 0: c = 1.f; s = 0.f; break;
        case 1: c = kC1; s = kS1; break;
        case 2: c = kR2; s = kR2; break;
        case 3: c = kS1; s = kC1; break;
        case 4: c = 0.f; s = 1.f; break;
        case 6: c = -kR2; s = kR2; break;
        case 9: c = -kC1; s = -kS1; break;
        default: c = 1.f; s = 0.f; break;   // not reached
    }
    return make_float2(c, inv ? s : -s);
}

template <int R>
__device__ __forceinline__ void dft(float2 *v, bool inv, const float2 *__restrict__ tw, int n);

template <>
__device__ __forceinline__ void dft<4>(float2 *v, bool inv, const float2 *__restrict__, int) {
    dft4(v[0], v[1], v[2], v[3], inv);
}

template <>
__device__ __forceinline__ void dft<8>(float2 *v, bool inv, const float2 *__restrict__, int) {
    float2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
    float2 o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
    dft4(e0, e1, e2, e3, inv);
    dft4(o0, o1, o2, o3, inv);
    const float sg = inv ? 1.f : -1.f;
    o1 = cmul(o1, make_float2(kR2, sg * kR2));
    o2 = rot_q(o2, inv);
    o3 = cmul(o3, make_float2(-kR2, sg * kR2));
    v[0] = cadd(e0, o0);
    v[4] = csub(e0, o0);
    v[1] = cadd(e1, o1);
    v[5] = csub(e1, o1);
    v[2] = cadd(e2, o2);
    v[6] = csub(e2, o2);
    v[3] = cadd(e3, o3);
    v[7] = csub(e3, o3);
}

template <>
__device__ __forceinline__ void dft<16>(float2 *v, bool inv, const float2 *__restrict__, int) {
    // X[k1 + 4 k2] = sum_q w16^(q k1) w4^(q k2) sum_s v[q + 4 s] w4^(s k1)
#pragma unroll
    for (int q = 0; q < 4; ++q) dft4(v[q], v[q + 4], v[q + 8], v[q + 12], inv);
#pragma unroll
    for (int q = 1; q < 4; ++q)
#pragma unroll
        for (int k1 = 1; k1 < 4; ++k1) v[q + 4 * k1] = cmul(v[q + 4 * k1], w16(q * k1, inv));
    float2 o[16];
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
        float2 a0 = v[0 + 4 * k1], a1 = v[1 + 4 * k1], a2 = v[2 + 4 * k1], a3 = v[3 + 4 * k1];
        dft4(a0, a1, a2, a3, inv);
        o[k1] = a0;
        o[k1 + 4] = a1;
        o[k1 + 8] = a2;
        o[k1 + 12] = a3;
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = o[i];
}

// Radix 16 whose middle half of inputs, v[4] .. v[11], is zero (the centred
// half of a sequence of N' = 2N points zero-padded to N'): the first level's
// four 4-point DFTs see (a, 0, 0, d) and reduce to two adds and a quarter
// turn each; v[4..11] need not be set.
__device__ __forceinline__ void dft16_zero_middle(float2 *v, bool inv) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float2 a = v[q], d = v[q + 12], rd = rot_q(d, inv);
        v[q] = cadd(a, d);
        v[q + 8] = csub(a, d);
        v[q + 4] = csub(a, rd);
        v[q + 12] = cadd(a, rd);
    }
#pragma unroll
    for (int q = 1; q < 4; ++q)
#pragma unroll
        for (int k1 = 1; k1 < 4; ++k1) v[q + 4 * k1] = cmul(v[q + 4 * k1], w16(q * k1, inv));
    float2 o[16];
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
        float2 a0 = v[0 + 4 * k1], a1 = v[1 + 4 * k1], a2 = v[2 + 4 * k1], a3 = v[3 + 4 * k1];
        dft4(a0, a1, a2, a3, inv);
        o[k1] = a0;
        o[k1 + 4] = a1;
        o[k1 + 8] = a2;
        o[k1 + 12] = a3;
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = o[i];
}

// cos and sin of 2 pi m / R for the odd radices R = 3, 5, 7 and 0 <= m < R
// (decimal expansions of the closed forms; sin is odd in m about R / 2).
__host__ __device__ constexpr double odd_cos(int R, int m) {
    const int k = m <= R / 2 ? m : R - m;
    return k == 0 ? 1.0
         : R == 3 ? -0.5
         : R == 5 ? (k == 1 ? 0.30901699437494742 : -0.80901699437494742)
         : (k == 1 ? 0.62348980185873353 : k == 2 ? -0.22252093395631440 : -0.90096886790241913);
}
__host__ __device__ constexpr double odd_sin(int R, int m) {
    const int k = m <= R / 2 ? m : R - m;
    const double s = k == 0 ? 0.0
                   : R == 3 ? 0.86602540378443865
                   : R == 5 ? (k == 1 ? 0.95105651629515357 : 0.58778525229247313)
                   : (k == 1 ? 0.78183148246802981 : k == 2 ? 0.97492791218182361 : 0.43388373911755812);
    return m <= R / 2 ? s : -s;
}

// Odd radix R = 2h + 1 in symmetric form.  With a_r = x_r + x_{R-r} and
// b_r = x_r - x_{R-r} (r = 1..h): X_0 = x_0 + sum a_r and, for k = 1..h,
// A_k = x_0 + sum_r cos(2 pi r k / R) a_r, B_k = sum_r sin(2 pi r k / R) b_r,
// X_k = A_k - i B_k and X_{R-k} = A_k + i B_k (the signs swap for the inverse).
template <int R>
__device__ __forceinline__ void dft_odd(float2 *v, bool inv) {
    constexpr int h = R / 2;
    float2 a[h + 1], b[h + 1];
#pragma unroll
    for (int r = 1; r <= h; ++r) {
        a[r] = cadd(v[r], v[R - r]);
        b[r] = csub(v[r], v[R - r]);
    }
    const float2 x0 = v[0];
    float2 s0 = x0;
#pragma unroll
    for (int r = 1; r <= h; ++r) s0 = cadd(s0, a[r]);
    v[0] = s0;
#pragma unroll
    for (int k = 1; k <= h; ++k) {
        float2 A = x0, B = make_float2(0.f, 0.f);
#pragma unroll
        for (int r = 1; r <= h; ++r) {
            const float c = (float)odd_cos(R, (r * k) % R), sn = (float)odd_sin(R, (r * k) % R);
            A.x = fmaf(c, a[r].x, A.x);
            A.y = fmaf(c, a[r].y, A.y);
            B.x = fmaf(sn, b[r].x, B.x);
            B.y = fmaf(sn, b[r].y, B.y);
        }
        const float2 minus = make_float2(A.x + B.y, A.y - B.x);   // A - i B
        const float2 plus = make_float2(A.x - B.y, A.y + B.x);    // A + i B
        v[k] = inv ? plus : minus;
        v[R - k] = inv ? minus : plus;
    }
}
template <>
__device__ __forceinline__ void dft<3>(float2 *v, bool inv, const float2 *__restrict__, int) {
    dft_odd<3>(v, inv);
}
template <>
__device__ __forceinline__ void dft<5>(float2 *v, bool inv, const float2 *__restrict__, int) {
    dft_odd<5>(v, inv);
}
template <>
__device__ __forceinline__ void dft<7>(float2 *v, bool inv, const float2 *__restrict__, int) {
    dft_odd<7>(v, inv);
}
// 10 = 2 x 5: five-point DFTs of the even and of the odd inputs, then
// X_k = E_k + w10^k O_k and X_{k+5} = E_k - w10^k O_k, w10 = exp(-+ 2 pi i / 10).
template <>
__device__ __forceinline__ void dft<10>(float2 *v, bool inv, const float2 *__restrict__, int) {
    float2 e[5] = {v[0], v[2], v[4], v[6], v[8]}, o[5] = {v[1], v[3], v[5], v[7], v[9]};
    dft_odd<5>(e, inv);
    dft_odd<5>(o, inv);
    // cos and sin of 2 pi k / 10, k = 1..4 (cos(pi/5) = (sqrt 5 + 1) / 4, cos(2 pi/5) = (sqrt 5 - 1) / 4)
    constexpr float c[5] = {1.f, 0.80901699437494742f, 0.30901699437494742f, -0.30901699437494742f,
                            -0.80901699437494742f};
    constexpr float sn[5] = {0.f, 0.58778525229247313f, 0.95105651629515357f, 0.95105651629515357f,
                             0.58778525229247313f};
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const float2 t = k == 0 ? o[0] : cmul(o[k], make_float2(c[k], inv ? sn[k] : -sn[k]));
        v[k] = cadd(e[k], t);
        v[k + 5] = csub(e[k], t);
    }
}

// v[m] *= w^m for m = 1..R-1, w = exp(-+ 2 pi i e / n).  The table holds w^m
// to half an ulp, but a warp's loads of w^m for m > 1 scatter over many
// sectors; so only w and w^4 are read and the other powers are products of
// them (at most five roundings: RMS error about 7e-8 against 2e-8 for the
// table, far below the FP32 transform's own rounding).
// The same with w and w^4 given (R = 16 or 8).
template <int R>
__device__ __forceinline__ void twiddle_powers(float2 *v, float2 w1, float2 w4) {
    static_assert(R == 16 || R == 8, "radix 16 or 8");
    const float2 w2 = cmul(w1, w1), w3 = cmul(w2, w1);
    v[1] = cmul(v[1], w1);
    v[2] = cmul(v[2], w2);
    v[3] = cmul(v[3], w3);
    v[4] = cmul(v[4], w4);
    v[5] = cmul(v[5], cmul(w4, w1));
    v[6] = cmul(v[6], cmul(w4, w2));
    v[7] = cmul(v[7], cmul(w4, w3));
    if constexpr (R == 16) {
        const float2 w8 = cmul(w4, w4), w12 = cmul(w8, w4);
        v[8] = cmul(v[8], w8);
        v[9] = cmul(v[9], cmul(w8, w1));
        v[10] = cmul(v[10], cmul(w8, w2));
        v[11] = cmul(v[11], cmul(w8, w3));
        v[12] = cmul(v[12], w12);
        v[13] = cmul(v[13], cmul(w12, w1));
        v[14] = cmul(v[14], cmul(w12, w2));
        v[15] = cmul(v[15], cmul(w12, w3));
    }
}

template <int R>
__device__ __forceinline__ void twiddle_all(float2 *v, const float2 *__restrict__ tw, int e, bool inv) {
    if constexpr (R == 16 || R == 8) {
        twiddle_powers<R>(v, twiddle(tw, e, inv), twiddle(tw, 4 * e, inv));
    } else if constexpr (R == 10) {
        // w^m from w and w^4, products at most two deep
        const float2 w1 = twiddle(tw, e, inv), w4 = twiddle(tw, 4 * e, inv);
        const float2 w2 = cmul(w1, w1), w3 = cmul(w2, w1), w8 = cmul(w4, w4);
        v[1] = cmul(v[1], w1);
        v[2] = cmul(v[2], w2);
        v[3] = cmul(v[3], w3);
        v[4] = cmul(v[4], w4);
        v[5] = cmul(v[5], cmul(w4, w1));
        v[6] = cmul(v[6], cmul(w4, w2));
        v[7] = cmul(v[7], cmul(w4, w3));
        v[8] = cmul(v[8], w8);
        v[9] = cmul(v[9], cmul(w8, w1));
    } else {
        // R <= 7: w^m from w by products, at most three roundings deep
        static_assert(R <= 7, "radices 3 to 7");
        const float2 w1 = twiddle(tw, e, inv), w2 = cmul(w1, w1);
        v[1] = cmul(v[1], w1);
        v[2] = cmul(v[2], w2);
        if constexpr (R >= 4) v[3] = cmul(v[3], cmul(w2, w1));
        if constexpr (R >= 5) v[4] = cmul(v[4], cmul(w2, w2));
        if constexpr (R >= 6) v[5] = cmul(v[5], cmul(cmul(w2, w2), w1));
        if constexpr (R >= 7) {
            const float2 w3 = cmul(w2, w1);
            v[6] = cmul(v[6], cmul(w3, w3));
        }
    }
}

// In-place decimation-in-time stage of radix R: for every block b of R*L
// positions and offset k < L, the R elements at b*R*L + k + m*L (m < R) are
// multiplied by w_{RL}^{k m}, transformed by an R-point DFT and written back
// to the same positions.  Butterflies own disjoint positions, so a thread
// can do them one after another and a stage needs no barrier between its
// reads and writes.  Work item q -> transform t = q % COUNT, butterfly q / COUNT.
// POW2: n, R and L are powers of two and the index arithmetic uses shifts.
// x / d for 0 <= x < 2^16, 1 <= d < 2^13, with mul = div_mul(d) (fft_plan.hpp)
__device__ __forceinline__ int div_small(int x, unsigned mul) {
    return mul ? (int)__umulhi((unsigned)x, mul) : x;
}

template <int R, int COUNT, bool POW2, class Store>
__device__ __forceinline__ void dit_stage(float2 *buf, const FftPlan &P, int L, unsigned Lmul, bool last,
                                          const float2 *__restrict__ tw, bool inv, int tid, int nthr,
                                          Store &store) {
    const int n = P.n, nb = n / R, total = COUNT * nb;
    int logL = 0, lgtw = 0;
    if constexpr (POW2) {
        logL = __ffs(L) - 1;
        lgtw = P.logn - logL - (__ffs(R) - 1);
    }
    const int twstep = POW2 ? 0 : n / (R * L);
    for (int q = tid; q < total; q += nthr) {
        const int t = q % COUNT, bq = q / COUNT;
        int blk, k;
        if constexpr (POW2) {
            blk = bq >> logL;
            k = bq & (L - 1);
        } else {
            blk = div_small(bq, Lmul);
            k = bq - blk * L;
        }
        const int base = blk * R * L + k;
        float2 *x = buf + t * P.stride;
        float2 v[R];
#pragma unroll
        for (int m = 0; m < R; ++m) v[m] = x[fft_pad(base + m * L, P.padshift)];
        if (k > 0) twiddle_all<R>(v, tw, POW2 ? k << lgtw : k * twstep, inv);
        dft<R>(v, inv, tw, n);
        if (last) {
#pragma unroll
            for (int m = 0; m < R; ++m) store(t, base + m * L, v[m]);
        } else {
#pragma unroll
            for (int m = 0; m < R; ++m) x[fft_pad(base + m * L, P.padshift)] = v[m];
        }
    }
    if (!last) __syncthreads();
}

// First stage: butterfly j of each transform reads inputs m*(n/R) + j, m < R,
// straight from load(t, e), and writes them to the digit-reversed positions
// g*R + m that the later in-place stages expect (g = the digits of j in
// reverse order).  A one-stage transform stores directly.
template <int R, int COUNT, bool POW2, class Load, class Store>
__device__ __forceinline__ void dit_first(float2 *buf, const FftPlan &P, const float2 *__restrict__ tw,
                                          bool inv, int tid, int nthr, Load &load, Store &store) {
    const int n = P.n, nb = n / R, total = COUNT * nb;
    for (int q = tid; q < total; q += nthr) {
        const int t = q % COUNT, j = q / COUNT;
        float2 v[R];
#pragma unroll
        for (int m = 0; m < R; ++m) v[m] = load(t, m * nb + j);
        dft<R>(v, inv, tw, n);
        if (P.nstages == 1) {
#pragma unroll
            for (int m = 0; m < R; ++m) store(t, m, v[m]);
            continue;
        }
        int g = 0;
        for (int i = 1; i < P.nstages; ++i) {
            if constexpr (POW2) {
                g += ((j >> P.lxw[i]) & (P.radix[i] - 1)) << P.lgw[i];
            } else {
                const int a = div_small(j, P.xw_mul[i]);
                g += (a - div_small(a, P.r_mul[i]) * P.radix[i]) * P.gw[i];
            }
        }
        float2 *x = buf + t * P.stride;
#pragma unroll
        for (int m = 0; m < R; ++m) x[fft_pad(g * R + m, P.padshift)] = v[m];
    }
    if (P.nstages > 1) __syncthreads();
}

}  // namespace fftdev

// Transform COUNT sequences of length P.n from load(t, e) to store(t, e, v)
// (t < COUNT), using the shared buffers buf + t * P.stride between stages.
// All threads of the CTA must call it; shared buffers may be reused after the
// caller's next barrier.  MIXED enables the odd radices (and integer
// division in the index arithmetic); without it n is a power of two and only
// radices 16, 8 and 4 are compiled.
template <bool MIXED, int COUNT, class Load, class Store>
__device__ __forceinline__ void fft_many(float2 *buf, const FftPlan &P, const float2 *__restrict__ tw, bool inv,
                                         int tid, int nthr, Load load, Store store) {
    constexpr bool POW2 = !MIXED;
    switch (P.radix[0]) {
        case 16: fftdev::dit_first<16, COUNT, POW2>(buf, P, tw, inv, tid, nthr, load, store); break;
        case 8: fftdev::dit_first<8, COUNT, POW2>(buf, P, tw, inv, tid, nthr, load, store); break;
        case 4: fftdev::dit_first<4, COUNT, POW2>(buf, P, tw, inv, tid, nthr, load, store); break;
        default:
            if constexpr (MIXED) {
                if (P.radix[0] == 10) fftdev::dit_first<10, COUNT, POW2>(buf, P, tw, inv, tid, nthr, load, store);
                else if (P.radix[0] == 7) fftdev::dit_first<7, COUNT, POW2>(buf, P, tw, inv, tid, nthr, load, store);
                else if (P.radix[0] == 5) fftdev::dit_first<5, COUNT, POW2>(buf, P, tw, inv, tid, nthr, load, store);
                else fftdev::dit_first<3, COUNT, POW2>(buf, P, tw, inv, tid, nthr, load, store);
            }
            break;
    }
    int L = P.radix[0];
    for (int s = 1; s < P.nstages; ++s) {
        const int R = P.radix[s];
        const bool last = s == P.nstages - 1;
        switch (R) {
            case 16: fftdev::dit_stage<16, COUNT, POW2>(buf, P, L, P.L_mul[s], last, tw, inv, tid, nthr, store); break;
            case 8: fftdev::dit_stage<8, COUNT, POW2>(buf, P, L, P.L_mul[s], last, tw, inv, tid, nthr, store); break;
            case 4: fftdev::dit_stage<4, COUNT, POW2>(buf, P, L, P.L_mul[s], last, tw, inv, tid, nthr, store); break;
            default:
                if constexpr (MIXED) {
                    if (R == 10)
                        fftdev::dit_stage<10, COUNT, POW2>(buf, P, L, P.L_mul[s], last, tw, inv, tid, nthr, store);
                    else if (R == 7)
                        fftdev::dit_stage<7, COUNT, POW2>(buf, P, L, P.L_mul[s], last, tw, inv, tid, nthr, store);
                    else if (R == 5)
                        fftdev::dit_stage<5, COUNT, POW2>(buf, P, L, P.L_mul[s], last, tw, inv, tid, nthr, store);
                    else
                        fftdev::dit_stage<3, COUNT, POW2>(buf, P, L, P.L_mul[s], last, tw, inv, tid, nthr, store);
                }
                break;
        }
        L *= R;
    }
}

// -- compile-time plans for the power-of-two sizes -----------------------------
//
// For N' = 512, 1024, 2048 and 4096 the radix sequence, the digit weights of
// the first stage, the padding and every stride are constants, so each padded
// shared-memory address is one base plus an immediate offset and each
// twiddle index is one multiply.  The layout and the arithmetic are those of
// the runtime engine above (same stride and padding), only specialised.

namespace fftst {

__host__ __device__ constexpr int ilog2(int v) { return v <= 1 ? 0 : 1 + ilog2(v / 2); }

template <int N> struct Radices;
template <> struct Radices<4096> { static constexpr int n = 3, r0 = 16, r1 = 16, r2 = 16; };
template <> struct Radices<2048> { static constexpr int n = 3, r0 = 16, r1 = 16, r2 = 8; };
template <> struct Radices<1024> { static constexpr int n = 3, r0 = 16, r1 = 8, r2 = 8; };
template <> struct Radices<512> { static constexpr int n = 3, r0 = 16, r1 = 8, r2 = 4; };

template <int N> struct Layout {
    static constexpr int shift = ilog2(N / Radices<N>::r0) < 4 ? 4 : ilog2(N / Radices<N>::r0);
    static constexpr int len = (N - 1) + ((N - 1) >> shift) + 1;
    static constexpr int stride = len + ((8 - len % 16) + 16) % 16;
    __host__ __device__ static constexpr int pad(int e) { return e + (e >> shift); }
};

// Crop pruning (N' = 2N, the centred half of a sequence is the crop): PRUNE_IN
// when the inputs outside it are zero, PRUNE_OUT when the outputs outside it
// are not wanted.  In the first stage, input m (N/R0) + j lies outside it for
// R0/4 <= m < 3 R0/4; in the last stage, output k + m (N/R) likewise.
constexpr int PRUNE_IN = 1, PRUNE_OUT = 2;

// First stage (radix R0): inputs m*(N/R0) + j, outputs to digit-reversed g*R0 + m.
template <int N, int COUNT, class Load, int PRUNE = 0>
__device__ __forceinline__ void first(float2 *buf, const float2 *__restrict__ tw, bool inv, int tid, int nthr,
                                      Load &load) {
    using Rd = Radices<N>;
    using Ly = Layout<N>;
    constexpr int R = Rd::r0, nb = N / R, total = COUNT * nb;
    constexpr bool pin = (PRUNE & PRUNE_IN) != 0;
    static_assert(!pin || R == 16, "input pruning is written for a radix-16 first stage");
    // j = d1 * r2 + d2 (x-order); g = d1 + d2 * r1 (position order)
    for (int q = tid; q < total; q += nthr) {
        const int t = q % COUNT, j = q / COUNT;
        float2 v[R];
#pragma unroll
        for (int m = 0; m < R; ++m)
            if (!pin || m < R / 4 || m >= 3 * R / 4) v[m] = load(t, m * nb + j);
        if constexpr (pin)
            fftdev::dft16_zero_middle(v, inv);
        else
            fftdev::dft<R>(v, inv, tw, N);
        const int d1 = j >> ilog2(Rd::r2), d2 = j & (Rd::r2 - 1);
        const int g = d1 + d2 * Rd::r1;
        float2 *x = buf + t * Ly::stride + Ly::pad(g * R);     // R divides 2^shift: one base
#pragma unroll
        for (int m = 0; m < R; ++m) x[m] = v[m];
    }
    __syncthreads();
}

// Later stage of radix R over span L (constant): in place, or to store() if LAST.
// Twiddle bases w, w^4 of the one butterfly a thread owns in a later stage
// (one transform, nthr >= N / R): they do not change from transform to
// transform, so a kernel that loops over many transforms reads them once.
struct StageTw {
    float2 w1, w4;
};

template <int N, int R, int L>
__device__ __forceinline__ StageTw stage_twiddles(const float2 *__restrict__ tw, bool inv, int tid) {
    constexpr int lgtw = ilog2(N / (R * L));
    const int k = tid & (L - 1);
    return StageTw{fftdev::twiddle(tw, k << lgtw, inv), fftdev::twiddle(tw, (4 * k) << lgtw, inv)};
}

template <int N, int COUNT, int R, int L, bool LAST, class Store, int PRUNE = 0>
__device__ __forceinline__ void later(float2 *buf, const float2 *__restrict__ tw, bool inv, int tid, int nthr,
                                      Store &store, const StageTw *pre = nullptr) {
    constexpr bool pout = LAST && (PRUNE & PRUNE_OUT) != 0;
    static_assert(!pout || (R % 4 == 0 && R * L == N), "output pruning needs the last stage, R a multiple of 4");
    using Ly = Layout<N>;
    constexpr int nb = N / R, total = COUNT * nb;
    constexpr int lgL = ilog2(L), lgtw = ilog2(N / (R * L));
    // pad(base + m L) with base = blk R L + k, k < L, is pad_base + m * step when
    //  (a) L is a multiple of 2^shift (the pad of m L is exact), or
    //  (b) R L divides 2^shift ((blk R L + k + m L) >> shift = (blk R L) >> shift);
    // otherwise each element is padded on its own.
    constexpr bool wide = (L >> Ly::shift) > 0;
    constexpr bool inblock = (R * L) <= (1 << Ly::shift);
    constexpr bool affine = wide || inblock;
    constexpr int step = wide ? L + (L >> Ly::shift) : L;
    auto at = [&](int pbase, int base, int m) {
        return affine ? pbase + m * step : Ly::pad(base + m * L);
    };
    for (int q = tid; q < total; q += nthr) {
        const int t = q % COUNT, bq = q / COUNT;
        const int blk = bq >> lgL, k = bq & (L - 1);
        const int base = blk * R * L + k;
        const int pbase = wide ? Ly::pad(base) : base + ((blk * R * L) >> Ly::shift);
        float2 *x = buf + t * Ly::stride;
        float2 v[R];
#pragma unroll
        for (int m = 0; m < R; ++m) v[m] = x[at(pbase, base, m)];
        if (k > 0) {
            if constexpr (R == 16 || R == 8) {
                if (pre) fftdev::twiddle_powers<R>(v, pre->w1, pre->w4);
                else fftdev::twiddle_all<R>(v, tw, k << lgtw, inv);
            } else {
                fftdev::twiddle_all<R>(v, tw, k << lgtw, inv);
            }
        }
        fftdev::dft<R>(v, inv, tw, N);
        if constexpr (LAST) {
#pragma unroll
            for (int m = 0; m < R; ++m)
                if (!pout || m < R / 4 || m >= 3 * R / 4) store(t, base + m * L, v[m]);
        } else {
#pragma unroll
            for (int m = 0; m < R; ++m) x[at(pbase, base, m)] = v[m];
        }
    }
    if constexpr (!LAST) __syncthreads();
}

// First stage for inputs already in the buffer, in natural order at 0..N-1
// (one transform, at most one butterfly per thread: nthr >= N / R0).  Each
// thread reads the R0 inputs m (N/R0) + tid (input m is zero where bit m of
// live is clear, whatever the buffer holds), the CTA synchronises, between()
// runs (the buffer's old contents are dead by then), and the outputs go to
// their padded digit-reversed slots.
template <int N, class Between>
__device__ __forceinline__ void first_inplace(float2 *buf, const float2 *__restrict__ tw, bool inv, int tid,
                                              Between &between, uint32_t live) {
    using Rd = Radices<N>;
    using Ly = Layout<N>;
    constexpr int R = Rd::r0, nb = N / R;
    const bool active = tid < nb;
    float2 v[R];
    if (active) {
#pragma unroll
        for (int m = 0; m < R; ++m) {
            const float2 x = buf[m * nb + tid];
            v[m] = (live >> m) & 1u ? x : make_float2(0.f, 0.f);
        }
    }
    __syncthreads();
    between();
    if (active) {
        fftdev::dft<R>(v, inv, tw, N);
        const int d1 = tid >> ilog2(Rd::r2), d2 = tid & (Rd::r2 - 1);
        float2 *x = buf + Ly::pad((d1 + d2 * Rd::r1) * R);
#pragma unroll
        for (int m = 0; m < R; ++m) x[m] = v[m];
    }
    __syncthreads();
}

}  // namespace fftst

// One transform of the compile-time size N whose input sits in buf in natural
// order (see first_inplace for live); later stages as in fft_static.
template <int N, int PRUNE = 0, class Between, class Store>
__device__ __forceinline__ void fft_static_inplace(float2 *buf, const float2 *__restrict__ tw, bool inv, int tid,
                                                   int nthr, Between between, Store store,
                                                   const fftst::StageTw &s2, const fftst::StageTw &s3,
                                                   uint32_t live = 0xffffffffu) {
    using Rd = fftst::Radices<N>;
    static_assert(Rd::n == 3, "three-stage plans only");
    static_assert((PRUNE & fftst::PRUNE_IN) == 0, "inputs already in the buffer are not pruned");
    fftst::first_inplace<N>(buf, tw, inv, tid, between, live);
    fftst::later<N, 1, Rd::r1, Rd::r0, false>(buf, tw, inv, tid, nthr, store, &s2);
    fftst::later<N, 1, Rd::r2, Rd::r0 * Rd::r1, true, Store, PRUNE>(buf, tw, inv, tid, nthr, store, &s3);
}

// COUNT transforms of the compile-time size N (see fft_many for the contract).
// s2, s3: the thread's twiddle bases of stages 2 and 3 (stage_twiddles), for
// COUNT = 1 callers that transform many sequences; null reads them per call.
template <int N, int COUNT, int PRUNE = 0, class Load, class Store>
__device__ __forceinline__ void fft_static(float2 *buf, const float2 *__restrict__ tw, bool inv, int tid, int nthr,
                                           Load load, Store store, const fftst::StageTw *s2 = nullptr,
                                           const fftst::StageTw *s3 = nullptr) {
    using Rd = fftst::Radices<N>;
    static_assert(Rd::n == 3, "three-stage plans only");
    fftst::first<N, COUNT, Load, PRUNE>(buf, tw, inv, tid, nthr, load);
    fftst::later<N, COUNT, Rd::r1, Rd::r0, false>(buf, tw, inv, tid, nthr, store, s2);
    fftst::later<N, COUNT, Rd::r2, Rd::r0 * Rd::r1, true, Store, PRUNE>(buf, tw, inv, tid, nthr, store, s3);
}

}  // namespace ws
