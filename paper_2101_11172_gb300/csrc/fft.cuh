// FFT engine for the w-plane transforms (Algorithm 5 step 3b, Algorithm 6
// step 3c).
//
// A CTA transforms a few length-n sequences cooperatively with the Stockham
// autosort formulation (every stage reads its butterfly inputs at stride n/R
// and writes them grouped by the running transform size Ns, so no
// bit-reversal pass is needed).  The first stage takes its inputs straight
// from the caller (global memory, with zero padding and screens applied on
// the fly) into registers and the last stage hands its outputs straight back
// (global stores, crops, accumulations); only the stages in between go
// through shared memory, in place: a stage loads all of its butterflies into
// registers and only then, after a barrier, stores the results.  Radices: 16,
// 8, 4 (power-of-two part) and 7, 5, 3.  Twiddles come from a table of
// exp(-2 pi i m / n) computed in double precision on the host.
//
// Shared-memory addressing pads one element every 16 (pad(e) = e + e/16),
// which keeps the strided accesses of the radix-16/8 stages free of bank
// conflicts.
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

// Odd radices: direct R-point DFT with roots of unity from the table.
template <int R>
__device__ __forceinline__ void dft_odd(float2 *v, bool inv, const float2 *__restrict__ tw, int n) {
    float2 o[R];
    const int step = n / R;
#pragma unroll
    for (int k = 0; k < R; ++k) {
        float2 acc = v[0];
#pragma unroll
        for (int r = 1; r < R; ++r) acc = cadd(acc, cmul(v[r], twiddle(tw, ((r * k) % R) * step, inv)));
        o[k] = acc;
    }
#pragma unroll
    for (int k = 0; k < R; ++k) v[k] = o[k];
}
template <>
__device__ __forceinline__ void dft<3>(float2 *v, bool inv, const float2 *__restrict__ tw, int n) {
    dft_odd<3>(v, inv, tw, n);
}
template <>
__device__ __forceinline__ void dft<5>(float2 *v, bool inv, const float2 *__restrict__ tw, int n) {
    dft_odd<5>(v, inv, tw, n);
}
template <>
__device__ __forceinline__ void dft<7>(float2 *v, bool inv, const float2 *__restrict__ tw, int n) {
    dft_odd<7>(v, inv, tw, n);
}

// One Stockham stage of radix R over `count` transforms.  Work item q maps to
// transform t = q % count and butterfly j = q / count (transforms interleaved
// so neighbouring lanes touch neighbouring columns of global memory).  The
// first stage reads its inputs through load(t, e) and the last stage hands
// its outputs to store(t, e, v); the others use the padded shared buffers
// (buf + t * stride).  EPT bounds the elements one thread holds (the host
// checks ceil(count * n / R / nthr) * R <= EPT).
template <int R, int EPT, class Load, class Store>
__device__ __forceinline__ void stage(float2 *buf, int stride, int count, int n, int Ns, bool first, bool last,
                                      const float2 *__restrict__ tw, bool inv, int tid, int nthr, Load &load,
                                      Store &store) {
    constexpr int MAXB = EPT / R;
    const int nb = n / R;
    const int total = count * nb;
    const int twstep = n / (Ns * R);
    float2 v[MAXB > 0 ? MAXB : 1][R];
#pragma unroll
    for (int b = 0; b < MAXB; ++b) {
        const int q = tid + b * nthr;
        if (q < total) {
            const int t = q % count, j = q / count;
            if (first) {
#pragma unroll
                for (int r = 0; r < R; ++r) v[b][r] = load(t, j + r * nb);
            } else {
                const float2 *x = buf + t * stride;
#pragma unroll
                for (int r = 0; r < R; ++r) v[b][r] = x[fft_pad(j + r * nb)];
            }
            if (Ns > 1) {
                const int k = j % Ns;
#pragma unroll
                for (int r = 1; r < R; ++r) v[b][r] = cmul(v[b][r], twiddle(tw, (k * r * twstep) % n, inv));
            }
            dft<R>(v[b], inv, tw, n);
        }
    }
    if (last) {
#pragma unroll
        for (int b = 0; b < MAXB; ++b) {
            const int q = tid + b * nthr;
            if (q < total) {
                const int t = q % count, j = q / count;
                const int idx = (j / Ns) * Ns * R + (j % Ns);
#pragma unroll
                for (int r = 0; r < R; ++r) store(t, idx + r * Ns, v[b][r]);
            }
        }
        return;
    }
    if (!first) __syncthreads();          // every read of this stage done before any write
#pragma unroll
    for (int b = 0; b < MAXB; ++b) {
        const int q = tid + b * nthr;
        if (q < total) {
            const int t = q % count, j = q / count;
            float2 *x = buf + t * stride;
            const int idx = (j / Ns) * Ns * R + (j % Ns);
#pragma unroll
            for (int r = 0; r < R; ++r) x[fft_pad(idx + r * Ns)] = v[b][r];
        }
    }
    __syncthreads();
}

}  // namespace fftdev

// Transform `count` sequences of length P.n (P.tpp of them per pass) from
// load(t, e) to store(t, e, v), using the padded shared buffers buf + t *
// stride (t < P.tpp) between stages.  All threads of the CTA must call it.
// MIXED enables the odd radices; without it only 16, 8 and 4 are compiled,
// which keeps the power-of-two transforms within the register budget.
// The caller must synchronise before reusing buf or reading what store wrote
// to shared memory.
template <int EPT, bool MIXED, class Load, class Store>
__device__ __forceinline__ void fft_many(float2 *buf, int stride, int count, const FftPlan &P,
                                         const float2 *__restrict__ tw, bool inv, int tid, int nthr, Load load,
                                         Store store) {
    for (int t0 = 0; t0 < count; t0 += P.tpp) {
        const int cnt = min(P.tpp, count - t0);
        auto ld = [&](int t, int e) { return load(t0 + t, e); };
        auto st = [&](int t, int e, float2 v) { store(t0 + t, e, v); };
        if (t0 > 0) __syncthreads();
        int Ns = 1;
        for (int s = 0; s < P.nstages; ++s) {
            const int R = P.radix[s];
            const bool first = s == 0, last = s == P.nstages - 1;
            switch (R) {
                case 16: fftdev::stage<16, EPT>(buf, stride, cnt, P.n, Ns, first, last, tw, inv, tid, nthr, ld, st); break;
                case 8: fftdev::stage<8, EPT>(buf, stride, cnt, P.n, Ns, first, last, tw, inv, tid, nthr, ld, st); break;
                case 4: fftdev::stage<4, EPT>(buf, stride, cnt, P.n, Ns, first, last, tw, inv, tid, nthr, ld, st); break;
                default:
                    if constexpr (MIXED) {
                        if (R == 7)
                            fftdev::stage<7, EPT>(buf, stride, cnt, P.n, Ns, first, last, tw, inv, tid, nthr, ld, st);
                        else if (R == 5)
                            fftdev::stage<5, EPT>(buf, stride, cnt, P.n, Ns, first, last, tw, inv, tid, nthr, ld, st);
                        else
                            fftdev::stage<3, EPT>(buf, stride, cnt, P.n, Ns, first, last, tw, inv, tid, nthr, ld, st);
                    }
                    break;
            }
            Ns *= R;
        }
    }
}

}  // namespace ws
