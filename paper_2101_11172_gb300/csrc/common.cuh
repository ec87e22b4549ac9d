// Device helpers shared by the CUDA translation units.
#pragma once

#include <cuda_runtime.h>

namespace ws {

// Stack layout of one w-plane: column blocks of CB = 4 grid columns, each
// block stored row after row, so cell (S, R) sits at ((R / 4) N' + S) 4 + R % 4.
// A block column of all N' rows is one contiguous run (the column transforms
// read and write it whole) and a 4-row strip of a block is 128 contiguous
// bytes (what the row transforms move).
constexpr int CB = 4;

__device__ __forceinline__ size_t tiled_index(int S, int R, int Np) {
    return ((size_t)(R >> 2) * Np + S) * CB + (R & 3);
}

// Image index c in [0, N) <-> grid index (stored modulo N') of the centred
// crop |x| < x0: c - N/2 wrapped into [0, N').
__device__ __forceinline__ int crop_to_grid(int c, int half, int Np) { return c < half ? c - half + Np : c - half; }

__device__ __forceinline__ int wrap_add(int a, int b, int n) {
    int s = a + b;
    return s >= n ? s - n : s;
}

// Taylor coefficient (pi/2)^n / n! of sin and cos of a quarter-turn argument.
__host__ __device__ constexpr double quarter_turn_coef(int n) {
    double v = 1.0;
    for (int i = 1; i <= n; ++i) v *= 1.5707963267948966 / i;
    return v;
}

// sin and cos of (pi/2) r for |r| <= 1/2 + 2^-11, i.e. |angle| < 0.787: the
// Taylor series of sin through the r^9 term and of cos through r^10, whose
// first omitted terms are below 1.8e-9 and 1.2e-10.
__device__ __forceinline__ void sincos_quarter(float r, float *s, float *c) {
    constexpr float s1 = (float)quarter_turn_coef(1), s3 = (float)-quarter_turn_coef(3),
                    s5 = (float)quarter_turn_coef(5), s7 = (float)-quarter_turn_coef(7),
                    s9 = (float)quarter_turn_coef(9);
    constexpr float c2 = (float)-quarter_turn_coef(2), c4 = (float)quarter_turn_coef(4),
                    c6 = (float)-quarter_turn_coef(6), c8 = (float)quarter_turn_coef(8),
                    c10 = (float)-quarter_turn_coef(10);
    const float r2 = r * r;
    float ps = fmaf(s9, r2, s7);
    ps = fmaf(ps, r2, s5);
    ps = fmaf(ps, r2, s3);
    ps = fmaf(ps, r2, s1);
    float pc = fmaf(c10, r2, c8);
    pc = fmaf(pc, r2, c6);
    pc = fmaf(pc, r2, c4);
    pc = fmaf(pc, r2, c2);
    *s = ps * r;
    *c = fmaf(pc, r2, 1.0f);
}

// exp(2 pi i t z) with z = hi + lo split so that t * hi is exact in FP32
// (hi is a multiple of 2^-13 of magnitude <= 1/2 and |t| < 2^11).  In quarter
// turns the phase is 4 t hi + 4 t lo: q, its nearest integer, is taken from
// the rounded sum, r = (4 t hi - q) + 4 t lo is formed with one rounding
// (4 t hi - q is exact), and sin and cos of (pi/2)(q + r) follow from those
// of (pi/2) r by the quadrant q mod 4.
__device__ __forceinline__ void phase_tz(float t, float2 z, float *s, float *c) {
    constexpr float kRound = 12582912.0f;            // 1.5 x 2^23: x + kRound holds rint(x) in its low bits
    const float t4 = 4.0f * t;
    const float h4 = t4 * z.x;                       // exact
    const float a = fmaf(t4, z.y, h4) + kRound;
    const float q = a - kRound;
    const float r = fmaf(t4, z.y, h4 - q);
    const unsigned k = __float_as_uint(a);           // q mod 4 in bits 0 and 1
    float ps, pc;
    sincos_quarter(r, &ps, &pc);
    // quadrant k: sin = (S, C, -S, -C)[k], cos = (C, -S, -C, S)[k]
    const bool odd = k & 1u;
    const float sv = odd ? pc : ps, cv = odd ? ps : pc;
    *s = __uint_as_float(__float_as_uint(sv) ^ ((k << 30) & 0x80000000u));
    *c = __uint_as_float(__float_as_uint(cv) ^ (((k + 1u) << 30) & 0x80000000u));
}

__device__ __forceinline__ void kahan_add(float &sum, float &comp, float v) {
    float y = v - comp;
    float t = sum + y;
    comp = (t - sum) - y;
    sum = t;
}

}  // namespace ws
