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

// exp(2 pi i t z) with z = hi + lo split so that t * hi is exact in FP32
// (hi is a multiple of 2^-13 of magnitude <= 1/2 and |t| < 2^11): the phase in
// turns is frac(t hi) + t lo, reduced exactly before the single rounding.
__device__ __forceinline__ void phase_tz(float t, float2 z, float *s, float *c) {
    float hi = t * z.x;
    float turns = fmaf(t, z.y, hi - rintf(hi));
    sincospif(2.0f * turns, s, c);
}

__device__ __forceinline__ void kahan_add(float &sum, float &comp, float v) {
    float y = v - comp;
    float t = sum + y;
    comp = (t - sum) - y;
    sum = t;
}

}  // namespace ws
