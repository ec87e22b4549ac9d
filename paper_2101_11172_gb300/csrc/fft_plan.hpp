// Host/device description of one shared-memory FFT (see fft.cuh).
#pragma once

#ifdef __CUDACC__
#define WS_HD __host__ __device__
#else
#define WS_HD
#endif

namespace ws {

struct FftPlan {
    int n;            // transform length
    int nstages;
    int radix[8];     // stage radices, first stage first
    int xw[8];        // first-stage digit weights: xw[i] = radix[i+1] * ... * radix[nstages-1]
    int gw[8];        // position weights: gw[i] = radix[1] * ... * radix[i-1]  (gw[1] = 1)
    int lxw[8], lgw[8];  // log2 of xw / gw when n is a power of two
    int logn;         // log2 n when n is a power of two
    int padshift;     // shared-memory padding: one slot after every 2^padshift elements
    int stride;       // float2 slots per transform buffer (== 8 mod 16)
    // ceil(2^32 / d) for the divisors d = xw[i], radix[i] and L[s] = radix[0] * ... *
    // radix[s-1] (0 where d = 1): x / d = umulhi(x, mul) exactly for 0 <= x < 2^16
    // and d < 2^13, since x (mul d - 2^32) < 2^32 (see div_small in fft.cuh)
    unsigned xw_mul[8], r_mul[8], L_mul[8];
};

// ceil(2^32 / d), or 0 for d = 1
WS_HD constexpr unsigned div_mul(int d) {
    return d <= 1 ? 0u : (unsigned)((4294967296ull + (unsigned long long)d - 1ull) / (unsigned long long)d);
}

// Shared-memory index of element e with one pad slot every 2^shift elements.
WS_HD constexpr int fft_pad(int e, int shift) { return e + (e >> shift); }

}  // namespace ws
