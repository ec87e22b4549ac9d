// Host/device description of one shared-memory FFT (see fft.cuh).
#pragma once

#ifdef __CUDACC__
#define WS_HD __host__ __device__
#else
#define WS_HD
#endif

namespace ws {

struct FftPlan {
    int n;          // transform length
    int nstages;
    int radix[8];   // stage radices, first stage first
    int tpp;        // transforms handled together per pass (1, 2 or 4)
};

// Shared-memory index of element e: one pad slot every 16 elements.
WS_HD constexpr int fft_pad(int e) { return e + (e >> 4); }
WS_HD constexpr int fft_padded_len(int n) { return n + (n >> 4) + 1; }

}  // namespace ws
