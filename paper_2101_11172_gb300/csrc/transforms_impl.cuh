// Kernel templates of the fused plane transforms (see transforms.cu).
//
// NP selects the FFT code: 0 = runtime plan, power of two; 1 = runtime plan
// with odd radices; 512, 1024, 2048, 4096 = the compile-time plans of
// fft.cuh.  Each translation unit instantiates Transforms<NP> for its sizes.
#pragma once

#include <cuda.h>

#include "common.cuh"
#include "fft.cuh"
#include "ws_internal.hpp"

namespace ws {
namespace tf {

constexpr int kThreads = 256;       // two rows or two columns per CTA
constexpr int kPerCta = 2;
constexpr int kRowThreads = 256;    // one row per CTA (inv_rows)
// Shared memory per CTA that still lets two CTAs share an SM (228 KB, 1 KB of it reserved per CTA).
constexpr size_t kTwoCtaSmem = 113 * 1024;

// Runtime-plan inv_rows keeps the z row in shared memory when the row buffer,
// the z row and the compensated sums still leave room for two CTAs per SM.
__host__ __device__ inline bool rows_keep_z(const FftPlan &F, int N) {
    return (size_t)F.stride * sizeof(float2) + (size_t)N * (sizeof(float2) + sizeof(float4)) + F.n / TU + 16 <=
           kTwoCtaSmem;
}

__device__ __forceinline__ int grid_to_crop(int g, int half, int Np) { return g < half ? g + half : g - (Np - half); }
__device__ __forceinline__ bool in_crop(int g, int half, int Np) { return g < half || g >= Np - half; }

// PRUNE (fftst::PRUNE_IN / PRUNE_OUT, compile-time plans with N' = 2N only):
// the inputs outside the centred half are zero / the outputs outside it are
// not wanted, and the transform skips them.
template <int NP, int COUNT, int PRUNE = 0, class Load, class Store>
__device__ __forceinline__ void plane_fft(float2 *buf, const FftPlan &F, const float2 *__restrict__ tw, bool inv,
                                          int tid, int nthr, Load load, Store store) {
    if constexpr (NP == 0)
        fft_many<false, COUNT>(buf, F, tw, inv, tid, nthr, load, store);
    else if constexpr (NP == 1)
        fft_many<true, COUNT>(buf, F, tw, inv, tid, nthr, load, store);
    else
        fft_static<NP, COUNT, PRUNE>(buf, tw, inv, tid, nthr, load, store);
}

// CROP: N' = 2N on a compile-time plan, so the crop is exactly the centred half.
template <int NP>
inline bool crop_half(const Launch &L) { return NP >= 512 && 2 * L.N == L.Np; }

// -- degridding --------------------------------------------------------------

// Planes per exact evaluation of the screen in fwd_rows: in between, each
// pixel's screened value advances one plane by a product with exp(-2 pi i z).
constexpr int kScreenSteps = 8;

// One CTA owns image row ii for a run of planes: the corrected row and its z
// stay in shared memory, so each plane costs the screen, one FFT and the
// stores of the strips some footprint reads.
//
// STEP keeps two more shared rows, the screened row g = row x exp(-2 pi i t z)
// and the step exp(-2 pi i z).  g is evaluated exactly on every kScreenSteps-th
// plane of the CTA's share; on the planes between, the FFT's first stage reads
// g and leaves g x step in its place for the next plane.  Each pixel is read
// by the same thread on every plane, so the update needs no barrier.
template <int NP, bool STEP, bool CROP>
__global__ void __launch_bounds__(kRowThreads, 2)
fwd_rows_kernel(Launch L, FftPlan F, const float2 *__restrict__ tw, const float2 *__restrict__ img,
                const float2 *__restrict__ zsplit, const uint8_t *__restrict__ col_occ, int plane0, int planes,
                float2 *__restrict__ stack) {
    extern __shared__ __align__(16) float2 sbuf[];
    const int Np = L.Np, N = L.N, half = N / 2;
    float2 *irow = sbuf + F.stride;                              // N (F.stride is even: 16-byte aligned)
    float2 *zrow = irow + N;                                     // N
    float2 *grow = zrow + N;                                     // N, STEP only: the screened row
    float2 *erow = grow + N;                                     // N, STEP only: exp(-2 pi i z)
    uint8_t *occ = reinterpret_cast<uint8_t *>(irow + (STEP ? 4 : 2) * N);   // ntu: strips of the current t-tile
    const int ii = blockIdx.x, tid = threadIdx.x;
    // this CTA's planes: an equal share of the chunk's valid planes
    const int nvalid = min(planes, L.Nw - plane0);
    const int per = (nvalid + (int)gridDim.y - 1) / (int)gridDim.y;
    const int p_begin = (int)blockIdx.y * per, p_end = min(nvalid, p_begin + per);
    if (p_begin >= p_end) return;
    const size_t pix0 = (size_t)ii * N;
    for (int jj = tid; jj < N; jj += kRowThreads) {
        irow[jj] = img[pix0 + jj];
        const float2 z = zsplit[pix0 + jj];
        zrow[jj] = z;
        if constexpr (STEP) {
            float sn, cs;
            phase_tz(1.f, z, &sn, &cs);
            erow[jj] = make_float2(cs, -sn);
        }
    }
    int occ_tt = -1;
    fftst::StageTw s2{}, s3{};                                  // the thread's twiddle bases, read once
    if constexpr (NP >= 512) {
        using Rd = fftst::Radices<NP>;
        s2 = fftst::stage_twiddles<NP, Rd::r1, Rd::r0>(tw, false, tid);
        s3 = fftst::stage_twiddles<NP, Rd::r2, Rd::r0 * Rd::r1>(tw, false, tid);
    }
    for (int p = p_begin; p < p_end; ++p) {
        const int pl = plane0 + p;
        const float t = (float)(pl + L.t_lo);
        float2 *plane = stack + (size_t)p * Np * Np;
        const int tt = pl / TT;
        __syncthreads();                     // row and z visible; the previous plane's last stage is done
        if (tt != occ_tt) {                  // uniform across the CTA
            for (int i = tid; i < L.ntu; i += kRowThreads) occ[i] = col_occ[tt * L.ntu + i];
            occ_tt = tt;
            __syncthreads();
        }
        // row x exp(-i phi), phi = 2 pi t z
        auto screened = [&](int jj) -> float2 {
            const float2 f = irow[jj];
            float sn, cs;
            phase_tz(t, zrow[jj], &sn, &cs);
            return make_float2(f.x * cs + f.y * sn, f.y * cs - f.x * sn);
        };
        bool step = false;                   // uniform: advance g to the next plane
        if constexpr (STEP) {
            if ((p - p_begin) % kScreenSteps == 0) {
                for (int jj = tid; jj < N; jj += kRowThreads) grow[jj] = screened(jj);
                __syncthreads();
            }
            step = (p + 1 - p_begin) % kScreenSteps != 0 && p + 1 < p_end;
        }
        auto load = [&](int, int J) -> float2 {
            if (!in_crop(J, half, Np)) return make_float2(0.f, 0.f);
            const int jj = grid_to_crop(J, half, Np);
            if constexpr (!STEP) {
                return screened(jj);
            } else {
                const float2 g = grow[jj];
                if (step) {
                    const float2 e = erow[jj];
                    grow[jj] = make_float2(g.x * e.x - g.y * e.y, g.x * e.y + g.y * e.x);
                }
                return g;
            }
        };
        // columns of this plane's t-tile that no footprint touches are never read
        auto store = [&](int, int R, float2 v) {
            if (occ[R / TU]) __stcs(plane + tiled_index(ii, R, Np), v);
        };
        if constexpr (NP >= 512)
            fft_static<NP, 1, CROP ? fftst::PRUNE_IN : 0>(sbuf, tw, false, tid, kRowThreads, load, store, &s2, &s3);
        else
            plane_fft<NP, 1>(sbuf, F, tw, false, tid, kRowThreads, load, store);
    }
}

template <int NP, bool CROP>
__global__ void __launch_bounds__(kThreads, 2)
fwd_cols_kernel(Launch L, FftPlan F, const float2 *__restrict__ tw, const uint8_t *__restrict__ tile_occ,
                const uint8_t *__restrict__ col_occ, int plane0, float2 *__restrict__ stack) {
    extern __shared__ __align__(16) float2 sbuf[];
    const int Np = L.Np, half = L.N / 2;
    const int R0 = blockIdx.x * kPerCta;                  // two of the four columns of a block
    const int tt = (plane0 + (int)blockIdx.y) / TT, tu = R0 / TU;
    if (plane0 + (int)blockIdx.y >= L.Nw) return;         // padding planes of the last t-tile: never read
    if (!col_occ[tt * L.ntu + tu]) return;                // no visibility reads these columns of this plane
    float2 *blk = stack + (size_t)blockIdx.y * Np * Np + (size_t)(R0 >> 2) * Np * CB + (R0 & 3);
    uint8_t *occ = reinterpret_cast<uint8_t *>(sbuf + kPerCta * F.stride);
    for (int i = threadIdx.x; i < L.ntv; i += kThreads) occ[i] = tile_occ[((size_t)tt * L.ntv + i) * L.ntu + tu];
    __syncthreads();
    // rows 0..N-1 hold the N transformed image rows; every other row is zero padding
    auto load = [&](int b, int S) -> float2 {
        if (!in_crop(S, half, Np)) return make_float2(0.f, 0.f);
        return __ldcs(blk + (size_t)grid_to_crop(S, half, Np) * CB + b);
    };
    auto store = [&](int b, int S, float2 v) {
        if (occ[S >> L.tv_log]) blk[(size_t)S * CB + b] = v;     // only tiles the gather reads
    };
    plane_fft<NP, kPerCta, CROP ? fftst::PRUNE_IN : 0>(sbuf, F, tw, false, threadIdx.x, kThreads, load, store);
}

// -- gridding ----------------------------------------------------------------

template <int NP, bool CROP>
__global__ void __launch_bounds__(kThreads, 2)
inv_cols_kernel(Launch L, FftPlan F, const float2 *__restrict__ tw, const uint8_t *__restrict__ tile_occ,
                const uint8_t *__restrict__ col_occ, int plane0, float2 *__restrict__ stack) {
    extern __shared__ __align__(16) float2 sbuf[];
    const int Np = L.Np, half = L.N / 2;
    const int R0 = blockIdx.x * kPerCta;
    const int tt = (plane0 + (int)blockIdx.y) / TT, tu = R0 / TU;
    if (plane0 + (int)blockIdx.y >= L.Nw) return;         // padding planes of the last t-tile: inv_rows skips them
    if (!col_occ[tt * L.ntu + tu]) return;                // all-zero columns: inv_rows skips them too
    float2 *blk = stack + (size_t)blockIdx.y * Np * Np + (size_t)(R0 >> 2) * Np * CB + (R0 & 3);
    uint8_t *occ = reinterpret_cast<uint8_t *>(sbuf + kPerCta * F.stride);
    for (int i = threadIdx.x; i < L.ntv; i += kThreads) occ[i] = tile_occ[((size_t)tt * L.ntv + i) * L.ntu + tu];
    __syncthreads();
    // gridding wrote only occupied tiles; every other cell is zero
    auto load = [&](int b, int S) -> float2 {
        return occ[S >> L.tv_log] ? __ldcs(blk + (size_t)S * CB + b) : make_float2(0.f, 0.f);
    };
    // keep the N crop rows, compacted into rows 0..N-1 (all reads precede these writes)
    auto store = [&](int b, int S, float2 v) {
        if (in_crop(S, half, Np)) blk[(size_t)grid_to_crop(S, half, Np) * CB + b] = v;
    };
    plane_fft<NP, kPerCta, CROP ? fftst::PRUNE_OUT : 0>(sbuf, F, tw, true, threadIdx.x, kThreads, load, store);
}

// -- TMA row copies and mbarriers ----------------------------------------------

__device__ __forceinline__ unsigned smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
    unsigned done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}
// Wait for the phase of the given parity to complete, giving up after
// `polls` polls (kWaitPolls: a few hundred milliseconds): false if it did not
// complete.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity, int polls = kWaitPolls) {
    for (int i = 0; i < polls; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        __nanosleep(64);
    }
    return false;
}
// Box of an image row: {8 floats, 1 row, min(256, N'/4) column blocks, 1 plane}
// of the stack's row map.
__device__ __forceinline__ void tma_row_box(float2 *dst, const CUtensorMap *map, int row, int block, int plane,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(0), "r"(row), "r"(block), "r"(plane), "r"(smem_addr(bar))
        : "memory");
}

// Shared-memory layout of the compile-time inv_rows: two 128-byte aligned row
// buffers (TMA destinations), z row, compensated sums, two mbarriers.
template <int NP>
struct RowsSmem {
    static constexpr size_t buf = (fftst::Layout<NP>::stride * sizeof(float2) + 127) / 128 * 128;
    static size_t bytes(int N) { return 128 + 2 * buf + (size_t)N * (sizeof(float2) + sizeof(float4)) + 16; }
};

// One CTA owns image row ii and sums the chunk's planes into a compensated
// accumulator in shared memory; the last FFT stage screens and accumulates.
//
// Compile-time plans double-buffer the row with TMA: as plane p starts, warp
// 0 copies plane p + 1's row into the other buffer in boxes of up to 256
// column blocks (8 KB), all completing on that buffer's mbarrier.  Strips no
// footprint touched hold stale data; the first FFT stage masks them to zero.
// Every wait is bounded; a CTA that gives up counts the failure in *timeouts,
// waits (bounded) for the copy in flight and returns.
template <int NP, bool CROP>
__global__ void __launch_bounds__(kRowThreads, 2)
inv_rows_kernel(Launch L, FftPlan F, const float2 *__restrict__ tw, const float2 *__restrict__ stack,
                const __grid_constant__ CUtensorMap row_map, const uint8_t *__restrict__ col_occ, int plane0,
                int planes, const float2 *__restrict__ zsplit, const float *__restrict__ corr,
                float4 *__restrict__ acc, int first, int last, float2 *__restrict__ dirty,
                unsigned long long *__restrict__ timeouts, int wait_polls) {
    extern __shared__ __align__(16) float2 sbuf[];
    const int Np = L.Np, N = L.N, half = N / 2;
    const int ii = blockIdx.x;
    const int tid = threadIdx.x;
    const size_t pix0 = (size_t)ii * N;
    const int nvalid = min(planes, L.Nw - plane0);
    if constexpr (NP >= 512) {
        using Sm = RowsSmem<NP>;
        constexpr int R0 = fftst::Radices<NP>::r0, nb = NP / R0;
        constexpr int kBoxBlocks = NP / CB < 256 ? NP / CB : 256, kRowBoxes = NP / CB / kBoxBlocks;
        // 128-byte aligned start, by pointer arithmetic on sbuf so that every
        // access below stays a shared-memory access
        float2 *base = sbuf + ((128u - (smem_addr(sbuf) & 127u)) & 127u) / sizeof(float2);
        constexpr int kBuf = (int)(Sm::buf / sizeof(float2));
        auto row_buf = [&](int p) { return base + (p & 1) * kBuf; };
        float2 *zrow = base + 2 * kBuf;                                   // N
        float4 *srow = reinterpret_cast<float4 *>(zrow + N);              // N: (sum re, sum im, comp re, comp im)
        uint64_t *bar = reinterpret_cast<uint64_t *>(srow + N);           // 2
        const int warp = tid >> 5, lane = tid & 31;
        // warp 0: copy plane p's row ii into buffer p & 1, kRowBoxes boxes of
        // kBoxBlocks column blocks (strips no footprint touched come along and
        // are masked to zero by the first stage)
        auto issue = [&](int p) {
            fence_proxy_async();             // the buffer's last generic reads precede these writes
            if (lane == 0) mbar_arrive_expect_tx(&bar[p & 1], (unsigned)(NP * sizeof(float2)));
            __syncwarp();
            if (lane < kRowBoxes)
                tma_row_box(row_buf(p) + lane * kBoxBlocks * CB, &row_map, ii, lane * kBoxBlocks, p, &bar[p & 1]);
        };
        if (tid == 0) {
            mbar_init(&bar[0], 1);
            mbar_init(&bar[1], 1);
            mbar_init_fence();
        }
        for (int jj = tid; jj < N; jj += kRowThreads) {
            zrow[jj] = zsplit[pix0 + jj];
            srow[jj] = first ? make_float4(0.f, 0.f, 0.f, 0.f) : acc[pix0 + jj];
        }
        using Rd = fftst::Radices<NP>;
        const fftst::StageTw s2 = fftst::stage_twiddles<NP, Rd::r1, Rd::r0>(tw, true, tid);
        const fftst::StageTw s3 = fftst::stage_twiddles<NP, Rd::r2, Rd::r0 * Rd::r1>(tw, true, tid);
        __syncthreads();
        if (warp == 0 && nvalid > 0) issue(0);
        uint32_t live = 0;                   // strips of this thread's first-stage inputs, one t-tile
        int live_tt = -1;
        for (int p = 0; p < nvalid; ++p) {
            const float t = (float)(plane0 + p + L.t_lo);
            const int tt = (plane0 + p) / TT;
            if (tt != live_tt) {             // threads past nb own no first-stage butterfly
                live = 0;
                if (tid < nb) {
#pragma unroll
                    for (int m = 0; m < R0; ++m)
                        live |= (uint32_t)(__ldg(col_occ + tt * L.ntu + (m * nb + tid) / TU) != 0) << m;
                }
                live_tt = tt;
            }
            const bool ok = mbar_wait(&bar[p & 1], (p >> 1) & 1, wait_polls);
            if (__syncthreads_or(!ok)) {     // uniform: give up on this row
                if (tid == 0) {
                    atomicAdd(timeouts, 1ull);
                    mbar_wait(&bar[p & 1], (p >> 1) & 1);   // drain the copy in flight (full limit)
                }
                __syncthreads();
                return;
            }
            // every thread is past plane p - 1, so its buffer is free for plane p + 1
            if (warp == 0 && p + 1 < nvalid) issue(p + 1);
            auto between = [] {};
            auto store = [&](int, int J, float2 v) {
                if (!in_crop(J, half, Np)) return;
                const int jj = grid_to_crop(J, half, Np);
                float sn, cs;
                phase_tz(t, zrow[jj], &sn, &cs);
                float4 a = srow[jj];
                kahan_add(a.x, a.z, v.x * cs - v.y * sn);
                kahan_add(a.y, a.w, v.x * sn + v.y * cs);
                srow[jj] = a;
            };
            fft_static_inplace<NP, CROP ? fftst::PRUNE_OUT : 0>(row_buf(p), tw, true, tid, kRowThreads, between, store,
                                                                  s2, s3, live);
        }
        __syncthreads();
        for (int jj = tid; jj < N; jj += kRowThreads) {
            const float4 a = srow[jj];
            if (last) {
                const float h = corr[pix0 + jj];
                dirty[pix0 + jj] = make_float2(h * (a.x - a.z), L.fold ? 0.f : h * (a.y - a.w));
            } else {
                acc[pix0 + jj] = a;
            }
        }
    } else {
        // the z row stays in shared memory where two CTAs per SM still fit, else
        // the screen reads z from global memory
        const bool keep_z = rows_keep_z(F, N);
        float2 *zrow = sbuf + F.stride;                          // N if keep_z (F.stride is even: 16-byte aligned)
        float4 *srow = reinterpret_cast<float4 *>(zrow + (keep_z ? N : 0));   // N: (sum re, sum im, comp re, comp im)
        uint8_t *occ = reinterpret_cast<uint8_t *>(srow + N);    // ntu: strips of the current t-tile
        const float2 *zsrc = keep_z ? zrow : zsplit + pix0;
        int occ_tt = -1;
        for (int jj = tid; jj < N; jj += kRowThreads) {
            if (keep_z) zrow[jj] = zsplit[pix0 + jj];
            srow[jj] = first ? make_float4(0.f, 0.f, 0.f, 0.f) : acc[pix0 + jj];
        }
        __syncthreads();
        for (int p = 0; p < nvalid; ++p) {
            const float2 *plane = stack + (size_t)p * Np * Np;
            const float t = (float)(plane0 + p + L.t_lo);
            const int tt = (plane0 + p) / TT;
            if (tt != occ_tt) {                  // uniform across the CTA; the previous plane ended with a barrier
                for (int i = tid; i < L.ntu; i += kRowThreads) occ[i] = col_occ[tt * L.ntu + i];
                __syncthreads();
                occ_tt = tt;
            }
            // column strips no footprint touched were never transformed: they are zero
            auto load = [&](int, int R) -> float2 {
                return occ[R / TU] ? __ldcs(plane + tiled_index(ii, R, Np)) : make_float2(0.f, 0.f);
            };
            auto store = [&](int, int J, float2 v) {
                if (!in_crop(J, half, Np)) return;
                const int jj = grid_to_crop(J, half, Np);
                float sn, cs;
                phase_tz(t, zsrc[jj], &sn, &cs);
                float4 a = srow[jj];
                kahan_add(a.x, a.z, v.x * cs - v.y * sn);
                kahan_add(a.y, a.w, v.x * sn + v.y * cs);
                srow[jj] = a;
            };
            plane_fft<NP, 1>(sbuf, F, tw, true, tid, kRowThreads, load, store);
            __syncthreads();
        }
        for (int jj = tid; jj < N; jj += kRowThreads) {
            const float4 a = srow[jj];
            if (last) {
                const float h = corr[pix0 + jj];
                dirty[pix0 + jj] = make_float2(h * (a.x - a.z), L.fold ? 0.f : h * (a.y - a.w));
            } else {
                acc[pix0 + jj] = a;
            }
        }
    }
}

// transform buffers + one occupancy byte per strip (at most N'/16 or N'/32 of them)
inline size_t smem2(const FftPlan &F) { return (size_t)kPerCta * F.stride * sizeof(float2) + F.n / TU + 16; }
inline size_t smem_fwd_rows(const FftPlan &F, int N, bool step) {
    return (size_t)F.stride * sizeof(float2) + (size_t)N * (step ? 4 : 2) * sizeof(float2) + F.n / TU + 16;
}
// fwd_rows steps its screen where the two extra rows still leave room for two
// CTAs per SM
inline bool fwd_rows_step(const FftPlan &F, int N) { return smem_fwd_rows(F, N, true) <= kTwoCtaSmem; }
// CTAs per image row in fwd_rows (each takes an equal share of the planes):
// enough rows x groups for about 32 CTAs per SM over the launch, so the SMs
// that finish first in the last round idle for a short CTA, not a long one
inline int row_groups(int N, int planes, int sms) {
    const int want = (32 * sms + N - 1) / N;
    return want < 1 ? 1 : (want > planes ? (planes > 0 ? planes : 1) : want);
}
inline size_t smem_rows(const FftPlan &F, int N) {
    return (size_t)F.stride * sizeof(float2) + (size_t)N * ((rows_keep_z(F, N) ? sizeof(float2) : 0) + sizeof(float4)) +
           F.n / TU + 16;
}
// inv_rows: compile-time plans keep two aligned row buffers and two mbarriers
template <int NP>
inline size_t smem_inv_rows(const FftPlan &F, int N) {
    if constexpr (NP >= 512)
        return RowsSmem<NP>::bytes(N);
    else
        return smem_rows(F, N);
}

// Raise a kernel's dynamic shared-memory limit to the device's opt-in maximum
// (after checking that this plan's need fits): kernels are shared by every
// plan, so a limit set to one plan's need could be too low for another's.
template <typename K>
cudaError_t allow_smem(K kernel, size_t bytes) {
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    if (bytes > (size_t)optin) return cudaErrorInvalidValue;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
}

// The stack as a 4-D FP32 tensor for TMA row copies: {8 floats of a column
// block's row, N' rows, N'/4 blocks, P planes}, boxes of min(256, N'/4) blocks of one row.
cudaError_t row_tensor_map(const ws_plan_s *p, CUtensorMap *map);

// Launchers of one FFT variant.
template <int NP>
struct Transforms {
    static cudaError_t setup(const FftPlan &F, int N) {
        cudaError_t e;
        const bool step = fwd_rows_step(F, N);
        if ((e = allow_smem(fwd_rows_kernel<NP, false, false>, smem_fwd_rows(F, N, false))) != cudaSuccess) return e;
        if ((e = allow_smem(fwd_rows_kernel<NP, false, true>, smem_fwd_rows(F, N, false))) != cudaSuccess) return e;
        if (step && (e = allow_smem(fwd_rows_kernel<NP, true, false>, smem_fwd_rows(F, N, true))) != cudaSuccess)
            return e;
        if (step && (e = allow_smem(fwd_rows_kernel<NP, true, true>, smem_fwd_rows(F, N, true))) != cudaSuccess)
            return e;
        if ((e = allow_smem(fwd_cols_kernel<NP, false>, smem2(F))) != cudaSuccess) return e;
        if ((e = allow_smem(fwd_cols_kernel<NP, true>, smem2(F))) != cudaSuccess) return e;
        if ((e = allow_smem(inv_cols_kernel<NP, false>, smem2(F))) != cudaSuccess) return e;
        if ((e = allow_smem(inv_cols_kernel<NP, true>, smem2(F))) != cudaSuccess) return e;
        if ((e = allow_smem(inv_rows_kernel<NP, false>, smem_inv_rows<NP>(F, N))) != cudaSuccess) return e;
        return allow_smem(inv_rows_kernel<NP, true>, smem_inv_rows<NP>(F, N));
    }
    static cudaError_t fwd_rows(const ws_plan_s *p, int chunk, int planes, cudaStream_t s) {
        const bool step = fwd_rows_step(p->fft, p->L.N), crop = crop_half<NP>(p->L);
        const dim3 grid(p->L.N, row_groups(p->L.N, planes, p->sms));
        const size_t smem = smem_fwd_rows(p->fft, p->L.N, step);
        auto go = [&](auto kernel) {
            kernel<<<grid, kRowThreads, smem, s>>>(p->L, p->fft, p->d_tw, p->d_img, p->d_zsplit, p->d_col_occ,
                                                   chunk * p->P, planes, p->d_stack);
        };
        if (step)
            crop ? go(fwd_rows_kernel<NP, true, true>) : go(fwd_rows_kernel<NP, true, false>);
        else
            crop ? go(fwd_rows_kernel<NP, false, true>) : go(fwd_rows_kernel<NP, false, false>);
        return cudaGetLastError();
    }
    static cudaError_t fwd_cols(const ws_plan_s *p, int chunk, int planes, cudaStream_t s) {
        const dim3 grid(p->L.Np / kPerCta, planes);
        if (crop_half<NP>(p->L))
            fwd_cols_kernel<NP, true><<<grid, kThreads, smem2(p->fft), s>>>(p->L, p->fft, p->d_tw, p->d_tile_occ,
                                                                         p->d_col_occ, chunk * p->P, p->d_stack);
        else
            fwd_cols_kernel<NP, false><<<grid, kThreads, smem2(p->fft), s>>>(p->L, p->fft, p->d_tw, p->d_tile_occ,
                                                                          p->d_col_occ, chunk * p->P, p->d_stack);
        return cudaGetLastError();
    }
    static cudaError_t inv_cols(const ws_plan_s *p, int chunk, int planes, cudaStream_t s) {
        const dim3 grid(p->L.Np / kPerCta, planes);
        if (crop_half<NP>(p->L))
            inv_cols_kernel<NP, true><<<grid, kThreads, smem2(p->fft), s>>>(p->L, p->fft, p->d_tw, p->d_tile_occ,
                                                                         p->d_col_occ, chunk * p->P, p->d_stack);
        else
            inv_cols_kernel<NP, false><<<grid, kThreads, smem2(p->fft), s>>>(p->L, p->fft, p->d_tw, p->d_tile_occ,
                                                                          p->d_col_occ, chunk * p->P, p->d_stack);
        return cudaGetLastError();
    }
    static cudaError_t inv_rows(const ws_plan_s *p, int chunk, int planes, bool first, bool last, float2 *dirty,
                                cudaStream_t s) {
        CUtensorMap map{};
        if constexpr (NP >= 512) {
            const cudaError_t e = row_tensor_map(p, &map);
            if (e != cudaSuccess) return e;
        }
        auto go = [&](auto kernel) {
            kernel<<<p->L.N, kRowThreads, smem_inv_rows<NP>(p->fft, p->L.N), s>>>(
                p->L, p->fft, p->d_tw, p->d_stack, map, p->d_col_occ, chunk * p->P, planes, p->d_zsplit, p->d_corr,
                p->d_acc, first ? 1 : 0, last ? 1 : 0, dirty, p->d_drop + 2, p->wait_polls);
        };
        crop_half<NP>(p->L) ? go(inv_rows_kernel<NP, true>) : go(inv_rows_kernel<NP, false>);
        return cudaGetLastError();
    }
};

// Entry points of one variant, exported by the translation unit that
// instantiates it (so every kernel is compiled exactly once).
struct Ops {
    cudaError_t (*setup)(const FftPlan &, int);
    cudaError_t (*fwd_rows)(const ws_plan_s *, int, int, cudaStream_t);
    cudaError_t (*fwd_cols)(const ws_plan_s *, int, int, cudaStream_t);
    cudaError_t (*inv_cols)(const ws_plan_s *, int, int, cudaStream_t);
    cudaError_t (*inv_rows)(const ws_plan_s *, int, int, bool, bool, float2 *, cudaStream_t);
};

template <int NP>
constexpr Ops ops_of() {
    return Ops{&Transforms<NP>::setup, &Transforms<NP>::fwd_rows, &Transforms<NP>::fwd_cols,
               &Transforms<NP>::inv_cols, &Transforms<NP>::inv_rows};
}

const Ops &ops_runtime_pow2();
const Ops &ops_runtime_mixed();
const Ops &ops_512();
const Ops &ops_1024();
const Ops &ops_2048();
const Ops &ops_4096();

}  // namespace tf
}  // namespace ws
