// CUDA kernels of the improved W-stacking hot path (sm_103a).
//
// Gridding (Algorithm 5):   prep -> bin -> per plane chunk: grid3d -> inv_cols -> inv_rows
//                           (transforms.cu: inverse DFTs, crop, x exp(2 pi i t z), sum over t,
//                           x h_x h_y h_z)
// Degridding (Algorithm 6): prep -> bin -> correct_image (x h_x h_y h_z) -> per plane chunk:
//                           fwd_rows -> fwd_cols (transforms.cu: x exp(-2 pi i t z), zero pad,
//                           forward DFTs) -> degrid3d (3-D correlation with C_x C_y C_z,
//                           x exp(-2 pi i w (n0-1)))
//
// Grid indices: row s (v direction) and column r (u direction) of a plane are
// stored modulo N'.  Because exp(2 pi i r j / N') is N'-periodic in r, a tap
// that runs past the grid edge wraps onto the opposite edge and the inverse
// DFT of the wrapped grid is exactly the sum over all integers r of Eq.
// gridded-dirty-map; the centred crop |x| < x0 is then rows/columns
// [N'-N/2, N') and [0, N/2).  Planes use the column-block layout of common.cuh.
#include <math.h>

#include <algorithm>
#include <atomic>

#include "common.cuh"
#include "ws_internal.hpp"

namespace ws {
namespace {

// An integer-valued double (|x| < 1e15) modulo n in [0, n): integer arithmetic,
// with the division only for the rare points more than a grid away.
__device__ __forceinline__ int wrap_index(double x, int n) {
    long long i = (long long)x;
    if (i < -n || i >= 2LL * n) i %= n;
    if (i < 0) i += n;
    if (i >= n) i -= n;
    return (int)i;
}

// ---------------------------------------------------------------------------
// Pre-processing (Section 3.3 tap rule, Section 5.2 scaling and pre-phase)
// ---------------------------------------------------------------------------
__global__ void prep_kernel(Launch L, const double *__restrict__ uvw, const float2 *__restrict__ vis,
                            int64_t M, int grid, VisRec *__restrict__ rec,
                            unsigned long long *__restrict__ drop) {
    // a grid-stride loop: the plan's constants in FP64 (W / 2, offsets) are formed
    // once per thread, not once per visibility (FP64 arithmetic is slow here)
    const int W = L.W;
    const double half_w = 0.5 * W, half_wm1 = 0.5 * (W - 1), t_off = (double)(W - 1) + L.t_lo;
    const double t_max = (double)(L.Nw - W);
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < M; k += (int64_t)gridDim.x * blockDim.x) {
        double u = uvw[3 * k], v = uvw[3 * k + 1], w = uvw[3 * k + 2];
        // Section 5.4, real sky: V(u, v, w) = conj V(-u, -v, -w), so w < 0 is gridded at
        // -(u, v, w) with the conjugate value (and degridded there, conjugated afterwards)
        const bool folded = L.fold && w < 0.0;
        if (folded) {
            u = -u;
            v = -v;
            w = -w;
        }
        VisRec r;
        r.r0 = r.s0 = 0;
        r.t0 = -1;
        r.nux = r.nuy = r.nuz = 0.f;
        r.vre = r.vim = 0.f;
        const double up = u * L.uv_scale, vp = v * L.uv_scale, wp = w * L.nscale;
        if (!(fabs(up) < 1e15) || !(fabs(vp) < 1e15)) {   // also catches NaN
            atomicAdd(&drop[0], 1ull);
            rec[k] = r;
            continue;
        }
        const double ft = floor(wp + half_w);
        const double t0 = ft - t_off;
        if (!(t0 >= 0.0 && t0 <= t_max)) {                 // NaN w fails too
            atomicAdd(&drop[1], 1ull);
            rec[k] = r;
            continue;
        }
        const double fu = floor(up + half_w), fv = floor(vp + half_w);
        const double ru = fu - (W - 1), rv = fv - (W - 1);
        r.r0 = wrap_index(ru, L.Np);
        r.s0 = wrap_index(rv, L.Np);
        r.t0 = (int)t0;
        r.nux = (float)(up + half_wm1 - fu);
        r.nuy = (float)(vp + half_wm1 - fv);
        r.nuz = (float)(wp + half_wm1 - ft);
        // pre-phase exp(+2 pi i w (n0 - 1)), argument reduced in FP64
        double turns = w * L.n0m1;
        turns -= rint(turns);
        float s, c;
        sincospif(2.0f * (float)turns, &s, &c);
        if (grid) {
            float2 V = vis[k];
            if (folded) V.y = -V.y;
            r.vre = V.x * c - V.y * s;
            r.vim = V.x * s + V.y * c;
        } else {
            r.vre = c;          // conjugate phase applied after degridding
            r.vim = -s;
        }
        rec[k] = r;
    }
}

// Gridding records of a bound visibility set: the set's records hold the
// degridding factor exp(-2 pi i w (n0 - 1)); gridding needs V exp(+2 pi i w
// (n0 - 1)), with V conjugated where a real-sky plan folded w < 0.
__global__ void bound_grid_records_kernel(Launch L, const double *__restrict__ uvw, const float2 *__restrict__ vis,
                                          int64_t M, const VisRec *__restrict__ brec, VisRec *__restrict__ rec) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= M) return;
    VisRec r = brec[k];
    float2 V = vis[k];
    if (L.fold && uvw[3 * k + 2] < 0.0) V.y = -V.y;
    const float c = r.vre, s = -r.vim;      // exp(+2 pi i w (n0 - 1)) = (c, s)
    r.vre = V.x * c - V.y * s;
    r.vim = V.x * s + V.y * c;
    rec[k] = r;
}

// ---------------------------------------------------------------------------
// Binning: counting sort of (visibility, bin) pairs by bin id
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t tile_id(const Launch &L, int tt, int tv, int tu) {
    return ((uint32_t)tt * L.ntv + tv) * L.ntu + tu;
}

// Gridding bin: a tile column (tv, tu) and the t-tile of the first tap.  A
// column's bins are contiguous, in t order.
__device__ __forceinline__ uint32_t column_bin(const Launch &L, int tv, int tu, int tt) {
    return ((uint32_t)tv * L.ntu + tu) * L.ntt + tt;
}

// The tile columns a footprint's W x W taps in (u, v) touch: 1 or 2 along each axis.
__device__ __forceinline__ void footprint_columns(const Launch &L, const VisRec &r, int *tu, int &nu_, int *tv,
                                                  int &nv_) {
    tu[0] = r.r0 / TU;
    tu[1] = wrap_add(r.r0, L.W - 1, L.Np) / TU;
    nu_ = tu[1] != tu[0] ? 2 : 1;
    tv[0] = r.s0 >> L.tv_log;
    tv[1] = wrap_add(r.s0, L.W - 1, L.Np) >> L.tv_log;
    nv_ = tv[1] != tv[0] ? 2 : 1;
}

// Bins of a record: its tile columns with the first tap's t-tile (grid), or
// the tile of its first tap (degrid).
template <bool GRID>
__device__ __forceinline__ int record_keys(const Launch &L, const VisRec &r, uint32_t *keys) {
    if (r.t0 < 0) return 0;
    if (!GRID) {
        keys[0] = tile_id(L, r.t0 / TT, r.s0 >> L.tv_log, r.r0 / TU);
        return 1;
    }
    int tu[2], tv[2], nu_, nv_;
    footprint_columns(L, r, tu, nu_, tv, nv_);
    int n = 0;
    for (int b = 0; b < nv_; ++b)
        for (int a = 0; a < nu_; ++a) keys[n++] = column_bin(L, tv[b], tu[a], r.t0 / TT);
    return n;
}

constexpr int kMaxKeys = 2 * 2;

// Counts the record's bins and marks the stack tiles its footprint touches.
// Every other cell of the stack is zero when gridding and never read when
// degridding, so the plane kernels skip it.
template <bool GRID>
__global__ void count_kernel(Launch L, const VisRec *__restrict__ rec, int64_t M, uint32_t *__restrict__ counts,
                             uint8_t *__restrict__ tile_occ) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= M) return;
    const VisRec r = rec[k];
    uint32_t keys[kMaxKeys];
    const int n = record_keys<GRID>(L, r, keys);
    for (int i = 0; i < n; ++i) atomicAdd(&counts[keys[i]], 1u);
    if (n == 0) return;
    int tu[2], tv[2], nu_, nv_;
    footprint_columns(L, r, tu, nu_, tv, nv_);
    const int tt1 = (r.t0 + L.W - 1) / TT;
    for (int tt = r.t0 / TT; tt <= tt1; ++tt)
        for (int b = 0; b < nv_; ++b)
            for (int a = 0; a < nu_; ++a) tile_occ[tile_id(L, tt, tv[b], tu[a])] = 1;   // stores only: no waits
}

template <bool GRID>
__global__ void scatter_kernel(Launch L, const VisRec *__restrict__ rec, int64_t M,
                               const uint32_t *__restrict__ offsets, uint32_t *__restrict__ fill,
                               uint32_t *__restrict__ list) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= M) return;
    uint32_t keys[kMaxKeys];
    int n = record_keys<GRID>(L, rec[k], keys);
    for (int i = 0; i < n; ++i) list[offsets[keys[i]] + atomicAdd(&fill[keys[i]], 1u)] = (uint32_t)k;
}

// Occupancy of the (t-tile, u-tile) strips of N' rows: any tile of the strip touched.
__global__ void strip_occ_kernel(Launch L, const uint8_t *__restrict__ tile_occ, int64_t ntiles,
                                 uint8_t *__restrict__ col_occ) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntiles || !tile_occ[t]) return;
    const int64_t c = (t / ((int64_t)L.ntu * L.ntv)) * L.ntu + t % L.ntu;
    if (!col_occ[c]) col_occ[c] = 1;
}

// Statistics only (WS_FLAG_TIMING): occupied tiles and occupied (t-tile,
// u-strip) strips of one t-tile per CTA.
__global__ void occ_count_kernel(Launch L, const uint8_t *__restrict__ tile_occ, const uint8_t *__restrict__ col_occ,
                                 uint32_t *__restrict__ counts) {
    const int tt = blockIdx.x;
    const int64_t per = (int64_t)L.ntu * L.ntv;
    uint32_t tiles = 0, strips = 0;
    for (int64_t i = threadIdx.x; i < per; i += blockDim.x) tiles += tile_occ[tt * per + i];
    for (int i = threadIdx.x; i < L.ntu; i += blockDim.x) strips += col_occ[(int64_t)tt * L.ntu + i];
    for (int o = 16; o > 0; o >>= 1) {
        tiles += __shfl_xor_sync(0xffffffffu, tiles, o);
        strips += __shfl_xor_sync(0xffffffffu, strips, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&counts[2 * tt], tiles);
        atomicAdd(&counts[2 * tt + 1], strips);
    }
}

// Exclusive scan of n uint32 (n <= 4096 * 4096): per-block scan of 4096
// elements, scan of the block sums in one block, then add back.
constexpr int kScanThreads = 1024;
constexpr int kScanPerBlock = 4 * kScanThreads;

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *total) {
    __shared__ uint32_t warp_sums[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[wid] = x;
    __syncthreads();
    if (wid == 0) {
        uint32_t s = warp_sums[lane];
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        warp_sums[lane] = s;
    }
    __syncthreads();
    uint32_t before = (wid ? warp_sums[wid - 1] : 0u) + x - v;
    *total = warp_sums[31];
    __syncthreads();
    return before;
}

__global__ void __launch_bounds__(kScanThreads) scan_block_kernel(const uint32_t *__restrict__ in,
                                                                  uint32_t *__restrict__ out,
                                                                  uint32_t *__restrict__ sums, int64_t n) {
    const int64_t base = (int64_t)blockIdx.x * kScanPerBlock + 4 * threadIdx.x;
    uint32_t a[4];
    for (int i = 0; i < 4; ++i) a[i] = base + i < n ? in[base + i] : 0u;
    uint32_t local = a[0] + a[1] + a[2] + a[3], total;
    uint32_t run = block_exclusive_scan(local, &total);
    for (int i = 0; i < 4; ++i) {
        if (base + i < n) out[base + i] = run;
        run += a[i];
    }
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanThreads) scan_sums_kernel(uint32_t *sums, int nb) {
    const int base = 4 * threadIdx.x;
    uint32_t a[4];
    for (int i = 0; i < 4; ++i) a[i] = base + i < nb ? sums[base + i] : 0u;
    uint32_t total;
    uint32_t run = block_exclusive_scan(a[0] + a[1] + a[2] + a[3], &total);
    for (int i = 0; i < 4; ++i) {
        if (base + i < nb) sums[base + i] = run;
        run += a[i];
    }
}

__global__ void scan_add_kernel(uint32_t *__restrict__ out, const uint32_t *__restrict__ sums, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += sums[i / kScanPerBlock];
}

// ---------------------------------------------------------------------------
// Gridding: Algorithm 5 steps 2 and 3a (Eq. gridded_vis).  One CTA owns one
// tile column -- TU grid columns x tv grid rows through every w-plane of the
// plane chunk -- and walks the column's bins in t order.  A bin holds the
// visibilities whose first tap lies in one t-tile, so their footprints reach
// at most TT + W - 1 consecutive planes: the CTA accumulates in a
// shared-memory ring of that many planes (plane t at ring slot t mod (TT + W
// - 1)), and before it adds a bin it writes out the planes that bin can no
// longer reach -- each occupied tile of the stack exactly once -- and clears
// their slots.  A visibility is one entry in each tile column its W x W taps
// in (u, v) touch (at most 2 x 2), whatever the planes its W taps in w span.
//
// A bin's entries are split evenly over the CTA's warps; a warp takes its
// share in chunks of up to kChunk entries, in three steps:
//   1. lane j prepares entry j of the chunk: its record, the part of its
//      W x W x W footprint that lies in the column and in the plane chunk
//      (first tap and tap count along u, v and w) and that part's first cell;
//   2. the warp evaluates the chunk's 3W weight polynomials C(r - u'),
//      C(s - v'), C(t - w'), one (entry, slot) pair per lane and round;
//   3. entry after entry, the lanes take the (row, plane) pairs of the part,
//      form C_y C_z V once each, and add C_x C_y C_z V along the part's run of
//      u taps with shared-memory reductions at immediate offsets.
// So the tap rule, the index arithmetic and the polynomials cost once per
// entry, and each tap costs one weight product and one reduction per
// component.
// ---------------------------------------------------------------------------
static_assert(kMaxDeg + 1 <= kCoefStride && kCoefStride % 4 == 0 && kMaxDeg == 16,
              "the Horner steps below read coefficients 0..16 as five float4");
static_assert(kMaxW <= 15, "tap counts and first taps are packed in 4 bits");
static_assert(ring_planes(kMaxW) <= 31, "ring slots are packed in 5 bits");
constexpr int kGeneral = -1;                       // item shape: the part wraps an axis of a small grid

// Dynamic shared memory of grid3d<W, R, DET> (grid_smem_bytes): the ring (re,
// im; FP32 sums, or 64-bit fixed-point sums for the deterministic mode), the
// weight table, and per warp the staged chunk (weights, items, values, nu).
template <int W, int R, bool DET>
struct GridSmem {
    static constexpr int S = 3 * W;                // weight slots per entry: u taps, v taps, w taps
    static constexpr int WX = wx_span(W);          // staged u weights, from the part's first tap
    static constexpr int SP = stage_stride(W);     // entry stride of the staged weights: u, v, w
    static constexpr int ES = DET ? 8 : 4;         // bytes per cell component
    static constexpr int RP = ring_planes(W);      // ring planes
    static constexpr int PS = plane_stride(R);     // cells per ring plane (padded)
    static constexpr size_t re = 0;
    static constexpr size_t im = re + ring_bytes(W, R, DET);
    static constexpr size_t coef = im + ring_bytes(W, R, DET);
    static constexpr size_t wt = coef + (size_t)S * kCoefStride * 4;
    static constexpr size_t item = wt + (size_t)kGridWarps * kChunk * SP * 4;
    static constexpr size_t val = item + (size_t)kGridWarps * kChunk * 16;
    static constexpr size_t nu = val + (size_t)kGridWarps * kChunk * 8;
    static constexpr size_t bytes = nu + (size_t)kGridWarps * kChunk * 16;
    static_assert(bytes == grid_smem_bytes(W, R, DET), "the host's size of the gridding shared memory");
    static_assert(coef % 16 == 0 && wt % 16 == 0 && item % 16 == 0 && nu % 16 == 0, "float4 / int4 alignment");
};

// Taps [a0, a1) of a footprint that land in a tile, at tile-local index a - off.
struct Span {
    int a0, a1, off;
};

// The footprint covers positions first .. first + W - 1 and the tile org ..
// org + T - 1 of a periodic axis of length n >= T: the tile starts d = org -
// first (mod n) past the footprint's start, and if it runs past n it also
// covers the footprint's first d + T - n positions.  Returns 0, 1 or 2 spans
// (two only when n < W + T, a grid of 32 rows).
__device__ __forceinline__ int tile_spans(int org, int first, int n, int W, int T, Span &s0, Span &s1) {
    int d = org - first;
    if (d < 0) d += n;
    const Span inside{d, min(W, d + T), d}, wrapped{0, min(W, d + T - n), d - n};
    const bool has_inside = d < W, has_wrapped = d + T > n;
    s0 = has_inside ? inside : wrapped;
    s1 = wrapped;
    return (int)has_inside + (int)has_wrapped;
}

// Shared-memory FP32 add with no returned value, at a byte offset fixed at compile time.
template <int OFF>
__device__ __forceinline__ void red_shared_at(unsigned addr, float v) {
    asm volatile("red.shared.add.f32 [%0+%1], %2;" ::"r"(addr), "n"(OFF), "f"(v) : "memory");
}

// The deterministic mode's shared-memory add: a contribution v becomes the
// 64-bit integer nearest v 2^scale, and integer sums do not depend on the
// order of their terms.
template <int OFF>
__device__ __forceinline__ void red_shared_fixed_at(unsigned addr, float v, int scale) {
    const unsigned long long q = (unsigned long long)__float2ll_rn(ldexpf(v, scale));
    asm volatile("red.shared.add.u64 [%0+%1], %2;" ::"r"(addr), "n"(OFF), "l"(q) : "memory");
}

// One contribution to a ring cell component at byte address addr + OFF.
template <bool DET, int OFF>
__device__ __forceinline__ void add_cell(unsigned addr, float v, int scale) {
    if constexpr (DET)
        red_shared_fixed_at<OFF>(addr, v, scale);
    else
        red_shared_at<OFF>(addr, v);
}

// Adds (pr, pi) x wx[a] to cells a = 0 .. na - 1 of a ring row (re and im at byte addresses).
template <int W, bool DET, int A = 0>
__device__ __forceinline__ void add_row(unsigned re, unsigned im, const float (&wx)[wx_span(W)], int na, float pr, float pi,
                                        int scale) {
    if constexpr (A < W) {
        if (A < na) {
            constexpr int ES = DET ? 8 : 4;
            add_cell<DET, ES * A>(re, pr * wx[A], scale);
            add_cell<DET, ES * A>(im, pi * wx[A], scale);
            add_row<W, DET, A + 1>(re, im, wx, na, pr, pi, scale);
        }
    }
}

// Index j of 0 .. n-1 taken in the order 0, n-1, 1, n-2, ...: the tile
// columns near the uv origin (both ends of the wrapped axes), which hold the
// most entries, start first and do not trail the launch.
__device__ __forceinline__ int centre_first(int j, int n) { return (j & 1) ? n - 1 - (j >> 1) : (j >> 1); }

// Writes out the ring's slices (t-tiles) s in [from, to), when the ring holds
// planes [from TT, from TT + RP): a slice that the chunk owns and a footprint
// touched (tile_occ) goes to the stack, its planes past the ring's end as
// zeros (no footprint reached them).  With `clear`, each thread zeroes the
// ring cells it has just read, which leaves the slices' ring planes zero for
// the planes that take their slots: every other cell of those planes is zero
// already (a slice no footprint touched, or outside the chunk, received no
// contribution, and padding cells never do).
template <int W, int R, bool DET>
__device__ __forceinline__ void flush_slices(int from, int to, const Launch &L, int tv, int tu, int chunk_tt0,
                                             int chunk_ntt, const uint8_t *__restrict__ tile_occ, int scale,
                                             unsigned char *smem, float2 *__restrict__ stack, bool clear) {
    using Sm = GridSmem<W, R, DET>;
    constexpr int RP = Sm::RP, PS = Sm::PS;
    const int ring_end = from * TT + RP;
    const int last = min(to, from + (RP + TT - 1) / TT);
    const size_t plane = (size_t)L.Np * L.Np;
    for (int sl = max(from, chunk_tt0); sl < min(last, chunk_tt0 + chunk_ntt); ++sl) {
        if (!tile_occ[((size_t)sl * L.ntv + tv) * L.ntu + tu]) continue;
        // pairs of cells, ordered (plane, column block, row, pair) so that each
        // column block's R rows go out as one contiguous run
        for (int i = threadIdx.x; i < TT * R * TU / 2; i += kGridThreads) {
            const int pair = i & 1, lr = (i >> 1) % R, blk = (i / (2 * R)) % (TU / CB), pl = i / (TU * R / 2);
            const int lc = blk * CB + 2 * pair;
            const int t = sl * TT + pl;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (t < ring_end) {
                const int cell = (t % RP) * PS + lr * kRowPad + lc;
                if constexpr (DET) {
                    long long *qre = reinterpret_cast<long long *>(smem + Sm::re);
                    long long *qim = reinterpret_cast<long long *>(smem + Sm::im);
                    v = make_float4(ldexpf(__ll2float_rn(qre[cell]), -scale), ldexpf(__ll2float_rn(qim[cell]), -scale),
                                    ldexpf(__ll2float_rn(qre[cell + 1]), -scale),
                                    ldexpf(__ll2float_rn(qim[cell + 1]), -scale));
                    if (clear) qre[cell] = qim[cell] = qre[cell + 1] = qim[cell + 1] = 0;
                } else {
                    float *sre = reinterpret_cast<float *>(smem + Sm::re);
                    float *sim = reinterpret_cast<float *>(smem + Sm::im);
                    v = make_float4(sre[cell], sim[cell], sre[cell + 1], sim[cell + 1]);
                    if (clear) sre[cell] = sim[cell] = sre[cell + 1] = sim[cell + 1] = 0.f;
                }
            }
            float2 *dst = stack + (size_t)(t - chunk_tt0 * TT) * plane + tiled_index(tv * R + lr, tu * TU + lc, L.Np);
            *reinterpret_cast<float4 *>(dst) = v;
        }
    }
}

// DET: the deterministic mode (WS_FLAG_DETERMINISTIC).  The ring sums in 64-bit
// fixed point with one scale 2^scale for the CTA, chosen so that no sum can
// exceed 2^62: |sum| <= E max|V~| wbound for the column's E entries, wbound
// bounding |C_x C_y C_z|.  The scale depends only on the column's set of
// entries, and integer additions do not depend on their order, so the stack
// -- and the dirty image -- come out bit for bit the same whatever order the
// binning's atomics and the warps' schedule give the entries.
template <int W, int R, bool DET>
__global__ void __launch_bounds__(kGridThreads, grid_ctas_per_sm(W, R, DET))
grid3d_kernel(Launch L, const float *__restrict__ coef, int deg, const VisRec *__restrict__ rec,
              const uint32_t *__restrict__ offsets, const uint32_t *__restrict__ list,
              const uint8_t *__restrict__ tile_occ, int chunk_tt0, int chunk_ntt, float wbound,
              float2 *__restrict__ stack) {
    using Sm = GridSmem<W, R, DET>;
    constexpr int PS = Sm::PS, RP = Sm::RP, ES = Sm::ES, S = Sm::S, SP = Sm::SP, WX = Sm::WX;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ unsigned col_max;                      // DET: max |V~| of the column's entries (float bits)
    const int tu = centre_first(blockIdx.x % L.ntu, L.ntu);
    const int tv = centre_first(blockIdx.x / L.ntu, L.ntv);
    // the bins whose footprints reach the chunk's planes [plo, phi)
    const int k_lo = max(0, chunk_tt0 - (TT + W - 2) / TT), k_hi = chunk_tt0 + chunk_ntt;
    const int plo = chunk_tt0 * TT, phi = plo + chunk_ntt * TT;
    const uint32_t *__restrict__ off = offsets + ((size_t)tv * L.ntu + tu) * L.ntt;
    const uint32_t all_beg = off[k_lo], all_end = off[k_hi];
    if (all_beg == all_end) return;                  // untouched column: the transforms treat it as zero
    float *scoef = reinterpret_cast<float *>(smem + Sm::coef);
    {
        float4 *qre = reinterpret_cast<float4 *>(smem + Sm::re), *qim = reinterpret_cast<float4 *>(smem + Sm::im);
        for (int i = threadIdx.x; i < (int)(ring_bytes(W, R, DET) / 16); i += kGridThreads) {
            qre[i] = make_float4(0.f, 0.f, 0.f, 0.f);
            qim[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
    if constexpr (DET) {
        if (threadIdx.x == 0) col_max = 0u;
        __syncthreads();
        float m = 0.f;
        for (uint32_t e = all_beg + threadIdx.x; e < all_end; e += kGridThreads) {
            const VisRec r = rec[list[e]];
            m = fmaxf(m, fmaxf(fabsf(r.vre), fabsf(r.vim)));
        }
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if ((threadIdx.x & 31) == 0) atomicMax(&col_max, __float_as_uint(m));   // non-negative floats order as integers
    }
    // slot l < 3W is (axis l / W, tap l % W); coef holds the (u, v) table and
    // then the w table, W x (deg + 1) each; coefficients past deg are zero
    for (int i = threadIdx.x; i < S * kCoefStride; i += kGridThreads) {
        const int l = i / kCoefStride, m = i - l * kCoefStride, axis = l / W, tap = l - axis * W;
        const int row = (axis == 2 ? W : 0) + tap;
        scoef[i] = m <= deg ? coef[row * (deg + 1) + m] : 0.f;
    }
    __syncthreads();
    const int Np = L.Np;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int u_org = tu * TU, v_org = tv * R;
    float *wts = reinterpret_cast<float *>(smem + Sm::wt) + warp * kChunk * SP;
    int4 *items = reinterpret_cast<int4 *>(smem + Sm::item) + warp * kChunk;
    float2 *vals = reinterpret_cast<float2 *>(smem + Sm::val) + warp * kChunk;
    float4 *nus = reinterpret_cast<float4 *>(smem + Sm::nu) + warp * kChunk;
    const unsigned re_base = (unsigned)__cvta_generic_to_shared(smem + Sm::re);
    const unsigned im_base = (unsigned)__cvta_generic_to_shared(smem + Sm::im);
    int scale = 0;                                   // DET: sums are kept as integers in units of 2^-scale
    if constexpr (DET) {
        const float bound = (float)(all_end - all_beg) * __uint_as_float(col_max) * wbound;
        if (bound > 0.f) {
            int ex;
            frexpf(bound, &ex);                          // bound < 2^ex
            scale = 62 - ex;
        }
    }
    int cur = -1;                                    // t-tile of the ring's first plane; -1: none yet
    for (int k = k_lo; k < k_hi; ++k) {
        const uint32_t beg = off[k], end = off[k + 1];
        if (beg == end) continue;
        if (cur >= 0) {
            // bin k reaches planes [k TT, k TT + RP): the ring's planes before k TT are final
            __syncthreads();
            flush_slices<W, R, DET>(cur, k, L, tv, tu, chunk_tt0, chunk_ntt, tile_occ, scale, smem, stack, true);
            __syncthreads();
        }
        cur = k;
        // this warp's share of the bin's entries
        const uint32_t E = end - beg;
        const uint32_t per = (E + kGridWarps - 1) / kGridWarps;
        const uint32_t wbeg = beg + min(E, warp * per), wend = beg + min(E, (warp + 1) * per);
        for (uint32_t cbeg = wbeg; cbeg < wend; cbeg += kChunk) {
            const int n = (int)min((uint32_t)kChunk, wend - cbeg);
            // 1. lane j: entry j's part of the footprint inside the column and the chunk's planes
            if (lane < n) {
                const uint32_t kv = list[cbeg + lane];
                const VisRec r = rec[kv];
                Span su[2], sv[2];
                const int nsu = tile_spans(u_org, r.r0, Np, W, TU, su[0], su[1]);
                const int nsv = tile_spans(v_org, r.s0, Np, W, R, sv[0], sv[1]);
                const int c0 = max(0, plo - r.t0), c1 = min(W, phi - r.t0);
                int4 it;
                if (nsu == 1 && nsv == 1) {
                    const int na = su[0].a1 - su[0].a0, nb = sv[0].a1 - sv[0].a0, nc = max(c1 - c0, 0);
                    const int slot = (r.t0 + c0) % RP;      // ring slot of the part's first plane
                    it.x = (sv[0].a0 - sv[0].off) * kRowPad + (su[0].a0 - su[0].off);
                    it.y = na | nb << 4 | nc << 8 | su[0].a0 << 12 | sv[0].a0 << 16 | c0 << 20 | slot << 24;
                    it.z = __float_as_int(1.0f / (float)nb);
                } else {
                    it.x = 0;
                    it.y = kGeneral;
                    it.z = 0;
                }
                it.w = (int)kv;
                items[lane] = it;
                vals[lane] = make_float2(r.vre, r.vim);
                nus[lane] = make_float4(r.nux, r.nuy, r.nuz, 0.f);
            }
            __syncwarp();
            // 2. the chunk's weights: pair q = (entry j, slot l), Horner from nu^16
            //    down; the u weights are kept from the part's first tap a0 on
            for (int q = lane; q < n * S; q += 32) {
                const int j = q / S, l = q - j * S, axis = l / W;
                const float4 nv = nus[j];
                const float nu = axis == 0 ? nv.x : (axis == 1 ? nv.y : nv.z);
                const float4 *c = reinterpret_cast<const float4 *>(scoef + l * kCoefStride);
                float acc = c[4].x;
#pragma unroll
                for (int b = 3; b >= 0; --b) {
                    const float4 c4 = c[b];
                    acc = fmaf(acc, nu, c4.w);
                    acc = fmaf(acc, nu, c4.z);
                    acc = fmaf(acc, nu, c4.y);
                    acc = fmaf(acc, nu, c4.x);
                }
                int pos = WX + l - W;
                if (axis == 0) {
                    const int y = items[j].y;
                    pos = l - (y == kGeneral ? 0 : (y >> 12) & 15);
                }
                if (pos >= 0) wts[j * SP + pos] = acc;
            }
            __syncwarp();
            // 3. add the chunk's entries one after the other
            for (int j = 0; j < n; ++j) {
                const int4 it = items[j];
                const float2 V = vals[j];
                const float *wt = wts + j * SP;
                if (it.y != kGeneral) {
                    const int na = it.y & 15, nb = (it.y >> 4) & 15, nc = (it.y >> 8) & 15;
                    const int b0 = (it.y >> 16) & 15, cw0 = (it.y >> 20) & 15;
                    const int slot0 = (it.y >> 24) & 31;
                    const float inv_nb = __int_as_float(it.z);
                    const int nbc = nb * nc;
                    // the part's u-tap weights (staged from its first tap on; those
                    // past na are not used), all read before the first reduction
                    float wx[WX];
#pragma unroll
                    for (int a4 = 0; a4 < WX / 4; ++a4) {
                        const float4 v = reinterpret_cast<const float4 *>(wt)[a4];
                        wx[4 * a4] = v.x;
                        wx[4 * a4 + 1] = v.y;
                        wx[4 * a4 + 2] = v.z;
                        wx[4 * a4 + 3] = v.w;
                    }
                    for (int q = lane; q < nbc; q += 32) {
                        // q = cc nb + bb, q < 144: (q + 1/2) / nb is at least 1/24 from an integer
                        const int cc = __float2int_rz(((float)q + 0.5f) * inv_nb), bb = q - cc * nb;
                        const float wyz = wt[WX + b0 + bb] * wt[WX + W + cw0 + cc];
                        int slot = slot0 + cc;
                        if (slot >= RP) slot -= RP;
                        const unsigned o = (unsigned)(it.x + slot * PS + bb * kRowPad) * ES;
                        add_row<W, DET>(re_base + o, im_base + o, wx, na, V.x * wyz, V.y * wyz, scale);
                    }
                } else {
                    // the part wraps around an axis (N' < W + R): every span pair, taps one by one
                    const VisRec r = rec[it.w];
                    Span su[2], sv[2];
                    const int nsu = tile_spans(u_org, r.r0, Np, W, TU, su[0], su[1]);
                    const int nsv = tile_spans(v_org, r.s0, Np, W, R, sv[0], sv[1]);
                    const int c0 = max(0, plo - r.t0), c1 = min(W, phi - r.t0);
                    for (int iu = 0; iu < nsu; ++iu)
                        for (int iv = 0; iv < nsv; ++iv) {
                            const int na = su[iu].a1 - su[iu].a0, nb = sv[iv].a1 - sv[iv].a0, nc = c1 - c0;
                            for (int q = lane; q < na * nb * nc; q += 32) {
                                const int a = su[iu].a0 + q % na, b = sv[iv].a0 + (q / na) % nb, c = c0 + q / (na * nb);
                                const float w = wt[a] * wt[WX + b] * wt[WX + W + c];
                                const unsigned o = (unsigned)(((r.t0 + c) % RP) * PS + (b - sv[iv].off) * kRowPad +
                                                              (a - su[iu].off)) *
                                                   ES;
                                add_cell<DET, 0>(re_base + o, V.x * w, scale);
                                add_cell<DET, 0>(im_base + o, V.y * w, scale);
                            }
                        }
                }
            }
            __syncwarp();                              // the chunk's staging is read before the next overwrites it
        }
    }
    __syncthreads();
    flush_slices<W, R, DET>(cur, cur + (RP + TT - 1) / TT, L, tv, tu, chunk_tt0, chunk_ntt, tile_occ, scale, smem,
                            stack, false);
}

// Algorithm 6 step 2: image x h_x h_y h_z.
// A real-sky plan (fold) reads only the real part of the image.
__global__ void correct_image_kernel(int64_t n, const float *__restrict__ corr,
                                     const float2 *__restrict__ image, int fold, float2 *__restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float h = corr[i];
    const float2 f = image[i];
    out[i] = make_float2(h * f.x, fold ? 0.f : h * f.y);
}

// Section 5.4: a visibility with w < 0 was degridded at -(u, v, w); the real
// sky's visibility at (u, v, w) is the conjugate of that.
__global__ void unfold_kernel(const double *__restrict__ uvw, int64_t M, float2 *__restrict__ vis) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= M) return;
    if (uvw[3 * k + 2] < 0.0) vis[k].y = -vis[k].y;
}

// ---------------------------------------------------------------------------
constexpr int kDegridThreads = 256;

// Degridding: Algorithm 6 steps 4-5.  One warp per visibility (visiting them
// in tile order for cache reuse); lanes over the W x W (a, b) columns of the
// footprint (W^2 / 32 rounded up per lane), W planes each.  All of a lane's
// gathers are issued before any is used, so a warp keeps up to 2 W loads in
// flight.  The polynomial table sits in shared memory for the weights.  Each
// chunk adds its planes' share to vis, in chunk order.
template <int W>
__global__ void __launch_bounds__(kDegridThreads, W <= 6 ? 5 : (W <= 8 ? 3 : 1))
degrid3d_kernel(Launch L, const float *__restrict__ coef, int deg, const VisRec *__restrict__ rec,
                const uint32_t *__restrict__ order, const uint32_t *__restrict__ n_order,
                const float2 *__restrict__ stack, int plane0, int planes, float2 *__restrict__ vis) {
    constexpr int kPasses = (W * W + 31) / 32;
    __shared__ float swt[kDegridThreads / 32][3 * W];
    // the (u, v) table, then the w table: 2W rows of kCoefStride coefficients, zero past deg
    __shared__ __align__(16) float scoef[2 * W * kCoefStride];
    for (int i = threadIdx.x; i < 2 * W * kCoefStride; i += kDegridThreads) {
        const int row = i / kCoefStride, m = i - row * kCoefStride;
        scoef[i] = m <= deg ? coef[row * (deg + 1) + m] : 0.f;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t n = (int64_t)*n_order;                   // entries of the sorted list (dropped ones excluded)
    const int64_t nwarps = (int64_t)gridDim.x * (kDegridThreads / 32);
    const int Np = L.Np;
    const size_t plane = (size_t)Np * Np;
    float *wt = swt[warp];
    // a grid of resident CTAs: each warp takes every nwarps-th visibility of the
    // tile-sorted list, so the warps in flight still gather from neighbouring cells
    for (int64_t widx = ((int64_t)blockIdx.x * kDegridThreads + threadIdx.x) >> 5; widx < n; widx += nwarps) {
        const uint32_t k = order[widx];
        const VisRec r = rec[k];
        if (r.t0 < 0) continue;
        const int c_lo = max(0, plane0 - r.t0);
        const int c_hi = min(W - 1, plane0 + planes - 1 - r.t0);
        if (c_lo > c_hi) continue;
        __syncwarp();                                       // the previous visibility's weights are read
        for (int l = lane; l < 3 * W; l += 32) {             // 3W > 32 for W >= 11
            const int axis = l / W, i = l - axis * W;
            const float nu = axis == 0 ? r.nux : (axis == 1 ? r.nuy : r.nuz);
            const float4 *c = reinterpret_cast<const float4 *>(scoef + ((axis == 2 ? W : 0) + i) * kCoefStride);
            float acc = c[4].x;                              // Horner from nu^16 down
#pragma unroll
            for (int b = 3; b >= 0; --b) {
                const float4 c4 = c[b];
                acc = fmaf(acc, nu, c4.w);
                acc = fmaf(acc, nu, c4.z);
                acc = fmaf(acc, nu, c4.y);
                acc = fmaf(acc, nu, c4.x);
            }
            wt[l] = acc;
        }
        __syncwarp();
        const int64_t t_rel = (int64_t)r.t0 - plane0;       // stack plane of tap c is t_rel + c
        const bool all_planes = c_lo == 0 && c_hi == W - 1; // uniform: the whole footprint is in the chunk
        float2 f[kPasses][W];
#pragma unroll
        for (int ps = 0; ps < kPasses; ++ps) {
            const int pair = lane + 32 * ps;
            const int a = pair % W, b = pair / W;
            const bool live = pair < W * W;
            const float2 *cell = stack + tiled_index(wrap_add(r.s0, live ? b : 0, Np), wrap_add(r.r0, a, Np), Np) +
                                 (size_t)t_rel * plane;
            if (all_planes) {
#pragma unroll
                for (int c = 0; c < W; ++c) f[ps][c] = live ? __ldg(cell + (size_t)c * plane) : make_float2(0.f, 0.f);
            } else {
#pragma unroll
                for (int c = 0; c < W; ++c) {
                    f[ps][c] = make_float2(0.f, 0.f);
                    if (live && c >= c_lo && c <= c_hi) f[ps][c] = __ldg(cell + (size_t)c * plane);
                }
            }
        }
        float ar = 0.f, ai = 0.f;
#pragma unroll
        for (int ps = 0; ps < kPasses; ++ps) {
            const int pair = lane + 32 * ps;
            if (pair >= W * W) break;
            const int a = pair % W, b = pair / W;
            float sr = 0.f, si = 0.f;
#pragma unroll
            for (int c = 0; c < W; ++c) {
                const float wc = wt[2 * W + c];
                sr = fmaf(wc, f[ps][c].x, sr);
                si = fmaf(wc, f[ps][c].y, si);
            }
            const float wab = wt[a] * wt[W + b];
            ar = fmaf(wab, sr, ar);
            ai = fmaf(wab, si, ai);
        }
        for (int o = 16; o > 0; o >>= 1) {
            ar += __shfl_xor_sync(0xffffffffu, ar, o);
            ai += __shfl_xor_sync(0xffffffffu, ai, o);
        }
        if (lane == 0) {
            float2 out = vis[k];
            out.x += ar * r.vre - ai * r.vim;
            out.y += ar * r.vim + ai * r.vre;
            vis[k] = out;
        }
    }
}

inline unsigned blocks_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

}  // namespace

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
cudaError_t launch_prep(const ws_plan_s *p, const double *uvw, const float2 *vis, int64_t M, bool grid,
                        cudaStream_t s) {
    if (M == 0) return cudaSuccess;
    const unsigned blocks = (unsigned)std::min<int64_t>(blocks_for(M, 256), (int64_t)p->sms * 8);
    prep_kernel<<<blocks, 256, 0, s>>>(p->L, uvw, vis, M, grid ? 1 : 0, p->d_rec, p->d_drop);
    return cudaGetLastError();
}

cudaError_t launch_bound_grid_records(const ws_plan_s *p, const double *uvw, const float2 *vis, int64_t M,
                                      cudaStream_t s) {
    if (M == 0) return cudaSuccess;
    bound_grid_records_kernel<<<blocks_for(M, 256), 256, 0, s>>>(p->L, uvw, vis, M, p->d_brec, p->d_rec);
    return cudaGetLastError();
}

cudaError_t launch_bin(ws_plan_s *p, int64_t M, bool grid, cudaStream_t s) {
    const int64_t n = p->ntiles + 1;
    cudaError_t e = cudaMemsetAsync(p->d_counts, 0, n * sizeof(uint32_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->d_tile_occ, 0, (size_t)p->ntiles, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->d_col_occ, 0, (size_t)p->L.ntt * p->L.ntu, s);
    if (e != cudaSuccess) return e;
    if (M > 0 && grid)
        count_kernel<true><<<blocks_for(M, 256), 256, 0, s>>>(p->L, p->d_rec, M, p->d_counts, p->d_tile_occ);
    else if (M > 0)
        count_kernel<false><<<blocks_for(M, 256), 256, 0, s>>>(p->L, p->d_rec, M, p->d_counts, p->d_tile_occ);
    const int nb = (int)((n + kScanPerBlock - 1) / kScanPerBlock);
    scan_block_kernel<<<nb, kScanThreads, 0, s>>>(p->d_counts, p->d_offsets, p->d_blocksums, n);
    scan_sums_kernel<<<1, kScanThreads, 0, s>>>(p->d_blocksums, nb);
    scan_add_kernel<<<blocks_for(n, 256), 256, 0, s>>>(p->d_offsets, p->d_blocksums, n);
    if (M == 0) return cudaGetLastError();
    e = cudaMemsetAsync(p->d_counts, 0, n * sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    if (grid)
        scatter_kernel<true><<<blocks_for(M, 256), 256, 0, s>>>(p->L, p->d_rec, M, p->d_offsets, p->d_counts,
                                                               p->d_list);
    else
        scatter_kernel<false><<<blocks_for(M, 256), 256, 0, s>>>(p->L, p->d_rec, M, p->d_offsets,
                                                                p->d_counts, p->d_list);
    strip_occ_kernel<<<blocks_for(p->ntiles, 256), 256, 0, s>>>(p->L, p->d_tile_occ, p->ntiles, p->d_col_occ);
    return cudaGetLastError();
}

cudaError_t launch_occ_count(const ws_plan_s *p, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(p->d_occ_counts, 0, (size_t)2 * p->L.ntt * sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    occ_count_kernel<<<p->L.ntt, 256, 0, s>>>(p->L, p->d_tile_occ, p->d_col_occ, p->d_occ_counts);
    return cudaGetLastError();
}

cudaError_t launch_grid_chunk(const ws_plan_s *p, int chunk, int planes, cudaStream_t s) {
    const int chunk_tt0 = chunk * (p->P / TT), chunk_ntt = planes / TT;
    const unsigned nblocks = (unsigned)p->L.ntu * p->L.ntv;      // one CTA per tile column
    if (chunk_ntt == 0) return cudaSuccess;
    const int R = p->L.tv;
    const bool det = (p->flags & WS_FLAG_DETERMINISTIC) != 0;
    auto go = [&](auto kernel, size_t smem) -> cudaError_t {
        if (smem > kMaxGridSmem) return cudaErrorInvalidValue;   // set_tile_rows keeps this from happening
        const cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        kernel<<<nblocks, kGridThreads, smem, s>>>(p->L, p->d_wcoef, p->wdeg, p->d_rec, p->d_offsets, p->d_list,
                                                   p->d_tile_occ, chunk_tt0, chunk_ntt, p->wbound, p->d_stack);
        return cudaGetLastError();
    };
#define WS_GRID_CASE(w)                                                                                       \
    case w:                                                                                                  \
        if (det) {                                                                                           \
            if (R == 16) return go(grid3d_kernel<w, 16, true>, GridSmem<w, 16, true>::bytes);                \
            if (R == 64) return go(grid3d_kernel<w, 64, true>, GridSmem<w, 64, true>::bytes);                \
            return go(grid3d_kernel<w, 32, true>, GridSmem<w, 32, true>::bytes);                             \
        }                                                                                                    \
        if (R == 16) return go(grid3d_kernel<w, 16, false>, GridSmem<w, 16, false>::bytes);                  \
        if (R == 64) return go(grid3d_kernel<w, 64, false>, GridSmem<w, 64, false>::bytes);                  \
        return go(grid3d_kernel<w, 32, false>, GridSmem<w, 32, false>::bytes);
    switch (p->L.W) {
        WS_GRID_CASE(1)
        WS_GRID_CASE(2)
        WS_GRID_CASE(3)
        WS_GRID_CASE(4)
        WS_GRID_CASE(5)
        WS_GRID_CASE(6)
        WS_GRID_CASE(7)
        WS_GRID_CASE(8)
        WS_GRID_CASE(9)
        WS_GRID_CASE(10)
        WS_GRID_CASE(11)
        WS_GRID_CASE(12)
        default:
            return cudaErrorInvalidValue;
    }
#undef WS_GRID_CASE
    return cudaGetLastError();
}

cudaError_t launch_correct_image(const ws_plan_s *p, const float2 *image, cudaStream_t s) {
    const int64_t n = (int64_t)p->L.N * p->L.N;
    correct_image_kernel<<<blocks_for(n, 256), 256, 0, s>>>(n, p->d_corr, image, p->L.fold, p->d_img);
    return cudaGetLastError();
}

cudaError_t launch_unfold(const ws_plan_s *p, const double *uvw, int64_t M, float2 *vis, cudaStream_t s) {
    (void)p;
    if (M == 0) return cudaSuccess;
    unfold_kernel<<<blocks_for(M, 256), 256, 0, s>>>(uvw, M, vis);
    return cudaGetLastError();
}

cudaError_t launch_degrid_chunk(const ws_plan_s *p, int chunk, int planes, int64_t M, float2 *vis,
                                cudaStream_t s) {
    if (M == 0) return cudaSuccess;
    // resident CTAs only (the kernel loops over the visibilities), at most one warp per visibility
    const int64_t want = blocks_for(M * 32, kDegridThreads);
    // CTAs per SM by (device, W), looked up once: the plan's device is current here
    auto resident = [&](auto kernel, int w) {
        constexpr int kDevices = 64;
        static std::atomic<int> per_sm[kDevices][kMaxW + 1];
        int b = p->dev >= 0 && p->dev < kDevices ? per_sm[p->dev][w].load(std::memory_order_relaxed) : 0;
        if (b == 0) {
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, kDegridThreads, 0) != cudaSuccess || b < 1)
                b = 1;
            if (p->dev >= 0 && p->dev < kDevices) per_sm[p->dev][w].store(b, std::memory_order_relaxed);
        }
        return (unsigned)std::min<int64_t>(want, (int64_t)p->sms * b);
    };
#define WS_DEGRID_CASE(w)                                                                                     \
    case w:                                                                                                  \
        degrid3d_kernel<w><<<resident(degrid3d_kernel<w>, w), kDegridThreads, 0, s>>>(                       \
            p->L, p->d_wcoef, p->wdeg, p->d_rec, p->d_list, p->d_offsets + p->ntiles, p->d_stack, chunk * p->P, \
            planes, vis);                                                                                    \
        break;
    switch (p->L.W) {
        WS_DEGRID_CASE(1)
        WS_DEGRID_CASE(2)
        WS_DEGRID_CASE(3)
        WS_DEGRID_CASE(4)
        WS_DEGRID_CASE(5)
        WS_DEGRID_CASE(6)
        WS_DEGRID_CASE(7)
        WS_DEGRID_CASE(8)
        WS_DEGRID_CASE(9)
        WS_DEGRID_CASE(10)
        WS_DEGRID_CASE(11)
        WS_DEGRID_CASE(12)
        default:
            return cudaErrorInvalidValue;
    }
#undef WS_DEGRID_CASE
    return cudaGetLastError();
}

}  // namespace ws
