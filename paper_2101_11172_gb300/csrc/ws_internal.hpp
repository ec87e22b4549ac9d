// Internal definitions shared by the plan (host) and the CUDA kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/ws.h"
#include "fft_plan.hpp"
#include "lmfit.hpp"

namespace ws {

#ifdef __CUDACC__
#define WS_HD __host__ __device__
#else
#define WS_HD
#endif

// Tiles of the stack: TT w-planes x tv grid rows (v) x TU grid columns (u).
// They bin the visibilities for degridding, mark the stack's occupancy for
// the plane transforms, and a tile column (all t-tiles of one (v, u) tile) is
// what one CTA of the gridding kernel owns.  tv is a plan parameter (16, 32 or
// 64 rows; a power of two that divides N', which is a multiple of 32, and
// whose gridding ring fits in shared memory), chosen by the tuner or left at
// TV; the plane count is padded to a multiple of TT.
constexpr int TU = 16;
constexpr int TV = 16;                 // default rows per tile
constexpr int kMinTileRows = 16, kMaxTileRows = 64;
constexpr int TT = 8;
constexpr int kMaxW = 12;
constexpr int kMaxW64 = 14;            // widths of FP64 plans (WS_FLAG_FP64)
constexpr int kMaxDeg = 16;

// Gridding kernel shape: 256 threads; each warp stages kChunk entries at a
// time.  Shared memory holds a ring of TT + W - 1 w-planes of the tile column
// (re and im, FP32 or, deterministic, 64-bit fixed point; rows padded to TU +
// 1 cells, planes to plane_stride cells), the weight table (3W slots of
// kCoefStride coefficients) and the warps' staged chunks (per entry its u
// weights from the first tap inside the tile, padded to a multiple of 4, then
// its v and w weights).
constexpr int kGridThreads = 256;
constexpr int kGridWarps = kGridThreads / 32;
constexpr int kChunk = 4;
constexpr int kRowPad = TU + 1;
constexpr int kCoefStride = 20;
constexpr size_t kMaxGridSmem = 227 * 1024;     // dynamic shared memory of one CTA
constexpr size_t kSmemPerSM = 228 * 1024;
WS_HD constexpr int ring_planes(int W) { return TT + W - 1; }
// Cells per ring plane: rows x 17 padded to 23 (mod 32).  The add loop's lanes
// take (row, plane) pairs of a footprint; with the row stride 17 and this
// plane stride their shared-memory banks collide least: 1.35 lanes per bank on
// average over the footprint shapes of W = 7, against 1.52 for 20 and 1.73
// for 8 (mod 32) (the ring's size is padded to 16 bytes for its clearing).
WS_HD constexpr int plane_stride(int rows) { return rows * kRowPad + ((23 - rows * kRowPad) % 32 + 32) % 32; }
WS_HD constexpr size_t ring_bytes(int W, int rows, bool det) {
    return ((size_t)ring_planes(W) * plane_stride(rows) * (det ? 8 : 4) + 15) / 16 * 16;   // one component
}
WS_HD constexpr int wx_span(int W) { return (W + 3) / 4 * 4; }                // staged u weights
WS_HD constexpr int stage_stride(int W) { return (wx_span(W) + 2 * W + 3) / 4 * 4; }   // floats per entry
WS_HD constexpr size_t grid_smem_bytes(int W, int rows, bool det) {
    return 2 * ring_bytes(W, rows, det)                                           // ring, re and im
           + (size_t)3 * W * kCoefStride * 4                                      // weight table
           + (size_t)kGridWarps * kChunk * stage_stride(W) * 4                    // staged weights
           + (size_t)kGridWarps * kChunk * (16 + 8 + 16);                         // items, values, nu
}
// CTAs of the gridding kernel that fit on one SM (1 KB reserved per CTA), at
// most 6.  Gridding is latency-bound and gains from every CTA that fits: on the
// survey (W = 7, 16-row tiles) 13.2 ms at 3 CTAs per SM, 11.0 at 4, 10.2 at 5 and
// 10.1 at 6, where the 4-entry chunks and 40 registers just fit.
WS_HD constexpr int grid_ctas_per_sm(int W, int rows, bool det) {
    return (int)(kSmemPerSM / (grid_smem_bytes(W, rows, det) + 1024)) < 1 ? 1
           : (int)(kSmemPerSM / (grid_smem_bytes(W, rows, det) + 1024)) > 6
               ? 6
               : (int)(kSmemPerSM / (grid_smem_bytes(W, rows, det) + 1024));
}
// Per-call device counters: visibilities dropped for non-finite u, v; for w
// outside the plan's range; and bounded device waits that gave up.
constexpr int kCounters = 3;
// Polls of a bounded mbarrier wait (a few hundred milliseconds) before it gives up.
constexpr int kWaitPolls = 1 << 20;

// One visibility after pre-processing: first grid point of its W x W x W
// footprint (u and v wrapped into [0, N'), t relative to the plan's t_lo;
// t0 < 0 marks a dropped visibility), the three offsets nu in [-1/2, 1/2)
// and a complex value (gridding: V exp(2 pi i w (n0 - 1)); degridding:
// exp(-2 pi i w (n0 - 1))).
struct __align__(16) VisRec {
    int32_t r0, s0, t0;
    float nux, nuy, nuz;
    float vre, vim;
};

struct DeviceTables {
    const float *wcoef;    // W x (deg+1) monomial coefficients of c_i(nu) in nu
    int W, deg;
};

struct Launch {            // geometry the kernels need
    int N, Np, W, Nw, t_lo;
    int ntu, ntv, ntt;     // tile counts along u, v, t
    int tv, tv_log;        // grid rows per tile (a power of two) and its log2
    double uv_scale;       // u' = u * uv_scale (= N' * dl)
    double nscale, n0m1;   // w' = w * nscale; n0 - 1
    int fold;              // WS_FLAG_HERMITIAN: w < 0 handled as the conjugate at -(u, v, w)
};

}  // namespace ws

struct ws_plan_s {
    int dev = -1;
    int sms = 1;                   // multiprocessors of dev (grid sizing)
    uint32_t flags = 0;
    ws::Launch L{};
    double x0 = 0.0, fov = 0.0, w_min = 0.0, w_max = 0.0;
    ws::LeastMisfitFit fit;
    int wdeg = 0;
    std::vector<float> wcoef_host;
    float wbound = 1.f;            // bound on |C_x C_y C_z| over all taps and offsets (deterministic gridding)

    // device tables (plan lifetime)
    float *d_wcoef = nullptr;      // 2 x W x (wdeg+1): taps along u and v, then along w
    int orig_bins = 0;             // > 0: original W-stacking with this many w-bins
    float *d_corr = nullptr;       // N x N: h(x_j) h(y_i) h(z_ij)
    float2 *d_zsplit = nullptr;    // N x N: z = hi + lo, hi a multiple of 2^-13
    // stack workspace
    int P = 0;                     // planes per chunk (multiple of TT)
    float2 *d_stack = nullptr;     // P x N' x N', column-block layout (common.cuh)
    float2 *d_tw = nullptr;        // N' twiddles exp(-2 pi i m / N')
    ws::FftPlan fft{};             // the N'-point plane transform
    bool fft_mixed = false;        // N' has a factor 3, 5 or 7
    // per-call buffers (grow on demand)
    ws::VisRec *d_rec = nullptr;
    int64_t rec_cap = 0;
    uint32_t *d_list = nullptr;
    int64_t list_cap = 0;
    uint32_t *d_counts = nullptr;  // ntiles + 1
    uint32_t *d_offsets = nullptr; // ntiles + 1
    uint32_t *d_blocksums = nullptr;
    int64_t ntiles = 0;
    uint8_t *d_tile_occ = nullptr; // ntiles: 1 if any visibility footprint touches the tile
    uint8_t *d_col_occ = nullptr;  // ntt x ntu: 1 if any tile of that (t-tile, u-tile) strip is touched
    float4 *d_acc = nullptr;       // N x N: (sum re, sum im, comp re, comp im)
    float2 *d_img = nullptr;       // N x N: corrected image (degridding)
    unsigned long long *d_drop = nullptr;   // kCounters: [0] non-finite uv, [1] w out of range, [2] timed-out waits
    unsigned long long *h_drop = nullptr;   // pinned mirror
    int wait_polls = ws::kWaitPolls;        // limit of inv_rows' first wait per plane (WS_WAIT_POLLS)
    // visibility set bound by ws_plan_bind_uvw: records (degridding form) and
    // both directions' bin lists, made once for that uvw
    const double *b_uvw = nullptr;
    int64_t b_M = -1;
    ws::VisRec *d_brec = nullptr;
    int64_t brec_cap = 0;
    uint32_t *d_blist_g = nullptr;          // gridding: (visibility, tile column) pairs by column and first-tap t-tile
    int64_t blist_g_cap = 0;
    uint32_t *d_blist_d = nullptr;          // degridding: visibilities by first-tap tile
    int64_t blist_d_cap = 0;
    uint32_t *d_boff_g = nullptr;           // ntiles + 1
    uint32_t *d_boff_d = nullptr;           // ntiles + 1
    uint8_t *d_btile_occ = nullptr;         // ntiles
    uint8_t *d_bcol_occ = nullptr;          // ntt x ntu
    unsigned long long *d_bdrop = nullptr;  // kCounters: the bound set's drop counts
    // FP64 plans (WS_FLAG_FP64): their own tables and one plane of workspace
    bool fp64 = false;
    double *d_cheb64 = nullptr;             // 2 x W x (degree+1): Chebyshev series of c_i(nu), (u, v) then w
    double *d_corr64 = nullptr;             // N x N
    double *d_z64 = nullptr;                // N x N
    double2 *d_plane64 = nullptr;           // N' x N'
    double2 *d_acc64 = nullptr;             // N x N
    double2 *d_tw64 = nullptr;              // N': exp(-2 pi i m / N')
    int fft64_log = 0;
    void *d_rec64 = nullptr;
    int64_t rec64_cap = 0;
    // occupancy statistics (WS_FLAG_TIMING): per t-tile, occupied tiles and
    // (t-tile, u-strip) strips, then the number of tile-list entries
    uint32_t *d_occ_counts = nullptr;       // 2 ntt
    uint32_t *h_occ_counts = nullptr;       // pinned: 2 ntt + 1
    int64_t last_dropped = 0;
    int64_t bytes = 0;
    // statistics (WS_FLAG_TIMING adds CUDA events around each stage)
    ws_stats_t stats{};
    struct Timed {
        int stage;
        cudaEvent_t start, stop;
    };
    std::vector<Timed> pending;           // recorded, not yet folded into stats
    std::vector<cudaEvent_t> free_events;
};

namespace ws {

void set_error(const std::string &msg);
ws_status cuda_fail(cudaError_t e, const char *what);

// Tile lists are indexed with 32-bit offsets and hold at most 12 entries per visibility.
constexpr int64_t kMaxVis = ((int64_t)1 << 31) / 12;

// Plan construction and the enqueue-only halves of ws_grid / ws_degrid (plan.cpp).
// own_stack = false leaves d_stack unset and P = 0 for a batch to assign.
ws_status plan_create(ws_plan_s **out, int32_t N, double x0, int32_t W, double fov, double w_min, double w_max,
                      uint32_t flags, bool own_stack, int32_t orig_bins = 0);
ws_status ensure_capacity(ws_plan_s *p, int64_t M, bool grid);
ws_status ensure_capacity64(ws_plan_s *p, int64_t M);
// Re-tile a plan with tv grid rows per tile: the per-tile tables are sized
// anew and a bound visibility set is dropped.  WS_ERR_ARG if tv is not 16, 32
// or 64, does not divide N', or gives a gridding ring larger than shared memory.
ws_status set_tile_rows(ws_plan_s *p, int tv);
// Whether tv rows per tile suit the plan (the conditions of set_tile_rows).
bool tile_rows_fit(const ws_plan_s *p, int tv);
ws_status enqueue_grid(ws_plan_s *p, const double *uvw, const float2 *vis, int64_t M, float2 *dirty,
                       cudaStream_t s);
ws_status enqueue_degrid(ws_plan_s *p, const float2 *image, const double *uvw, int64_t M, float2 *vis,
                         cudaStream_t s);

// Tuning cache (tune.cpp): key of (GPU, N', W); lookup and store of the tile rows.
std::string tune_key(int dev, int Np, int W);
bool tune_lookup(const char *path, const std::string &key, int *tile_rows);
bool tune_store(const char *path, const std::string &key, int tile_rows, const int *cand, const float *ms, int n);

// FP64 path (fp64.cu).
size_t fp64_record_bytes();
ws_status enqueue_grid64(ws_plan_s *p, const double *uvw, const double2 *vis, int64_t M, double2 *dirty,
                         cudaStream_t s);
ws_status enqueue_degrid64(ws_plan_s *p, const double2 *image, const double *uvw, int64_t M, double2 *vis,
                           cudaStream_t s);

// Launchers (wstack.cu).
cudaError_t launch_prep(const ws_plan_s *p, const double *uvw, const float2 *vis, int64_t M,
                        bool grid, cudaStream_t s);
cudaError_t launch_bound_grid_records(const ws_plan_s *p, const double *uvw, const float2 *vis, int64_t M,
                                      cudaStream_t s);
// Binning (gridding: by tile column and first-tap t-tile; degridding: by
// first-tap tile) and the stack's occupancy maps, from the records d_rec.
cudaError_t launch_bin(ws_plan_s *p, int64_t M, bool grid, cudaStream_t s);
cudaError_t launch_occ_count(const ws_plan_s *p, cudaStream_t s);
cudaError_t launch_grid_chunk(const ws_plan_s *p, int chunk, int planes, cudaStream_t s);
cudaError_t launch_correct_image(const ws_plan_s *p, const float2 *image, cudaStream_t s);
cudaError_t launch_unfold(const ws_plan_s *p, const double *uvw, int64_t M, float2 *vis, cudaStream_t s);
cudaError_t launch_degrid_chunk(const ws_plan_s *p, int chunk, int planes, int64_t M,
                                float2 *vis, cudaStream_t s);

// Plane transforms (transforms.cu).
size_t transform_smem_bytes(const FftPlan &F, int N);
cudaError_t setup_transform_kernels(const FftPlan &F, int N);
cudaError_t launch_fwd_rows(const ws_plan_s *p, int chunk, int planes, cudaStream_t s);
cudaError_t launch_fwd_cols(const ws_plan_s *p, int chunk, int planes, cudaStream_t s);
cudaError_t launch_inv_cols(const ws_plan_s *p, int chunk, int planes, cudaStream_t s);
cudaError_t launch_inv_rows(const ws_plan_s *p, int chunk, int planes, bool first, bool last, float2 *dirty,
                            cudaStream_t s);

}  // namespace ws
