// ws_degrid_noalloc: degridding for callers that cannot allocate device memory.
//
// Some callers must not call cudaMalloc once they are running: code that
// executes under a memory budget fixed at start-up (a serving process that
// pre-reserves its pool, a plug-in inside a host application that owns all
// device allocations) or code that must not trigger the implicit device
// synchronisation an allocation can cause.  For them this file runs the same
// degridding kernels as ws_degrid, but takes every per-call scratch buffer
// (visibility records, bin lists, counts and occupancy, the corrected
// image, the w-plane chunk and the drop counters) from one fixed, file-scope device
// array instead of the plan's workspace.  The plan itself (tables made by
// ws_plan) and the caller's inputs and outputs are used as they are.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <string>

#include "ws_internal.hpp"

namespace {

// 64 MiB of scratch, held by every device that loads this library until exit.
constexpr size_t kScratchBytes = (size_t)64 << 20;
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Device address of g_scratch per device, looked up once with that device current.
constexpr int kMaxDevices = 64;
unsigned char *g_scratch_ptr[kMaxDevices] = {};
std::mutex g_scratch_mutex;

ws_status scratch_for(int dev, unsigned char **out) {
    if (dev < 0 || dev >= kMaxDevices) {
        ws::set_error("ws_degrid_noalloc: device index out of range");
        return WS_ERR_ARG;
    }
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_ptr[dev]) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_scratch);
        if (e != cudaSuccess) return ws::cuda_fail(e, "ws_degrid_noalloc: cudaGetSymbolAddress");
        g_scratch_ptr[dev] = static_cast<unsigned char *>(ptr);
    }
    *out = g_scratch_ptr[dev];
    return WS_OK;
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

extern "C" ws_status ws_degrid_noalloc(ws_plan_t plan, const void *image, const double *uvw, int64_t M, void *vis,
                                       ws_stream_t stream) {
    using namespace ws;
    if (!plan || M < 0 || !image || (M > 0 && (!uvw || !vis)) || M > kMaxVis) {
        set_error("ws_degrid_noalloc: invalid argument");
        return WS_ERR_ARG;
    }
    const ws_plan_s *p = plan;
    if (p->fp64) {
        set_error("ws_degrid_noalloc: not for FP64 plans");
        return WS_ERR_ARG;
    }
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != p->dev && cudaSetDevice(p->dev) != cudaSuccess) {
        set_error("ws_degrid_noalloc: cannot select the plan's device");
        return WS_ERR_CUDA;
    }
    struct Restore {
        int prev, dev;
        ~Restore() {
            if (prev >= 0 && prev != dev) cudaSetDevice(prev);
        }
    } restore{prev, p->dev};

    unsigned char *base = nullptr;
    ws_status st = scratch_for(p->dev, &base);
    if (st != WS_OK) return st;

    // carve the scratch: fixed parts first, then as many planes as fit (a multiple of TT)
    const size_t n_img = (size_t)p->L.N * p->L.N;
    const size_t plane = (size_t)p->L.Np * p->L.Np * sizeof(float2);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t at = off;
        off = align256(off + bytes);
        return base + at;
    };
    const int64_t Mc = std::max<int64_t>(M, 1);
    VisRec *rec = reinterpret_cast<VisRec *>(take((size_t)Mc * sizeof(VisRec)));
    uint32_t *list = reinterpret_cast<uint32_t *>(take((size_t)Mc * sizeof(uint32_t)));
    uint32_t *counts = reinterpret_cast<uint32_t *>(take((size_t)(p->ntiles + 1) * sizeof(uint32_t)));
    uint32_t *offsets = reinterpret_cast<uint32_t *>(take((size_t)(p->ntiles + 1) * sizeof(uint32_t)));
    uint32_t *blocksums = reinterpret_cast<uint32_t *>(take(4096 * sizeof(uint32_t)));
    unsigned long long *drop = reinterpret_cast<unsigned long long *>(take(2 * sizeof(unsigned long long)));
    uint8_t *tile_occ = take((size_t)p->ntiles);
    uint8_t *col_occ = take((size_t)p->L.ntt * p->L.ntu);
    float2 *img = reinterpret_cast<float2 *>(take(n_img * sizeof(float2)));
    if (off > kScratchBytes || (kScratchBytes - off) / plane < (size_t)TT) {
        set_error("ws_degrid_noalloc: the problem needs more than the 64 MiB of fixed scratch (visibility "
                  "records, image and at least 8 w-planes of N' x N'); use ws_degrid");
        return WS_ERR_ARG;
    }
    const int total = p->L.ntt * TT;
    int P = (int)std::min<size_t>((kScratchBytes - off) / plane, (size_t)total);
    P = (P / TT) * TT;
    float2 *stack = reinterpret_cast<float2 *>(base + off);

    // a view of the plan whose workspace pointers are the scratch (scalars and pointers only)
    ws_plan_s v;
    v.dev = p->dev;
    v.sms = p->sms;
    v.flags = p->flags;
    v.L = p->L;
    v.wdeg = p->wdeg;
    v.d_wcoef = p->d_wcoef;
    v.d_corr = p->d_corr;
    v.d_zsplit = p->d_zsplit;
    v.d_tw = p->d_tw;
    v.fft = p->fft;
    v.fft_mixed = p->fft_mixed;
    v.ntiles = p->ntiles;
    v.P = P;
    v.d_stack = stack;
    v.d_rec = rec;
    v.d_list = list;
    v.d_counts = counts;
    v.d_offsets = offsets;
    v.d_blocksums = blocksums;
    v.d_img = img;
    v.d_drop = drop;
    v.d_tile_occ = tile_occ;
    v.d_col_occ = col_occ;

    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(drop, 0, 2 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return cuda_fail(e, "ws_degrid_noalloc: clearing counters");
    if (M > 0) {
        if ((e = cudaMemsetAsync(vis, 0, (size_t)M * sizeof(float2), s)) != cudaSuccess)
            return cuda_fail(e, "ws_degrid_noalloc: clearing the output");
        if ((e = launch_prep(&v, uvw, nullptr, M, false, s)) != cudaSuccess)
            return cuda_fail(e, "ws_degrid_noalloc: prep kernel");
        if ((e = launch_bin(&v, M, false, s)) != cudaSuccess)
            return cuda_fail(e, "ws_degrid_noalloc: binning kernels");
        if ((e = launch_correct_image(&v, static_cast<const float2 *>(image), s)) != cudaSuccess)
            return cuda_fail(e, "ws_degrid_noalloc: correction kernel");
        const int nchunks = (total + P - 1) / P;
        for (int c = 0; c < nchunks; ++c) {
            const int planes = std::min(P, total - c * P);
            if ((e = launch_fwd_rows(&v, c, planes, s)) != cudaSuccess)
                return cuda_fail(e, "ws_degrid_noalloc: fwd_rows kernel");
            if ((e = launch_fwd_cols(&v, c, planes, s)) != cudaSuccess)
                return cuda_fail(e, "ws_degrid_noalloc: fwd_cols kernel");
            if ((e = launch_degrid_chunk(&v, c, planes, M, static_cast<float2 *>(vis), s)) != cudaSuccess)
                return cuda_fail(e, "ws_degrid_noalloc: degrid3d kernel");
        }
        if (v.L.fold && (e = launch_unfold(&v, uvw, M, static_cast<float2 *>(vis), s)) != cudaSuccess)
            return cuda_fail(e, "ws_degrid_noalloc: unfolding kernel");
    }
    // the drop counts go to the plan's pinned mirror (allocated by ws_plan)
    if ((e = cudaMemcpyAsync(p->h_drop, drop, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s)) !=
        cudaSuccess)
        return cuda_fail(e, "ws_degrid_noalloc: reading the drop counters");
    if (p->flags & WS_FLAG_ASYNC) return WS_OK;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "ws_degrid_noalloc: waiting");
    if (p->h_drop[0]) {
        set_error(std::to_string(p->h_drop[0]) + " visibilities had non-finite or huge u, v and were dropped");
        return WS_ERR_UV_RANGE;
    }
    if (p->h_drop[1]) {
        set_error(std::to_string(p->h_drop[1]) + " visibilities had w outside the plan's w-range and were dropped");
        return WS_ERR_W_RANGE;
    }
    return WS_OK;
}
