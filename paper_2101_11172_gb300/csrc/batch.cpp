// Batches of independent gridding / degridding problems (ws_batch_*).
//
// The paper treats one observation at a time; a serving system sees many at
// once -- channels, snapshots, fields -- with different image sizes, w-ranges
// and visibility counts.  A batch holds one plan per instance (Section 5.3
// sizing, Section 3.3 kernels, exactly as ws_plan builds them) but no
// per-plan w-stack: the instances are dealt to K branches and each branch
// owns one slice of a shared workspace, which its instances use one after
// the other.  A call enqueues every instance's kernels on its branch's stream,
// forked from and joined back into one capture stream, and captures the lot
// into a CUDA graph; later calls with the same data pointers replay the graph
// (one launch from the host), calls with new pointers capture a new one.
//
// K = 0 at creation defers the choice: the first call picks the gridding
// tile rows for each image size (tune_tiles), then times the graph for
// K = 1, 2 and 4 (those whose slices still hold TT planes of the largest
// instance) and keeps the fastest.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "ws_internal.hpp"

using namespace ws;

namespace {

constexpr int kMaxBranches = 8;

struct Graph {
    std::vector<const void *> key;     // the data pointers it was captured with
    cudaGraphExec_t exec = nullptr;
};

}  // namespace

struct ws_batch_s {
    int dev = -1;
    uint32_t flags = 0;
    std::vector<ws_plan_s *> plans;
    std::vector<int64_t> M;
    std::vector<double> cost;          // relative work of each instance (for dealing)
    float2 *workspace = nullptr;
    size_t workspace_bytes = 0;
    int K = 0;                         // branches in use (0 until tuned)
    std::vector<int> branch_of;        // instance -> branch for the current K
    cudaStream_t origin = nullptr;     // capture stream
    cudaStream_t br[kMaxBranches] = {};
    cudaEvent_t fork = nullptr, join[kMaxBranches] = {};
    cudaEvent_t ready = nullptr, tuned = nullptr;   // order the tuning runs after, and before, the caller's stream
    Graph graph[2];                    // 0 = grid, 1 = degrid
};

namespace {

void destroy_graph(Graph &g) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    g.exec = nullptr;
    g.key.clear();
}

void release_batch(ws_batch_s *b) {
    if (!b) return;
    if (b->dev >= 0) cudaSetDevice(b->dev);
    cudaDeviceSynchronize();
    for (Graph &g : b->graph) destroy_graph(g);
    for (ws_plan_s *p : b->plans) {
        if (p) p->d_stack = nullptr;   // the batch's workspace, freed below
        ws_destroy(p);
    }
    cudaFree(b->workspace);
    for (int k = 0; k < kMaxBranches; ++k) {
        if (b->br[k]) cudaStreamDestroy(b->br[k]);
        if (b->join[k]) cudaEventDestroy(b->join[k]);
    }
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->ready) cudaEventDestroy(b->ready);
    if (b->tuned) cudaEventDestroy(b->tuned);
    if (b->origin) cudaStreamDestroy(b->origin);
    delete b;
}

size_t plane_bytes(const ws_plan_s *p) { return (size_t)p->L.Np * p->L.Np * sizeof(float2); }

// Deal instances to K branches (largest first, each to the least-loaded
// branch) and give each plan its branch's slice of the workspace.  False if a
// slice cannot hold TT planes of some instance dealt to it.
bool assign(ws_batch_s *b, int K) {
    const int n = (int)b->plans.size();
    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return b->cost[a] > b->cost[c]; });
    std::vector<double> load(K, 0.0);
    b->branch_of.assign(n, 0);
    for (int i : order) {
        const int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        b->branch_of[i] = k;
        load[k] += b->cost[i];
    }
    const size_t slice = (b->workspace_bytes / (size_t)K) & ~(size_t)255;
    for (int i = 0; i < n; ++i) {
        ws_plan_s *p = b->plans[i];
        const int total = p->L.ntt * TT;
        const size_t fit = slice / plane_bytes(p);
        if (fit < (size_t)TT) return false;
        p->P = (int)std::min<size_t>((size_t)total, (fit / TT) * TT);
        p->d_stack = reinterpret_cast<float2 *>(reinterpret_cast<char *>(b->workspace) + slice * b->branch_of[i]);
    }
    b->K = K;
    return true;
}

// Capture one call of every instance into an executable graph.
ws_status capture(ws_batch_s *b, int dir, const std::vector<const void *> &ptr, cudaGraphExec_t *exec) {
    const int n = (int)b->plans.size();
    cudaError_t e = cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "ws_batch: beginning the capture");
    ws_status st = WS_OK;
    e = cudaEventRecord(b->fork, b->origin);
    for (int k = 0; k < b->K && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(b->br[k], b->fork, 0);
    if (e != cudaSuccess) st = cuda_fail(e, "ws_batch: forking the branches");
    for (int i = 0; i < n && st == WS_OK; ++i) {
        ws_plan_s *p = b->plans[i];
        cudaStream_t s = b->br[b->branch_of[i]];
        const void *a = ptr[3 * i], *c = ptr[3 * i + 1];
        void *out = const_cast<void *>(ptr[3 * i + 2]);
        if (dir == 0)
            st = enqueue_grid(p, static_cast<const double *>(a), static_cast<const float2 *>(c), b->M[i],
                              static_cast<float2 *>(out), s);
        else
            st = enqueue_degrid(p, static_cast<const float2 *>(a), static_cast<const double *>(c), b->M[i],
                                static_cast<float2 *>(out), s);
        if (st == WS_OK) {
            e = cudaMemcpyAsync(p->h_drop, p->d_drop, kCounters * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                                s);
            if (e != cudaSuccess) st = cuda_fail(e, "ws_batch: reading drop counters");
        }
    }
    for (int k = 0; k < b->K && st == WS_OK; ++k) {
        e = cudaEventRecord(b->join[k], b->br[k]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->origin, b->join[k], 0);
        if (e != cudaSuccess) st = cuda_fail(e, "ws_batch: joining the branches");
    }
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(b->origin, &g);
    if (st == WS_OK && e != cudaSuccess) st = cuda_fail(e, "ws_batch: ending the capture");
    if (st == WS_OK) {
        e = cudaGraphInstantiate(exec, g, 0);
        if (e != cudaSuccess) st = cuda_fail(e, "ws_batch: instantiating the graph");
    }
    if (g) cudaGraphDestroy(g);
    return st;
}

// Device milliseconds of one launch of exec on the capture stream (after one untimed launch).
ws_status time_graph(ws_batch_s *b, cudaGraphExec_t exec, float *ms) {
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    cudaError_t e = cudaEventCreate(&t0);
    if (e == cudaSuccess) e = cudaEventCreate(&t1);
    if (e == cudaSuccess) e = cudaGraphLaunch(exec, b->origin);
    if (e == cudaSuccess) e = cudaEventRecord(t0, b->origin);
    if (e == cudaSuccess) e = cudaGraphLaunch(exec, b->origin);
    if (e == cudaSuccess) e = cudaEventRecord(t1, b->origin);
    if (e == cudaSuccess) e = cudaEventSynchronize(t1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, t0, t1);
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    return e == cudaSuccess ? WS_OK : cuda_fail(e, "ws_batch: timing a branch count");
}

// Enqueue instance i's call of direction dir (0 grid, 1 degrid) on stream s.
ws_status enqueue_instance(ws_batch_s *b, int i, int dir, const std::vector<const void *> &ptr, cudaStream_t s) {
    ws_plan_s *p = b->plans[i];
    const void *a = ptr[3 * i], *c = ptr[3 * i + 1];
    void *out = const_cast<void *>(ptr[3 * i + 2]);
    if (dir == 0)
        return enqueue_grid(p, static_cast<const double *>(a), static_cast<const float2 *>(c), b->M[i],
                            static_cast<float2 *>(out), s);
    return enqueue_degrid(p, static_cast<const float2 *>(a), static_cast<const double *>(c), b->M[i],
                          static_cast<float2 *>(out), s);
}

// Tile rows per image size: for every N' in the batch without an entry in the
// tuning cache (WS_TUNE_CACHE), time this call's direction on the instance of
// that size with the most visibilities for 16, 32 and 64 rows per tile, and
// give every instance of that size the fastest (recorded in the cache when one
// is named).  Runs on the batch's stream with one workspace slice per branch.
ws_status tune_tiles(ws_batch_s *b, int dir, const std::vector<const void *> &ptr) {
    const int n = (int)b->plans.size();
    const char *cache = std::getenv("WS_TUNE_CACHE");
    std::vector<int> sizes;
    for (ws_plan_s *p : b->plans)
        if (std::find(sizes.begin(), sizes.end(), p->L.Np) == sizes.end()) sizes.push_back(p->L.Np);
    if (!assign(b, 1)) return WS_OK;            // tune() reports the workspace problem
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    cudaError_t e = cudaEventCreate(&t0);
    if (e == cudaSuccess) e = cudaEventCreate(&t1);
    ws_status st = e == cudaSuccess ? WS_OK : cuda_fail(e, "ws_batch: timing tile shapes");
    for (int Np : sizes) {
        if (st != WS_OK) break;
        int big = -1;
        for (int i = 0; i < n; ++i)
            if (b->plans[i]->L.Np == Np && (big < 0 || b->M[i] > b->M[big])) big = i;
        const std::string key = tune_key(b->dev, Np, b->plans[big]->L.W);
        int cached = 0;
        if (tune_lookup(cache, key, &cached) || b->M[big] == 0) continue;
        int cand[3], nc = 0;
        float ms[3] = {0.f, 0.f, 0.f};
        for (int c : {16, 32, 64})
            if (tile_rows_fit(b->plans[big], c)) cand[nc++] = c;
        for (int k = 0; k < nc && st == WS_OK; ++k) {
            st = set_tile_rows(b->plans[big], cand[k]);
            if (st != WS_OK) break;
            st = enqueue_instance(b, big, dir, ptr, b->origin);          // untimed
            if (st == WS_OK && (e = cudaEventRecord(t0, b->origin)) != cudaSuccess) st = cuda_fail(e, "ws_batch");
            if (st == WS_OK) st = enqueue_instance(b, big, dir, ptr, b->origin);
            if (st == WS_OK && (e = cudaEventRecord(t1, b->origin)) == cudaSuccess &&
                (e = cudaEventSynchronize(t1)) == cudaSuccess)
                e = cudaEventElapsedTime(&ms[k], t0, t1);
            if (st == WS_OK && e != cudaSuccess) st = cuda_fail(e, "ws_batch: timing tile shapes");
        }
        if (st != WS_OK) break;
        int k = 0;
        for (int j = 1; j < nc; ++j)
            if (ms[j] < ms[k]) k = j;
        for (int i = 0; i < n && st == WS_OK; ++i)
            if (b->plans[i]->L.Np == Np) st = set_tile_rows(b->plans[i], cand[k]);
        if (st == WS_OK && cache && *cache) tune_store(cache, key, cand[k], cand, ms, nc);
    }
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    b->K = 0;
    return st;
}

// Pick K by timing this call's graph for K = 1, 2, 4; leaves the best graph in g.
ws_status tune(ws_batch_s *b, int dir, const std::vector<const void *> &ptr, Graph &g) {
    float best = 0.f;
    int best_K = 0;
    const int n = (int)b->plans.size();
    ws_status tst = tune_tiles(b, dir, ptr);
    if (tst != WS_OK) return tst;
    for (int K : {1, 2, 4}) {
        if (K > n && K > 1) break;
        if (!assign(b, K)) continue;
        cudaGraphExec_t exec = nullptr;
        ws_status st = capture(b, dir, ptr, &exec);
        float ms = 0.f;
        if (st == WS_OK) st = time_graph(b, exec, &ms);
        if (st != WS_OK) {
            if (exec) cudaGraphExecDestroy(exec);
            return st;
        }
        if (best_K == 0 || ms < best) {
            best = ms;
            best_K = K;
            destroy_graph(g);
            g.exec = exec;
            g.key = ptr;
        } else {
            cudaGraphExecDestroy(exec);
        }
    }
    if (best_K == 0) {
        set_error("ws_batch: the workspace cannot hold 8 w-planes of the largest instance");
        return WS_ERR_OOM;
    }
    assign(b, best_K);
    return WS_OK;
}

ws_status run(ws_batch_s *b, int dir, const std::vector<const void *> &ptr, cudaStream_t stream) {
    if (cudaSetDevice(b->dev) != cudaSuccess) {
        set_error("ws_batch: cannot select the batch's device");
        return WS_ERR_CUDA;
    }
    Graph &g = b->graph[dir];
    if (!g.exec || g.key != ptr) {
        destroy_graph(g);
        if (b->K == 0) {
            // the first call decides K; the other direction's graph must then be recaptured.
            // The timing runs execute on the batch's own stream: they start after the
            // work already queued on the caller's stream (which may still be producing
            // this call's inputs, or using memory the outputs now occupy) and the
            // caller's stream waits for them in turn.
            destroy_graph(b->graph[1 - dir]);
            cudaError_t e = cudaEventRecord(b->ready, stream);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(b->origin, b->ready, 0);
            if (e != cudaSuccess) return cuda_fail(e, "ws_batch: ordering the tuning runs");
            ws_status st = tune(b, dir, ptr, g);
            e = cudaEventRecord(b->tuned, b->origin);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(stream, b->tuned, 0);
            if (st != WS_OK) return st;
            if (e != cudaSuccess) return cuda_fail(e, "ws_batch: ordering the tuning runs");
        } else {
            ws_status st = capture(b, dir, ptr, &g.exec);
            if (st != WS_OK) return st;
            g.key = ptr;
        }
    }
    cudaError_t e = cudaGraphLaunch(g.exec, stream);
    if (e != cudaSuccess) return cuda_fail(e, "ws_batch: launching the graph");
    if (b->flags & WS_FLAG_ASYNC) return WS_OK;
    e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_fail(e, "ws_batch: waiting for the stream");
    for (size_t i = 0; i < b->plans.size(); ++i) {
        const ws_plan_s *p = b->plans[i];
        if (p->h_drop[2]) {
            set_error("instance " + std::to_string(i) + ": " + std::to_string(p->h_drop[2]) +
                      " device waits for copies gave up; the output is incomplete");
            return WS_ERR_TIMEOUT;
        }
        if (p->h_drop[0] || p->h_drop[1]) {
            set_error("instance " + std::to_string(i) + ": " + std::to_string(p->h_drop[0] + p->h_drop[1]) +
                      " visibilities were dropped (" + (p->h_drop[0] ? "non-finite u, v" : "w outside the range") +
                      ")");
            return p->h_drop[0] ? WS_ERR_UV_RANGE : WS_ERR_W_RANGE;
        }
    }
    return WS_OK;
}

}  // namespace

extern "C" {

ws_status ws_batch_create(ws_batch_t *out, int32_t n, const ws_instance_t *inst, double x0, int32_t W,
                          int32_t branches, int64_t workspace_bytes, uint32_t flags) {
    if (!out) {
        set_error("ws_batch_create: out is NULL");
        return WS_ERR_ARG;
    }
    *out = nullptr;
    if (n < 1 || !inst || branches < 0 || branches > kMaxBranches || workspace_bytes < 0) {
        set_error("ws_batch_create: need n >= 1 instances and 0 <= branches <= 8");
        return WS_ERR_ARG;
    }
    if (flags & ~(uint32_t)(WS_FLAG_ASYNC | WS_FLAG_NO_Z_OFFSET | WS_FLAG_HERMITIAN | WS_FLAG_DIVIDE_BY_N |
                            WS_FLAG_DETERMINISTIC)) {
        set_error("ws_batch_create: only WS_FLAG_ASYNC, WS_FLAG_NO_Z_OFFSET, WS_FLAG_HERMITIAN, WS_FLAG_DIVIDE_BY_N "
                  "and WS_FLAG_DETERMINISTIC apply to batches");
        return WS_ERR_ARG;
    }
    for (int32_t i = 0; i < n; ++i)
        if (inst[i].M < 0 || inst[i].M > kMaxVis) {
            set_error("ws_batch_create: instance " + std::to_string(i) + " has an invalid visibility count");
            return WS_ERR_ARG;
        }
    ws_batch_s *b = new (std::nothrow) ws_batch_s;
    if (!b) {
        set_error("ws_batch_create: out of host memory");
        return WS_ERR_OOM;
    }
    b->flags = flags;
    cudaError_t e = cudaGetDevice(&b->dev);
    if (e != cudaSuccess) {
        delete b;
        return cuda_fail(e, "ws_batch_create: no CUDA device");
    }
    ws_status st = WS_OK;
    size_t largest_plane = 0;
    for (int32_t i = 0; i < n && st == WS_OK; ++i) {
        ws_plan_s *p = nullptr;
        st = plan_create(&p, inst[i].N, x0, W, inst[i].fov, inst[i].w_min, inst[i].w_max,
                         flags & (WS_FLAG_NO_Z_OFFSET | WS_FLAG_HERMITIAN | WS_FLAG_DIVIDE_BY_N | WS_FLAG_DETERMINISTIC),
                         false);
        if (st != WS_OK) {
            set_error("ws_batch_create: instance " + std::to_string(i) + ": " + ws_last_error());
            break;
        }
        b->plans.push_back(p);
        b->M.push_back(inst[i].M);
        // plane passes of both transforms plus the gridding work, in bytes moved
        b->cost.push_back(2.0 * (double)p->L.Nw * (double)plane_bytes(p) +
                          (double)inst[i].M * W * W * W * 8.0);
        largest_plane = std::max(largest_plane, plane_bytes(p));
        st = ensure_capacity(p, std::max<int64_t>(inst[i].M, 1), true);
    }
    if (st == WS_OK) {
        size_t want = (size_t)workspace_bytes;
        if (want == 0) {
            size_t free_b = 0, total_b = 0;
            cudaMemGetInfo(&free_b, &total_b);
            want = (size_t)(0.6 * (double)free_b);
            // no more than K slices that each hold the whole stack of the largest instance
            size_t largest_stack = 0;
            for (ws_plan_s *p : b->plans)
                largest_stack = std::max(largest_stack, (size_t)p->L.ntt * TT * plane_bytes(p));
            const int kmax = std::min<int>(branches > 0 ? branches : 4, n);
            want = std::min(want, (size_t)kmax * (largest_stack + 256));
        }
        if (want < (size_t)TT * largest_plane) {
            set_error("ws_batch_create: the workspace cannot hold 8 w-planes of the largest instance");
            st = WS_ERR_OOM;
        } else {
            e = cudaMalloc((void **)&b->workspace, want);
            if (e != cudaSuccess) st = cuda_fail(e, "ws_batch_create: allocating the shared workspace");
            b->workspace_bytes = want;
        }
    }
    if (st == WS_OK) {
        e = cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ready, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->tuned, cudaEventDisableTiming);
        for (int k = 0; k < kMaxBranches && e == cudaSuccess; ++k) {
            e = cudaStreamCreateWithFlags(&b->br[k], cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join[k], cudaEventDisableTiming);
        }
        if (e != cudaSuccess) st = cuda_fail(e, "ws_batch_create: creating streams");
    }
    if (st == WS_OK && branches > 0 && !assign(b, std::min<int>(branches, n))) {
        set_error("ws_batch_create: a workspace slice cannot hold 8 w-planes of its largest instance");
        st = WS_ERR_OOM;
    }
    if (st != WS_OK) {
        const std::string msg = ws_last_error();
        release_batch(b);
        set_error(msg);
        return st;
    }
    *out = b;
    return WS_OK;
}

ws_status ws_batch_grid(ws_batch_t b, const double *const *uvw, const void *const *vis, void *const *dirty,
                        ws_stream_t stream) {
    if (!b || !uvw || !vis || !dirty) {
        set_error("ws_batch_grid: invalid argument");
        return WS_ERR_ARG;
    }
    std::vector<const void *> ptr;
    for (size_t i = 0; i < b->plans.size(); ++i) {
        if (!dirty[i] || (b->M[i] > 0 && (!uvw[i] || !vis[i]))) {
            set_error("ws_batch_grid: NULL pointer for instance " + std::to_string(i));
            return WS_ERR_ARG;
        }
        ptr.push_back(uvw[i]);
        ptr.push_back(vis[i]);
        ptr.push_back(dirty[i]);
    }
    return run(b, 0, ptr, reinterpret_cast<cudaStream_t>(stream));
}

ws_status ws_batch_degrid(ws_batch_t b, const void *const *image, const double *const *uvw, void *const *vis,
                          ws_stream_t stream) {
    if (!b || !image || !uvw || !vis) {
        set_error("ws_batch_degrid: invalid argument");
        return WS_ERR_ARG;
    }
    std::vector<const void *> ptr;
    for (size_t i = 0; i < b->plans.size(); ++i) {
        if (!image[i] || (b->M[i] > 0 && (!uvw[i] || !vis[i]))) {
            set_error("ws_batch_degrid: NULL pointer for instance " + std::to_string(i));
            return WS_ERR_ARG;
        }
        ptr.push_back(image[i]);
        ptr.push_back(uvw[i]);
        ptr.push_back(vis[i]);
    }
    return run(b, 1, ptr, reinterpret_cast<cudaStream_t>(stream));
}

ws_status ws_batch_info(ws_batch_t b, int32_t i, ws_plan_info_t *info, int32_t *branch) {
    if (!b || i < 0 || i >= (int32_t)b->plans.size() || !info) {
        set_error("ws_batch_info: invalid argument");
        return WS_ERR_ARG;
    }
    ws_status st = ws_plan_info(b->plans[i], info);
    if (branch) *branch = b->K > 0 ? b->branch_of[i] : -1;
    return st;
}

ws_status ws_batch_branches(ws_batch_t b, int32_t *branches) {
    if (!b || !branches) {
        set_error("ws_batch_branches: invalid argument");
        return WS_ERR_ARG;
    }
    *branches = b->K;
    return WS_OK;
}

ws_status ws_batch_destroy(ws_batch_t b) {
    release_batch(b);
    return WS_OK;
}

}  // extern "C"
