// Tuning of the plan's gridding tile (ws_plan_tune) and its result cache.
//
// The rows per gridding tile (16, 32 or 64) trade the number of (visibility,
// tile) entries against shared memory per CTA and the granularity of the
// stack's occupancy: fewer rows give more CTAs per SM and a finer skip of
// empty tiles in the column transforms, more rows split fewer footprints.
// The same tiles bin the visibilities for degridding.  The best choice
// depends on N', W, the visibility distribution and the GPU, so it is
// measured: the tuner times one ws_grid plus one ws_degrid on the caller's
// data for every candidate and keeps the fastest.
//
// The cache is a small JSON object, one entry per "<GPU name>|N'=<N'>|W=<W>":
//   {"NVIDIA GB300|N'=4096|W=7": {"tile_rows": 32, "ms": {"16": 71.2, "32": 66.9, "64": 68.4}}}
// ws_plan_tune reads and writes it; ws_plan and ws_batch_create apply the
// entry for their (N', W) when the environment variable WS_TUNE_CACHE names
// such a file.
#include <cuda_runtime.h>
#include <unistd.h>

#include <cstdio>
#include <cstdlib>
#include <fstream>
#include <sstream>
#include <string>

#include "ws_internal.hpp"

namespace ws {
namespace {

std::string read_file(const char *path) {
    std::ifstream f(path, std::ios::binary);
    if (!f) return std::string();
    std::ostringstream ss;
    ss << f.rdbuf();
    return ss.str();
}

// Position of the value object of "key" in the cache text, or npos.
size_t find_entry(const std::string &text, const std::string &key) {
    const std::string quoted = "\"" + key + "\"";
    size_t at = text.find(quoted);
    if (at == std::string::npos) return std::string::npos;
    at = text.find('{', at + quoted.size());
    return at;
}

// The entry's object text {...} (no nested braces beyond one level).
std::string entry_text(const std::string &text, size_t open) {
    int depth = 0;
    for (size_t i = open; i < text.size(); ++i) {
        if (text[i] == '{') ++depth;
        if (text[i] == '}' && --depth == 0) return text.substr(open, i - open + 1);
    }
    return std::string();
}

}  // namespace

std::string tune_key(int dev, int Np, int W) {
    cudaDeviceProp prop{};
    std::string name = "unknown GPU";
    if (cudaGetDeviceProperties(&prop, dev) == cudaSuccess) name = prop.name;
    for (char &c : name)
        if (c == '"' || c == '\\' || c == '|') c = ' ';
    return name + "|N'=" + std::to_string(Np) + "|W=" + std::to_string(W);
}

bool tune_lookup(const char *path, const std::string &key, int *tile_rows) {
    if (!path || !*path) return false;
    const std::string text = read_file(path);
    const size_t open = find_entry(text, key);
    if (open == std::string::npos) return false;
    const std::string e = entry_text(text, open);
    const size_t at = e.find("\"tile_rows\"");
    if (at == std::string::npos) return false;
    const size_t colon = e.find(':', at);
    if (colon == std::string::npos) return false;
    const int v = std::atoi(e.c_str() + colon + 1);
    if (v != 16 && v != 32 && v != 64) return false;
    *tile_rows = v;
    return true;
}

bool tune_store(const char *path, const std::string &key, int tile_rows, const int *cand, const float *ms, int n) {
    std::string text = read_file(path);
    std::ostringstream entry;
    entry << "{\"tile_rows\": " << tile_rows << ", \"ms\": {";
    for (int i = 0; i < n; ++i) entry << (i ? ", " : "") << "\"" << cand[i] << "\": " << ms[i];
    entry << "}}";
    const size_t open = find_entry(text, key);
    if (open != std::string::npos) {
        const std::string old = entry_text(text, open);
        text.replace(open, old.size(), entry.str());
    } else {
        const size_t close = text.rfind('}');
        const bool empty = text.find('"') == std::string::npos;
        const std::string item = "\"" + key + "\": " + entry.str();
        if (close == std::string::npos) text = "{\n " + item + "\n}\n";
        else text = text.substr(0, close) + (empty ? " " : ",\n ") + item + "\n}\n";
    }
    const std::string tmp = std::string(path) + ".tmp" + std::to_string((long)getpid());
    {
        std::ofstream f(tmp, std::ios::binary | std::ios::trunc);
        if (!f) return false;
        f << text;
        if (!f) return false;
    }
    return std::rename(tmp.c_str(), path) == 0;
}

}  // namespace ws

using namespace ws;

extern "C" ws_status ws_plan_tune(ws_plan_t plan, const double *uvw, const void *vis, const void *image, int64_t M,
                                  const char *cache_path, ws_stream_t stream, int32_t *tile_rows) {
    if (!plan || M <= 0 || M > kMaxVis || !uvw || !vis || !image) {
        set_error("ws_plan_tune: invalid argument");
        return WS_ERR_ARG;
    }
    ws_plan_s *p = plan;
    if (p->fp64) {
        set_error("ws_plan_tune: not for FP64 plans");
        return WS_ERR_ARG;
    }
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != p->dev && cudaSetDevice(p->dev) != cudaSuccess) {
        set_error("ws_plan_tune: cannot select the plan's device");
        return WS_ERR_CUDA;
    }
    struct Restore {
        int prev, dev;
        ~Restore() {
            if (prev >= 0 && prev != dev) cudaSetDevice(prev);
        }
    } restore{prev, p->dev};
    const std::string key = tune_key(p->dev, p->L.Np, p->L.W);
    int best = 0;
    if (tune_lookup(cache_path, key, &best) && tile_rows_fit(p, best)) {
        const ws_status st = set_tile_rows(p, best);
        if (st == WS_OK && tile_rows) *tile_rows = best;
        return st;
    }
    int cand[3], n = 0;
    for (int c : {16, 32, 64})
        if (tile_rows_fit(p, c)) cand[n++] = c;
    float ms[3] = {0.f, 0.f, 0.f};
    float2 *dirty = nullptr, *vout = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc((void **)&dirty, (size_t)p->L.N * p->L.N * sizeof(float2));
    if (e == cudaSuccess) e = cudaMalloc((void **)&vout, (size_t)M * sizeof(float2));
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    ws_status st = e == cudaSuccess ? WS_OK : cuda_fail(e, "ws_plan_tune: allocating scratch");
    const ws_stats_t saved = p->stats;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    auto ok = [](ws_status x) { return x == WS_OK || x == WS_ERR_UV_RANGE || x == WS_ERR_W_RANGE; };
    for (int i = 0; i < n && st == WS_OK; ++i) {
        st = set_tile_rows(p, cand[i]);
        if (st != WS_OK) break;
        // one untimed pass (buffers grown, kernels loaded), then one timed
        ws_status a = ws_grid(p, uvw, vis, M, dirty, stream);
        ws_status b = ok(a) ? ws_degrid(p, image, uvw, M, vout, stream) : a;
        if (!ok(b)) {
            st = b;
            break;
        }
        e = cudaEventRecord(e0, s);
        a = ws_grid(p, uvw, vis, M, dirty, stream);
        b = ok(a) ? ws_degrid(p, image, uvw, M, vout, stream) : a;
        if (!ok(b)) {
            st = b;
            break;
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms[i], e0, e1);
        if (e != cudaSuccess) st = cuda_fail(e, "ws_plan_tune: timing a tile shape");
    }
    p->stats = saved;
    if (st == WS_OK) {
        int k = 0;
        for (int i = 1; i < n; ++i)
            if (ms[i] < ms[k]) k = i;
        best = cand[k];
        st = set_tile_rows(p, best);
        if (st == WS_OK && cache_path && *cache_path && !tune_store(cache_path, key, best, cand, ms, n)) {
            set_error(std::string("ws_plan_tune: cannot write the tuning cache ") + cache_path);
            st = WS_ERR_ARG;
        }
        if (tile_rows) *tile_rows = best;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(dirty);
    cudaFree(vout);
    return st;
}
