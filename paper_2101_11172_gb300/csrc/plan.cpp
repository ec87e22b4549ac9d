// Plan construction and the C ABI entry points (host side).
//
// ws_plan   Section 5.3 (Eq. n_params / n_params_no_offset, Eq. N_{w'}+W),
//           Section 5.1 (Eq. z-on-sphere), Section 3.3 (least-misfit C, h)
// ws_grid   Algorithm 5
// ws_degrid Algorithm 6
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>

#include "ws_internal.hpp"

namespace ws {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

ws_status cuda_fail(cudaError_t e, const char *what) {
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? WS_ERR_OOM : WS_ERR_CUDA;
}

namespace {

bool seven_smooth(int64_t n) {
    for (int p : {2, 3, 5, 7})
        while (n % p == 0) n /= p;
    return n == 1;
}

// Smallest multiple of 32 with no prime factor above 7 that is >= N/(2 x0).
int64_t fft_size(int N, double x0) {
    double need = N / (2.0 * x0);
    int64_t n = 32 * std::max<int64_t>(1, (int64_t)std::ceil(need / 32.0 - 1e-12));
    while (!seven_smooth(n)) n += 32;
    return n;
}

// Device-side guard: makes the plan's device current for the call's scope.
struct DeviceScope {
    int prev = -1;
    bool ok = true;
    explicit DeviceScope(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceScope() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

template <typename T>
cudaError_t dev_alloc(T **ptr, size_t count, int64_t *bytes) {
    *ptr = nullptr;
    if (count == 0) return cudaSuccess;
    cudaError_t e = cudaMalloc((void **)ptr, count * sizeof(T));
    if (e == cudaSuccess) *bytes += (int64_t)(count * sizeof(T));
    return e;
}

void release(ws_plan_s *p) {
    if (!p) return;
    DeviceScope scope(p->dev >= 0 ? p->dev : 0);
    for (auto &t : p->pending) {
        cudaEventDestroy(t.start);
        cudaEventDestroy(t.stop);
    }
    for (cudaEvent_t e : p->free_events) cudaEventDestroy(e);
    cudaFree(p->d_wcoef);
    cudaFree(p->d_corr);
    cudaFree(p->d_zsplit);
    cudaFree(p->d_stack);
    cudaFree(p->d_tw);
    cudaFree(p->d_rec);
    cudaFree(p->d_list);
    cudaFree(p->d_counts);
    cudaFree(p->d_offsets);
    cudaFree(p->d_blocksums);
    cudaFree(p->d_acc);
    cudaFree(p->d_tile_occ);
    cudaFree(p->d_col_occ);
    cudaFree(p->d_img);
    cudaFree(p->d_drop);
    cudaFree(p->d_occ_counts);
    cudaFree(p->d_brec);
    cudaFree(p->d_blist_g);
    cudaFree(p->d_blist_d);
    cudaFree(p->d_boff_g);
    cudaFree(p->d_boff_d);
    cudaFree(p->d_btile_occ);
    cudaFree(p->d_bcol_occ);
    cudaFree(p->d_bdrop);
    cudaFree(p->d_cheb64);
    cudaFree(p->d_corr64);
    cudaFree(p->d_z64);
    cudaFree(p->d_plane64);
    cudaFree(p->d_acc64);
    cudaFree(p->d_tw64);
    cudaFree(p->d_rec64);
    if (p->h_drop) cudaFreeHost(p->h_drop);
    if (p->h_occ_counts) cudaFreeHost(p->h_occ_counts);
    delete p;
}

cudaEvent_t take_event(ws_plan_s *p) {
    if (!p->free_events.empty()) {
        cudaEvent_t e = p->free_events.back();
        p->free_events.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

// Fold completed stage events into the statistics (waits for them).
void fold_pending(ws_plan_s *p) {
    for (auto &t : p->pending) {
        float ms = 0.f;
        if (cudaEventSynchronize(t.stop) == cudaSuccess && cudaEventElapsedTime(&ms, t.start, t.stop) == cudaSuccess)
            p->stats.stage_ms[t.stage] += ms;
        p->free_events.push_back(t.start);
        p->free_events.push_back(t.stop);
    }
    p->pending.clear();
}

// Times one stage on the call's stream when the plan has WS_FLAG_TIMING.
struct StageTimer {
    ws_plan_s *p;
    cudaStream_t s;
    int stage;
    cudaEvent_t a = nullptr, b = nullptr;
    StageTimer(ws_plan_s *p_, cudaStream_t s_, int stage_, int launches) : p(p_), s(s_), stage(stage_) {
        p->stats.stage_launches[stage] += launches;
        p->stats.kernel_launches += launches;
        if (!(p->flags & WS_FLAG_TIMING)) return;
        if (p->pending.size() > 4096) fold_pending(p);
        a = take_event(p);
        b = take_event(p);
        if (a && b) cudaEventRecord(a, s);
    }
    ~StageTimer() {
        if (a && b) {
            cudaEventRecord(b, s);
            p->pending.push_back({stage, a, b});
        } else {
            if (a) p->free_events.push_back(a);
            if (b) p->free_events.push_back(b);
        }
    }
};

// Radices of an N'-point transform: 16, 8, 4 for the power of two (N' is a
// multiple of 32, so no radix 2 is needed), then 7, 5, 3; plus the digit
// weights of the first stage's reversal and the shared-memory layout.
bool fft_make_plan(int n, FftPlan *F) {
    int a = 0, m = n;
    while (m % 2 == 0) {
        m /= 2;
        ++a;
    }
    // the power-of-two radices for 2^a (none for radix 2: a = 1 is not possible)
    auto pow2_radix = [](int a) { return (a >= 8 || a == 4 || a == 7) ? 16 : (a == 3 || a == 5 || a == 6) ? 8 : 4; };
    auto pow2_stages = [&](int a) {
        int s = 0;
        for (; a > 0; ++s) {
            if (a == 1) return 99;
            const int r = pow2_radix(a);
            a -= r == 16 ? 4 : (r == 8 ? 3 : 2);
        }
        return s;
    };
    // one factor 2 and one factor 5 make a radix-10 stage where that saves a stage
    // (N' = 5600 = 2^5 5^2 7: 16, 10, 7, 5 instead of 8, 4, 7, 5, 5)
    const bool ten = m % 5 == 0 && a >= 1 && pow2_stages(a - 1) < pow2_stages(a);
    if (ten) {
        --a;
        m /= 5;
    }
    int ns = 0;
    while (a > 0) {
        if (a == 1) return false;
        const int r = pow2_radix(a);
        F->radix[ns++] = r;
        a -= r == 16 ? 4 : (r == 8 ? 3 : 2);
        if (ns >= 8) return false;
    }
    if (ten) F->radix[ns++] = 10;
    for (int p : {7, 5, 3})
        while (m % p == 0) {
            if (ns >= 8) return false;
            F->radix[ns++] = p;
            m /= p;
        }
    if (m != 1) return false;
    F->n = n;
    F->nstages = ns;
    auto log2i = [](int v) {
        int l = 0;
        while ((1 << l) < v) ++l;
        return (1 << l) == v ? l : -1;
    };
    int L = 1;
    for (int i = 0; i < ns; ++i) {
        int xw = 1, gw = 1;
        for (int l = i + 1; l < ns; ++l) xw *= F->radix[l];
        for (int l = 1; l < i; ++l) gw *= F->radix[l];
        F->xw[i] = xw;
        F->gw[i] = gw;
        F->lxw[i] = log2i(xw);
        F->lgw[i] = log2i(gw);
        F->xw_mul[i] = div_mul(xw);
        F->r_mul[i] = div_mul(F->radix[i]);
        F->L_mul[i] = div_mul(L);
        L *= F->radix[i];
    }
    F->logn = log2i(n);
    int shift = 4;
    while ((2 << shift) <= n / F->radix[0]) ++shift;
    F->padshift = shift;
    int len = (n - 1) + ((n - 1) >> shift) + 1;
    F->stride = len + ((8 - len % 16) + 16) % 16;     // == 8 (mod 16)
    return true;
}

// Occupied algorithmic bytes of one call per stage, from the occupancy counts
// the call copied to h_occ_counts.  Per plane, a column pass reads or writes
// the occupied tiles (tv x TU cells each) and the N crop rows of every
// occupied (t-tile, u-strip) strip; a row pass the N rows of the occupied
// strips; gridding writes whole occupied tiles (TT planes) and reads one
// record and one list entry per (visibility, bin) pair; degridding gathers
// from the occupied tiles and reads and writes its output once per chunk.
void add_occupied_bytes(ws_plan_s *p, bool grid, int64_t M) {
    const Launch &L = p->L;
    const double tile_plane = (double)L.tv * TU * sizeof(float2), strip_plane = (double)L.N * TU * sizeof(float2);
    double t_valid = 0.0, s_valid = 0.0, t_full = 0.0;
    for (int tt = 0; tt < L.ntt; ++tt) {
        const double valid = std::min(TT, L.Nw - tt * TT);
        t_valid += valid * p->h_occ_counts[2 * tt];
        s_valid += valid * p->h_occ_counts[2 * tt + 1];
        t_full += (double)TT * p->h_occ_counts[2 * tt];
    }
    const double entries = p->h_occ_counts[2 * L.ntt];
    const double img = (double)L.N * L.N;
    const int nchunks = (L.ntt * TT + p->P - 1) / p->P;
    double *b = p->stats.stage_bytes;
    if (grid) {
        b[WS_STAGE_PREP] += (double)M * (24 + 8 + sizeof(VisRec));
        b[WS_STAGE_GRID3D] += t_full * tile_plane + entries * (sizeof(uint32_t) + sizeof(VisRec));
        b[WS_STAGE_COLS_INV] += t_valid * tile_plane + s_valid * strip_plane;
        b[WS_STAGE_ROWS_INV] += s_valid * strip_plane + img * (sizeof(float2) + sizeof(float) + sizeof(float2)) +
                                (nchunks - 1) * img * 2 * sizeof(float4);
    } else {
        b[WS_STAGE_PREP] += (double)M * (24 + sizeof(VisRec));
        b[WS_STAGE_CORRECT] += img * (sizeof(float2) + sizeof(float) + sizeof(float2));
        b[WS_STAGE_ROWS_FWD] += nchunks * img * 2 * sizeof(float2) + s_valid * strip_plane;
        b[WS_STAGE_COLS_FWD] += s_valid * strip_plane + t_valid * tile_plane;
        b[WS_STAGE_DEGRID3D] += t_valid * tile_plane + entries * (sizeof(uint32_t) + sizeof(VisRec)) +
                                nchunks * (double)M * 2 * sizeof(float2);
    }
}

// Statistics only: occupancy counts of this call to the host (WS_FLAG_TIMING).
cudaError_t copy_occ_counts(ws_plan_s *p, cudaStream_t s) {
    if (!(p->flags & WS_FLAG_TIMING)) return cudaSuccess;
    cudaError_t e = launch_occ_count(p, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(p->h_occ_counts, p->d_occ_counts, (size_t)2 * p->L.ntt * sizeof(uint32_t),
                            cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(p->h_occ_counts + 2 * p->L.ntt, p->d_offsets + p->ntiles, sizeof(uint32_t),
                            cudaMemcpyDeviceToHost, s);
    return e;
}

ws_status finish_call(ws_plan_s *p, cudaStream_t s, bool grid, int64_t M) {
    cudaError_t e = cudaMemcpyAsync(p->h_drop, p->d_drop, kCounters * sizeof(unsigned long long),
                                    cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_fail(e, "reading the drop counters");
    if (p->flags & WS_FLAG_ASYNC) return WS_OK;
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "waiting for the stream");
    p->last_dropped = (int64_t)(p->h_drop[0] + p->h_drop[1]);
    p->stats.waits_timed_out += (int64_t)p->h_drop[2];
    if ((p->flags & WS_FLAG_TIMING) && M > 0) add_occupied_bytes(p, grid, M);
    if (p->h_drop[2]) {
        set_error(std::to_string(p->h_drop[2]) + " device waits for copies gave up; the output is incomplete");
        return WS_ERR_TIMEOUT;
    }
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

}  // namespace

bool tile_rows_fit(const ws_plan_s *p, int tv) {
    return (tv == 16 || tv == 32 || tv == 64) && p->L.Np % tv == 0 &&
           grid_smem_bytes(p->L.W, tv, (p->flags & WS_FLAG_DETERMINISTIC) != 0) <= kMaxGridSmem;
}

ws_status set_tile_rows(ws_plan_s *p, int tv) {
    if (!tile_rows_fit(p, tv)) {
        set_error("tile rows must be 16, 32 or 64, divide N' = " + std::to_string(p->L.Np) +
                  " and give a gridding ring that fits in shared memory (W = " + std::to_string(p->L.W) + ")");
        return WS_ERR_ARG;
    }
    if (tv == p->L.tv) return WS_OK;
    const int ntv = p->L.Np / tv;
    const int64_t ntiles = (int64_t)p->L.ntu * ntv * p->L.ntt;
    if (ntiles + 1 > (int64_t)4096 * 4096) {
        set_error("too many gridding tiles for " + std::to_string(tv) + " rows per tile");
        return WS_ERR_ARG;
    }
    cudaError_t e = cudaDeviceSynchronize();         // the per-tile tables may be in use
    if (e != cudaSuccess) return cuda_fail(e, "re-tiling: synchronize");
    uint32_t **tables32[] = {&p->d_counts, &p->d_offsets, &p->d_boff_g, &p->d_boff_d};
    uint8_t **tables8[] = {&p->d_tile_occ, &p->d_btile_occ};
    for (uint32_t **t : tables32) {
        if (*t) p->bytes -= (p->ntiles + 1) * (int64_t)sizeof(uint32_t);
        cudaFree(*t);
        *t = nullptr;
    }
    for (uint8_t **t : tables8) {
        if (*t) p->bytes -= p->ntiles;
        cudaFree(*t);
        *t = nullptr;
    }
    // the bound set's other buffers are kept; its tables are made again by the next bind
    cudaFree(p->d_bcol_occ);
    cudaFree(p->d_bdrop);
    if (p->d_bcol_occ) p->bytes -= (int64_t)p->L.ntt * p->L.ntu;
    if (p->d_bdrop) p->bytes -= kCounters * (int64_t)sizeof(unsigned long long);
    p->d_bcol_occ = nullptr;
    p->d_bdrop = nullptr;
    p->b_uvw = nullptr;
    p->b_M = -1;
    p->L.tv = tv;
    p->L.tv_log = tv == 16 ? 4 : (tv == 32 ? 5 : 6);
    p->L.ntv = ntv;
    p->ntiles = ntiles;
    if ((e = dev_alloc(&p->d_counts, (size_t)ntiles + 1, &p->bytes)) != cudaSuccess ||
        (e = dev_alloc(&p->d_offsets, (size_t)ntiles + 1, &p->bytes)) != cudaSuccess ||
        (e = dev_alloc(&p->d_tile_occ, (size_t)ntiles, &p->bytes)) != cudaSuccess)
        return cuda_fail(e, "re-tiling: allocating the per-tile tables");
    return WS_OK;
}

// FP64 plans: grow the record buffer to hold M visibilities.
ws_status ensure_capacity64(ws_plan_s *p, int64_t M) {
    const int64_t need = std::max<int64_t>(M, 1);
    if (need <= p->rec64_cap) return WS_OK;
    cudaFree(p->d_rec64);
    p->bytes -= p->rec64_cap * (int64_t)fp64_record_bytes();
    p->rec64_cap = 0;
    p->d_rec64 = nullptr;
    cudaError_t e = cudaMalloc(&p->d_rec64, (size_t)need * fp64_record_bytes());
    if (e != cudaSuccess) return cuda_fail(e, "allocating FP64 visibility records");
    p->bytes += need * (int64_t)fp64_record_bytes();
    p->rec64_cap = need;
    return WS_OK;
}

// Grow the per-call buffers to hold M visibilities.
ws_status ensure_capacity(ws_plan_s *p, int64_t M, bool grid) {
    if (M > p->rec_cap) {
        cudaFree(p->d_rec);
        p->bytes -= p->rec_cap * (int64_t)sizeof(ws::VisRec);
        p->rec_cap = 0;
        cudaError_t e = dev_alloc(&p->d_rec, (size_t)M, &p->bytes);
        if (e != cudaSuccess) return cuda_fail(e, "allocating visibility records");
        p->rec_cap = M;
    }
    // gridding: at most 2 x 2 tile columns per visibility
    const int64_t per = grid ? 4 : 1;
    const int64_t need = M * per;
    if (need > p->list_cap) {
        cudaFree(p->d_list);
        p->bytes -= p->list_cap * 4;
        p->list_cap = 0;
        cudaError_t e = dev_alloc(&p->d_list, (size_t)need, &p->bytes);
        if (e != cudaSuccess) return cuda_fail(e, "allocating bin lists");
        p->list_cap = need;
    }
    return WS_OK;
}

}  // namespace ws

using namespace ws;

extern "C" {

const char *ws_last_error(void) { return g_last_error.c_str(); }

ws_status ws_plan(ws_plan_t *out, int32_t N, double x0, int32_t W, double fov, double w_min, double w_max,
                  uint32_t flags) {
    return ws::plan_create(out, N, x0, W, fov, w_min, w_max, flags, true, 0);
}

ws_status ws_plan_original(ws_plan_t *out, int32_t N, double x0, int32_t W, double fov, double w_min, double w_max,
                           int32_t Nw, uint32_t flags) {
    if (Nw < 1 || W % 2 == 0) {
        if (out) *out = nullptr;
        set_error("ws_plan_original: need Nw >= 1 bins and an odd W");
        return WS_ERR_ARG;
    }
    if (flags & WS_FLAG_NO_Z_OFFSET) {
        if (out) *out = nullptr;
        set_error("ws_plan_original: the original method has no z offset to remove");
        return WS_ERR_ARG;
    }
    return ws::plan_create(out, N, x0, W, fov, w_min, w_max, flags, true, Nw);
}

}  // extern "C"

namespace ws {

ws_status plan_create(ws_plan_s **out, int32_t N, double x0, int32_t W, double fov, double w_min, double w_max,
                      uint32_t flags, bool own_stack, int32_t orig_bins) {
    if (!out) {
        set_error("ws_plan: out is NULL");
        return WS_ERR_ARG;
    }
    *out = nullptr;
    if (N < 16 || N > 4096 || N % 8) {
        set_error("ws_plan: N must be a multiple of 8 in [16, 4096]");
        return WS_ERR_ARG;
    }
    if (!(x0 > 0.0 && x0 <= 0.5)) {
        set_error("ws_plan: need 0 < x0 <= 0.5");
        return WS_ERR_ARG;
    }
    const bool fp64 = (flags & WS_FLAG_FP64) != 0;
    if (W < 1 || W > (fp64 ? kMaxW64 : kMaxW)) {
        set_error(fp64 ? "ws_plan: need 1 <= W <= 14 (FP64 plans)" : "ws_plan: need 1 <= W <= 12 (14 with WS_FLAG_FP64)");
        return WS_ERR_ARG;
    }
    if (fp64 && (orig_bins > 0 || !own_stack)) {
        set_error("ws_plan: WS_FLAG_FP64 is for ws_plan only (not original W-stacking plans or batches)");
        return WS_ERR_ARG;
    }
    const double lmax = 0.5 * fov;
    if (!(fov > 0.0) || !(2.0 * lmax * lmax < 1.0)) {
        set_error("ws_plan: need fov > 0 with the map corner inside the unit circle");
        return WS_ERR_ARG;
    }
    if (!std::isfinite(w_min) || !std::isfinite(w_max) || w_min > w_max) {
        set_error("ws_plan: need finite w_min <= w_max");
        return WS_ERR_ARG;
    }
    if (flags & ~(uint32_t)(WS_FLAG_ASYNC | WS_FLAG_NO_Z_OFFSET | WS_FLAG_TIMING | WS_FLAG_HERMITIAN |
                            WS_FLAG_DIVIDE_BY_N | WS_FLAG_FP64 | WS_FLAG_DETERMINISTIC)) {
        set_error("ws_plan: unknown flag bits");
        return WS_ERR_ARG;
    }
    const int64_t Np = fft_size(N, x0);
    if (Np > 6144) {
        set_error("ws_plan: FFT grid N' = N/(2 x0) rounded up must not exceed 6144");
        return WS_ERR_ARG;
    }
    if (fp64 && ((Np & (Np - 1)) != 0 || Np > 4096)) {
        set_error("ws_plan: FP64 plans need a power-of-two N' <= 4096, got " + std::to_string(Np));
        return WS_ERR_ARG;
    }
    ws_plan_s *p = new (std::nothrow) ws_plan_s;
    if (!p) {
        set_error("ws_plan: out of host memory");
        return WS_ERR_OOM;
    }
    p->flags = flags;
    p->fov = fov;
    p->w_min = w_min;
    p->w_max = w_max;
    p->x0 = N / (2.0 * (double)Np);
    // Eq. n_params: z in [-z0, z0] with z0 = x0 (or Eq. n_params_no_offset: n0 = 1)
    const double r2 = 2.0 * lmax * lmax;
    const double one_minus_nmin = r2 / (1.0 + std::sqrt(1.0 - r2));
    double nscale, n0;
    if (orig_bins > 0) {
        // Algorithms 3 and 4: orig_bins w-bins over the (folded) w-range, phase
        // exp(2 pi i w[t] (n - 1)) so n0 = 1; the w-range is folded first
        double a = w_min, b = w_max;
        if (flags & WS_FLAG_HERMITIAN) {
            if (a < 0.0 && b <= 0.0) {
                const double t = -a;
                a = -b;
                b = t;
            } else if (a < 0.0) {
                b = std::max(-a, b);
                a = 0.0;
            }
        }
        if (!(b > a)) {
            set_error("ws_plan_original: need w_max > w_min");
            delete p;
            return WS_ERR_ARG;
        }
        nscale = orig_bins / (b - a);
        n0 = 1.0;
        // t x z_hi must stay exact in FP32: |z| = |n - 1| / n_scale <= 1/2
        if (one_minus_nmin / nscale > 0.5) {
            set_error("ws_plan_original: fewer bins than 2 (n_max - n_min)(w_max - w_min); Eq. N_w asks for pi times more");
            delete p;
            return WS_ERR_ARG;
        }
    } else if (flags & WS_FLAG_NO_Z_OFFSET) {
        nscale = one_minus_nmin / p->x0;
        n0 = 1.0;
    } else {
        nscale = one_minus_nmin / (2.0 * p->x0);
        n0 = 1.0 - p->x0 * nscale;
    }
    // Section 5.4: with a real sky every w < 0 is folded to -w, so the w-range folds too
    if (flags & WS_FLAG_HERMITIAN) {
        const double a = std::fabs(w_min), b = std::fabs(w_max);
        if (w_min >= 0.0) {
        } else if (w_max <= 0.0) {
            w_min = b;
            w_max = a;
        } else {
            w_min = 0.0;
            w_max = std::max(a, b);
        }
    }
    // planes: first tap of w'_min to last tap of w'_max (Section 3.3 tap rule)
    const long long t_lo = (long long)std::floor(nscale * w_min + 0.5 * W) - (W - 1);
    const long long t_hi = (long long)std::floor(nscale * w_max + 0.5 * W);
    if (t_lo < -2040 || t_hi > 2040 - TT) {
        set_error("ws_plan: w-range needs more than ~4000 w-planes (plane index |t| must stay below 2040)");
        delete p;
        return WS_ERR_ARG;
    }
    Launch &L = p->L;
    L.N = N;
    L.Np = (int)Np;
    L.W = W;
    L.t_lo = (int)t_lo;
    L.Nw = (int)(t_hi - t_lo + 1);
    L.ntu = (int)(Np / TU);
    // TV rows per tile, or 16 where a TV-row gridding ring would not fit in shared memory
    L.tv = grid_smem_bytes(W, TV, (flags & WS_FLAG_DETERMINISTIC) != 0) <= kMaxGridSmem ? TV : 16;
    L.tv_log = L.tv == 16 ? 4 : (L.tv == 32 ? 5 : 6);
    L.ntv = (int)(Np / L.tv);
    L.ntt = (L.Nw + TT - 1) / TT;
    L.uv_scale = Np * (fov / N);
    L.nscale = nscale;
    L.n0m1 = n0 - 1.0;
    L.fold = (flags & WS_FLAG_HERMITIAN) ? 1 : 0;
    p->ntiles = (int64_t)L.ntu * L.ntv * L.ntt;
    if (p->ntiles + 1 > (int64_t)4096 * 4096) {
        set_error("ws_plan: too many gridding tiles (N' x N' x planes too large)");
        delete p;
        return WS_ERR_ARG;
    }

    std::string err;
    if (!fit_least_misfit(W, p->x0, &p->fit, &err)) {
        set_error("ws_plan: " + err);
        delete p;
        return WS_ERR_ARG;
    }
    p->fft_mixed = (Np & (Np - 1)) != 0;
    if (!fft_make_plan((int)Np, &p->fft) || transform_smem_bytes(p->fft, N) > (size_t)227 * 1024) {
        set_error("ws_plan: no transform plan for N' = " + std::to_string(Np));
        delete p;
        return WS_ERR_ARG;
    }
    std::vector<double> mono;
    monomial_weights(p->fit, 1e-10, kMaxDeg, &p->wdeg, &mono);
    // two tables of W x (deg + 1): taps along u and v, then taps along w.  The
    // original method bins in w: only the middle tap (the nearest plane for odd W,
    // Section 3.3 tap rule) carries weight 1.
    p->wcoef_host.assign(mono.begin(), mono.end());
    if (orig_bins > 0) {
        std::vector<float> zt((size_t)W * (p->wdeg + 1), 0.f);
        zt[(size_t)((W - 1) / 2) * (p->wdeg + 1)] = 1.f;
        p->wcoef_host.insert(p->wcoef_host.end(), zt.begin(), zt.end());
    } else {
        p->wcoef_host.insert(p->wcoef_host.end(), mono.begin(), mono.end());
    }
    p->orig_bins = orig_bins;
    {
        // |c_i(nu)| at most wmax over the taps of each table (sampled finely; the weights are
        // smooth), so |C_x C_y C_z| <= wmax_uv^2 wmax_w; 2 % margin for the FP32 evaluation
        const int D1 = p->wdeg + 1;
        double wmax[2] = {0.0, 0.0};
        for (int tab = 0; tab < 2; ++tab)
            for (int i = 0; i < W; ++i)
                for (int k = 0; k <= 2048; ++k) {
                    const double nu = -0.5 + k / 2048.0;
                    double acc = 0.0;
                    for (int m = p->wdeg; m >= 0; --m) acc = acc * nu + p->wcoef_host[((size_t)tab * W + i) * D1 + m];
                    wmax[tab] = std::max(wmax[tab], std::fabs(acc));
                }
        p->wbound = (float)(1.02 * wmax[0] * wmax[0] * wmax[1]);
    }

    // correction image h(x_j) h(y_i) h(z_ij) and the split z_ij (Eq. z-on-sphere)
    const double dl = fov / N;
    std::vector<double> hx(N);
    for (int j = 0; j < N; ++j) hx[j] = h_series(p->fit, (j - N / 2) / (double)Np);
    std::vector<float> corr((size_t)N * N);
    std::vector<float2> zs((size_t)N * N);
    std::vector<double> corr64(fp64 ? (size_t)N * N : 0), z64(fp64 ? (size_t)N * N : 0);
    for (int i = 0; i < N; ++i) {
        const double m = (i - N / 2) * dl;
        for (int j = 0; j < N; ++j) {
            const double l = (j - N / 2) * dl;
            const double rr = l * l + m * m;
            const double nm1 = -rr / (1.0 + std::sqrt(1.0 - rr));
            double z = (nm1 + (1.0 - n0)) / nscale;
            // Section 5.2: the operators act on f = I / n; WS_FLAG_DIVIDE_BY_N folds the 1/n in here
            const double inv_n = (flags & WS_FLAG_DIVIDE_BY_N) ? 1.0 / (1.0 + nm1) : 1.0;
            if (orig_bins > 0) {
                corr[(size_t)i * N + j] = (float)(hx[i] * hx[j] * inv_n);   // Algorithm 3 step 5: 2-D correction
            } else {
                z = std::min(std::max(z, -p->x0), p->x0);
                const double c = hx[i] * hx[j] * h_series(p->fit, z) * inv_n;
                corr[(size_t)i * N + j] = (float)c;
                if (fp64) {
                    corr64[(size_t)i * N + j] = c;
                    z64[(size_t)i * N + j] = z;
                }
            }
            const double hi = std::nearbyint(z * 8192.0) / 8192.0;
            zs[(size_t)i * N + j] = make_float2((float)hi, (float)(z - hi));
        }
    }

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        ws_status st = cuda_fail(e, "ws_plan: no CUDA device");
        delete p;
        return st;
    }
    p->dev = dev;
    if (cudaDeviceGetAttribute(&p->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || p->sms < 1) p->sms = 1;
    const size_t plane_bytes = (size_t)Np * Np * sizeof(float2);
    // planes per chunk: all planes if they fit the budget, else a multiple of TT
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    size_t budget = (size_t)(0.6 * (double)free_b);
    if (const char *env = std::getenv("WS_STACK_BYTES")) budget = (size_t)std::strtoull(env, nullptr, 10);
    int P = fp64 ? 0 : L.ntt * TT;
    if (fp64) own_stack = false;                  // FP64 plans work one plane at a time
    if (const char *env = std::getenv("WS_PLANES_PER_CHUNK")) {
        int want = std::atoi(env);
        if (want > 0) P = std::min(P, std::max(TT, (want / TT) * TT));
    }
    const int fit_planes = (int)std::min<size_t>(budget / plane_bytes, (size_t)1 << 20);
    if (fit_planes < P) P = std::max(TT, (fit_planes / TT) * TT);
    if (fp64) P = 0;
    p->P = own_stack ? P : 0;             // a batch hands the plan a shared stack later

    ws_status st = WS_OK;
    const char *what = nullptr;
#define WS_TRY(call, msg)              \
    do {                               \
        e = (call);                    \
        if (e != cudaSuccess) {        \
            what = msg;                \
            goto fail;                 \
        }                              \
    } while (0)
    WS_TRY(dev_alloc(&p->d_wcoef, p->wcoef_host.size(), &p->bytes), "allocating weight table");
    WS_TRY(cudaMemcpy(p->d_wcoef, p->wcoef_host.data(), p->wcoef_host.size() * sizeof(float),
                      cudaMemcpyHostToDevice), "uploading weight table");
    WS_TRY(dev_alloc(&p->d_corr, corr.size(), &p->bytes), "allocating correction image");
    WS_TRY(cudaMemcpy(p->d_corr, corr.data(), corr.size() * sizeof(float), cudaMemcpyHostToDevice),
           "uploading correction image");
    WS_TRY(dev_alloc(&p->d_zsplit, zs.size(), &p->bytes), "allocating z table");
    WS_TRY(cudaMemcpy(p->d_zsplit, zs.data(), zs.size() * sizeof(float2), cudaMemcpyHostToDevice),
           "uploading z table");
    if (own_stack) WS_TRY(dev_alloc(&p->d_stack, (size_t)P * Np * Np, &p->bytes), "allocating the w-stack chunk");
    {
        std::vector<float2> tw((size_t)Np);
        for (int64_t m = 0; m < Np; ++m) {
            const double ang = 2.0 * 3.14159265358979323846 * (double)m / (double)Np;
            tw[m] = make_float2((float)std::cos(ang), (float)-std::sin(ang));
        }
        WS_TRY(dev_alloc(&p->d_tw, tw.size(), &p->bytes), "allocating twiddles");
        WS_TRY(cudaMemcpy(p->d_tw, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice),
               "uploading twiddles");
    }
    WS_TRY(setup_transform_kernels(p->fft, N), "configuring transform kernels");
    WS_TRY(dev_alloc(&p->d_counts, (size_t)p->ntiles + 1, &p->bytes), "allocating tile counts");
    WS_TRY(dev_alloc(&p->d_offsets, (size_t)p->ntiles + 1, &p->bytes), "allocating tile offsets");
    WS_TRY(dev_alloc(&p->d_blocksums, (size_t)4096, &p->bytes), "allocating scan sums");
    WS_TRY(dev_alloc(&p->d_acc, (size_t)N * N, &p->bytes), "allocating the accumulator");
    WS_TRY(dev_alloc(&p->d_tile_occ, (size_t)p->ntiles, &p->bytes), "allocating tile occupancy");
    WS_TRY(dev_alloc(&p->d_col_occ, (size_t)L.ntt * L.ntu, &p->bytes), "allocating strip occupancy");
    WS_TRY(dev_alloc(&p->d_img, (size_t)N * N, &p->bytes), "allocating the corrected image");
    WS_TRY(dev_alloc(&p->d_drop, (size_t)kCounters, &p->bytes), "allocating drop counters");
    WS_TRY(cudaMallocHost((void **)&p->h_drop, kCounters * sizeof(unsigned long long)), "allocating pinned counters");
    std::memset(p->h_drop, 0, kCounters * sizeof(unsigned long long));
    if (fp64) {
        p->fp64 = true;
        const int D = p->fit.degree;
        std::vector<double> cheb2(p->fit.cheb.begin(), p->fit.cheb.end());
        cheb2.insert(cheb2.end(), p->fit.cheb.begin(), p->fit.cheb.end());
        std::vector<double2> tw64((size_t)Np);
        for (int64_t m = 0; m < Np; ++m) {
            const double ang = 2.0 * 3.14159265358979323846 * (double)m / (double)Np;
            tw64[m] = make_double2(std::cos(ang), -std::sin(ang));
        }
        (void)D;
        WS_TRY(dev_alloc(&p->d_cheb64, cheb2.size(), &p->bytes), "allocating FP64 weights");
        WS_TRY(cudaMemcpy(p->d_cheb64, cheb2.data(), cheb2.size() * sizeof(double), cudaMemcpyHostToDevice),
               "uploading FP64 weights");
        WS_TRY(dev_alloc(&p->d_corr64, corr64.size(), &p->bytes), "allocating FP64 correction");
        WS_TRY(cudaMemcpy(p->d_corr64, corr64.data(), corr64.size() * sizeof(double), cudaMemcpyHostToDevice),
               "uploading FP64 correction");
        WS_TRY(dev_alloc(&p->d_z64, z64.size(), &p->bytes), "allocating FP64 z");
        WS_TRY(cudaMemcpy(p->d_z64, z64.data(), z64.size() * sizeof(double), cudaMemcpyHostToDevice),
               "uploading FP64 z");
        WS_TRY(dev_alloc(&p->d_tw64, tw64.size(), &p->bytes), "allocating FP64 twiddles");
        WS_TRY(cudaMemcpy(p->d_tw64, tw64.data(), tw64.size() * sizeof(double2), cudaMemcpyHostToDevice),
               "uploading FP64 twiddles");
        WS_TRY(dev_alloc(&p->d_plane64, (size_t)Np * Np, &p->bytes), "allocating the FP64 plane");
        WS_TRY(dev_alloc(&p->d_acc64, (size_t)N * N, &p->bytes), "allocating the FP64 accumulator");
        p->fft64_log = 0;
        while ((1LL << p->fft64_log) < Np) ++p->fft64_log;
    }
    if (flags & WS_FLAG_TIMING) {
        WS_TRY(dev_alloc(&p->d_occ_counts, (size_t)2 * L.ntt, &p->bytes), "allocating occupancy counts");
        WS_TRY(cudaMallocHost((void **)&p->h_occ_counts, ((size_t)2 * L.ntt + 1) * sizeof(uint32_t)),
               "allocating pinned occupancy counts");
        std::memset(p->h_occ_counts, 0, ((size_t)2 * L.ntt + 1) * sizeof(uint32_t));
    }
#undef WS_TRY
    // the tuned tile rows for this (GPU, N', W), when a tuning cache is named
    if (const char *cache = std::getenv("WS_TUNE_CACHE")) {
        int tv = 0;
        // an entry that does not fit this plan (rows not dividing N', a ring too large) is ignored
        if (tune_lookup(cache, tune_key(dev, (int)Np, W), &tv) && tv != L.tv && tile_rows_fit(p, tv)) {
            st = set_tile_rows(p, tv);
            if (st != WS_OK) {
                release(p);
                return st;
            }
        }
    }
    *out = p;
    return WS_OK;
fail:
    st = cuda_fail(e, what);
    release(p);
    return st;
}

namespace {

// For the scope of one call on the bound visibility set: the plan's tile
// lists, offsets and occupancy maps (and, for degridding, its records) are
// the bound set's.  A plan serves one call at a time, so the swap is private
// to the call; the destructor puts the per-call buffers back.
struct BoundView {
    ws_plan_s *p;
    bool active;
    VisRec *rec;
    uint32_t *list, *offsets;
    uint8_t *tile_occ, *col_occ;
    BoundView(ws_plan_s *p_, bool active_, bool grid)
        : p(p_), active(active_), rec(p_->d_rec), list(p_->d_list), offsets(p_->d_offsets),
          tile_occ(p_->d_tile_occ), col_occ(p_->d_col_occ) {
        if (!active) return;
        if (!grid) p->d_rec = p->d_brec;
        p->d_list = grid ? p->d_blist_g : p->d_blist_d;
        p->d_offsets = grid ? p->d_boff_g : p->d_boff_d;
        p->d_tile_occ = p->d_btile_occ;
        p->d_col_occ = p->d_bcol_occ;
    }
    ~BoundView() {
        p->d_rec = rec;
        p->d_list = list;
        p->d_offsets = offsets;
        p->d_tile_occ = tile_occ;
        p->d_col_occ = col_occ;
    }
};

bool is_bound(const ws_plan_s *p, const double *uvw, int64_t M) {
    return p->b_uvw != nullptr && uvw == p->b_uvw && M == p->b_M;
}

}  // namespace

ws_status enqueue_grid(ws_plan_s *p, const double *uvw, const float2 *vis, int64_t M, float2 *dirty,
                       cudaStream_t s) {
    const bool bound = is_bound(p, uvw, M);
    cudaError_t e = bound ? cudaMemcpyAsync(p->d_drop, p->d_bdrop, kCounters * sizeof(unsigned long long),
                                            cudaMemcpyDeviceToDevice, s)
                          : cudaMemsetAsync(p->d_drop, 0, kCounters * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return cuda_fail(e, "ws_grid: clearing counters");
    p->stats.calls += 1;
    if (bound) {
        // the bound set's records, with this call's values and the gridding pre-phase
        StageTimer t(p, s, WS_STAGE_PREP, M > 0 ? 1 : 0);
        if ((e = launch_bound_grid_records(p, uvw, vis, M, s)) != cudaSuccess)
            return cuda_fail(e, "ws_grid: bound records kernel");
    } else {
        {
            StageTimer t(p, s, WS_STAGE_PREP, M > 0 ? 1 : 0);
            if ((e = launch_prep(p, uvw, vis, M, true, s)) != cudaSuccess) return cuda_fail(e, "ws_grid: prep kernel");
        }
        StageTimer t(p, s, WS_STAGE_BIN, (M > 0 ? 6 : 3) + ((p->flags & WS_FLAG_TIMING) ? 1 : 0));
        if ((e = launch_bin(p, M, true, s)) != cudaSuccess) return cuda_fail(e, "ws_grid: binning kernels");
    }
    BoundView view(p, bound, true);
    if ((e = copy_occ_counts(p, s)) != cudaSuccess) return cuda_fail(e, "ws_grid: occupancy statistics");
    // test knob: the poll limit of inv_rows' first wait for each plane's row copy
    p->wait_polls = kWaitPolls;
    if (const char *env = std::getenv("WS_WAIT_POLLS")) {
        const long v = std::strtol(env, nullptr, 10);
        if (v >= 0 && v < kWaitPolls) p->wait_polls = (int)v;
    }
    const int total = p->L.ntt * TT;
    const int nchunks = (total + p->P - 1) / p->P;
    for (int c = 0; c < nchunks; ++c) {
        const int planes = std::min(p->P, total - c * p->P);
        {
            StageTimer t(p, s, WS_STAGE_GRID3D, 1);
            if ((e = launch_grid_chunk(p, c, planes, s)) != cudaSuccess)
                return cuda_fail(e, "ws_grid: grid3d kernel");
        }
        {
            StageTimer t(p, s, WS_STAGE_COLS_INV, 1);
            if ((e = launch_inv_cols(p, c, planes, s)) != cudaSuccess)
                return cuda_fail(e, "ws_grid: inv_cols kernel");
        }
        {
            StageTimer t(p, s, WS_STAGE_ROWS_INV, 1);
            if ((e = launch_inv_rows(p, c, planes, c == 0, c == nchunks - 1, dirty, s)) != cudaSuccess)
                return cuda_fail(e, "ws_grid: inv_rows kernel");
        }
    }
    return WS_OK;
}

ws_status enqueue_degrid(ws_plan_s *p, const float2 *image, const double *uvw, int64_t M, float2 *vis,
                         cudaStream_t s) {
    const bool bound = is_bound(p, uvw, M);
    cudaError_t e = bound ? cudaMemcpyAsync(p->d_drop, p->d_bdrop, kCounters * sizeof(unsigned long long),
                                            cudaMemcpyDeviceToDevice, s)
                          : cudaMemsetAsync(p->d_drop, 0, kCounters * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return cuda_fail(e, "ws_degrid: clearing counters");
    if (M == 0) return WS_OK;
    if ((e = cudaMemsetAsync(vis, 0, (size_t)M * sizeof(float2), s)) != cudaSuccess)
        return cuda_fail(e, "ws_degrid: clearing the output");
    p->stats.calls += 1;
    if (!bound) {
        {
            StageTimer t(p, s, WS_STAGE_PREP, 1);
            if ((e = launch_prep(p, uvw, nullptr, M, false, s)) != cudaSuccess)
                return cuda_fail(e, "ws_degrid: prep kernel");
        }
        StageTimer t(p, s, WS_STAGE_BIN, 6 + ((p->flags & WS_FLAG_TIMING) ? 1 : 0));
        if ((e = launch_bin(p, M, false, s)) != cudaSuccess) return cuda_fail(e, "ws_degrid: binning kernels");
    }
    BoundView view(p, bound, false);
    if ((e = copy_occ_counts(p, s)) != cudaSuccess) return cuda_fail(e, "ws_degrid: occupancy statistics");
    {
        StageTimer t(p, s, WS_STAGE_CORRECT, 1);
        if ((e = launch_correct_image(p, image, s)) != cudaSuccess)
            return cuda_fail(e, "ws_degrid: correction kernel");
    }
    const int total = p->L.ntt * TT;
    const int nchunks = (total + p->P - 1) / p->P;
    for (int c = 0; c < nchunks; ++c) {
        const int planes = std::min(p->P, total - c * p->P);
        {
            StageTimer t(p, s, WS_STAGE_ROWS_FWD, 1);
            if ((e = launch_fwd_rows(p, c, planes, s)) != cudaSuccess)
                return cuda_fail(e, "ws_degrid: fwd_rows kernel");
        }
        {
            StageTimer t(p, s, WS_STAGE_COLS_FWD, 1);
            if ((e = launch_fwd_cols(p, c, planes, s)) != cudaSuccess)
                return cuda_fail(e, "ws_degrid: fwd_cols kernel");
        }
        {
            StageTimer t(p, s, WS_STAGE_DEGRID3D, 1);
            if ((e = launch_degrid_chunk(p, c, planes, M, vis, s)) != cudaSuccess)
                return cuda_fail(e, "ws_degrid: degrid3d kernel");
        }
    }
    if (p->L.fold && (e = launch_unfold(p, uvw, M, vis, s)) != cudaSuccess)
        return cuda_fail(e, "ws_degrid: unfolding kernel");
    return WS_OK;
}

}  // namespace ws

extern "C" {

ws_status ws_grid(ws_plan_t plan, const double *uvw, const void *vis, int64_t M, void *dirty,
                  ws_stream_t stream) {
    if (!plan || M < 0 || !dirty || (M > 0 && (!uvw || !vis)) || M > kMaxVis) {
        set_error("ws_grid: invalid argument");
        return WS_ERR_ARG;
    }
    ws_plan_s *p = plan;
    DeviceScope scope(p->dev);
    if (!scope.ok) {
        set_error("ws_grid: cannot select the plan's device");
        return WS_ERR_CUDA;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (p->fp64) {
        ws_status st = ensure_capacity64(p, M);
        if (st != WS_OK) return st;
        st = enqueue_grid64(p, uvw, static_cast<const double2 *>(vis), M, static_cast<double2 *>(dirty), s);
        if (st != WS_OK) return st;
        return finish_call(p, s, true, 0);
    }
    ws_status st = ensure_capacity(p, std::max<int64_t>(M, 1), true);
    if (st != WS_OK) return st;
    st = enqueue_grid(p, uvw, static_cast<const float2 *>(vis), M, static_cast<float2 *>(dirty), s);
    if (st != WS_OK) return st;
    return finish_call(p, s, true, M);
}

ws_status ws_degrid(ws_plan_t plan, const void *image, const double *uvw, int64_t M, void *vis,
                    ws_stream_t stream) {
    if (!plan || M < 0 || !image || (M > 0 && (!uvw || !vis)) || M > kMaxVis) {
        set_error("ws_degrid: invalid argument");
        return WS_ERR_ARG;
    }
    ws_plan_s *p = plan;
    DeviceScope scope(p->dev);
    if (!scope.ok) {
        set_error("ws_degrid: cannot select the plan's device");
        return WS_ERR_CUDA;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (p->fp64) {
        ws_status st = ensure_capacity64(p, M);
        if (st != WS_OK) return st;
        st = enqueue_degrid64(p, static_cast<const double2 *>(image), uvw, M, static_cast<double2 *>(vis), s);
        if (st != WS_OK) return st;
        return finish_call(p, s, false, 0);
    }
    ws_status st = ensure_capacity(p, std::max<int64_t>(M, 1), false);
    if (st != WS_OK) return st;
    st = enqueue_degrid(p, static_cast<const float2 *>(image), uvw, M, static_cast<float2 *>(vis), s);
    if (st != WS_OK) return st;
    return finish_call(p, s, false, M);
}

ws_status ws_plan_dropped(ws_plan_t plan, int64_t *dropped) {
    if (!plan || !dropped) {
        set_error("ws_plan_dropped: invalid argument");
        return WS_ERR_ARG;
    }
    DeviceScope scope(plan->dev);
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "ws_plan_dropped: synchronize");
    plan->last_dropped = (int64_t)(plan->h_drop[0] + plan->h_drop[1]);
    *dropped = plan->last_dropped;
    return WS_OK;
}

ws_status ws_plan_bind_uvw(ws_plan_t plan, const double *uvw, int64_t M, ws_stream_t stream) {
    if (!plan || M < 0 || M > kMaxVis) {
        set_error("ws_plan_bind_uvw: invalid argument");
        return WS_ERR_ARG;
    }
    ws_plan_s *p = plan;
    if (p->fp64) {
        set_error("ws_plan_bind_uvw: not for FP64 plans");
        return WS_ERR_ARG;
    }
    p->b_uvw = nullptr;                      // invalid until the new set is complete
    p->b_M = -1;
    if (!uvw) return WS_OK;
    DeviceScope scope(p->dev);
    if (!scope.ok) {
        set_error("ws_plan_bind_uvw: cannot select the plan's device");
        return WS_ERR_CUDA;
    }
    const int64_t Mc = std::max<int64_t>(M, 1);
    const int64_t per = 4;                                         // tile columns per visibility, at most
    cudaError_t e = cudaSuccess;
    auto grow = [&](auto **ptr, int64_t *cap, int64_t need, const char *what) -> bool {
        if (need <= *cap) return true;
        cudaFree(*ptr);
        p->bytes -= *cap * (int64_t)sizeof(**ptr);
        *cap = 0;
        if ((e = dev_alloc(ptr, (size_t)need, &p->bytes)) != cudaSuccess) {
            cuda_fail(e, what);
            return false;
        }
        *cap = need;
        return true;
    };
    if (!grow(&p->d_brec, &p->brec_cap, Mc, "ws_plan_bind_uvw: allocating records") ||
        !grow(&p->d_blist_g, &p->blist_g_cap, Mc * per, "ws_plan_bind_uvw: allocating gridding lists") ||
        !grow(&p->d_blist_d, &p->blist_d_cap, Mc, "ws_plan_bind_uvw: allocating degridding lists"))
        return e == cudaErrorMemoryAllocation ? WS_ERR_OOM : WS_ERR_CUDA;
    if (!p->d_boff_g) {
        const char *what = nullptr;
        if ((e = dev_alloc(&p->d_boff_g, (size_t)p->ntiles + 1, &p->bytes)) != cudaSuccess) what = "offsets";
        else if ((e = dev_alloc(&p->d_boff_d, (size_t)p->ntiles + 1, &p->bytes)) != cudaSuccess) what = "offsets";
        else if ((e = dev_alloc(&p->d_btile_occ, (size_t)p->ntiles, &p->bytes)) != cudaSuccess) what = "occupancy";
        else if ((e = dev_alloc(&p->d_bcol_occ, (size_t)p->L.ntt * p->L.ntu, &p->bytes)) != cudaSuccess) what = "occupancy";
        else if ((e = dev_alloc(&p->d_bdrop, (size_t)kCounters, &p->bytes)) != cudaSuccess) what = "counters";
        if (what) {
            ws_status st = cuda_fail(e, "ws_plan_bind_uvw: allocating the bound set's tables");
            cudaFree(p->d_boff_g);
            cudaFree(p->d_boff_d);
            cudaFree(p->d_btile_occ);
            cudaFree(p->d_bcol_occ);
            cudaFree(p->d_bdrop);
            p->d_boff_g = p->d_boff_d = nullptr;
            p->d_btile_occ = p->d_bcol_occ = nullptr;
            p->d_bdrop = nullptr;
            return st;
        }
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if ((e = cudaMemsetAsync(p->d_drop, 0, kCounters * sizeof(unsigned long long), s)) != cudaSuccess)
        return cuda_fail(e, "ws_plan_bind_uvw: clearing counters");
    {
        // records in the degridding form, both directions' lists and the occupancy,
        // written straight into the bound set's buffers
        VisRec *rec = p->d_rec;
        uint32_t *list = p->d_list, *offsets = p->d_offsets;
        uint8_t *tile_occ = p->d_tile_occ, *col_occ = p->d_col_occ;
        p->d_rec = p->d_brec;
        p->d_list = p->d_blist_g;
        p->d_offsets = p->d_boff_g;
        p->d_tile_occ = p->d_btile_occ;
        p->d_col_occ = p->d_bcol_occ;
        e = launch_prep(p, uvw, nullptr, M, false, s);
        if (e == cudaSuccess) e = launch_bin(p, M, true, s);
        p->d_list = p->d_blist_d;
        p->d_offsets = p->d_boff_d;
        if (e == cudaSuccess) e = launch_bin(p, M, false, s);
        p->d_rec = rec;
        p->d_list = list;
        p->d_offsets = offsets;
        p->d_tile_occ = tile_occ;
        p->d_col_occ = col_occ;
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(p->d_bdrop, p->d_drop, kCounters * sizeof(unsigned long long), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "ws_plan_bind_uvw: pre-processing and binning");
    p->b_uvw = uvw;
    p->b_M = M;
    return WS_OK;
}

ws_status ws_plan_stats(ws_plan_t plan, ws_stats_t *stats, int32_t reset) {
    if (!plan || !stats) {
        set_error("ws_plan_stats: invalid argument");
        return WS_ERR_ARG;
    }
    DeviceScope scope(plan->dev);
    fold_pending(plan);
    *stats = plan->stats;
    if (reset) plan->stats = ws_stats_t{};
    return WS_OK;
}

ws_status ws_plan_info(ws_plan_t plan, ws_plan_info_t *info) {
    if (!plan || !info) {
        set_error("ws_plan_info: invalid argument");
        return WS_ERR_ARG;
    }
    info->N = plan->L.N;
    info->Np = plan->L.Np;
    info->W = plan->L.W;
    info->Nw = plan->L.Nw;
    info->t_lo = plan->L.t_lo;
    info->planes_per_chunk = plan->P;
    info->x0 = plan->x0;
    info->n0 = plan->L.n0m1 + 1.0;
    info->nscale = plan->L.nscale;
    info->error_bound = plan->fit.E;
    info->workspace_bytes = plan->bytes;
    info->tile_rows = plan->L.tv;
    return WS_OK;
}

ws_status ws_destroy(ws_plan_t plan) {
    if (!plan) return WS_OK;
    {
        DeviceScope scope(plan->dev);
        cudaDeviceSynchronize();
    }
    release(plan);
    return WS_OK;
}

}  // extern "C"
