/* ws.h -- C ABI of the GB300 improved W-stacking gridder/degridder.
 *
 * Implements the hot path of Ye, Gull, Tan & Nikolic 2021, "High accuracy
 * wide field imaging method in radio interferometry":
 *   ws_degrid  Algorithm 6 (model image -> visibilities, 3-D degridding)
 *   ws_grid    Algorithm 5 (visibilities -> dirty image, 3-D gridding)
 * with least-misfit gridding functions C and corrections h (Section 3.3) in
 * all three directions, W_x = W_y = W_z = W and x0 = y0 = z0.
 *
 * Normalisation.  Both operators are plain sums (no 1/M natural weighting,
 * no 2 l_max or 4 l_max m_max factor, unnormalised FFTs), approximating
 *   degrid: V_k    = sum_{i,j} f[i][j] exp(-2 pi i (u_k l_j + v_k m_i + w_k (n_ij - 1)))
 *   grid:   d[i][j] = sum_k V_k    exp(+2 pi i (u_k l_j + v_k m_i + w_k (n_ij - 1)))
 * (Eq. fourier_visibility and its adjoint), so that they are exact adjoints
 * of each other: <ws_degrid(f), V> = <f, ws_grid(V)> under the plain complex
 * inner products, up to FP32 rounding.  f is the sky brightness divided by n
 * (Section 5.2); the caller applies weights and scale factors.
 *
 * Coordinates.  Image pixel [i][j] (row i along m, column j along l, both
 * -N/2..N/2-1 after subtracting N/2) sits at l_j = (j - N/2) fov/N,
 * m_i = (i - N/2) fov/N; n_ij = sqrt(1 - l^2 - m^2).  uvw are in wavelengths.
 *
 * Memory.  Every data pointer is DEVICE memory owned by the caller; the
 * library never frees it.  Images are complex64 (interleaved float re, im)
 * N x N row-major; visibilities complex64 length M; uvw double M x 3
 * (u, v, w per row).  The plan owns its tables and workspace (device memory
 * it allocates and frees).
 *
 * Streams.  Work is enqueued on the given stream (0 = legacy default
 * stream).  Unless the plan was made with WS_FLAG_ASYNC, each call ends by
 * waiting for its stream and reading back the count of visibilities it had
 * to drop; WS_FLAG_ASYNC skips that wait and the count is available from
 * ws_plan_dropped().  A plan must not be used by two calls at once.
 *
 * Errors.  Nothing aborts or traps.  Every function returns a ws_status;
 * ws_last_error() returns a message for the calling thread's latest failure.
 */
#ifndef WS_H
#define WS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ws_plan_s *ws_plan_t;
typedef struct CUstream_st *ws_stream_t;   /* the same type as cudaStream_t */

typedef enum {
    WS_OK = 0,
    WS_ERR_ARG = 1,        /* invalid argument or plan parameters */
    WS_ERR_UV_RANGE = 2,   /* a u or v was not finite (NaN/inf); those visibilities were dropped */
    WS_ERR_W_RANGE = 3,    /* a w fell outside the plan's [w_min, w_max]; those were dropped */
    WS_ERR_CUDA = 4,       /* a CUDA call failed */
    WS_ERR_OOM = 5,        /* device memory could not be allocated */
    WS_ERR_TIMEOUT = 6     /* a bounded device wait gave up */
} ws_status;

enum {
    WS_FLAG_ASYNC = 1u << 0,       /* do not wait for the stream at the end of each call */
    WS_FLAG_NO_Z_OFFSET = 1u << 1, /* Eq. n_params_no_offset: n0 = 1, z in [-z0, 0] */
    WS_FLAG_TIMING = 1u << 2,      /* record CUDA events around every stage (see ws_plan_stats) */
    WS_FLAG_HERMITIAN = 1u << 3,   /* real sky (Section 5.4): a visibility at w < 0 is handled as the
                                      conjugate visibility at (-u, -v, -w), so only |w| needs planes.
                                      ws_degrid reads only the real part of the image; ws_grid returns
                                      the real dirty image Re(sum_k V_k exp(+2 pi i ...)) with a zero
                                      imaginary part.  The plan's w-range is folded the same way. */
    WS_FLAG_DIVIDE_BY_N = 1u << 4, /* images are the sky brightness I rather than f = I / n (Section 5.2):
                                      ws_degrid uses I / n and ws_grid returns its dirty image divided
                                      by n, which keeps the two adjoint */
    WS_FLAG_FP64 = 1u << 5,        /* everything in double precision, for measuring the method's error
                                      where it falls below FP32 rounding (W up to 14, Section 6.3):
                                      images, visibilities and dirty images are complex128 (interleaved
                                      double re, im), the weights, w-stack, transforms, screens and sums
                                      FP64.  Plain per-plane kernels, not tuned for throughput (their
                                      gridding sums with FP64 atomics, so it is reproducible to FP64
                                      rounding, not bit for bit); N' must be a power of two <= 4096.  Not for ws_plan_original, batches,
                                      ws_plan_bind_uvw, ws_plan_tune or ws_degrid_noalloc. */
    WS_FLAG_DETERMINISTIC = 1u << 6 /* bit-for-bit reproducible gridding: each gridding CTA sums its tile
                                      column in 64-bit fixed point (a power-of-two scale per column keeps
                                      every sum below 2^62, resolution about 1e-19 of the column's largest
                                      possible sum), so ws_grid's dirty image does not depend on the order
                                      of the visibilities or of the GPU's atomics.  Slower gridding (twice
                                      the shared memory per CTA); degridding is deterministic anyway.  For
                                      the FP32 path (not WS_FLAG_FP64 plans). */
};

/* Stages of one call, in execution order (Algorithm 5 / Algorithm 6 steps). */
enum {
    WS_STAGE_PREP = 0,      /* scale u, v, w; first taps; offsets nu; pre-phase */
    WS_STAGE_BIN,           /* counting sort of visibilities into bins; stack occupancy */
    WS_STAGE_GRID3D,        /* Alg. 5 steps 2-3a: 3-D least-misfit gridding into the w-stack */
    WS_STAGE_COLS_INV,      /* Alg. 5 steps 3b-3c, first half: inverse DFT along v, crop rows */
    WS_STAGE_ROWS_INV,      /* Alg. 5 steps 3b-5, second half: inverse DFT along u, crop,
                               w-screen, sum over planes, correction */
    WS_STAGE_CORRECT,       /* Alg. 6 step 2: image x correction */
    WS_STAGE_ROWS_FWD,      /* Alg. 6 steps 3a-3c, first half: w-screen, zero pad, DFT along l */
    WS_STAGE_COLS_FWD,      /* Alg. 6 step 3c, second half: zero pad, DFT along m */
    WS_STAGE_DEGRID3D,      /* Alg. 6 steps 4-5: 3-D correlation with C, post-phase */
    WS_NSTAGES
};

typedef struct {
    int64_t calls;                     /* ws_grid + ws_degrid calls since the last reset */
    int64_t kernel_launches;           /* kernel launches of the counted calls */
    double stage_ms[WS_NSTAGES];       /* device time per stage (WS_FLAG_TIMING plans only) */
    int64_t stage_launches[WS_NSTAGES];/* kernel launches per stage */
    double stage_bytes[WS_NSTAGES];    /* occupied algorithmic bytes per stage (WS_FLAG_TIMING plans,
                                          calls that wait for their stream): the bytes each stage must
                                          move for the w-stack tiles and column strips that some
                                          visibility footprint touches (every other stack cell is zero
                                          in gridding and never read in degridding), plus its inputs
                                          and outputs; 0 for the binning stage */
    int64_t waits_timed_out;           /* bounded device waits that gave up (WS_ERR_TIMEOUT calls) */
} ws_stats_t;

typedef struct {
    int32_t N;             /* image side */
    int32_t Np;            /* FFT grid side N' (multiple of 32, 7-smooth, >= N/(2 x0)) */
    int32_t W;             /* kernel width in u, v and w */
    int32_t Nw;            /* number of w-planes (Eq. N_{w'}+W, exact for the w-range) */
    int32_t t_lo;          /* first plane index t (plane t sits at w = t / n_scale) */
    int32_t planes_per_chunk;  /* planes held in device memory at once */
    double x0;             /* effective cropping parameter N/(2 N') = y0 = z0 */
    double n0;             /* Eq. n_params */
    double nscale;         /* Eq. n_params */
    double error_bound;    /* E of Eq. norm_bound for (W, x0) from the plan's own fit */
    int64_t workspace_bytes;   /* device bytes the plan currently holds */
    int32_t tile_rows;     /* grid rows per gridding tile: 16 unless tuned (ws_plan_tune) */
} ws_plan_info_t;

/* Build a plan.
 *   N       image side, a multiple of 8, 16..4096
 *   x0      image cropping parameter, 0 < x0 <= 0.5 (Section 3.3 box); N' is
 *           rounded up, so the effective x0 = N/(2 N') <= x0; N' <= 6144
 *   W       least-misfit kernel width, 1..12 (1..14 with WS_FLAG_FP64)
 *   fov     full field of view in direction cosines (l, m in [-fov/2, fov/2)),
 *           0 < fov and (fov/2)^2 * 2 < 1
 *   w_min, w_max  the w-range (wavelengths) every later call must respect
 *   flags   WS_FLAG_*
 * Fits C and h (Section 3.3), sizes the w-stack (Section 5.3), uploads the
 * correction image h_x h_y h_z(z(x, y)) (Algorithm 5 step 5) and z(x, y)
 * (Eq. z-on-sphere) to the current CUDA device.  Returns WS_ERR_ARG for bad
 * parameters, WS_ERR_OOM / WS_ERR_CUDA on device failures; *out is set only on
 * success. */
ws_status ws_plan(ws_plan_t *out, int32_t N, double x0, int32_t W, double fov,
                  double w_min, double w_max, uint32_t flags);

/* The original W-stacking (Algorithms 3 and 4), for comparison with the
 * improved method: Nw w-bins of equal width over [w_min, w_max] (folded first
 * under WS_FLAG_HERMITIAN), each visibility in its nearest bin, 2-D
 * least-misfit gridding of width W in u and v, bin phase
 * exp(2 pi i w[t] (n - 1)) and the 2-D correction h_x h_y only.  Bins are
 * centred on multiples of the bin width (Algorithm 3 centres them on
 * w_min + (t + 1/2) dw: the same method on a shifted lattice).  Eq. N_w gives
 * the customary count Nw >= 2 pi (n_max - n_min)(w_max - w_min); the error
 * falls only as 1 / Nw (Section 6.2).  W must be odd; plans with fewer than
 * 2 (n_max - n_min)(w_max - w_min) bins, or with WS_FLAG_NO_Z_OFFSET, return
 * WS_ERR_ARG.  The plan is used with ws_grid, ws_degrid and the other plan
 * calls like any other. */
ws_status ws_plan_original(ws_plan_t *out, int32_t N, double x0, int32_t W, double fov,
                           double w_min, double w_max, int32_t Nw, uint32_t flags);

/* Algorithm 6: image (device complex64 N x N, read) -> vis (device complex64
 * M, overwritten), for uvw (device double M x 3).  M = 0 is allowed.
 * Visibilities with w outside [w_min, w_max] or non-finite u, v are written as
 * 0 and counted; the call then returns WS_ERR_W_RANGE / WS_ERR_UV_RANGE (after
 * finishing all other visibilities). */
ws_status ws_degrid(ws_plan_t plan, const void *image, const double *uvw, int64_t M,
                    void *vis, ws_stream_t stream);

/* Algorithm 5: vis (device complex64 M, read) at uvw (device double M x 3) ->
 * dirty (device complex64 N x N, overwritten).  Out-of-range visibilities are
 * skipped and counted as for ws_degrid.  The row transforms of N' = 512 ..
 * 4096 wait for their TMA row copies with a bounded wait (2^20 polls); a wait
 * that gives up leaves dirty incomplete, is counted in ws_stats_t
 * waits_timed_out, and the call returns WS_ERR_TIMEOUT.  The environment
 * variable WS_WAIT_POLLS, read at every call, sets the poll limit of the
 * first wait for each plane's row (0 gives up at once; the wait that drains
 * a copy in flight before the CTA returns keeps the full limit), so that the
 * timeout path can be exercised without any fault. */
ws_status ws_grid(ws_plan_t plan, const double *uvw, const void *vis, int64_t M,
                  void *dirty, ws_stream_t stream);

/* Bind a visibility coordinate set to the plan.  The tap rule of Section 3.3,
 * the offsets nu, the pre-phase exp(2 pi i w (n0 - 1)) and the sort of the
 * visibilities into bins depend on uvw alone, so a consumer that
 * calls ws_grid and ws_degrid many times on the same uvw (conjugate
 * gradients, autograd, any iterative imager) can have them made once.  This
 * call makes them for both directions, with the occupancy of the w-stack,
 * into plan-owned buffers (allocated on first use, grown as needed).  Later
 * ws_grid / ws_degrid calls whose uvw pointer and M equal the bound ones skip
 * that work and give the same results as unbound calls.  Calls with any other
 * uvw or M run unbound, as before.
 *   uvw  device double M x 3, or NULL to unbind (the buffers are kept)
 * The caller must keep the bound array allocated and unchanged until it binds
 * another set or unbinds: the plan does not see later changes to its contents.
 * Visibilities the bound set drops (non-finite u, v; w outside the plan's
 * range) are reported by every later call on it, as for an unbound call.
 * Waits for the stream before it returns. */
ws_status ws_plan_bind_uvw(ws_plan_t plan, const double *uvw, int64_t M, ws_stream_t stream);

/* Tune the plan's gridding tile.  The stack is tiled in 8 w-planes x
 * tile_rows grid rows x 16 grid columns: gridding gives one CTA each column of
 * tiles, degridding bins the visibilities by tile (the gather order), and the
 * plane transforms skip the tiles no footprint touches.  tile_rows = 16, 32
 * or 64 trades entries per visibility against shared memory per CTA and the
 * occupancy granularity; the fastest depends on N', W, the data and the GPU.
 * This call times one ws_grid plus one ws_degrid per candidate on the
 * caller's data (uvw, vis: M visibilities; image: N x N; device memory, read
 * only) on `stream`, keeps the fastest, and reports it in *tile_rows (may be
 * NULL).  With cache_path non-NULL the result is read from, or else written
 * to, that JSON file under the key "<GPU name>|N'=<N'>|W=<W>" (a cached
 * entry skips the timing).  ws_plan and ws_batch_create apply the cached
 * entry for their (N', W) when the environment variable WS_TUNE_CACHE names
 * the file; an entry the plan cannot take (rows that do not divide N', or a
 * gridding ring too large for shared memory, as 64 rows are for deterministic
 * plans at W = 7) is ignored, and the tuner does not time such shapes.  Re-tiling drops a bound visibility set.  The tuning allocates
 * scratch outputs and synchronises the device; call it at set-up, not in a
 * loop.  The paper has no counterpart: tile shapes are a property of this
 * GPU implementation. */
ws_status ws_plan_tune(ws_plan_t plan, const double *uvw, const void *vis, const void *image, int64_t M,
                       const char *cache_path, ws_stream_t stream, int32_t *tile_rows);

/* Allocation-free degridding.  The paper has no counterpart: this entry point
 * exists for callers that cannot allocate device memory while they run (a
 * process whose device memory budget is fixed at start-up, a plug-in whose
 * host application owns every allocation, code that must not trigger the
 * synchronisation an allocation can imply).  It computes the same result as
 * ws_degrid, with the same arguments and status codes, but takes all of its
 * per-call scratch (visibility records, bin lists, the corrected image, the
 * w-plane chunk) from one 64 MiB array in device memory that the library
 * holds on every device that loads it, until the process exits.  It calls no
 * cudaMalloc or cudaFree and allocates nothing else on the device.
 *   - The plan (made earlier by ws_plan, which does allocate) supplies the
 *     tables; the caller supplies inputs and outputs as for ws_degrid.
 *   - Problems whose records, image and at least 8 w-planes of N' x N' do not
 *     fit in the 64 MiB are rejected with WS_ERR_ARG and a message.
 *   - The first call on a device looks up the array's device address (a
 *     runtime symbol query that may load the module); make that first call
 *     before capturing the stream into a graph.
 *   - Every call on a device shares the one array: calls whose GPU work
 *     overlaps (different streams, or different host threads) race and give
 *     wrong results.  Serialise them. */
ws_status ws_degrid_noalloc(ws_plan_t plan, const void *image, const double *uvw, int64_t M,
                            void *vis, ws_stream_t stream);

/* Visibilities dropped by the plan's latest call (waits for that call). */
ws_status ws_plan_dropped(ws_plan_t plan, int64_t *dropped);

/* Plan parameters and sizes. */
ws_status ws_plan_info(ws_plan_t plan, ws_plan_info_t *info);

/* Counters of the plan's calls since the last reset; waits for the plan's
 * pending timed work.  reset != 0 clears them afterwards.  Stage times are
 * zero unless the plan was made with WS_FLAG_TIMING. */
ws_status ws_plan_stats(ws_plan_t plan, ws_stats_t *stats, int32_t reset);

/* Release the plan's device memory (waits for its work). */
ws_status ws_destroy(ws_plan_t plan);

/* ---- Batches of independent problems -----------------------------------
 * Many observations or channels at once, each with its own image size,
 * field, w-range and visibility count (x0, W and flags shared).  The paper
 * has no counterpart; this is the serving form of Algorithms 5 and 6.  The
 * batch builds one plan per instance, exactly as ws_plan would, but no
 * per-plan w-stack: it deals the instances to `branches` parallel branches
 * (largest first, each to the least-loaded branch) and gives each branch one
 * slice of a shared workspace, used by its instances in turn.  A call runs
 * every instance's kernels, each branch on its own stream, captured once into
 * a CUDA graph; later calls with the same data pointers replay that graph,
 * calls with other pointers capture a new one.  Results are those of
 * ws_grid / ws_degrid on each instance alone.
 *
 * Pointer arguments are HOST arrays of n DEVICE pointers (instance order);
 * each instance's buffers follow the ws_grid / ws_degrid layouts.  The batch
 * must not be used by two calls at once; buffers must stay valid while a
 * replayed graph may use them. */
typedef struct ws_batch_s *ws_batch_t;

typedef struct {
    int32_t N;             /* image side (as for ws_plan) */
    double fov;            /* field of view (as for ws_plan) */
    double w_min, w_max;   /* w-range (as for ws_plan) */
    int64_t M;             /* visibilities of this instance (fixed for the batch's life) */
} ws_instance_t;

/* Build a batch of n >= 1 instances.
 *   x0, W            as for ws_plan, shared by all instances
 *   branches         1..8 parallel branches, or 0: the first call picks the
 *                    gridding tile rows (16, 32 or 64) for each image size by
 *                    timing that size's largest instance (unless the tuning
 *                    cache named by WS_TUNE_CACHE has them; new results are
 *                    added to it), then times the call with 1, 2 and 4
 *                    branches and keeps the fastest
 *   workspace_bytes  device bytes shared by the branches' w-stacks; 0 = the
 *                    smaller of 60% of free memory and what `branches` (or 4)
 *                    whole stacks of the largest instance need.  Each slice
 *                    must hold 8 planes of its largest instance (WS_ERR_OOM)
 *   flags            WS_FLAG_ASYNC, WS_FLAG_NO_Z_OFFSET, WS_FLAG_HERMITIAN
 * Per-instance parameter errors return WS_ERR_ARG naming the instance. */
ws_status ws_batch_create(ws_batch_t *out, int32_t n, const ws_instance_t *inst, double x0, int32_t W,
                          int32_t branches, int64_t workspace_bytes, uint32_t flags);

/* Algorithm 5 on every instance: uvw[i] (device double M_i x 3), vis[i]
 * (device complex64 M_i) -> dirty[i] (device complex64 N_i x N_i).  Unless
 * WS_FLAG_ASYNC, waits for the stream and returns WS_ERR_UV_RANGE /
 * WS_ERR_W_RANGE naming the first instance that dropped visibilities. */
ws_status ws_batch_grid(ws_batch_t batch, const double *const *uvw, const void *const *vis,
                        void *const *dirty, ws_stream_t stream);

/* Algorithm 6 on every instance: image[i] (device complex64 N_i x N_i),
 * uvw[i] -> vis[i] (device complex64 M_i, overwritten). */
ws_status ws_batch_degrid(ws_batch_t batch, const void *const *image, const double *const *uvw,
                          void *const *vis, ws_stream_t stream);

/* Plan parameters of instance i and the branch it runs on (-1 before the
 * branch count is chosen); branch may be NULL. */
ws_status ws_batch_info(ws_batch_t batch, int32_t i, ws_plan_info_t *info, int32_t *branch);

/* Branch count in use (0 until the first call of a batch made with branches = 0). */
ws_status ws_batch_branches(ws_batch_t batch, int32_t *branches);

/* Release the batch's plans, workspace, streams and graphs (waits for its work). */
ws_status ws_batch_destroy(ws_batch_t batch);

/* Message for the calling thread's latest non-WS_OK status ("" if none). */
const char *ws_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* WS_H */
