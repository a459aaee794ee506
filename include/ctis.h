/*
 * ctis.h - C ABI of the GB300 CTIS reconstruction library (libctis.so).
 *
 * The library implements the data-parallel hot path of shift-invariant CTIS
 * reconstruction (White, Bell, Haygood): the forward projection H f, the back
 * projection H^T r and the EM iteration of Eq. 2 built from them, as
 * hand-written sm_103a CUDA kernels.
 *
 * Problem statement (Sec. 2): a field stop of a x alpha pixels is observed at
 * w wavelengths on a gamma x xi focal-plane array (FPA). One calibration image
 * per wavelength is the response to a point source at field-stop pixel (0,0);
 * under shift-invariance, field-stop pixel (p, r) produces the same image
 * shifted by (p, r). H therefore has n = gamma*xi rows and m = a*alpha*w
 * columns, and H f = sum_s sum_k v_{s,k} f_s(x - x_k, y - y_k) (Eqs. 1, 8, 12).
 *
 * Layouts (all dense, row-major, no padding in caller buffers):
 *   datacube f   : f[s][r][p], element j = s*a*alpha + r*a + p (the zero-based
 *                  j of the Sec. 3 index map), s < w, r < alpha, p < a.
 *   FPA image g  : g[y][x], element i = x + gamma*y, x < gamma, y < xi.
 *   PSF          : CSR over wavelengths: psf_ptr[w+1] (psf_ptr[0] = 0), then
 *                  per nonzero k the FPA coordinates psf_x[k], psf_y[k] of the
 *                  response to field-stop pixel (0,0) and its value psf_val[k].
 *
 * Conventions:
 *   - Every function returns a ctis_status (0 = success). Errors detected on
 *     the host return before anything is enqueued. Kernels report device-side
 *     failures (a bounded wait that gave up) through ctis_plan_check().
 *   - Device pointers are caller-owned (allocate them with any allocator; the
 *     library never frees them). Host pointers are read during the call only.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream). Calls are
 *     asynchronous and stream-ordered unless stated otherwise.
 *   - A plan owns device workspace, so calls on one plan must not overlap in
 *     time: issue them on one stream (or synchronise between streams).
 *   - A plan is bound to the CUDA device that was current at creation; calls
 *     must be made with that device current.
 */
#ifndef CTIS_H
#define CTIS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ctis_plan ctis_plan;

typedef enum {
    CTIS_OK = 0,
    CTIS_ERR_INVALID_ARG = -1,   /* bad size, pointer, flag or PSF entry        */
    CTIS_ERR_OUT_OF_BOUNDS = -2, /* a shifted PSF nonzero leaves the FPA         */
    CTIS_ERR_NOMEM = -3,         /* device or host allocation failed             */
    CTIS_ERR_CUDA = -4,          /* a CUDA runtime/driver call failed            */
    CTIS_ERR_TIMEOUT = -5,       /* a kernel's bounded wait gave up              */
    CTIS_ERR_UNSUPPORTED = -6    /* valid request this build cannot serve        */
} ctis_status;

/* Storage type of the datacube f and of the PSF values inside a plan. */
enum { CTIS_F32 = 0, CTIS_BF16 = 1 };

/* FPA boundary reading (ctis_plan_options.boundary). Eq. 7's circulant would
 * wrap a shifted nonzero past the FPA edge into another row; a physical shift
 * loses it. REJECT (default): every shifted nonzero must stay on the FPA, so
 * both readings agree. CLIP: the physical reading: shifted nonzeros off the
 * FPA are dropped (lost light), and h = H^T 1 then varies per voxel. WRAP:
 * Eq. 7 taken literally, for comparison: PSF nonzeros must lie on the FPA
 * (c_s has n entries) and a shifted copy lands in row
 * (x + p + gamma (y + r)) mod n, so one past the right edge re-enters at the
 * left of the next FPA row and one past the last row at the top. The plan
 * stores it as the CLIP reading of the PSF together with each nonzero's
 * images at (x - gamma, y + 1), (x, y - xi) and (x - gamma, y + 1 - xi)
 * (those whose shifted copies can meet the FPA): each shifted copy re-enters
 * at exactly one of them. ctis_plan_export_taps then lists the images too,
 * and ctis_plan_set_values, ctis_psf_grad and ctis_unrolled_nll_grad return
 * CTIS_ERR_UNSUPPORTED (an image must keep its original's value). */
enum { CTIS_BOUNDARY_REJECT = 0, CTIS_BOUNDARY_CLIP = 1, CTIS_BOUNDARY_WRAP = 2 };

/* ctis_reconstruct flags. Without an INIT flag, f_dev holds the initial guess. */
enum {
    CTIS_INIT_ONES = 1,  /* f^(1) = 1 (Algorithm 1)                     */
    CTIS_INIT_HTG = 2    /* f^(1) = H^T g (Sec. 2, alternative guess)   */
};

/* Per-forward-pass statistics (float64), CTIS_NSTATS values each, taken over
 * the pixels where H f > 0 (the support of the model image):
 *   [0] sum H f                       (model flux)
 *   [1] sum g                         (measured flux on the support)
 *   [2] sum g log(H f) - H f          (Poisson log-likelihood, no constant)
 *   [3] sum (g - H f)^2               (squared residual norm)          */
enum { CTIS_STAT_FLUX_HF = 0, CTIS_STAT_FLUX_G = 1, CTIS_STAT_LOGLIK = 2,
       CTIS_STAT_RESID2 = 3, CTIS_NSTATS = 4 };

/* Create a plan: validate and merge the calibration PSFs, check that every
 * shifted nonzero stays on the FPA (0 <= x_k, x_k + a - 1 < gamma, same for y
 * with alpha and xi; otherwise CTIS_ERR_OUT_OF_BOUNDS), group nonzeros into
 * spot clusters, build the per-tile work lists of both projectors, compute
 * h = H^T 1 (Eq. 2; per wavelength the sum of its PSF values) in float64 and
 * upload everything. All PSF arrays are host memory, copied. Values must be
 * finite and >= 0. Duplicate (x, y) entries of one wavelength add up.
 * dtype is CTIS_F32 or CTIS_BF16 (BF16: f and PSF values are stored in
 * bfloat16, arithmetic accumulates in float32). Blocks until the plan's device
 * data is uploaded. On failure *out is set to NULL. */
int ctis_plan_create(ctis_plan** out, int a, int alpha, int w, int gamma, int xi,
                     const int32_t* psf_ptr, const int32_t* psf_x,
                     const int32_t* psf_y, const float* psf_val, int dtype);

/* Optional plan settings (zero-initialise, set struct_size). */
typedef struct {
    int struct_size;       /* sizeof(ctis_plan_options)                         */
    int tasks_per_item;    /* > 0: tiles cut into work items of at most this many
                              cluster tasks, assigned to CTAs longest first     */
    int item_overhead_q;   /* > 0: balanced split: the tiles' tasks, in tile
                              order, cut into one run of equal estimated cost
                              per CTA, with a per-item overhead of this many
                              quarter tasks. Exclusive with tasks_per_item;
                              both 0 = the candidate with the smallest
                              estimated busiest CTA                             */
    int cta_skew_permille; /* 0..900: schedule for CTAs whose speed falls
                              linearly from 1 + skew to 1 - skew over the block
                              indices (the SM's warp schedulers favour the CTAs
                              resident first); 0 = equal speeds                 */
    int boundary;          /* CTIS_BOUNDARY_REJECT (0), _CLIP or _WRAP; CLIP
                              accepts PSF coordinates in [-2^24, 2^24), WRAP
                              those on the FPA                                  */
    int forward_tile;      /* CTIS_TILE_32X32 (0, default) or CTIS_TILE_32X16:
                              the forward's output tiles until ctis_plan_autotune
                              picks the faster shape                            */
    int reserved[2];       /* must be 0                                          */
} ctis_plan_options;

/* Forward tile shapes (FPA pixels, columns x rows). 32 x 16 tiles waste less
 * of the footprints of small field stops (a footprint covers whole tiles)
 * but carry each window's fixed costs over half the outputs. */
enum { CTIS_TILE_32X32 = 0, CTIS_TILE_32X16 = 1 };

/* ctis_plan_create with options; opt may be NULL (all defaults). */
int ctis_plan_create_ex(ctis_plan** out, int a, int alpha, int w, int gamma, int xi,
                        const int32_t* psf_ptr, const int32_t* psf_x, const int32_t* psf_y,
                        const float* psf_val, int dtype, const ctis_plan_options* opt);

/* Host-only view of the tables a plan would build (no device is touched):
 * for one projector (forward != 0: FPA tiles x spot clusters, Eqs. 8 and 12;
 * else voxel tiles x the clusters of their wavelength, Eq. 14), the PSF is
 * merged and clustered as ctis_plan_create does, and the work lists are built
 * and scheduled (options as in ctis_plan_options) over n_ctas persistent CTAs
 * of info.warps_per_cta warps. block_sm: NULL, or [n_ctas] the SM id of each
 * CTA (as the plan's placement probe reports; ids in [0, 4096)). The outputs
 * are host arrays sized from info (fill info first with all arrays NULL,
 * then call again); any array may be NULL:
 *   clusters      [3 * clusters]  (s, X, Y): wavelength and FPA origin of each
 *                                 K x K spot cluster
 *   tile_xyp      [3 * tiles]     (x0, y0, plane) of each output tile
 *   tile_task_ptr [tiles + 1]     CSR offsets of the tiles' tasks
 *   task_cluster  [tasks]         the cluster of each task, tile order
 *   warp_begin    [warps + 1]     each warp's range of work items
 *   item_tile     [witems]        the tile of each warp's work item
 *   item_chunk    [2 * witems]    (chunk index, chunks of the tile)
 *   item_range    [2 * witems]    [begin, end) of the item's tasks, in tile
 *                                 task order (warp w of a CTA runs the w-th
 *                                 part of the CTA's item)
 * Errors: those of ctis_plan_create (except device ones); CTIS_ERR_INVALID_ARG
 * for a bad n_ctas, block_sm or info. */
typedef struct {
    int struct_size;       /* sizeof(ctis_tables_info), set by the caller */
    int64_t clusters, cluster_k, tiles, tasks, witems, warps, warps_per_cta;
    int64_t tile_w, tile_h;
    int64_t chunk, split_q, skew_pm;   /* the schedule, as in ctis_plan_info */
    int64_t load_milli;                /* estimated latest CTA, tasks per warp x1000 */
} ctis_tables_info;

int ctis_tables_inspect(int a, int alpha, int w, int gamma, int xi, const int32_t* psf_ptr,
                        const int32_t* psf_x, const int32_t* psf_y, const float* psf_val, int dtype,
                        const ctis_plan_options* opt, int forward, int n_ctas,
                        const int32_t* block_sm, ctis_tables_info* info, int32_t* clusters,
                        int32_t* tile_xyp, int32_t* tile_task_ptr, int32_t* task_cluster,
                        int32_t* warp_begin, int32_t* item_tile, int32_t* item_chunk,
                        int32_t* item_range);

/* Release the plan and its device memory (synchronises the device first).
 * NULL is accepted. */
int ctis_plan_destroy(ctis_plan* plan);

/* Sizes and derived quantities of a plan (host call, no device work). */
typedef struct {
    int64_t a, alpha, w, gamma, xi, m, n;
    int64_t nnz;                 /* merged PSF nonzeros, all wavelengths       */
    int64_t clusters;            /* spot clusters after grouping               */
    int64_t cluster_k;           /* cluster box side K (K x K taps)            */
    int64_t fwd_tiles, fwd_tasks, fwd_items;
    int64_t adj_tiles, adj_tasks, adj_items;
    int64_t scratch_bytes;       /* device workspace owned by the plan         */
    int64_t dtype;
    int64_t fwd_warps, adj_warps;          /* persistent warps per launch        */
    int64_t fwd_chunk, adj_chunk;          /* tasks per work item (chunk schedule;
                                              0 under the balanced split)       */
    int64_t fwd_load_milli, adj_load_milli;/* busiest warp's scheduled tasks x1000 */
    int64_t fwd_split_q, adj_split_q;      /* balanced split's item overhead in
                                              quarter tasks; 0 = chunk schedule */
    int64_t fwd_skew_pm, adj_skew_pm;      /* CTA priority skew of the schedule  */
    int64_t boundary;                      /* CTIS_BOUNDARY_*                    */
    int64_t fwd_tile_w, fwd_tile_h;        /* the forward's tile shape (FPA pixels;
                                              ctis_plan_autotune may change it)  */
} ctis_plan_info;

int ctis_plan_get_info(const ctis_plan* plan, ctis_plan_info* info);

/* Copy the merged PSF table to host arrays: for each merged nonzero, sorted by
 * (s, y, x), its wavelength, FPA coordinates and value (as stored: float32, or
 * bfloat16 widened to float32), plus h[w] (float32 as used by the update;
 * under CTIS_BOUNDARY_CLIP the per-wavelength sum of the values, which the
 * voxels whose light partly leaves the FPA do not reach: their h is
 * H^T 1 per voxel; under CTIS_BOUNDARY_WRAP the sum of the nonzeros on the
 * FPA, which every voxel reaches). Arrays must hold info.nnz entries (h: w entries). Any
 * pointer may be NULL. */
int ctis_plan_export_taps(const ctis_plan* plan, int32_t* s, int32_t* x, int32_t* y,
                          float* val, float* h);

/* Device index map of the Sec. 3 embedding (I_w kron E): out_dev[j] = position
 * in the stacked FPA vectors v = (v_1 .. v_w) of datacube element j,
 * i = x + gamma*y + s*n for j = (p, r, s) with x = p, y = r. int64, m entries. */
int ctis_index_map(const ctis_plan* plan, int64_t* out_dev, void* stream);

/* hf_dev = H f_dev (Eqs. 1, 8). f_dev: m elements of the plan's dtype;
 * hf_dev: n float32. */
int ctis_forward(const ctis_plan* plan, const void* f_dev, float* hf_dev, void* stream);

/* out_dev = H^T r_dev (Eq. 14). r_dev: n float32; out_dev: m float32. */
int ctis_adjoint(const ctis_plan* plan, const float* r_dev, float* out_dev, void* stream);

/* k EM updates (Eq. 2, Algorithm 1): per iteration u = g / (H f) (0 where
 * H f = 0), then f <- f * (H^T u) / h (0 where h = 0).
 * g_dev: n float32 counts. f_dev: m elements of the plan's dtype; read as the
 * initial guess unless an INIT flag is given, overwritten with f^(k+1).
 * stats_dev: NULL, or device float64[(k+1)*CTIS_NSTATS]: row t holds the
 * statistics of H f^(t+1) for t < k (computed by the iteration's forward
 * pass) and row k those of the returned f (one extra forward pass).
 * The k iterations are replayed from a CUDA graph cached in the plan
 * (re-captured when pointers, k, flags or the stream's capture state change). */
int ctis_reconstruct(const ctis_plan* plan, const float* g_dev, void* f_dev, int k,
                     int flags, double* stats_dev, void* stream);

/* Other solvers on the same projector pair (Sec. 2 lists ART and MART among
 * the usual CTIS solvers and the scheme is solver agnostic; their
 * simultaneous forms): k updates of `solver`, with relaxation `relax` in
 * (0, 2] (ignored by EM), fused into the same two launches per iteration:
 *   CTIS_SOLVER_EM:    exactly ctis_reconstruct.
 *   CTIS_SOLVER_SART:  u = (g - H f) / r with r = H 1 (0 where r = 0), then
 *                      f <- max(f + relax * (H^T u) / h, 0) (simultaneous ART,
 *                      Andersen and Kak).
 *   CTIS_SOLVER_SMART: u = log(g / H f) where g > 0 and H f > 0 (0 elsewhere),
 *                      then f <- f * exp(relax * (H^T u) / h) (simultaneous
 *                      MART, Byrne).
 * Voxels with h = 0 keep their value under SART and SMART. Arguments,
 * statistics and graph caching as ctis_reconstruct. SART builds r on its
 * first call (a forward projection of ones, synchronous; again after
 * ctis_plan_set_values), so that call must not be made while the stream is
 * being captured (CTIS_ERR_INVALID_ARG). */
enum { CTIS_SOLVER_EM = 0, CTIS_SOLVER_SART = 1, CTIS_SOLVER_SMART = 2 };
int ctis_reconstruct_solver(const ctis_plan* plan, const float* g_dev, void* f_dev, int k,
                            int flags, int solver, float relax, double* stats_dev, void* stream);

/* Kernel timing. When enabled, ctis_reconstruct records a CUDA event pair
 * (as event-record nodes of its cached graph) around every projector launch.
 * ctis_plan_kernel_times waits for those events and reports, for the most
 * recent ctis_reconstruct, the summed device time in milliseconds and the
 * number of forward and adjoint launches. Any output pointer may be NULL. */
int ctis_plan_set_profiling(ctis_plan* plan, int enable);

/* Test and measurement hooks. With CTIS_DEBUG_DROP_COPIES the gather
 * kernels arm each copy's barrier without issuing the copy, so every wait of
 * every warp runs out (after about 2^31 SM cycles, ~1 s), the kernel records
 * the failure, skips its remaining copies and returns; ctis_plan_check then
 * reports CTIS_ERR_TIMEOUT and the context stays usable. Results are
 * undefined while it is set. CTIS_DEBUG_SERIAL_LAUNCH launches the projector
 * kernels as plain launches instead of with programmatic dependent launch
 * (by default a projector kernel is scheduled as soon as every CTA of the
 * stream's previous projector has finished its work, and its prologue, which
 * reads only the plan's work lists, runs while that grid drains and exits;
 * the results are the same either way). flags = 0 restores normal operation. Waits for the
 * device and drops the plan's cached graphs. */
enum { CTIS_DEBUG_DROP_COPIES = 1, CTIS_DEBUG_SERIAL_LAUNCH = 2 };
int ctis_plan_set_debug(ctis_plan* plan, int flags);
int ctis_plan_kernel_times(const ctis_plan* plan, double* fwd_ms, int* n_fwd, double* adj_ms,
                           int* n_adj);

/* Wavelength-sharded EM reconstruction (Eqs. 2, 3 and 8). H f is the sum over
 * wavelength blocks of H_s f_s, so the ranks of a job that each own a
 * contiguous slice of the wavelengths can run one reconstruction together:
 * every rank creates a plan for its slice alone (the slice's wavelengths,
 * their calibration images, psf_ptr rebased to 0) and calls this with its
 * part of the datacube. Each iteration, the rank forms its slice's partial
 * image q_r = sum over its s of H_s f_s into a plan-owned device buffer of n
 * float32 and calls reduce(q, n, reduce_ctx, stream), which must replace q,
 * stream-ordered on `stream`, with the sum over the ranks (an all-reduce, for
 * instance NCCL's on the caller's communicator; every rank must add in the
 * same order so that all hold the same sum); then u = g / q (0 where q = 0)
 * and the statistics of q, and the slice's adjoint and multiplicative update,
 * are local. The reduction is the only exchange: n floats per iteration
 * (k + 1 with statistics, the last for the final iterate). reduce may be
 * NULL: the slice's own image is then the whole H f (a single rank with the
 * whole datacube, or a test). g_dev (n float32, the whole measurement, on
 * every rank), f_dev (the slice's datacube, m_slice elements of the plan's
 * dtype; the initial guess unless CTIS_INIT_ONES), stats_dev (NULL or
 * float64[(k + 1) * CTIS_NSTATS], identical on every rank) as in
 * ctis_reconstruct (CTIS_INIT_HTG gives the slice's own columns of H^T g,
 * local to the rank). Not captured in a CUDA graph (the callback runs on the
 * host between launches); EM only. Returns what the launches return, or
 * CTIS_ERR_CUDA when reduce returns nonzero. */
typedef int (*ctis_reduce_fn)(float* q_dev, int64_t n, void* reduce_ctx, void* stream);
int ctis_reconstruct_sharded(ctis_plan* plan, const float* g_dev, void* f_dev, int k, int flags,
                             double* stats_dev, ctis_reduce_fn reduce, void* reduce_ctx,
                             void* stream);

/* Average device time of one EM launch of each projector, from CUDA events
 * around `reps` back-to-back launches on `stream` (after two warm-up
 * launches): the forward with the ratio epilogue and float64 tile statistics
 * (g_dev the measurement, as in ctis_reconstruct), and the adjoint with the
 * multiplicative update, on the plan's current schedules; milliseconds per
 * launch in *fwd_ms and *adj_ms. No event sits between the launches, so the
 * figures carry no event-record overhead (the profiled reconstruction's
 * per-launch events of ctis_plan_kernel_times do). The plan's internal
 * datacube and FPA copies are overwritten; no caller buffer is written.
 * Synchronous. The paper has no counterpart (a measurement utility). */
int ctis_plan_time_launches(ctis_plan* plan, const float* g_dev, int reps, double* fwd_ms,
                            double* adj_ms, void* stream);

/* FP32 FMA-pipe microbenchmark (the measured ceiling of the projectors'
 * roofline; the paper has no counterpart): `blocks` CTAs of `threads`
 * threads, each thread advancing 8 independent chains by 4 fused
 * multiply-adds per iteration for `iters` iterations (scalar FFMA, or FFMA2
 * pairs when `packed`): blocks * threads * iters * 32 FMAs (twice that when
 * packed), 2 FLOP each. Writes one float per thread to out_dev (device,
 * blocks * threads floats) so the chains are kept. Asynchronous on `stream`;
 * the caller times it. Returns CTIS_ERR_INVALID_ARG for sizes out of range
 * (threads a multiple of 32 in [32, 1024]), CTIS_ERR_CUDA if the launch
 * fails. */
int ctis_fma_peak(int packed, int blocks, int threads, int iters, float* out_dev, void* stream);

/* H f like ctis_forward, but with the projection's scratch (the x-shifted
 * copies of f, chunk partial sums and tile tickets) taken from a
 * fixed array inside the library instead of the plan's workspace. The paper
 * has no counterpart; this exists for callers that cannot call cudaMalloc
 * when they project (allocation-free real-time loops, code whose device
 * memory all belongs to its own pool, or code running under a stream capture
 * that rejects allocation). The call allocates nothing and calls no
 * allocating routine.
 *   - The array holds CTIS_STATIC_SCRATCH_BYTES (64 MiB) per GPU from the
 *     moment the library is loaded on that GPU until the process exits.
 *     Plans whose forward needs more return CTIS_ERR_UNSUPPORTED (the
 *     realistic 128x128x64 -> 1024^2 workload needs about 35 MiB; the
 *     256x256x128 -> 2048^2 one does not fit).
 *   - The first call on a device looks up the array's device address with
 *     that device current; make that first call before any stream capture.
 *   - Every call on a device shares the one array, and it keeps the last
 *     call's contents (each call clears what must start at zero). Calls whose
 *     executions overlap on the GPU (other streams, other threads, other
 *     plans) race on it: serialise them.
 *   - A device-side wait that gives up is reported by ctis_plan_check, as
 *     for ctis_forward (the error flag is the plan's own). */
#define CTIS_STATIC_SCRATCH_BYTES (64u << 20)
int ctis_forward_static_scratch(const ctis_plan* plan, const void* f_dev, float* hf_dev,
                                void* stream);

/* k EM updates on many frames at once. Frame i is reconstructed with plan
 * plans[plan_idx[i]] from g_dev[i] (n float32) into f_dev[i] (m elements of
 * that plan's dtype; read as the initial guess unless an INIT flag is given),
 * exactly as ctis_reconstruct would, with every frame's own statistics:
 * stats_dev is NULL or device float64[nframes][k+1][CTIS_NSTATS] (frame
 * order as given). Frames of one plan run as extra copies of its work lists,
 * so each iteration is one forward and one adjoint launch per plan covering
 * all of its frames; the whole call is one CUDA graph, cached for the next
 * call with the same arguments (per-frame pointers included). A plan keeps
 * the workspace of the last frame count it served (datacube and FPA copies,
 * partial sums and statistics for every frame). Host arrays: plans[nplans]
 * (distinct), plan_idx, g_dev and f_dev [nframes]; they may be freed when the
 * call returns. */
int ctis_reconstruct_batched(ctis_plan* const* plans, int nplans, int nframes,
                             const int* plan_idx, const float* const* g_dev,
                             void* const* f_dev, int k, int flags, double* stats_dev,
                             void* stream);

/* ctis_reconstruct_batched with the update rule of `solver` and relaxation
 * `relax` (as ctis_reconstruct_solver; CTIS_SOLVER_EM is exactly
 * ctis_reconstruct_batched). Each frame equals its single-frame
 * ctis_reconstruct_solver run bit for bit. SART builds a plan's row sums
 * on its first use (synchronous). */
int ctis_reconstruct_batched_solver(ctis_plan* const* plans, int nplans, int nframes,
                                    const int* plan_idx, const float* const* g_dev,
                                    void* const* f_dev, int k, int flags, int solver, float relax,
                                    double* stats_dev, void* stream);

/* ---- gradients (the differentiable form of the projector pair) ----------
 * The PSF values are the parameters: tap t of wavelength s, at FPA offset
 * (x_t, y_t) for field-stop pixel (0, 0), adds v_t f_s(p, r) to pixel
 * (x_t + p, y_t + r) (Sec. 2), so H is linear in every v_t. Taps are
 * indexed in ctis_plan_export_taps order (merged, sorted by (s, y, x)). */

/* Replace the plan's tap values (host float32[nnz], finite and >= 0),
 * rounded to the plan's dtype, and recompute h = H^T 1 (Eq. 2); not under
 * CTIS_BOUNDARY_WRAP (CTIS_ERR_UNSUPPORTED). Waits for all
 * device work first (queued kernels may read the old tables); the plan's
 * cached reconstruction graph stays valid and uses the new values. */
int ctis_plan_set_values(ctis_plan* plan, const float* vals);

/* dval_dev[t] = sum_{p,r} f_s(p, r) * r(x_t + p, y_t + r): the gradient of
 * <r, H f> with respect to v_t (s = tap t's wavelength). f_dev: m elements of
 * the plan's dtype; r_dev: n float32; dval_dev: nnz float32. Sums are float32
 * in a fixed order (reproducible). Not under CTIS_BOUNDARY_WRAP
 * (CTIS_ERR_UNSUPPORTED). */
int ctis_psf_grad(const ctis_plan* plan, const void* f_dev, const float* r_dev,
                  float* dval_dev, void* stream);

/* The Poisson negative log-likelihood after k EM updates (Eq. 2) and its
 * gradient through the updates:
 *   f^(0) = f0 (or all ones when f0_dev is NULL), f^(t+1) = EM(f^(t)),
 *   L = sum_i q_i - g_i log q_i over q = H f^(k), pixels with q_i > 0;
 *   nll_dev[0] = L (float64), dval_dev[t] = dL/dv_t (including the
 *   dependence of h = H^T 1 on v), df0_dev = dL/df0 when not NULL (float32).
 * The iterates are checkpointed (the plan keeps (k+1)*m float32 of workspace,
 * grown on demand); the backward pass recomputes each step's projections.
 * float32 plans with CTIS_BOUNDARY_REJECT or _CLIP (under CLIP h = H^T 1 is
 * per voxel, and its dependence on v goes through the taps whose shifted
 * copy lands on the FPA); CTIS_ERR_UNSUPPORTED otherwise; 0 <= k <= 4096. */
int ctis_unrolled_nll_grad(ctis_plan* plan, const float* g_dev, const float* f0_dev, int k,
                           double* nll_dev, float* dval_dev, float* df0_dev, void* stream);

/* Autotuner: for each projector, times the plan's EM launches (forward with
 * the ratio and statistics, adjoint with the update) over candidate work
 * schedules on this GPU, with g_dev (n float32) as the measurement and f = 1,
 * and keeps the fastest. Candidates: the plan's model choice, work items of
 * at most 16..192 cluster tasks assigned longest first, and the balanced
 * split with item overheads of 2..24 quarter tasks, some of them also with
 * CTA priority skews of 100..300 permille (ctis_plan_options); the four
 * fastest of a first pass are timed again, interleaved, before the choice.
 * The forward is tuned once per tile shape (CTIS_TILE_*), and the shapes'
 * winners are timed against each other, interleaved, over three rounds: the
 * plan keeps the faster shape with its schedule (ctis_plan_get_info reports
 * both). Synchronous; overwrites the plan's internal copies and drops its
 * cached graphs (the next ctis_reconstruct re-captures). Results stay
 * deterministic for a given shape and schedule but may differ in the last
 * bits between them (partial sums are grouped differently). */
int ctis_plan_autotune(ctis_plan* plan, const float* g_dev, void* stream);

/* Reschedules one projector's work lists (forward != 0: the forward) as the
 * options of ctis_plan_options would: tasks_per_item > 0 chunks assigned
 * longest first, item_overhead_q > 0 the balanced split (exclusive), both 0
 * the model's choice; cta_skew_permille in [0, 900]. Reapplies a schedule the
 * autotuner chose (ctis_plan_get_info reports it). Synchronous; drops the
 * plan's cached graphs. */
int ctis_plan_set_schedule(ctis_plan* plan, int forward, int tasks_per_item, int item_overhead_q,
                           int cta_skew_permille);

/* The paper's own (WBH) form of the projectors, for comparison with the
 * gather path: H_s = C_s E with C_s the length-n circulant whose first column
 * is the calibration image c_s (Eq. 7), so H f = F^-1 sum_s d_s (.) F E f_s
 * (Eqs. 11, 13) and H^T u = E^T stack_s F^-1 (conj(d_s) (.) F u) (Eqs. 14,
 * 17), d_s = F c_s, F the length-n real-to-complex transform (cuFFT, float32).
 * Built on the first call (w x (n/2+1) complex spectra and as many work
 * vectors, ~4 w n float32 of device memory). float32 plans with
 * CTIS_BOUNDARY_REJECT or _WRAP (the transform's product is circular: it is
 * the WRAP reading, which REJECT's rule makes equal to the others);
 * CTIS_ERR_UNSUPPORTED otherwise. Calls on one
 * plan share its workspace: issue them on one stream.
 *   ctis_fft_forward:     hf_dev (n) = H f_dev (m), dense layouts as ctis_forward.
 *   ctis_fft_adjoint:     out_dev (m) = H^T r_dev (n).
 *   ctis_fft_reconstruct: k EM updates (Eq. 2, Algorithm 1) of f_dev in place,
 *                         from ones with CTIS_INIT_ONES, else from f_dev. */
int ctis_fft_forward(ctis_plan* plan, const float* f_dev, float* hf_dev, void* stream);
int ctis_fft_adjoint(ctis_plan* plan, const float* r_dev, float* out_dev, void* stream);
int ctis_fft_reconstruct(ctis_plan* plan, const float* g_dev, float* f_dev, int k, int flags,
                         void* stream);

/* Wait for the plan's work on `stream`, then report (and clear) any device-side
 * failure recorded by its kernels: CTIS_OK or CTIS_ERR_TIMEOUT. */
int ctis_plan_check(const ctis_plan* plan, void* stream);

/* Human-readable name of a status code (static string). */
const char* ctis_status_string(int status);

/* Details of the last error on the calling thread (static thread-local string). */
const char* ctis_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* CTIS_H */
