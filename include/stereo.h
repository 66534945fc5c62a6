/*
 * libstereo: GB300 (sm_103a) implementation of the data-parallel hot path of
 * the iterative, tunable stereo method of Pillai, Ramalingam and Leonard
 * ("High-Performance and Tunable Stereo Reconstruction", Alg. 1-4).
 *
 * Two layers of entry points:
 *   1. The request API (stereo_create / stereo_submit / stereo_poll /
 *      stereo_release / stereo_destroy): the problem statement of Alg. 1 --
 *      given a rectified grey-scale pair (I_l, I_r), return the semi-dense
 *      disparity D_f and its cost C_f on the high-gradient pixels Omega_I.
 *   2. Stage entry points (stereo_census ... stereo_resample_match): one call
 *      per step of the method on caller-owned device buffers, for callers
 *      that run their own pipeline and for step-by-step verification.
 *
 * Conventions for every call:
 *   - Images are row-major uint8 with row stride W.  Pixel (u, v) is column
 *     u, row v; linear index v*W + u ("raster order").
 *   - Device pointers must be CUDA device (or managed) memory on the current
 *     device; "host" pointers are ordinary or pinned host memory.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Stage calls are asynchronous on that stream unless stated.
 *   - Return value: STEREO_OK (0) or a negative STEREO_E_* code.  Argument
 *     errors are detected on the host before anything is launched; CUDA
 *     launch errors come back as STEREO_E_CUDA.
 *   - The caller owns all buffers passed to stage calls.  Buffers handed out
 *     by stereo_poll are owned by the library until stereo_release.
 *   - Limits: 5 <= W, H <= 8192, W*H < 2^27, 1 <= dmax <= 256.
 */
#ifndef STEREO_H
#define STEREO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define STEREO_OK 0
#define STEREO_E_INVAL (-1)     /* bad argument (size, pointer, threshold) */
#define STEREO_E_NOMEM (-2)     /* request larger than the memory budget, or out of device memory */
#define STEREO_E_BUSY (-3)      /* no free slot and the queue is full: retry later */
#define STEREO_E_PENDING (-4)   /* poll timed out: result not ready yet */
#define STEREO_E_TIMEOUT (-5)   /* a bounded device-side wait gave up */
#define STEREO_E_INTERNAL (-6)  /* host-step failure (e.g. triangulation) */
#define STEREO_E_CUDA (-7)      /* a CUDA call failed */
#define STEREO_E_NOTFOUND (-8)  /* unknown ticket */
#define STEREO_E_CAP (-9)       /* a caller-provided output buffer is too small */

/* Tunables of Table 1 (G-scope) plus the readings this library fixes where the
 * paper gives no value.  Thresholds are census-bit counts in [0, 24]. */
typedef struct {
    int device;                /* CUDA device ordinal */
    size_t mem_budget_bytes;   /* device memory for in-flight requests (0 = 4 GiB) */
    void* arena;               /* optional caller-provided device arena of mem_budget_bytes
                                  (e.g. from the PyTorch caching allocator); NULL = the
                                  library calls cudaMalloc once at create time */
    int max_slots;             /* requests in flight at once (1 = plain per-pair path) */
    int max_queue;             /* submitted-but-not-admitted requests before STEREO_E_BUSY */
    int t_lo, t_hi;            /* Alg. 3 validation thresholds, 0 <= t_lo <= t_hi < 24 */
    int t_grad;                /* Omega_I: |dI/du| + |dI/dv| >= t_grad; 0 = the dense
                                  variant (every pixel inside the 2-pixel border evaluated) */
    int t_fast;                /* FAST-9 intensity threshold */
    int kp_per_bin;            /* keypoints kept per 12x10 bin, 1..32 */
    int uniq_margin;           /* epipolar uniqueness margin in census bits */
    int host_threads;          /* host triangulation workers (0 = 1) */
    void* stream;              /* cudaStream_t for all work (NULL = library creates one) */
    int profile;               /* N > 0: time the kernel launches of one GPU round in N (the
                                  sampled position within each N rounds rotates) with
                                  CUDA events on `stream` and accumulate per-kind durations in
                                  stereo_stats (1 = every round; event nodes lengthen a round,
                                  so a larger N disturbs the timing less); 0 = off */
    int inject_mesh_failure;   /* testing: the n-th host mesh step of the context (1-based) fails
                                  as if the triangulation had failed (STEREO_E_INTERNAL); 0 = off */
    int batch_window_us;       /* continuous batching: when some requests are ready for a GPU
                                  stage while others are still in their host step, wait up to
                                  this long for more of them before launching; 0 = the default
                                  (with device meshes, a request about to take its first pass
                                  waits up to 4 ms for the requests of its seed round still in
                                  their seed host step, so a burst submitted together runs its
                                  passes together; with host meshes, launch at once);
                                  < 0 = never wait */
    int autotune;              /* 1 = at create, time the kernels' work-shape candidates on a
                                  synthetic round of tune_w x tune_h pairs and keep the fastest
                                  (results do not depend on it; see stereo_get_tuning) */
    int tune_w, tune_h;        /* frame of the synthetic tuning round (0 = 1242 x 375) */
    int host_mesh;             /* 1 = triangulate S_it on the host between passes (the earlier
                                  design, kept for comparison); 0 = only S_1's mesh on the host,
                                  every later mesh re-tessellated on the GPU (stereo_delaunay_insert's
                                  kernels), with no host step between passes.  Same results. */
    int inject_wait_timeout;   /* testing: n > 0 makes the context use the bulk-copy validate
                                  (stereo_validate_bulk's kernel, the one kernel with device-side
                                  waits) and, in its n-th GPU round with an iteration stage, has
                                  that kernel's producer issue no copy, so every bounded wait gives
                                  up after a second: the round's requests fail with
                                  STEREO_E_TIMEOUT and the context stays usable; 0 = off */
} stereo_config;

/* Fill *cfg with the defaults: t_lo 4, t_hi 8, t_grad 8, t_fast 20,
 * kp_per_bin 4, uniq_margin 2, max_slots 1, max_queue 64, 4 GiB budget. */
void stereo_default_config(stereo_config* cfg);

typedef struct {
    const float* disparity;    /* D_f, H*W device fp32; 0 where never validated */
    const uint8_t* cost;       /* C_f, H*W device uint8 census bits; t_hi where never validated */
    const uint8_t* mask;       /* H*W device uint8 of the last pass: bit0 in Omega_I,
                                  bit1 evaluated (has a prior), bit2 C < t_lo, bit3 C > t_hi */
    const int32_t* planeidx;   /* H*W device int32 plane index of the last pass (-1 = no triangle) */
    int w, h;
    int iters;
    const int32_t* n_support;  /* host, iters entries: |S_it| for it = 1..iters */
    const int32_t* n_tri;      /* host, iters entries: triangles of G(S_it) */
    const float* support;      /* host, (u, v, d) triples of S_1 .. S_iters concatenated */
    double latency_ms;         /* submit -> result ready, host clock */
    double host_mesh_ms;       /* time spent in the host steps (support-set merge, triangulation,
                                  planes, raster lists), summed over passes */
    int status;                /* STEREO_OK or the request's error */
} stereo_result;

typedef struct stereo_ctx stereo_ctx;

/* Alg. 1 as a service.  stereo_create makes a context on cfg->device. */
int stereo_create(const stereo_config* cfg, stereo_ctx** out);

/* Device memory one request of this shape takes from the context's budget
 * (mem_budget_bytes) while in flight under cfg: its frame buffers, cell
 * records, device mesh (unless cfg->host_mesh) and staging; a budget of k times
 * this admits k such requests at once.  No counterpart in the paper.  Returns
 * 0 for invalid arguments. */
size_t stereo_request_bytes(const stereo_config* cfg, int w, int h, int dmax, int iters, int cell);

/* Submit one pair (I_l, I_r) with N_D = dmax, n_iters = iters and the initial
 * occupancy-grid size sz_occ = cell (Alg. 1, Table 1).  left/right may be host
 * or device pointers (detected); they are copied before the call returns, so
 * the caller may reuse them at once.  *ticket_out identifies the request.
 * Errors: STEREO_E_INVAL (sizes, thresholds, null pointers), STEREO_E_NOMEM
 * (needs more than the whole budget), STEREO_E_BUSY (queue full). */
int stereo_submit(stereo_ctx* ctx, int stream_id, const uint8_t* left, const uint8_t* right,
                  int w, int h, int dmax, int iters, int cell, uint64_t* ticket_out);

/* One pair of a batch submission: the arguments of stereo_submit, and
 * optional destinations of the results.  out_disparity (w*h fp32 D_f),
 * out_cost (w*h bytes C_f) and out_mask (w*h bytes of mask bits, as
 * stereo_result.mask), each NULL or a caller buffer that receives the result
 * before the request is reported done: the library copies it in the GPU round
 * that finishes the request, so a poll finds it in place.  Page-locked host
 * memory and device memory are written by the copy kernel of that round;
 * pageable host memory is copied with cudaMemcpyAsync (slower).  The buffers
 * stay the caller's and must stay valid until the request is done. */
typedef struct {
    int stream_id;
    const uint8_t* left;
    const uint8_t* right;
    int w, h, dmax, iters, cell;
    float* out_disparity;
    uint8_t* out_cost;
    uint8_t* out_mask;
} stereo_pair;

/* stereo_submit for n pairs at once, for callers serving many cameras: the
 * inputs are copied with one synchronisation and the pairs queued together,
 * so they start in the same GPU round (no counterpart in the paper, which
 * takes one pair).  Every pair is checked first: an invalid one rejects the
 * batch (STEREO_E_INVAL, nothing queued), as does one that needs more than
 * the whole budget (STEREO_E_NOMEM).  Pairs are then taken in order while the
 * queue has room; tickets_out[i] receives the ticket of pair i.  Returns the
 * number of pairs taken (1..n), or STEREO_E_BUSY when none could be, or
 * STEREO_E_CUDA / STEREO_E_NOMEM when copying failed (nothing queued). */
int stereo_submit_batch(stereo_ctx* ctx, const stereo_pair* pairs, int n, uint64_t* tickets_out);

/* Wait up to timeout_us (<0 = forever, 0 = test only) for a ticket.  On
 * STEREO_OK, *out describes the result; its buffers stay valid until
 * stereo_release.  STEREO_E_PENDING = not ready yet.  A request that failed
 * returns its error code (out->status holds it too). */
int stereo_poll(stereo_ctx* ctx, uint64_t ticket, stereo_result* out, int timeout_us);

/* stereo_poll, then the result copied into the caller's host buffers: D_f
 * (w*h fp32), C_f and the mask (w*h bytes each); a NULL buffer is skipped.
 * The copies run on the calling thread's own stream (other requests keep
 * computing meanwhile) and have landed when the call returns; page-locked
 * buffers copy fastest, pageable ones work too.  No counterpart in the paper:
 * it delivers Alg. 1's output D_f to host memory in one call.  Returns what
 * stereo_poll returns, or STEREO_E_CUDA if a copy failed. */
int stereo_poll_host(stereo_ctx* ctx, uint64_t ticket, stereo_result* out, int timeout_us,
                     float* disparity, uint8_t* cost, uint8_t* mask);

/* Return a finished request's buffers to the pool. */
int stereo_release(stereo_ctx* ctx, uint64_t ticket);

/* stereo_poll and stereo_release for n tickets at once, for callers serving
 * many cameras (one call and one lock instead of n; no counterpart in the
 * paper).  stereo_poll_batch waits up to timeout_us (<0 = forever, 0 = test
 * only) until every ticket is done, then fills out[i] as stereo_poll would for
 * tickets[i] (out[i].status is that request's own status).  Returns STEREO_OK
 * when all are done (whatever their status), STEREO_E_PENDING when the time
 * ran out first (out is then unspecified), STEREO_E_NOTFOUND when a ticket is
 * unknown (nothing waited for), STEREO_E_INVAL for null pointers or n < 1.
 * stereo_release_batch releases every done request among tickets[0..n) and
 * returns STEREO_OK, or the first error stereo_release would have returned for
 * one of them (the others are still released). */
int stereo_poll_batch(stereo_ctx* ctx, const uint64_t* tickets, int n, stereo_result* out, int timeout_us);
int stereo_release_batch(stereo_ctx* ctx, const uint64_t* tickets, int n);

/* Cancel queued work, wait for in-flight work, free everything. */
void stereo_destroy(stereo_ctx* ctx);

/* Text of the last failing CUDA call inside the library (error name, code,
 * source line, call), or "" when none failed.  The string is a thread-local
 * copy, valid until the next call from the same thread. */
const char* stereo_last_error(void);

/* Kernel kinds of the per-kind counters in stereo_stats. */
#define STEREO_K_CENSUS 0        /* census + Omega_I */
#define STEREO_K_FAST_SCORE 1    /* FAST-9 scores */
#define STEREO_K_FAST_BINS 2     /* non-maximum suppression + per-bin top-K */
#define STEREO_K_MATCH_KP 3      /* epipolar match of the keypoints */
#define STEREO_K_RASTER_CLEAR 4  /* plane-index map reset to -1 (inside the raster in the engine) */
#define STEREO_K_RASTER 5        /* scan conversion of the triangles */
#define STEREO_K_VALIDATE 6      /* fused interpolate + cost + refine */
#define STEREO_K_RESAMPLE 7      /* per-cell resample + epipolar match */
#define STEREO_K_FILL 8          /* cell-record resets (inside the raster in the engine) */
#define STEREO_K_MESH 9          /* re-tessellation, planes and raster lists on the device */
#define STEREO_K_KINDS 10

/* Counters of the context since creation.  kernel_launches counts every
 * kernel the library launched; batched_pairs sums the pairs each launch
 * covered (batched_pairs / kernel_launches = mean pairs per launch).  With
 * profile = N > 0, kind_ms[k] holds the summed CUDA-event durations of the
 * kind_timed[k] launches of kind k that were timed (those of every N-th
 * round; kind_ms[k] / kind_timed[k] is the mean launch time), and
 * kind_bytes[k] the algorithmic bytes all kind_launches[k] launches had to move (census:
 * 2 B/px read + 8.125 B/px written; raster clear and raster: 4 B/px written each; validate:
 * 13.125 B/px read (12.125 on a first pass) + 6 B/px written; mesh: 16 B per cell record read,
 * 16 B per new support point and 72 B per triangle of the new mesh written). */
typedef struct {
    long long kernel_launches;
    long long requests_done;
    long long batched_pairs;
    long long gpu_rounds;
    double host_mesh_ms;
    long long kind_launches[STEREO_K_KINDS];
    double kind_ms[STEREO_K_KINDS];
    double kind_bytes[STEREO_K_KINDS];
    double round_ms;              /* wall time inside GPU rounds (host preparation to synchronisation) */
    double graph_ms;              /* of which capturing and updating / instantiating the round's graph */
    double exec_ms;               /* of which from the graph launch to the round's synchronisation */
    long long graph_instantiations; /* rounds whose graph could not be updated in place */
    long long kind_timed[STEREO_K_KINDS]; /* launches of each kind timed with events (see profile) */
    /* device re-tessellation, summed over the passes of every request: passes, insertion
     * rounds and flip rounds of the launch that served each (a launch serves several
     * pairs), edge flips, and points inserted */
    long long mesh_passes, mesh_insert_rounds, mesh_flip_rounds, mesh_flips, mesh_points;
    long long mesh_edge_points;  /* of the points, those that lay on an edge when inserted */
} stereo_stats;
int stereo_get_stats(stereo_ctx* ctx, stereo_stats* out);

/* No counterpart in the paper (the paper has one CPU thread and no kernels).
 * The kernels' work shapes in use: the raster's small-triangle threshold
 * (bounding-box pixels; smaller boxes go to warp batches), the box pixels of
 * a warp batch, the column width of a large-triangle work item, and the
 * fused validate's blocks per SM and launch mode (1 = one launch for every
 * cell-side class).  With autotune, also the measured best times of the
 * synthetic round.  None of these change any result.  Returns STEREO_OK, or
 * STEREO_E_INVAL for a null argument; *out is caller-owned memory the call fills. */
typedef struct {
    int small_area, batch_area, raster_cols;
    int validate_blocks_per_sm, validate_mixed;
    int autotuned;
    double raster_us, validate_us;  /* best candidate's time (autotune), else 0 */
} stereo_tuning;
int stereo_get_tuning(stereo_ctx* ctx, stereo_tuning* out);

/* ---------------------------------------------------------------------------
 * Stage entry points.  All pointers device unless marked host.
 * ------------------------------------------------------------------------- */

/* Census 5x5 transform (Sec. III-C, "Census window-based matching on a 5x5
 * patch") of both images, and the Omega_I bit map of the left image (Sec. III,
 * high-gradient subset).  Census code bit b (b = 0..23) enumerates the
 * non-centre offsets row by row (dy = -2..2, dx = -2..2, bit 0 at (-2,-2)) and
 * is set when that neighbour is strictly darker than the centre; pixels within
 * 2 of the border get code 0.  Omega_I: 2 <= u < W-2, 2 <= v < H-2 and
 * |L(u+1,v) - L(u-1,v)| + |L(u,v+1) - L(u,v-1)| >= t_grad; stored as bit (u & 31)
 * of word v*ceil(W/32) + u/32.  Outputs: cL, cR: W*H uint32; omega:
 * H*ceil(W/32) uint32.  Any output pointer may be NULL to skip it. */
int stereo_census(const uint8_t* left, const uint8_t* right, int w, int h, int t_grad,
                  uint32_t* cL, uint32_t* cR, uint32_t* omega, void* stream);

/* FAST keypoints sampled from 12x10 spatial bins (Sec. III-A, SparseStereo).
 * FAST-9 on the radius-3 circle with threshold t_fast; score = max over the
 * brighter and darker circle sets of the summed excess over t_fast; 3x3
 * non-maximum suppression (equal scores go to the smaller raster index);
 * per bin (bx = 12u/W, by = 10v/H) the K best by (score desc, raster index
 * asc).  out_uv: 120*K slots of (u, v) int32 pairs in bin raster order then
 * rank, (-1, -1) for empty slots.  scratch: W*H int16 score map. */
int stereo_fast(const uint8_t* left, int w, int h, int t_fast, int K, int16_t* scratch,
                int32_t* out_uv, void* stream);

/* Epipolar matching along rows (Sec. III-A; Alg. 4 SparseEpipolarStereo).
 * For query (u, v): d* = first argmin over d in [0, min(dmax-1, u-2)] of
 * popcount(cL(u,v) ^ cR(u-d,v)); accepted when cost(d*) < t_lo and every d
 * with |d - d*| >= 2 costs at least cost(d*) + margin.  q_uv: n (u, v) pairs
 * (entries with u < 0 are skipped); out_d: n int32, d* or -1. */
int stereo_epipolar_match(const uint32_t* cL, const uint32_t* cR, int w, int h,
                          const int32_t* q_uv, int n, int dmax, int t_lo, int margin,
                          int32_t* out_d, void* stream);

/* Delaunay triangulation of support points (Sec. III-A, DelaunayTriangulation;
 * host, synchronous).  uv: n (u, v) int32 pairs in canonical order (sorted by
 * (v, u), no duplicates, 0 <= u, v <= 16383 so the exact int64 predicates
 * cannot overflow).  Cocircular ties resolve by symbolic perturbation of
 * the lifted coordinate u^2 + v^2 (smaller index = larger perturbation), which
 * makes the triangulation unique.  tri (host): up to cap sorted index triples
 * (i < j < k) in ascending order.  Returns the triangle count or a negative
 * error (STEREO_E_CAP when cap is too small; 2n suffices). */
int stereo_delaunay(const int32_t* uv, int n, int32_t* tri, int cap);

/* stereo_delaunay with the top levels of the divide and conquer on up to
 * `threads` host threads (1, 2, 4 or 8; other counts round down; the halves
 * of a split below 2048 points stay on one thread).  Same arguments, result
 * and errors as stereo_delaunay: the splits and merges are the same, only
 * their threads differ.  The engine uses the same routine with its idle host
 * workers at the end of a burst. */
int stereo_delaunay_parallel(const int32_t* uv, int n, int32_t* tri, int cap, int threads);

/* The re-tessellation between passes on the device (Alg. 1: the
 * DelaunayTriangulation of S_{it+1} = S_it + the new points of a resampling,
 * Alg. 4): the points are inserted into the given triangulation of S_it and
 * the mesh is flipped to the triangulation stereo_delaunay defines, on the
 * GPU, as the engine does between passes.  uv: n >= 3 (u, v) pairs in
 * canonical order and tri: T sorted index triples, the triangulation
 * stereo_delaunay returns for them (host).  uv_new (host): m (u, v) pixels of
 * a w x h frame, each covered by the old mesh's plane-index map (inside its
 * hull, or on a top or left hull edge: the pixels a pass can evaluate); a
 * pixel already in uv, or repeated, is skipped (an existing point keeps its
 * pixel).  tri_out (host): up to cap sorted index triples in ascending
 * order, indices into the union sorted by (v, u).  Synchronous; allocates
 * and frees device memory of its own on the current device.  Returns the
 * triangle count, or STEREO_E_INVAL (arguments, or a new point outside the
 * old mesh), STEREO_E_CAP (cap too small; 2 (n + m) suffices),
 * STEREO_E_NOMEM, STEREO_E_CUDA or STEREO_E_INTERNAL. */
int stereo_delaunay_insert(const int32_t* uv, int n, const int32_t* tri, int T, const int32_t* uv_new, int m,
                           int w, int h, int32_t* tri_out, int cap);

/* Disparity plane d = a*u + b*v + c per triangle (Eq. 3, "solving a linear
 * system"; host, synchronous): Cramer's rule in fp64 over the vertices in
 * index order, rounded to fp32.  d: n fp32 support disparities; abc: 3*T. */
int stereo_planes(const int32_t* uv, const float* d, const int32_t* tri, int T, float* abc);

/* Scratch bytes stereo_raster needs for T triangles: 2 * (T + 1) +
 * 2 * ceil(T / 1024) int32 of work lists (rounded up to 256 bytes). */
size_t stereo_raster_scratch_bytes(int T);

/* Pixel -> triangle lookup table (Sec. III-B) and DisparityInterpolation
 * (Alg. 1, Eq. 3) in one pass.  A pixel (u, v), sampled at integer
 * coordinates, belongs to a triangle when every edge function is positive or
 * zero on a top or left edge; this partitions the hull.  The table is built
 * by exact scan conversion.  Per covered pixel: planeidx = t and
 * D_it = fma(a_t, u, fma(b_t, v, c_t)) in fp32; outside the hull -1 and NaN.
 * tri_uv: T * 6 int32 vertex coordinates (u0,v0,u1,v1,u2,v2); abc: T * 3 fp32
 * plane coefficients (needed when D_it is given).  planeidx (int32) and D_it
 * (fp32), W*H each, 16-byte aligned; either may be NULL, not both.  scratch:
 * at least stereo_raster_scratch_bytes(T) bytes of device memory. */
int stereo_raster(const int32_t* tri_uv, const float* abc, int T, int w, int h, int32_t* planeidx,
                  float* D_it, void* scratch, size_t scratch_bytes, void* stream);

/* stereo_raster without a scratch argument, for callers that cannot allocate
 * device memory where they run the raster (a real-time loop whose memory is
 * all allocated up front, or code running while another component owns the
 * device allocator).  The
 * paper has no counterpart: it is a memory-management variant of
 * stereo_raster with the same arguments and results otherwise.  Its work
 * lists live in one file-scope device array sized for at most 262143
 * triangles (just over 2 MiB, held by every GPU that loads the library until exit);
 * larger T returns STEREO_E_CAP.  The first call on each device looks up the
 * array's device address (no allocation); make that first call before any
 * stream capture.  The address is kept for the life of the process: after a
 * cudaDeviceReset the entry point must not be called again.  All calls share
 * the array: calls that overlap on the GPU race and must be serialised by the
 * caller. */
int stereo_raster_noalloc(const int32_t* tri_uv, const float* abc, int T, int w, int h,
                          int32_t* planeidx, float* D_it, void* stream);

/* One pass of CostEvaluation (Alg. 2) + DisparityRefinement (Alg. 3) over
 * Omega_I on the interpolated prior D_it (NaN = no triangle).  A pixel in
 * Omega_I is evaluated when k = rint(D_it) keeps the right window inside the
 * image (2 <= u - k <= W - 3); its cost is C = popcount(cL(u,v) ^ cR(u-k,v)).
 * Then, as Alg. 3 in raster order: C < C_f => (D_f, C_f) <- (D_it, C); per
 * sz x sz cell the least C below t_lo (first in raster order on ties) and the
 * largest C above t_hi (first in raster order) are kept as keys:
 *   cg_key[cell] = (C << 27) | (v*W + u),  cb_key[cell] = ((24 - C) << 27) | (v*W + u),
 * 0xFFFFFFFF when empty; both arrays, ceil(H/sz)*ceil(W/sz) entries, must hold
 * 0xFFFFFFFF on entry (atomic minimum), or both be NULL to skip the cells.
 * first_pass = 1 treats D_f, C_f as their initial values (0, t_hi) without
 * reading them, and writes every pixel.  mask (W*H bytes) is required;
 * NULL returns STEREO_E_INVAL. */
int stereo_validate(const uint32_t* cL, const uint32_t* cR, const uint32_t* omega, const float* D_it,
                    int w, int h, int sz, int t_lo, int t_hi, int first_pass, float* D_f,
                    uint8_t* C_f, uint8_t* mask, uint32_t* cg_key, uint32_t* cb_key, void* stream);

/* stereo_validate as a pipelined kernel: one producer warp per block stages
 * each 128x8 tile's inputs into shared memory with asynchronous bulk copies
 * (cp.async.bulk, completion on mbarriers) while eight consumer warps evaluate
 * earlier tiles; the right-census columns a tile row needs are staged too.
 * Same results as stereo_validate.  cL, cR, omega, D_it and C_f must be
 * 16-byte aligned.  err_flag: device int the kernel sets to 1 if one of its
 * bounded waits gave up (the outputs are then incomplete); the caller clears
 * it and reads it after the stream synchronises. */
int stereo_validate_bulk(const uint32_t* cL, const uint32_t* cR, const uint32_t* omega, const float* D_it,
                         int w, int h, int sz, int t_lo, int t_hi, int first_pass, float* D_f,
                         uint8_t* C_f, uint8_t* mask, uint32_t* cg_key, uint32_t* cb_key, int* err_flag,
                         void* stream);

/* SupportResampling (Alg. 4) per cell, fused with SparseEpipolarStereo on the
 * invalid cells: for each cell with a cg key, cg_d = D_it at that pixel; for
 * each cell with a cb key, x_d = the epipolar match of that pixel (as
 * stereo_epipolar_match) or -1.  Cells without keys get cg_d = NaN and
 * x_d = -1.  The caller merges them in cell raster order. */
int stereo_resample_match(const uint32_t* cg_key, const uint32_t* cb_key, int ncells, const float* D_it,
                          const uint32_t* cL, const uint32_t* cR, int w, int h, int dmax,
                          int t_lo, int margin, float* cg_d, int32_t* x_d, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* STEREO_H */
