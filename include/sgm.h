/*
 * sgm.h -- C ABI of the GB300 (sm_103a) Semi-Global Matching hot path.
 *
 * Method: Hernandez-Juarez et al., "Embedded real-time stereo estimation via
 * Semi-Global Matching on the GPU", arXiv 1610.04121.  The library computes,
 * for a rectified pair (base = left image, match = right image):
 *   1. the 9x7 center-symmetric Census feature of every pixel (Eq. 1);
 *   2. the matching cost MC(x,y,d) = bitcount(F_base(x,y) XOR F_match(x-d,y))
 *      for d in [0, D) (Eq. 2);
 *   3. the aggregated cost L_r along 2, 4 or 8 path directions (Eq. 3);
 *   4. the summed cost S = sum_r L_r and the winner-take-all disparity
 *      argmin_d S, lowest d on ties (Eq. 4);
 *   5. a 3x3 median filter of that disparity (Section 2, stage 4).
 * The problem statement is "two rectified images in, one disparity image out"
 * (Section 2, Fig. 2).  All arithmetic is integer and the output is exact.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  Images   uint8, row-major, pitch = W bytes, H rows.
 *  Output   uint8 disparity, row-major, pitch = W (values 0 .. D-1).
 *  W, H     >= 1.
 *  D        one of 32, 64, 96, 128, 160, 192, 224, 256.
 *  P1, P2   penalties of Eq. 3, each in [0, 224] (keeps every L_r <= 255);
 *           P2 <= 193 in a context created with SGM_FLAG_CENSUS_FULL.
 *  n_paths  2 (left-to-right, top-to-bottom), 4 (adds right-to-left and
 *           bottom-to-top) or 8 (adds the four diagonals) (Section 4).
 *  Borders  the feature is 0 where the 9x7 window leaves the image, and a
 *           match column x-d < 0 uses the feature 0; the first pixel of each
 *           path takes L_r = MC; the median copies the one-pixel border ring.
 *  Pointers "host or device": the library asks the CUDA runtime which kind a
 *           pointer is.  Host memory may be pageable (copied through the
 *           context's arena with cudaMemcpyAsync) or pinned (copied to and
 *           from the arena by a staging kernel).  Device pointers must be on
 *           the context's device and are used in place.
 *  Ownership the caller owns every buffer it passes; the library never frees
 *           or keeps a caller pointer beyond the call, except for
 *           sgm_submit (see there).  The library owns its context, its device
 *           work arena and its CUDA graphs.
 *  Errors   every function returns an sgm_status; nothing is thrown across
 *           the ABI.  sgm_last_error(ctx) gives a human-readable reason for
 *           the last failure on that context (thread-local to the context).
 *  Threads  one context must not be used by two threads at once, except that
 *           sgm_submit / sgm_poll may be called from any thread.
 */
#ifndef SGM_GB300_H
#define SGM_GB300_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define SGM_API __attribute__((visibility("default")))
#else
#define SGM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sgm_ctx sgm_ctx;

typedef enum sgm_status {
    SGM_OK = 0,
    SGM_EAGAIN = 1,      /* sgm_poll: the request is still running; sgm_submit: shed by the admission bound */
    SGM_EINVAL = -1,     /* bad argument (sizes, D, penalties, paths, null pointer, unknown ticket) */
    SGM_ENOMEM = -2,     /* device memory (or the context's memory cap) exhausted */
    SGM_ECUDA = -3,      /* a CUDA runtime call failed; see sgm_last_error */
    SGM_ETIMEDOUT = -4,  /* sgm_poll: the timeout elapsed */
    SGM_ECANCELED = -5,  /* the request was cancelled by sgm_destroy */
    SGM_EDEVICE = -6     /* a batched kernel rejected a work-list descriptor (the device status word) */
} sgm_status;

/* sgm_create flags. */
#define SGM_FLAG_STAGE_TIMING 1u /* record a CUDA event between the kernels of every path (sgm_stage_times) */
#define SGM_FLAG_CENSUS_FULL 2u  /* features: the full 9x7 Census (62 bits, every pixel of the window against \
                                    the centre) in place of the CSCT of Eq. 1; matching costs reach 62, so \
                                    P2 must not exceed 255 - 62 = 193 */

/* Limits checked by every entry point. */
#define SGM_MAX_D 256
#define SGM_MAX_PENALTY 224

/* One pair of a batch (sgm_compute_batch).  Pointers as described above. */
typedef struct sgm_pair {
    const uint8_t *left;
    const uint8_t *right;
    uint8_t *disp_out;
    int32_t W, H, D, P1, P2, n_paths;
} sgm_pair;

/*
 * Create a context on CUDA device `device` (makes it current for the calling
 * thread).  `mem_cap_bytes` caps the device memory the context may hold for
 * its work arena and served requests (0 = no cap beyond the device's free
 * memory).  `flags` is 0 or a combination of SGM_FLAG_STAGE_TIMING and
 * SGM_FLAG_CENSUS_FULL; the Census type holds for every entry point of the
 * context (sgm_compute_static always uses the CSCT).  On success *out
 * receives the context.
 * Test hooks, read from the environment here (host side only; no kernel is
 * made to fault): SGM_TEST_FAIL_ALLOC=n makes the context's n-th device or
 * pinned-host allocation fail as if memory were exhausted (the call that
 * needed it returns SGM_ENOMEM, or sgm_create itself for its own first
 * allocations, and the context stays usable); SGM_TEST_BAD_JOB=n gives the
 * first n batched waves one sweep descriptor with a wrong D, which its kernel
 * skips and reports through the device status word (SGM_EDEVICE).
 * Errors: SGM_EINVAL (null out, bad device, unknown flag), SGM_ENOMEM,
 * SGM_ECUDA.
 */
SGM_API int sgm_create(sgm_ctx **out, int device, size_t mem_cap_bytes, unsigned flags);

/*
 * Destroy a context: requests submitted and not yet finished are cancelled
 * (their tickets then poll as SGM_ECANCELED is no longer observable, since
 * the context is gone); the call waits for work already on the GPU to end,
 * then frees every device and host resource.  NULL is accepted (no-op).
 */
SGM_API int sgm_destroy(sgm_ctx *ctx);

/* Text of the last error on this context ("" if none); valid until the next
 * call on the context.  Accepts NULL (returns a static message). */
SGM_API const char *sgm_last_error(const sgm_ctx *ctx);

/*
 * Make the context enqueue its work on `cuda_stream` (a cudaStream_t of the
 * context's device, or NULL for the context's own stream; the default
 * stream, whose handle is NULL, is selected with cudaStreamLegacy or
 * cudaStreamPerThread).  The caller keeps the stream alive while the context
 * uses it.
 */
SGM_API int sgm_set_stream(sgm_ctx *ctx, void *cuda_stream);

/*
 * Blocking disparity computation (Section 2, stages 1-5): copies host
 * inputs in if needed, runs the whole path on the GPU, copies the result out
 * if `disp_out` is host memory, and returns when `disp_out` holds the
 * median-filtered disparity.  Uses the context's arena (grown on demand).
 * Errors: SGM_EINVAL, SGM_ENOMEM, SGM_ECUDA, SGM_EDEVICE.
 */
SGM_API int sgm_compute(sgm_ctx *ctx, const uint8_t *left, const uint8_t *right, int W, int H, int D, int P1, int P2,
                int n_paths, uint8_t *disp_out);

/* Post-filter flags of sgm_compute_ex (the post-filters Section 5 of the
 * paper announces; the paper gives no definition, these are the readings). */
#define SGM_POST_SUBPIXEL 1u    /* parabola vertex through S(d-1), S(d), S(d+1) at the winner d */
#define SGM_POST_LR_CHECK 2u    /* left-right consistency check */
#define SGM_POST_ADAPTIVE_P2 4u /* P2 per step from the base image's intensity step */
#define SGM_DISP16_INVALID 0xFFFFu

/*
 * sgm_compute with post-filters; `post` is 0 or a combination of the
 * SGM_POST_* flags; disp16_out is uint16 [H][W] in 1/16 pixel.  Pointers as
 * sgm_compute (host or device); blocking.
 *   - ADAPTIVE_P2: the step q -> p of every path uses
 *     P2(p, q) = max(P1, P2 / (1 + |I(p) - I(q)|)) (integer division, I the
 *     base image) in place of P2 in Eq. 3; needs max(P1, P2) <= 255 - 31
 *     (255 - 62 with SGM_FLAG_CENSUS_FULL).
 *   - SUBPIXEL: at the winner d of Eq. 4 with 0 < d < D-1 the value is
 *     16 d + floor((16 (S(d-1) - S(d+1)) + den) / (2 den)),
 *     den = S(d-1) + S(d+1) - 2 S(d) (the vertex offset rounded to 1/16,
 *     halves up; within [-8, 8]); else 16 d.
 *   - the 3x3 median (Section 2) then runs on these values (border ring
 *     copied);
 *   - LR_CHECK: the right image's disparity d_R is the same matching pass on
 *     the mirrored pair (base = mirrored right, match = mirrored left), read
 *     back in original columns; left pixel x with winner d is kept when
 *     x - d >= 0 and |d - d_R(x - d)| <= 1, else the output is
 *     SGM_DISP16_INVALID.
 * With post = 0 the output is 16 x that of sgm_compute.  Stage timing does
 * not cover this entry point.  Errors as sgm_compute (SGM_EINVAL also for
 * unknown flags and the adaptive P2 bound).
 */
SGM_API int sgm_compute_ex(sgm_ctx *ctx, const uint8_t *left, const uint8_t *right, int W, int H, int D, int P1,
                           int P2, int n_paths, unsigned post, uint16_t *disp16_out);

/* Non-blocking sgm_compute_ex for device pointers only (as sgm_compute_async). */
SGM_API int sgm_compute_ex_async(sgm_ctx *ctx, const uint8_t *left, const uint8_t *right, int W, int H, int D,
                                 int P1, int P2, int n_paths, unsigned post, uint16_t *disp16_out);

/*
 * Non-blocking form for device pointers only: enqueues the whole path on the
 * context's stream and returns at once.  `left`, `right` and `disp_out` must
 * be device memory; the caller synchronises the stream before reading
 * `disp_out`.  The launch sequence for one (W, H, D, P1, P2, n_paths) and one
 * set of pointers is captured once into a CUDA graph and replayed.
 * Errors: SGM_EINVAL (including host pointers), SGM_ENOMEM, SGM_ECUDA.
 */
SGM_API int sgm_compute_async(sgm_ctx *ctx, const uint8_t *left, const uint8_t *right, int W, int H, int D, int P1, int P2,
                      int n_paths, uint8_t *disp_out);

/*
 * Batched computation of `n` independent pairs of possibly different sizes,
 * D, penalties and path counts (the paper's scaling argument, Section 4,
 * applied to many pairs at once).  Pairs are grouped by (D, path count, sum
 * width); every stage of a group is one persistent grid whose blocks take
 * units (tiles, row segments, blocks of sweep lines) from a device work list
 * covering the group's pairs, longest chains first.  A wave (the pairs whose
 * buffers fit the memory budget at once, at most 16 groups) is one CUDA
 * graph launch, the groups on concurrent branches; the graph is captured
 * once per wave shape and replayed with the lists rewritten.  The first wave
 * of a new set of pair shapes autotunes the sweep grid (persistent blocks per
 * SM from {2, 3, 4, 5}: one warm-up and five timed runs each, the lowest
 * median wins; the call blocks meanwhile).  Pointers of each pair as in
 * sgm_compute (all host or all device per pair).  Blocking.
 * Each pair's result is bit-identical to sgm_compute of that pair alone.
 * Errors: SGM_EINVAL (n < 0, null pairs, any invalid pair), SGM_ENOMEM,
 * SGM_ECUDA, SGM_EDEVICE (a kernel rejected a descriptor; the context
 * stays usable).
 */
SGM_API int sgm_compute_batch(sgm_ctx *ctx, int n, const sgm_pair *pairs);

/*
 * Served form: queue one pair and return a ticket at once.  A scheduler
 * thread owned by the context admits queued requests in arrival order while
 * device memory (within mem_cap_bytes) allows, batches whatever is admitted
 * into one launch sequence (the batched path of sgm_compute_batch, each
 * batch on its own stream with its own arena from a device-resident pool),
 * and keeps up to two batches in flight on the GPU: requests that arrive
 * while a batch runs are admitted into the next one as soon as a slot is
 * free.  Each result is bit-identical to sgm_compute of that pair alone.
 * The caller keeps left/right/disp_out alive and unmodified until sgm_poll
 * returns something other than SGM_EAGAIN for the ticket.
 * With an admission bound set (sgm_set_admission_bound) a request whose
 * estimated wait exceeds it is shed: SGM_EAGAIN, nothing queued, no ticket.
 * Errors: SGM_EINVAL (bad pair or null ticket), SGM_ENOMEM (the pair alone
 * exceeds the memory cap).
 */
SGM_API int sgm_submit(sgm_ctx *ctx, const uint8_t *left, const uint8_t *right, int W, int H, int D, int P1, int P2,
               int n_paths, uint8_t *disp_out, uint64_t *ticket);

/*
 * Wait up to `timeout_us` microseconds (0 = just test, < 0 = wait forever)
 * for a submitted request.  Returns SGM_OK once `disp_out` holds the result
 * (the ticket is then retired), SGM_EAGAIN if timeout_us == 0 and it is not
 * done, SGM_ETIMEDOUT if the wait elapsed, SGM_EINVAL for an unknown ticket,
 * or the request's own error status.
 */
SGM_API int sgm_poll(sgm_ctx *ctx, uint64_t ticket, int64_t timeout_us);

/*
 * Served-request statistics since the context was created:
 * out[0] = completed requests, out[1] = p50 latency (us), out[2] = p99
 * latency (us), out[3] = max latency (us); latency = completion of the
 * request's batch on the GPU (its last copy) minus submit time.  `n_out`
 * must be >= 4.  With n_out >= 8 also: out[4] = batches launched, out[5] =
 * mean pairs per batch, out[6] = most batches in flight at once, out[7] =
 * disparity evaluations (W*H*D) of the completed requests.  With n_out >= 10
 * also: out[8] = requests shed by the admission bound, out[9] = the measured
 * service rate: disparity evaluations per second of time with a served batch
 * in flight, over the context's life (0 before the first batch finishes).
 * With n_out >= 13 also the current state: out[10] = requests queued and not
 * yet admitted, out[11] = batches in flight, out[12] = device bytes held by
 * the served slots' arenas (the pool's occupancy).
 */
SGM_API int sgm_served_stats(sgm_ctx *ctx, double *out, int n_out);

/*
 * Admission bound of the served form: sgm_submit sheds (SGM_EAGAIN) a
 * request whose estimated wait exceeds max_wait_us.  The estimate is the
 * disparity evaluations (W*H*D) queued or running, the new request's
 * included, over the service rate measured so far (every evaluation served
 * over the time the GPU had a served batch in flight); before the first
 * batch has finished nothing is shed.  0 (the default) = no bound.
 * Errors: SGM_EINVAL (null context, max_wait_us < 0).
 */
SGM_API int sgm_set_admission_bound(sgm_ctx *ctx, int64_t max_wait_us);

/*
 * The autotuners' results as a JSON file: the 4-path sweep schedule per
 * (W, H, D, n_paths, Census type, byte sums) key and the batched sweep grid
 * per set of pair shapes.  sgm_load_tuning merges a saved file into a context
 * on a device with the same SM count, so that a new process skips the timed
 * tuning runs.  Nothing else of a context persists.
 * Errors: SGM_EINVAL (null context or path, a file that cannot be written or
 * read, is malformed, or was tuned on a device with another SM count).
 */
SGM_API int sgm_save_tuning(const sgm_ctx *ctx, const char *path);
SGM_API int sgm_load_tuning(sgm_ctx *ctx, const char *path);

/*
 * Start a new statistics window for sgm_served_stats (for example after a
 * warm-up): clears the latencies, batch counts and DE total; requests in
 * flight are counted in the new window when they complete.
 * Errors: SGM_EINVAL (null context).
 */
SGM_API int sgm_served_reset_stats(sgm_ctx *ctx);

/*
 * Debug form of sgm_compute for localising a mismatch stage by stage.  All
 * pointers are host pointers; each optional output may be NULL:
 *   Fb, Fm   uint32 [H][W]    Census features of left and right (Eq. 1); uint64 [H][W]
 *                             in a context created with SGM_FLAG_CENSUS_FULL
 *   MC       uint8  [H][W][D] matching cost (Eq. 2), d fastest
 *   S        uint16 [H][W][D] summed aggregated cost (Eq. 4's sum)
 *   raw      uint8  [H][W]    winner-take-all disparity before the median
 *   disp     uint8  [H][W]    final disparity
 * A 4-path problem runs the schedule forced by sgm_set_schedule, else
 * SGM_SCHED_V_THEN_H (it is not autotuned).  Errors as sgm_compute.
 */
SGM_API int sgm_debug_stages(sgm_ctx *ctx, const uint8_t *left, const uint8_t *right, int W, int H, int D, int P1, int P2,
                     int n_paths, void *Fb, void *Fm, uint8_t *MC, uint16_t *S, uint8_t *raw, uint8_t *disp);

/*
 * Per-kernel device times (milliseconds) of the most recent path this context
 * enqueued through sgm_compute / sgm_compute_async, in launch order; needs a
 * context created with SGM_FLAG_STAGE_TIMING.  Waits for that path to finish.
 * Writes min(n, stages) values to ms_out and returns the number of stages
 * (5 for 2 or 4 paths, 7 for 8 paths), or a negative sgm_status.  Stage
 * names, in order (sgm_stage_name): census, cost, then the sweeps, then
 * median.  Sweeps with 2 paths: sweep_h (left to right), sweep_v (top to
 * bottom with the winner-take-all).  With 4 paths: sweep_v+h1 (the whole
 * vertical pair beside the first halves of the horizontal pair), sweep_h2
 * (the horizontal second halves with the winner-take-all).  With 8 paths:
 * sweep_h (the horizontal pair with the first halves of the three
 * vertical-type pairs), sweep_diag+, sweep_diag-, sweep_v.
 */
SGM_API int sgm_stage_times(sgm_ctx *ctx, float *ms_out, int n);

/* Name of stage i of a path with n_paths directions, or NULL. */
SGM_API const char *sgm_stage_name(int n_paths, int i);

/*
 * The bounds-checked build (the library compiled with -DSGM_BOUNDS_CHECK,
 * `python -m paper_1610_04121_gb300.build --bounds-check`): every global
 * access of the kernels, and the shared-memory feature indices of the cost
 * kernels, is tested against the extent of its array; a violation records a
 * site number in a device fault word and skips the access (no trap).  The
 * synchronous calls (sgm_compute, sgm_compute_ex, sgm_compute_batch,
 * sgm_debug_stages, and sgm_poll for served requests) then return
 * SGM_EDEVICE.  sgm_bounds_checked() is 1 in that build, else 0;
 * sgm_bounds_fault() returns and clears the first recorded site (0: none),
 * for callers of the asynchronous entry points.
 */
SGM_API int sgm_bounds_checked(void);
SGM_API unsigned sgm_bounds_fault(void);

/* Path count (2, 4 or 8) of the path that sgm_stage_times reports on, or 0
 * when none has been enqueued with SGM_FLAG_STAGE_TIMING. */
SGM_API int sgm_stage_paths(const sgm_ctx *ctx);

/* Name of stage i of the path that sgm_stage_times reports on (it follows
 * that path's sweep schedule: with SGM_SCHED_H_THEN_V the 4-path sweeps are
 * sweep_h+v1, sweep_v2; with SGM_SCHED_PAIRS pairs_vh, pairs_h_wta), or NULL. */
SGM_API const char *sgm_stage_label(const sgm_ctx *ctx, int i);

/*
 * Sweep schedules of the 4-path plain path (sgm_compute, sgm_compute_async;
 * Eq. 3 along the four paths of Section 4, then Eq. 4):
 *   SGM_SCHED_V_THEN_H  the whole vertical pair (writing S) beside the first
 *                       halves of the horizontal pair, then the horizontal
 *                       second halves with the winner-take-all;
 *   SGM_SCHED_H_THEN_V  the whole horizontal pair beside the vertical first
 *                       halves, then the vertical second halves with the
 *                       winner-take-all;
 *   SGM_SCHED_PAIRS     two lines per warp over 2 x 2 pixel quads: the whole
 *                       vertical pair beside min(W, H) steps of each
 *                       horizontal direction, then the rest of the
 *                       horizontal directions with the winner-take-all
 *                       beside a parallel winner-take-all over the columns
 *                       both horizontal directions passed (the longest
 *                       chain is max(W, H) steps).  Not offered when its
 *                       quad records would pass 4 GiB.
 * All give bit-identical results.  By default the context autotunes: the
 * first call for a new (W, H, D, Census type, byte-sum) key runs the path
 * with each schedule (once to warm up, then five times timed with CUDA
 * events on the context's stream; that call blocks meanwhile) and keeps the
 * one with the lowest median for the key; a stream under capture is not
 * tuned (the first schedule is used).  sgm_set_schedule(ctx, s) forces
 * schedule s; -1 restores autotuning.
 * Errors: SGM_EINVAL (null context, unknown schedule).
 */
#define SGM_SCHED_V_THEN_H 0
#define SGM_SCHED_H_THEN_V 1
#define SGM_SCHED_PAIRS 2
SGM_API int sgm_set_schedule(sgm_ctx *ctx, int schedule);

/* The schedule the context uses for this problem: the forced one, the tuned
 * one, SGM_SCHED_V_THEN_H for 2 and 8 paths, or -1 when not tuned yet. */
SGM_API int sgm_schedule_for(const sgm_ctx *ctx, int W, int H, int D, int P1, int P2, int n_paths);

/*
 * Kernel launches issued by this context so far (every launch of this
 * library's kernels, counted on the host when enqueued; a replayed graph
 * adds the launches it contains).
 */
SGM_API uint64_t sgm_kernel_launches(const sgm_ctx *ctx);

/* Library version string. */
SGM_API const char *sgm_version(void);

/*
 * Allocation-free form of sgm_compute_async, for callers that cannot allocate
 * device memory: code running where cudaMalloc is forbidden or unavailable
 * (an embedding runtime that owns all device memory, a plugin that may only
 * use what its host hands it, or a real-time loop that must never allocate).
 * The paper has no counterpart: it is an interface addition of this library.
 *
 * `left`, `right` and `disp_out` are device pointers on the current device;
 * the call enqueues the whole path on `cuda_stream` (NULL = the legacy default
 * stream) and returns without waiting.  It needs no context and calls no
 * cudaMalloc, cudaFree or other allocating routine: every intermediate lives
 * in one static device array of 48 MiB that each GPU which loads the library
 * keeps until the process exits.  The intermediates take 8 W H bytes for the
 * features, W H (3 D) bytes (2 paths) or W H (4 D) bytes (4 or 8 paths) for
 * the per-pixel records and W H for the raw disparity; sizes that do not fit
 * are rejected with SGM_EINVAL (320x240 with D = 128 and 8 paths fits, about
 * 40 MB; 640x480 with D = 128 does not).
 *
 * The first call on a device looks up the array's device address and sets
 * kernel attributes; make that first call before any stream capture.  Every
 * call shares the one array and leaves the last call's contents in it (no
 * part of it needs to start at zero: each byte is written before it is read),
 * so calls that overlap on the GPU -- on different streams, or from different
 * threads -- race: serialise them.  Results are bit-identical to sgm_compute.
 * Errors (sgm_last_error(NULL) gives the text): SGM_EINVAL (null or host
 * pointer, bad sizes, D, penalties or paths, scratch too small), SGM_ECUDA.
 */
SGM_API int sgm_compute_static(const uint8_t *left, const uint8_t *right, int W, int H, int D, int P1, int P2,
                               int n_paths, uint8_t *disp_out, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* SGM_GB300_H */
