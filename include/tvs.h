/*
 * tvs.h -- C ABI of the GB300 (sm_103a) total-viewshed library, an
 * implementation of the sDEM method (skewed Digital Elevation Model) of
 * Sanchez-Fernandez, Romero, Bandera and Tabik, arXiv 2003.02200.
 *
 * What a call computes (section 3 and 4.1 of the paper):
 *   every DEM cell is a point of view (POV) lifted by the observer height h0;
 *   for each of n directions theta_k = k*pi/n the DEM is relocated into a
 *   skewed layout in which every sampled line of sight is one contiguous row
 *   (Kernel-1, Alg. 6); every sample of every row is then a virtual POV that
 *   walks its row forward and backward, keeping the running maximum elevation
 *   angle (Kernel-2, Alg. 7 and 8), and the measure of its visible ring
 *   sectors is blended back onto the DEM cells (Kernel-3, Alg. 9) and summed
 *   over directions.  Result: the visible area of every cell, in the square of
 *   the grid-step unit (m^2 for metres), scaled by the Pappus factor pi/(2n)
 *   (the pi/360 of the ring-sector area equation for n = 180).
 *
 * Conventions shared by every entry point:
 *   - DEM: rows x cols float32, row-major, rows north to south, columns west
 *     to east (section 4.1); rows >= 2 and cols >= 2.
 *   - n_sectors counts directions over 180 degrees (each direction is walked
 *     both ways, so 180 means one-degree sectors).
 *   - max_range_m <= 0 or +inf means unlimited; otherwise only targets within
 *     floor(max_range_m / (step_m * sqrt(1 + t^2))) steps count.
 *   - Every function returns TVS_OK (0) or a negative TVS_ERR_* code; the
 *     message of the last failure on the calling thread is tvs_last_error().
 *   - A handle is not thread-safe: one call at a time per handle.  Calls of
 *     one handle on different CUDA streams must not overlap on the GPU (they
 *     share the handle's device scratch).
 */
#ifndef TVS_H
#define TVS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TVS_ABI_VERSION 2

#define TVS_OK            0
#define TVS_ERR_ARG     (-1)  /* bad pointer, size, step, height, count or non-finite value */
#define TVS_ERR_OOM     (-2)  /* the work does not fit the HBM budget, or cudaMalloc failed */
#define TVS_ERR_CUDA    (-3)  /* CUDA runtime error (no device, launch failure, ...) */
#define TVS_ERR_TIMEOUT (-4)  /* a bounded wait gave up (tvs_server_wait); no kernel of the
                                 library waits on a flag or a barrier of another CTA */
#define TVS_ERR_STATE   (-5)  /* handle in a state that cannot serve the call */

typedef struct tvs_ctx* tvs_handle;

/* One direction k of n (section 4.1 step 1; Alg. 6 covers 0..45 degrees and the
 * other eighths use a D4 view of the DEM).  Host-side description. */
typedef struct {
    int32_t  frame;   /* 0 identity, 1 transpose, 2 transpose + mirrored columns, 3 mirrored rows */
    int32_t  m;       /* reduced angle alpha = pi*m/(2n), 0 <= alpha <= pi/4 */
    int32_t  H, W;    /* shape of the view; W is the walk axis */
    int32_t  D;       /* dest(W-1): shift of the last column, in rows */
    int32_t  R;       /* rows of the skewed layout, H + D */
    uint64_t t_fx;    /* llround(tan(alpha) * 2^32) */
    double   t;       /* t_fx * 2^-32 */
    double   g;       /* 1 + t^2, the (1/cos s)^2 factor of Alg. 7 */
    int64_t  K;       /* walk limit in steps (INT64_MAX when unlimited) */
} tvs_direction_info;

/* Per-kernel timing kept while profiling is on (CUDA events on the launch stream). */
typedef struct {
    char     name[32];
    int64_t  launches;
    double   total_ms;
    double   units;        /* algorithmic units summed over launches (see unit) */
    char     unit[16];     /* "evals" for the sweep and the point walks, "bytes" for the
                              memory kernels, "cells" (cell x POV pairs) for the map raster */
} tvs_kernel_stats;

/* ABI version of the loaded library (TVS_ABI_VERSION).  Host only. */
int tvs_abi_version(void);

/* Create a handle bound to CUDA device `device`.  hbm_budget_bytes caps the
 * device scratch the handle may hold (0 = min(16 GiB, 60% of free memory)).
 * The handle owns its scratch; the caller owns every input and output.
 * Errors: TVS_ERR_ARG (out == NULL, bad device), TVS_ERR_CUDA (no usable GPU). */
int tvs_create(tvs_handle* out, int device, size_t hbm_budget_bytes);

/* Release the handle and its device scratch.  NULL is accepted. */
void tvs_destroy(tvs_handle h);

/* Message of the last failing call made by this thread ("" if none).  The
 * pointer stays valid until the thread's next failing call. */
const char* tvs_last_error(tvs_handle h);

/* Total viewshed from HOST memory (Alg. 4, computed the sDEM way of section 4).
 * dem: rows*cols float32 elevations (metres), row-major, finite.
 * step_m > 0: grid step; obs_height_m: h0 >= 0 (finite); n_sectors >= 1.
 * out: rows*cols float32, visible area of each cell in m^2, laid out like dem.
 * Synchronous: on return `out` holds the result.  The library copies dem to
 * the device and out back inside the call.
 * Errors: TVS_ERR_ARG, TVS_ERR_OOM, TVS_ERR_CUDA. */
int tvs_total_viewshed(tvs_handle h, const float* dem, int rows, int cols, double step_m,
                       double obs_height_m, int n_sectors, double max_range_m, float* out);

/* Same computation on DEVICE memory, ordered on `cuda_stream` (a cudaStream_t,
 * NULL = legacy default stream).  d_dem and d_out are device pointers of
 * rows*cols float32 on the handle's device (they may not overlap).  The call
 * returns once the work is enqueued; d_out is complete when the stream reaches
 * that point.  Elevations are not scanned for NaN/inf on this path (the result
 * of a non-finite DEM is unspecified).  Scratch is (re)allocated inside the call
 * when the job needs more than the handle holds; that allocation synchronises
 * the device once.  Errors: TVS_ERR_ARG, TVS_ERR_OOM, TVS_ERR_CUDA. */
int tvs_total_viewshed_device(tvs_handle h, const float* d_dem, int rows, int cols, double step_m,
                              double obs_height_m, int n_sectors, double max_range_m, float* d_out,
                              void* cuda_stream);

/* Same computation as tvs_total_viewshed_device, for callers that cannot
 * allocate device memory (a framework whose caching allocator owns the GPU's
 * memory budget, or a latency-bound loop that must not pay the device-wide
 * synchronisation of cudaMalloc/cudaFree).  It takes no handle and allocates
 * nothing: all scratch lives in one file-scope device array of 64 MiB, reserved
 * when the library's device code is loaded and held by every GPU that loads it
 * until the process exits.  The paper has no counterpart to this entry point.
 * Runs on the calling thread's current device, ordered on `cuda_stream`
 * (a cudaStream_t, NULL = legacy default stream); d_dem, d_out (rows*cols
 * float32 each, not overlapping) and the stream must belong to that device.
 * The first call on a device resolves the array's device address
 * (cudaGetSymbolAddress).  The entry point cannot be captured into a CUDA
 * graph: its tables reach the device through copies from host memory that the
 * next call reuses, so a call on a capturing stream returns TVS_ERR_ARG.
 * Every call shares the one array (it keeps the last call's contents; the
 * entry point resets what must start at zero), so calls that overlap on the
 * GPU race: order them on one stream or synchronise between them.  Its host
 * tables are static too (not on the calling thread's stack, so a worker
 * thread with a small stack may call it), and host threads take turns
 * through the entry point.
 * Limits: n_sectors <= 1024, and the job must fit 64 MiB: 16 bytes per DEM
 * cell (exact running totals) plus 8 bytes per skewed sample of at least one
 * direction (a diagonal direction of an S x S DEM has about 2 S^2 samples, so
 * S <= 1440 fits; larger jobs return TVS_ERR_OOM with a message).
 * Errors: TVS_ERR_ARG, TVS_ERR_OOM, TVS_ERR_CUDA. */
int tvs_total_viewshed_device_noalloc(const float* d_dem, int rows, int cols, double step_m,
                                      double obs_height_m, int n_sectors, double max_range_m, float* d_out,
                                      void* cuda_stream);

/* One DEM of a batch: device buffers of rows*cols float32 each (they may not
 * overlap) and the same parameters as tvs_total_viewshed_device. */
typedef struct {
    const float* d_dem;
    float* d_out;
    int rows, cols;
    double step_m;
    double obs_height_m;
    int n_sectors;
    double max_range_m;
} tvs_job;

/* Total viewsheds of njobs DEMs of any sizes and parameters in one pass
 * (section 4.1 applied to each DEM): the (DEM, direction) pairs of all jobs are
 * planned together into chunks that fit the handle's HBM budget, and each chunk
 * runs one launch per kernel for all of its DEMs, so small DEMs share the GPU
 * instead of running one after another.  Each job's result is bit for bit
 * what tvs_total_viewshed_device gives for it: per-cell totals are exact sums
 * of FP32 partial sums over fixed groups of 8 directions, so they do not
 * depend on which chunk or which CTA added a group (the one exception: a
 * budget too small for 8 directions of a job cuts inside a group, which moves
 * results by FP32 rounding only).  Stream-ordered like
 * tvs_total_viewshed_device.
 * Errors: TVS_ERR_ARG (a bad job: the message names its index), TVS_ERR_OOM,
 * TVS_ERR_CUDA. */
int tvs_total_viewshed_batch(tvs_handle h, const tvs_job* jobs, int njobs, void* cuda_stream);

/* A prepared batch: the plan of a fixed set of jobs (same buffers, same
 * parameters every time), its own device scratch (hbm_budget_bytes, 0 = the
 * handle's budget), its tables uploaded once, and its launch sequence captured
 * once in a CUDA graph.  tvs_batch_launch replays the graph on a stream; the
 * caller may change the contents of the jobs' d_dem between launches, not the
 * pointers or parameters.  Launches of one prepared batch must not overlap on
 * the GPU (they share its scratch).  tvs_batch_destroy is NULL-safe. */
typedef struct tvs_batch* tvs_batch_handle;

typedef struct {
    int32_t  jobs;
    int32_t  chunks;            /* chunks of (DEM, direction) pairs */
    int32_t  kernels_per_launch;
    int32_t  pad_;
    double   evals;             /* evaluations of one launch (the work count) */
    double   scratch_bytes;
} tvs_batch_info;

int tvs_batch_create(tvs_handle h, const tvs_job* jobs, int njobs, size_t hbm_budget_bytes,
                     tvs_batch_handle* out);
int tvs_batch_launch(tvs_batch_handle b, void* cuda_stream);
int tvs_batch_get_info(tvs_batch_handle b, tvs_batch_info* info);
void tvs_batch_destroy(tvs_batch_handle b);

/* Launch choices of a handle (no effect on results, only on speed, except
 * fp32_decisions).
 * small_pov_below_w: every skewed row of a direction whose walk axis is
 *   shorter than this is swept with 4 POVs per lane group (default 0: none);
 * p4_cost_pct: the other rows pick 4 or 8 POVs per lane group row by row,
 *   whichever needs fewer warp items x walk steps x POVs x step cost, where a
 *   4-POV step costs p4_cost_pct percent of an 8-POV step per POV (default
 *   107; 1 << 20 keeps every such row on 8; 0 in tvs_set_tuning = default);
 * sweep_max_warps: warps per sweep CTA, 0 = as many as shared memory allows,
 *   at most 16 (default 0; certified launches whose rows need one staged row
 *   per pair of warps take at most 12 when pruning, where the 12-warp build
 *   runs without register spills and was measured faster);
 * unskew_ctas_per_sm: a chunk whose DEMs have fewer cell tiles than this many
 *   per SM splits its directions into ranges across CTAs (1 to 4, default 2);
 * prune: exact horizon pruning in the sweep (1, default) or none (0): a group
 *   of POVs stops walking once no remaining target can rise above its running
 *   maximum elevation angle (bounded through the row's suffix maximum with
 *   monotone rounding), which leaves every result bit for bit the same;
 *   the work count (evaluations) stays the unpruned one.
 * fp32_decisions: 0 (default) takes every visibility decision (Alg. 8's
 *   comparison of a target's elevation angle with the running maximum) as
 *   exact arithmetic on the blended heights takes it -- FP32 decisions proved
 *   by an error bound, double-float and FP64 walks where the bound does not
 *   settle one -- so each per-sample measure equals the FP64 definition's;
 *   1 takes them in single precision as the paper's kernels declare heights
 *   and slopes (float in Alg. 6-8): (1 - r) a + r b, h = z + h0,
 *   (z - h) * (1/d) rounded at every step, which flips near-ties.  This
 *   field changes results (by such flips only). */
typedef struct {
    int32_t small_pov_below_w;
    int32_t sweep_max_warps;
    int32_t unskew_ctas_per_sm;
    int32_t p4_cost_pct;
    int32_t prune;
    int32_t fp32_decisions;
} tvs_tuning;

int tvs_get_tuning(tvs_handle h, tvs_tuning* t);
int tvs_set_tuning(tvs_handle h, const tvs_tuning* t);

/* Autotuner: times candidate tunings on the caller's jobs (each candidate
 * runs the whole batch once to warm up and once timed with CUDA events on the
 * handle's stream), searching one choice at a time, keeps the fastest in the
 * handle and returns it in *best and its batch time in *best_ms (both
 * optional).  The jobs' outputs are overwritten.  Synchronous. */
int tvs_autotune(tvs_handle h, const tvs_job* jobs, int njobs, tvs_tuning* best, double* best_ms);

/* Direction table entry k of n for a rows x cols DEM (host only, no GPU). */
int tvs_direction(int n_sectors, int k, int rows, int cols, double step_m, double max_range_m,
                  tvs_direction_info* info);

/* Work count of a job: the number of (virtual POV, direction, target) visits,
 * sum over directions, skewed rows and their usable samples of
 * min(L_fwd, K) + min(L_bwd, K).  Host only; returns a negative code on bad args. */
int64_t tvs_count_evals(int rows, int cols, int n_sectors, double step_m, double max_range_m);

/* Host-only test hook of the batch planner (no GPU): plans njobs whole jobs
 * -- job j a rows[j] x cols[j] DEM with n_sectors[j] directions, step_m[j]
 * and max_range_m[j] (the observer height does not change a plan) -- the way
 * tvs_total_viewshed_batch does on the device path under a scratch budget of
 * budget_bytes on a GPU of num_sms SMs with smem_optin bytes of opt-in shared
 * memory per CTA (0: the planner ignores the sweep's shared-memory layouts),
 * with exact pruning `prune` (0/1) and FP32 decisions `fp32_decisions` (0/1).
 * Writes, for every planned (job, direction) instance in launch order, its
 * job inst_job[i], its direction inst_k[i] and its chunk inst_chunk[i]
 * (chunks are launched in order, each one pass of the pipeline), and the
 * counts *ninst and *nchunks.  The three arrays are the caller's, of
 * inst_cap entries, at least the jobs' total number of directions.  Errors:
 * TVS_ERR_ARG (NULL pointers, bad job arguments, inst_cap too small),
 * TVS_ERR_OOM (a direction does not fit the budget). */
int tvs_debug_plan(const int32_t* rows, const int32_t* cols, const int32_t* n_sectors, const double* step_m,
                   const double* max_range_m, int njobs, uint64_t budget_bytes, int num_sms, int smem_optin,
                   int prune, int fp32_decisions, int32_t* inst_job, int32_t* inst_k, int32_t* inst_chunk,
                   int inst_cap, int32_t* ninst, int32_t* nchunks);

/* Row map of direction k computed by the device kernel that the sweep uses,
 * copied to host arrays: dest[j], frac[j] for j < W (integer row shift and
 * 32-bit fraction of j*t), jlo[p], jhi[p] for p < R (usable columns of skewed
 * row p, whose base row is p - D; jlo > jhi when empty) and *R.  dest and frac
 * need max(rows, cols) entries, jlo and jhi rows + cols entries.  Synchronous. */
int tvs_debug_rowmap(tvs_handle h, int rows, int cols, int n_sectors, int k, int32_t* dest,
                     uint32_t* frac, int32_t* jlo, int32_t* jhi, int32_t* R);

/* Skew + sweep of a single direction k on a HOST DEM, returning the per-sample
 * visible measure cv (forward + backward, squared steps, an exact integer) of
 * every skewed row: cv[p * W + j] for p < R, j < W, -1 where the sample is not
 * usable.  cv needs (rows + cols) * max(rows, cols) entries.  Synchronous. */
int tvs_debug_direction_cv(tvs_handle h, const float* dem, int rows, int cols, double step_m,
                           double obs_height_m, int n_sectors, double max_range_m, int k,
                           int32_t* cv, int32_t* R, int32_t* W);

/* Test hook: the sweep checks the indices of its staging, per-block margins,
 * flagged-POV list and exact walks against their buffers; the first violation
 * on the current device (code, index, bound, CTA; all zero when none) is
 * copied to out[0..3] after a device synchronisation, and cleared when
 * `clear` is non-zero.  A violation means a library bug: the access was
 * skipped instead of faulting.  Errors: TVS_ERR_ARG, TVS_ERR_CUDA. */
int tvs_debug_sweep_check(int32_t* out, int clear);

/* Test and profiling hook: event counts of the certified sweep on the current
 * device since the last clear, after a device synchronisation: out[0] exact
 * walks (POVs with a decision inside its FP32 margin), out[1] of them walked
 * in FP64 (a decision inside the double-float margin too), out[2] SM clock
 * cycles warps spent walking flagged POVs exactly, out[3] cycles warps spent
 * in the certified sweep in all (out[2] / out[3] is the share of the exact
 * walks).  out holds 4 entries.  Errors: TVS_ERR_ARG, TVS_ERR_CUDA. */
int tvs_debug_sweep_stats(uint64_t* out, int clear);

/* Turn per-kernel timing on (1) or off (0); turning it on clears the counters.
 * While on, each launch is bracketed by CUDA events on its stream. */
int tvs_profile_enable(tvs_handle h, int on);

/* Read the per-kernel counters (synchronises the recorded events).  Writes up
 * to max entries to stats and their number to *count. */
int tvs_profile_read(tvs_handle h, tvs_kernel_stats* stats, int max, int* count);

/* ---------------------------------------------- singular / multiple viewsheds --
 * The visible area of each of npov points of view (section 2.1: the singular
 * viewshed of Alg. 1-3; several POVs give the multiple viewshed of the
 * paper's first experiment).  pov_ij: HOST array of npov (row, col) pairs of
 * DEM cells.  d_dem: rows*cols float32 on the device; d_area: npov float32 on
 * the device (m^2); stream-ordered like tvs_total_viewshed_device (the POV
 * list is copied before the call returns).  Modes:
 *   TVS_POINTS_SDEM:   the sDEM discretisation; area[q] is bit for bit the
 *                      value tvs_total_viewshed gives for that cell;
 *   TVS_POINTS_DIRECT: Alg. 1-3 by definition, lines of sight through the
 *                      POV cell itself (no virtual POVs); the difference from
 *                      TVS_POINTS_SDEM is the sDEM discretisation.
 * Work per POV: n_sectors x 2 lines x (forward + backward) walks.
 * Errors: TVS_ERR_ARG (NULL pointer, bad job, a POV outside the DEM, unknown
 * mode), TVS_ERR_OOM, TVS_ERR_CUDA. */
#define TVS_POINTS_SDEM   0
#define TVS_POINTS_DIRECT 1

int tvs_viewshed_points(tvs_handle h, const float* d_dem, int rows, int cols, double step_m, double obs_height_m,
                        int n_sectors, double max_range_m, const int32_t* pov_ij, int npov, int mode, float* d_area,
                        void* cuda_stream);

/* Work count of tvs_viewshed_points: the number of targets its walks visit,
 * sum over the npov POVs (pov_ij: HOST (row, col) pairs), the n_sectors
 * directions, the lines (SDEM: the usable virtual POVs; DIRECT: the line
 * through the cell) and both sides of min(usable targets, K).  Host only;
 * returns a negative code on bad arguments. */
int64_t tvs_count_point_evals(int rows, int cols, int n_sectors, double step_m, double max_range_m,
                              const int32_t* pov_ij, int npov, int mode);

/* Visibility map of a list of POVs (the boolean map of a singular viewshed,
 * section 1; with several POVs, how many see each cell).  Reading (the paper
 * gives no cell rule): the 2n half-lines of Alg. 1 cut the plane into sectors
 * of width pi/n around their axes; a cell belongs to the sector whose axis is
 * nearest to the direction from the POV (a double-precision angle) and is
 * visible iff the sample of that half-line, drawn through the POV cell as in
 * TVS_POINTS_DIRECT, at the cell's walk-axis column is visible (slope
 * strictly above every earlier one); cells the half-line does not reach
 * (past the DEM or the walk limit) are not visible, the POV's own cell is.
 * d_count: rows*cols int32 on the device, written with the number of the
 * npov POVs (pov_ij: HOST (row, col) pairs) that see each cell.
 * Stream-ordered.  Errors: TVS_ERR_ARG, TVS_ERR_OOM, TVS_ERR_CUDA. */
int tvs_visibility_map(tvs_handle h, const float* d_dem, int rows, int cols, double step_m, double obs_height_m,
                       int n_sectors, double max_range_m, const int32_t* pov_ij, int npov, int32_t* d_count,
                       void* cuda_stream);

/* ------------------------------------------------------- request server --
 * Serving total viewsheds to callers that submit DEMs as they arrive (the
 * paper computes one DEM at a time; this is an addition).  A server owns one
 * device allocation of hbm_budget_bytes, split into `lanes` step scratch slots
 * of step_slot_bytes and a resident arena that holds, for every admitted
 * request, its DEM, its output and its exact running totals (24 bytes per
 * cell).  Requests are admitted in submission order while the arena has room
 * and fewer than max_active are admitted.  A scheduler thread runs the GPU in
 * steps: one step is one pass of the pipeline (row map, skew, sweep, unskew)
 * over slices of several admitted requests' directions, whole groups of 8
 * directions at a time, taken in policy order until about step_evals
 * evaluations are in the step.  A request that arrives while steps run joins
 * the next step; with 2 lanes the next step is enqueued while the current one
 * runs.  Results are exact-sum totals, so each request's output is bit for bit
 * what tvs_total_viewshed gives for it alone, whatever it shared its steps
 * with.  Finished outputs are copied to the caller's host buffer.
 * All server calls are thread-safe. */
typedef struct tvs_server* tvs_server_handle;

#define TVS_POLICY_DEADLINE 0  /* earliest (submit time + evals / rate_hint) first */
#define TVS_POLICY_FIFO     1  /* submission order */
#define TVS_POLICY_SRPT     2  /* fewest remaining evaluations first */

typedef struct {
    size_t  hbm_budget_bytes;  /* whole server; 0 = min(80 GiB, 85% of free memory) */
    size_t  step_slot_bytes;   /* scratch of one lane; 0 = min(4 GiB, budget / 8) */
    double  step_evals;        /* evaluations per step (work count, before pruning); 0 = 1.6e11 */
    double  rate_hint;         /* evaluations per second the deadline policy assumes; 0 = 5e12 */
    int32_t max_active;        /* admitted requests at once; 0 = 256 */
    int32_t policy;            /* TVS_POLICY_*; 0 = deadline */
    int32_t lanes;             /* steps in flight, 1 or 2; 0 = 2 */
    int32_t fail_after_steps;  /* test hook: > 0 makes enqueueing step N+1 fail as a
                                  CUDA error would (the host-side failure path); 0 = off */
} tvs_server_config;

#define TVS_REQ_QUEUED   0     /* submitted, waiting for arena room */
#define TVS_REQ_ADMITTED 1     /* resident, no step yet */
#define TVS_REQ_RUNNING  2     /* in at least one enqueued step */
#define TVS_REQ_DONE     3     /* output copied to the caller's buffer */
#define TVS_REQ_FAILED   4     /* see error and message */

typedef struct {
    int32_t state;             /* TVS_REQ_* */
    int32_t error;             /* TVS_OK, or the failure's TVS_ERR_* code */
    int32_t steps;             /* steps that carried directions of the request */
    int32_t n_sectors;
    double  t_submit;          /* seconds on the server clock (tvs_server_clock) */
    double  t_admit;           /* -1 until admitted */
    double  t_first;           /* first step enqueued, -1 before */
    double  t_done;            /* completion observed, -1 before */
    double  evals;             /* work count of the request */
    char    message[128];      /* failure message, "" otherwise */
} tvs_request_info;

typedef struct {
    int64_t submitted, completed, failed;
    int64_t steps;             /* steps enqueued */
    int64_t kernels;           /* kernel launches enqueued */
    double  evals;             /* evaluations enqueued */
    double  arena_bytes;       /* resident arena size */
    double  arena_peak_bytes;  /* most of it ever in use */
    int32_t queued, active;    /* right now */
    int32_t max_step_jobs;     /* most requests one step carried */
    int32_t lanes;
} tvs_server_stats;

/* Create a server on `device` (cfg may be NULL: all defaults).  Errors:
 * TVS_ERR_ARG (bad config), TVS_ERR_OOM (the budget cannot be allocated or
 * leaves no arena), TVS_ERR_CUDA. */
int tvs_server_create(int device, const tvs_server_config* cfg, tvs_server_handle* out);

/* Submit one total viewshed.  dem (rows*cols float32, host memory, finite) and
 * out (rows*cols float32, host memory) must stay valid and untouched until the
 * request is DONE or FAILED; page-locked buffers make the copies asynchronous.
 * The other arguments mean what they mean for tvs_total_viewshed.  Returns at
 * once with the request's ticket.  Errors: TVS_ERR_ARG, TVS_ERR_OOM (the
 * request can never fit the arena or one 8-direction group of it can never
 * fit a step slot), TVS_ERR_STATE (the server is shutting down or failed). */
int tvs_server_submit(tvs_server_handle s, const float* dem, int rows, int cols, double step_m,
                      double obs_height_m, int n_sectors, double max_range_m, float* out, int64_t* ticket);

/* Wait until the request is DONE (returns TVS_OK) or FAILED (returns its
 * error), or until timeout_s seconds passed (TVS_ERR_TIMEOUT; < 0 waits
 * without limit).  TVS_ERR_ARG for an unknown ticket. */
int tvs_server_wait(tvs_server_handle s, int64_t ticket, double timeout_s);

/* State and timestamps of a request. */
int tvs_server_query(tvs_server_handle s, int64_t ticket, tvs_request_info* info);

/* Drop the record of a finished (DONE or FAILED) request: its ticket becomes
 * unknown.  A server keeps every record until then, so long-running callers
 * forget the requests they have collected.  TVS_ERR_STATE while the request
 * is still in flight. */
int tvs_server_forget(tvs_server_handle s, int64_t ticket);

/* Counters of the server. */
int tvs_server_get_stats(tvs_server_handle s, tvs_server_stats* stats);

/* Seconds since the server was created (steady clock; the t_* fields of
 * tvs_request_info use it). */
double tvs_server_clock(tvs_server_handle s);

/* Stop the server: requests not yet admitted fail with TVS_ERR_STATE,
 * admitted ones run to completion, then the threads exit and the device
 * memory is released.  NULL is accepted. */
void tvs_server_destroy(tvs_server_handle s);

#ifdef __cplusplus
}
#endif

#endif /* TVS_H */
