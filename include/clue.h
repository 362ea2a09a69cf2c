/*
 * clue.h -- C ABI of the GB300 CLUE library (libclue.so).
 *
 * CLUE (Rovere et al., arXiv 2001.09761) clusters the hits of a calorimeter
 * event layer by layer: a fixed square grid per layer (Sec. 2.1, Eqs. 1-2),
 * the local density rho (Eq. 3, Algorithm 1), the nearest-higher nh and
 * separation delta (Eq. 4, Algorithm 2), the seed / outlier decision with
 * follower lists (Sec. 2.2, Eq. 5, Algorithm 3) and the expansion of cluster
 * ids down the follower chains (Algorithm 3).  The input is one structure of
 * arrays over all layers of an event (Sec. 3).
 *
 * Arithmetic contract (identical on every call, every bin size and every
 * launch shape, so results are reproducible bit for bit):
 *   - distances are compared squared in fp32: dx = x_j - x_i, dy = y_j - y_i,
 *     d2 = dx*dx + dy*dy, each operation rounded to nearest, no fused
 *     multiply-add; thresholds are squared once in fp32;
 *   - chi is flat unless clue_opts.chi says otherwise: rho_i is the exact sum
 *     of w_j (or fl(chi(d_ij) w_j)) over all hits j of i's layer with
 *     d2 < d_c^2 (j = i included), rounded once to the nearest fp32, ties to
 *     even: a function of the neighbour set alone (Eq. 3 sums over a set);
 *   - nh_i is the hit j of i's layer with rho_j > rho_i and d2 < d_m^2,
 *     d_m = max(delta_c, delta_o), of smallest d2, the smaller index on a tie;
 *     -1 (and delta = +inf) when there is none;
 *   - seed iff rho > rho_c and delta^2 > delta_c^2; outlier iff rho < rho_c and
 *     delta^2 > delta_o^2; every other hit with nh != -1 follows its nh;
 *   - cluster ids are numbered 0..k-1 per event in ascending seed index and
 *     passed from each seed to all its descendants; outliers, their
 *     descendants, and non-seed hits with no nearest-higher get -1.
 *
 * Memory and threading: every array argument of clue_run / clue_run_batch is
 * a DEVICE pointer (e.g. a torch CUDA tensor's data pointer) on the context's
 * device, owned by the caller, and must stay valid until clue_sync returns.
 * Work is queued on the context's stream and returns before it finishes.
 * The context owns a grow-only scratch arena (allocated once per size, as the
 * paper's Sec. 4.2 allocates once before the event loop).  A context is used
 * by one host thread at a time.  A run is refused (CLUE_ERR_STATE) while the
 * caller is capturing the context's stream into a CUDA graph of its own: the
 * library captures and replays repeated calls itself.
 *
 * Errors: every call returns CLUE_OK (0) or a CLUE_ERR_* code; nothing aborts
 * and nothing traps on the device.  Errors in the inputs (a NaN or infinite
 * coordinate or energy, a layer outside [0, max_layers)) are detected on the
 * device and returned by the next clue_sync; the outputs of that run are then
 * unspecified.
 */
#ifndef CLUE_H
#define CLUE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CLUE_OK 0
#define CLUE_ERR_ARG 1      /* invalid argument (null pointer, bad size or parameter) */
#define CLUE_ERR_INPUT 2    /* invalid input values found on the device */
#define CLUE_ERR_OOM 3      /* device or pinned host allocation failed */
#define CLUE_ERR_CUDA 4     /* a CUDA runtime call failed (see clue_last_message) */
#define CLUE_ERR_TIMEOUT 5  /* a bounded device-side wait gave up */
#define CLUE_ERR_STATE 6    /* call not valid in the context's current state */

typedef struct clue_ctx clue_ctx;

/* Context options.  Fill with clue_default_opts, then override. */
typedef struct clue_opts {
    int32_t device;      /* CUDA device ordinal */
    float x_min, x_max;  /* grid extent (cm); hits outside fall into edge bins */
    float y_min, y_max;
    int32_t max_layers;  /* layer ids must lie in [0, max_layers) */
    float bin_size;      /* grid bin size (cm); 0 = from the tuning table */
    int32_t block_size;  /* threads per block of the density kernels (32..256, a
                            multiple of 32); 0 = from the tuning table, whose
                            block line the autotuner sets from 128, 256 and
                            512; its default (block 0) picks, per run, 256
                            for runs of at least one tile per SM (512 when the
                            run's staging leaves room for only two CTAs of
                            256 per SM) and 1024 for runs of fewer tiles */
    int32_t use_graphs;  /* 1 = capture a repeated call into a CUDA graph and replay it */
    void *stream;        /* cudaStream_t to queue work on; NULL = context-owned stream */
    int32_t expand;      /* how ids reach the followers (identical results):
                            CLUE_EXPAND_FRONTIER = follower lists walked level by
                            level from the seeds (Algorithm 3's expansion, k-way);
                            CLUE_EXPAND_CHASE = each follower follows its nh chain
                            up to the first hit with a final id (n-way) */
    int32_t chi;         /* density kernel chi(d) of Eq. 3: CLUE_CHI_FLAT (1, the
                            default), CLUE_CHI_GAUSSIAN exp(-d^2 / (2 s^2)),
                            CLUE_CHI_EXPONENTIAL exp(-d / s); the term added is
                            fl(chi(d) * w), with exp computed by a fixed fp32
                            sequence (Cody-Waite reduction, degree-7 Taylor) */
    float chi_param;     /* s > 0 for the Gaussian and exponential kernels */
    int64_t max_scratch_bytes; /* 0 = no limit; otherwise a run whose scratch
                                  would exceed it fails with CLUE_ERR_OOM before
                                  any allocation (memory budgets, tests) */
    int32_t walk_limit;  /* most steps the device may take to pass an id down one
                            hit's chain of nearest-highers (Algorithm 3's
                            expansion): a bounded walk of min(64, walk_limit)
                            steps, then pointer-jumping rounds (each at least
                            doubles the distance covered, so a chain of depth D
                            needs about log2(D / 64) + 1).  0 = no limit beyond
                            the 40 rounds that cover any chain.  A hit whose chain
                            needs more gets -1 and the next clue_sync returns
                            CLUE_ERR_TIMEOUT (the device never waits unbounded) */
    int32_t density;     /* kernels of rho (Eq. 3) and nh / delta (Eq. 4), identical
                            results: CLUE_DENSITY_FUSED = one kernel per tile of hits
                            computes rho, nh and the decision (rho of the tile's
                            halo computed again per tile); CLUE_DENSITY_SEPARATE = a
                            rho kernel, then an nh kernel; CLUE_DENSITY_AUTO (the
                            default) = fused where the run's grid rows are sparse
                            enough for the smallest staging, else separate */
} clue_opts;

#define CLUE_CHI_FLAT 0
#define CLUE_CHI_GAUSSIAN 1
#define CLUE_CHI_EXPONENTIAL 2

#define CLUE_EXPAND_FRONTIER 0
#define CLUE_EXPAND_CHASE 1

#define CLUE_DENSITY_AUTO 0
#define CLUE_DENSITY_FUSED 1
#define CLUE_DENSITY_SEPARATE 2

/* Defaults: device 0, extent [-250, 250]^2, 128 layers, tuned bin/block,
 * graphs on, own stream, expansion by chasing (CLUE_EXPAND_CHASE), flat chi
 * (Eq. 3, Algorithm 1), no scratch or walk limit, density kernels by run. */
void clue_default_opts(clue_opts *opts);

/* Create a context on opts->device.  *out receives the context.  The
 * context holds what Sec. 4.2 allocates once before the event loop (the
 * device scratch every run reuses, grown only when a larger run needs it) and
 * the fixed grid's extent and layer count (Sec. 2.1).
 * Errors: CLUE_ERR_ARG (null, extent not finite/increasing, max_layers < 1,
 * bin_size < 0, block_size, expand or chi out of range, chi_param not > 0
 * for a non-flat chi, walk_limit < 0), CLUE_ERR_CUDA. */
int clue_create(clue_ctx **out, const clue_opts *opts);

/* Release the context and everything it owns, after waiting for its queued
 * work: the one-time release after the last event of Sec. 4.2. */
void clue_destroy(clue_ctx *ctx);

/* Queue later work on another stream (cudaStream_t; NULL = the context's own).
 * The paper has no counterpart: stream placement is a deployment concern. */
int clue_set_stream(clue_ctx *ctx, void *stream);

/*
 * Cluster one event of n hits (Sec. 2, Algorithms 1-3).
 *   x, y      float32[n]  hit coordinates (cm)
 *   layer     int32[n]    layer id in [0, max_layers)
 *   energy    float32[n]  hit weight w (Eq. 3)
 *   n         0 <= n <= 2^31 - 2 (n = 0 is a no-op)
 *   dc        cut-off distance d_c > 0 (Eq. 2-3)
 *   rhoc      density threshold rho_c (finite)
 *   delta_c   seed separation delta_c >= 0 (Sec. 2.2)
 *   delta_o   outlier separation delta_o >= 0 (Sec. 2.2)
 *   cluster_id int32[n] out: cluster id 0..k-1, or -1 for noise
 *   is_seed    uint8[n] out: 1 for seeds, else 0
 * All arrays are device pointers; see the header comment for ownership.
 * Errors: CLUE_ERR_ARG, CLUE_ERR_OOM, CLUE_ERR_CUDA (immediately);
 * CLUE_ERR_INPUT, CLUE_ERR_TIMEOUT (from the next clue_sync).
 */
int clue_run(clue_ctx *ctx, const float *x, const float *y, const int32_t *layer,
             const float *energy, int64_t n, float dc, float rhoc, float delta_c,
             float delta_o, int32_t *cluster_id, uint8_t *is_seed);

/*
 * Cluster a batch of independent events in one pass (one launch per stage for
 * the whole batch): Sec. 3's pipeline of one kernel per CLUE step over one
 * structure of arrays, with many events' hits in that structure instead of
 * one event's; each event is clustered exactly as clue_run clusters it
 * alone (Algorithms 1-3).  Event e owns hits [offsets[e], offsets[e+1]) of the
 * concatenated device arrays x, y, layer, energy, cluster_id, is_seed.
 *   offsets   HOST int64[n_events + 1], offsets[0] = 0, non-decreasing,
 *             offsets[n_events] <= 2^31 - 2
 *   n_events  >= 0
 * Cluster ids are numbered per event (each event starts at 0).
 * The same parameters apply to every event.  Errors as clue_run.
 */
int clue_run_batch(clue_ctx *ctx, const float *x, const float *y, const int32_t *layer,
                   const float *energy, const int64_t *offsets, int32_t n_events, float dc,
                   float rhoc, float delta_c, float delta_o, int32_t *cluster_id,
                   uint8_t *is_seed);

/*
 * As clue_run_batch, but every array (x, y, layer, energy, cluster_id,
 * is_seed, offsets) is a HOST pointer (pinned memory is fastest): the
 * end-to-end path whose host-device copies Table 2 of Sec. 4.2 lists as
 * "cuda memcpy".  The call
 * copies the inputs to context-owned device buffers, clusters, copies the
 * results back and returns when they are in host memory (it synchronises).
 * A batch of 8M hits or more is split at event boundaries into chunks of
 * about N/8 and a last one of about N/32, pipelined over three streams:
 * chunk c+1 is copied in and chunk c-1 copied out while chunk c is clustered.
 * Errors: as clue_run_batch, including CLUE_ERR_INPUT / CLUE_ERR_TIMEOUT.
 */
int clue_run_batch_host(clue_ctx *ctx, const float *x, const float *y, const int32_t *layer,
                        const float *energy, const int64_t *offsets, int32_t n_events,
                        float dc, float rhoc, float delta_c, float delta_o,
                        int32_t *cluster_id, uint8_t *is_seed);

/*
 * (The paper has no counterpart: a staging helper for servers.)
 * Queue the copies of one event's inputs, n hits of the arrays x, y, layer,
 * energy (host or device; pinned host memory gives asynchronous copies, and
 * pageable host memory may be reused once the call returns), into the DEVICE
 * arrays dx, dy, dlayer, denergy at element offset `offset`, on `stream`
 * (cudaStream_t; NULL = legacy default stream).  For servers that stage
 * events into a resident batch buffer as they arrive (one call instead of
 * four).  No context needed.  Errors: CLUE_ERR_ARG, CLUE_ERR_CUDA.
 */
int clue_stage_event(const float *x, const float *y, const int32_t *layer,
                     const float *energy, int64_t n, float *dx, float *dy, int32_t *dlayer,
                     float *denergy, int64_t offset, void *stream);

/* Wait for the context's queued work (the kernels of Sec. 3 run
 * asynchronously; results are complete once they have all finished); returns
 * the first deferred error (CLUE_ERR_INPUT, CLUE_ERR_TIMEOUT, CLUE_ERR_CUDA)
 * or CLUE_OK, and clears it. */
int clue_sync(clue_ctx *ctx);

/*
 * Copy per-hit intermediates of the last run into caller DEVICE arrays of the
 * last run's total hit count (any may be NULL): rho (Eq. 3), delta (sqrt of
 * the fp32 squared separation, +inf when none, Eq. 4) and nh (Eq. 4, index
 * within the hit's event, -1 when none).  Queued on the context's stream.
 * Errors: CLUE_ERR_STATE before any run.
 */
int clue_get_intermediates(clue_ctx *ctx, float *rho, float *delta, int32_t *nh);

/*
 * Tune the grid bin size (Sec. 2.1 leaves it free; results do not depend on
 * it) and the tile length (hits per CTA, so hits per thread) per event-size
 * class (each class timed on its own events, copied into a context-owned
 * sub-batch), and the density kernels' block size (Sec. 3 times block sizes
 * 1024 and 256; here timed on the whole batch) for the given device batch (same
 * arguments as clue_run_batch; results of the trial runs are written to
 * cluster_id / is_seed).  Every candidate gives bit-identical results; only
 * speed differs.  `reps` timed repetitions per candidate (>= 1).
 * Synchronises.  Errors as clue_run_batch.
 */
int clue_autotune(clue_ctx *ctx, const float *x, const float *y, const int32_t *layer,
                  const float *energy, const int64_t *offsets, int32_t n_events, float dc,
                  float rhoc, float delta_c, float delta_o, int32_t *cluster_id,
                  uint8_t *is_seed, int32_t reps);

/* Write the tuning table as text into buf (capacity cap bytes,
 * NUL-terminated): a comment line, then per class "class <lo> <hi>
 * <bin_scale> <tile_hits>" (bin size = bin_scale * 2 d_c; tile_hits: hits
 * per CTA of the per-tile kernels, a multiple of 32 up to 1024) for the six
 * classes (edges 0, 32768, 100000, 316228, 1000000, 3162278 hits), then
 * "block <threads>" (0 = by run size) and "band <staged records>" (the
 * density kernels' staging capacity, 0 = by run).  Returns the length
 * needed, or a negative CLUE_ERR_* code.  (No counterpart in the paper:
 * tuning state.) */
int64_t clue_get_tuning(clue_ctx *ctx, char *buf, int64_t cap);

/* Replace the tuning table from text in the format of clue_get_tuning (a
 * class line without <tile_hits> keeps 1024).  Errors: CLUE_ERR_ARG on
 * malformed text or values out of range. */
int clue_set_tuning(clue_ctx *ctx, const char *text);

/* (No counterpart in the paper beyond the per-kernel times of Table 2.)
 * Per-kernel timing: when on (1), the next runs record a CUDA event before
 * the first kernel and after each kernel (or launch group: a prefix sum's
 * three kernels count as one).  clue_stage_times waits for the last profiled
 * run and writes up to `cap` durations in ms, in launch order, and their
 * names (comma-separated, into names if not NULL, capacity names_cap); it
 * returns the number of entries, or a negative CLUE_ERR_* code
 * (-CLUE_ERR_STATE when no profiled run exists).  clue_stage_times_back does
 * the same for the profiled run `back` runs before the last (0 = the last;
 * the last 4 profiled runs stay readable), so a caller can read a run's times
 * while later runs are queued, without draining the stream each run. */
int clue_set_profiling(clue_ctx *ctx, int32_t on);
int clue_stage_times(clue_ctx *ctx, float *ms, int32_t cap, char *names, int64_t names_cap);
int clue_stage_times_back(clue_ctx *ctx, int32_t back, float *ms, int32_t cap, char *names,
                          int64_t names_cap);

/* Number of kernels the last run launched (for launch accounting; no
 * counterpart in the paper). */
int32_t clue_last_launch_count(clue_ctx *ctx);

/* Device bytes the context's scratch arena holds now (the one-time
 * allocation of Sec. 4.2). */
int64_t clue_scratch_bytes(clue_ctx *ctx);

/*
 * Single-event clustering that allocates nothing (the paper has no
 * counterpart: this is a deployment variant of clue_run).
 *
 * For callers that cannot allocate device memory -- code running inside
 * another framework's memory pool, a real-time loop where an allocation could
 * block or fail, or a plugin whose host owns every device allocation.  It runs
 * the same kernels as clue_run, so results are bit-identical to clue_run's,
 * but every scratch array lives in one fixed array in the library's device
 * memory (about 14.7 MB, held on every GPU that loads the library until the
 * process exits).  It needs no context and calls no allocator, neither CUDA's
 * nor any other.
 *
 *   x, y, layer, energy, cluster_id, is_seed: DEVICE arrays of n entries on
 *     the current device, as in clue_run (caller-owned)
 *   n          0 <= n <= CLUE_STATIC_MAX_HITS (larger n: CLUE_ERR_ARG, nothing runs)
 *   dc, rhoc, delta_c, delta_o: as in clue_run
 *   x_min..y_max, max_layers: the grid extent and layer count (as clue_opts);
 *     1 <= max_layers <= CLUE_STATIC_MAX_CELLS; the bins are widened until
 *     max_layers * (bins per layer) fits CLUE_STATIC_MAX_CELLS (results do not
 *     depend on the bin size)
 *   stream     cudaStream_t to run on (NULL = the legacy default stream)
 *
 * The call is synchronous: it returns after the results are in cluster_id /
 * is_seed, with CLUE_OK, CLUE_ERR_ARG, CLUE_ERR_INPUT (NaN/Inf or bad layer,
 * outputs unspecified), CLUE_ERR_TIMEOUT, CLUE_ERR_OOM (first call on a
 * device only, see below) or CLUE_ERR_CUDA.
 * The first call on each device sets the call up there (once per device,
 * with that device current): it loads the library's device code on that
 * device, which reserves the array, and looks up the array's device address.
 * That first call can therefore block, and it fails with CLUE_ERR_OOM when
 * the device has no room left for the array; make it at set-up time, before
 * any stream capture.  Later calls on that device allocate nothing.  Every call shares the one array and keeps what the previous call
 * left in it (the call clears what must start at zero): calls that overlap on
 * the GPU -- from several host threads or on several streams at once -- race
 * and give wrong results.
 */
#define CLUE_STATIC_MAX_HITS 65536
#define CLUE_STATIC_MAX_CELLS 1048576
int clue_run_static(const float *x, const float *y, const int32_t *layer, const float *energy,
                    int64_t n, float dc, float rhoc, float delta_c, float delta_o, float x_min,
                    float x_max, float y_min, float y_max, int32_t max_layers,
                    int32_t *cluster_id, uint8_t *is_seed, void *stream);

/*
 * Continuous-batching server (the paper has no counterpart: its events are
 * clustered one at a time; this serves a stream of them on one GPU).
 *
 * Events arrive one per clue_server_submit, from any host thread, at any
 * time.  A worker thread admits each into the device region being filled
 * while the region has room (hits, events) and the memory budget covers it
 * (otherwise the event waits), copies its inputs there on a copy stream at
 * once, and launches a filled region as one clue_run_batch as soon as fewer
 * than max_inflight batches are queued on the device; the results are copied
 * back into the event's own output arrays and a stream callback then marks
 * the event done.  Each event's results are the same bytes as clue_run gives
 * for the event alone.
 */
typedef struct clue_server clue_server;

typedef struct clue_server_opts {
    int64_t region_hits;          /* hits per device region: the largest event taken */
    int32_t n_regions;            /* regions, >= 2: one fills while others run */
    int32_t max_inflight;         /* batches queued on the device at once (<= n_regions - 1) */
    int32_t max_events_per_batch; /* events per batch at most */
    int64_t mem_budget_bytes;     /* 0 = none; else each admitted hit holds 141 bytes
                                     against it until its event is done */
} clue_server_opts;

/* Defaults: regions of 16M hits, 3 regions, 2 batches in flight, 512 events
 * per batch, no budget. */
void clue_server_default_opts(clue_server_opts *opts);

/* Create a server on opts->device with its own context (clue_opts as for
 * clue_create; opts->stream is ignored: the server owns its streams), the
 * clustering parameters of every event (as clue_run) and an optional tuning
 * table (text of clue_get_tuning, or NULL).  Allocates its regions
 * (n_regions x region_hits x 21 bytes) and starts its worker thread.
 * Errors: CLUE_ERR_ARG, CLUE_ERR_OOM, CLUE_ERR_CUDA. */
int clue_server_create(clue_server **out, const clue_opts *opts,
                       const clue_server_opts *server_opts, float dc, float rhoc,
                       float delta_c, float delta_o, const char *tuning);

/* Queue one event of n hits.  x, y, layer, energy (inputs) and cluster_id,
 * is_seed (outputs) are arrays of n entries in host or device memory (host
 * memory should be pinned: pageable memory makes the copies synchronous);
 * the caller keeps all six valid until the event's clue_server_wait returns.
 * *ticket identifies the event.  Errors:
 * CLUE_ERR_ARG (null pointers, n < 0, n above region_hits or the budget:
 * nothing queued), CLUE_ERR_STATE (the server is stopping). */
int clue_server_submit(clue_server *server, const float *x, const float *y,
                       const int32_t *layer, const float *energy, int64_t n,
                       int32_t *cluster_id, uint8_t *is_seed, int64_t *ticket);

/* Wait until the ticket's event is done: its results are in its output
 * arrays.  timeout_s < 0 waits without limit.  Returns CLUE_OK once it is
 * done, with the event's outcome in *status (CLUE_OK, or CLUE_ERR_INPUT /
 * CLUE_ERR_TIMEOUT raised on the device by its batch, or CLUE_ERR_CUDA) and
 * *latency_ms from submission to the results in its output arrays (either may be
 * NULL); the ticket is then released.  Returns CLUE_ERR_TIMEOUT, the ticket
 * kept, if the event is not done in time; CLUE_ERR_ARG for an unknown or
 * released ticket. */
int clue_server_wait(clue_server *server, int64_t ticket, double timeout_s, int32_t *status,
                     double *latency_ms);

/* Counters into out[6] (if not NULL): events done, hits done, batches
 * launched, events rejected, seconds from the first submission to the last
 * completion, mean events per batch; and up to `cap` per-event latencies in
 * ms (completion order) into latency_ms.  Returns the number of latencies
 * recorded, or a negative CLUE_ERR_* code. */
int64_t clue_server_stats(clue_server *server, double *out, double *latency_ms, int64_t cap);

/* Start the counters and latencies of clue_server_stats again from zero
 * (e.g. after a warm-up).  Errors: CLUE_ERR_ARG. */
int clue_server_reset_stats(clue_server *server);

/* Finish every queued event, stop the worker and release everything. */
void clue_server_destroy(clue_server *server);

/* Human-readable text of a CLUE_ERR_* code (the paper has no counterpart:
 * error reporting of this library). */
const char *clue_strerror(int code);

/* Text of the last CUDA error the context saw ("" if none; no counterpart in
 * the paper). */
const char *clue_last_message(clue_ctx *ctx);

/* Library version string (no counterpart in the paper). */
const char *clue_version(void);

#ifdef __cplusplus
}
#endif

#endif /* CLUE_H */
