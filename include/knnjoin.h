/*
 * knnjoin.h -- C ABI of the B300 exact K-nearest-neighbour self-join.
 *
 * The operation (Gowanlock, "Hybrid KNN-Join", Sec. 2.1, problem statement):
 * for every point p_i of a data set D of n points in d dimensions, find its K
 * nearest neighbours under the Euclidean distance, the point itself excluded.
 * This library computes it on one GPU with the paper's GPU method -- a grid
 * index built on the device (Sec. 3.1, 4.6), a search distance chosen from a
 * sampled distance histogram (Sec. 4.4), a density-ordered query work queue
 * (Sec. 4.5, Fig. 4) and a per-query scan of the 3^n adjacent cells (Alg. 1,
 * GPUJoinKernel) -- made exact and self-contained: a query whose K-th
 * neighbour is not certified by the cells scanned is re-queued with a wider
 * ring of cells (the paper re-queues failed queries, Alg. 1, Sec. 4.3) until
 * it is.
 *
 * Result convention (the paper fixes neither precision nor tie order; this
 * library fixes both):
 *   D(i,j)  = canonical FP64 squared distance: t_k = fl64(fl64((double)x_ik -
 *             (double)x_jk)^2), summed left to right in FP64, no fused
 *             multiply-add;
 *   row i   = the K indices j != i smallest under (D(i,j), j), ascending;
 *   dist    = correctly rounded sqrt(D(i,j)) in FP64.
 * Another point with the same coordinates as p_i is a neighbour at distance 0.
 *
 * Conventions common to all calls:
 *   - Points are row-major float32 [n][d]; ids are int32 [n][K]; distances
 *     are float64 [n][K].  Pointers may be host or device memory (detected
 *     per call); device pointers must belong to the context's device
 *     (device memory of another GPU is rejected with KNN_ERR_INVALID).
 *   - The caller owns every buffer it passes.  The library never frees or
 *     retains them past the call (blocking calls) or past the poll that
 *     returns a final status (submitted jobs).  The library owns its index
 *     and scratch memory, allocated through the optional hook in
 *     knnjoin_config, until knnjoin_destroy.
 *   - No call aborts, exits or traps.  Errors are returned as a status; the
 *     message is available from knnjoin_last_error.  After KNN_ERR_CUDA the
 *     context must be destroyed.
 *   - A context is used by one host thread at a time.
 */
#ifndef KNNJOIN_H
#define KNNJOIN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct knnjoin_ctx knnjoin_ctx;
typedef struct knnjoin_index knnjoin_index;  /* resident index (knnjoin_index_create) */

typedef enum {
    KNN_OK = 0,
    KNN_ERR_INVALID = 1,    /* bad argument: see knnjoin_last_error */
    KNN_ERR_NOMEM = 2,      /* device or host allocation failed */
    KNN_ERR_CUDA = 3,       /* CUDA runtime error; destroy the context */
    KNN_ERR_NOT_READY = 4,  /* submitted job still running */
    KNN_ERR_TIMEOUT = 5,    /* a bounded wait expired */
    KNN_ERR_CANCELLED = 6,  /* job was cancelled */
    KNN_ERR_QUEUE_FULL = 7  /* serving queue has no free slot */
} knnjoin_status;

typedef struct {
    int device;               /* CUDA device ordinal */
    void *stream;             /* cudaStream_t to run on; NULL = the context makes its own */
    void *(*alloc)(size_t bytes, void *user);  /* optional device allocator: returns device memory
                                                   of the context's GPU, 256-byte aligned as
                                                   cudaMalloc's, or NULL (KNN_ERR_NOMEM); a pointer
                                                   not 16-byte aligned is freed and the call fails
                                                   with KNN_ERR_INVALID */
    void (*free)(void *ptr, void *user);       /* matching free */
    void *user;
    size_t hbm_budget_bytes;  /* admission limit of batched/served jobs; 0 = 90% of free memory */
    int max_jobs;             /* serving queue slots (jobs waiting to start); 0 = 1024 */
    const char *tune_cache_path; /* JSON file of autotuned cell-width multipliers:
                                    read at create, rewritten by knnjoin_autotune;
                                    NULL = tuning kept in memory only */
    float width_mult;         /* cell side = width_mult * eps_min (Sec. 4.4); 0 = the
                                 autotuned value for (d, K, floor(log2 n)) if any,
                                 else 1.25.  Speed only: results never depend on it */
    int workers;              /* concurrent join pipelines for batched/served jobs; 0 = 8 */
    int policy;               /* 0: certified rings (default): a query is re-queued one level
                                 up until its K-th neighbour is closer than the faces of its
                                 scanned box.  1: the paper's GPU-Only policy (Alg. 1, Sec. 4.4):
                                 one global eps (cell side eps, eps_0 = eps_min), a query fails
                                 when fewer than K neighbours lie within eps, and failed queries
                                 are redone on a grid re-indexed with eps += eps_min / 2.
                                 Results are identical; speed differs */
    int out_chunk_mb;         /* results bound for host memory are computed in chunks of
                                 query rows whose device output is at most this many MiB,
                                 each copied out before the next (0 = only when the results
                                 exceed half of the free device memory) */
    int large_first;          /* batched/served joins with at least 2^25 output entries (n*K)
                                 run on high-priority streams, so their blocks are scheduled
                                 ahead of smaller joins sharing the GPU (shorter tail latency
                                 for large jobs, a little longer for small ones); 0 = off */
    int batch_union;          /* knnjoin_self_join_batch: 1 = scan the batch's joins together.
                                 Every join runs its own pass loop (index, density queue,
                                 re-queue) on a stream and host thread of its own, and each
                                 pass's scan is one launch per group of joins with the same
                                 d and buffer size, over the union of their work items
                                 ordered dense first across joins (Sec. 4.5 work queue).
                                 0 = the worker pool runs whole joins concurrently.
                                 Results are identical either way */
    int tail_queries;         /* tail strategy (Sec. 5.4): when at most this many queries are
                                 left uncertified -- after an epoch of the paper's policy, or
                                 after the second pass of the default one -- they are finished
                                 in one pass over the whole grid (a box that contains every
                                 point certifies every query) instead of further widening.
                                 0 = max(1024, queries / 100); negative = never.  Results are
                                 identical; the number of passes changes */
    int reserved[2];
} knnjoin_config;

/* One self-join (batched and served calls). */
typedef struct {
    const float *points;  /* [n][d] float32 */
    int64_t n;
    int d;
    int K;
    int32_t *out_ids;     /* [n][K] */
    double *out_dist;     /* [n][K] */
} knnjoin_job;

/* Counters of the last join run by a context (or of a submitted job). */
typedef struct {
    int64_t n;
    int d, K;
    int passes;                    /* passes of the re-queue loop */
    int start_level;
    int64_t pass_queries[16];      /* active queries per pass (pass 0: every query of the join,
                                      or of the first output chunk) */
    int64_t candidates;            /* candidate distance evaluations, all passes */
    int64_t band_entries;          /* exact re-scores (FP64-canonical) */
    int64_t overflow_queries;      /* queries redone with exact keys */
    double eps_mean, eps_min;      /* Sec. 4.4 search distance */
    double cell_width;             /* level-0 cell side */
    int key_bits;
    int fixed_point;               /* 1 = integer fast path for exact distances */
    double ms_total;               /* device time of the join (events) */
    double ms_index;               /* device time up to the first pass */
    double ms_scan;                /* device time of the scan kernel launches */
    int64_t launches;              /* kernel launches of the join */
    double ms_queue;               /* served/batched: submit -> start (host clock) */
    double ms_wall;                /* served/batched: submit -> done (host clock) */
    double ms_pass[16];            /* device time of each pass's scan launches */
    int64_t pass_candidates[16];   /* candidate distance evaluations of each pass */
    double width_mult;             /* cell-width multiplier the join used */
    int64_t chunks;                /* output chunks (1 unless out_chunk_mb applied) */
    int64_t buffer_entries;        /* candidate buffer per query in the scan (64, 128 or 256;
                                      the smallest holding K + 32 unless autotuned larger) */
} knnjoin_stats;

/* Create a context on cfg->device (cfg may be NULL: device 0, own stream).
 * Returns KNN_ERR_INVALID for a bad device, KNN_ERR_CUDA if CUDA fails. */
knnjoin_status knnjoin_create(const knnjoin_config *cfg, knnjoin_ctx **out);

/* Free every resource of the context.  NULL is a no-op. */
void knnjoin_destroy(knnjoin_ctx *ctx);

/* Blocking exact KNN self-join (Sec. 2.1; method Alg. 1 / Sec. 3-4).
 *   points   : float32 [n][d], host or device
 *   n        : 2 <= n <= 2^31 - 1
 *   d        : 1 <= d <= 8
 *   K        : 1 <= K <= min(n - 1, 256)
 *   out_ids  : int32 [n][K], host or device; row i ascending by (D, id)
 *   out_dist : float64 [n][K], host or device; correctly rounded sqrt(D)
 * KNN_ERR_INVALID on bad sizes, NULL pointers or a non-finite coordinate
 * (detected on the device; the outputs are then unspecified). */
knnjoin_status knnjoin_self_join(knnjoin_ctx *ctx, const float *points, int64_t n, int d, int K,
                                 int32_t *out_ids, double *out_dist);

/* R x S join (the same method with a query set apart from the data set;
 * the paper notes, in Sec. 2.1, that its self-join applies directly to it):
 * for each of the nq query points, the K nearest of the n data points under
 * (D(r, j), j) ascending, j the data point's row.  Nothing is excluded: a
 * query equal to a data point has it as a neighbour at distance 0.
 *   queries  row-major float32 [nq][d], host or device;
 *   points   row-major float32 [n][d], host or device;
 *   out_ids  int32 [nq][K] (data rows), out_dist float64 [nq][K].
 * The grid covers the bounding box of both sets; the search distance and the
 * index are the data set's.  Returns KNN_ERR_INVALID for nq < 1, n < 2,
 * n or nq > 2^31 - 1, d outside [1, 8], K outside [1, min(n, 256)], NULL
 * pointers or a NaN/Inf coordinate in either set. */
knnjoin_status knnjoin_join(knnjoin_ctx *ctx, const float *queries, int64_t nq, const float *points, int64_t n,
                            int d, int K, int32_t *out_ids, double *out_dist);

/* One shard of a self-join: the rows [row_begin, row_end) of the result of
 * knnjoin_self_join on the same points (bit for bit), written to out_ids /
 * out_dist of row_end - row_begin rows (row r of the shard is point
 * row_begin + r).  Queries are independent given all points, so a join is
 * split over GPUs by giving each its own row range: each GPU indexes all n
 * points (deterministic, so every GPU builds the same index) and answers its
 * rows, with no exchange between GPUs (the paper's future-work note on
 * multi-GPU joins, Sec. 6, Discussion and Conclusions).  0 <= row_begin < row_end <= n, else
 * KNN_ERR_INVALID; other rules as knnjoin_self_join. */
knnjoin_status knnjoin_self_join_rows(knnjoin_ctx *ctx, const float *points, int64_t n, int d, int K,
                                      int64_t row_begin, int64_t row_end, int32_t *out_ids, double *out_dist);

/* Cost-balanced shards of a self-join (the paper's multi-GPU note, Sec. 6:
 * its density-ordered work queue split over a node's GPUs).  Equal row
 * counts are unequal work when the input is spatially ordered or skewed, so
 * the queries are taken in the index's key order (cells contiguous) and cut
 * into nshards ranges of equal estimated cost: a query in a cell whose 3^d
 * neighbourhood holds N points costs N (its candidates at ring 1, Alg. 1).
 * knnjoin_shard_bounds: bounds int64 [nshards + 1] (host) receives the cut
 *   points, sorted query positions 0 = bounds[0] <= ... <= bounds[nshards] =
 *   n; costs double [nshards] (host, optional) each range's estimated cost.
 *   Deterministic: every GPU computes the same bounds for the same points.
 * knnjoin_self_join_range: the queries at sorted positions [pos_begin,
 *   pos_end): out_rows int64 [m] (host or device) receives the original row
 *   of each output row, out_ids / out_dist [m][K] (m = pos_end - pos_begin)
 *   the rows of knnjoin_self_join for those points, bit for bit.
 * Both require the default policy (knnjoin_config.policy = 0); otherwise as
 * knnjoin_self_join, and 0 <= pos_begin < pos_end <= n, 1 <= nshards <=
 * 4096, else KNN_ERR_INVALID. */
knnjoin_status knnjoin_shard_bounds(knnjoin_ctx *ctx, const float *points, int64_t n, int d, int K, int nshards,
                                    int64_t *bounds, double *costs);
knnjoin_status knnjoin_self_join_range(knnjoin_ctx *ctx, const float *points, int64_t n, int d, int K,
                                       int64_t pos_begin, int64_t pos_end, int64_t *out_rows, int32_t *out_ids,
                                       double *out_dist);

/* Resident index: index a data set once and keep it on the device, then
 * answer R x S queries against it (the same result as knnjoin_join with these
 * points: for each query row the K nearest data rows under (D, j), nothing
 * excluded).  The paper indexes a data set once on the GPU and sends it query
 * batches (Sec. 3.1 index, Sec. 4.3 batches); serving keeps the index of a
 * data set between requests instead of rebuilding it per join.
 *
 * knnjoin_index_create: points row-major float32 [n][d], host or device,
 *   read during the call only (the index keeps its own copy, sorted); K is
 *   the neighbour count the search distance is chosen for (queries may ask
 *   for another).  Size rules as knnjoin_self_join.  *out receives the index,
 *   owned by the library until knnjoin_index_destroy or knnjoin_destroy of
 *   the context.  The index holds about (24 + 4 d + 4 pad(d)) n bytes of
 *   device memory plus its cell maps (pad(d) = 2, 4 or 8).
 * knnjoin_index_query: queries row-major float32 [nq][d], host or device;
 *   out_ids int32 [nq][K], out_dist float64 [nq][K], host or device;
 *   1 <= K <= min(n, 256).  The grid is the data's: queries outside its box
 *   are answered exactly (boundary cells, wider rings), only more slowly.
 *   Calls on one index are serialised; different indexes run concurrently
 *   (each has its own stream).  Work queued on the context's stream before
 *   the call completes first.  KNN_ERR_INVALID for nq < 1, K out of range,
 *   NULL pointers or a NaN/Inf query coordinate.
 * knnjoin_index_stats: counters of the index's last call (create or query).
 * knnjoin_index_destroy: frees the index; NULL or an already destroyed index
 *   is ignored. */
knnjoin_status knnjoin_index_create(knnjoin_ctx *ctx, const float *points, int64_t n, int d, int K,
                                    knnjoin_index **out);
knnjoin_status knnjoin_index_query(knnjoin_index *index, const float *queries, int64_t nq, int K,
                                   int32_t *out_ids, double *out_dist);
knnjoin_status knnjoin_index_stats(knnjoin_index *index, knnjoin_stats *out);
void knnjoin_index_destroy(knnjoin_index *index);

/* Autotuning (not in the paper; its analogues are the search-distance factor
 * study of Sec. 5.4 and the task-granularity study of Sec. 4.7): time the
 * self-join of these points at a fixed list of cell-width multipliers (1.0 ..
 * 1.625, best of two runs each, outputs in library scratch), then at the best
 * one the next larger candidate buffer per query (e.g. 128 instead of 64
 * entries for K <= 32, which also halves the queries per work item); keep the
 * fastest pair for the key (d, K, floor(log2 n)) -- used by later joins of the
 * context (and its worker pool) unless the config fixed width_mult -- and
 * rewrite tune_cache_path if set.  Same validation as knnjoin_self_join;
 * *best_width_mult receives the chosen multiplier (the buffer size is reported
 * in knnjoin_stats.buffer_entries of later joins). */
knnjoin_status knnjoin_autotune(knnjoin_ctx *ctx, const float *points, int64_t n, int d, int K,
                                float *best_width_mult);

/* Blocking: run njobs independent self-joins (same conventions as
 * knnjoin_self_join per job) concurrently on the context's worker pipelines
 * (each its own stream and scratch), admitted by device-memory footprint.
 * Work queued on the context's stream before the call completes first.
 * Returns the first failing job's status. */
knnjoin_status knnjoin_self_join_batch(knnjoin_ctx *ctx, const knnjoin_job *jobs, int njobs);

/* Serving: enqueue a join and return at once with *job_id.  Jobs start in
 * arrival order as soon as a worker pipeline is free and the job's device
 * memory footprint fits the budget beside the running ones (continuous
 * batching: jobs overlap on the GPU).  The caller keeps the job's buffers
 * alive until knnjoin_poll returns a status other than KNN_ERR_NOT_READY.
 * KNN_ERR_QUEUE_FULL if max_jobs jobs are already waiting; KNN_ERR_INVALID
 * for bad arguments (checked at submission). */
knnjoin_status knnjoin_submit(knnjoin_ctx *ctx, const knnjoin_job *job, uint64_t *job_id);

/* KNN_OK when the job finished, KNN_ERR_NOT_READY while it runs, else its
 * error.  Polling a finished job again returns KNN_ERR_INVALID. */
knnjoin_status knnjoin_poll(knnjoin_ctx *ctx, uint64_t job_id);

/* Cancel a job that has not started; a later poll returns KNN_ERR_CANCELLED. */
knnjoin_status knnjoin_cancel(knnjoin_ctx *ctx, uint64_t job_id);

/* Counters of a job (job_id 0: the last blocking join). */
knnjoin_status knnjoin_get_stats(knnjoin_ctx *ctx, uint64_t job_id, knnjoin_stats *out);

/* Diagnostic, not part of a join: how often ranking by the FP32 filter
 * distance alone would have changed a self-join's result.  The join filters
 * with an FP32 squared distance and ranks in canonical FP64 (Sec. 4, the
 * kernel; Sec. 2.1 defines the result); this call takes exact result rows
 * (out_ids of knnjoin_self_join for these points and K) and, for each listed
 * query row i, forms the FP32-only row: the K smallest j != i under
 * (d2_32(i, j), j), d2_32 being the scan kernels' own FP32 expression, by a
 * brute-force scan of all n points on the device.
 *   points      row-major float32 [n][d], host or device;
 *   ids         int32 [n][K] exact rows, host or device;
 *   rows        int64 [nrows] query rows to check, HOST memory, each in [0, n);
 *   out_counts  int64 [3], host: [0] rows whose FP32-only row differs at any
 *               position, [1] positions that differ, summed over the rows,
 *               [2] exact ids absent from the FP32-only row, summed.
 * Cost: nrows * n FP32 distance evaluations.  KNN_ERR_INVALID for the
 * self-join's size rules, nrows < 1, a row outside [0, n), device-memory
 * rows, NULL pointers, or an ids row holding an index outside [0, n) or the
 * row itself. */
knnjoin_status knnjoin_fp32_mismatch(knnjoin_ctx *ctx, const float *points, int64_t n, int d, int K,
                                     const int32_t *ids, const int64_t *rows, int64_t nrows,
                                     int64_t *out_counts);

/* Message of the last error on this context ("" if none).  Valid until the
 * next call on the context. */
const char *knnjoin_last_error(knnjoin_ctx *ctx);

/* Largest n accepted by knnjoin_self_join_noalloc. */
#define KNN_NOALLOC_MAX_POINTS 65536

/* The paper has no counterpart to this entry point: it is a variant of
 * knnjoin_self_join for callers that must not allocate -- code running
 * inside another framework's memory pool or under a hard memory cap, or an
 * embedding that forbids cudaMalloc/cudaFree behind its back.  It allocates
 * nothing: its scratch is one fixed 32 MiB device array inside the library
 * (held by every GPU that loads the library until the process exits).
 *   points   : float32 [n][d], DEVICE memory (host pointers are rejected)
 *   n, d, K  : as knnjoin_self_join, and n <= KNN_NOALLOC_MAX_POINTS
 *   out_ids  : int32 [n][K], device memory
 *   out_dist : float64 [n][K], device memory
 *   stream   : cudaStream_t to run on (NULL = the legacy default stream)
 *   errbuf   : optional buffer of errlen bytes for the error message
 * The results are identical to knnjoin_self_join's.  The call blocks until
 * the join is done; an error return also waits for any kernels the call
 * had queued, so on every return the GPU has stopped using the array.
 * KNN_ERR_INVALID for sizes beyond the limits, host or managed pointers, or
 * outputs on a GPU other than the points'; KNN_ERR_NOMEM ("fixed scratch
 * array exhausted") if an unusually spread-out input needs the cell tables
 * of more grid levels than the array holds.  All calls share the one array,
 * which keeps the previous call's contents; calls that overlap on the GPU
 * race, so the caller serialises them.  The first call on a device sets up
 * that device (looks up the array's address, creates timing events): make
 * it before any stream capture. */
knnjoin_status knnjoin_self_join_noalloc(const float *points, int64_t n, int d, int K,
                                         int32_t *out_ids, double *out_dist, void *stream,
                                         char *errbuf, size_t errlen);

/* Diagnostic: the density-ordered work queue of a self-join's first pass
 * (Sec. 4.5, Fig. 4: the queries ordered by the number of points in their
 * grid cell, densest first).  Runs the self-join of points (host or device,
 * [n][d]; results discarded) and writes to out_sizes (int64, host, cap
 * entries) the cell count of each query in queue order; *out_len receives
 * the queue's length (n).  Cells of equal counts follow in (level, cell
 * key) order.  Size rules as knnjoin_self_join. */
knnjoin_status knnjoin_work_queue(knnjoin_ctx *ctx, const float *points, int64_t n, int d, int K, int64_t *out_sizes,
                                  int64_t cap, int64_t *out_len);

/* Diagnostic: the grid index of a self-join as the join builds it (steps
 * a3-a5: Sec. 3.1 grid index, Sec. 4.6 GPU indexing).  Runs steps a1-a5 for
 * points (host or device, [n][d]; size rules as knnjoin_self_join), then
 * fills the host buffers given (each may be NULL):
 *   keys  uint64 [n]: the Morton keys of the points' level-0 cells (bit b of
 *         cell coordinate k at key bit b*d + k), in sorted order;
 *   perm  uint32 [n]: the original index of each sorted position (the sort
 *         is stable: equal keys keep their original order);
 *   grid  double [3 + 2d]: the level-0 cell side w0, the key bits per
 *         dimension, the face origin lo[k] and the largest cell index
 *         cmax0[k] per dimension (cell c of dimension k spans
 *         [fl32(c w0 + lo[k]), fl32((c + 1) w0 + lo[k])), clamped to
 *         [0, cmax0[k]]), and the kind of level `level`'s cell table
 *         (1 dense, 0 hash map, -1 when nprobe = 0 and no table was built);
 *   probe_runs uint32 [nprobe][2]: for each of the nprobe level-`level` cell
 *         keys in probe_keys (uint64, host; the level-0 key shifted right by
 *         d * level), the run [begin, end) of sorted positions that the cell
 *         table the scan uses at that level returns -- (0, 0) for a cell
 *         without points or beyond the level's grid.
 * KNN_ERR_INVALID for level outside [0, key bits per dimension], device
 * pointers for the dump's buffers, or probe arguments given by halves. */
knnjoin_status knnjoin_index_dump(knnjoin_ctx *ctx, const float *points, int64_t n, int d, int K, int level,
                                  uint64_t *keys, uint32_t *perm, double *grid, const uint64_t *probe_keys,
                                  int64_t nprobe, uint32_t *probe_runs);

/* Library version string. */
const char *knnjoin_version(void);

#ifdef __cplusplus
}
#endif

#endif /* KNNJOIN_H */
