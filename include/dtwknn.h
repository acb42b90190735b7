/*
 * dtwknn.h - C ABI of the GB300 (sm_103a) exact nearest-neighbour DTW
 * retrieval cascade of D. Lemire, "Faster Retrieval with a Two-Pass
 * Dynamic-Time-Warping Lower Bound" (arXiv:0811.3301).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Series are fp32, row-major and contiguous: a set of `count` series of
 *    length n is a [count][n] array.  Indices are 0-based (the paper's are
 *    1-based, Sec. 2).
 *  - n >= 1 and n <= DTW_MAX_N.  w >= 0 is the locality constraint of
 *    Sec. 4: x_i and y_j may be aligned only if |i - j| <= w; any w >= n - 1
 *    means no constraint.  p is 1 or 2 (the l_p norm of Sec. 2); the DTW
 *    entry points dtw_band and dtw_band_noalloc also take p = 4 and
 *    p = infinity (DTW_P_INF), the other measures of App. C.
 *  - Distances and bounds are returned with the p-th root taken, as the
 *    paper defines them (DTW_p = q_{1,1}^(1/p), Sec. 4).  Internally the
 *    kernels compare in power space.
 *  - Unless an entry point says otherwise, array pointers are DEVICE
 *    pointers owned by the caller, and outputs are preallocated by the caller.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  Calls are asynchronous on it unless documented otherwise.
 *  - Inputs must be finite; NaN or Inf inputs give unspecified results.
 *  - Every call returns a dtw_status; on failure dtw_last_error() gives a
 *    message for the calling host thread and no output is written.
 *  - Calls that need scratch memory take it from a per-device workspace
 *    that the library grows on demand with cudaMalloc; growth synchronises
 *    the device, so the first call at a new size must not be made inside a
 *    CUDA stream capture.  Calls that use the workspace must not overlap on
 *    the GPU (one such call at a time per device).
 */
#ifndef DTWKNN_H
#define DTWKNN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DTW_MAX_N 4096 /* longest supported series */
#define DTW_MAX_K 128  /* largest supported neighbour count */
#define DTW_P_INF 0    /* p = infinity: DTW_inf, the largest cost along the best path (Sec. 4) */

typedef enum {
    DTW_OK = 0,
    DTW_ERR_INVALID_ARG = 1, /* a size, pointer or parameter is out of range */
    DTW_ERR_CUDA = 2,        /* a CUDA runtime call or kernel launch failed */
    DTW_ERR_OOM = 3,         /* the workspace could not be grown */
    DTW_ERR_TIMEOUT = 4,     /* a bounded device-side wait gave up */
    DTW_ERR_NO_BUCKET = 5,   /* no database series has the query's length */
    DTW_ERR_INTERNAL = 6     /* an internal consistency check failed */
} dtw_status;

/* Cascade variants for knn_search_ex (Sec. 7 and Sec. 8). */
typedef enum {
    DTW_MODE_IMPROVED = 0, /* LB_Keogh, then LB_Improved, then DTW (Algorithm 3) */
    DTW_MODE_KEOGH = 1,    /* LB_Keogh, then DTW (Algorithm 2) */
    DTW_MODE_NOPRUNE = 2   /* every candidate gets a full DTW (validation) */
} dtw_mode;

/* Counters of one knn_search call, summed over queries. */
typedef struct {
    int64_t candidates;      /* (query, candidate) pairs: Q * N */
    int64_t seeds;           /* pairs whose DTW was computed first to seed the threshold */
    int64_t pruned_summary;  /* pairs discarded by the piecewise-sum bound (Sec. 9) */
    int64_t pruned_keogh;    /* pairs discarded by LB_Keogh */
    int64_t pruned_improved; /* pairs discarded by LB_Improved */
    int64_t dtw_computed;    /* non-seed pairs whose DTW was started */
    int64_t dtw_abandoned;   /* of which abandoned early (row minimum above the threshold) */
    int64_t dtw_cells;       /* in-band cells (|i - j| <= w) of the DP rows those DTWs evaluated;
                                a completed pair has n (2w + 1) - w (w + 1) */
    int64_t seed_cells;      /* in-band cells evaluated by the seed DTWs */
    int64_t dtw_lane_rows;   /* thread-per-pair DTW: rows its warps stepped, 32 per row of a
                                chunk's longest pair (dtw_rows / this = lane use);
                                0 when the warp path ran the stage */
    int64_t dtw_rows;        /* DP rows evaluated by the non-seed DTWs */
    int64_t seed_rows;       /* DP rows evaluated by the seed DTWs */
} dtw_stats;

typedef struct {
    int32_t mode;  /* a dtw_mode */
    float slack;   /* relative pruning slack; the kernels use the larger of this
                      and the worst-case fp32 rounding bound of the compared sums */
    int32_t seeds; /* candidates per query (lowest bound first) whose DTW seeds the
                      threshold; 0 selects the default (16, at least k, at most N) */
    int32_t parts; /* parts d of the piecewise-sum bound (Sec. 9) computed for every pair
                      before LB_Keogh, which then runs only on its survivors; 0 selects
                      the default (n / 8 when n >= 64, else off), -1 disables it (LB_Keogh
                      of every pair), otherwise 1 <= d <= n */
    int32_t dtw_path; /* DTW kernel of the cascade's DTW stages: 0 chooses (one warp per
                         pair for bands wider than 208 slots and for the few seeds of
                         long series, else one thread per pair),
                         1 one thread per pair where the band fits, 2 one warp per pair
                         (one row per lane and step for bands of 409 and 289 slots, two
                         pairs per warp otherwise),
                         3 one warp per two pairs (16-lane groups) where the band allows,
                         4 one thread per pair in launches of 64 rows (pairs still alive
                         at a launch's last row are resumed by the next one), where the
                         band fits one thread's registers (2w + 1 <= 64, or <= 208 for
                         p = 1 and 2) and n > 128; 0 uses 4 for bands of up to 64
                         slots in runs of at least 2^24 (query, candidate) pairs */
    int32_t filter_path; /* LB_Keogh / LB_Improved filter kernel: 0 chooses (batches of eight
                            pairs per warp for series of 128 or 256 elements with the
                            piecewise-sum pre-filter, else one warp per pair), 1 one warp
                            per pair, 2 batches where they apply */
    int32_t lb_abandon;  /* 1: stop summing a pair's LB_Keogh / LB_Improved once the partial
                            sums (tested every 256 indices) exceed the threshold, on series
                            longer than 256 whose rows are streamed; 0 or -1: never.  The
                            result is the same either way */
} dtw_options;

/*
 * Warping envelope (Sec. 5): U(y)_i = max { y_k : |k - i| <= w } and
 * L(y)_i = min { y_k : |k - i| <= w }, k restricted to the series, for each of
 * `count` series y [count][n].  Outputs U, L are [count][n].  The result is
 * exact (min and max do not round).  The paper computes it with the
 * streaming Algorithm 1 (Sec. 6); this library uses a block-parallel
 * doubling scheme with the same result.
 */
dtw_status dtw_envelope(const float *y, int64_t count, int32_t n, int32_t w,
                        float *U, float *L, void *stream);

/*
 * LB_Keogh_p(x, y) = || x - H(x, y) ||_p (Sec. 7, Eq. 1) of every candidate
 * x = cand[c] (cand is [N][n]) against one query y given by its envelope
 * U = U(y), L = L(y) ([n] each).  out[c] receives the bound (root taken), [N].
 */
dtw_status lb_keogh(const float *cand, int64_t N, const float *U, const float *L,
                    int32_t n, int32_t p, float *out, void *stream);

/*
 * Piecewise-sum bound of Sec. 9 for every candidate x = cand[c] against one
 * query envelope U, L: with the cover of d parts C_j (floor(n/d) indices each,
 * the last part takes the rest) and D_j the distance from sum_{C_j} x to
 * [sum_{C_j} L, sum_{C_j} U], out[c] = sum_j D_j (p = 1, the paper's bound) or
 * sqrt(sum_j D_j^2 / max_j |C_j|) (p = 2).  Both are at most LB_Keogh_p.
 * 1 <= d <= n.  out is [N].
 */
dtw_status lb_piecewise(const float *cand, int64_t N, const float *U, const float *L,
                        int32_t n, int32_t d, int32_t p, float *out, void *stream);

/*
 * LB_Improved_p(x, y) with LB_Improved_p^p = LB_Keogh_p(x, y)^p +
 * LB_Keogh_p(y, H(x, y))^p (Sec. 8) for every candidate x = cand[c] against
 * the query q [n] with envelope U, L ([n] each, computed with the same w).
 * out[c] receives the bound (root taken), [N].  The second sum is evaluated
 * from the candidates' own envelopes and the envelopes of U and L, which
 * give the same terms as the envelope of the projection H; uses the
 * workspace (2 N n + 4 n floats).
 */
dtw_status lb_improved(const float *cand, int64_t N, const float *q, const float *U,
                       const float *L, int32_t n, int32_t w, int32_t p, float *out,
                       void *stream);

/*
 * Band-constrained DTW_p (Sec. 4 recursion) of the pairs (x[c], y) for
 * c < N: x is [N][n]; y is one series [n] when y_stride == 0, or [N][n] when
 * y_stride == n (pair c uses y + c * n).  p is 1, 2, 4 or DTW_P_INF; for
 * DTW_P_INF a cell holds max(|x_i - y_j|, min(predecessors)) (Sec. 4) and the
 * result is DTW_inf.  If threshold is finite, a pair whose DTW_p provably
 * exceeds it (the minimum of a row of the dynamic program is above
 * threshold^p, or threshold for DTW_inf: an exact test since costs are
 * non-negative) is abandoned and gets +INF; +INF disables abandoning.  out is
 * [N] (root taken).
 */
dtw_status dtw_band(const float *x, const float *y, int64_t N, int32_t y_stride,
                    int32_t n, int32_t w, int32_t p, float threshold, float *out,
                    void *stream);

/*
 * Exact k nearest neighbours under DTW_p with band w (Sec. 7-8 problem
 * statement, generalised from 1 to k neighbours): for each of the Q queries
 * [Q][n], the k database series db [N][n] of smallest DTW_p, ordered by
 * (distance, index) ascending, so that ties go to the lower index.  The
 * cascade computes the query envelopes, LB_Keogh of every pair, the DTW of
 * the lowest-bound seeds, LB_Improved of the LB_Keogh survivors and a DTW
 * with early abandoning of the LB_Improved survivors, every stage pruning
 * against the current k-th best distance.
 * out_idx [Q][k] (int64) and out_dist [Q][k] (fp32, root taken) receive the
 * result; when k > N the tail is idx -1, distance +INF.
 * db, queries, out_idx and out_dist may each be host or device memory; host
 * inputs are copied in, and host outputs make the call synchronous.
 * stats (host, nullable) receives counters and also makes the call
 * synchronous.
 */
dtw_status knn_search(const float *db, int64_t N, const float *queries, int64_t Q,
                      int32_t n, int32_t w, int32_t p, int32_t k, int64_t *out_idx,
                      float *out_dist, dtw_stats *stats, void *stream);

/*
 * Triangle-inequality experiment of App. B: for N triples (x_i, y_i, z_i)
 * (x, y, z each [N][n]), ratio[i] = DTW_p(x_i, z_i) / (DTW_p(x_i, y_i) +
 * DTW_p(y_i, z_i)) with band w (the paper uses no constraint: w >= n - 1).
 * A ratio above 1 is a violation of the triangle inequality; 0 / 0 gives 0
 * and c / 0 (c > 0) gives +INF.  dist3 (nullable, [3][N]) receives the three
 * distances DTW_p(x,y), DTW_p(y,z), DTW_p(x,z).  Uses the workspace.
 */
dtw_status dtw_triangle(const float *x, const float *y, const float *z, int64_t N, int32_t n,
                        int32_t w, int32_t p, float *ratio, float *dist3, void *stream);

/* knn_search with a cascade mode, slack and seed count (opt may be NULL). */
dtw_status knn_search_ex(const float *db, int64_t N, const float *queries, int64_t Q,
                         int32_t n, int32_t w, int32_t p, int32_t k,
                         const dtw_options *opt, int64_t *out_idx, float *out_dist,
                         dtw_stats *stats, void *stream);

/*
 * Candidate sharding (Sec. 7-8 problem statement: the candidates of a query
 * are independent, so the database can be split by candidate range over
 * several GPUs or processes, each searching every query in its own shard).
 * A shard's own seeds give each query a threshold that is at least that
 * shard's k-th smallest DTW, and the smallest of these over the shards is at
 * least the k-th smallest over the whole database, so every shard may prune
 * with it: a true neighbour never exceeds it.
 *
 * knn_seed_thresholds runs the first stages of knn_search_ex on this shard
 * (query envelopes, the bound of every pair, the DTW of the lowest-bound
 * seeds) and writes thr_out[q] [Q], the k-th smallest seed DTW of query q
 * (+INF when the shard has fewer than k seeds), in the cascade's power units:
 * DTW_p^p for p = 1, 2, 4 and DTW_inf for p = DTW_P_INF (no root taken).
 *
 * knn_search_bounded is knn_search_ex with query q's threshold lowered to
 * thr_in[q] (same units; NaN and negative values are ignored) once its seeds
 * are done.  The result lists only the shard's candidates whose DTW does not
 * exceed the final threshold (the rest of a list is idx -1, +INF); when
 * thr_in is the minimum of every shard's thr_out, merging the shards' lists
 * by (distance, index) gives the exact k nearest neighbours of the whole
 * database.  The shards' indices are their own (0-based in the shard).
 *
 * knn_merge_topk merges R lists per query: idx, dist [R][Q][k_in] (device;
 * indices below 2^31, -1 / +INF for empty entries, distances >= 0) into
 * out_idx, out_dist [Q][k] (device), the k smallest (distance, index) per
 * query, padded with -1 / +INF.  Asynchronous on stream.
 *
 * thr_out and thr_in may be host or device memory (a host thr_out makes the
 * call synchronous); other arguments as in knn_search_ex.
 */
dtw_status knn_seed_thresholds(const float *db, int64_t N, const float *queries, int64_t Q,
                               int32_t n, int32_t w, int32_t p, int32_t k,
                               const dtw_options *opt, float *thr_out, void *stream);
dtw_status knn_search_bounded(const float *db, int64_t N, const float *queries, int64_t Q,
                              int32_t n, int32_t w, int32_t p, int32_t k,
                              const dtw_options *opt, const float *thr_in, int64_t *out_idx,
                              float *out_dist, dtw_stats *stats, void *stream);
dtw_status knn_merge_topk(const int64_t *idx, const float *dist, int32_t R, int64_t Q,
                          int32_t k_in, int32_t k, int64_t *out_idx, float *out_dist,
                          void *stream);

/*
 * Stage timing.  While enabled, knn_search records a pair of CUDA events on
 * its stream around each stage (stage index: DTW_STAGE_*), so that the
 * device time of each kernel is measured on the stream it runs on.
 * dtw_profile_read waits for the recorded events, adds their elapsed times
 * into *out (milliseconds and launch counts per stage) and, if reset is
 * non-zero, forgets them.  Recording costs two event records per stage.
 */
enum {
    DTW_STAGE_ENVELOPE = 0,
    DTW_STAGE_LB_KEOGH = 1,
    DTW_STAGE_SEED_SELECT = 2,
    DTW_STAGE_SEED_DTW = 3,
    DTW_STAGE_SEED_KTH = 4,
    DTW_STAGE_LB_IMPROVED = 5,
    DTW_STAGE_DTW = 6,
    DTW_STAGE_FINALIZE = 7,
    DTW_STAGE_DB_PREP = 8, /* per-call database terms: part sums, row envelopes */
    DTW_STAGE_GROUP = 9,   /* survivors of the bounds grouped by query and ordered by bound */
    DTW_NUM_STAGES = 10
};
typedef struct {
    double ms[DTW_NUM_STAGES];        /* device time of each stage, summed over its runs */
    int64_t launches[DTW_NUM_STAGES]; /* kernels each stage launched (the DTW stage in row
                                         phases: one per phase) */
} dtw_profile;

dtw_status dtw_profile_enable(int32_t on);
dtw_status dtw_profile_read(dtw_profile *out, int32_t reset);

/*
 * dtw_band_noalloc: dtw_band (same arguments, same results) for callers that
 * cannot call cudaMalloc or cudaFree, such as a service whose device memory is
 * owned by another allocator or a loop that must not stall on cudaFree's
 * device-wide synchronisation.  The paper has no counterpart: this is a
 * deployment variant.  Its scratch is a fixed 8 MiB array of device memory
 * that belongs to the library and is held on every GPU that loads it until
 * the process exits; it never allocates.  A call whose scratch (the padded
 * query copies: about 16 * (n + w + 2*C + 8) bytes per query row, with C the band
 * slot count, plus 256 bytes) does not fit returns DTW_ERR_INVALID_ARG.  All
 * calls share the array, so calls that overlap on the GPU race.  The first
 * call in each CUDA context of a device (the primary context is created anew
 * after cudaDeviceReset) looks up the array's device address and keeps it for
 * that context's later calls; make that first call before any stream capture.
 */
dtw_status dtw_band_noalloc(const float *x, const float *y, int64_t N, int32_t y_stride,
                            int32_t n, int32_t w, int32_t p, float threshold, float *out,
                            void *stream);

/*
 * Multi-length index.  The paper states the search for one query length; a
 * database holding series of several lengths is searched bucket by bucket,
 * since LB_Keogh, LB_Improved and the band DTW of Sec. 4-8 compare series of
 * equal length only.  An index owns one bucket per length (copied into
 * device memory it allocates) and answers batches of queries of mixed
 * length n, band w and neighbour count k.  Each query gets exactly the result
 * knn_search gives for it against its bucket with the index's options
 * (same neighbours, same distances); batching, streams, graphs and tuning
 * change only the speed.
 *
 * Batch execution: queries of equal (n, w, k) form a group; each group is one
 * cascade run (the stages of knn_search for a block of queries), and the
 * groups run concurrently on a pool of streams forked from and joined back
 * to the caller's stream.  Flags:
 *   DTW_BATCH_GRAPH     capture the batch's device work as a CUDA graph the
 *                       first time a batch of the same group shapes (lengths,
 *                       bands, k, queries per group, tuning) is seen, and
 *                       replay it afterwards; up to 16 graphs are cached.
 *   DTW_BATCH_AUTOTUNE  before running, time candidate parameters (Sec. 9
 *                       parts, seeds, filter segment length) on up to 256 of
 *                       the group's own queries for every (n, w, k) that has
 *                       no tuning yet, and keep the fastest (synchronous).
 *   DTW_BATCH_SERIAL    run the groups one after another on the caller's stream.
 *   DTW_BATCH_PER_QUERY run every query as its own cascade (one query per
 *                       launch of each stage), one after another: the
 *                       unbatched baseline.  GRAPH is ignored with it.
 *   DTW_BATCH_PERSISTENT after each group's first stages (envelopes, the
 *                       stored bound of every pair, seeds and their
 *                       threshold), run the rest of the cascade for all
 *                       groups in one persistent launch over a device queue
 *                       of (query, candidate chunk) items: each warp takes an
 *                       item and runs LB_Keogh, LB_Improved and the band DTW
 *                       (one warp per pair) on that chunk, against the
 *                       query's live threshold, which every completed DTW
 *                       lowers at once; one more launch forms every query's
 *                       top-k.  Needs the default cascade mode, p in {1, 2},
 *                       bands 2w + 1 <= 512 and groups small enough for one
 *                       cascade run (about 2^27 / N queries); otherwise the
 *                       call fails with DTW_ERR_INVALID_ARG.  With AUTOTUNE
 *                       the candidate chunk length is also timed (512 to
 *                       4096) the first time, on the batch itself.
 *                       Combines with GRAPH; not with SERIAL or PER_QUERY.
 * Memory: the index grows a device arena for the largest batch seen (growth
 * synchronises the device and drops the cached graphs) and a pinned host map
 * of one entry per query.  Calls on one index are serialised by a mutex, and
 * the device work of successive searches is ordered on the index's side.
 */
typedef struct dtw_index dtw_index;

enum {
    DTW_BATCH_GRAPH = 1,
    DTW_BATCH_AUTOTUNE = 2,
    DTW_BATCH_SERIAL = 4,
    DTW_BATCH_PER_QUERY = 8,
    DTW_BATCH_PERSISTENT = 16
};

/* Cascade parameters of one (n, w, k); see dtw_options for parts, seeds and dtw_path.
 * seg_len: candidates per filter segment (512, 1024, 2048 or 4096; 0: for n <= 256
 * 4096 when the bucket holds 65,536 series or more, else 2048; 1024 for longer series). ms: time of the
 * tuning sample in milliseconds, or -1 when the values are the defaults. */
typedef struct {
    int32_t parts;
    int32_t seeds;
    int32_t seg_len;
    float ms;
    int32_t dtw_path; /* as in dtw_options */
    int32_t filter_warps; /* warps per LB_Improved filter CTA, 1..8; 0: chosen from occupancy */
} dtw_tuning;

typedef struct {
    int32_t buckets;
    int32_t graphs_cached;
    int64_t resident_bytes; /* bucket series and their part sums */
    int64_t arena_bytes;    /* batch workspace */
    int64_t graph_captures;
    int64_t graph_replays;
} dtw_index_stats;

/* Creates an empty index for DTW_p on the current device.  opt (nullable)
 * gives the cascade mode, slack and the default seeds and parts. */
dtw_status dtw_index_create(int32_t p, const dtw_options *opt, dtw_index **out);

/* Adds the bucket of length n: db [N][n], host or device memory, is copied
 * into memory the index owns (synchronous).  One bucket per length. */
dtw_status dtw_index_add_bucket(dtw_index *ix, const float *db, int64_t N, int32_t n);

/* Times candidate parameters on sample [count][n] (host or device) and stores
 * the fastest for (n, w, k); out (nullable) receives them.  Synchronous. */
dtw_status dtw_index_tune(dtw_index *ix, const float *sample, int64_t count, int32_t n,
                          int32_t w, int32_t k, dtw_tuning *out);

/* Reads (defaults when untuned) or sets the parameters used for (n, w, k). */
dtw_status dtw_index_get_tuning(dtw_index *ix, int32_t n, int32_t w, int32_t k, dtw_tuning *out);
dtw_status dtw_index_set_tuning(dtw_index *ix, int32_t n, int32_t w, int32_t k, const dtw_tuning *t);

/*
 * Batched exact k-NN: query i has length q_len[i], band q_w[i] and
 * neighbour count q_k[i] (host arrays of Q entries); the queries' values are
 * concatenated in order in `queries` (sum of q_len floats, host or device).
 * out_idx [Q][k_stride] (int64) and out_dist [Q][k_stride] (fp32, root taken),
 * both host or both device memory, receive each query's neighbours ordered by
 * (distance, index); entries past q_k[i], and past the bucket size, are
 * idx -1, distance +INF.  1 <= q_k[i] <= k_stride <= DTW_MAX_K.  A query whose
 * length has no bucket fails the call with DTW_ERR_NO_BUCKET before any work.
 * stats (nullable) receives the counters summed over the batch; stats and host
 * outputs make the call synchronous.
 */
dtw_status dtw_index_search(dtw_index *ix, const float *queries, int64_t Q,
                            const int32_t *q_len, const int32_t *q_w, const int32_t *q_k,
                            int32_t k_stride, int32_t flags, int64_t *out_idx,
                            float *out_dist, dtw_stats *stats, void *stream);

dtw_status dtw_index_info(dtw_index *ix, dtw_index_stats *out);

/* Frees the index (waits for its work). */
dtw_status dtw_index_destroy(dtw_index *ix);

/*
 * Request server: continuous batching of k-NN queries over an index.  Each
 * request (one query of any length that has a bucket, its band w and k) is
 * queued on arrival.  A scheduler thread owns `slots` batch slots; each slot
 * has its own device arena of slot_bytes (reserved at creation, never grown),
 * pinned staging buffers and streams.  Whenever a slot is free it admits the
 * oldest waiting requests, as many as the arena holds (admission by memory)
 * and at most max_batch, and launches them as one batch (dtw_index_search's
 * execution); batches of different slots run on the device at the same time,
 * so requests that arrive while others are on the GPU start as soon as a slot
 * frees.  max_wait_us > 0 lets a partial batch wait that long for more
 * arrivals while another batch is running.  Each request's result equals
 * what knn_search gives it alone.  The paper has no counterpart: this is the
 * deployment layer around its method.
 */
typedef struct dtw_server dtw_server;

typedef struct {
    int32_t slots;      /* batches in flight at once, 1..16 (default 4) */
    int32_t max_batch;  /* requests per batch, 1..65536 (default 512) */
    int64_t slot_bytes; /* device arena per slot; 0: 2 GiB */
    int32_t max_wait_us;
    int32_t flags;      /* DTW_BATCH_GRAPH, DTW_BATCH_SERIAL or DTW_BATCH_PER_QUERY for every batch */
    int32_t batch_timeout_ms; /* watchdog: a batch still running this long after launch completes
                                 its requests with DTW_ERR_TIMEOUT (their buffers are not written;
                                 the slot stays reserved until the device finishes); 0: none */
} dtw_server_config;

typedef struct {
    uint64_t ticket;
    int32_t status;     /* DTW_OK, or the error that ended the request's batch */
    int32_t k;
    int64_t arrival_ns; /* dtw_monotonic_ns clock */
    int64_t admit_ns;   /* its batch was formed */
    int64_t done_ns;    /* its results were in the caller's buffers */
} dtw_completion;

typedef struct {
    int64_t submitted, completed, failed, batches;
    int64_t max_inflight_batches, max_batch_seen;
    int64_t pending, inflight_batches;
    int64_t timed_out; /* requests completed by the watchdog */
} dtw_server_stats;

/* Starts a server on ix (which must outlive it); cfg may be NULL (defaults).
 * Reserves slots * slot_bytes of device memory. */
dtw_status dtw_server_create(dtw_index *ix, const dtw_server_config *cfg, dtw_server **out);

/* Queues one request: query [n] (host, copied), band w, k neighbours.  Its
 * result is written to out_idx [k] and out_dist [k] (host memory that must
 * stay valid until the request's completion is polled).  arrival_ns (0: now)
 * is the request's arrival time on the dtw_monotonic_ns clock.  Fails with
 * DTW_ERR_INVALID_ARG when the query holds a NaN or an infinity (they break
 * the ordering of the bounds), DTW_ERR_NO_BUCKET when no bucket has length n,
 * DTW_ERR_OOM when a batch of this request alone does not fit slot_bytes. */
dtw_status dtw_server_submit(dtw_server *srv, const float *query, int32_t n, int32_t w, int32_t k,
                             int64_t *out_idx, float *out_dist, int64_t arrival_ns, uint64_t *ticket);

/* Takes up to max completion records (waiting up to wait_ms for the first). */
dtw_status dtw_server_poll(dtw_server *srv, dtw_completion *out, int32_t max, int32_t *count,
                           int32_t wait_ms);

dtw_status dtw_server_info(dtw_server *srv, dtw_server_stats *out);

/* Completes every queued request, then stops the scheduler and frees the server. */
dtw_status dtw_server_destroy(dtw_server *srv);

/* The server's clock (CLOCK_MONOTONIC), nanoseconds. */
int64_t dtw_monotonic_ns(void);

/* Message of the last failed call on this host thread ("" if none). */
const char *dtw_last_error(void);

/* Library version string. */
const char *dtw_version(void);

#ifdef __cplusplus
}
#endif

#endif /* DTWKNN_H */
