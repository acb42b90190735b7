// Host-side plan, workspace layout and launch sequence of one cascade run
// (Algorithms 2/3 for a batch of equal-length queries against one database).
// Internal: the public ABI is include/dtwknn.h.
#pragma once

#include "common.cuh"
#include "dtw.cuh"

namespace dtwk {

// Bump allocator over a workspace block; sizes are rounded to 256 bytes.  With
// base == nullptr it only measures.
struct Carve {
    size_t off = 0;
    char *base = nullptr;
    template <typename T>
    T *take(size_t count) {
        size_t bytes = (count * sizeof(T) + 255) & ~size_t(255);
        T *p = reinterpret_cast<T *>(base ? base + off : nullptr);
        off += bytes;
        return p;
    }
};

// Sizes and parameters of one run: database of N rows of length n, at most Qc
// queries per run, band w (clamped to n-1), k neighbours.
struct CascadePlan {
    int64_t N;
    int n, we, p, k, mode;
    DtwGeom g;
    float slack;
    int parts;       // piecewise-sum parts d, or -1 (pre-filter off)
    bool summary;    // parts > 0
    PartGeom pg;
    int S;           // seeds per query
    int64_t Qc;      // queries per run
    int seg_len;     // candidates per filter segment
    int filter_warps;
    bool seeds_on_threads;  // seeds of long series one thread per pair (runs that overlap with others)
    int nseg;        // sub-segments per query
    int seg_per_cta; // filter segments per CTA
    int dtw_path;    // 0 auto, 1 thread per pair, 2 warp per pair (main DTW stage)
    int dtw_phase;   // main DTW stage on the thread-per-pair register path in row phases of this many rows (0: off)
    int64_t cont_cap;  // entries of each row-phase continuation list
    int filter_path; // 1 one warp per pair, 2 batches of eight pairs per warp
    int lb_abandon;  // early abandoning inside the bound sums (streamed long rows)
    int order_first; // pairs per query the DTW stage takes first, by ascending bound (0: filter order)
};

// Device buffers of one run, carved from a workspace.
struct CascadeWs {
    float *U, *L, *UL, *LU, *copies, *lb, *PU, *PL, *seed_res, *lbi_u, *pair_lbi, *pair_res;
    unsigned long long *tile_min, *misc;
    float *cont_state[2];    // row-phase continuation lists (dtw_phase > 0)
    int64_t *cont_pi[2];
    Pair *seed_pairs, *pairs_u, *pairs;
    uint32_t *gmin, *bsf;
    int32_t *qcount, *qstart, *qstart_b, *seg_start, *seg_count;
};

// o.parts: 0 = default (n/8 for n >= 64, else off), -1 = off, else d.
// o.seeds: 0 = default (16); clamped to [k, 32] and to N.
// seg_len: 0 = default (for n <= 256: 4096 when N >= 65536, else 2048; 1024 for
// longer series); filter_warps: 0 = default.
CascadePlan make_plan(int64_t N, int64_t Qmax, int n, int w, int p, int k, const dtw_options &o,
                      int seg_len = 0, int filter_warps = 0);
CascadeWs carve_ws(const CascadePlan &pl, Carve &cv);
size_t cascade_ws_bytes(const CascadePlan &pl);

// One run over qn <= pl.Qc queries q [qn][n] (device).  PX [N][parts] and
// xmax_bits are the database part sums and max |x| (launch_summarize), used
// when pl.summary; XU, XL [N][n] the database rows' envelopes for band pl.we
// (launch_envelope), used when pl.mode is DTW_MODE_IMPROVED.  counters: CNT_ALLOC device words (run counters, seed-stage
// counters, the error word CNT_ERR), accumulated, zeroed by the caller.  Outputs
// out_idx/out_dist [qn][k] (device).  Asynchronous on s; allocates nothing.
cudaError_t cascade_run(const CascadePlan &pl, const CascadeWs &ws, const float *db, const float *PX,
                        const unsigned *xmax_bits, const float *XU, const float *XL, const float *q, int qn,
                        int64_t *out_idx, float *out_dist, unsigned long long *counters, cudaStream_t s,
                        const float *thr_in = nullptr, float *thr_out = nullptr, bool prefix_only = false);

// The device buffers of one run (cascade_run's view of ws and its
// arguments), for callers that launch stages themselves.
CascadeBufs cascade_bufs(const CascadePlan &pl, const CascadeWs &ws, const float *db, const float *XU, const float *XL,
                         const float *q, int qn, int64_t *out_idx, float *out_dist, unsigned long long *counters);

// The first stages of a run (asynchronous on s, allocates nothing): the
// queries' envelopes and padded copies, the stored bound of every pair (the
// piecewise-sum bound or LB_Keogh), the seeds, their DTW and the seed
// threshold.  Afterwards b.bsf / b.gmin hold each query's threshold, b.lb
// its bounds (NaN at the seeds) and the seed slots their DTW^p.
cudaError_t cascade_prefix(const CascadePlan &pl, const CascadeWs &ws, const CascadeBufs &b, const float *PX,
                           const unsigned *xmax_bits, cudaStream_t s);

// Whether a run under pl reads the database envelopes XU, XL.
inline bool plan_needs_db_envelope(const CascadePlan &pl) { return pl.N > 0 && pl.mode == DTW_MODE_IMPROVED; }

// The database terms a run reads, computed from db [N][n]: the part sums PX
// [N][parts] and max |x| (xmax_bits, 8 bytes) when pl.summary, and the row
// envelopes XU, XL [N][n] when plan_needs_db_envelope(pl).  Timed as stage
// DTW_STAGE_DB_PREP.
cudaError_t prepare_database(const CascadePlan &pl, const float *db, float *PX, unsigned *xmax_bits, float *XU,
                             float *XL, cudaStream_t s);

// Adds the statistics of Q queries run under pl, from the host copy of the
// CNT_ALLOC counter words, to st.
void cascade_stats(const CascadePlan &pl, int64_t Q, const unsigned long long *h, dtw_stats *st);

// Stage timing (dtw_profile_enable / dtw_profile_read).  Stages launched while
// a stream is being captured are not timed.
void profile_set(bool on);
cudaError_t profile_collect(double *ms, int64_t *launches, bool reset);

}  // namespace dtwk
