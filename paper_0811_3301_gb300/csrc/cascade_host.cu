// Host side of one cascade run (Algorithms 2/3 over a batch of queries of one
// length against one database): the plan (sizes and parameters), the
// workspace layout and the launch sequence.  Used by knn_search and by the
// multi-length index.  All launches are asynchronous on one stream and
// allocate nothing, so a run can be captured in a CUDA graph.
#include <cmath>
#include <mutex>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "cascade_host.cuh"

namespace dtwk {

// ---------------------------------------------------------------------------
// stage timing
// ---------------------------------------------------------------------------
static bool g_prof_on = false;
static std::mutex g_prof_mu;
struct StageEvents {
    int stage;
    cudaEvent_t a, b;
    int kernels;  // kernels the stage launched between the two events
};
static std::vector<StageEvents> g_prof_events;

void profile_set(bool on) { g_prof_on = on; }

cudaError_t profile_collect(double *ms, int64_t *launches, bool reset) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (auto &ev : g_prof_events) {
        cudaError_t e = cudaEventSynchronize(ev.b);
        if (e != cudaSuccess) return e;
        float t = 0.0f;
        e = cudaEventElapsedTime(&t, ev.a, ev.b);
        if (e != cudaSuccess) return e;
        if (ev.stage >= 0 && ev.stage < DTW_NUM_STAGES) {
            ms[ev.stage] += t;
            launches[ev.stage] += ev.kernels;
        }
    }
    if (reset) {
        for (auto &ev : g_prof_events) {
            cudaEventDestroy(ev.a);
            cudaEventDestroy(ev.b);
        }
        g_prof_events.clear();
    }
    return cudaSuccess;
}

static const char *const kStageNames[DTW_NUM_STAGES] = {"envelope", "lb_keogh",    "seed_select", "seed_dtw",
                                                         "seed_kth", "lb_improved", "dtw",         "finalize",
                                                         "db_prep",  "group"};

// Marks a stage with an NVTX range (host side, for timeline tools; no cost
// without one attached) and, when profiling is on and the stream is not being
// captured, records a pair of events around it.
struct StageTimer {
    StageEvents ev{};
    bool on = false;
    cudaStream_t s;
    StageTimer(int stage, cudaStream_t st) : s(st) {
        nvtxRangePushA(stage >= 0 && stage < DTW_NUM_STAGES ? kStageNames[stage] : "stage");
        if (!g_prof_on) return;
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
            cudaGetLastError();
            return;
        }
        ev.stage = stage;
        ev.kernels = 1;
        if (cudaEventCreate(&ev.a) != cudaSuccess || cudaEventCreate(&ev.b) != cudaSuccess) {
            cudaGetLastError();
            return;
        }
        on = true;
        cudaEventRecord(ev.a, s);
    }
    ~StageTimer() {
        nvtxRangePop();
        if (!on) return;
        cudaEventRecord(ev.b, s);
        std::lock_guard<std::mutex> lk(g_prof_mu);
        g_prof_events.push_back(ev);
    }
};

#define RUN_TRY(expr)                   \
    do {                                \
        cudaError_t e_ = (expr);        \
        if (e_ != cudaSuccess) return e_; \
    } while (0)

static cudaError_t launch_dtw_any(const DtwJob &j, const DtwGeom &g, cudaStream_t s) {
    return launch_dtw_by_p(j, g, s);
}

// One warp per pair (dtw_lanes.cuh) or one thread per pair for a DTW stage of
// at most `npairs` pairs.  A thread-per-pair DTW of a long series takes
// n (2w+1) dependent cell updates, so when the pairs are too few to fill the
// GPU (about 2^17 threads) the stage time is that latency; the warp path
// shortens it many-fold.  That is the case of the seeds of long series.  The
// main stage lists many pairs, where one thread per pair has the higher
// throughput, unless the caller (or the autotuner) asks for the warp path.
// Bands wider than one thread's registers always take the warp path.  When
// the run overlaps with others (the groups of an index batch, on concurrent
// streams), their kernels fill the SMs that one seed launch leaves idle, so
// the seeds take the thread path's higher throughput instead (batched
// workload: 345 K -> 401 K q/s; a lone run: 8,000 seeds of n = 1,024,
// w = 102, 1.18 -> 1.86 ms).
static int use_lanes(const CascadePlan &pl, int64_t npairs, bool main_stage) {
    if (dtw_lanes_cl(pl.n, pl.we) == 0) return 0;
    if (!main_stage && pl.seeds_on_threads && (pl.dtw_path == 0 || pl.dtw_path >= 4)) return 0;
    if (pl.dtw_path == 3) return main_stage ? 2 : 1;
    if (pl.dtw_path >= 4) return main_stage ? 0 : ((pl.n >= 512 && npairs < ((int64_t)1 << 17)) ? 1 : 0);
    if (pl.dtw_path == 2) return 1;
    if (pl.dtw_path == 1) return 0;
    if (main_stage) return 0;
    return (pl.n >= 512 && npairs < ((int64_t)1 << 17)) ? 1 : 0;
}

// ---------------------------------------------------------------------------
// plan and workspace
// ---------------------------------------------------------------------------
CascadePlan make_plan(int64_t N, int64_t Qmax, int n, int w, int p, int k, const dtw_options &o, int seg_len,
                      int filter_warps) {
    CascadePlan pl{};
    pl.N = N;
    pl.n = n;
    pl.we = w < n - 1 ? w : n - 1;
    pl.p = p;
    pl.k = k;
    pl.mode = o.mode;
    pl.g = dtw_geom(n, pl.we);
    pl.slack = fmaxf(o.slack, auto_slack(n));
    pl.parts = o.parts == 0 ? (n >= 64 ? n / 8 : -1) : o.parts;
    if (pl.parts > n) pl.parts = n;
    if (N <= 0) pl.parts = -1;
    pl.summary = pl.parts > 0;
    pl.pg = part_geom(n, pl.summary ? pl.parts : 1);
    int S = o.seeds > 0 ? o.seeds : 16;
    if (S < k) S = k;
    if (S > 32) S = 32;
    if (S > N) S = (int)N;
    if (S < 1) S = 1;
    pl.S = N > 0 ? S : 0;
    // query chunk: bounds the Q*N-sized buffers
    const int64_t pair_budget = (int64_t)1 << 27;
    int64_t Qc = N > 0 ? pair_budget / N : Qmax;
    if (Qc < 1) Qc = 1;
    if (Qc > 32768) Qc = 32768;  // grid limit of the per-query kernels
    if (Qc > Qmax) Qc = Qmax;
    if (Qc < 1) Qc = 1;
    pl.Qc = Qc;
    // continuation lists of the row phases: pairs still alive at a phase's
    // end; a pair that finds its list full runs on in place
    pl.cont_cap = N > 0 ? std::min<int64_t>(Qc * N, Qc * 2048) : 0;
    // filter segments: longer ones amortise more of a CTA's setup; for series
    // up to 256 (chunks in registers) 4096 measured fastest on large databases
    // (2048 keeps enough CTAs on smaller ones), 1024 for longer series
    pl.seg_len = seg_len > 0 ? seg_len : (n <= 256 ? (N >= 65536 ? 4096 : 2048) : 1024);
    pl.dtw_path = o.dtw_path;
    // The main DTW stage in row phases of 64 rows (k_dtw_reg4p, k_dtw_regp):
    // bands on the register path (up to 64 slots, or 208 for p = 1 and 2),
    // series longer than two phases.  Asked for by dtw_path 4; by default for
    // bands of up to 64 slots in runs of at least 2^24 pairs, where the stage
    // is long enough for the phases' state traffic and extra launches to pay
    // (100,000 x 256, 1,000 queries: DTW stage 1.44 -> 1.37 ms).  Wider bands
    // measured slower in phases (n = 1,024, w = 102: 12.9 -> 14.5 ms), their
    // 209-slot states outweighing the lanes regained.
    const bool phase_ok = !pl.g.wide && pl.g.C <= (p == 1 || p == 2 ? kDtwRegMaxC : kDtwGroupMaxC) &&
                          n > 2 * kDtwPhaseRows && pl.mode != DTW_MODE_NOPRUNE && N > 0;
    const bool phase_big = o.dtw_path == 0 && pl.g.C <= kDtwGroupMaxC && Qc * N >= ((int64_t)1 << 24);
    pl.dtw_phase = (phase_ok && (o.dtw_path == 4 || phase_big)) ? kDtwPhaseRows : 0;
    pl.lb_abandon = o.lb_abandon > 0 ? 1 : 0;
    // The DTW stage takes every query's lowest-bound pairs first (a multiple
    // of 32, at least 2k), so that each query's threshold falls to near its
    // final value early and its remaining pairs are skipped or abandoned
    // sooner.  The order changes which non-neighbours are computed, never
    // the result.
    pl.order_first = pl.mode == DTW_MODE_NOPRUNE ? 0 : 32 * ((k + 15) / 16);
    // filter kernel: pairs in batches of eight per warp where that kernel
    // applies (the default), else one warp per pair
    const bool batch_ok = N > 0 && lbi_batch_applies(n, pl.summary, pl.mode == DTW_MODE_IMPROVED);
    pl.filter_path = (batch_ok && o.filter_path != 1) ? 2 : 1;
    pl.filter_warps = lbi_filter_warps(n, pl.we, std::max(pl.S, 1), pl.seg_len, p, filter_warps);
    const int64_t nsegs = N > 0 ? (N + pl.seg_len - 1) / pl.seg_len : 1;
    pl.nseg = (int)nsegs * pl.filter_warps;
    // filter CTAs: about sixteen waves of four CTAs per SM; each takes a few
    // consecutive segments of its query to amortise the query staging, and
    // the CTAs of all queries that scan one group of segments run close
    // together, so the group's rows stay in L2 (two segments of 4,096
    // candidates: about 1.1x the algorithmic DRAM bytes, against 1.8x with
    // five)
    const int64_t target = (int64_t)device_sm_count() * 64;
    int64_t spc = (Qc * nsegs) / target;
    pl.seg_per_cta = (int)std::max<int64_t>(1, std::min<int64_t>(spc, nsegs));
    return pl;
}

CascadeWs carve_ws(const CascadePlan &pl, Carve &cv) {
    CascadeWs l{};
    const int64_t Qc = pl.Qc;
    const int64_t Nc = pl.N > 0 ? pl.N : 1;
    const int n = pl.n;
    l.U = cv.take<float>((size_t)Qc * n);
    l.L = cv.take<float>((size_t)Qc * n);
    l.UL = plan_needs_db_envelope(pl) ? cv.take<float>((size_t)Qc * n) : nullptr;
    l.LU = plan_needs_db_envelope(pl) ? cv.take<float>((size_t)Qc * n) : nullptr;
    l.copies = cv.take<float>((size_t)Qc * 4 * pl.g.ylen);
    l.lb = cv.take<float>((size_t)Qc * Nc);
    l.PU = pl.summary ? cv.take<float>((size_t)Qc * pl.parts) : nullptr;
    l.PL = pl.summary ? cv.take<float>((size_t)Qc * pl.parts) : nullptr;
    l.tile_min = cv.take<unsigned long long>((size_t)Qc * lbk_tiles((int)Nc));
    l.seed_pairs = cv.take<Pair>((size_t)Qc * std::max(pl.S, 1));
    l.seed_res = cv.take<float>((size_t)Qc * std::max(pl.S, 1));
    l.gmin = cv.take<uint32_t>((size_t)Qc * pl.k);
    l.bsf = cv.take<uint32_t>((size_t)Qc);
    l.pairs_u = cv.take<Pair>((size_t)Qc * Nc);
    l.lbi_u = cv.take<float>((size_t)Qc * Nc);
    l.qcount = cv.take<int32_t>((size_t)Qc);
    l.qstart = cv.take<int32_t>((size_t)Qc);
    l.qstart_b = cv.take<int32_t>((size_t)Qc);
    l.pairs = cv.take<Pair>((size_t)Qc * Nc);
    l.pair_lbi = cv.take<float>((size_t)Qc * Nc);
    l.pair_res = cv.take<float>((size_t)Qc * Nc);
    l.seg_start = cv.take<int32_t>((size_t)Qc * pl.nseg);
    l.seg_count = cv.take<int32_t>((size_t)Qc * pl.nseg);
    l.misc = cv.take<unsigned long long>(16);
    for (int h = 0; h < 2; ++h) {
        l.cont_state[h] = pl.dtw_phase > 0 ? cv.take<float>((size_t)pl.cont_cap * (pl.g.C + 1)) : nullptr;
        l.cont_pi[h] = pl.dtw_phase > 0 ? cv.take<int64_t>((size_t)pl.cont_cap) : nullptr;
    }
    return l;
}

size_t cascade_ws_bytes(const CascadePlan &pl) {
    Carve cv;
    carve_ws(pl, cv);
    return cv.off;
}

// ---------------------------------------------------------------------------
// one run over qn <= Qc queries
// ---------------------------------------------------------------------------
CascadeBufs cascade_bufs(const CascadePlan &pl, const CascadeWs &l, const float *db, const float *XU, const float *XL,
                         const float *q, int qn, int64_t *out_idx, float *out_dist, unsigned long long *counters) {
    const int64_t N = pl.N;
    const int64_t Nc = N > 0 ? N : 1;
    CascadeBufs b{};
    b.db = db;
    b.queries = q;
    b.U = l.U;
    b.L = l.L;
    b.UL = l.UL;
    b.LU = l.LU;
    b.XU = XU;
    b.XL = XL;
    b.qc.data = l.copies;
    b.qc.padl = pl.g.padl;
    b.qc.ylen = pl.g.ylen;
    b.N = (int)N;
    b.Q = qn;
    b.n = pl.n;
    b.w = pl.we;
    b.p = pl.p;
    b.k = pl.k;
    b.mode = pl.mode;
    b.slack = pl.slack;
    b.lb = l.lb;
    b.tile_min = l.tile_min;
    b.ntiles = lbk_tiles((int)Nc);
    b.S = pl.S;
    b.seed_pairs = l.seed_pairs;
    b.seed_res = l.seed_res;
    b.gmin = l.gmin;
    b.bsf = l.bsf;
    b.pairs_u = l.pairs_u;
    b.lbi_u = l.lbi_u;
    b.qcount = l.qcount;
    b.qstart = l.qstart;
    b.qstart_b = l.qstart_b;
    b.order_first = pl.order_first;
    b.pair_total = l.misc + 4;
    b.lead_total = l.misc + 8;
    b.lbi_inline = pl.mode == DTW_MODE_IMPROVED ? 1 : 0;
    b.summary = pl.summary ? 1 : 0;
    b.summary_scale = (pl.summary && pl.p == 2) ? (float)pl.pg.smax : 1.0f;
    b.pairs = l.pairs;
    b.pair_lbi = l.pair_lbi;
    b.pair_res = l.pair_res;
    b.pair_cap = (int64_t)qn * Nc;
    b.pair_count = l.misc + 0;
    b.seg_len = pl.seg_len;
    b.seg_per_cta = pl.seg_per_cta;
    b.filter_warps = pl.filter_warps;
    b.filter_path = pl.filter_path;
    b.lb_abandon = pl.lb_abandon;
    b.dev_err = reinterpret_cast<unsigned *>(counters + CNT_ERR);
    b.nseg = N > 0 ? pl.nseg : 0;
    b.seg_start = l.seg_start;
    b.seg_count = l.seg_count;
    b.cursor = l.misc + 2;
    b.counters = counters;
    b.out_idx = out_idx;
    b.out_dist = out_dist;
    return b;
}

// The DTW job of a run's seed pairs (their results go to the seed slots).
static DtwJob seed_job(const CascadePlan &pl, const CascadeWs &l, const CascadeBufs &b) {
    DtwJob js{};
    js.db = b.db;
    js.n = pl.n;
    js.w = pl.we;
    js.p = pl.p;
    js.k = pl.k;
    js.qc = b.qc;
    js.pairs = l.seed_pairs;
    js.npairs = (int64_t)b.Q * pl.S;
    js.slack = pl.slack;
    js.bsf = l.bsf;
    js.gmin = l.gmin;
    js.res = l.seed_res;
    js.cursor = l.misc + 1;
    js.counters = b.counters + CNT_NUM;
    // On the warp path, where each warp computes its seeds one after another,
    // they run with early abandoning against the live threshold, which the
    // seeds that complete first set and lower (an abandoned seed's DTW
    // exceeds a threshold that is itself at least the final k-th best
    // distance, so it cannot be a neighbour).  One thread per pair runs all
    // seeds at once, so there the checks would only cost.
    js.lanes = use_lanes(pl, js.npairs, false);
    js.abandon = (js.lanes && pl.mode != DTW_MODE_NOPRUNE) ? 1 : 0;
    return js;
}

cudaError_t cascade_prefix(const CascadePlan &pl, const CascadeWs &l, const CascadeBufs &b, const float *PX,
                           const unsigned *xmax_bits, cudaStream_t s) {
    if (plan_needs_db_envelope(pl) && (b.XU == nullptr || b.XL == nullptr)) return cudaErrorInvalidValue;
    const int n = pl.n, p = pl.p, qn = b.Q;
    const int64_t N = pl.N;
    RUN_TRY(cudaMemsetAsync(l.misc, 0, 16 * sizeof(unsigned long long), s));
    {
        StageTimer tm(DTW_STAGE_ENVELOPE, s);
        RUN_TRY(launch_envelope(b.queries, qn, n, pl.we, l.U, l.L, b.qc, pl.g.padl, s, l.UL, l.LU));
    }
    if (N <= 0) return cudaSuccess;
    {
        StageTimer tm(DTW_STAGE_LB_KEOGH, s);
        if (pl.summary) {
            // piecewise-sum bound of every pair: the tile kernel on the d part sums
            RUN_TRY(launch_query_summary(l.U, l.L, qn, n, pl.parts, xmax_bits, l.PU, l.PL, 1, s));
            RUN_TRY(launch_lbk_tile(PX, (int)N, l.PU, l.PL, qn, pl.parts, p, l.lb, l.tile_min, s));
        } else {
            RUN_TRY(launch_lbk_tile(b.db, (int)N, l.U, l.L, qn, n, p, l.lb, l.tile_min, s));
        }
    }
    {
        StageTimer tm(DTW_STAGE_SEED_SELECT, s);
        RUN_TRY(launch_seed_select(b, s));
    }
    {
        StageTimer tm(DTW_STAGE_SEED_DTW, s);
        RUN_TRY(launch_dtw_any(seed_job(pl, l, b), pl.g, s));
    }
    {
        StageTimer tm(DTW_STAGE_SEED_KTH, s);
        RUN_TRY(launch_seed_kth(b, s));
    }
    return cudaSuccess;
}

cudaError_t cascade_run(const CascadePlan &pl, const CascadeWs &l, const float *db, const float *PX,
                        const unsigned *xmax_bits, const float *XU, const float *XL, const float *q, int qn,
                        int64_t *out_idx, float *out_dist, unsigned long long *counters, cudaStream_t s,
                        const float *thr_in, float *thr_out, bool prefix_only) {
    const CascadeBufs b = cascade_bufs(pl, l, db, XU, XL, q, qn, out_idx, out_dist, counters);
    RUN_TRY(cascade_prefix(pl, l, b, PX, xmax_bits, s));
    const int64_t N = pl.N;
    if (thr_in || thr_out) {
        // thresholds exchanged with other shards of the database: lowered
        // before the filter, and/or reported after the seeds
        StageTimer tm(DTW_STAGE_SEED_KTH, s);
        RUN_TRY(launch_threshold_io(b.bsf, qn, N > 0, thr_in, thr_out, s));
    }
    if (prefix_only) return cudaSuccess;
    if (N > 0) {
        {
            StageTimer tm(DTW_STAGE_LB_IMPROVED, s);
            RUN_TRY(cudaMemsetAsync(l.qcount, 0, (size_t)qn * sizeof(int32_t), s));
            RUN_TRY(launch_lbi_filter(b, s));
        }
        {
            StageTimer tm(DTW_STAGE_GROUP, s);
            RUN_TRY(launch_group_by_query(b, s));
        }
        DtwJob jp = seed_job(pl, l, b);
        jp.pairs = l.pairs;
        jp.npairs = (int64_t)qn * N;
        jp.npairs_dev = b.pair_total;
        jp.pair_lbi = pl.mode == DTW_MODE_NOPRUNE ? nullptr : l.pair_lbi;
        jp.abandon = pl.mode == DTW_MODE_NOPRUNE ? 0 : 1;
        jp.res = l.pair_res;
        jp.cursor = b.cursor;
        jp.counters = counters;
        jp.lanes = use_lanes(pl, jp.npairs, true);
        // the grouped pairs' result slots hold their LB_Keogh^p (k_gather)
        jp.tU = jp.abandon ? l.U : nullptr;
        jp.tL = jp.abandon ? l.L : nullptr;
        {
            StageTimer tm(DTW_STAGE_DTW, s);
            if (pl.dtw_phase > 0 && !jp.lanes) {
                // row phases: every listed pair's first rows (the leading
                // region's pairs to the end), then the deferred pairs from
                // one list to the other, a phase per launch
                unsigned long long *cnt[2] = {l.misc + 9, l.misc + 10};
                jp.ph.lead = b.lead_total;
                jp.ph.cap = pl.cont_cap;
                int h = 0;
                for (int r0 = 0; r0 < pl.n; r0 += pl.dtw_phase, h ^= 1) {
                    jp.ph.row_begin = r0;
                    jp.ph.row_end = std::min(pl.n, r0 + pl.dtw_phase);
                    const bool first = r0 == 0;
                    jp.ph.in_state = first ? nullptr : l.cont_state[h ^ 1];
                    jp.ph.in_pi = first ? nullptr : l.cont_pi[h ^ 1];
                    jp.ph.in_count = first ? nullptr : cnt[h ^ 1];
                    jp.ph.out_state = l.cont_state[h];
                    jp.ph.out_pi = l.cont_pi[h];
                    jp.ph.out_count = cnt[h];
                    jp.cursor = l.misc + 11;
                    RUN_TRY(cudaMemsetAsync(cnt[h], 0, sizeof(unsigned long long), s));
                    RUN_TRY(cudaMemsetAsync(jp.cursor, 0, sizeof(unsigned long long), s));
                    RUN_TRY(launch_dtw_phase_by_p(jp, pl.g, s));
                }
                tm.ev.kernels = (pl.n + pl.dtw_phase - 1) / pl.dtw_phase;
            } else {
                RUN_TRY(launch_dtw_any(jp, pl.g, s));
            }
        }
    }
    {
        StageTimer tm(DTW_STAGE_FINALIZE, s);
        RUN_TRY(launch_finalize(b, s));
    }
    return cudaSuccess;
}

cudaError_t prepare_database(const CascadePlan &pl, const float *db, float *PX, unsigned *xmax_bits, float *XU,
                             float *XL, cudaStream_t s) {
    StageTimer tm(DTW_STAGE_DB_PREP, s);
    if (pl.summary) {
        RUN_TRY(cudaMemsetAsync(xmax_bits, 0, sizeof(unsigned long long), s));
        RUN_TRY(launch_summarize(db, pl.N, pl.n, pl.parts, PX, xmax_bits, s));
    }
    if (plan_needs_db_envelope(pl)) RUN_TRY(launch_envelope(db, pl.N, pl.n, pl.we, XU, XL, QueryCopies{}, 0, s));
    return cudaSuccess;
}

void cascade_stats(const CascadePlan &pl, int64_t Q, const unsigned long long *h, dtw_stats *st) {
    const int64_t N = pl.N;
    const int64_t seeds = N > 0 ? Q * (int64_t)pl.S : 0;
    st->candidates += Q * N;
    st->seeds += seeds;
    if (pl.summary) {
        st->pruned_summary += Q * N - seeds - (int64_t)h[CNT_SUMMARY_PASS];
        st->pruned_keogh += (int64_t)h[CNT_SUMMARY_PASS] - (int64_t)h[CNT_KEOGH_PASS];
    } else {
        st->pruned_keogh += Q * N - seeds - (int64_t)h[CNT_KEOGH_PASS];
    }
    st->pruned_improved += (int64_t)h[CNT_KEOGH_PASS] - (int64_t)h[CNT_LBI_PASS] + (int64_t)h[CNT_DTW_SKIP];
    st->dtw_computed += (int64_t)h[CNT_DTW_COMPUTED];
    st->dtw_abandoned += (int64_t)h[CNT_DTW_ABANDONED];
    st->dtw_cells += (int64_t)h[CNT_DTW_CELLS];
    st->seed_cells += (int64_t)h[CNT_NUM + CNT_DTW_CELLS];
    st->dtw_lane_rows += (int64_t)h[CNT_DTW_LANE_ROWS];
    st->dtw_rows += (int64_t)h[CNT_DTW_ROWS];
    st->seed_rows += (int64_t)h[CNT_NUM + CNT_DTW_ROWS];
}

}  // namespace dtwk
