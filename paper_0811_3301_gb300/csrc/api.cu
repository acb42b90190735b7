// C ABI of the DTW retrieval cascade (include/dtwknn.h): argument checks,
// the per-device workspace, host/device staging and the launch sequence of
// knn_search.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "dtw.cuh"

namespace dtwk {

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local char g_err[512] = "";

static dtw_status fail(dtw_status st, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return st;
}

// Sets this thread's last-error message (used by entry points defined in
// other translation units).
void set_error_message(const char *msg) { snprintf(g_err, sizeof(g_err), "%s", msg ? msg : ""); }

#define CUDA_TRY(expr)                                                                    \
    do {                                                                                  \
        cudaError_t e_ = (expr);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(DTW_ERR_CUDA, "%s failed: %s", #expr, cudaGetErrorString(e_));     \
    } while (0)

int device_sm_count() {
    static int cache[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (cache[dev] == 0) {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        cache[dev] = v > 0 ? v : 1;
    }
    return cache[dev];
}

// ---------------------------------------------------------------------------
// workspace: one growable device allocation per device
// ---------------------------------------------------------------------------
struct Workspace {
    void *base = nullptr;
    size_t cap = 0;
};
static Workspace g_ws[64];
static std::mutex g_ws_mu;

static dtw_status workspace_get(size_t bytes, void **out) {
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(DTW_ERR_INTERNAL, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_ws_mu);
    Workspace &w = g_ws[dev];
    if (w.cap < bytes) {
        if (w.base) {
            cudaError_t e = cudaFree(w.base);  // synchronises the device
            w.base = nullptr;
            w.cap = 0;
            if (e != cudaSuccess) return fail(DTW_ERR_CUDA, "cudaFree: %s", cudaGetErrorString(e));
        }
        size_t want = bytes + bytes / 8 + (1u << 20);
        cudaError_t e = cudaMalloc(&w.base, want);
        if (e != cudaSuccess) {
            cudaGetLastError();
            w.base = nullptr;
            return fail(DTW_ERR_OOM, "workspace of %zu bytes: %s", want, cudaGetErrorString(e));
        }
        w.cap = want;
    }
    *out = w.base;
    return DTW_OK;
}

// Bump allocator over a workspace block; sizes are rounded to 256 bytes.
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

static bool is_device_ptr(const void *p) {
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

static dtw_status check_common(int32_t n, int32_t w, int32_t p) {
    if (n < 1 || n > DTW_MAX_N) return fail(DTW_ERR_INVALID_ARG, "n=%d outside [1, %d]", n, DTW_MAX_N);
    if (w < 0) return fail(DTW_ERR_INVALID_ARG, "w=%d must be >= 0", w);
    if (p != 1 && p != 2) return fail(DTW_ERR_INVALID_ARG, "p=%d must be 1 or 2", p);
    return DTW_OK;
}

static dtw_status check_band(int32_t n, int32_t w) {
    int we = w < n - 1 ? w : n - 1;
    if (2 * we + 1 > 2048)
        return fail(DTW_ERR_INVALID_ARG, "DTW band 2*min(w,n-1)+1 = %d exceeds 2048", 2 * we + 1);
    return DTW_OK;
}

// ---------------------------------------------------------------------------
// stage timing (dtw_profile_enable / dtw_profile_read)
// ---------------------------------------------------------------------------
struct StageEvents {
    int stage;
    cudaEvent_t a, b;
};
static bool g_prof_on = false;
static std::mutex g_prof_mu;
static std::vector<StageEvents> g_prof_events;

struct StageTimer {
    StageEvents ev{};
    bool on = false;
    cudaStream_t s;
    StageTimer(int stage, cudaStream_t st) : s(st) {
        on = g_prof_on;
        if (!on) return;
        ev.stage = stage;
        if (cudaEventCreate(&ev.a) != cudaSuccess || cudaEventCreate(&ev.b) != cudaSuccess) {
            cudaGetLastError();
            on = false;
            return;
        }
        cudaEventRecord(ev.a, s);
    }
    ~StageTimer() {
        if (!on) return;
        cudaEventRecord(ev.b, s);
        std::lock_guard<std::mutex> lk(g_prof_mu);
        g_prof_events.push_back(ev);
    }
};

static cudaError_t launch_dtw(const DtwJob &j, const DtwGeom &g, cudaStream_t s) {
    return j.p == 1 ? launch_dtw_p1(j, g, s) : launch_dtw_p2(j, g, s);
}

}  // namespace dtwk

using namespace dtwk;

extern "C" {

const char *dtw_last_error(void) { return g_err; }

dtw_status dtw_profile_enable(int32_t on) {
    g_err[0] = 0;
    g_prof_on = on != 0;
    return DTW_OK;
}

dtw_status dtw_profile_read(dtw_profile *out, int32_t reset) {
    g_err[0] = 0;
    if (!out) return fail(DTW_ERR_INVALID_ARG, "null pointer");
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (auto &ev : g_prof_events) {
        cudaError_t e = cudaEventSynchronize(ev.b);
        if (e != cudaSuccess) return fail(DTW_ERR_CUDA, "cudaEventSynchronize: %s", cudaGetErrorString(e));
        float ms = 0.0f;
        e = cudaEventElapsedTime(&ms, ev.a, ev.b);
        if (e != cudaSuccess) return fail(DTW_ERR_CUDA, "cudaEventElapsedTime: %s", cudaGetErrorString(e));
        if (ev.stage >= 0 && ev.stage < DTW_NUM_STAGES) {
            out->ms[ev.stage] += ms;
            out->launches[ev.stage] += 1;
        }
    }
    if (reset) {
        for (auto &ev : g_prof_events) {
            cudaEventDestroy(ev.a);
            cudaEventDestroy(ev.b);
        }
        g_prof_events.clear();
    }
    return DTW_OK;
}

const char *dtw_version(void) { return "dtwknn 0.1 (sm_103a)"; }

dtw_status dtw_envelope(const float *y, int64_t count, int32_t n, int32_t w, float *U, float *L,
                        void *stream) {
    g_err[0] = 0;
    if (n < 1 || n > DTW_MAX_N) return fail(DTW_ERR_INVALID_ARG, "n=%d outside [1, %d]", n, DTW_MAX_N);
    if (w < 0) return fail(DTW_ERR_INVALID_ARG, "w=%d must be >= 0", w);
    if (count < 0 || count > INT32_MAX) return fail(DTW_ERR_INVALID_ARG, "count=%lld out of range", (long long)count);
    if (count == 0) return DTW_OK;
    if (!y || !U || !L) return fail(DTW_ERR_INVALID_ARG, "null pointer");
    CUDA_TRY(launch_envelope(y, count, n, w, U, L, QueryCopies{}, 0, (cudaStream_t)stream));
    return DTW_OK;
}

dtw_status lb_keogh(const float *cand, int64_t N, const float *U, const float *L, int32_t n,
                    int32_t p, float *out, void *stream) {
    g_err[0] = 0;
    dtw_status st = check_common(n, 0, p);
    if (st != DTW_OK) return st;
    if (N < 0) return fail(DTW_ERR_INVALID_ARG, "N=%lld must be >= 0", (long long)N);
    if (N == 0) return DTW_OK;
    if (!cand || !U || !L || !out) return fail(DTW_ERR_INVALID_ARG, "null pointer");
    CUDA_TRY(launch_lbk_single(cand, N, U, L, n, p, out, (cudaStream_t)stream));
    return DTW_OK;
}

dtw_status lb_piecewise(const float *cand, int64_t N, const float *U, const float *L, int32_t n, int32_t d,
                        int32_t p, float *out, void *stream) {
    g_err[0] = 0;
    dtw_status st = check_common(n, 0, p);
    if (st != DTW_OK) return st;
    if (d < 1 || d > n) return fail(DTW_ERR_INVALID_ARG, "d=%d outside [1, n=%d]", d, n);
    if (N < 0) return fail(DTW_ERR_INVALID_ARG, "N=%lld must be >= 0", (long long)N);
    if (N == 0) return DTW_OK;
    if (!cand || !U || !L || !out) return fail(DTW_ERR_INVALID_ARG, "null pointer");
    void *ws = nullptr;
    if ((st = workspace_get(((size_t)N * d + 2 * (size_t)d) * sizeof(float) + 256, &ws)) != DTW_OK) return st;
    CUDA_TRY(launch_lbp_single(cand, N, U, L, n, d, p, out, (float *)ws, (cudaStream_t)stream));
    return DTW_OK;
}

dtw_status lb_improved(const float *cand, int64_t N, const float *q, const float *U, const float *L,
                       int32_t n, int32_t w, int32_t p, float *out, void *stream) {
    g_err[0] = 0;
    dtw_status st = check_common(n, w, p);
    if (st != DTW_OK) return st;
    if (N < 0) return fail(DTW_ERR_INVALID_ARG, "N=%lld must be >= 0", (long long)N);
    if (N == 0) return DTW_OK;
    if (!cand || !q || !U || !L || !out) return fail(DTW_ERR_INVALID_ARG, "null pointer");
    CUDA_TRY(launch_lbi_single(cand, N, q, U, L, n, w, p, out, (cudaStream_t)stream));
    return DTW_OK;
}

dtw_status dtw_band(const float *x, const float *y, int64_t N, int32_t y_stride, int32_t n, int32_t w,
                    int32_t p, float threshold, float *out, void *stream) {
    g_err[0] = 0;
    dtw_status st = check_common(n, w, p);
    if (st != DTW_OK) return st;
    if ((st = check_band(n, w)) != DTW_OK) return st;
    if (N < 0 || N > INT32_MAX) return fail(DTW_ERR_INVALID_ARG, "N=%lld out of range", (long long)N);
    if (y_stride != 0 && y_stride != n)
        return fail(DTW_ERR_INVALID_ARG, "y_stride=%d must be 0 or n=%d", y_stride, n);
    if (std::isnan(threshold) || threshold < 0.0f)
        return fail(DTW_ERR_INVALID_ARG, "threshold must be >= 0 or +INF");
    if (N == 0) return DTW_OK;
    if (!x || !y || !out) return fail(DTW_ERR_INVALID_ARG, "null pointer");
    cudaStream_t s = (cudaStream_t)stream;
    const int we = w < n - 1 ? w : n - 1;
    const DtwGeom g = dtw_geom(n, we);
    const int64_t nq = y_stride ? N : 1;
    Carve cv;
    cv.take<float>((size_t)nq * 4 * g.ylen);
    cv.take<unsigned long long>(1);
    void *ws = nullptr;
    if ((st = workspace_get(cv.off, &ws)) != DTW_OK) return st;
    Carve c2;
    c2.base = (char *)ws;
    QueryCopies qc;
    qc.data = c2.take<float>((size_t)nq * 4 * g.ylen);
    qc.padl = g.padl;
    qc.ylen = g.ylen;
    unsigned long long *cursor = c2.take<unsigned long long>(1);
    CUDA_TRY(launch_query_copies(y, nq, n, qc, s));
    CUDA_TRY(cudaMemsetAsync(cursor, 0, sizeof(unsigned long long), s));
    DtwJob j{};
    j.db = x;
    j.n = n;
    j.w = we;
    j.p = p;
    j.k = 1;
    j.qc = qc;
    j.pairs = nullptr;
    j.npairs = N;
    j.per_pair_y = y_stride ? 1 : 0;
    j.fixed_thr = std::isinf(threshold) ? INFINITY : (p == 1 ? threshold : threshold * threshold);
    j.abandon = std::isinf(threshold) ? 0 : 1;
    j.res = out;
    j.root_out = 1;
    j.cursor = cursor;
    CUDA_TRY(launch_dtw(j, g, s));
    return DTW_OK;
}

dtw_status knn_search_ex(const float *db, int64_t N, const float *queries, int64_t Q, int32_t n,
                         int32_t w, int32_t p, int32_t k, const dtw_options *opt, int64_t *out_idx,
                         float *out_dist, dtw_stats *stats, void *stream) {
    g_err[0] = 0;
    dtw_status st = check_common(n, w, p);
    if (st != DTW_OK) return st;
    if ((st = check_band(n, w)) != DTW_OK) return st;
    if (N < 0 || N > INT32_MAX / 2) return fail(DTW_ERR_INVALID_ARG, "N=%lld out of range", (long long)N);
    if (Q < 0 || Q > INT32_MAX / 2) return fail(DTW_ERR_INVALID_ARG, "Q=%lld out of range", (long long)Q);
    if (k < 1 || k > DTW_MAX_K) return fail(DTW_ERR_INVALID_ARG, "k=%d outside [1, %d]", k, DTW_MAX_K);
    dtw_options o{DTW_MODE_IMPROVED, 1e-6f, 0, 0};
    if (opt) o = *opt;
    if (o.parts < -1 || o.parts > n) return fail(DTW_ERR_INVALID_ARG, "parts=%d outside [-1, n=%d]", o.parts, n);
    if (o.mode < DTW_MODE_IMPROVED || o.mode > DTW_MODE_NOPRUNE)
        return fail(DTW_ERR_INVALID_ARG, "mode=%d unknown", o.mode);
    if (!(o.slack >= 0.0f) || std::isinf(o.slack)) return fail(DTW_ERR_INVALID_ARG, "slack must be finite and >= 0");
    if (o.seeds < 0) return fail(DTW_ERR_INVALID_ARG, "seeds=%d must be >= 0", o.seeds);
    if (stats) memset(stats, 0, sizeof(*stats));
    if (Q == 0) return DTW_OK;
    if (!queries || !out_idx || !out_dist || (N > 0 && !db)) return fail(DTW_ERR_INVALID_ARG, "null pointer");
    cudaStream_t s = (cudaStream_t)stream;

    const int we = w < n - 1 ? w : n - 1;
    const DtwGeom g = dtw_geom(n, we);
    const float slack = fmaxf(o.slack, auto_slack(n));
    // piecewise-sum pre-filter (Sec. 9): d parts
    const int parts = o.parts == 0 ? (n >= 64 ? n / 8 : -1) : o.parts;
    const bool summary = parts > 0 && N > 0;
    const PartGeom pg = part_geom(n, summary ? parts : 1);
    int S = o.seeds > 0 ? o.seeds : 16;
    if (S < k) S = k;
    if (S > 32) S = 32;
    if (S > N) S = (int)N;
    if (S < 1) S = 1;

    const bool db_dev = N == 0 || is_device_ptr(db);
    const bool q_dev = is_device_ptr(queries);
    const bool oi_dev = is_device_ptr(out_idx);
    const bool od_dev = is_device_ptr(out_dist);

    // query chunk: bounds the Q*N-sized buffers
    const int64_t pair_budget = (int64_t)1 << 27;
    int64_t Qc = N > 0 ? pair_budget / N : Q;
    if (Qc < 1) Qc = 1;
    if (Qc > 32768) Qc = 32768;  // grid.y limit of the per-query kernels
    if (Qc > Q) Qc = Q;
    const int seg_len = 1024;
    const int filter_warps = lbi_filter_warps(n, we, S, seg_len);
    // sub-segments per query: candidate segments x filter warps
    const int nseg = N > 0 ? (int)((N + seg_len - 1) / seg_len) * filter_warps : 1;
    const int64_t Nc = N > 0 ? N : 1;

    auto layout = [&](Carve &cv) {
        struct L {
            float *db, *q, *U, *L, *copies, *lb, *seed_res, *pair_lbi, *pair_res, *out_dist, *lbi_u, *PX, *PU, *PL;
            Pair *seed_pairs, *pairs, *pairs_u;
            int32_t *qcount, *qstart;
            uint32_t *gmin, *bsf;
            int32_t *seg_start, *seg_count;
            unsigned long long *misc, *tile_min;
            int64_t *out_idx;
        } l;
        l.db = db_dev ? nullptr : cv.take<float>((size_t)N * n);
        l.q = cv.take<float>((size_t)Qc * n);
        l.U = cv.take<float>((size_t)Qc * n);
        l.L = cv.take<float>((size_t)Qc * n);
        l.copies = cv.take<float>((size_t)Qc * 4 * g.ylen);
        l.lb = cv.take<float>((size_t)Qc * Nc);
        l.PX = summary ? cv.take<float>((size_t)N * parts) : nullptr;
        l.PU = summary ? cv.take<float>((size_t)Qc * parts) : nullptr;
        l.PL = summary ? cv.take<float>((size_t)Qc * parts) : nullptr;
        l.tile_min = cv.take<unsigned long long>((size_t)Qc * lbk_tiles((int)Nc));
        l.seed_pairs = cv.take<Pair>((size_t)Qc * S);
        l.seed_res = cv.take<float>((size_t)Qc * S);
        l.gmin = cv.take<uint32_t>((size_t)Qc * k);
        l.bsf = cv.take<uint32_t>((size_t)Qc);
        l.pairs_u = cv.take<Pair>((size_t)Qc * Nc);
        l.lbi_u = cv.take<float>((size_t)Qc * Nc);
        l.qcount = cv.take<int32_t>((size_t)Qc);
        l.qstart = cv.take<int32_t>((size_t)Qc);

        l.pairs = cv.take<Pair>((size_t)Qc * Nc);
        l.pair_lbi = cv.take<float>((size_t)Qc * Nc);
        l.pair_res = cv.take<float>((size_t)Qc * Nc);
        l.seg_start = cv.take<int32_t>((size_t)Qc * nseg);
        l.seg_count = cv.take<int32_t>((size_t)Qc * nseg);
        l.misc = cv.take<unsigned long long>(32);
        l.out_idx = oi_dev ? nullptr : cv.take<int64_t>((size_t)Q * k);
        l.out_dist = od_dev ? nullptr : cv.take<float>((size_t)Q * k);
        return l;
    };
    Carve sizing;
    layout(sizing);
    void *ws = nullptr;
    if ((st = workspace_get(sizing.off, &ws)) != DTW_OK) return st;
    Carve cv;
    cv.base = (char *)ws;
    auto l = layout(cv);

    const float *dbd = db;
    if (!db_dev) {
        CUDA_TRY(cudaMemcpyAsync(l.db, db, (size_t)N * n * sizeof(float), cudaMemcpyHostToDevice, s));
        dbd = l.db;
    }
    int64_t *oidx = oi_dev ? out_idx : l.out_idx;
    float *odist = od_dev ? out_dist : l.out_dist;
    unsigned long long *pair_count = l.misc + 0;
    unsigned long long *cur_seed = l.misc + 1;
    unsigned long long *cur_pairs = l.misc + 2;
    unsigned long long *counters = l.misc + 8;
    unsigned long long *seed_counters = l.misc + 16;
    CUDA_TRY(cudaMemsetAsync(counters, 0, 2 * CNT_NUM * sizeof(unsigned long long), s));
    unsigned *xmax_bits = reinterpret_cast<unsigned *>(l.misc + 24);
    if (summary) {
        // part sums of the database rows, once per call
        CUDA_TRY(cudaMemsetAsync(xmax_bits, 0, sizeof(unsigned long long), s));
        CUDA_TRY(launch_summarize(dbd, N, n, parts, l.PX, xmax_bits, s));
    }

    for (int64_t q0 = 0; q0 < Q; q0 += Qc) {
        const int qn = (int)((Q - q0) < Qc ? (Q - q0) : Qc);
        const float *qd;
        if (q_dev) {
            qd = queries + q0 * n;
        } else {
            CUDA_TRY(cudaMemcpyAsync(l.q, queries + q0 * n, (size_t)qn * n * sizeof(float),
                                     cudaMemcpyHostToDevice, s));
            qd = l.q;
        }
        CUDA_TRY(cudaMemsetAsync(l.misc, 0, 8 * sizeof(unsigned long long), s));
        QueryCopies qc;
        qc.data = l.copies;
        qc.padl = g.padl;
        qc.ylen = g.ylen;
        {
            StageTimer tm(DTW_STAGE_ENVELOPE, s);
            CUDA_TRY(launch_envelope(qd, qn, n, we, l.U, l.L, qc, g.padl, s));
        }

        CascadeBufs b{};
        b.db = dbd;
        b.queries = qd;
        b.U = l.U;
        b.L = l.L;
        b.qc = qc;
        b.N = (int)N;
        b.Q = qn;
        b.n = n;
        b.w = we;
        b.p = p;
        b.k = k;
        b.mode = o.mode;
        b.slack = slack;
        b.lb = l.lb;
        b.tile_min = l.tile_min;
        b.ntiles = lbk_tiles((int)Nc);
        b.S = N > 0 ? S : 0;
        b.seed_pairs = l.seed_pairs;
        b.seed_res = l.seed_res;
        b.gmin = l.gmin;
        b.bsf = l.bsf;
        b.pairs_u = l.pairs_u;
        b.lbi_u = l.lbi_u;
        b.qcount = l.qcount;
        b.qstart = l.qstart;
        b.pair_total = l.misc + 4;
        b.lbi_inline = o.mode == DTW_MODE_IMPROVED ? 1 : 0;
        b.summary = summary ? 1 : 0;
        b.summary_scale = (summary && p == 2) ? (float)pg.smax : 1.0f;
        b.pairs = l.pairs;
        b.pair_lbi = l.pair_lbi;
        b.pair_res = l.pair_res;
        b.pair_cap = (int64_t)qn * Nc;
        b.pair_count = pair_count;
        b.seg_len = seg_len;
        b.nseg = N > 0 ? nseg : 0;
        b.seg_start = l.seg_start;
        b.seg_count = l.seg_count;
        b.cursor = cur_pairs;
        b.counters = counters;
        b.out_idx = oidx + q0 * k;
        b.out_dist = odist + q0 * k;

        if (N > 0) {
            {
                StageTimer tm(DTW_STAGE_LB_KEOGH, s);
                if (summary) {
                    // piecewise-sum bound of every pair (the tile kernel on the d part sums)
                    CUDA_TRY(launch_query_summary(l.U, l.L, qn, n, parts, xmax_bits, l.PU, l.PL, 1, s));
                    CUDA_TRY(launch_lbk_tile(l.PX, (int)N, l.PU, l.PL, qn, parts, p, l.lb, l.tile_min, s));
                } else {
                    CUDA_TRY(launch_lbk_tile(dbd, (int)N, l.U, l.L, qn, n, p, l.lb, l.tile_min, s));
                }
            }
            {
                StageTimer tm(DTW_STAGE_SEED_SELECT, s);
                CUDA_TRY(launch_seed_select(b, s));
            }
            DtwJob js{};
            js.db = dbd;
            js.n = n;
            js.w = we;
            js.p = p;
            js.k = k;
            js.qc = qc;
            js.pairs = l.seed_pairs;
            js.npairs = (int64_t)qn * S;
            js.slack = slack;
            js.bsf = l.bsf;
            js.gmin = l.gmin;
            js.abandon = 0;
            js.res = l.seed_res;
            js.cursor = cur_seed;
            js.counters = seed_counters;
            {
                StageTimer tm(DTW_STAGE_SEED_DTW, s);
                CUDA_TRY(launch_dtw(js, g, s));
            }
            {
                StageTimer tm(DTW_STAGE_SEED_KTH, s);
                CUDA_TRY(launch_seed_kth(b, s));
            }
            {
                StageTimer tm(DTW_STAGE_LB_IMPROVED, s);
                CUDA_TRY(cudaMemsetAsync(l.qcount, 0, (size_t)qn * sizeof(int32_t), s));
                CUDA_TRY(launch_lbi_filter(b, s));
                CUDA_TRY(launch_group_by_query(b, s));
            }
            DtwJob jp = js;
            jp.pairs = l.pairs;
            jp.npairs = (int64_t)qn * Nc;
            jp.npairs_dev = b.pair_total;
            jp.pair_lbi = o.mode == DTW_MODE_NOPRUNE ? nullptr : l.pair_lbi;
            jp.abandon = o.mode == DTW_MODE_NOPRUNE ? 0 : 1;
            jp.res = l.pair_res;
            jp.cursor = cur_pairs;
            jp.counters = counters;
            {
                StageTimer tm(DTW_STAGE_DTW, s);
                CUDA_TRY(launch_dtw(jp, g, s));
            }
        }
        {
            StageTimer tm(DTW_STAGE_FINALIZE, s);
            CUDA_TRY(launch_finalize(b, s));
        }
    }
    if (!oi_dev)
        CUDA_TRY(cudaMemcpyAsync(out_idx, l.out_idx, (size_t)Q * k * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    if (!od_dev)
        CUDA_TRY(cudaMemcpyAsync(out_dist, l.out_dist, (size_t)Q * k * sizeof(float), cudaMemcpyDeviceToHost, s));
    if (stats || !oi_dev || !od_dev) {
        unsigned long long h[2 * CNT_NUM];
        if (stats) CUDA_TRY(cudaMemcpyAsync(h, counters, sizeof(h), cudaMemcpyDeviceToHost, s));
        CUDA_TRY(cudaStreamSynchronize(s));
        if (stats) {
            const int64_t seeds = N > 0 ? Q * (int64_t)S : 0;
            stats->candidates = Q * N;
            stats->seeds = seeds;
            if (summary) {
                stats->pruned_summary = Q * N - seeds - (int64_t)h[CNT_SUMMARY_PASS];
                stats->pruned_keogh = (int64_t)h[CNT_SUMMARY_PASS] - (int64_t)h[CNT_KEOGH_PASS];
            } else {
                stats->pruned_summary = 0;
                stats->pruned_keogh = Q * N - seeds - (int64_t)h[CNT_KEOGH_PASS];
            }
            stats->pruned_improved = (int64_t)h[CNT_KEOGH_PASS] - (int64_t)h[CNT_LBI_PASS] + (int64_t)h[CNT_DTW_SKIP];
            stats->dtw_computed = (int64_t)h[CNT_DTW_COMPUTED];
            stats->dtw_abandoned = (int64_t)h[CNT_DTW_ABANDONED];
            stats->dtw_cells = (int64_t)h[CNT_DTW_ROWS] * (2 * we + 1);
            stats->seed_cells = (int64_t)h[CNT_NUM + CNT_DTW_ROWS] * (2 * we + 1);
        }
    }
    return DTW_OK;
}

dtw_status knn_search(const float *db, int64_t N, const float *queries, int64_t Q, int32_t n, int32_t w,
                      int32_t p, int32_t k, int64_t *out_idx, float *out_dist, dtw_stats *stats,
                      void *stream) {
    return knn_search_ex(db, N, queries, Q, n, w, p, k, nullptr, out_idx, out_dist, stats, stream);
}

}  // extern "C"
