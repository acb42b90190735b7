// C ABI of the DTW retrieval cascade (include/dtwknn.h): argument checks,
// the per-device workspace, host/device staging and the launch sequence of
// knn_search.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "cascade_host.cuh"

namespace dtwk {

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local char g_err[512] = "";

dtw_status fail(dtw_status st, const char *fmt, ...) {
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

// dtw_band takes p in {1, 2, 4} or DTW_P_INF (0); the bounds and the cascade take p in {1, 2}.
static dtw_status check_dtw_p(int32_t n, int32_t w, int32_t p) {
    if (p == 4 || p == DTW_P_INF) return check_common(n, w, 1);
    return check_common(n, w, p);
}

// A threshold on DTW_p in the units the kernels compare (DTW_p^p; DTW_inf itself).
float threshold_power(float t, int32_t p) {
    if (std::isinf(t)) return INFINITY;
    if (p == 2) return t * t;
    if (p == 4) return (t * t) * (t * t);
    return t;
}

static dtw_status check_band(int32_t n, int32_t w) {
    int we = w < n - 1 ? w : n - 1;
    if (2 * we + 1 > 2048)
        return fail(DTW_ERR_INVALID_ARG, "DTW band 2*min(w,n-1)+1 = %d exceeds 2048", 2 * we + 1);
    return DTW_OK;
}

static cudaError_t launch_dtw(const DtwJob &j, const DtwGeom &g, cudaStream_t s) {
    return launch_dtw_by_p(j, g, s);
}

dtw_status check_dtw_band_args(const float *x, const float *y, int64_t N, int32_t y_stride, int32_t n, int32_t w,
                               int32_t p, float threshold, const float *out, bool *empty) {
    *empty = false;
    dtw_status st = check_dtw_p(n, w, p);
    if (st != DTW_OK) return st;
    if ((st = check_band(n, w)) != DTW_OK) return st;
    if (N < 0 || N > INT32_MAX) return fail(DTW_ERR_INVALID_ARG, "N=%lld out of range", (long long)N);
    if (y_stride != 0 && y_stride != n)
        return fail(DTW_ERR_INVALID_ARG, "y_stride=%d must be 0 or n=%d", y_stride, n);
    if (std::isnan(threshold) || threshold < 0.0f)
        return fail(DTW_ERR_INVALID_ARG, "threshold must be >= 0 or +INF");
    if (N == 0) {
        *empty = true;
        return DTW_OK;
    }
    if (!x || !y || !out) return fail(DTW_ERR_INVALID_ARG, "null pointer");
    return DTW_OK;
}

}  // namespace dtwk

using namespace dtwk;

extern "C" {

const char *dtw_last_error(void) { return g_err; }

dtw_status dtw_profile_enable(int32_t on) {
    g_err[0] = 0;
    profile_set(on != 0);
    return DTW_OK;
}

dtw_status dtw_profile_read(dtw_profile *out, int32_t reset) {
    g_err[0] = 0;
    if (!out) return fail(DTW_ERR_INVALID_ARG, "null pointer");
    CUDA_TRY(profile_collect(out->ms, out->launches, reset != 0));
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
    cudaStream_t s = (cudaStream_t)stream;
    const int we = w < n - 1 ? w : n - 1;
    // the candidates' envelopes and the query's second-order envelopes U(L),
    // L(U) (the envelope of L gives U(L), that of U gives L(U))
    auto layout = [&](Carve &cv, float *&XU, float *&XL, float *&UL, float *&LU, float *&t0, float *&t1) {
        XU = cv.take<float>((size_t)N * n);
        XL = cv.take<float>((size_t)N * n);
        UL = cv.take<float>((size_t)n);
        LU = cv.take<float>((size_t)n);
        t0 = cv.take<float>((size_t)n);
        t1 = cv.take<float>((size_t)n);
    };
    float *XU, *XL, *UL, *LU, *t0, *t1;
    Carve sizing;
    layout(sizing, XU, XL, UL, LU, t0, t1);
    void *ws = nullptr;
    if ((st = workspace_get(sizing.off, &ws)) != DTW_OK) return st;
    Carve cv;
    cv.base = (char *)ws;
    layout(cv, XU, XL, UL, LU, t0, t1);
    CUDA_TRY(launch_envelope(cand, N, n, we, XU, XL, QueryCopies{}, 0, s));
    CUDA_TRY(launch_envelope(L, 1, n, we, UL, t0, QueryCopies{}, 0, s));
    CUDA_TRY(launch_envelope(U, 1, n, we, t1, LU, QueryCopies{}, 0, s));
    CUDA_TRY(launch_lbi_single(cand, N, q, U, L, XU, XL, UL, LU, n, p, out, s));
    return DTW_OK;
}

dtw_status dtw_band(const float *x, const float *y, int64_t N, int32_t y_stride, int32_t n, int32_t w,
                    int32_t p, float threshold, float *out, void *stream) {
    g_err[0] = 0;
    bool empty = false;
    dtw_status st = check_dtw_band_args(x, y, N, y_stride, n, w, p, threshold, out, &empty);
    if (st != DTW_OK || empty) return st;
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
    j.fixed_thr = threshold_power(threshold, p);
    j.abandon = std::isinf(threshold) ? 0 : 1;
    j.res = out;
    j.root_out = 1;
    j.cursor = cursor;
    CUDA_TRY(launch_dtw(j, g, s));
    return DTW_OK;
}

dtw_status dtw_triangle(const float *x, const float *y, const float *z, int64_t N, int32_t n, int32_t w, int32_t p,
                        float *ratio, float *dist3, void *stream) {
    g_err[0] = 0;
    dtw_status st = check_common(n, w, p);
    if (st != DTW_OK) return st;
    if ((st = check_band(n, w)) != DTW_OK) return st;
    if (N < 0 || N > INT32_MAX) return fail(DTW_ERR_INVALID_ARG, "N=%lld out of range", (long long)N);
    if (N == 0) return DTW_OK;
    if (!x || !y || !z || !ratio) return fail(DTW_ERR_INVALID_ARG, "null pointer");
    cudaStream_t s = (cudaStream_t)stream;
    const int we = w < n - 1 ? w : n - 1;
    const DtwGeom g = dtw_geom(n, we);
    auto layout = [&](Carve &cv, QueryCopies &qc, float *&d3, unsigned long long *&cur) {
        qc.data = cv.take<float>((size_t)N * 4 * g.ylen);
        qc.padl = g.padl;
        qc.ylen = g.ylen;
        d3 = dist3 ? nullptr : cv.take<float>((size_t)3 * N);
        cur = cv.take<unsigned long long>(3);
    };
    QueryCopies qc;
    float *d3 = nullptr;
    unsigned long long *cur = nullptr;
    Carve sizing;
    layout(sizing, qc, d3, cur);
    void *ws = nullptr;
    if ((st = workspace_get(sizing.off, &ws)) != DTW_OK) return st;
    Carve cv;
    cv.base = (char *)ws;
    layout(cv, qc, d3, cur);
    float *d = dist3 ? dist3 : d3;  // [3][N]: DTW_p(x,y), DTW_p(y,z), DTW_p(x,z)
    CUDA_TRY(cudaMemsetAsync(cur, 0, 3 * sizeof(unsigned long long), s));
    DtwJob j{};
    j.n = n;
    j.w = we;
    j.p = p;
    j.k = 1;
    j.qc = qc;
    j.npairs = N;
    j.per_pair_y = 1;
    j.fixed_thr = INFINITY;
    j.root_out = 1;
    // pairs (x_i, y_i)
    CUDA_TRY(launch_query_copies(y, N, n, qc, s));
    j.db = x;
    j.res = d;
    j.cursor = cur;
    CUDA_TRY(launch_dtw(j, g, s));
    // pairs (y_i, z_i) and (x_i, z_i) share the copies of z
    CUDA_TRY(launch_query_copies(z, N, n, qc, s));
    j.db = y;
    j.res = d + N;
    j.cursor = cur + 1;
    CUDA_TRY(launch_dtw(j, g, s));
    j.db = x;
    j.res = d + 2 * N;
    j.cursor = cur + 2;
    CUDA_TRY(launch_dtw(j, g, s));
    CUDA_TRY(launch_triangle_ratio(d, d + N, d + 2 * N, N, ratio, s));
    return DTW_OK;
}

}  // extern "C"

// knn_search_ex, with per-query thresholds from other shards of the database
// (thr_in, lowered into each query's threshold after its seeds) and/or the
// seeds' thresholds reported (thr_out); prefix_only stops after the seeds.
static dtw_status knn_run(const float *db, int64_t N, const float *queries, int64_t Q, int32_t n, int32_t w,
                          int32_t p, int32_t k, const dtw_options *opt, int64_t *out_idx, float *out_dist,
                          dtw_stats *stats, void *stream, const float *thr_in, float *thr_out, bool prefix_only) {
    g_err[0] = 0;
    dtw_status st = check_common(n, w, p);
    if (st != DTW_OK) return st;
    if ((st = check_band(n, w)) != DTW_OK) return st;
    if (N < 0 || N > INT32_MAX / 2) return fail(DTW_ERR_INVALID_ARG, "N=%lld out of range", (long long)N);
    if (Q < 0 || Q > INT32_MAX / 2) return fail(DTW_ERR_INVALID_ARG, "Q=%lld out of range", (long long)Q);
    if (k < 1 || k > DTW_MAX_K) return fail(DTW_ERR_INVALID_ARG, "k=%d outside [1, %d]", k, DTW_MAX_K);
    dtw_options o{DTW_MODE_IMPROVED, 1e-6f, 0, 0, 0, 0, 0};
    if (opt) o = *opt;
    if (o.parts < -1 || o.parts > n) return fail(DTW_ERR_INVALID_ARG, "parts=%d outside [-1, n=%d]", o.parts, n);
    if (o.mode < DTW_MODE_IMPROVED || o.mode > DTW_MODE_NOPRUNE)
        return fail(DTW_ERR_INVALID_ARG, "mode=%d unknown", o.mode);
    if (!(o.slack >= 0.0f) || std::isinf(o.slack)) return fail(DTW_ERR_INVALID_ARG, "slack must be finite and >= 0");
    if (o.seeds < 0) return fail(DTW_ERR_INVALID_ARG, "seeds=%d must be >= 0", o.seeds);
    if (o.dtw_path < 0 || o.dtw_path > 4) return fail(DTW_ERR_INVALID_ARG, "dtw_path=%d outside [0, 4]", o.dtw_path);
    if (o.filter_path < 0 || o.filter_path > 2)
        return fail(DTW_ERR_INVALID_ARG, "filter_path=%d outside [0, 2]", o.filter_path);
    if (stats) memset(stats, 0, sizeof(*stats));
    if (Q == 0) return DTW_OK;
    if (!queries || (N > 0 && !db)) return fail(DTW_ERR_INVALID_ARG, "null pointer");
    if (!prefix_only && (!out_idx || !out_dist)) return fail(DTW_ERR_INVALID_ARG, "null pointer");
    if (prefix_only && !thr_out) return fail(DTW_ERR_INVALID_ARG, "null pointer");
    cudaStream_t s = (cudaStream_t)stream;

    const CascadePlan pl = make_plan(N, Q, n, w, p, k, o);
    const bool db_dev = N == 0 || is_device_ptr(db);
    const bool q_dev = is_device_ptr(queries);
    const bool oi_dev = prefix_only || is_device_ptr(out_idx);
    const bool od_dev = prefix_only || is_device_ptr(out_dist);
    const bool ti_dev = !thr_in || is_device_ptr(thr_in);
    const bool to_dev = !thr_out || is_device_ptr(thr_out);
    const int64_t Qc = pl.Qc;

    struct Extra {
        float *db, *q, *PX, *XU, *XL, *out_dist, *thr_in, *thr_out;
        int64_t *out_idx;
        unsigned long long *counters, *xmax;
    };
    auto layout = [&](Carve &cv, Extra &x) {
        x.db = db_dev ? nullptr : cv.take<float>((size_t)N * n);
        x.q = q_dev ? nullptr : cv.take<float>((size_t)Qc * n);
        x.PX = pl.summary ? cv.take<float>((size_t)N * pl.parts) : nullptr;
        x.XU = plan_needs_db_envelope(pl) ? cv.take<float>((size_t)N * n) : nullptr;
        x.XL = plan_needs_db_envelope(pl) ? cv.take<float>((size_t)N * n) : nullptr;
        x.counters = cv.take<unsigned long long>(CNT_ALLOC);
        x.xmax = cv.take<unsigned long long>(1);
        x.out_idx = oi_dev ? nullptr : cv.take<int64_t>((size_t)Q * k);
        x.out_dist = od_dev ? nullptr : cv.take<float>((size_t)Q * k);
        x.thr_in = ti_dev ? nullptr : cv.take<float>((size_t)Q);
        x.thr_out = to_dev ? nullptr : cv.take<float>((size_t)Q);
        return carve_ws(pl, cv);
    };
    Carve sizing;
    Extra x{};
    layout(sizing, x);
    void *wsp = nullptr;
    if ((st = workspace_get(sizing.off, &wsp)) != DTW_OK) return st;
    Carve cv;
    cv.base = (char *)wsp;
    const CascadeWs ws = layout(cv, x);

    const float *dbd = db;
    if (!db_dev) {
        CUDA_TRY(cudaMemcpyAsync(x.db, db, (size_t)N * n * sizeof(float), cudaMemcpyHostToDevice, s));
        dbd = x.db;
    }
    int64_t *oidx = oi_dev ? out_idx : x.out_idx;
    float *odist = od_dev ? out_dist : x.out_dist;
    const float *tin = thr_in;
    if (!ti_dev) {
        CUDA_TRY(cudaMemcpyAsync(x.thr_in, thr_in, (size_t)Q * sizeof(float), cudaMemcpyHostToDevice, s));
        tin = x.thr_in;
    }
    float *tout = to_dev ? thr_out : x.thr_out;
    CUDA_TRY(cudaMemsetAsync(x.counters, 0, CNT_ALLOC * sizeof(unsigned long long), s));
    unsigned *xmax_bits = reinterpret_cast<unsigned *>(x.xmax);
    // part sums and row envelopes of the database, once per call
    CUDA_TRY(prepare_database(pl, dbd, x.PX, xmax_bits, x.XU, x.XL, s));
    for (int64_t q0 = 0; q0 < Q; q0 += Qc) {
        const int qn = (int)((Q - q0) < Qc ? (Q - q0) : Qc);
        const float *qd;
        if (q_dev) {
            qd = queries + q0 * n;
        } else {
            CUDA_TRY(cudaMemcpyAsync(x.q, queries + q0 * n, (size_t)qn * n * sizeof(float),
                                     cudaMemcpyHostToDevice, s));
            qd = x.q;
        }
        CUDA_TRY(cascade_run(pl, ws, dbd, x.PX, xmax_bits, x.XU, x.XL, qd, qn, oidx ? oidx + q0 * k : nullptr,
                             odist ? odist + q0 * k : nullptr, x.counters, s, tin ? tin + q0 : nullptr,
                             tout ? tout + q0 : nullptr, prefix_only));
    }
    if (!to_dev)
        CUDA_TRY(cudaMemcpyAsync(thr_out, x.thr_out, (size_t)Q * sizeof(float), cudaMemcpyDeviceToHost, s));
    if (!oi_dev)
        CUDA_TRY(cudaMemcpyAsync(out_idx, x.out_idx, (size_t)Q * k * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    if (!od_dev)
        CUDA_TRY(cudaMemcpyAsync(out_dist, x.out_dist, (size_t)Q * k * sizeof(float), cudaMemcpyDeviceToHost, s));
    if (stats || !oi_dev || !od_dev || !to_dev) {
        // a synchronising call also reports a bounded device-side wait that
        // gave up (the outputs are then not valid)
        unsigned long long h[CNT_ALLOC];
        CUDA_TRY(cudaMemcpyAsync(h, x.counters, sizeof(h), cudaMemcpyDeviceToHost, s));
        CUDA_TRY(cudaStreamSynchronize(s));
        if (h[CNT_ERR] != 0)
            return fail((dtw_status)h[CNT_ERR], "a device-side wait of the cascade gave up (status %llu)",
                        (unsigned long long)h[CNT_ERR]);
        if (stats) cascade_stats(pl, Q, h, stats);
    }
    return DTW_OK;
}

extern "C" {

dtw_status knn_search_ex(const float *db, int64_t N, const float *queries, int64_t Q, int32_t n,
                         int32_t w, int32_t p, int32_t k, const dtw_options *opt, int64_t *out_idx,
                         float *out_dist, dtw_stats *stats, void *stream) {
    return knn_run(db, N, queries, Q, n, w, p, k, opt, out_idx, out_dist, stats, stream, nullptr, nullptr, false);
}

dtw_status knn_search(const float *db, int64_t N, const float *queries, int64_t Q, int32_t n, int32_t w,
                      int32_t p, int32_t k, int64_t *out_idx, float *out_dist, dtw_stats *stats,
                      void *stream) {
    return knn_search_ex(db, N, queries, Q, n, w, p, k, nullptr, out_idx, out_dist, stats, stream);
}

dtw_status knn_seed_thresholds(const float *db, int64_t N, const float *queries, int64_t Q, int32_t n,
                               int32_t w, int32_t p, int32_t k, const dtw_options *opt, float *thr_out,
                               void *stream) {
    return knn_run(db, N, queries, Q, n, w, p, k, opt, nullptr, nullptr, nullptr, stream, nullptr, thr_out, true);
}

dtw_status knn_search_bounded(const float *db, int64_t N, const float *queries, int64_t Q, int32_t n,
                              int32_t w, int32_t p, int32_t k, const dtw_options *opt, const float *thr_in,
                              int64_t *out_idx, float *out_dist, dtw_stats *stats, void *stream) {
    if (!thr_in && Q > 0) {
        g_err[0] = 0;
        return fail(DTW_ERR_INVALID_ARG, "null pointer");
    }
    return knn_run(db, N, queries, Q, n, w, p, k, opt, out_idx, out_dist, stats, stream, thr_in, nullptr, false);
}

dtw_status knn_merge_topk(const int64_t *idx, const float *dist, int32_t R, int64_t Q, int32_t k_in, int32_t k,
                          int64_t *out_idx, float *out_dist, void *stream) {
    g_err[0] = 0;
    if (R < 1 || k_in < 1 || k < 1 || k > DTW_MAX_K || Q < 0 || Q > INT32_MAX / 2 ||
        (int64_t)R * k_in > INT32_MAX / 2)
        return fail(DTW_ERR_INVALID_ARG, "R=%d, k_in=%d, k=%d, Q=%lld out of range", R, k_in, k, (long long)Q);
    if (Q == 0) return DTW_OK;
    if (!idx || !dist || !out_idx || !out_dist) return fail(DTW_ERR_INVALID_ARG, "null pointer");
    if (!is_device_ptr(idx) || !is_device_ptr(dist) || !is_device_ptr(out_idx) || !is_device_ptr(out_dist))
        return fail(DTW_ERR_INVALID_ARG, "knn_merge_topk takes device buffers");
    CUDA_TRY(launch_merge_topk(idx, dist, R, (int)Q, k_in, k, out_idx, out_dist, (cudaStream_t)stream));
    return DTW_OK;
}

}  // extern "C"
