// Multi-length index (dtw_index_*): length buckets resident on the device,
// batched search over queries of mixed length n, band w and neighbour count k.
// A batch is split into groups of equal (n, w, k); every group is one cascade
// run (Algorithm 3 for a block of queries, cascade_host.cu) on its own stream
// of a pool, so groups of different lengths overlap on the device.  The whole
// batch (gather, fork, runs, join, scatter) can be captured once as a CUDA
// graph and replayed for later batches of the same group shapes.  An
// autotuner times the cascade parameters (piecewise-sum parts, seeds, filter
// segment length) per (n, w, k).
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "index_impl.cuh"

namespace dtwk {

void set_error_message(const char *msg);

dtw_status ix_fail(dtw_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    set_error_message(buf);
    return st;
}

#define IX_TRY(expr)                                                                       \
    do {                                                                                   \
        cudaError_t e_ = (expr);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return ix_fail(DTW_ERR_CUDA, "%s failed: %s", #expr, cudaGetErrorString(e_));  \
    } while (0)

// ---------------------------------------------------------------------------
// gather / scatter kernels
// ---------------------------------------------------------------------------
__global__ void k_gather_queries(const float *__restrict__ staged, const QMap *__restrict__ map, int64_t Q,
                                 float *__restrict__ grouped) {
    for (int64_t i = blockIdx.x; i < Q; i += gridDim.x) {
        const int64_t src = map[i].src, dst = map[i].dst;
        const int len = map[i].len;
        for (int t = threadIdx.x; t < len; t += blockDim.x) grouped[dst + t] = staged[src + t];
    }
}

__global__ void k_scatter_results(const int64_t *__restrict__ gidx, const float *__restrict__ gdist,
                                  const QMap *__restrict__ map, int64_t Q, int k_stride,
                                  int64_t *__restrict__ out_idx, float *__restrict__ out_dist) {
    const int64_t total = Q * k_stride;
    for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < total; o += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = o / k_stride;
        const int j = (int)(o - i * k_stride);
        const int kg = map[i].kg;
        if (j < kg) {
            out_idx[o] = gidx[map[i].osrc + j];
            out_dist[o] = gdist[map[i].osrc + j];
        } else {
            out_idx[o] = -1;
            out_dist[o] = kInf;
        }
    }
}

static cudaError_t launch_gather(const float *staged, const QMap *map, int64_t Q, float *grouped, cudaStream_t s) {
    if (Q <= 0) return cudaSuccess;
    const int blocks = (int)std::min<int64_t>(Q, 4 * (int64_t)device_sm_count());
    k_gather_queries<<<blocks, 128, 0, s>>>(staged, map, Q, grouped);
    return cudaGetLastError();
}

static cudaError_t launch_scatter(const int64_t *gidx, const float *gdist, const QMap *map, int64_t Q, int k_stride,
                                  int64_t *oidx, float *odist, cudaStream_t s) {
    const int64_t total = Q * k_stride;
    if (total <= 0) return cudaSuccess;
    const int blocks = (int)std::min<int64_t>((total + 255) / 256, 4 * (int64_t)device_sm_count());
    k_scatter_results<<<blocks, 256, 0, s>>>(gidx, gdist, map, Q, k_stride, oidx, odist);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// slots
// ---------------------------------------------------------------------------
dtw_status slot_init(Slot &sl, int pool_size) {
    IX_TRY(cudaStreamCreateWithFlags(&sl.origin, cudaStreamNonBlocking));
    IX_TRY(cudaEventCreateWithFlags(&sl.fork, cudaEventDisableTiming));
    IX_TRY(cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming));
    IX_TRY(cudaEventCreateWithFlags(&sl.hmap_free, cudaEventDisableTiming));
    sl.pool.resize(pool_size);
    sl.join.resize(pool_size);
    for (int i = 0; i < pool_size; ++i) {
        IX_TRY(cudaStreamCreateWithFlags(&sl.pool[i], cudaStreamNonBlocking));
        IX_TRY(cudaEventCreateWithFlags(&sl.join[i], cudaEventDisableTiming));
    }
    return DTW_OK;
}

static void slot_clear_graphs(Slot &sl) {
    for (auto &g : sl.graphs) cudaGraphExecDestroy(g.exec);
    sl.graphs.clear();
}

void slot_release(Slot &sl) {
    slot_clear_graphs(sl);
    if (sl.origin) cudaStreamSynchronize(sl.origin);
    for (auto st : sl.pool) cudaStreamSynchronize(st);
    if (sl.arena) cudaFree(sl.arena);
    if (sl.hmap) cudaFreeHost(sl.hmap);
    if (sl.hptab) cudaFreeHost(sl.hptab);
    for (auto st : sl.pool) cudaStreamDestroy(st);
    for (auto ev : sl.join) cudaEventDestroy(ev);
    if (sl.fork) cudaEventDestroy(sl.fork);
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.hmap_free) cudaEventDestroy(sl.hmap_free);
    if (sl.origin) cudaStreamDestroy(sl.origin);
    sl = Slot{};
}

// Grows the slot's arena to at least `bytes` (synchronises the device and
// drops the cached graphs, which hold arena addresses).
dtw_status slot_reserve(Slot &sl, size_t bytes) {
    if (sl.arena_cap >= bytes) return DTW_OK;
    IX_TRY(cudaDeviceSynchronize());
    slot_clear_graphs(sl);
    if (sl.arena) {
        cudaFree(sl.arena);
        sl.arena = nullptr;
        sl.arena_cap = 0;
    }
    const size_t want = bytes + bytes / 8 + (1u << 20);
    cudaError_t e = cudaMalloc(&sl.arena, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        sl.arena = nullptr;
        return ix_fail(DTW_ERR_OOM, "index arena of %zu bytes: %s", want, cudaGetErrorString(e));
    }
    sl.arena_cap = want;
    return DTW_OK;
}

static dtw_status slot_reserve_map(Slot &sl, int64_t Q) {
    if ((int64_t)sl.hmap_cap >= Q) return DTW_OK;
    IX_TRY(cudaEventSynchronize(sl.hmap_free));
    if (sl.hmap) cudaFreeHost(sl.hmap);
    sl.hmap = nullptr;
    sl.hmap_cap = 0;
    const size_t want = (size_t)std::max<int64_t>(Q, 1024);
    cudaError_t e = cudaHostAlloc((void **)&sl.hmap, want * sizeof(QMap), cudaHostAllocDefault);
    if (e != cudaSuccess) {
        cudaGetLastError();
        sl.hmap = nullptr;
        return ix_fail(DTW_ERR_OOM, "pinned query map of %zu entries: %s", want, cudaGetErrorString(e));
    }
    sl.hmap_cap = want;
    return DTW_OK;
}

static dtw_status slot_reserve_ptab(Slot &sl, size_t G) {
    if (sl.hptab_cap >= G) return DTW_OK;
    IX_TRY(cudaEventSynchronize(sl.hmap_free));
    if (sl.hptab) cudaFreeHost(sl.hptab);
    sl.hptab = nullptr;
    sl.hptab_cap = 0;
    const size_t want = std::max<size_t>(G, 64);
    cudaError_t e = cudaHostAlloc((void **)&sl.hptab, want * sizeof(PersistGroup), cudaHostAllocDefault);
    if (e != cudaSuccess) {
        cudaGetLastError();
        sl.hptab = nullptr;
        return ix_fail(DTW_ERR_OOM, "pinned group table of %zu entries: %s", want, cudaGetErrorString(e));
    }
    sl.hptab_cap = want;
    return DTW_OK;
}

// ---------------------------------------------------------------------------
// buckets and part sums
// ---------------------------------------------------------------------------
int find_bucket(const dtw_index *ix, int n) {
    for (size_t b = 0; b < ix->buckets.size(); ++b)
        if (ix->buckets[b].n == n) return (int)b;
    return -1;
}

// Part sums of bucket b for d parts (computed on first use, synchronously).
dtw_status ensure_sums(dtw_index *ix, int b, int parts, const PartSums **out) {
    Bucket &bk = ix->buckets[b];
    for (const auto &ps : bk.sums)
        if (ps.parts == parts) {
            *out = &ps;
            return DTW_OK;
        }
    PartSums ps{};
    ps.parts = parts;
    const size_t px_bytes = ((size_t)bk.N * parts * sizeof(float) + 255) & ~size_t(255);
    cudaError_t e = cudaMalloc(&ps.PX, px_bytes + 256);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return ix_fail(DTW_ERR_OOM, "part sums of %lld x %d: %s", (long long)bk.N, parts, cudaGetErrorString(e));
    }
    ps.xmax = reinterpret_cast<unsigned long long *>(reinterpret_cast<char *>(ps.PX) + px_bytes);
    cudaStream_t s = ix->slot.origin;
    IX_TRY(cudaMemsetAsync(ps.xmax, 0, sizeof(unsigned long long), s));
    IX_TRY(launch_summarize(bk.db, bk.N, bk.n, parts, ps.PX, reinterpret_cast<unsigned *>(ps.xmax), s));
    IX_TRY(cudaStreamSynchronize(s));
    bk.sums.push_back(ps);
    *out = &bk.sums.back();
    return DTW_OK;
}

// Envelopes of bucket b's rows for band w (computed on first use,
// synchronously; w already clamped to n - 1).
dtw_status ensure_env(dtw_index *ix, int b, int w, const DbEnvelope **out) {
    Bucket &bk = ix->buckets[b];
    for (const auto &ev : bk.envs)
        if (ev.w == w) {
            *out = &ev;
            return DTW_OK;
        }
    DbEnvelope ev{};
    ev.w = w;
    const size_t row_bytes = ((size_t)bk.N * bk.n * sizeof(float) + 255) & ~size_t(255);
    cudaError_t e = cudaMalloc(&ev.XU, 2 * row_bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return ix_fail(DTW_ERR_OOM, "envelopes of %lld x %d: %s", (long long)bk.N, bk.n, cudaGetErrorString(e));
    }
    ev.XL = reinterpret_cast<float *>(reinterpret_cast<char *>(ev.XU) + row_bytes);
    cudaStream_t s = ix->slot.origin;
    e = launch_envelope(bk.db, bk.N, bk.n, w, ev.XU, ev.XL, QueryCopies{}, 0, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaFree(ev.XU);
        return ix_fail(DTW_ERR_CUDA, "bucket envelopes: %s", cudaGetErrorString(e));
    }
    bk.envs.push_back(ev);
    *out = &bk.envs.back();
    return DTW_OK;
}

Tuning tuning_for(const dtw_index *ix, int n, int w, int k) {
    auto it = ix->tuned.find(TuneKey{n, w, k});
    if (it != ix->tuned.end()) return it->second;
    Tuning t{};
    t.parts = ix->opt.parts;
    t.seeds = ix->opt.seeds;
    t.seg_len = 0;
    t.ms = -1.0f;
    t.dtw_path = ix->opt.dtw_path;
    t.filter_warps = 0;
    return t;
}

CascadePlan plan_for(const dtw_index *ix, int b, int w, int k, int64_t qmax, const Tuning &t) {
    const Bucket &bk = ix->buckets[b];
    dtw_options o = ix->opt;
    o.parts = t.parts;
    o.seeds = t.seeds;
    o.dtw_path = t.dtw_path;
    return make_plan(bk.N, qmax, bk.n, w, ix->p, k, o, t.seg_len, t.filter_warps);
}

// ---------------------------------------------------------------------------
// batch layout in the slot arena
// ---------------------------------------------------------------------------
BatchLayout layout_batch(Carve &cv, int64_t Q, int64_t total, int64_t gout, int k_stride,
                         const std::vector<GroupRun> &groups, bool shared_ws) {
    BatchLayout L{};
    L.staged = cv.take<float>((size_t)std::max<int64_t>(total, 1));
    L.map = cv.take<QMap>((size_t)std::max<int64_t>(Q, 1));
    // each group's queries start on a 16-byte boundary (vector loads)
    L.grouped = cv.take<float>((size_t)std::max<int64_t>(total + 4 * (int64_t)groups.size(), 1));
    L.gidx = cv.take<int64_t>((size_t)std::max<int64_t>(gout, 1));
    L.gdist = cv.take<float>((size_t)std::max<int64_t>(gout, 1));
    L.oidx = cv.take<int64_t>((size_t)std::max<int64_t>(Q * k_stride, 1));
    L.odist = cv.take<float>((size_t)std::max<int64_t>(Q * k_stride, 1));
    L.counters = cv.take<unsigned long long>(std::max<size_t>(groups.size(), 1) * CNT_ALLOC);
    L.ptab = cv.take<PersistGroup>(std::max<size_t>(groups.size(), 1));
    L.pcursor = cv.take<unsigned long long>(1);
    L.ws.resize(groups.size());
    if (shared_ws) {
        const size_t off0 = cv.off;
        size_t end = off0;
        for (size_t g = 0; g < groups.size(); ++g) {
            cv.off = off0;
            L.ws[g] = carve_ws(groups[g].pl, cv);
            end = std::max(end, cv.off);
        }
        cv.off = end;
    } else {
        for (size_t g = 0; g < groups.size(); ++g) L.ws[g] = carve_ws(groups[g].pl, cv);
    }
    return L;
}

// ---------------------------------------------------------------------------
// batch preparation: validation, grouping, plans
// ---------------------------------------------------------------------------
dtw_status prepare_batch(dtw_index *ix, int64_t Q, const int32_t *q_len, const int32_t *q_w, const int32_t *q_k,
                         int32_t k_stride, int32_t flags, Batch &bt) {
    if (Q < 0 || Q > INT32_MAX / 2) return ix_fail(DTW_ERR_INVALID_ARG, "Q=%lld out of range", (long long)Q);
    if (k_stride < 1 || k_stride > DTW_MAX_K)
        return ix_fail(DTW_ERR_INVALID_ARG, "k_stride=%d outside [1, %d]", k_stride, DTW_MAX_K);
    if (Q > 0 && (!q_len || !q_w || !q_k)) return ix_fail(DTW_ERR_INVALID_ARG, "null pointer");
    const bool per_query = (flags & DTW_BATCH_PER_QUERY) != 0;
    bt = Batch{};
    bt.Q = Q;
    bt.k_stride = k_stride;
    bt.flags = flags;
    bt.qbucket.resize(Q);
    bt.qoff.resize(Q);
    std::map<std::array<int, 3>, int> gid;
    int64_t total = 0;
    for (int64_t i = 0; i < Q; ++i) {
        const int n = q_len[i], w = q_w[i], k = q_k[i];
        if (n < 1 || n > DTW_MAX_N) return ix_fail(DTW_ERR_INVALID_ARG, "query %lld: n=%d out of range", (long long)i, n);
        if (w < 0) return ix_fail(DTW_ERR_INVALID_ARG, "query %lld: w=%d must be >= 0", (long long)i, w);
        if (k < 1 || k > k_stride)
            return ix_fail(DTW_ERR_INVALID_ARG, "query %lld: k=%d outside [1, k_stride=%d]", (long long)i, k, k_stride);
        const int b = find_bucket(ix, n);
        if (b < 0) return ix_fail(DTW_ERR_NO_BUCKET, "query %lld: no bucket of length %d", (long long)i, n);
        const int we = w < n - 1 ? w : n - 1;
        if (2 * we + 1 > 2048)
            return ix_fail(DTW_ERR_INVALID_ARG, "query %lld: DTW band %d exceeds 2048", (long long)i, 2 * we + 1);
        bt.qbucket[i] = b;
        bt.qoff[i] = total;
        total += n;
        std::array<int, 3> key{b, we, k};
        auto it = gid.find(key);
        int g;
        if (it == gid.end()) {
            g = (int)bt.groups.size();
            gid[key] = g;
            GroupRun gr{};
            gr.bucket = b;
            gr.w = we;
            gr.k = k;
            bt.groups.push_back(gr);
        } else {
            g = it->second;
        }
        bt.groups[g].members.push_back(i);
    }
    bt.total = total;
    // heaviest groups first, so they start first on the stream pool
    std::stable_sort(bt.groups.begin(), bt.groups.end(), [&](const GroupRun &a, const GroupRun &b) {
        const Bucket &ba = ix->buckets[a.bucket], &bb = ix->buckets[b.bucket];
        const double ca = (double)a.members.size() * ba.N * ba.n * (2.0 * a.w + 1.0);
        const double cb = (double)b.members.size() * bb.N * bb.n * (2.0 * b.w + 1.0);
        return ca > cb;
    });
    int64_t qdst = 0, gout = 0;
    for (size_t g = 0; g < bt.groups.size(); ++g) {
        GroupRun &gr = bt.groups[g];
        const Bucket &bk = ix->buckets[gr.bucket];
        gr.qn = (int)gr.members.size();
        gr.t = tuning_for(ix, bk.n, gr.w, gr.k);
        gr.pl = plan_for(ix, gr.bucket, gr.w, gr.k, per_query ? 1 : gr.qn, gr.t);
        // groups that run side by side on the stream pool: seeds one thread per pair
        gr.pl.seeds_on_threads = bt.groups.size() > 1 && !per_query;
        qdst = (qdst + 3) & ~int64_t(3);
        gr.qoff = qdst;
        gr.ooff = gout;
        qdst += (int64_t)gr.qn * bk.n;
        gout += (int64_t)gr.qn * gr.k;
        gr.stream = (int)(g % ix->slot.pool.size());
    }
    bt.gout = gout;
    if (flags & DTW_BATCH_PERSISTENT) {
        if (flags & (DTW_BATCH_SERIAL | DTW_BATCH_PER_QUERY))
            return ix_fail(DTW_ERR_INVALID_ARG, "DTW_BATCH_PERSISTENT does not combine with SERIAL or PER_QUERY");
        if (ix->p != 1 && ix->p != 2)
            return ix_fail(DTW_ERR_INVALID_ARG, "DTW_BATCH_PERSISTENT needs p in {1, 2}");
        for (const auto &gr : bt.groups) {
            if (gr.pl.mode != DTW_MODE_IMPROVED)
                return ix_fail(DTW_ERR_INVALID_ARG, "DTW_BATCH_PERSISTENT needs the LB_Improved cascade mode");
            const PersistShape sh = persist_shape(gr.pl.n, gr.pl.we);
            if (sh.g == 0)
                return ix_fail(DTW_ERR_INVALID_ARG, "DTW_BATCH_PERSISTENT: band %d of n=%d exceeds 512",
                               2 * gr.pl.we + 1, gr.pl.n);
            // every query-copy index the lane groups read: column -w (row 0, slot 0)
            // up to n - 1 + w + CL (row n - 1, the top slot of the band's last lane)
            if (gr.pl.g.padl < gr.pl.we || (int64_t)gr.pl.g.padl + gr.pl.n + gr.pl.we + sh.cl > gr.pl.g.ylen)
                return ix_fail(DTW_ERR_INTERNAL, "DTW_BATCH_PERSISTENT: query copies too short for n=%d, w=%d",
                               gr.pl.n, gr.pl.we);
            if (gr.qn > gr.pl.Qc)
                return ix_fail(DTW_ERR_INVALID_ARG,
                               "DTW_BATCH_PERSISTENT: %d queries of length %d exceed one cascade run (%lld)", gr.qn,
                               gr.pl.n, (long long)gr.pl.Qc);
        }
    }
    return DTW_OK;
}

// Part sums of every group that uses the pre-filter, and the row envelopes
// of every group that computes LB_Improved (outside any capture).
dtw_status bind_sums(dtw_index *ix, Batch &bt) {
    for (auto &gr : bt.groups) {
        gr.PX = nullptr;
        gr.xmax = nullptr;
        gr.XU = nullptr;
        gr.XL = nullptr;
        if (plan_needs_db_envelope(gr.pl)) {
            const DbEnvelope *ev = nullptr;
            dtw_status st = ensure_env(ix, gr.bucket, gr.pl.we, &ev);
            if (st != DTW_OK) return st;
            gr.XU = ev->XU;
            gr.XL = ev->XL;
        }
        if (gr.pl.summary) {
            const PartSums *ps = nullptr;
            dtw_status st = ensure_sums(ix, gr.bucket, gr.pl.parts, &ps);
            if (st != DTW_OK) return st;
            gr.PX = ps->PX;
            gr.xmax = reinterpret_cast<const unsigned *>(ps->xmax);
        }
    }
    return DTW_OK;
}

void fill_map(const Batch &bt, QMap *hmap) {
    for (const auto &gr : bt.groups) {
        for (int j = 0; j < gr.qn; ++j) {
            const int64_t i = gr.members[j];
            QMap m;
            m.src = bt.qoff[i];
            m.len = gr.pl.n;
            m.dst = gr.qoff + (int64_t)j * gr.pl.n;
            m.osrc = gr.ooff + (int64_t)j * gr.k;
            m.kg = gr.k;
            hmap[i] = m;
        }
    }
}

// The persistent arm's group table (host copy), for the batch laid out as L.
// Returns the number of work items (total over the groups).
static int64_t fill_ptab(const dtw_index *ix, const Batch &bt, const BatchLayout &L, PersistGroup *tab) {
    int64_t items = 0, qbase = 0;
    for (size_t g = 0; g < bt.groups.size(); ++g) {
        const GroupRun &gr = bt.groups[g];
        const Bucket &bk = ix->buckets[gr.bucket];
        const CascadeWs &ws = L.ws[g];
        const CascadeBufs b = cascade_bufs(gr.pl, ws, bk.db, gr.XU, gr.XL, L.grouped + gr.qoff, gr.qn,
                                           L.gidx + gr.ooff, L.gdist + gr.ooff, L.counters + g * CNT_ALLOC);
        PersistGroup pg{};
        pg.db = bk.db;
        pg.XU = gr.XU;
        pg.XL = gr.XL;
        pg.queries = b.queries;
        pg.U = b.U;
        pg.L = b.L;
        pg.UL = b.UL;
        pg.LU = b.LU;
        pg.qc = b.qc;
        pg.lb = b.lb;
        pg.bsf = b.bsf;
        pg.gmin = b.gmin;
        pg.seed_pairs = b.seed_pairs;
        pg.seed_res = b.seed_res;
        pg.out_idx = b.out_idx;
        pg.out_dist = b.out_dist;
        pg.counters = b.counters;
        pg.N = (int)bk.N;
        pg.Q = gr.qn;
        pg.n = gr.pl.n;
        pg.w = gr.pl.we;
        pg.p = gr.pl.p;
        pg.k = gr.pl.k;
        pg.S = gr.pl.S;
        pg.chunk = ix->persist_chunk;
        pg.nchunks = (int)((bk.N + pg.chunk - 1) / pg.chunk);
        const PersistShape sh = persist_shape(gr.pl.n, gr.pl.we);
        pg.dg = sh.g;
        pg.cl = sh.cl;
        pg.vec = (gr.pl.n % 4 == 0) && ((reinterpret_cast<uintptr_t>(bk.db) & 15) == 0) &&
                 ((reinterpret_cast<uintptr_t>(b.queries) & 15) == 0);
        pg.summary = gr.pl.summary ? 1 : 0;
        pg.slack = gr.pl.slack;
        pg.summary_scale = b.summary_scale;
        pg.item0 = items;
        pg.qbase = qbase;
        items += (int64_t)pg.Q * pg.nchunks;
        qbase += pg.Q;
        tab[g] = pg;
    }
    return items;
}

// Persistent arm: each group's first stages on the pool streams, then one
// persistent launch over every group's (query, candidate chunk) items and
// one launch for every query's top-k, then the scatter to batch order.
static cudaError_t enqueue_batch_persistent(dtw_index *ix, Slot &sl, const Batch &bt, const BatchLayout &L,
                                            cudaStream_t s, int64_t items) {
    const size_t G = bt.groups.size();
    cudaError_t e;
    if ((e = cudaMemsetAsync(L.counters, 0, std::max<size_t>(G, 1) * CNT_ALLOC * sizeof(unsigned long long), s)) !=
        cudaSuccess)
        return e;
    if ((e = cudaMemsetAsync(L.pcursor, 0, sizeof(unsigned long long), s)) != cudaSuccess) return e;
    if ((e = launch_gather(L.staged, L.map, bt.Q, L.grouped, s)) != cudaSuccess) return e;
    std::vector<char> used(sl.pool.size(), 0);
    if ((e = cudaEventRecord(sl.fork, s)) != cudaSuccess) return e;
    for (const auto &gr : bt.groups) used[gr.stream] = 1;
    for (size_t i = 0; i < sl.pool.size(); ++i)
        if (used[i] && (e = cudaStreamWaitEvent(sl.pool[i], sl.fork, 0)) != cudaSuccess) return e;
    int64_t queries = 0;
    for (size_t g = 0; g < G; ++g) {
        const GroupRun &gr = bt.groups[g];
        const Bucket &bk = ix->buckets[gr.bucket];
        const CascadeBufs b = cascade_bufs(gr.pl, L.ws[g], bk.db, gr.XU, gr.XL, L.grouped + gr.qoff, gr.qn,
                                           L.gidx + gr.ooff, L.gdist + gr.ooff, L.counters + g * CNT_ALLOC);
        if ((e = cascade_prefix(gr.pl, L.ws[g], b, gr.PX, gr.xmax, sl.pool[gr.stream])) != cudaSuccess) return e;
        queries += gr.qn;
    }
    for (size_t i = 0; i < sl.pool.size(); ++i) {
        if (!used[i]) continue;
        if ((e = cudaEventRecord(sl.join[i], sl.pool[i])) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(s, sl.join[i], 0)) != cudaSuccess) return e;
    }
    if ((e = launch_persistent(L.ptab, (int)G, items, queries, ix->p, L.pcursor, s)) != cudaSuccess) return e;
    return launch_scatter(L.gidx, L.gdist, L.map, bt.Q, bt.k_stride, L.oidx, L.odist, s);
}

// The device work of one batch, from the staged queries and map to the
// scattered outputs, enqueued on `s` (and the pool, forked from s).
static cudaError_t enqueue_batch(dtw_index *ix, Slot &sl, const Batch &bt, const BatchLayout &L, cudaStream_t s,
                                 int64_t items) {
    if (bt.flags & DTW_BATCH_PERSISTENT) return enqueue_batch_persistent(ix, sl, bt, L, s, items);
    const size_t G = bt.groups.size();
    const bool per_query = (bt.flags & DTW_BATCH_PER_QUERY) != 0;
    const bool serial = per_query || (bt.flags & DTW_BATCH_SERIAL) != 0;
    cudaError_t e;
    if ((e = cudaMemsetAsync(L.counters, 0, std::max<size_t>(G, 1) * CNT_ALLOC * sizeof(unsigned long long), s)) !=
        cudaSuccess)
        return e;
    if ((e = launch_gather(L.staged, L.map, bt.Q, L.grouped, s)) != cudaSuccess) return e;
    std::vector<char> used(sl.pool.size(), 0);
    if (!serial) {
        if ((e = cudaEventRecord(sl.fork, s)) != cudaSuccess) return e;
        for (const auto &gr : bt.groups) used[gr.stream] = 1;
        for (size_t i = 0; i < sl.pool.size(); ++i)
            if (used[i] && (e = cudaStreamWaitEvent(sl.pool[i], sl.fork, 0)) != cudaSuccess) return e;
    }
    for (size_t g = 0; g < G; ++g) {
        const GroupRun &gr = bt.groups[g];
        const Bucket &bk = ix->buckets[gr.bucket];
        cudaStream_t gs = serial ? s : sl.pool[gr.stream];
        unsigned long long *cnt = L.counters + g * CNT_ALLOC;
        const int64_t step = per_query ? 1 : gr.pl.Qc;
        for (int64_t q0 = 0; q0 < gr.qn; q0 += step) {
            const int qn = (int)std::min<int64_t>(step, gr.qn - q0);
            e = cascade_run(gr.pl, L.ws[g], bk.db, gr.PX, gr.xmax, gr.XU, gr.XL, L.grouped + gr.qoff + q0 * bk.n,
                            qn, L.gidx + gr.ooff + q0 * gr.k, L.gdist + gr.ooff + q0 * gr.k, cnt, gs);
            if (e != cudaSuccess) return e;
        }
    }
    if (!serial) {
        for (size_t i = 0; i < sl.pool.size(); ++i) {
            if (!used[i]) continue;
            if ((e = cudaEventRecord(sl.join[i], sl.pool[i])) != cudaSuccess) return e;
            if ((e = cudaStreamWaitEvent(s, sl.join[i], 0)) != cudaSuccess) return e;
        }
    }
    return launch_scatter(L.gidx, L.gdist, L.map, bt.Q, bt.k_stride, L.oidx, L.odist, s);
}

static std::vector<int64_t> graph_key(const dtw_index *ix, const Batch &bt) {
    std::vector<int64_t> key{bt.Q, bt.k_stride, bt.total, bt.flags, (int64_t)bt.groups.size(), ix->persist_chunk};
    for (const auto &gr : bt.groups) {
        key.insert(key.end(),
                   {gr.bucket, gr.w, gr.k, gr.qn, gr.pl.parts, gr.pl.S, gr.pl.seg_len, gr.pl.dtw_path,
                    gr.pl.filter_warps, gr.stream});
    }
    return key;
}

// Runs a prepared batch on slot sl: stages the queries and the map, runs the
// device work (replaying or capturing a graph when DTW_BATCH_GRAPH is set)
// and copies the outputs.  Asynchronous on s unless outputs are host memory.
dtw_status run_batch(dtw_index *ix, Slot &sl, Batch &bt, const float *queries, bool q_dev, int64_t *out_idx,
                     float *out_dist, bool out_dev, cudaStream_t s, unsigned long long *counters_host) {
    dtw_status st;
    if ((st = bind_sums(ix, bt)) != DTW_OK) return st;
    const bool per_query = (bt.flags & DTW_BATCH_PER_QUERY) != 0;
    Carve sizing;
    layout_batch(sizing, bt.Q, bt.total, bt.gout, bt.k_stride, bt.groups, per_query);
    if ((st = slot_reserve(sl, sizing.off)) != DTW_OK) return st;
    if ((st = slot_reserve_map(sl, bt.Q)) != DTW_OK) return st;
    const bool persistent = (bt.flags & DTW_BATCH_PERSISTENT) != 0;
    if (persistent && (st = slot_reserve_ptab(sl, bt.groups.size())) != DTW_OK) return st;
    Carve cv;
    cv.base = sl.arena;
    const BatchLayout L = layout_batch(cv, bt.Q, bt.total, bt.gout, bt.k_stride, bt.groups, per_query);

    // the previous batch of this slot may still read the map and arena
    IX_TRY(cudaStreamWaitEvent(s, sl.done, 0));
    IX_TRY(cudaEventSynchronize(sl.hmap_free));
    fill_map(bt, sl.hmap);
    if (bt.total > 0)
        IX_TRY(cudaMemcpyAsync(L.staged, queries, (size_t)bt.total * sizeof(float),
                               q_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    IX_TRY(cudaMemcpyAsync(L.map, sl.hmap, (size_t)bt.Q * sizeof(QMap), cudaMemcpyHostToDevice, s));
    int64_t items = 0;
    if (persistent) {
        items = fill_ptab(ix, bt, L, sl.hptab);
        IX_TRY(cudaMemcpyAsync(L.ptab, sl.hptab, bt.groups.size() * sizeof(PersistGroup), cudaMemcpyHostToDevice, s));
    }
    IX_TRY(cudaEventRecord(sl.hmap_free, s));

    const bool use_graph = (bt.flags & DTW_BATCH_GRAPH) != 0 && !per_query;
    if (use_graph) {
        const std::vector<int64_t> key = graph_key(ix, bt);
        GraphEntry *hit = nullptr;
        for (auto &g : sl.graphs)
            if (g.key == key) hit = &g;
        if (!hit) {
            // capture on the slot's own stream; the graph is launched on s
            IX_TRY(cudaStreamBeginCapture(sl.origin, cudaStreamCaptureModeRelaxed));
            cudaError_t e = enqueue_batch(ix, sl, bt, L, sl.origin, items);
            cudaGraph_t graph = nullptr;
            cudaError_t e2 = cudaStreamEndCapture(sl.origin, &graph);
            if (e != cudaSuccess || e2 != cudaSuccess) {
                if (graph) cudaGraphDestroy(graph);
                cudaGetLastError();
                return ix_fail(DTW_ERR_CUDA, "graph capture: %s",
                               cudaGetErrorString(e != cudaSuccess ? e : e2));
            }
            cudaGraphExec_t exec = nullptr;
            e = cudaGraphInstantiate(&exec, graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) return ix_fail(DTW_ERR_CUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
            if (sl.graphs.size() >= 16) {
                auto lru = std::min_element(sl.graphs.begin(), sl.graphs.end(),
                                            [](const GraphEntry &a, const GraphEntry &b) { return a.last_use < b.last_use; });
                cudaGraphExecDestroy(lru->exec);
                sl.graphs.erase(lru);
            }
            sl.graphs.push_back(GraphEntry{key, exec, 0});
            hit = &sl.graphs.back();
            ++sl.captures;
        }
        hit->last_use = ++sl.tick;
        IX_TRY(cudaGraphLaunch(hit->exec, s));
        ++sl.replays;
    } else {
        cudaError_t e = enqueue_batch(ix, sl, bt, L, s, items);
        if (e != cudaSuccess) return ix_fail(DTW_ERR_CUDA, "batch launch: %s", cudaGetErrorString(e));
    }
    if (bt.Q > 0) {
        const cudaMemcpyKind kind = out_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        IX_TRY(cudaMemcpyAsync(out_idx, L.oidx, (size_t)bt.Q * bt.k_stride * sizeof(int64_t), kind, s));
        IX_TRY(cudaMemcpyAsync(out_dist, L.odist, (size_t)bt.Q * bt.k_stride * sizeof(float), kind, s));
    }
    if (counters_host)
        IX_TRY(cudaMemcpyAsync(counters_host, L.counters, bt.groups.size() * CNT_ALLOC * sizeof(unsigned long long),
                               cudaMemcpyDeviceToHost, s));
    IX_TRY(cudaEventRecord(sl.done, s));
    return DTW_OK;
}

size_t batch_bytes(const Batch &bt) {
    Carve sizing;
    layout_batch(sizing, bt.Q, bt.total, bt.gout, bt.k_stride, bt.groups, (bt.flags & DTW_BATCH_PER_QUERY) != 0);
    return sizing.off;
}

// ---------------------------------------------------------------------------
// autotuner
// ---------------------------------------------------------------------------
// Times candidate parameter sets on `qn` queries (device) of bucket b and
// keeps the fastest.  The result of the search does not depend on the
// parameters (the cascade is exact); only its speed does.  Coordinate descent:
// parts, then seeds, then the filter segment length, then the DTW kernel
// (thread or warp per pair, or thread per pair in row phases), then the
// filter's warps per CTA, each with the others at their best so far.
dtw_status tune_group(dtw_index *ix, int b, int w, int k, const float *qdev, int qn, Tuning *out) {
    const Bucket &bk = ix->buckets[b];
    const int n = bk.n;
    const int we = w < n - 1 ? w : n - 1;
    cudaStream_t s = ix->slot.origin;
    std::vector<int> parts_c{-1};
    for (int div : {32, 16, 8, 4}) {
        const int d = n / div;
        if (d >= 4 && std::find(parts_c.begin(), parts_c.end(), d) == parts_c.end()) parts_c.push_back(d);
    }
    std::vector<int> seeds_c;
    for (int sd : {std::max(k, 4), 8, 16, 32})
        if (sd >= k && sd <= 32 && std::find(seeds_c.begin(), seeds_c.end(), sd) == seeds_c.end()) seeds_c.push_back(sd);
    const std::vector<int> seg_c{512, 1024, 2048, 4096};
    std::vector<int> path_c{1};
    if (dtw_lanes_cl(n, we) > 0) {
        path_c.push_back(2);
        if (2 * we + 1 <= 512) path_c.push_back(3);
    }
    // row phases only for the bands of up to 64 slots: wider ones measured
    // slower in phases
    if (n > 2 * kDtwPhaseRows && 2 * we + 1 <= kDtwGroupMaxC) path_c.push_back(4);
    const std::vector<int> fw_c{0, 4, 5, 6, 7, 8};

    // scratch sized for the largest candidate plan
    size_t ws_max = 0;
    for (int pc : parts_c)
        for (int sd : seeds_c)
            for (int sg : seg_c)
                for (int dp : {0, 4}) {
                    Tuning t{pc, sd, sg, 0.0f, dp, 0};
                    ws_max = std::max(ws_max, cascade_ws_bytes(plan_for(ix, b, we, k, qn, t)));
                }
    Carve cv0;
    cv0.take<int64_t>((size_t)qn * k);
    cv0.take<float>((size_t)qn * k);
    cv0.take<unsigned long long>(CNT_ALLOC);
    const size_t head = cv0.off;
    char *buf = nullptr;
    cudaError_t e = cudaMalloc(&buf, head + ws_max);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return ix_fail(DTW_ERR_OOM, "autotuner scratch of %zu bytes: %s", head + ws_max, cudaGetErrorString(e));
    }
    Carve cv;
    cv.base = buf;
    int64_t *oidx = cv.take<int64_t>((size_t)qn * k);
    float *odist = cv.take<float>((size_t)qn * k);
    unsigned long long *cnt = cv.take<unsigned long long>(CNT_ALLOC);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    dtw_status st = DTW_OK;

    auto time_one = [&](const Tuning &t, float *ms) -> dtw_status {
        const CascadePlan pl = plan_for(ix, b, we, k, qn, t);
        const float *PX = nullptr;
        const unsigned *xm = nullptr;
        if (pl.summary) {
            const PartSums *ps = nullptr;
            dtw_status s2 = ensure_sums(ix, b, pl.parts, &ps);
            if (s2 != DTW_OK) return s2;
            PX = ps->PX;
            xm = reinterpret_cast<const unsigned *>(ps->xmax);
        }
        const float *XU = nullptr, *XL = nullptr;
        if (plan_needs_db_envelope(pl)) {
            const DbEnvelope *ev = nullptr;
            dtw_status s2 = ensure_env(ix, b, pl.we, &ev);
            if (s2 != DTW_OK) return s2;
            XU = ev->XU;
            XL = ev->XL;
        }
        Carve c2;
        c2.base = buf + head;
        const CascadeWs ws = carve_ws(pl, c2);
        float best = INFINITY;
        for (int rep = 0; rep < 3; ++rep) {
            IX_TRY(cudaEventRecord(e0, s));
            for (int64_t q0 = 0; q0 < qn; q0 += pl.Qc) {
                const int m = (int)std::min<int64_t>(pl.Qc, qn - q0);
                IX_TRY(cascade_run(pl, ws, bk.db, PX, xm, XU, XL, qdev + q0 * n, m, oidx + q0 * k, odist + q0 * k,
                                   cnt, s));
            }
            IX_TRY(cudaEventRecord(e1, s));
            IX_TRY(cudaEventSynchronize(e1));
            float t_ms = 0.0f;
            IX_TRY(cudaEventElapsedTime(&t_ms, e0, e1));
            if (rep > 0) best = std::min(best, t_ms);  // rep 0 warms up
        }
        *ms = best;
        return DTW_OK;
    };

    Tuning best = tuning_for(ix, n, we, k);
    best.parts = ix->opt.parts == 0 ? (n >= 64 ? n / 8 : -1) : ix->opt.parts;
    best.seeds = ix->opt.seeds > 0 ? ix->opt.seeds : 16;
    best.seg_len = 0;
    best.dtw_path = ix->opt.dtw_path;
    best.filter_warps = 0;
    float best_ms = INFINITY;
    if ((st = time_one(best, &best_ms)) != DTW_OK) goto done;
    for (int axis = 0; axis < 5; ++axis) {
        const std::vector<int> &cands =
            axis == 0 ? parts_c : axis == 1 ? seeds_c : axis == 2 ? seg_c : axis == 3 ? path_c : fw_c;
        for (int v : cands) {
            Tuning t = best;
            if (axis == 0) t.parts = v;
            if (axis == 1) t.seeds = v;
            if (axis == 2) t.seg_len = v;
            if (axis == 3) t.dtw_path = v;
            if (axis == 4) t.filter_warps = v;
            if (t.parts == best.parts && t.seeds == best.seeds && t.seg_len == best.seg_len &&
                t.dtw_path == best.dtw_path && t.filter_warps == best.filter_warps)
                continue;
            float ms = INFINITY;
            if ((st = time_one(t, &ms)) != DTW_OK) goto done;
            if (ms < best_ms) {
                best_ms = ms;
                best = t;
            }
        }
    }
    best.ms = best_ms;
    ix->tuned[TuneKey{n, we, k}] = best;
    if (out) *out = best;
done:
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamSynchronize(s);
    cudaFree(buf);
    return st;
}

// Autotunes every group of the batch whose (n, w, k) has no tuning yet, on
// up to 256 of its own queries (copied to the device).
static dtw_status autotune_batch(dtw_index *ix, const Batch &bt, const float *queries, bool q_dev) {
    for (const auto &gr : bt.groups) {
        const Bucket &bk = ix->buckets[gr.bucket];
        if (ix->tuned.count(TuneKey{bk.n, gr.w, gr.k})) continue;
        const int m = std::min(gr.qn, 256);
        float *qd = nullptr;
        IX_TRY(cudaMalloc(&qd, (size_t)m * bk.n * sizeof(float)));
        dtw_status st = DTW_OK;
        for (int j = 0; j < m && st == DTW_OK; ++j) {
            cudaError_t e = cudaMemcpyAsync(qd + (size_t)j * bk.n, queries + bt.qoff[gr.members[j]],
                                            (size_t)bk.n * sizeof(float),
                                            q_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, ix->slot.origin);
            if (e != cudaSuccess) st = ix_fail(DTW_ERR_CUDA, "autotune copy: %s", cudaGetErrorString(e));
        }
        if (st == DTW_OK) st = tune_group(ix, gr.bucket, gr.w, gr.k, qd, m, nullptr);
        cudaStreamSynchronize(ix->slot.origin);
        cudaFree(qd);
        if (st != DTW_OK) return st;
    }
    return DTW_OK;
}

// Times the persistent arm on the batch itself for candidate chunk lengths
// (work items of 512 to 4096 candidates) and keeps the fastest for the index.
// Outputs go to a scratch area of the arena; synchronous.
static dtw_status tune_persist_chunk(dtw_index *ix, Batch &bt, const float *queries, bool q_dev, cudaStream_t s) {
    const int keep = ix->persist_chunk;
    const int flags = bt.flags;
    bt.flags &= ~DTW_BATCH_GRAPH;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    IX_TRY(cudaEventCreate(&e0));
    IX_TRY(cudaEventCreate(&e1));
    int64_t *oi = nullptr;
    float *od = nullptr;
    dtw_status st = DTW_OK;
    cudaError_t ce = cudaMalloc(&oi, (size_t)bt.Q * bt.k_stride * (sizeof(int64_t) + sizeof(float)));
    if (ce != cudaSuccess) {
        cudaGetLastError();
        st = ix_fail(DTW_ERR_OOM, "persistent tuning outputs: %s", cudaGetErrorString(ce));
    }
    od = reinterpret_cast<float *>(oi + bt.Q * bt.k_stride);
    float best_ms = INFINITY;
    int best = keep;
    for (int chunk : {512, 1024, 2048, 4096}) {
        if (st != DTW_OK) break;
        ix->persist_chunk = chunk;
        float ms = INFINITY;
        for (int rep = 0; rep < 3 && st == DTW_OK; ++rep) {
            if (cudaEventRecord(e0, s) != cudaSuccess) st = ix_fail(DTW_ERR_CUDA, "event record failed");
            if (st == DTW_OK) st = run_batch(ix, ix->slot, bt, queries, q_dev, oi, od, true, s, nullptr);
            if (st == DTW_OK && (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess))
                st = ix_fail(DTW_ERR_CUDA, "persistent tuning: %s", cudaGetErrorString(cudaGetLastError()));
            float t = 0.0f;
            if (st == DTW_OK && cudaEventElapsedTime(&t, e0, e1) == cudaSuccess && rep > 0) ms = std::min(ms, t);
        }
        if (st == DTW_OK && ms < best_ms) {
            best_ms = ms;
            best = chunk;
        }
    }
    cudaStreamSynchronize(s);
    if (oi) cudaFree(oi);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    bt.flags = flags;
    ix->persist_chunk = st == DTW_OK ? best : keep;
    if (st == DTW_OK) ix->persist_tuned = true;
    return st;
}

bool ptr_on_device(const void *p) {
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

void batch_stats(const Batch &bt, const unsigned long long *h, dtw_stats *st) {
    memset(st, 0, sizeof(*st));
    for (size_t g = 0; g < bt.groups.size(); ++g)
        cascade_stats(bt.groups[g].pl, bt.groups[g].qn, h + g * CNT_ALLOC, st);
}

}  // namespace dtwk

using namespace dtwk;

namespace {
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};
}  // namespace

extern "C" {

dtw_status dtw_index_create(int32_t p, const dtw_options *opt, dtw_index **out) {
    set_error_message("");
    if (!out) return ix_fail(DTW_ERR_INVALID_ARG, "null pointer");
    *out = nullptr;
    if (p != 1 && p != 2) return ix_fail(DTW_ERR_INVALID_ARG, "p=%d must be 1 or 2", p);
    dtw_options o{DTW_MODE_IMPROVED, 1e-6f, 0, 0, 0, 0, 0};
    if (opt) o = *opt;
    if (o.mode < DTW_MODE_IMPROVED || o.mode > DTW_MODE_NOPRUNE)
        return ix_fail(DTW_ERR_INVALID_ARG, "mode=%d unknown", o.mode);
    if (!(o.slack >= 0.0f) || std::isinf(o.slack)) return ix_fail(DTW_ERR_INVALID_ARG, "slack must be finite and >= 0");
    if (o.seeds < 0) return ix_fail(DTW_ERR_INVALID_ARG, "seeds=%d must be >= 0", o.seeds);
    if (o.parts < -1) return ix_fail(DTW_ERR_INVALID_ARG, "parts=%d must be >= -1", o.parts);
    if (o.dtw_path < 0 || o.dtw_path > 4) return ix_fail(DTW_ERR_INVALID_ARG, "dtw_path=%d outside [0, 4]", o.dtw_path);
    if (o.filter_path < 0 || o.filter_path > 2)
        return ix_fail(DTW_ERR_INVALID_ARG, "filter_path=%d outside [0, 2]", o.filter_path);
    auto *ix = new dtw_index();
    ix->p = p;
    ix->opt = o;
    if (cudaGetDevice(&ix->device) != cudaSuccess) {
        cudaGetLastError();
        delete ix;
        return ix_fail(DTW_ERR_CUDA, "no CUDA device");
    }
    dtw_status st = slot_init(ix->slot, 16);
    if (st != DTW_OK) {
        slot_release(ix->slot);
        delete ix;
        return st;
    }
    *out = ix;
    return DTW_OK;
}

dtw_status dtw_index_add_bucket(dtw_index *ix, const float *db, int64_t N, int32_t n) {
    set_error_message("");
    if (!ix || !db) return ix_fail(DTW_ERR_INVALID_ARG, "null pointer");
    if (n < 1 || n > DTW_MAX_N) return ix_fail(DTW_ERR_INVALID_ARG, "n=%d outside [1, %d]", n, DTW_MAX_N);
    if (N < 1 || N > INT32_MAX / 2) return ix_fail(DTW_ERR_INVALID_ARG, "N=%lld out of range", (long long)N);
    std::lock_guard<std::mutex> lk(ix->mu);
    DeviceGuard dg(ix->device);
    if (find_bucket(ix, n) >= 0) return ix_fail(DTW_ERR_INVALID_ARG, "a bucket of length %d exists", n);
    Bucket bk{};
    bk.n = n;
    bk.N = N;
    cudaError_t e = cudaMalloc(&bk.db, (size_t)N * n * sizeof(float));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return ix_fail(DTW_ERR_OOM, "bucket of %lld x %d: %s", (long long)N, n, cudaGetErrorString(e));
    }
    e = cudaMemcpyAsync(bk.db, db, (size_t)N * n * sizeof(float), cudaMemcpyDefault, ix->slot.origin);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ix->slot.origin);
    if (e != cudaSuccess) {
        cudaFree(bk.db);
        return ix_fail(DTW_ERR_CUDA, "bucket copy: %s", cudaGetErrorString(e));
    }
    ix->buckets.push_back(bk);
    // part sums for the default pre-filter
    const int parts = ix->opt.parts == 0 ? (n >= 64 ? n / 8 : -1) : std::min<int>(ix->opt.parts, n);
    if (parts > 0) {
        const PartSums *ps = nullptr;
        dtw_status st = ensure_sums(ix, (int)ix->buckets.size() - 1, parts, &ps);
        if (st != DTW_OK) return st;
    }
    // row envelopes for the usual band w = floor(n / 10)
    if (ix->opt.mode == DTW_MODE_IMPROVED) {
        const DbEnvelope *ev = nullptr;
        dtw_status st = ensure_env(ix, (int)ix->buckets.size() - 1, std::min(n / 10, n - 1), &ev);
        if (st != DTW_OK) return st;
    }
    return DTW_OK;
}

dtw_status dtw_index_tune(dtw_index *ix, const float *sample, int64_t count, int32_t n, int32_t w, int32_t k,
                          dtw_tuning *out) {
    set_error_message("");
    if (!ix || !sample) return ix_fail(DTW_ERR_INVALID_ARG, "null pointer");
    if (count < 1 || count > 32768) return ix_fail(DTW_ERR_INVALID_ARG, "count=%lld outside [1, 32768]", (long long)count);
    if (w < 0) return ix_fail(DTW_ERR_INVALID_ARG, "w=%d must be >= 0", w);
    if (k < 1 || k > DTW_MAX_K) return ix_fail(DTW_ERR_INVALID_ARG, "k=%d outside [1, %d]", k, DTW_MAX_K);
    std::lock_guard<std::mutex> lk(ix->mu);
    DeviceGuard dg(ix->device);
    const int b = find_bucket(ix, n);
    if (b < 0) return ix_fail(DTW_ERR_NO_BUCKET, "no bucket of length %d", n);
    const int we = w < n - 1 ? w : n - 1;
    if (2 * we + 1 > 2048) return ix_fail(DTW_ERR_INVALID_ARG, "DTW band %d exceeds 2048", 2 * we + 1);
    float *qd = nullptr;
    IX_TRY(cudaMalloc(&qd, (size_t)count * n * sizeof(float)));
    cudaError_t e = cudaMemcpyAsync(qd, sample, (size_t)count * n * sizeof(float), cudaMemcpyDefault, ix->slot.origin);
    dtw_status st = e == cudaSuccess ? DTW_OK : ix_fail(DTW_ERR_CUDA, "sample copy: %s", cudaGetErrorString(e));
    Tuning t{};
    if (st == DTW_OK) st = tune_group(ix, b, we, k, qd, (int)count, &t);
    cudaStreamSynchronize(ix->slot.origin);
    cudaFree(qd);
    if (st == DTW_OK && out) {
        out->parts = t.parts;
        out->seeds = t.seeds;
        out->seg_len = t.seg_len;
        out->ms = t.ms;
        out->dtw_path = t.dtw_path;
        out->filter_warps = t.filter_warps;
    }
    return st;
}

dtw_status dtw_index_get_tuning(dtw_index *ix, int32_t n, int32_t w, int32_t k, dtw_tuning *out) {
    set_error_message("");
    if (!ix || !out) return ix_fail(DTW_ERR_INVALID_ARG, "null pointer");
    std::lock_guard<std::mutex> lk(ix->mu);
    if (find_bucket(ix, n) < 0) return ix_fail(DTW_ERR_NO_BUCKET, "no bucket of length %d", n);
    const int we = w < n - 1 ? w : n - 1;
    const Tuning t = tuning_for(ix, n, we, k);
    out->parts = t.parts;
    out->seeds = t.seeds;
    out->seg_len = t.seg_len;
    out->ms = t.ms;
    out->dtw_path = t.dtw_path;
    out->filter_warps = t.filter_warps;
    return DTW_OK;
}

dtw_status dtw_index_set_tuning(dtw_index *ix, int32_t n, int32_t w, int32_t k, const dtw_tuning *t) {
    set_error_message("");
    if (!ix || !t) return ix_fail(DTW_ERR_INVALID_ARG, "null pointer");
    if (t->parts < -1 || t->parts > n || t->seeds < 0 || t->seeds > 32 ||
        (t->seg_len != 0 && t->seg_len != 512 && t->seg_len != 1024 && t->seg_len != 2048 && t->seg_len != 4096) ||
        t->dtw_path < 0 ||
        t->dtw_path > 4 ||
        t->filter_warps < 0 || t->filter_warps > 8)
        return ix_fail(DTW_ERR_INVALID_ARG, "tuning out of range (parts in [-1, n], seeds in [0, 32], seg_len "
                                            "0/512/1024/2048/4096, dtw_path 0-4, filter_warps 0-8)");
    if (w < 0 || k < 1 || k > DTW_MAX_K) return ix_fail(DTW_ERR_INVALID_ARG, "w or k out of range");
    std::lock_guard<std::mutex> lk(ix->mu);
    if (find_bucket(ix, n) < 0) return ix_fail(DTW_ERR_NO_BUCKET, "no bucket of length %d", n);
    const int we = w < n - 1 ? w : n - 1;
    ix->tuned[TuneKey{n, we, k}] = Tuning{t->parts, t->seeds, t->seg_len, t->ms, t->dtw_path, t->filter_warps};
    return DTW_OK;
}

dtw_status dtw_index_search(dtw_index *ix, const float *queries, int64_t Q, const int32_t *q_len, const int32_t *q_w,
                            const int32_t *q_k, int32_t k_stride, int32_t flags, int64_t *out_idx, float *out_dist,
                            dtw_stats *stats, void *stream) {
    set_error_message("");
    if (!ix) return ix_fail(DTW_ERR_INVALID_ARG, "null pointer");
    if (flags & ~(DTW_BATCH_GRAPH | DTW_BATCH_AUTOTUNE | DTW_BATCH_SERIAL | DTW_BATCH_PER_QUERY |
                  DTW_BATCH_PERSISTENT))
        return ix_fail(DTW_ERR_INVALID_ARG, "flags=0x%x has unknown bits", flags);
    std::lock_guard<std::mutex> lk(ix->mu);
    DeviceGuard dg(ix->device);
    Batch bt;
    dtw_status st = prepare_batch(ix, Q, q_len, q_w, q_k, k_stride, flags, bt);
    if (st != DTW_OK) return st;
    if (stats) memset(stats, 0, sizeof(*stats));
    if (Q == 0) return DTW_OK;
    if (!queries || !out_idx || !out_dist) return ix_fail(DTW_ERR_INVALID_ARG, "null pointer");
    const bool q_dev = ptr_on_device(queries);
    const bool oi_dev = ptr_on_device(out_idx), od_dev = ptr_on_device(out_dist);
    if (oi_dev != od_dev) return ix_fail(DTW_ERR_INVALID_ARG, "out_idx and out_dist must both be host or both device memory");
    cudaStream_t s = (cudaStream_t)stream;
    if (flags & DTW_BATCH_AUTOTUNE) {
        if ((st = autotune_batch(ix, bt, queries, q_dev)) != DTW_OK) return st;
        Batch again;
        if ((st = prepare_batch(ix, Q, q_len, q_w, q_k, k_stride, flags, again)) != DTW_OK) return st;
        bt = std::move(again);
        if ((flags & DTW_BATCH_PERSISTENT) && !ix->persist_tuned) {
            if ((st = tune_persist_chunk(ix, bt, queries, q_dev, s)) != DTW_OK) return st;
            if ((st = prepare_batch(ix, Q, q_len, q_w, q_k, k_stride, flags, again)) != DTW_OK) return st;
            bt = std::move(again);
        }
    }
    std::vector<unsigned long long> h;
    if (stats) h.assign(bt.groups.size() * CNT_ALLOC, 0);
    if ((st = run_batch(ix, ix->slot, bt, queries, q_dev, out_idx, out_dist, oi_dev, s, stats ? h.data() : nullptr)) !=
        DTW_OK)
        return st;
    if (stats || !oi_dev) IX_TRY(cudaStreamSynchronize(s));
    if (stats) batch_stats(bt, h.data(), stats);
    return DTW_OK;
}

dtw_status dtw_index_info(dtw_index *ix, dtw_index_stats *out) {
    set_error_message("");
    if (!ix || !out) return ix_fail(DTW_ERR_INVALID_ARG, "null pointer");
    std::lock_guard<std::mutex> lk(ix->mu);
    memset(out, 0, sizeof(*out));
    out->buckets = (int32_t)ix->buckets.size();
    for (const auto &bk : ix->buckets) {
        out->resident_bytes += (int64_t)bk.N * bk.n * sizeof(float);
        for (const auto &ps : bk.sums) out->resident_bytes += (int64_t)bk.N * ps.parts * sizeof(float);
    }
    out->arena_bytes = (int64_t)ix->slot.arena_cap;
    out->graphs_cached = (int32_t)ix->slot.graphs.size();
    out->graph_captures = ix->slot.captures;
    out->graph_replays = ix->slot.replays;
    return DTW_OK;
}

dtw_status dtw_index_destroy(dtw_index *ix) {
    set_error_message("");
    if (!ix) return DTW_OK;
    {
        std::lock_guard<std::mutex> lk(ix->mu);
        DeviceGuard dg(ix->device);
        slot_release(ix->slot);
        for (auto &bk : ix->buckets) {
            for (auto &ps : bk.sums) cudaFree(ps.PX);
            for (auto &ev : bk.envs) cudaFree(ev.XU);
            cudaFree(bk.db);
        }
        ix->buckets.clear();
    }
    delete ix;
    return DTW_OK;
}

}  // extern "C"
