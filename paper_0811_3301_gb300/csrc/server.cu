// Request server (dtw_server_*): continuous batching of k-NN queries over a
// multi-length index.  Requests arrive one at a time (any length with a
// bucket, any band and k) and wait in a FIFO.  A scheduler thread owns a few
// batch slots, each with its own device arena, pinned staging buffers and
// stream pool: whenever a slot is free it admits the oldest waiting requests
// into a batch, as many as fit the slot's arena (admission by memory) up to a
// batch-size cap, and launches the batch; batches of different slots run on
// the device at the same time.  When a slot's batch completes, its results
// are copied to the requests' buffers and completion records (with arrival,
// admission and completion times) are posted for dtw_server_poll.
#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "index_impl.cuh"

namespace dtwk {
void set_error_message(const char *msg);

static int64_t now_ns() {
    return (int64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

struct Request {
    uint64_t ticket;
    int n, w, k;
    std::vector<float> q;
    int64_t *out_idx;
    float *out_dist;
    int64_t arrival, admit;
};

struct ServerSlot {
    Slot sl;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    bool busy = false;
    std::vector<Request> reqs;
    Batch bt;
    int k_stride = 1;
    int64_t launched_ns = 0;
    bool timed_out = false;  // its requests were completed by the watchdog
    float *hq = nullptr;  // pinned staged queries
    size_t hq_cap = 0;
    int64_t *hoi = nullptr;  // pinned outputs [max_batch][DTW_MAX_K]
    float *hod = nullptr;
};

// Upper bound of the arena bytes of a batch, kept per group as requests are
// added (the exact figure is checked once the batch is formed).
struct Admission {
    std::map<std::array<int, 3>, std::pair<int, size_t>> groups;  // (bucket, w, k) -> (queries, workspace)
    int64_t Q = 0, total = 0, gout = 0;
    int kmax = 1;
    size_t ws = 0;
    size_t bound() const {
        const size_t G = groups.size();
        return ws + 2 * ((size_t)total * 4 + 256) + (size_t)Q * sizeof(QMap) + 256 + (size_t)gout * 12 + 512 +
               (size_t)Q * kmax * 12 + 512 + (G + 1) * CNT_ALLOC * 8 + 256 + 4096;
    }
};

}  // namespace dtwk

using namespace dtwk;

struct dtw_server {
    dtw_index *ix = nullptr;
    dtw_server_config cfg{};
    std::vector<ServerSlot> slots;
    std::deque<Request> pending;
    std::deque<dtw_completion> done;
    std::mutex mu;
    std::condition_variable cv, done_cv;
    std::thread th;
    bool stop = false;
    uint64_t next_ticket = 1;
    dtw_server_stats st{};
    int inflight = 0;
};

namespace dtwk {

static size_t request_ws(dtw_index *ix, int b, int w, int k, int qn) {
    const Tuning t = tuning_for(ix, ix->buckets[b].n, w, k);
    return cascade_ws_bytes(plan_for(ix, b, w, k, qn, t));
}

// Admits the oldest pending requests into slot ss and launches the batch.
// Called by the scheduler with srv->mu held (lk); the lock is released while
// the batch is prepared and launched, so that submissions are not held up.
static void launch_slot(dtw_server *srv, ServerSlot &ss, std::unique_lock<std::mutex> &lk) {
    dtw_index *ix = srv->ix;
    const size_t cap = (size_t)srv->cfg.slot_bytes;
    Admission adm;
    ss.reqs.clear();
    std::unique_lock<std::mutex> ilk0(ix->mu);
    while (!srv->pending.empty() && (int)ss.reqs.size() < srv->cfg.max_batch) {
        const Request &r = srv->pending.front();
        const int b = find_bucket(ix, r.n);
        const int we = r.w < r.n - 1 ? r.w : r.n - 1;
        Admission next = adm;
        auto &g = next.groups[{b, we, r.k}];
        next.ws -= g.second;
        g.first += 1;
        g.second = request_ws(ix, b, we, r.k, g.first);
        next.ws += g.second;
        next.Q += 1;
        next.total += r.n;
        next.gout += r.k;
        next.kmax = std::max(next.kmax, r.k);
        if (next.bound() > cap && !ss.reqs.empty()) break;  // memory admission
        adm = next;
        ss.reqs.push_back(std::move(srv->pending.front()));
        srv->pending.pop_front();
    }
    ilk0.unlock();
    if (ss.reqs.empty()) return;
    const int64_t Q = (int64_t)ss.reqs.size();
    std::vector<int32_t> lens(Q), ws(Q), ks(Q);
    int kmax = 1;
    int64_t off = 0;
    for (int64_t i = 0; i < Q; ++i) {
        const Request &r = ss.reqs[i];
        lens[i] = r.n;
        ws[i] = r.w;
        ks[i] = r.k;
        kmax = std::max(kmax, r.k);
        std::memcpy(ss.hq + off, r.q.data(), (size_t)r.n * sizeof(float));
        off += r.n;
    }
    ss.k_stride = kmax;
    const int64_t t_admit = now_ns();
    for (auto &r : ss.reqs) r.admit = t_admit;
    dtw_status st;
    lk.unlock();
    {
        std::lock_guard<std::mutex> ilk(ix->mu);
        st = prepare_batch(ix, Q, lens.data(), ws.data(), ks.data(), kmax, srv->cfg.flags, ss.bt);
        if (st == DTW_OK && batch_bytes(ss.bt) > cap) st = ix_fail(DTW_ERR_OOM, "batch exceeds the slot arena");
        if (st == DTW_OK)
            st = run_batch(ix, ss.sl, ss.bt, ss.hq, false, ss.hoi, ss.hod, false, ss.stream, nullptr);
    }
    if (st == DTW_OK && cudaEventRecord(ss.ev, ss.stream) != cudaSuccess) st = DTW_ERR_CUDA;
    lk.lock();
    if (st != DTW_OK) {
        // the batch failed before running: complete its requests with the error
        const int64_t t = now_ns();
        for (auto &r : ss.reqs)
            srv->done.push_back(dtw_completion{r.ticket, (int32_t)st, r.k, r.arrival, r.admit, t});
        srv->st.completed += Q;
        srv->st.failed += Q;
        ss.reqs.clear();
        srv->done_cv.notify_all();
        return;
    }
    ss.busy = true;
    ss.timed_out = false;
    ss.launched_ns = now_ns();
    srv->inflight += 1;
    srv->st.batches += 1;
    srv->st.max_inflight_batches = std::max<int64_t>(srv->st.max_inflight_batches, srv->inflight);
    srv->st.max_batch_seen = std::max<int64_t>(srv->st.max_batch_seen, Q);
}

// The watchdog: completes a slot's requests with DTW_ERR_TIMEOUT when its
// batch has run past the deadline (srv->mu held).  The slot is released only
// when the device work ends (finish_slot), since it still uses the buffers.
static void expire_slot(dtw_server *srv, ServerSlot &ss) {
    const int64_t t = now_ns();
    for (auto &r : ss.reqs)
        srv->done.push_back(dtw_completion{r.ticket, (int32_t)DTW_ERR_TIMEOUT, r.k, r.arrival, r.admit, t});
    srv->st.completed += (int64_t)ss.reqs.size();
    srv->st.failed += (int64_t)ss.reqs.size();
    srv->st.timed_out += (int64_t)ss.reqs.size();
    ss.reqs.clear();
    ss.timed_out = true;
    srv->done_cv.notify_all();
}

// Delivers the results of a completed slot (srv->mu held).
static void finish_slot(dtw_server *srv, ServerSlot &ss, cudaError_t e) {
    const int64_t t = now_ns();
    for (size_t i = 0; i < ss.reqs.size(); ++i) {
        Request &r = ss.reqs[i];
        if (e == cudaSuccess) {
            std::memcpy(r.out_idx, ss.hoi + i * ss.k_stride, (size_t)r.k * sizeof(int64_t));
            std::memcpy(r.out_dist, ss.hod + i * ss.k_stride, (size_t)r.k * sizeof(float));
        }
        srv->done.push_back(dtw_completion{r.ticket, e == cudaSuccess ? (int32_t)DTW_OK : (int32_t)DTW_ERR_CUDA, r.k,
                                           r.arrival, r.admit, t});
    }
    srv->st.completed += (int64_t)ss.reqs.size();
    if (e != cudaSuccess) srv->st.failed += (int64_t)ss.reqs.size();
    ss.reqs.clear();
    ss.busy = false;
    srv->inflight -= 1;
    srv->done_cv.notify_all();
}

static void scheduler(dtw_server *srv) {
    cudaSetDevice(srv->ix->device);
    std::unique_lock<std::mutex> lk(srv->mu);
    for (;;) {
        bool progress = false;
        for (auto &ss : srv->slots) {
            if (!ss.busy) continue;
            const cudaError_t e = cudaEventQuery(ss.ev);
            if (e == cudaErrorNotReady) {
                if (!ss.timed_out && srv->cfg.batch_timeout_ms > 0 &&
                    now_ns() - ss.launched_ns > (int64_t)srv->cfg.batch_timeout_ms * 1000000) {
                    expire_slot(srv, ss);
                    progress = true;
                }
                continue;
            }
            if (e != cudaSuccess) cudaGetLastError();
            finish_slot(srv, ss, e);
            progress = true;
        }
        if (!srv->pending.empty()) {
            // a partial batch waits up to max_wait_us for company while
            // another batch is on the device
            const bool full = (int)srv->pending.size() >= srv->cfg.max_batch;
            const bool waited = now_ns() - srv->pending.front().arrival >= (int64_t)srv->cfg.max_wait_us * 1000;
            if (full || waited || srv->inflight == 0) {
                for (auto &ss : srv->slots) {
                    if (ss.busy || srv->pending.empty()) continue;
                    launch_slot(srv, ss, lk);
                    progress = true;
                }
            }
        }
        if (srv->stop && srv->pending.empty() && srv->inflight == 0) break;
        if (!progress) {
            if (srv->inflight > 0 || !srv->pending.empty())
                srv->cv.wait_for(lk, std::chrono::microseconds(20));
            else
                srv->cv.wait_for(lk, std::chrono::milliseconds(5));
        }
    }
}

}  // namespace dtwk

extern "C" {

int64_t dtw_monotonic_ns(void) { return now_ns(); }

dtw_status dtw_server_create(dtw_index *ix, const dtw_server_config *cfg, dtw_server **out) {
    set_error_message("");
    if (!ix || !out) return ix_fail(DTW_ERR_INVALID_ARG, "null pointer");
    *out = nullptr;
    dtw_server_config c{4, 512, 0, 0, 0, 0};
    if (cfg) c = *cfg;
    if (c.slots < 1 || c.slots > 16) return ix_fail(DTW_ERR_INVALID_ARG, "slots=%d outside [1, 16]", c.slots);
    if (c.max_batch < 1 || c.max_batch > 65536)
        return ix_fail(DTW_ERR_INVALID_ARG, "max_batch=%d outside [1, 65536]", c.max_batch);
    if (c.slot_bytes < 0 || c.max_wait_us < 0 || c.batch_timeout_ms < 0)
        return ix_fail(DTW_ERR_INVALID_ARG, "negative slot_bytes, max_wait_us or batch_timeout_ms");
    if (c.flags & ~(DTW_BATCH_GRAPH | DTW_BATCH_SERIAL | DTW_BATCH_PER_QUERY))
        return ix_fail(DTW_ERR_INVALID_ARG, "flags=0x%x: only GRAPH, SERIAL and PER_QUERY apply", c.flags);
    if (c.slot_bytes == 0) c.slot_bytes = (int64_t)2 << 30;
    auto *srv = new dtw_server();
    srv->ix = ix;
    srv->cfg = c;
    srv->slots.resize(c.slots);
    int maxn = 1;
    for (const auto &bk : ix->buckets) maxn = std::max(maxn, bk.n);
    dtw_status st = DTW_OK;
    {
        std::lock_guard<std::mutex> lk(ix->mu);
        int prev = -1;
        cudaGetDevice(&prev);
        cudaSetDevice(ix->device);
        for (auto &ss : srv->slots) {
            if ((st = slot_init(ss.sl, (int)ix->slot.pool.size())) != DTW_OK) break;
            if ((st = slot_reserve(ss.sl, (size_t)c.slot_bytes)) != DTW_OK) break;
            if (cudaStreamCreateWithFlags(&ss.stream, cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&ss.ev, cudaEventDisableTiming) != cudaSuccess) {
                st = ix_fail(DTW_ERR_CUDA, "stream or event creation failed");
                break;
            }
            ss.hq_cap = (size_t)c.max_batch * maxn;
            if (cudaHostAlloc((void **)&ss.hq, ss.hq_cap * sizeof(float), cudaHostAllocDefault) != cudaSuccess ||
                cudaHostAlloc((void **)&ss.hoi, (size_t)c.max_batch * DTW_MAX_K * sizeof(int64_t),
                              cudaHostAllocDefault) != cudaSuccess ||
                cudaHostAlloc((void **)&ss.hod, (size_t)c.max_batch * DTW_MAX_K * sizeof(float),
                              cudaHostAllocDefault) != cudaSuccess) {
                cudaGetLastError();
                st = ix_fail(DTW_ERR_OOM, "pinned staging buffers");
                break;
            }
            // the pinned query map, sized once so that no batch allocates
            QMap *hm = nullptr;
            if (cudaHostAlloc((void **)&hm, (size_t)c.max_batch * sizeof(QMap), cudaHostAllocDefault) != cudaSuccess) {
                cudaGetLastError();
                st = ix_fail(DTW_ERR_OOM, "pinned query map");
                break;
            }
            ss.sl.hmap = hm;
            ss.sl.hmap_cap = (size_t)c.max_batch;
        }
        if (prev >= 0) cudaSetDevice(prev);
    }
    if (st != DTW_OK) {
        for (auto &ss : srv->slots) {
            if (ss.hq) cudaFreeHost(ss.hq);
            if (ss.hoi) cudaFreeHost(ss.hoi);
            if (ss.hod) cudaFreeHost(ss.hod);
            if (ss.ev) cudaEventDestroy(ss.ev);
            if (ss.stream) cudaStreamDestroy(ss.stream);
            slot_release(ss.sl);
        }
        delete srv;
        return st;
    }
    srv->th = std::thread(scheduler, srv);
    *out = srv;
    return DTW_OK;
}

dtw_status dtw_server_submit(dtw_server *srv, const float *query, int32_t n, int32_t w, int32_t k, int64_t *out_idx,
                             float *out_dist, int64_t arrival_ns, uint64_t *ticket) {
    set_error_message("");
    if (!srv || !query || !out_idx || !out_dist) return ix_fail(DTW_ERR_INVALID_ARG, "null pointer");
    if (n < 1 || n > DTW_MAX_N) return ix_fail(DTW_ERR_INVALID_ARG, "n=%d out of range", n);
    if (w < 0) return ix_fail(DTW_ERR_INVALID_ARG, "w=%d must be >= 0", w);
    if (k < 1 || k > DTW_MAX_K) return ix_fail(DTW_ERR_INVALID_ARG, "k=%d outside [1, %d]", k, DTW_MAX_K);
    for (int32_t i = 0; i < n; ++i)
        if (!std::isfinite(query[i]))
            return ix_fail(DTW_ERR_INVALID_ARG, "query value %d is not finite (NaN or infinity)", i);
    dtw_index *ix = srv->ix;
    int b;
    size_t need;
    {
        std::lock_guard<std::mutex> lk(ix->mu);
        b = find_bucket(ix, n);
        if (b < 0) return ix_fail(DTW_ERR_NO_BUCKET, "no bucket of length %d", n);
        const int we = w < n - 1 ? w : n - 1;
        if (2 * we + 1 > 2048) return ix_fail(DTW_ERR_INVALID_ARG, "DTW band %d exceeds 2048", 2 * we + 1);
        Admission one;
        one.groups[{b, we, k}] = {1, request_ws(ix, b, we, k, 1)};
        one.ws = one.groups.begin()->second.second;
        one.Q = 1;
        one.total = n;
        one.gout = k;
        one.kmax = k;
        need = one.bound();
    }
    if (need > (size_t)srv->cfg.slot_bytes)
        return ix_fail(DTW_ERR_OOM, "one query of length %d needs %zu bytes, above slot_bytes", n, need);
    Request r;
    r.n = n;
    r.w = w;
    r.k = k;
    r.q.assign(query, query + n);
    r.out_idx = out_idx;
    r.out_dist = out_dist;
    r.arrival = arrival_ns > 0 ? arrival_ns : now_ns();
    r.admit = 0;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        if (srv->stop) return ix_fail(DTW_ERR_INVALID_ARG, "server is stopping");
        r.ticket = srv->next_ticket++;
        if (ticket) *ticket = r.ticket;
        srv->pending.push_back(std::move(r));
        srv->st.submitted += 1;
    }
    srv->cv.notify_one();
    return DTW_OK;
}

dtw_status dtw_server_poll(dtw_server *srv, dtw_completion *out, int32_t max, int32_t *count, int32_t wait_ms) {
    set_error_message("");
    if (!srv || !count || (max > 0 && !out)) return ix_fail(DTW_ERR_INVALID_ARG, "null pointer");
    *count = 0;
    std::unique_lock<std::mutex> lk(srv->mu);
    if (srv->done.empty() && wait_ms > 0)
        srv->done_cv.wait_for(lk, std::chrono::milliseconds(wait_ms), [&] { return !srv->done.empty(); });
    int c = 0;
    while (c < max && !srv->done.empty()) {
        out[c++] = srv->done.front();
        srv->done.pop_front();
    }
    *count = c;
    return DTW_OK;
}

dtw_status dtw_server_info(dtw_server *srv, dtw_server_stats *out) {
    set_error_message("");
    if (!srv || !out) return ix_fail(DTW_ERR_INVALID_ARG, "null pointer");
    std::lock_guard<std::mutex> lk(srv->mu);
    *out = srv->st;
    out->pending = (int64_t)srv->pending.size();
    out->inflight_batches = srv->inflight;
    return DTW_OK;
}

dtw_status dtw_server_destroy(dtw_server *srv) {
    set_error_message("");
    if (!srv) return DTW_OK;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stop = true;
    }
    srv->cv.notify_all();
    if (srv->th.joinable()) srv->th.join();
    {
        std::lock_guard<std::mutex> lk(srv->ix->mu);
        int prev = -1;
        cudaGetDevice(&prev);
        cudaSetDevice(srv->ix->device);
        for (auto &ss : srv->slots) {
            if (ss.stream) cudaStreamSynchronize(ss.stream);
            if (ss.hq) cudaFreeHost(ss.hq);
            if (ss.hoi) cudaFreeHost(ss.hoi);
            if (ss.hod) cudaFreeHost(ss.hod);
            if (ss.ev) cudaEventDestroy(ss.ev);
            if (ss.stream) cudaStreamDestroy(ss.stream);
            slot_release(ss.sl);
        }
        if (prev >= 0) cudaSetDevice(prev);
    }
    delete srv;
    return DTW_OK;
}

}  // extern "C"
