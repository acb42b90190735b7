// Internal structures of the multi-length index (index.cu) and the request
// server (server.cu).  Internal: the public ABI is include/dtwknn.h.
#pragma once

#include <mutex>
#include <vector>
#include <map>

#include "cascade_host.cuh"
#include "persist.cuh"

namespace dtwk {

// One query of a batch: where its values are staged, where its group's run
// reads them, and where its result row is.
struct QMap {
    int64_t src;   // offset in the staged batch (floats)
    int64_t dst;   // offset in the grouped query buffer (floats)
    int64_t osrc;  // offset of its row in the group outputs (entries)
    int32_t len;   // n
    int32_t kg;    // its group's k
};

struct GraphEntry {
    std::vector<int64_t> key;
    cudaGraphExec_t exec;
    uint64_t last_use;
};

// Device arena, pinned query map and streams of one batch in flight.
struct Slot {
    char *arena = nullptr;
    size_t arena_cap = 0;
    QMap *hmap = nullptr;  // pinned host copy of the map
    size_t hmap_cap = 0;
    PersistGroup *hptab = nullptr;  // pinned host copy of the persistent group table
    size_t hptab_cap = 0;
    cudaEvent_t hmap_free = nullptr;  // the map's last host-to-device copy has completed
    cudaEvent_t done = nullptr;       // the slot's last batch has completed
    cudaStream_t origin = nullptr;    // capture stream
    std::vector<cudaStream_t> pool;
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> join;
    std::vector<GraphEntry> graphs;
    uint64_t tick = 0;
    int64_t captures = 0, replays = 0;
};

struct PartSums {
    int parts;
    float *PX;                 // [N][parts], owns the allocation
    unsigned long long *xmax;  // max |x| over the bucket (float bits in the low word)
};

// Envelopes of a bucket's rows for one band (LB_Improved's second sum).
struct DbEnvelope {
    int w;
    float *XU;  // [N][n], owns the allocation (XL follows it)
    float *XL;  // [N][n]
};

struct Bucket {
    int n;
    int64_t N;
    float *db;  // [N][n], owned
    std::vector<PartSums> sums;
    std::vector<DbEnvelope> envs;
};

struct TuneKey {
    int n, w, k;
    bool operator<(const TuneKey &o) const {
        if (n != o.n) return n < o.n;
        if (w != o.w) return w < o.w;
        return k < o.k;
    }
};

struct Tuning {
    int parts, seeds, seg_len;
    float ms;          // time of the tuning sample, -1 if not tuned
    int dtw_path;      // as in dtw_options
    int filter_warps;  // 0: from occupancy
};

// Queries of one batch with equal (bucket, w, k).
struct GroupRun {
    int bucket, w, k, qn;
    std::vector<int64_t> members;  // batch positions, in order
    Tuning t;
    CascadePlan pl;
    int64_t qoff;  // grouped query buffer offset (floats)
    int64_t ooff;  // group outputs offset (entries)
    int stream;    // pool stream index
    const float *PX;
    const unsigned *xmax;
    const float *XU, *XL;
};

struct Batch {
    int64_t Q = 0, total = 0, gout = 0;
    int k_stride = 1, flags = 0;
    std::vector<int> qbucket;
    std::vector<int64_t> qoff;  // offset of each query in the caller's flat array
    std::vector<GroupRun> groups;
};

struct BatchLayout {
    float *staged, *grouped, *gdist, *odist;
    QMap *map;
    int64_t *gidx, *oidx;
    unsigned long long *counters;
    PersistGroup *ptab;          // the persistent arm's group table (device)
    unsigned long long *pcursor; // its work-item cursor
    std::vector<CascadeWs> ws;
};

dtw_status ix_fail(dtw_status st, const char *fmt, ...);
dtw_status slot_init(Slot &sl, int pool_size);
void slot_release(Slot &sl);
dtw_status slot_reserve(Slot &sl, size_t bytes);
bool ptr_on_device(const void *p);

}  // namespace dtwk

struct dtw_index {
    int device = 0, p = 1;
    dtw_options opt{};
    std::vector<dtwk::Bucket> buckets;
    std::map<dtwk::TuneKey, dtwk::Tuning> tuned;
    dtwk::Slot slot;  // used by dtw_index_search
    int persist_chunk = 2048;  // candidates per work item of the persistent arm
    bool persist_tuned = false;
    std::mutex mu;
};

namespace dtwk {

int find_bucket(const dtw_index *ix, int n);
dtw_status ensure_sums(dtw_index *ix, int b, int parts, const PartSums **out);
dtw_status ensure_env(dtw_index *ix, int b, int w, const DbEnvelope **out);
Tuning tuning_for(const dtw_index *ix, int n, int w, int k);
CascadePlan plan_for(const dtw_index *ix, int b, int w, int k, int64_t qmax, const Tuning &t);
dtw_status prepare_batch(dtw_index *ix, int64_t Q, const int32_t *q_len, const int32_t *q_w, const int32_t *q_k,
                         int32_t k_stride, int32_t flags, Batch &bt);
size_t batch_bytes(const Batch &bt);
dtw_status run_batch(dtw_index *ix, Slot &sl, Batch &bt, const float *queries, bool q_dev, int64_t *out_idx,
                     float *out_dist, bool out_dev, cudaStream_t s, unsigned long long *counters_host);
void batch_stats(const Batch &bt, const unsigned long long *h, dtw_stats *st);
dtw_status tune_group(dtw_index *ix, int b, int w, int k, const float *qdev, int qn, Tuning *out);

}  // namespace dtwk
