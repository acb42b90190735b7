// Persistent form of the mixed-length batch (index.cu, DTW_BATCH_PERSISTENT).
// Internal: the public ABI is include/dtwknn.h.
#pragma once

#include "cascade_host.cuh"

namespace dtwk {

// One (bucket, w, k) group of a batch, as the persistent kernel reads it:
// the bucket's rows and row envelopes, the group's query terms and padded
// copies (made by cascade_prefix), its bound matrix (bounds on entry;
// completed DTWs are written back into it with the sign bit set), its
// thresholds, seeds and outputs.
struct PersistGroup {
    const float *db, *XU, *XL;          // [N][n]
    const float *queries, *U, *L, *UL, *LU;  // [Q][n]
    QueryCopies qc;
    float *lb;                          // [Q][N]
    uint32_t *bsf, *gmin;               // [Q], [Q][k] (fp32 bits)
    const Pair *seed_pairs;             // [S][Q]
    const float *seed_res;              // [S][Q]
    int64_t *out_idx;                   // [Q][k]
    float *out_dist;                    // [Q][k]
    unsigned long long *counters;       // the group's counter block (CNT_ALLOC words)
    int64_t item0;                      // first work item of the group
    int64_t qbase;                      // first query of the group among all the batch's groups
    int N, Q, n, w, p, k, S, chunk, nchunks;
    int dg, cl;                         // DTW lane groups: G lanes per pair, CL band slots per lane
    int vec, summary;
    float slack, summary_scale;
};

// Lane groups of the persistent kernel's DTW for band w of series of length
// n: G lanes per pair (4, 8, 16 or 32; the smallest with G * 16 >= 2w + 1)
// and CL band slots per lane (4, 8 or 16; the smallest with G * CL >=
// 2w + 1); {0, 0} when 2w + 1 > 512.
struct PersistShape {
    int g, cl;
};
PersistShape persist_shape(int n, int w);

// The persistent filter + DTW over every group's (query, candidate-chunk)
// items (groups: device table of G entries, total_items items; cursor zeroed
// by the caller), then the top-k of every query (total_queries over all
// groups).  Asynchronous on s.
cudaError_t launch_persistent(const PersistGroup *groups, int G, int64_t total_items, int64_t total_queries,
                              int p, unsigned long long *cursor, cudaStream_t s);

}  // namespace dtwk
