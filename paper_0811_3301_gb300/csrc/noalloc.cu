// dtw_band_noalloc: dtw_band for callers that cannot call cudaMalloc.
//
// Some callers of this library cannot allocate device memory at the point
// where they need a DTW: for example a service whose device memory is owned
// and fully reserved by another allocator (a framework's caching pool), or a
// latency-critical loop that must not stall on the device-wide
// synchronisation of cudaFree when the library's workspace would grow.
// This entry point takes the scratch that dtw_band needs (the four padded,
// shifted copies of the query rows and the work cursor) from a fixed array
// in device memory that is part of the library itself, so it never calls
// cudaMalloc, cudaFree or any allocating routine.
//
// Costs and limits:
//  - the array, kNoAllocScratchBytes = 8 MiB, is held on every GPU that
//    loads the library until the process exits;
//  - a call whose scratch does not fit is rejected with DTW_ERR_INVALID_ARG;
//  - every call uses the same array, so calls that overlap on the GPU (on
//    different streams, or from different host threads) race on it; the
//    previous call's contents remain, and everything that must start at
//    zero (the cursor) is cleared by each call;
//  - the first call on a device looks up the array's device address with
//    cudaGetSymbolAddress while that device is current; make that first call
//    before any stream capture.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <mutex>

#include "common.cuh"
#include "dtw.cuh"

namespace dtwk {

constexpr size_t kNoAllocScratchBytes = size_t(8) << 20;

// The scratch.  In host code this name is only a host-side stand-in for the
// symbol; the device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

static void *g_noalloc_addr[64] = {nullptr};
static std::mutex g_noalloc_mu;

void set_error_message(const char *msg);  // api.cu

static dtw_status noalloc_fail(dtw_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    set_error_message(buf);
    return st;
}

// Device address of the scratch array on the current device (looked up once
// per device, with that device current).
static dtw_status noalloc_scratch(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return noalloc_fail(DTW_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= 64) return noalloc_fail(DTW_ERR_INTERNAL, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (g_noalloc_addr[dev] == nullptr) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            return noalloc_fail(DTW_ERR_CUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
        }
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return DTW_OK;
}

}  // namespace dtwk

using namespace dtwk;

extern "C" dtw_status dtw_band_noalloc(const float *x, const float *y, int64_t N, int32_t y_stride,
                                       int32_t n, int32_t w, int32_t p, float threshold, float *out,
                                       void *stream) {
    set_error_message("");
    if (n < 1 || n > DTW_MAX_N) return noalloc_fail(DTW_ERR_INVALID_ARG, "n=%d outside [1, %d]", n, DTW_MAX_N);
    if (w < 0) return noalloc_fail(DTW_ERR_INVALID_ARG, "w=%d must be >= 0", w);
    if (p != 1 && p != 2 && p != 4 && p != DTW_P_INF)
        return noalloc_fail(DTW_ERR_INVALID_ARG, "p=%d must be 1, 2, 4 or DTW_P_INF (0)", p);
    const int we = w < n - 1 ? w : n - 1;
    if (2 * we + 1 > 2048)
        return noalloc_fail(DTW_ERR_INVALID_ARG, "DTW band 2*min(w,n-1)+1 = %d exceeds 2048", 2 * we + 1);
    if (N < 0 || N > INT32_MAX) return noalloc_fail(DTW_ERR_INVALID_ARG, "N=%lld out of range", (long long)N);
    if (y_stride != 0 && y_stride != n)
        return noalloc_fail(DTW_ERR_INVALID_ARG, "y_stride=%d must be 0 or n=%d", y_stride, n);
    if (std::isnan(threshold) || threshold < 0.0f)
        return noalloc_fail(DTW_ERR_INVALID_ARG, "threshold must be >= 0 or +INF");
    if (N == 0) return DTW_OK;
    if (!x || !y || !out) return noalloc_fail(DTW_ERR_INVALID_ARG, "null pointer");

    const DtwGeom g = dtw_geom(n, we);
    const int64_t nq = y_stride ? N : 1;
    const size_t copies_bytes = ((size_t)nq * 4 * g.ylen * sizeof(float) + 255) & ~size_t(255);
    const size_t need = copies_bytes + 256;  // + the work cursor
    if (need > kNoAllocScratchBytes)
        return noalloc_fail(DTW_ERR_INVALID_ARG,
                            "dtw_band_noalloc needs %zu bytes of scratch for N=%lld, n=%d, w=%d, "
                            "y_stride=%d; its fixed scratch holds %zu bytes",
                            need, (long long)N, n, w, y_stride, kNoAllocScratchBytes);
    void *scratch = nullptr;
    dtw_status st = noalloc_scratch(&scratch);
    if (st != DTW_OK) return st;

    cudaStream_t s = (cudaStream_t)stream;
    QueryCopies qc;
    qc.data = reinterpret_cast<float *>(scratch);
    qc.padl = g.padl;
    qc.ylen = g.ylen;
    unsigned long long *cursor =
        reinterpret_cast<unsigned long long *>(reinterpret_cast<char *>(scratch) + copies_bytes);
    cudaError_t e = launch_query_copies(y, nq, n, qc, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(cursor, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return noalloc_fail(DTW_ERR_CUDA, "scratch set-up: %s", cudaGetErrorString(e));
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
    j.fixed_thr = std::isinf(threshold) ? INFINITY
                  : (p == 2 ? threshold * threshold
                            : (p == 4 ? (threshold * threshold) * (threshold * threshold) : threshold));
    j.abandon = std::isinf(threshold) ? 0 : 1;
    j.res = out;
    j.root_out = 1;
    j.cursor = cursor;
    e = launch_dtw_by_p(j, g, s);
    if (e != cudaSuccess) return noalloc_fail(DTW_ERR_CUDA, "DTW launch: %s", cudaGetErrorString(e));
    return DTW_OK;
}
