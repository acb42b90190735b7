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
// cudaMalloc, cudaFree or any allocating routine.  Its arguments are checked
// by the same code as dtw_band's, and it launches the same kernels.
//
// Costs and limits:
//  - the array, kNoAllocScratchBytes = 8 MiB, is held on every GPU that
//    loads the library until the process exits;
//  - a call whose scratch does not fit is rejected with DTW_ERR_INVALID_ARG;
//  - every call uses the same array, so calls that overlap on the GPU (on
//    different streams, or from different host threads) race on it; the
//    previous call's contents remain, and everything that must start at
//    zero (the cursor) is cleared by each call;
//  - the first call in each CUDA context of a device (the primary context is
//    created anew after cudaDeviceReset) looks up the array's device address
//    with cudaGetSymbolAddress while that device is current, and keeps it for
//    the later calls in that context; make that first call before any stream
//    capture.
#include <cmath>
#include <cstdio>
#include <mutex>

#include "common.cuh"
#include "dtw.cuh"

namespace dtwk {

constexpr size_t kNoAllocScratchBytes = size_t(8) << 20;

// The scratch.  In host code this name is only a host-side stand-in for the
// symbol; the device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

void set_error_message(const char *msg);  // api.cu

// Per device ordinal: the context (by its process-unique id) in which the
// address was looked up, and the address.
struct NoallocAddr {
    unsigned long long ctx_id = 0;
    void *addr = nullptr;
};
static NoallocAddr g_noalloc_addr[64];
static std::mutex g_noalloc_mu;

// The driver's cuCtxGetCurrent and cuCtxGetId, reached through the runtime
// (the library does not link the driver library itself).
typedef int (*CtxGetCurrentFn)(void **);
typedef int (*CtxGetIdFn)(void *, unsigned long long *);

// Process-unique id of the context current on this thread; 0 when none is.
static bool current_context_id(unsigned long long *id) {
    static CtxGetCurrentFn get_cur = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = q1;
        void *f1 = nullptr, *f2 = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
            q1 == cudaDriverEntryPointSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
            q2 == cudaDriverEntryPointSuccess) {
            get_cur = reinterpret_cast<CtxGetCurrentFn>(f1);
            get_id = reinterpret_cast<CtxGetIdFn>(f2);
        }
        cudaGetLastError();
    });
    *id = 0;
    if (!get_cur || !get_id) return false;
    void *ctx = nullptr;
    if (get_cur(&ctx) != 0) return false;
    if (ctx == nullptr) return true;
    return get_id(ctx, id) == 0;
}

// Device address of the scratch array in the current device's current
// context, looked up with cudaGetSymbolAddress once per context while that
// device is current.  The lookup also makes the device's primary context
// current when no context was yet.
static dtw_status noalloc_scratch(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(DTW_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= 64) return fail(DTW_ERR_INTERNAL, "device ordinal %d out of range", dev);
    unsigned long long id = 0;
    if (!current_context_id(&id)) return fail(DTW_ERR_CUDA, "cannot identify the current CUDA context");
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    NoallocAddr &a = g_noalloc_addr[dev];
    if (id == 0 || a.ctx_id != id) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            a.ctx_id = 0;
            return fail(DTW_ERR_CUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
        }
        if (id == 0 && (!current_context_id(&id) || id == 0))
            return fail(DTW_ERR_CUDA, "cannot identify the current CUDA context");
        a.addr = p;
        a.ctx_id = id;
    }
    *out = a.addr;
    return DTW_OK;
}

}  // namespace dtwk

using namespace dtwk;

extern "C" dtw_status dtw_band_noalloc(const float *x, const float *y, int64_t N, int32_t y_stride,
                                       int32_t n, int32_t w, int32_t p, float threshold, float *out,
                                       void *stream) {
    set_error_message("");
    bool empty = false;
    dtw_status st = check_dtw_band_args(x, y, N, y_stride, n, w, p, threshold, out, &empty);
    if (st != DTW_OK || empty) return st;
    const int we = w < n - 1 ? w : n - 1;
    const DtwGeom g = dtw_geom(n, we);
    const int64_t nq = y_stride ? N : 1;
    const size_t copies_bytes = ((size_t)nq * 4 * g.ylen * sizeof(float) + 255) & ~size_t(255);
    const size_t need = copies_bytes + 256;  // + the work cursor
    if (need > kNoAllocScratchBytes)
        return fail(DTW_ERR_INVALID_ARG,
                    "dtw_band_noalloc needs %zu bytes of scratch for N=%lld, n=%d, w=%d, "
                    "y_stride=%d; its fixed scratch holds %zu bytes",
                    need, (long long)N, n, w, y_stride, kNoAllocScratchBytes);
    void *scratch = nullptr;
    st = noalloc_scratch(&scratch);
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
    if (e != cudaSuccess) return fail(DTW_ERR_CUDA, "scratch set-up: %s", cudaGetErrorString(e));
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
    e = launch_dtw_by_p(j, g, s);
    if (e != cudaSuccess) return fail(DTW_ERR_CUDA, "DTW launch: %s", cudaGetErrorString(e));
    return DTW_OK;
}
