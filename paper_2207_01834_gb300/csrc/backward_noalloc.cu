// pg_knn_backward_noalloc: the k-NN gradient computed in a fixed, library-owned
// device buffer, for callers that cannot let a library allocate GPU memory.
//
// Who needs it: applications that reserve (nearly) all device memory for their
// own pool at start-up, so a cudaMalloc inside a library either fails or
// breaks their accounting; processes under a hard per-process memory cap; and
// latency-critical loops that must not pay for (or synchronise on) a device
// allocation.  This entry point uses only a statically sized __device__ array
// that is part of the loaded library image, so it never calls cudaMalloc,
// cudaMallocAsync, cudaFree or any allocating library routine.
//
// Costs and rules: the array (about 25 MiB) is resident on every GPU that
// loads the library until the process exits.  Every call uses the same array,
// so calls whose work overlaps on the GPU (for example on two streams at once)
// race with each other and must be serialised by the caller.  The array keeps
// the previous call's contents; everything the computation needs zeroed is
// cleared on each call.  Outside stream capture every call looks up the
// array's device address (cudaGetSymbolAddress) with the calling thread's
// device current, so a device reset is picked up by the next call; under
// capture the address found by the last uncaptured call on that device is
// used, so the first call on a device (and the first after a device reset)
// must come before any capture.
#include <mutex>

#include "internal.h"
#include "sort.h"

namespace pg {
size_t knn_backward_scratch_bytes(int64_t n, int64_t P);
pg_status knn_backward_run_ws(const float *data, int64_t n, const float *queries, int64_t m, int dim, int k,
                              const int32_t *idx, const float *g, float *gq, float *gp, void *scratch,
                              int *radix_ws, cudaStream_t s);
}  // namespace pg

using namespace pg;

namespace {

constexpr int64_t kMaxPairs = int64_t(1) << 20;    // m * k
constexpr int64_t kMaxPoints = int64_t(1) << 20;   // n
// main region: keys, values and two temporaries (4 words per pair) + segment
// bounds (2 words per data point), rounded to 256 bytes; it must hold
// knn_backward_scratch_bytes(n, m * k) for every accepted size
constexpr size_t kMainBytes = ((size_t)(4 * kMaxPairs + 2 * kMaxPoints) * 4 + 256 + 255) / 256 * 256;
// radix workspace of the sort of kMaxPairs keys, sized from the sort's and the
// scan's own tile constants
constexpr size_t kRadixWords = (size_t)radix_ws_words_ce(kMaxPairs);
static_assert(kRadixWords >= (size_t)radix_ws_words_ce(kMaxPairs - 1) && kRadixWords > 2 * kRadixDigits,
              "radix workspace reserve");
constexpr size_t kScratchBytes = kMainBytes + (kRadixWords * 4 + 255) / 256 * 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
void *g_addr[256] = {};   // last address looked up per device (used only under stream capture)

// Device address of the array in the current device's context.  Outside
// stream capture it is looked up on every call (so a device reset or a new
// primary context is picked up); under capture, where the lookup could load
// the module, the address of the last call on this device is used.
pg_status scratch_address(cudaStream_t s, void **out) {
    int dev = 0;
    PG_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 256) return fail(PG_EUNSUPPORTED, "pg_knn_backward_noalloc: device index out of range");
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
        (void)cudaGetLastError();   // not a sticky error; treat the stream as capturing
        cs = cudaStreamCaptureStatusActive;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (cs == cudaStreamCaptureStatusNone) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        g_addr[dev] = p;
    } else if (!g_addr[dev]) {
        return fail(PG_EINVAL,
                    "pg_knn_backward_noalloc: the first call on a device must come before any stream capture");
    }
    *out = g_addr[dev];
    return PG_OK;
}

}  // namespace

extern "C" pg_status pg_knn_backward_noalloc(const float *data, int64_t n, const float *queries, int64_t m,
                                             int dim, int k, const int32_t *idx, const float *grad_dist,
                                             float *grad_queries, float *grad_data, void *stream) {
    if (k < 1 || k > PG_MAX_K) return fail(PG_EINVAL, "pg_knn_backward_noalloc: k must be in [1, 64]");
    if (dim < 1 || dim > PG_MAX_DIM) return fail(PG_EINVAL, "pg_knn_backward_noalloc: dim must be in [1, 16]");
    if (n < 0 || m < 0) return fail(PG_EINVAL, "pg_knn_backward_noalloc: n and m must be >= 0");
    if (n > kMaxPoints)
        return fail(PG_EINVAL, "pg_knn_backward_noalloc: n exceeds the fixed scratch limit of 1048576 data points");
    // m is bounded before m * k is formed (no overflow for any m)
    if (m > kMaxPairs / k)
        return fail(PG_EINVAL,
                    "pg_knn_backward_noalloc: m*k exceeds the fixed scratch limit of 1048576 (query, neighbour) pairs");
    const int64_t P = m * (int64_t)k;
    if (knn_backward_scratch_bytes(n, P) > kMainBytes || (size_t)radix_ws_words(P) > kRadixWords)
        return fail(PG_EUNSUPPORTED, "pg_knn_backward_noalloc: scratch layout does not fit the fixed array");
    if (m > 0 && (!queries || !idx || !grad_dist)) return fail(PG_EINVAL, "pg_knn_backward_noalloc: NULL input");
    if (n > 0 && !data && (grad_data || (m > 0 && grad_queries)))
        return fail(PG_EINVAL, "pg_knn_backward_noalloc: NULL data");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    void *base = nullptr;
    PG_TRY(scratch_address(s, &base));
    unsigned char *b = static_cast<unsigned char *>(base);
    return knn_backward_run_ws(data, n, queries, m, dim, k, idx, grad_dist, grad_queries, grad_data, b,
                               reinterpret_cast<int *>(b + kMainBytes), s);
}
