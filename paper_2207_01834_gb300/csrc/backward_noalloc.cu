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
// cleared on each call.  The first call on a device looks up the array's device
// address (cudaGetSymbolAddress) with that device current; make that first
// call before any stream capture.
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
// bounds (2 words per data point), rounded to 256 bytes
constexpr size_t kMainBytes = ((size_t)(4 * kMaxPairs + 2 * kMaxPoints) * 4 + 256 + 255) / 256 * 256;
// radix workspace: two 256 x tiles tables + scan partials (tiles of 2048 items)
constexpr size_t kRadixWords = 2 * 256 * (size_t)(kMaxPairs / 2048) + 1 + ((256 * (kMaxPairs / 2048)) / 4096 + 2);
constexpr size_t kScratchBytes = kMainBytes + (kRadixWords * 4 + 255) / 256 * 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
void *g_addr[256] = {};

// Device address of the array on the current device (looked up once per device).
pg_status scratch_address(void **out) {
    int dev = 0;
    PG_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 256) return fail(PG_EUNSUPPORTED, "pg_knn_backward_noalloc: device index out of range");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        g_addr[dev] = p;
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
    if (m * (int64_t)k > kMaxPairs)
        return fail(PG_EINVAL,
                    "pg_knn_backward_noalloc: m*k exceeds the fixed scratch limit of 1048576 (query, neighbour) pairs");
    if (m > 0 && (!queries || !idx || !grad_dist)) return fail(PG_EINVAL, "pg_knn_backward_noalloc: NULL input");
    if (n > 0 && !data && (grad_data || (m > 0 && grad_queries)))
        return fail(PG_EINVAL, "pg_knn_backward_noalloc: NULL data");
    void *base = nullptr;
    PG_TRY(scratch_address(&base));
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    unsigned char *b = static_cast<unsigned char *>(base);
    return knn_backward_run_ws(data, n, queries, m, dim, k, idx, grad_dist, grad_queries, grad_data, b,
                               reinterpret_cast<int *>(b + kMainBytes), s);
}
