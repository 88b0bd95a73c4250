// Runtime services of the library: error state, device memory, launch
// counting and the kernel timer used for roofline measurements.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace pg {

static thread_local std::string g_last_error;
static std::atomic<uint64_t> g_launches{0};
static std::atomic<int> g_fail_alloc_after{0};

void set_error(pg_status code, const std::string &msg) {
    (void)code;
    g_last_error = msg;
}

pg_status fail(pg_status code, const std::string &msg) {
    set_error(code, msg);
    return code;
}

pg_status cuda_fail(cudaError_t e, const char *what) {
    std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    if (e == cudaErrorMemoryAllocation) return fail(PG_ENOMEM, m);
    return fail(PG_ECUDA, m);
}

static std::once_flag g_pool_once;

static void configure_pool() {
    // Keep freed blocks in the default pool so repeated builds and queries do
    // not return memory to the driver between calls.
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) != cudaSuccess) return;
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
}

pg_status dalloc(void **p, size_t bytes, cudaStream_t s) {
    *p = nullptr;
    int left = g_fail_alloc_after.load();
    if (left > 0) {
        if (g_fail_alloc_after.fetch_sub(1) == 1)
            return fail(PG_ENOMEM, "device allocation failed (injected)");
    }
    std::call_once(g_pool_once, configure_pool);
    cudaError_t e = cudaMallocAsync(p, bytes ? bytes : 16, s);
    if (e != cudaSuccess) {
        *p = nullptr;
        return cuda_fail(e, "cudaMallocAsync");
    }
    return PG_OK;
}

void dfree(void *p, cudaStream_t s) {
    if (p) cudaFreeAsync(p, s);
}

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
// ---------------------------------------------------------------- small reads
// A few device words reach the host through a kernel that stores them into
// mapped pinned host memory, not through a copy engine: a bulk transfer the
// caller has in flight on another stream (results going back to the host)
// then cannot delay the library's own control reads.
namespace {
__global__ void k_read_small(const int *__restrict__ src, int *dst, int words) {
    const int i = threadIdx.x;
    if (i < words) dst[i] = src[i];
}
constexpr size_t kReadSmallBytes = 1024;
thread_local std::map<int, int *> t_mapped;   // device -> mapped buffer (kept for the thread's life)
}  // namespace

// Fills and small uploads by kernels, for the same reason: neither waits
// behind a bulk copy in flight on a copy engine.
namespace {
__global__ void k_fill_words(uint32_t *__restrict__ p, uint32_t v, size_t n) {
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if ((reinterpret_cast<uintptr_t>(p) & 15) == 0) {
        uint4 *q = reinterpret_cast<uint4 *>(p);
        const uint4 vv = make_uint4(v, v, v, v);
        for (size_t j = i; j < n / 4; j += stride) q[j] = vv;
        for (size_t j = n / 4 * 4 + i; j < n; j += stride) p[j] = v;
    } else {
        for (size_t j = i; j < n; j += stride) p[j] = v;
    }
}
struct SmallBlob {
    uint32_t w[kStoreSmallBytes / 4];
};
__global__ void k_store_words(uint32_t *__restrict__ dst, SmallBlob b, int words) {
    const int i = threadIdx.x;
    if (i < words) dst[i] = b.w[i];
}
}  // namespace

pg_status fill_words(void *dst, uint32_t value, size_t words, cudaStream_t s) {
    if (words == 0) return PG_OK;
    const int grid = (int)std::min<size_t>((words / 4 + 255) / 256 + 1, (size_t)num_sms() * 8);
    k_fill_words<<<grid, 256, 0, s>>>(static_cast<uint32_t *>(dst), value, words);
    count_launch();
    return check_launch("fill_words");
}

pg_status store_small(void *dev_dst, const void *host_src, size_t bytes, cudaStream_t s) {
    if (bytes == 0) return PG_OK;
    if (bytes > kStoreSmallBytes || bytes % 4) return fail(PG_EINVAL, "store_small: at most 256 bytes, whole words");
    SmallBlob b;
    memcpy(b.w, host_src, bytes);
    k_store_words<<<1, (int)(kStoreSmallBytes / 4), 0, s>>>(static_cast<uint32_t *>(dev_dst), b, (int)(bytes / 4));
    count_launch();
    return check_launch("store_small");
}

pg_status read_small(void *host_dst, const void *dev_src, size_t bytes, cudaStream_t s) {
    if (bytes == 0) return PG_OK;
    if (bytes > kReadSmallBytes || bytes % 4) return fail(PG_EINVAL, "read_small: at most 1024 bytes, whole words");
    int dev = 0;
    PG_CUDA(cudaGetDevice(&dev));
    int *&buf = t_mapped[dev];
    if (!buf) PG_CUDA(cudaHostAlloc(reinterpret_cast<void **>(&buf), kReadSmallBytes, cudaHostAllocMapped | cudaHostAllocPortable));
    k_read_small<<<1, (int)(kReadSmallBytes / 4), 0, s>>>(static_cast<const int *>(dev_src), buf, (int)(bytes / 4));
    count_launch();
    PG_TRY(check_launch("read_small"));
    PG_CUDA(cudaStreamSynchronize(s));
    memcpy(host_dst, buf, bytes);
    return PG_OK;
}


pg_status check_launch(const char *what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, what);
    return PG_OK;
}

int num_sms() {
    static int sms = 0;
    if (sms == 0) {
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        sms = v > 0 ? v : 1;
    }
    return sms;
}

// ---------------------------------------------------------------- kernel timer
struct TimedLaunch {
    std::string name;
    cudaEvent_t a, b;
};
static std::mutex g_prof_mu;
static std::vector<TimedLaunch> g_prof;
static std::atomic<int> g_prof_on{0};

KTimer::KTimer(const char *nm, cudaStream_t st) : name(nm), s(st) {
    if (!g_prof_on.load()) return;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
        a = b = nullptr;
        return;
    }
    cudaEventRecord(a, s);
}

KTimer::~KTimer() {
    if (!a) return;
    cudaEventRecord(b, s);
    std::lock_guard<std::mutex> g(g_prof_mu);
    g_prof.push_back({name, a, b});
}

}  // namespace pg

using namespace pg;

extern "C" {

const char *pg_last_error(void) { return g_last_error.c_str(); }

const char *pg_version(void) { return "pargeo-gb300 0.1 (sm_103a)"; }

uint64_t pg_launch_count(void) { return g_launches.load(); }

pg_status pg_profile_enable(int on) {
    g_prof_on.store(on ? 1 : 0);
    return PG_OK;
}

pg_status pg_profile_read(const char *prefix, double *total_ms, int64_t *launches) {
    if (!total_ms || !launches) return fail(PG_EINVAL, "pg_profile_read: null output");
    std::vector<TimedLaunch> keep, take;
    {
        std::lock_guard<std::mutex> g(g_prof_mu);
        for (auto &t : g_prof) {
            if (!prefix || t.name.compare(0, strlen(prefix), prefix) == 0) take.push_back(t);
            else keep.push_back(t);
        }
        g_prof.swap(keep);
    }
    double tot = 0.0;
    int64_t cnt = 0;
    pg_status st = PG_OK;
    for (auto &t : take) {
        cudaError_t e = cudaEventSynchronize(t.b);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t.a, t.b);
        if (e != cudaSuccess && st == PG_OK) st = cuda_fail(e, "pg_profile_read");
        tot += ms;
        ++cnt;
        cudaEventDestroy(t.a);
        cudaEventDestroy(t.b);
    }
    *total_ms = tot;
    *launches = cnt;
    return st;
}

pg_status pg_debug_fail_alloc_after(int n) {
    g_fail_alloc_after.store(n > 0 ? n : 0);
    return PG_OK;
}

}  // extern "C"
