// Shared device/host helpers of the sm_103a k-NN library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "pargeo_gpu.h"

namespace pg {

// ---------------------------------------------------------------- status
struct Error {
    pg_status code;
    std::string msg;
};

void set_error(pg_status code, const std::string &msg);
pg_status fail(pg_status code, const std::string &msg);
pg_status cuda_fail(cudaError_t e, const char *what);

#define PG_CUDA(call)                                                     \
    do {                                                                  \
        cudaError_t e_ = (call);                                          \
        if (e_ != cudaSuccess) return ::pg::cuda_fail(e_, #call);         \
    } while (0)

#define PG_TRY(call)                                                      \
    do {                                                                  \
        pg_status s_ = (call);                                            \
        if (s_ != PG_OK) return s_;                                       \
    } while (0)

// ---------------------------------------------------------------- memory
// Stream-ordered device allocation from the device's default pool (kept
// cached across calls).  Honours the allocation fault-injection hook.
pg_status dalloc(void **p, size_t bytes, cudaStream_t s);
void dfree(void *p, cudaStream_t s);

template <class T>
pg_status dalloc_n(T **p, size_t n, cudaStream_t s) {
    return dalloc(reinterpret_cast<void **>(p), n * sizeof(T), s);
}

// RAII scratch buffer (freed stream-ordered).
struct Scratch {
    void *p = nullptr;
    cudaStream_t s = nullptr;
    Scratch() = default;
    Scratch(const Scratch &) = delete;
    Scratch &operator=(const Scratch &) = delete;
    ~Scratch() { release(); }
    pg_status alloc(size_t bytes, cudaStream_t st) {
        release();
        s = st;
        return dalloc(&p, bytes ? bytes : 16, st);
    }
    void release() {
        if (p) dfree(p, s);
        p = nullptr;
    }
    template <class T>
    T *as() const { return reinterpret_cast<T *>(p); }
};

// ---------------------------------------------------------------- launches
void count_launch();
// Kernel timer bracket (active only while profiling is enabled).
struct KTimer {
    const char *name;
    cudaStream_t s;
    cudaEvent_t a = nullptr, b = nullptr;
    KTimer(const char *nm, cudaStream_t st);
    ~KTimer();
};
pg_status check_launch(const char *what);
// Copy up to 1024 bytes (whole words) of device memory to the host, in stream
// order, without a copy engine; synchronises the stream.
pg_status read_small(void *host_dst, const void *dev_src, size_t bytes, cudaStream_t s);

inline int ceil_div_i(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }
int num_sms();

// Programmatic dependent launch.  A kernel launched with launch_pdl may be
// scheduled while the kernel before it in the stream is still running; it
// calls pdl_wait() before touching anything, which returns once every kernel
// before it has completed and its writes are visible (a no-op for a normal
// launch).  pdl_trigger() then lets the kernel after it be scheduled early,
// so the launch latency between dependent kernels is hidden.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <class... Exp, class... Act>
cudaError_t launch_pdl(void (*kernel)(Exp...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Act &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<Exp>(args)...);
}

// ---------------------------------------------------------------- layout
// Coordinates stored per point: the dimension class DC >= dim (zero padded).
inline int dim_class(int dim) {
    if (dim <= 8) return dim < 2 ? 2 : dim;
    return dim <= 12 ? 12 : 16;
}
// float4 words per bucket entry: DC coordinates + the id.
__host__ __device__ constexpr int bucket_w(int dc) { return (dc + 1 + 3) / 4; }
// float4 words per node record: lo0, hi0, lo1, hi1 (DC each) + 4 ints.
__host__ __device__ constexpr int node_w(int dc) { return dc + 1; }

constexpr unsigned DEAD_ID = 0xFFFFFFFFu;

// Descriptor of one tree as seen by the traversal kernels.
struct TreeDesc {
    const float4 *bucket;
    const float4 *nodes;
    const int *parent;        // per node: 2*parent + side (-1 at the root); may be NULL
    const int *leaf_parent;   // per bucket entry: code of its leaf; may be NULL
    int root_ref;
    int root_cnt;   // >0 leaf root, 0 internal root, <0 empty / dead
    float root_lo[PG_MAX_DIM];
    float root_hi[PG_MAX_DIM];
};

// Result of building one tree inside one thread block.
struct CtaTree {
    int root_ref, root_cnt, nodes, depth;
};

// ---------------------------------------------------------------- float order
// Monotone map float -> int so that integer min/max order equals float order.
__device__ __forceinline__ int f2o(float f) {
    int i = __float_as_int(f);
    return i >= 0 ? i : (i ^ 0x7fffffff);
}
__device__ __forceinline__ float o2f(int i) { return __int_as_float(i >= 0 ? i : (i ^ 0x7fffffff)); }

// ---------------------------------------------------------------- distance
// Squared distance accumulated as one fixed chain of rounded operations so
// that a box lower bound (per-coordinate gaps no larger in magnitude) never
// exceeds the distance of a point inside the box: every step is monotone.
template <int DC>
__device__ __forceinline__ float sqdist(const float *a, const float *b) {
    float d0 = __fsub_rn(a[0], b[0]);
    float acc = __fmul_rn(d0, d0);
#pragma unroll
    for (int c = 1; c < DC; ++c) {
        float dc = __fsub_rn(a[c], b[c]);
        acc = __fmaf_rn(dc, dc, acc);
    }
    return acc;
}

template <int DC>
__device__ __forceinline__ float boxdist(const float *q, const float *lo, const float *hi) {
    float g0 = fmaxf(fmaxf(__fsub_rn(lo[0], q[0]), __fsub_rn(q[0], hi[0])), 0.f);
    float acc = __fmul_rn(g0, g0);
#pragma unroll
    for (int c = 1; c < DC; ++c) {
        float g = fmaxf(fmaxf(__fsub_rn(lo[c], q[c]), __fsub_rn(q[c], hi[c])), 0.f);
        acc = __fmaf_rn(g, g, acc);
    }
    return acc;
}

}  // namespace pg
