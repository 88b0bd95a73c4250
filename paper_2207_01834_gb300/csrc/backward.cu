// Gradient of the selected squared k-NN distances (not in the paper; the
// derivative of D(q, p) = |q - p|^2 written out):
//   L = sum_{i,j} g_ij * D(q_i, p_{idx_ij})
//   dL/dq_i = sum_j 2 g_ij (q_i - p_{idx_ij})
//   dL/dp_t = -sum_{(i,j): idx_ij = t} 2 g_ij (q_i - p_t)
// Only the indices are kept from the forward pass; distances are recomputed
// from the coordinates.  The query gradient is a per-query sum over its k
// slots in slot order.  The data gradient is a scatter; to make it bitwise
// deterministic the (index, pair) list is sorted stably by index and every
// data point sums its contributions in ascending pair order (no float
// atomics).
#include <algorithm>

#include "internal.h"
#include "sort.h"

namespace pg {

namespace {

constexpr int BT = 256;

// Coordinate loops run to the dimension class DC (compile time) and skip
// c >= dim, so registers and instructions follow the real dimension.
template <int DC>
__global__ void k_bwd_queries(const float *__restrict__ data, int64_t n, const float *__restrict__ queries, int64_t m,
                              int dim, int k, const int32_t *__restrict__ idx, const float *__restrict__ g,
                              float *__restrict__ gq) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    float q[DC], acc[DC];
#pragma unroll
    for (int c = 0; c < DC; ++c) {
        q[c] = c < dim ? queries[i * dim + c] : 0.f;
        acc[c] = 0.f;
    }
    for (int j = 0; j < k; ++j) {
        const int t = idx[i * k + j];
        if (t < 0 || t >= n) continue;   // padding (or out of range): no contribution
        const float w = 2.f * g[i * k + j];
#pragma unroll
        for (int c = 0; c < DC; ++c)
            if (c < dim) acc[c] = __fmaf_rn(w, __fsub_rn(q[c], data[(int64_t)t * dim + c]), acc[c]);
    }
#pragma unroll
    for (int c = 0; c < DC; ++c)
        if (c < dim) gq[i * dim + c] = acc[c];
}

// Sort keys: the data index, or n for padding slots (sorted last, ignored).
__global__ void k_bwd_keys(const int32_t *__restrict__ idx, int64_t P, uint32_t n, uint32_t *__restrict__ keys) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    const int t = idx[p];
    keys[p] = (t >= 0 && (uint32_t)t < n) ? (uint32_t)t : n;
}

__global__ void k_bwd_bounds(const uint32_t *__restrict__ skeys, int64_t P, uint32_t n, int *__restrict__ lo,
                             int *__restrict__ hi) {
    const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= P) return;
    const uint32_t key = skeys[x];
    if (key >= n) return;
    if (x == 0 || skeys[x - 1] != key) lo[key] = (int)x;
    if (x == P - 1 || skeys[x + 1] != key) hi[key] = (int)(x + 1);
}

template <int DC>
__global__ void k_bwd_data(const float *__restrict__ data, const float *__restrict__ queries, int64_t n, int dim,
                           int k, const uint32_t *__restrict__ svals, const float *__restrict__ g,
                           const int *__restrict__ lo, const int *__restrict__ hi, float *__restrict__ gp) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    float p[DC], acc[DC];
#pragma unroll
    for (int c = 0; c < DC; ++c) {
        p[c] = c < dim ? data[t * dim + c] : 0.f;
        acc[c] = 0.f;
    }
    const int a = lo[t], b = hi[t];
    for (int x = a; x < b; ++x) {
        const uint32_t pr = svals[x];
        const int64_t i = pr / (uint32_t)k;
        const float w = -2.f * g[pr];
#pragma unroll
        for (int c = 0; c < DC; ++c)
            if (c < dim) acc[c] = __fmaf_rn(w, __fsub_rn(queries[i * dim + c], p[c]), acc[c]);
    }
#pragma unroll
    for (int c = 0; c < DC; ++c)
        if (c < dim) gp[t * dim + c] = acc[c];
}

inline int grid_of(int64_t n) { return std::max(1, ceil_div_i(n, BT)); }

#define PG_DC_SWITCH(dim, CASE)                                                             \
    switch (dim_class(dim)) {                                                               \
        CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8) CASE(12) CASE(16)           \
        default: return fail(PG_EUNSUPPORTED, "dimension class");                          \
    }

pg_status launch_bwd_queries(const float *data, int64_t n, const float *queries, int64_t m, int dim, int k,
                             const int32_t *idx, const float *g, float *gq, cudaStream_t s) {
#define PG_CASE(D)                                                                                  \
    case D: k_bwd_queries<D><<<grid_of(m), BT, 0, s>>>(data, n, queries, m, dim, k, idx, g, gq); break;
    PG_DC_SWITCH(dim, PG_CASE)
#undef PG_CASE
    count_launch();
    return PG_OK;
}

pg_status launch_bwd_data(const float *data, const float *queries, int64_t n, int dim, int k, const uint32_t *sv,
                          const float *g, const int *lo, const int *hi, float *gp, cudaStream_t s) {
#define PG_CASE(D)                                                                                  \
    case D: k_bwd_data<D><<<grid_of(n), BT, 0, s>>>(data, queries, n, dim, k, sv, g, lo, hi, gp); break;
    PG_DC_SWITCH(dim, PG_CASE)
#undef PG_CASE
    count_launch();
    return PG_OK;
}

}  // namespace

// Scratch layout for the data gradient (P = m*k pairs): keys, vals, two
// temporaries (P each), segment bounds (2n).
size_t knn_backward_scratch_bytes(int64_t n, int64_t P) {
    return sizeof(uint32_t) * (size_t)(4 * P) + sizeof(int) * (size_t)(2 * n) + 256;
}

pg_status knn_backward_run(const float *data, int64_t n, const float *queries, int64_t m, int dim, int k,
                           const int32_t *idx, const float *g, float *gq, float *gp, void *scratch,
                           cudaStream_t s) {
    if (gq && m > 0) {
        PG_TRY(launch_bwd_queries(data, n, queries, m, dim, k, idx, g, gq, s));
    }
    if (gp && n > 0) {
        const int64_t P = m * k;
        uint32_t *keys = reinterpret_cast<uint32_t *>(scratch);
        uint32_t *vals = keys + P, *tk = vals + P, *tv = tk + P;
        int *lo = reinterpret_cast<int *>(tv + P), *hi = lo + n;
        PG_CUDA(cudaMemsetAsync(lo, 0, sizeof(int) * (size_t)(2 * n), s));
        uint32_t *sk = keys, *sv = vals;
        if (P > 0) {
            k_bwd_keys<<<grid_of(P), BT, 0, s>>>(idx, P, (uint32_t)n, keys);
            count_launch();
            int bits = 1;
            while (bits < 32 && ((uint64_t)1 << bits) <= (uint64_t)n) ++bits;   // keys in [0, n]
            PG_TRY(radix_sort_pairs(keys, vals, true, tk, tv, P, bits, s, &sk, &sv));
            k_bwd_bounds<<<grid_of(P), BT, 0, s>>>(sk, P, (uint32_t)n, lo, hi);
            count_launch();
        }
        KTimer kt("knn_backward_data", s);
        PG_TRY(launch_bwd_data(data, queries, n, dim, k, sv, g, lo, hi, gp, s));
    }
    return check_launch("knn backward");
}

// The same computation on caller-provided scratch (knn_backward_scratch_bytes
// plus radix_ws_words ints after it): no allocation.
pg_status knn_backward_run_ws(const float *data, int64_t n, const float *queries, int64_t m, int dim, int k,
                              const int32_t *idx, const float *g, float *gq, float *gp, void *scratch,
                              int *radix_ws, cudaStream_t s) {
    if (gq && m > 0) {
        PG_TRY(launch_bwd_queries(data, n, queries, m, dim, k, idx, g, gq, s));
    }
    if (gp && n > 0) {
        const int64_t P = m * k;
        uint32_t *keys = reinterpret_cast<uint32_t *>(scratch);
        uint32_t *vals = keys + P, *tk = vals + P, *tv = tk + P;
        int *lo = reinterpret_cast<int *>(tv + P), *hi = lo + n;
        PG_CUDA(cudaMemsetAsync(lo, 0, sizeof(int) * (size_t)(2 * n), s));
        uint32_t *sk = keys, *sv = vals;
        if (P > 0) {
            k_bwd_keys<<<grid_of(P), BT, 0, s>>>(idx, P, (uint32_t)n, keys);
            count_launch();
            int bits = 1;
            while (bits < 32 && ((uint64_t)1 << bits) <= (uint64_t)n) ++bits;
            PG_TRY(radix_sort_pairs_ws(keys, vals, true, tk, tv, P, bits, radix_ws, s, &sk, &sv));
            k_bwd_bounds<<<grid_of(P), BT, 0, s>>>(sk, P, (uint32_t)n, lo, hi);
            count_launch();
        }
        PG_TRY(launch_bwd_data(data, queries, n, dim, k, sv, g, lo, hi, gp, s));
    }
    return check_launch("knn backward");
}

}  // namespace pg

using namespace pg;

extern "C" pg_status pg_knn_backward(const float *data, int64_t n, const float *queries, int64_t m, int dim, int k,
                                     const int32_t *idx, const float *grad_dist, float *grad_queries,
                                     float *grad_data, void *stream) {
    if (k < 1 || k > PG_MAX_K) return fail(PG_EINVAL, "pg_knn_backward: k must be in [1, 64]");
    if (dim < 1 || dim > PG_MAX_DIM) return fail(PG_EINVAL, "pg_knn_backward: dim must be in [1, 16]");
    if (n < 0 || m < 0 || n >= ((int64_t)1 << 31) || m >= ((int64_t)1 << 31))
        return fail(PG_EINVAL, "pg_knn_backward: n and m must be in [0, 2^31)");
    if (m * (int64_t)k >= ((int64_t)1 << 31)) return fail(PG_EINVAL, "pg_knn_backward: m*k must be < 2^31");
    if (m > 0 && (!queries || !idx || !grad_dist)) return fail(PG_EINVAL, "pg_knn_backward: NULL input");
    if (n > 0 && !data && (grad_data || (m > 0 && grad_queries))) return fail(PG_EINVAL, "pg_knn_backward: NULL data");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    Scratch sc;
    if (grad_data && n > 0) PG_TRY(sc.alloc(knn_backward_scratch_bytes(n, m * (int64_t)k), s));
    return knn_backward_run(data, n, queries, m, dim, k, idx, grad_dist, grad_queries, grad_data, sc.p, s);
}
