// Chooses the traversal kernel instance for a (dimension class, k) request.
//
// Every traversal variant returns the same exact answer (paper App. A.1.3:
// each query is searched independently), so the choice only changes speed.
// A call names its variant, or asks for the automatic one (PG_KNN_AUTO):
// then the calling thread's override (pg_knn_set_variant) applies if set,
// else the tune table entry for (dimension class, k class, all-kNN or
// separate queries) that an autotuner recorded (pg_knn_tune_set), else the
// built-in default.
#include <atomic>

#include "internal.h"

namespace pg {

#define PG_DECL(DCN)                                                                                      \
    pg_status knn_launch_dc##DCN(const TreeDesc *, int, const float *, const float4 *, const int32_t *,     \
                                 const int32_t *, int64_t, int, int, int32_t *, float *, int,              \
                                 unsigned long long *,                                                     \
                                 cudaStream_t);
PG_DECL(2) PG_DECL(3) PG_DECL(4) PG_DECL(5) PG_DECL(6) PG_DECL(7) PG_DECL(8) PG_DECL(12) PG_DECL(16)
#undef PG_DECL

int k_class(int k) {
    if (k <= 1) return 1;
    if (k <= 2) return 2;
    if (k <= 4) return 4;
    if (k <= 8) return 8;
    if (k <= 10) return 10;
    if (k <= 16) return 16;
    if (k <= 32) return 32;
    return 64;
}

namespace {

constexpr int kDcSlots = 9;   // dimension classes 2, 3, 4, 5, 6, 7, 8, 12, 16
constexpr int kKSlots = 8;    // k classes 1, 2, 4, 8, 10, 16, 32, 64

int dc_slot(int dc) {
    if (dc <= 8) return dc < 2 ? 0 : dc - 2;
    return dc <= 12 ? 7 : 8;
}
int k_slot(int k) {
    switch (k_class(k)) {
        case 1: return 0;
        case 2: return 1;
        case 4: return 2;
        case 8: return 3;
        case 10: return 4;
        case 16: return 5;
        case 32: return 6;
        default: return 7;
    }
}

thread_local int t_override = 0;                      // pg_knn_set_variant of this thread
std::atomic<int> g_tune[kDcSlots][kKSlots][2];         // 0: no entry (zero-initialised)
std::atomic<bool> g_touch{false};                      // count touched records / entries
unsigned long long *g_touch_dev = nullptr;             // [node records, bucket entries] (one device)

// Built-in choice when nothing else is set: the postponed-leaf traversal,
// the fastest measured variant on 2D-5D all-kNN and separate queries, with
// its k-list as a shared-memory heap for k > 16 (3D uniform, 2M points, 1M
// queries, k = 64: 7.2 against 10.2 ms); warp per query from 7 dimensions
// and k >= 16 (7D clustered, 1M queries: k = 16 28.3 against 32.9 ms, k = 64
// 55.6 against 107 ms) and from 5 dimensions and k > 32 (5D clustered, k = 64:
// 30.3 against 32.8 ms; all-kNN even).
int default_variant(int dc, int k, bool /*self*/) {
    if ((dc >= 7 && k >= 16) || (dc >= 5 && k > 32)) return PG_KNN_WARP;
    return k > 16 ? PG_KNN_POSTPONED_HEAP : PG_KNN_POSTPONED;
}

}  // namespace

bool valid_variant(int v) { return v >= PG_KNN_AUTO && v <= PG_KNN_POSTPONED_HEAP; }

int resolve_variant(int requested, int dc, int k, bool self) {
    if (requested != PG_KNN_AUTO) return requested;
    if (t_override != PG_KNN_AUTO) return t_override;
    const int v = g_tune[dc_slot(dc)][k_slot(k)][self ? 1 : 0].load(std::memory_order_relaxed);
    return v != PG_KNN_AUTO ? v : default_variant(dc, k, self);
}

pg_status knn_launch(const TreeDesc *trees_dev, int ntrees, int dc, const float *queries,
                     const float4 *self_bucket, const int32_t *order, const int32_t *start_leaf, int64_t m,
                     int dim, int k, int32_t *out_idx, float *out_dist, int requested, cudaStream_t s) {
    if (m == 0) return PG_OK;
    if (!valid_variant(requested)) return fail(PG_EINVAL, "k-NN: unknown traversal variant");
    int variant = resolve_variant(requested, dc, k, self_bucket != nullptr);
    if (g_touch.load() && (variant == PG_KNN_POSTPONED || variant == PG_KNN_POSTPONED_HEAP)) {
        if (!g_touch_dev) {
            PG_CUDA(cudaMalloc(&g_touch_dev, 2 * sizeof(unsigned long long)));
            PG_CUDA(cudaMemset(g_touch_dev, 0, 2 * sizeof(unsigned long long)));
        }
        variant = kKnnCountingInstance;   // the counting instance of the same traversal
    }
    unsigned long long *touch = g_touch_dev;
    switch (dc) {
        case 2: return knn_launch_dc2(trees_dev, ntrees, queries, self_bucket, order, start_leaf, m, dim, k, out_idx, out_dist, variant, touch, s);
        case 3: return knn_launch_dc3(trees_dev, ntrees, queries, self_bucket, order, start_leaf, m, dim, k, out_idx, out_dist, variant, touch, s);
        case 4: return knn_launch_dc4(trees_dev, ntrees, queries, self_bucket, order, start_leaf, m, dim, k, out_idx, out_dist, variant, touch, s);
        case 5: return knn_launch_dc5(trees_dev, ntrees, queries, self_bucket, order, start_leaf, m, dim, k, out_idx, out_dist, variant, touch, s);
        case 6: return knn_launch_dc6(trees_dev, ntrees, queries, self_bucket, order, start_leaf, m, dim, k, out_idx, out_dist, variant, touch, s);
        case 7: return knn_launch_dc7(trees_dev, ntrees, queries, self_bucket, order, start_leaf, m, dim, k, out_idx, out_dist, variant, touch, s);
        case 8: return knn_launch_dc8(trees_dev, ntrees, queries, self_bucket, order, start_leaf, m, dim, k, out_idx, out_dist, variant, touch, s);
        case 12: return knn_launch_dc12(trees_dev, ntrees, queries, self_bucket, order, start_leaf, m, dim, k, out_idx, out_dist, variant, touch, s);
        case 16: return knn_launch_dc16(trees_dev, ntrees, queries, self_bucket, order, start_leaf, m, dim, k, out_idx, out_dist, variant, touch, s);
        default: return fail(PG_EUNSUPPORTED, "dimension class");
    }
}

}  // namespace pg

extern "C" pg_status pg_knn_touch_enable(int on) {
    pg::g_touch.store(on != 0);
    return PG_OK;
}

extern "C" pg_status pg_knn_touch_read(int64_t *node_records, int64_t *bucket_entries) {
    if (!node_records || !bucket_entries) return pg::fail(PG_EINVAL, "pg_knn_touch_read: NULL argument");
    unsigned long long h[2] = {0, 0};
    if (pg::g_touch_dev) {
        PG_CUDA(cudaDeviceSynchronize());
        PG_CUDA(cudaMemcpy(h, pg::g_touch_dev, sizeof(h), cudaMemcpyDeviceToHost));
        PG_CUDA(cudaMemset(pg::g_touch_dev, 0, sizeof(h)));
    }
    *node_records = (int64_t)h[0];
    *bucket_entries = (int64_t)h[1];
    return PG_OK;
}

extern "C" pg_status pg_knn_set_variant(int variant) {
    if (!pg::valid_variant(variant)) return pg::fail(PG_EINVAL, "pg_knn_set_variant: unknown traversal variant");
    pg::t_override = variant;
    return PG_OK;
}

extern "C" pg_status pg_knn_tune_set(int dim, int k, int all_knn, int variant) {
    if (dim < 1 || dim > PG_MAX_DIM) return pg::fail(PG_EINVAL, "pg_knn_tune_set: dim must be in [1, 16]");
    if (k < 1 || k > PG_MAX_K) return pg::fail(PG_EINVAL, "pg_knn_tune_set: k must be in [1, 64]");
    if (!pg::valid_variant(variant)) return pg::fail(PG_EINVAL, "pg_knn_tune_set: unknown traversal variant");
    pg::g_tune[pg::dc_slot(pg::dim_class(dim))][pg::k_slot(k)][all_knn ? 1 : 0].store(variant);
    return PG_OK;
}

extern "C" pg_status pg_knn_tune_get(int dim, int k, int all_knn, int *variant) {
    if (!variant) return pg::fail(PG_EINVAL, "pg_knn_tune_get: variant is NULL");
    if (dim < 1 || dim > PG_MAX_DIM) return pg::fail(PG_EINVAL, "pg_knn_tune_get: dim must be in [1, 16]");
    if (k < 1 || k > PG_MAX_K) return pg::fail(PG_EINVAL, "pg_knn_tune_get: k must be in [1, 64]");
    *variant = pg::resolve_variant(PG_KNN_AUTO, pg::dim_class(dim), k, all_knn != 0);
    return PG_OK;
}
