// Chooses the traversal kernel instance for a (dimension class, k) request.
#include "internal.h"

namespace pg {

#define PG_DECL(DCN)                                                                                      \
    pg_status knn_launch_dc##DCN(const TreeDesc *, int, const float *, const float4 *, const int32_t *,     \
                                 int64_t, int, int, int32_t *, float *, int, unsigned long long *,         \
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

static int g_variant = 0;   // 0 automatic, 1 thread per query, 2 warp packets, 3 postponed leaves
static bool g_touch = false;                   // count touched records / entries (postponed leaves)
static unsigned long long *g_touch_dev = nullptr;   // [node records, bucket entries] (one device)

void set_knn_variant(int v) { g_variant = v; }
// automatic: thread per query (measured faster on 3D all-kNN so far)
int knn_variant() { return g_variant == 0 ? 1 : g_variant; }

pg_status knn_launch(const TreeDesc *trees_dev, int ntrees, int dc, const float *queries,
                     const float4 *self_bucket, const int32_t *order, int64_t m, int dim, int k, int32_t *out_idx,
                     float *out_dist, cudaStream_t s) {
    if (m == 0) return PG_OK;
    int variant = knn_variant();
    if (g_touch && variant == 3) {
        if (!g_touch_dev) {
            PG_CUDA(cudaMalloc(&g_touch_dev, 2 * sizeof(unsigned long long)));
            PG_CUDA(cudaMemset(g_touch_dev, 0, 2 * sizeof(unsigned long long)));
        }
        variant = 4;   // the counting instance of the same traversal
    }
    unsigned long long *touch = g_touch_dev;
    switch (dc) {
        case 2: return knn_launch_dc2(trees_dev, ntrees, queries, self_bucket, order, m, dim, k, out_idx, out_dist, variant, touch, s);
        case 3: return knn_launch_dc3(trees_dev, ntrees, queries, self_bucket, order, m, dim, k, out_idx, out_dist, variant, touch, s);
        case 4: return knn_launch_dc4(trees_dev, ntrees, queries, self_bucket, order, m, dim, k, out_idx, out_dist, variant, touch, s);
        case 5: return knn_launch_dc5(trees_dev, ntrees, queries, self_bucket, order, m, dim, k, out_idx, out_dist, variant, touch, s);
        case 6: return knn_launch_dc6(trees_dev, ntrees, queries, self_bucket, order, m, dim, k, out_idx, out_dist, variant, touch, s);
        case 7: return knn_launch_dc7(trees_dev, ntrees, queries, self_bucket, order, m, dim, k, out_idx, out_dist, variant, touch, s);
        case 8: return knn_launch_dc8(trees_dev, ntrees, queries, self_bucket, order, m, dim, k, out_idx, out_dist, variant, touch, s);
        case 12: return knn_launch_dc12(trees_dev, ntrees, queries, self_bucket, order, m, dim, k, out_idx, out_dist, variant, touch, s);
        case 16: return knn_launch_dc16(trees_dev, ntrees, queries, self_bucket, order, m, dim, k, out_idx, out_dist, variant, touch, s);
        default: return fail(PG_EUNSUPPORTED, "dimension class");
    }
}

}  // namespace pg

extern "C" pg_status pg_knn_touch_enable(int on) {
    pg::g_touch = on != 0;
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
    if (variant < 0 || variant > 3) return pg::fail(PG_EINVAL, "pg_knn_set_variant: variant must be 0..3");
    pg::set_knn_variant(variant);
    return PG_OK;
}
