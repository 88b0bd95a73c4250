// C ABI: static kd-tree build, k-NN query, export.
#include <cstring>
#include <new>

#include "internal.h"

namespace pg {
pg_status build_rows(const float *pts, int64_t n, int dim, int leaf, int rule, cudaStream_t s, pg_tree *t);
}

using namespace pg;

static pg_status check_dim(int dim) {
    if (dim < 1 || dim > PG_MAX_DIM) return fail(PG_EINVAL, "dim must be in [1, 16]");
    return PG_OK;
}

extern "C" {

pg_status pg_tree_build(const float *points, int64_t n, int dim, int leaf_size, void *stream, pg_tree **out) {
    return pg_tree_build_split(points, n, dim, leaf_size, PG_SPLIT_SPATIAL, stream, out);
}

pg_status pg_tree_build_split(const float *points, int64_t n, int dim, int leaf_size, int split_rule, void *stream,
                              pg_tree **out) {
    if (!out) return fail(PG_EINVAL, "pg_tree_build: out is NULL");
    if (split_rule != PG_SPLIT_SPATIAL && split_rule != PG_SPLIT_OBJECT)
        return fail(PG_EINVAL, "pg_tree_build_split: unknown split rule");
    *out = nullptr;
    PG_TRY(check_dim(dim));
    if (n < 0 || n >= (int64_t)1 << 31) return fail(PG_EINVAL, "pg_tree_build: n must be in [0, 2^31)");
    if (n > 0 && !points) return fail(PG_EINVAL, "pg_tree_build: points is NULL");
    if (leaf_size < 1 || leaf_size > PG_MAX_LEAF) return fail(PG_EINVAL, "pg_tree_build: leaf_size must be in [1, 256]");
    pg_tree *t = new (std::nothrow) pg_tree();
    if (!t) return fail(PG_ENOMEM, "pg_tree_build: host allocation");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    pg_status st = build_rows(points, n, dim, leaf_size, split_rule, s, t);
    if (st != PG_OK) {
        tree_release(t);
        delete t;
        return st;
    }
    *out = t;
    return PG_OK;
}

pg_status pg_knn(const pg_tree *tree, const float *queries, int64_t m, int k, int32_t *out_idx, float *out_dist,
                 void *stream) {
    return pg_knn_ex(tree, queries, m, k, PG_KNN_AUTO, out_idx, out_dist, stream);
}

pg_status pg_knn_ex(const pg_tree *tree, const float *queries, int64_t m, int k, int variant, int32_t *out_idx,
                    float *out_dist, void *stream) {
    if (!tree) return fail(PG_EINVAL, "pg_knn: tree is NULL");
    if (k < 1 || k > PG_MAX_K) return fail(PG_EINVAL, "pg_knn: k must be in [1, 64]");
    if (m < 0 || m >= (int64_t)1 << 31) return fail(PG_EINVAL, "pg_knn: m must be in [0, 2^31)");
    if (!queries && m != tree->n) return fail(PG_EINVAL, "pg_knn: all-kNN (queries == NULL) needs m == n");
    if (m > 0 && (!out_idx || !out_dist)) return fail(PG_EINVAL, "pg_knn: output pointer is NULL");
    if (!valid_variant(variant)) return fail(PG_EINVAL, "pg_knn: unknown traversal variant");
    if (m == 0) return PG_OK;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (tree->n == 0) {
        // Nothing to find: every slot is padding.
        return knn_launch(tree->desc, 1, tree->dc, queries, nullptr, nullptr, nullptr, m, tree->dim, k, out_idx,
                          out_dist, variant, s);
    }
    if (!queries)   // all-kNN: bucket order is already tree order
        return knn_launch(tree->desc, 1, tree->dc, nullptr, tree->bucket, nullptr, nullptr, m, tree->dim, k,
                          out_idx, out_dist, variant, s);
    // Queries sorted by the leaf they fall in: the processing order and, per
    // position, that leaf (where a bottom-up search starts).
    Scratch ord;
    const bool sorted = m >= kOrderMinQueries;
    if (sorted) {
        PG_TRY(ord.alloc(sizeof(int32_t) * (size_t)(2 * m), s));
        PG_TRY(query_order(tree, queries, m, tree->dim, ord.as<int32_t>(), s, ord.as<int32_t>() + m));
    }
    return knn_launch(tree->desc, 1, tree->dc, queries, nullptr, sorted ? ord.as<int32_t>() : nullptr,
                      sorted ? ord.as<int32_t>() + m : nullptr, m, tree->dim, k, out_idx, out_dist, variant, s);
}

pg_status pg_tree_free(pg_tree *tree) {
    if (!tree) return PG_OK;
    tree_release(tree);
    delete tree;
    return PG_OK;
}

pg_status pg_tree_info(const pg_tree *t, pg_tree_info_t *info) {
    if (!t || !info) return fail(PG_EINVAL, "pg_tree_info: NULL argument");
    PG_TRY(tree_sync_meta(const_cast<pg_tree *>(t)));
    memset(info, 0, sizeof(*info));
    info->n = t->n;
    info->dim = t->dim;
    info->dim_class = t->dc;
    info->leaf_size = t->leaf_size;
    info->num_nodes = t->num_nodes;
    info->depth = t->depth;
    info->node_floats = 4 * node_w(t->dc);
    info->point_floats = 4 * bucket_w(t->dc);
    info->root_ref = t->root_ref;
    info->root_cnt = t->root_cnt;
    for (int c = 0; c < PG_MAX_DIM; ++c) {
        info->root_lo[c] = t->root_lo[c];
        info->root_hi[c] = t->root_hi[c];
    }
    return PG_OK;
}

pg_status pg_tree_export(const pg_tree *t, float *nodes, int32_t *split_dim, float *split_val, float *bucket) {
    if (!t) return fail(PG_EINVAL, "pg_tree_export: tree is NULL");
    PG_TRY(tree_sync_meta(const_cast<pg_tree *>(t)));
    cudaStream_t s = t->stream;
    const size_t nn = (size_t)t->num_nodes;
    if (nodes && nn) PG_CUDA(cudaMemcpyAsync(nodes, t->nodes, sizeof(float4) * node_w(t->dc) * nn, cudaMemcpyDeviceToHost, s));
    if (split_dim && nn) PG_CUDA(cudaMemcpyAsync(split_dim, t->split_dim, sizeof(int) * nn, cudaMemcpyDeviceToHost, s));
    if (split_val && nn) PG_CUDA(cudaMemcpyAsync(split_val, t->split_val, sizeof(float) * nn, cudaMemcpyDeviceToHost, s));
    if (bucket && t->n) PG_CUDA(cudaMemcpyAsync(bucket, t->bucket, sizeof(float4) * bucket_w(t->dc) * (size_t)t->n, cudaMemcpyDeviceToHost, s));
    PG_CUDA(cudaStreamSynchronize(s));
    return PG_OK;
}

}  // extern "C"
