// Internal structures and host-side launchers shared by the library's
// translation units.  Nothing here is part of the C ABI.
#pragma once

#include <vector>

#include "common.cuh"

struct pg_tree {
    int64_t n = 0;
    int dim = 0;
    int dc = 2;
    int leaf_size = 16;
    int num_nodes = 0;
    int node_cap = 0;
    int depth = 0;
    int root_ref = -1;
    int root_cnt = -1;           // >0 leaf root, 0 internal root, <0 empty
    float root_lo[PG_MAX_DIM] = {0};
    float root_hi[PG_MAX_DIM] = {0};
    float4 *bucket = nullptr;    // n * bucket_w(dc)
    float4 *nodes = nullptr;     // node_cap * node_w(dc)
    int *split_dim = nullptr;    // node_cap
    float *split_val = nullptr;  // node_cap
    int2 *node_range = nullptr;  // node_cap: bucket range [x, y) of the node
    int *parent = nullptr;       // node_cap: 2*parent_node + side, or -1 at the root
    int *leaf_parent = nullptr;  // n: the code of the leaf holding each bucket entry
    pg::TreeDesc *desc = nullptr;  // device copy of this tree's descriptor
    cudaStream_t stream = nullptr;
    int64_t live = 0;            // live points (BDL trees lose points on erase)
    // A build enqueued under stream capture leaves its root, depth, node count
    // and root box in device memory (meta); they are read back into the
    // fields above when a host-side call first needs them.
    int *meta = nullptr;
    bool meta_pending = false;
};

namespace pg {

// ---- runtime.cu
// Fill `words` 32-bit words with `value`, and store up to kStoreSmallBytes of
// host data into device memory, by kernels (stream-ordered; no copy engine, so
// neither waits behind a caller's bulk copy in flight).
constexpr size_t kStoreSmallBytes = 256;
pg_status fill_words(void *dst, uint32_t value, size_t words, cudaStream_t s);
pg_status store_small(void *dev_dst, const void *host_src, size_t bytes, cudaStream_t s);

// ---- scan.cu
// out[0..n] = exclusive prefix sums of in[0..n-1]; out[n] = total.
pg_status exclusive_scan(const int *in, int *out, int64_t n, cudaStream_t s);

// ---- build.cu
// Pack row-major points (n*dim) into bucket entries with ids (ids == NULL: i).
pg_status pack_points(const float *pts, const int32_t *ids, int64_t n, int dim, int dc,
                      float4 *out, cudaStream_t s);
// Gather rows of a row-major store by id list into bucket entries.
pg_status gather_points(const float *store, const int32_t *ids, int64_t n, int dim, int dc,
                        float4 *out, cudaStream_t s);
// Build a tree over packed bucket entries.  Takes ownership of `packed`
// (it becomes the tree's bucket array or is freed).
pg_status build_packed(float4 *packed, int64_t n, int dim, int leaf, cudaStream_t s, pg_tree *t);
void tree_release(pg_tree *t);
// Device-level splitting of many independent trees at once (build.cu).
// Tree t starts as the segment [t_start[t], t_end[t]) of P with tight box
// t_box[t*2*DC ...] (DC lows then DC highs, order-preserving ints); seg_of[i]
// must hold the tree of position i (-1 for unused positions).  `levels`
// levels are enqueued without host waits; segments of up to fin_max points,
// and at the last level every segment that could still split, go to the
// finisher list `fin` (start, end, parent, side, depth, lo, hi; fin_cap
// entries per field; parent -(t+2) marks the root of tree t).  A finisher
// segment [st, en) owns node slots [st, en) and must put its root in slot
// en - 1, which its parent record (or roots[2t], roots[2t+1] for a tree root)
// already names; level nodes get slots from node_off on.
// The control block holds the node count, the finisher count and the number
// of levels that moved points (its parity names the buffer that holds the
// final order: P if even).
struct ForestArgs {
    int64_t n;
    int ntrees, leaf, fin_max, levels, seg_cap, fin_cap, node_off;
    float4 *P, *Q;
    int *seg_of, *seg_of_nx;
    const int *t_start, *t_end, *t_box;
    float4 *nodes;
    int *n_sdim;
    float *n_sval;
    int2 *n_range;
    int *n_parent, *roots;
    // carved from one scratch block by forest_carve
    int *seg_a, *seg_b, *lvl, *fin, *ctl, *scan_ws;
    unsigned *tiles;
};
struct ForestCtl {
    int nb, fin, scatters;   // word indices in the control block
};
int64_t forest_words(int dc, int seg_cap, int fin_cap, int64_t n);
void forest_carve(ForestArgs &fa, int *words, int dc);
ForestCtl forest_ctl();
pg_status forest_levels(int dc, const ForestArgs &fa, cudaStream_t s);

pg_status tree_upload_desc(pg_tree *t);
TreeDesc tree_desc(const pg_tree *t);
// Words of a tree's device metadata block (see k_tree_meta in build.cu).
constexpr int kTreeMetaWords = 8 + 2 * PG_MAX_DIM;
// Read back the host-side metadata of a tree built under stream capture
// (waits for its stream); a no-op for other trees.
pg_status tree_sync_meta(pg_tree *t);

// ---- knn_dispatch.cu
// k-NN over `ntrees` trees described in device memory.  If self_bucket is not
// NULL the queries are the m bucket entries of that array and the output row
// is the entry's id; otherwise queries are row-major m*dim floats.
// order (may be NULL): processing order of the queries (a permutation of
// 0..m-1 that puts queries of the same leaf next to each other).
// start_leaf (may be NULL): per processing position, the bucket position in
// tree 0 of the leaf the query falls in; traversals that search from the
// bottom start there and then search the other trees from their roots.
// self_bucket may be given only with ntrees == 1; tree 0 must have its
// parent links (parent, leaf_parent) when either is given.
// variant: a PG_KNN_* traversal, or PG_KNN_AUTO for the automatic choice.
pg_status knn_launch(const TreeDesc *trees_dev, int ntrees, int dc, const float *queries,
                     const float4 *self_bucket, const int32_t *order, const int32_t *start_leaf, int64_t m,
                     int dim, int k, int32_t *out_idx, float *out_dist, int variant, cudaStream_t s);
int k_class(int k);
bool valid_variant(int v);
// The variant PG_KNN_AUTO resolves to for this thread and request.
int resolve_variant(int requested, int dc, int k, bool self);
// Internal launch code of the counting instance of the postponed-leaf kernel.
constexpr int kKnnCountingInstance = 100;

// ---- order.cu
// Queries sorted by the leaf of `t` they fall in (stable); order gets m ints.
// leaf_ref (may be NULL) gets, per sorted position, the bucket position of
// that query's leaf (m ints).
pg_status query_order(const pg_tree *t, const float *queries, int64_t m, int dim, int32_t *order, cudaStream_t s,
                      int32_t *leaf_ref = nullptr);
constexpr int64_t kOrderMinQueries = 4096;

}  // namespace pg
