/*
 * pargeo_gpu.h — C ABI of the GB300 (sm_103a) kd-tree / BDL-tree k-NN library.
 *
 * The library builds kd-trees over Euclidean point sets and answers batched
 * exact k-nearest-neighbour queries over one tree or over the BDL-tree's
 * log-structured forest of static trees (ParGeo, Wang et al., ESA 2022:
 * Section 5 and Appendix A).  It also provides the gradient of the selected
 * squared distances and a batched multi-cloud Chamfer path.
 *
 * Conventions shared by every call
 *   - Points are float32, row-major: point i occupies p[i*dim .. i*dim+dim-1].
 *     dim is 1..16.  Coordinates must be finite; squared distances must not
 *     overflow float32 (|coordinates| well below 1e18).
 *   - "device" pointers are CUDA device (or managed) memory of the current
 *     device; "host" pointers are ordinary CPU memory.  The caller owns every
 *     buffer it passes.  The library copies its inputs and never keeps a
 *     caller pointer after a call returns.
 *   - stream: a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Calls that take a stream are stream-ordered: they enqueue work and may
 *     return before it finishes; results are valid once the stream reaches
 *     them.  Some calls read small counts back to the host and therefore
 *     synchronise with the stream; each such call says so.
 *   - k-NN output: per query, k slots ordered by ascending (squared distance,
 *     index).  out_idx is the data row (trees) or the point id (BDL); out_dist
 *     is the squared Euclidean distance computed in float32.  When fewer than
 *     k points are available the remaining slots hold index -1 and +inf.
 *   - Errors: every call returns a pg_status.  On PG_EINVAL nothing was
 *     launched and the outputs are untouched.  pg_last_error() describes the
 *     last failure of the calling thread.
 */
#ifndef PARGEO_GPU_H
#define PARGEO_GPU_H

#include <stdint.h>

#if defined(__GNUC__)
#define PG_API __attribute__((visibility("default")))
#else
#define PG_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PG_OK = 0,
    PG_EINVAL = 1,        /* invalid argument (nothing launched)              */
    PG_ENOMEM = 2,        /* device or host allocation failed                 */
    PG_ECUDA = 3,         /* a CUDA runtime call failed                       */
    PG_ETIMEOUT = 4,      /* a bounded device-side wait gave up               */
    PG_EUNSUPPORTED = 5   /* valid request the library does not support       */
} pg_status;

typedef struct pg_tree pg_tree;   /* one static kd-tree (opaque)                */
typedef struct pg_bdl pg_bdl;     /* one BDL-tree forest (opaque)               */

/* Limits checked by every call. */
#define PG_MAX_DIM 16
#define PG_MAX_K 64
#define PG_MAX_LEAF 256
#define PG_DEPTH_CAP 48   /* nodes deeper than this become leaves              */

/* Split rules of pg_tree_build_split (paper Section 4: splits by spatial
 * median or by object median). */
#define PG_SPLIT_SPATIAL 0
#define PG_SPLIT_OBJECT 1

/* ------------------------------------------------------------------------
 * Static kd-tree (paper Section 5 intro; construction Appendix A.1.1).
 * ---------------------------------------------------------------------- */

/*
 * Build a kd-tree over n points (device, n*dim float32).  Every internal node
 * cuts its tight bounding box in half along its widest dimension (the paper's
 * spatial-median split, Section 6 "Construction"); a node with at most
 * leaf_size points, with all points equal, or at depth PG_DEPTH_CAP is a leaf.
 * n may be 0 (empty tree).  leaf_size in [1, PG_MAX_LEAF]; n < 2^31.
 * Synchronises with `stream` about twice per build (it reads the root box,
 * for the finite check, and the level loop's end flag once the expected
 * depth is reached), never once per level; the root record and the tree
 * descriptor are written on the device, and the tree's host-side fields
 * (pg_tree_info, pg_tree_export, range search, k-NN graph) are read back,
 * with a wait on the tree's stream, by the first such call.
 * Under stream capture (spatial-median split only) it waits on nothing: the
 * level loop is enqueued as a device-driven loop (a conditional WHILE node
 * of the graph being captured, its body captured from a side stream; capture
 * in thread-local or relaxed mode), the finisher takes its work count from
 * the device, and the descriptor is written by a kernel, so a build and the
 * k-NN calls on the tree can be captured into one CUDA graph and replayed on
 * new data of the same size.  The tree's host-side fields (pg_tree_info,
 * pg_tree_export, range search, k-NN graph) are read back, with a wait on
 * the tree's stream, by the first such call after the graph has run; a
 * non-finite coordinate is then reported by that call, not by the build.
 * On success *out receives a handle owned by the caller (free with
 * pg_tree_free).  Errors: PG_EINVAL, PG_ENOMEM, PG_ECUDA.
 */
PG_API pg_status pg_tree_build(const float *points, int64_t n, int dim, int leaf_size, void *stream,
                        pg_tree **out);

/*
 * As pg_tree_build with a choice of split rule (paper Section 4: the split is
 * by spatial median or by object median).  PG_SPLIT_SPATIAL is
 * pg_tree_build.  PG_SPLIT_OBJECT: the split dimension is the widest extent of
 * the node's tight box as before, and a node of c points sends its
 * floor(c / 2) smallest points along it to the left child (ties by bucket
 * position), so left coordinates <= split value <= right coordinates, where
 * the split value is the first right point's coordinate; the tree is
 * balanced.  k-NN answers do not depend on the rule.  Errors: as
 * pg_tree_build, and PG_EINVAL for another rule.
 */
PG_API pg_status pg_tree_build_split(const float *points, int64_t n, int dim, int leaf_size, int split_rule,
                                     void *stream, pg_tree **out);

/* Traversal kernels of the k-NN calls (paper App. A.1.3 searches every query
 * independently; every variant returns the same exact answer, bit for bit,
 * so the choice changes only speed):
 *   PG_KNN_THREAD     one thread per query walks its own path;
 *   PG_KNN_PACKET     the 32 queries of a warp, adjacent in tree order, share
 *                     one walk and every lane scans every leaf any of them
 *                     needs;
 *   PG_KNN_POSTPONED  one thread per query with postponed leaves: lanes walk
 *                     nodes until each holds a leaf, then scan their leaves
 *                     together;
 *   PG_KNN_WARP       one warp per query: the lanes split each leaf's points
 *                     and expand up to 32 nodes at a time, the k-list is
 *                     spread over the lanes (one or two keys each) and
 *                     merged by ballot and shuffle; for higher dimensions
 *                     and large k;
 *   PG_KNN_POSTPONED_HEAP  PG_KNN_POSTPONED with the k-list of each query
 *                     kept as a binary max-heap in shared memory (k >= 11:
 *                     lists of 16, 32 or 64 slots) instead of a sorted
 *                     register list: an insertion costs about log2(k)
 *                     steps instead of one per slot; smaller k is
 *                     PG_KNN_POSTPONED itself;
 *   PG_KNN_AUTO       the calling thread's pg_knn_set_variant choice if set,
 *                     else the tune table entry for the request's dimension
 *                     class, k class and kind (all-kNN or separate queries)
 *                     (pg_knn_tune_set), else PG_KNN_WARP for dimension
 *                     classes from 7 with k >= 16 and from 5 with k > 32,
 *                     PG_KNN_POSTPONED_HEAP for other k > 16 and
 *                     PG_KNN_POSTPONED otherwise. */
#define PG_KNN_AUTO 0
#define PG_KNN_THREAD 1
#define PG_KNN_PACKET 2
#define PG_KNN_POSTPONED 3
#define PG_KNN_WARP 4
#define PG_KNN_POSTPONED_HEAP 5

/*
 * Exact k-NN of m query points (device, m*dim float32) against the tree's
 * points (paper Appendix A.1.3, "Data-Parallel k-NN": every query searched
 * independently; subtrees whose bounding box is farther than the current k-th
 * distance are pruned).  queries == NULL means all-kNN: the queries are the
 * tree's own points and m must equal the tree's n; row i of the output then
 * belongs to input point i (each point finds itself at distance 0).
 * out_idx (device, m*k int32) and out_dist (device, m*k float32).
 * k in [1, PG_MAX_K].  The traversal is PG_KNN_AUTO's choice.
 * Stream-ordered, no synchronisation.  Separate queries (m >= 4096) are first
 * ordered by the leaf they fall in (scratch of 8 * m bytes), so that a warp's
 * queries are neighbours.  Errors: PG_EINVAL, PG_ENOMEM, PG_ECUDA.
 */
PG_API pg_status pg_knn(const pg_tree *tree, const float *queries, int64_t m, int k, int32_t *out_idx,
                 float *out_dist, void *stream);

/* pg_knn with the traversal named per call (a PG_KNN_* value): two threads,
 * or two trees, can use different variants at once.  Errors: as pg_knn, and
 * PG_EINVAL for an unknown variant. */
PG_API pg_status pg_knn_ex(const pg_tree *tree, const float *queries, int64_t m, int k, int variant,
                           int32_t *out_idx, float *out_dist, void *stream);

/* Release a tree.  Work that uses the tree must be ordered before this call on
 * the tree's build stream.  NULL is accepted. */
PG_API pg_status pg_tree_free(pg_tree *tree);

/* Shape of a built tree, for export and inspection. */
typedef struct {
    int64_t n;           /* number of points                                   */
    int32_t dim;         /* coordinate count of the input                      */
    int32_t dim_class;   /* DC: coordinates stored per point (>= dim, padded 0)*/
    int32_t leaf_size;
    int32_t num_nodes;   /* node slots (some may be unused: cnt fields -1)     */
    int32_t depth;       /* deepest leaf                                       */
    int32_t node_floats; /* 32-bit words per node record = 4*DC + 4            */
    int32_t point_floats;/* 32-bit words per bucket entry = 4*ceil((DC+1)/4)   */
    int32_t root_ref;    /* root child reference (see pg_tree_export)          */
    int32_t root_cnt;
    float root_lo[PG_MAX_DIM]; /* tight box of all points (first dim entries)  */
    float root_hi[PG_MAX_DIM];
} pg_tree_info_t;

PG_API pg_status pg_tree_info(const pg_tree *tree, pg_tree_info_t *info);

/*
 * Copy a tree's layout to host memory (synchronises with the tree's stream).
 *   nodes      num_nodes * node_floats words.  Node record: float lo0[DC],
 *              hi0[DC], lo1[DC], hi1[DC] (the tight boxes of the two children),
 *              then int32 ref0, cnt0, ref1, cnt1.  cnt > 0: the child is a leaf
 *              holding bucket entries [ref, ref+cnt); cnt == 0: the child is
 *              the internal node `ref`; cnt < 0: the child holds no live point.
 *   split_dim  num_nodes int32 and split_val num_nodes float32: the node sends
 *              x with x[split_dim] < split_val to child 0, the rest to child 1.
 *   bucket     n * point_floats words: coordinates (DC floats, zero padded)
 *              with the point's index (int32 bits) at word DC.
 * Any of the pointers may be NULL to skip that array.
 */
PG_API pg_status pg_tree_export(const pg_tree *tree, float *nodes, int32_t *split_dim, float *split_val,
                         float *bucket);

/*
 * k-NN graph of the tree's points (paper Section 4, geometric graph
 * generators: the k-NN graph comes from the kd-tree's k-NN search).  Point i is
 * joined to its k nearest OTHER points, i.e. the k smallest (squared distance,
 * row) pairs over rows != i; edges are undirected, each listed once as
 * (u, v) with u < v, all sorted by (u, v).  Rows are the tree's input rows.
 *   k          1..63.
 *   capacity   edges out_edges can hold (int32 pairs); n * k always suffices.
 *   out_edges  device, 2 * capacity int32 (u0, v0, u1, v1, ...), or NULL to
 *              only count.
 *   out_count  host: the number of edges (written even when the edges are
 *              not, so a caller can size a second call).
 * Stream-ordered; synchronises the stream once to read the count.  Errors:
 * PG_EINVAL (NULL tree/out_count, k or capacity out of range, n * k >= 2^31,
 * or capacity below the edge count with out_edges given: nothing written);
 * PG_ENOMEM for scratch (about 40 * n * k bytes).
 */
PG_API pg_status pg_knn_graph(const pg_tree *tree, int k, int64_t capacity, int32_t *out_edges,
                              int64_t *out_count, void *stream);

/*
 * Range search (paper Section 4: the kd-tree supports k-NN and range search;
 * Table 1 "kd-tree Range Search").  For each query q, every point p of the
 * tree with D(q, p) <= radius^2, D the squared Euclidean distance in float32
 * (the same rounded chain as pg_knn) and radius^2 rounded to float32 once.
 *   queries      device, m * dim row-major float32, or NULL for the tree's own
 *                points (then m must equal n and row i is input row i).
 *   radius       finite, >= 0.
 *   capacity     int32 slots in out_idx.
 *   out_idx      device, the concatenated result rows (tree input rows), or
 *                NULL to compute only the offsets.  Row order: the order of
 *                the tree walk (deterministic for a given tree and query).
 *   out_offsets  device, m + 1 int64: query i's points are
 *                out_idx[out_offsets[i] .. out_offsets[i+1]).
 *   out_total    host: the number of results (written before any capacity
 *                error, so a caller can size a second call).
 * Stream-ordered; synchronises the stream once to read the total.  Errors:
 * PG_EINVAL (NULL tree/out_offsets/out_total, m out of [0, 2^31), queries
 * NULL with m != n, radius negative or not finite, more than 2^31 - 2
 * results, or capacity below the total with out_idx given: offsets written,
 * indices not); PG_ENOMEM for scratch (8 * m + 4 * m bytes).
 */
PG_API pg_status pg_range(const pg_tree *tree, const float *queries, int64_t m, float radius, int64_t capacity,
                          int32_t *out_idx, int64_t *out_offsets, int64_t *out_total, void *stream);

/*
 * Range search, second half: writes the result rows of the search that a
 * pg_range call with out_idx == NULL sized (same tree, queries, m and radius)
 * from the offsets that call returned, without counting again.  Same rows as
 * pg_range with out_idx would write.
 *   offsets      device, m + 1 int64, as pg_range wrote them.
 *   capacity     int32 slots in out_idx (at least offsets[m]).
 *   out_idx      device; row i goes to out_idx[offsets[i] .. offsets[i+1]).
 * Nothing is written outside a row's own offsets or at or above capacity,
 * whatever the offsets hold.  Stream-ordered; synchronises the stream once to
 * read the row check.  Errors: PG_EINVAL (NULL tree, NULL offsets or out_idx
 * with m > 0 and n > 0, m out of [0, 2^31), queries NULL with m != n, radius
 * negative or not finite, capacity < 0, or a row whose point count differs
 * from its offsets or does not fit below capacity: the offsets do not belong
 * to this search, and such rows are incomplete); PG_ENOMEM for scratch
 * (4 * m + 4 bytes).
 */
PG_API pg_status pg_range_fill(const pg_tree *tree, const float *queries, int64_t m, float radius,
                               const int64_t *offsets, int64_t capacity, int32_t *out_idx, void *stream);

/*
 * The calling thread's traversal override: every later PG_KNN_AUTO request of
 * this thread (pg_knn, pg_bdl_knn, pg_knn_graph, and the *_ex calls given
 * PG_KNN_AUTO) uses `variant`; PG_KNN_AUTO clears it.  Other threads are not
 * affected.  Errors: PG_EINVAL for an unknown variant.
 */
PG_API pg_status pg_knn_set_variant(int variant);

/*
 * Tune table of PG_KNN_AUTO (process-wide, safe to call from any thread):
 * requests whose dimension class (dim 1-2, 3, ..., 8, 9-12, 13-16), k class
 * (1, 2, 3-4, 5-8, 9-10, 11-16, 17-32, 33-64) and kind (all_knn != 0: the
 * tree's own points; 0: separate queries) match use `variant`; PG_KNN_AUTO
 * removes the entry.  An autotuner that timed the variants on its workload
 * records its choice here.  pg_knn_tune_get returns the variant a
 * PG_KNN_AUTO request of the calling thread resolves to.  Errors: PG_EINVAL
 * for dim, k or variant out of range or a NULL output.
 */
PG_API pg_status pg_knn_tune_set(int dim, int k, int all_knn, int variant);
PG_API pg_status pg_knn_tune_get(int dim, int k, int all_knn, int *variant);

/*
 * Touched-bytes counters of the traversal (measurement only; no counterpart in
 * the paper).  While enabled (on != 0), every later PG_KNN_POSTPONED or
 * PG_KNN_POSTPONED_HEAP launch in this process runs an instance of the
 * postponed-leaf kernel (register k-list; both lists hold the same pairs at
 * every step, so both walk alike) that also counts, over all its queries, the
 * node records and the bucket entries it loads; the answer is unchanged.  pg_knn_touch_read synchronises the device, returns the counts
 * accumulated since the last read (zeros if nothing was counted) and resets
 * them.  Bytes: node_records * 16 * (DC + 1), bucket_entries * 16 *
 * ceil((DC + 1) / 4), DC the dimension class.  The counters live on the device
 * current at the first counted launch.  Errors: PG_EINVAL for NULL outputs.
 */
PG_API pg_status pg_knn_touch_enable(int on);
PG_API pg_status pg_knn_touch_read(int64_t *node_records, int64_t *bucket_entries);

/* ------------------------------------------------------------------------
 * BDL-tree (paper Section 5; Appendix A.2 Insert_L, A.3 Erase_L, A.4 kNN_L).
 * A forest of static kd-trees in slots i = 0, 1, ... with capacity
 * 2^i * buffer_size plus a buffer tree of capacity buffer_size.
 * All BDL calls run on the stream given to pg_bdl_create and synchronise with
 * it (they read counts back to drive the forest bookkeeping).
 * ---------------------------------------------------------------------- */

/* Create an empty forest.  dim in [1,16], buffer_size (X) >= 1,
 * leaf_size in [1, PG_MAX_LEAF]. */
PG_API pg_status pg_bdl_create(int dim, int64_t buffer_size, int leaf_size, void *stream, pg_bdl **out);

/*
 * Insert a batch of cnt points (device, cnt*dim float32) with Insert_L: the
 * batch's cnt mod X last points go to the buffer tree; if the buffer then
 * holds X or more points its X smallest ids join the batch; the full-tree
 * bitmask becomes F + floor(cnt/X) (+1 on buffer overflow); trees whose bit
 * clears are destroyed and their live points, with the batch, rebuild the
 * trees whose bit sets, lowest slot first, each filled to capacity, the
 * highest new slot taking what remains.
 * Points receive consecutive ids in input order, continuing from earlier
 * inserts; out_ids (device, cnt int32, may be NULL) receives them.
 * All or nothing: every new tree is built before the forest changes, so on
 * an error (PG_ENOMEM, PG_ECUDA) the forest holds what it held before the
 * call and the next insert hands out the same ids.
 */
PG_API pg_status pg_bdl_insert(pg_bdl *bdl, const float *points, int64_t cnt, int32_t *out_ids);

/*
 * Erase with Erase_L: every live point whose coordinates are bitwise equal to
 * one of the cnt points (device, cnt*dim float32) is removed from its tree;
 * then every tree left with fewer than half of its capacity is destroyed and
 * its live points are reinserted with Insert_L (the buffer tree is exempt).
 * Points not present are ignored.  On an error the erase has either removed
 * nothing or removed every match (queries are exact either way); in the
 * second case a failed reinsertion leaves the under-full trees in place and
 * erasing the same points again is harmless.
 */
PG_API pg_status pg_bdl_erase(pg_bdl *bdl, const float *points, int64_t cnt);

/*
 * Exact k-NN of m queries over the whole forest: one k-buffer per query is
 * carried across every non-empty tree (kNN_L), so the answer is the k-NN of
 * the live point set.  out_idx holds point ids.  Arguments as in pg_knn
 * (queries must not be NULL); the traversal is PG_KNN_AUTO's choice.
 */
PG_API pg_status pg_bdl_knn(const pg_bdl *bdl, const float *queries, int64_t m, int k, int32_t *out_idx,
                     float *out_dist);

/* pg_bdl_knn with the traversal named per call (a PG_KNN_* value). */
PG_API pg_status pg_bdl_knn_ex(const pg_bdl *bdl, const float *queries, int64_t m, int k, int variant,
                               int32_t *out_idx, float *out_dist);

/* Number of live points. */
PG_API pg_status pg_bdl_size(const pg_bdl *bdl, int64_t *live);

/*
 * Forest bookkeeping, to host memory: *F = bitmask of occupied slots,
 * slot_live[i] (64 entries) = live points of slot i (0 when empty),
 * *buffer_live = live points in the buffer tree, *next_id = ids handed out.
 */
PG_API pg_status pg_bdl_structure(const pg_bdl *bdl, uint64_t *F, int64_t *slot_live,
                           int64_t *buffer_live, int64_t *next_id);

/* Where every id lives, to host memory (next_id int8 entries): slot index,
 * -2 for the buffer tree, -1 for erased ids. */
PG_API pg_status pg_bdl_slot_of(const pg_bdl *bdl, int8_t *slot_of);

PG_API pg_status pg_bdl_free(pg_bdl *bdl);

/* ------------------------------------------------------------------------
 * Gradient (not in the paper: derivative of the selected squared distances).
 * ---------------------------------------------------------------------- */

/*
 * For L = sum_{i<m, j<k} grad_dist[i*k+j] * |q_i - p_{idx[i*k+j]}|^2:
 *   grad_queries[i]  = sum_j 2 g_ij (q_i - p_idx(i,j))            (m*dim)
 *   grad_data[t]     = -sum_{(i,j): idx_ij = t} 2 g_ij (q_i - p_t) (n*dim)
 * Distances are recomputed from the coordinates (float32).  Entries with
 * idx < 0 (padding) or idx >= n are skipped.  grad_data is summed per data point in ascending
 * (i, j) order after a stable sort by index, so the result is bitwise
 * deterministic.  All pointers are device memory; either gradient may be
 * NULL.  Outputs are overwritten (not accumulated).  Stream-ordered.
 */
PG_API pg_status pg_knn_backward(const float *data, int64_t n, const float *queries, int64_t m, int dim,
                          int k, const int32_t *idx, const float *grad_dist, float *grad_queries,
                          float *grad_data, void *stream);

/*
 * pg_knn_backward_noalloc — the paper has no counterpart (library service).
 * Same inputs, outputs and results as pg_knn_backward, computed without any
 * device allocation, for callers that cannot let a library allocate GPU
 * memory: applications that reserve all device memory for their own pool at
 * start-up, processes under a hard memory cap, and loops that must not pay
 * for or synchronise on an allocation.  It works in one statically sized
 * __device__ array (about 25 MiB) that stays resident on every GPU that loads
 * the library until the process exits, and calls no cudaMalloc, cudaFree or
 * allocating library routine.
 * Limits: n <= 1,048,576 data points and m*k <= 1,048,576 (query, neighbour)
 * pairs; larger requests return PG_EINVAL and launch nothing.
 * All calls share the array: calls whose GPU work overlaps (for example on two
 * streams at once) race and must be serialised by the caller.  Outside stream
 * capture every call looks up the array's device address with the calling
 * thread's device current; under capture the address found by the last
 * uncaptured call on that device is reused, so make the first call on a
 * device, and the first after a device reset, before any capture (a captured
 * first call returns PG_EINVAL).  One context per device is assumed: the
 * runtime's primary context.  Stream-ordered otherwise.
 */
PG_API pg_status pg_knn_backward_noalloc(const float *data, int64_t n, const float *queries, int64_t m,
                                         int dim, int k, const int32_t *idx, const float *grad_dist,
                                         float *grad_queries, float *grad_data, void *stream);

/* ------------------------------------------------------------------------
 * Batched multi-cloud Chamfer path (not in the paper: many uneven point
 * clouds built and queried in one persistent launch over a work queue).
 * ---------------------------------------------------------------------- */

/*
 * npairs cloud pairs.  a (device, a_off[npairs]*dim) holds the A clouds back
 * to back; a_off (HOST, npairs+1 int64) their row offsets; likewise b/b_off.
 * For every pair i and both directions it finds the k nearest neighbours of
 * each point of A_i in B_i and of each point of B_i in A_i, and writes
 *   loss[i]  (device, npairs float32) = sum of the selected squared distances
 *   idx_ab   (device, |a|*k int32)   neighbour rows local to B_i
 *   idx_ba   (device, |b|*k int32)   neighbour rows local to A_i
 *   dist_ab / dist_ba (device float32, same shapes; may be NULL)
 * leaf_size as in pg_tree_build.  Each cloud must hold >= 1 point.
 * One persistent kernel builds every cloud's kd-tree and answers every query
 * chunk from a work queue (builds first, largest first; a query chunk waits,
 * bounded, for its two trees).  The plan (layout, queue, a CUDA graph of the
 * launch sequence) is cached per (offsets, dim, k, leaf_size); each call
 * replays the graph on `stream` and synchronises once to read the wait
 * status.  Calls from several host threads run one at a time (the cached
 * plans' buffers are shared).  Errors: PG_EINVAL, PG_ENOMEM, PG_ECUDA,
 * PG_ETIMEOUT (a wait gave up).
 */
PG_API pg_status pg_batched_chamfer(const float *a, const int64_t *a_off, const float *b,
                             const int64_t *b_off, int npairs, int dim, int k, int leaf_size,
                             float *loss, int32_t *idx_ab, int32_t *idx_ba, float *dist_ab,
                             float *dist_ba, void *stream);

/*
 * Backward twin: given upstream dL/dloss[i] (device, npairs float32) and the
 * indices written by pg_batched_chamfer, writes grad_a (|a|*dim) and grad_b
 * (|b|*dim), float32, device, deterministic as in pg_knn_backward.
 */
PG_API pg_status pg_batched_chamfer_backward(const float *a, const int64_t *a_off, const float *b,
                                      const int64_t *b_off, int npairs, int dim, int k,
                                      const int32_t *idx_ab, const int32_t *idx_ba,
                                      const float *grad_loss, float *grad_a, float *grad_b,
                                      void *stream);

/* ------------------------------------------------------------------------
 * Diagnostics.
 * ---------------------------------------------------------------------- */

/* Message of the calling thread's last failure ("" if none). */
PG_API const char *pg_last_error(void);

/* Library version string. */
PG_API const char *pg_version(void);

/* Number of kernels this library has launched in this process. */
PG_API uint64_t pg_launch_count(void);

/*
 * Kernel timing: while enabled, the library brackets each launch of the
 * kernels it times with CUDA events on the launching stream.
 * pg_profile_read synchronises, then returns the summed milliseconds and the
 * launch count recorded for kernels whose name starts with `prefix`, and
 * clears them.
 */
PG_API pg_status pg_profile_enable(int on);
PG_API pg_status pg_profile_read(const char *prefix, double *total_ms, int64_t *launches);

/* Fault injection for tests: the n-th device allocation from now fails with
 * PG_ENOMEM (n <= 0 disables).  Host-side only; no GPU fault is involved. */
PG_API pg_status pg_debug_fail_alloc_after(int n);

/*
 * Fault injection for tests of the batched path's bounded waits: with
 * skip_publish != 0 the build items never set their ready flags, so every
 * query item waits until `wait_limit` spins (about 100 ns each; <= 0 restores
 * the default of about two seconds) and pg_batched_chamfer returns
 * PG_ETIMEOUT.  No GPU fault is involved.
 */
PG_API pg_status pg_debug_batched_faults(int skip_publish, long long wait_limit);

#ifdef __cplusplus
}
#endif

#endif /* PARGEO_GPU_H */
