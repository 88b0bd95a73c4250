// Range search on the kd-tree (paper Section 4: the kd-tree supports k-NN and
// range search; Table 1 "kd-tree Range Search").  A query (q, r) returns every
// point p with D(q, p) <= r^2, D the squared Euclidean distance computed in
// float32 with the same chain of rounded operations as the k-NN search, and
// r^2 rounded to float32 once.
//
// One thread per query walks the tree depth first and enters a child when its
// tight box lies within r^2 (the box distance never exceeds the distance of
// a point inside the box, so nothing inside the ball is skipped).  Two passes
// make the output deterministic without atomics: the first counts each
// query's points, an exclusive scan turns the counts into row offsets, and
// the second writes each row's indices in the order of the walk.  The fill
// pass writes a row only inside its offsets and below the capacity, and flags
// a row whose count differs from them, so offsets from another call can
// never make it write out of bounds.
#include <algorithm>

#include "internal.h"
#include "knn_kernel.cuh"

namespace pg {

namespace {

constexpr int RT = 128;

template <int DC, bool FILL>
__global__ void __launch_bounds__(RT) k_range(const TreeDesc *__restrict__ trees, const float *__restrict__ queries,
                                              const float4 *__restrict__ self_bucket,
                                              const int32_t *__restrict__ order, int64_t m, int dim, float r2,
                                              int *__restrict__ counts, const int64_t *__restrict__ offs,
                                              int64_t capacity, int32_t *__restrict__ out_idx,
                                              int *__restrict__ bad) {
    const int64_t pos = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (pos >= m) return;
    constexpr int NW = node_w(DC);
    const TreeDesc &T = trees[0];
    float q[DC];
    int64_t row;
    if (self_bucket) {
        unsigned qid;
        load_point<DC>(self_bucket, pos, q, qid);
        row = qid;
    } else {
        row = order ? (int64_t)order[pos] : pos;
#pragma unroll
        for (int c = 0; c < DC; ++c) q[c] = c < dim ? queries[row * dim + c] : 0.f;
    }
    int64_t found = 0, o0 = 0, o1 = 0, lim = 0;
    if (FILL) {
        o0 = offs[row];
        o1 = offs[row + 1];
        lim = o0 < 0 ? 0 : max((int64_t)0, min(o1, capacity) - o0);
    }
    auto scan = [&](int ref, int cnt) {
        for (int i = ref; i < ref + cnt; ++i) {
            float p[DC];
            unsigned pid;
            load_point<DC>(T.bucket, i, p, pid);
            if (sqdist<DC>(q, p) <= r2) {
                if (FILL && found < lim) out_idx[o0 + found] = (int32_t)pid;
                ++found;
            }
        }
    };
    if (T.root_cnt >= 0) {
        float rlo[DC], rhi[DC];
#pragma unroll
        for (int c = 0; c < DC; ++c) { rlo[c] = T.root_lo[c]; rhi[c] = T.root_hi[c]; }
        if (boxdist<DC>(q, rlo, rhi) <= r2) {
            if (T.root_cnt > 0) {
                scan(T.root_ref, T.root_cnt);
            } else {
                int stack[KNN_STACK];
                int sp = 0;
                stack[sp++] = T.root_ref;
                while (sp > 0) {
                    const int ref = stack[--sp];
                    float rec[4 * NW];
                    const float4 *np = T.nodes + (size_t)ref * NW;
#pragma unroll
                    for (int w = 0; w < NW; ++w) {
                        const float4 f = __ldg(np + w);
                        rec[4 * w] = f.x; rec[4 * w + 1] = f.y; rec[4 * w + 2] = f.z; rec[4 * w + 3] = f.w;
                    }
                    const int *ri = reinterpret_cast<const int *>(rec + 4 * DC);
                    // right child first on the stack so the left one is walked first
#pragma unroll
                    for (int ch = 1; ch >= 0; --ch) {
                        const int r = ri[2 * ch], c = ri[2 * ch + 1];
                        if (c < 0 || boxdist<DC>(q, rec + 2 * ch * DC, rec + 2 * ch * DC + DC) > r2) continue;
                        if (c > 0) scan(r, c);
                        else if (sp < KNN_STACK) stack[sp++] = r;
                    }
                }
            }
        }
    }
    if (!FILL) counts[row] = (int)found;
    else if (bad && (found != o1 - o0 || found > lim)) atomicExch(bad, 1);
}

__global__ void k_range_total(const int *__restrict__ counts, int64_t m, unsigned long long *__restrict__ total) {
    unsigned long long t = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
        t += (unsigned)counts[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(total, t);
}

__global__ void k_range_offsets(const int *__restrict__ pre, int64_t m, int64_t *__restrict__ offsets) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i <= m) offsets[i] = pre[i];
}

// One pass: fill == false counts each query's points into counts; fill ==
// true writes the rows given by offs (m + 1 int64) into out_idx.
struct RangePass {
    int *counts = nullptr;
    const int64_t *offs = nullptr;
    int64_t capacity = 0;
    int32_t *out_idx = nullptr;
    int *bad = nullptr;
    bool fill = false;
};

template <int DC>
pg_status range_pass(const pg_tree *t, const float *queries, const int32_t *order, int64_t m, float r2,
                     const RangePass &a, cudaStream_t s) {
    const int grid = std::max(1, ceil_div_i(m, RT));
    const float4 *self = queries ? nullptr : t->bucket;
    if (a.fill)
        k_range<DC, true><<<grid, RT, 0, s>>>(t->desc, queries, self, order, m, t->dim, r2, a.counts, a.offs,
                                               a.capacity, a.out_idx, a.bad);
    else
        k_range<DC, false><<<grid, RT, 0, s>>>(t->desc, queries, self, order, m, t->dim, r2, a.counts, a.offs,
                                                a.capacity, a.out_idx, a.bad);
    count_launch();
    return check_launch("range search");
}

pg_status range_dispatch(const pg_tree *t, const float *queries, const int32_t *order, int64_t m, float r2,
                         const RangePass &a, cudaStream_t s) {
    switch (t->dc) {
        case 2: return range_pass<2>(t, queries, order, m, r2, a, s);
        case 3: return range_pass<3>(t, queries, order, m, r2, a, s);
        case 4: return range_pass<4>(t, queries, order, m, r2, a, s);
        case 5: return range_pass<5>(t, queries, order, m, r2, a, s);
        case 6: return range_pass<6>(t, queries, order, m, r2, a, s);
        case 7: return range_pass<7>(t, queries, order, m, r2, a, s);
        case 8: return range_pass<8>(t, queries, order, m, r2, a, s);
        case 12: return range_pass<12>(t, queries, order, m, r2, a, s);
        case 16: return range_pass<16>(t, queries, order, m, r2, a, s);
        default: return fail(PG_EUNSUPPORTED, "dimension class");
    }
}

pg_status range_args(const pg_tree *tree, const float *queries, int64_t m, float radius, int64_t capacity) {
    if (m < 0 || m >= (int64_t)1 << 31) return fail(PG_EINVAL, "range search: m must be in [0, 2^31)");
    if (!queries && m != tree->n) return fail(PG_EINVAL, "range search: all-points search (queries == NULL) needs m == n");
    if (!(radius >= 0.f && radius <= 3.4e38f)) return fail(PG_EINVAL, "range search: radius must be finite and >= 0");
    if (capacity < 0) return fail(PG_EINVAL, "range search: capacity must be >= 0");
    return PG_OK;
}

}  // namespace

}  // namespace pg

using namespace pg;

extern "C" pg_status pg_range(const pg_tree *tree, const float *queries, int64_t m, float radius, int64_t capacity,
                              int32_t *out_idx, int64_t *out_offsets, int64_t *out_total, void *stream) {
    if (!tree || !out_offsets || !out_total) return fail(PG_EINVAL, "pg_range: NULL argument");
    PG_TRY(tree_sync_meta(const_cast<pg_tree *>(tree)));
    PG_TRY(range_args(tree, queries, m, radius, capacity));
    *out_total = 0;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (m == 0) {
        PG_CUDA(cudaMemsetAsync(out_offsets, 0, sizeof(int64_t), s));
        return PG_OK;
    }
    const float r2 = radius * radius;
    Scratch cnt, ord, tot;
    PG_TRY(cnt.alloc(sizeof(int) * (size_t)(2 * m + 2), s));
    int *counts = cnt.as<int>(), *pre = counts + m + 1;
    if (tree->n == 0) {
        PG_CUDA(cudaMemsetAsync(out_offsets, 0, sizeof(int64_t) * (size_t)(m + 1), s));
        return PG_OK;
    }
    const bool sorted = queries && m >= kOrderMinQueries;
    if (sorted) {
        PG_TRY(ord.alloc(sizeof(int32_t) * (size_t)m, s));
        PG_TRY(query_order(tree, queries, m, tree->dim, ord.as<int32_t>(), s));
    }
    const int32_t *order = sorted ? ord.as<int32_t>() : nullptr;
    RangePass cp;
    cp.counts = counts;
    PG_TRY(range_dispatch(tree, queries, order, m, r2, cp, s));
    PG_TRY(tot.alloc(sizeof(unsigned long long), s));
    PG_CUDA(cudaMemsetAsync(tot.p, 0, sizeof(unsigned long long), s));
    k_range_total<<<std::min(ceil_div_i(m, 256), num_sms() * 8), 256, 0, s>>>(counts, m, tot.as<unsigned long long>());
    count_launch();
    unsigned long long total = 0;
    PG_TRY(read_small(&total, tot.p, sizeof(total), s));
    *out_total = (int64_t)total;
    if (total >= ((unsigned long long)1 << 31) - 1)
        return fail(PG_EINVAL, "pg_range: more than 2^31 - 2 results");
    PG_TRY(exclusive_scan(counts, pre, m, s));
    k_range_offsets<<<ceil_div_i(m + 1, 256), 256, 0, s>>>(pre, m, out_offsets);
    count_launch();
    if (!out_idx) return check_launch("range offsets");
    if (capacity < (int64_t)total) return fail(PG_EINVAL, "pg_range: capacity is below the result count");
    RangePass fp;
    fp.offs = out_offsets;
    fp.capacity = capacity;
    fp.out_idx = out_idx;
    fp.fill = true;
    return range_dispatch(tree, queries, order, m, r2, fp, s);
}

extern "C" pg_status pg_range_fill(const pg_tree *tree, const float *queries, int64_t m, float radius,
                                   const int64_t *offsets, int64_t capacity, int32_t *out_idx, void *stream) {
    if (!tree) return fail(PG_EINVAL, "pg_range_fill: NULL tree");
    PG_TRY(tree_sync_meta(const_cast<pg_tree *>(tree)));
    PG_TRY(range_args(tree, queries, m, radius, capacity));
    if (m == 0 || tree->n == 0) return PG_OK;   // every row is empty
    if (!offsets || !out_idx) return fail(PG_EINVAL, "pg_range_fill: NULL offsets or out_idx");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    Scratch ord, flag;
    PG_TRY(flag.alloc(sizeof(int), s));
    PG_TRY(fill_words(flag.p, 0u, 1, s));
    const bool sorted = queries && m >= kOrderMinQueries;
    if (sorted) {
        PG_TRY(ord.alloc(sizeof(int32_t) * (size_t)m, s));
        PG_TRY(query_order(tree, queries, m, tree->dim, ord.as<int32_t>(), s));
    }
    RangePass fp;
    fp.offs = offsets;
    fp.capacity = capacity;
    fp.out_idx = out_idx;
    fp.bad = flag.as<int>();
    fp.fill = true;
    PG_TRY(range_dispatch(tree, queries, sorted ? ord.as<int32_t>() : nullptr, m, radius * radius, fp, s));
    int bad = 0;
    PG_TRY(read_small(&bad, flag.p, sizeof(int), s));
    if (bad) return fail(PG_EINVAL, "pg_range_fill: the offsets do not match this tree, query set and radius");
    return PG_OK;
}
