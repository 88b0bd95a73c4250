// Data-parallel exact k-NN traversal (paper Appendix A.1.3 "Data-Parallel
// k-NN" and Section 5 / Appendix A.4 kNN_L over the BDL forest).
//
// One thread per query.  The query's k best candidates live in registers as
// an ascending list of (squared distance, id) pairs.  The paper's 2k buffer
// with periodic selection keeps the same set; a sorted register list needs no
// selection step and no memory.  Every tree of the forest is searched in turn
// with the same list, so the answer is the k-NN of the union (kNN_L).
//
// Search order per tree: from the root, at each internal node both children's
// tight boxes are measured; the nearer child is visited next and the farther
// one is pushed on a small stack with its box distance.  A child is skipped
// when its box lies farther than the current k-th distance (strictly, so that
// equal-distance candidates with smaller ids are still found).  Box distance
// and point distance use the same monotone chain of rounded operations, so a
// box bound never exceeds the distance of a point inside it: the result is
// exactly the k smallest (float32 distance, id) pairs.
#pragma once

#include "common.cuh"

namespace pg {

constexpr int KNN_THREADS = 128;
constexpr int KNN_STACK = PG_DEPTH_CAP + 2;

template <int KC>
struct KList {
    float d[KC];
    unsigned id[KC];

    // Slots below KC-k hold -inf sentinels that never move, so a list of
    // compile-time capacity KC serves any runtime k <= KC.
    __device__ __forceinline__ void init(int k) {
#pragma unroll
        for (int j = 0; j < KC; ++j) {
            const bool sentinel = j < KC - k;
            d[j] = sentinel ? -__int_as_float(0x7f800000) : __int_as_float(0x7f800000);
            id[j] = DEAD_ID;
        }
    }
    __device__ __forceinline__ float kth() const { return d[KC - 1]; }

    __device__ __forceinline__ static bool less(float a, unsigned ia, float b, unsigned ib) {
        return a < b || (a == b && ia < ib);
    }
    // Insert (x, ix) if it precedes the current k-th pair.
    __device__ __forceinline__ void offer(float x, unsigned ix) {
        if (!less(x, ix, d[KC - 1], id[KC - 1])) return;
#pragma unroll
        for (int j = KC - 1; j > 0; --j) {
            const bool shift = less(x, ix, d[j - 1], id[j - 1]);
            const bool here = !shift && less(x, ix, d[j], id[j]);
            const float nd = shift ? d[j - 1] : (here ? x : d[j]);
            const unsigned ni = shift ? id[j - 1] : (here ? ix : id[j]);
            d[j] = nd;
            id[j] = ni;
        }
        if (less(x, ix, d[0], id[0])) { d[0] = x; id[0] = ix; }
    }
};

template <int DC>
__device__ __forceinline__ void load_point(const float4 *__restrict__ bucket, int64_t i, float *p, unsigned &pid) {
    constexpr int W = bucket_w(DC);
    float v[4 * W];
#pragma unroll
    for (int w = 0; w < W; ++w) {
        float4 f = __ldg(bucket + i * W + w);
        v[4 * w] = f.x; v[4 * w + 1] = f.y; v[4 * w + 2] = f.z; v[4 * w + 3] = f.w;
    }
#pragma unroll
    for (int c = 0; c < DC; ++c) p[c] = v[c];
    pid = __float_as_uint(v[DC]);
}

template <int DC, int KC>
__device__ __forceinline__ void scan_leaf(const float4 *__restrict__ bucket, int ref, int cnt, const float *q,
                                          KList<KC> &L) {
    for (int i = ref; i < ref + cnt; ++i) {
        float p[DC];
        unsigned pid;
        load_point<DC>(bucket, i, p, pid);
        L.offer(sqdist<DC>(q, p), pid);
    }
}

template <int DC, int KC>
__device__ __forceinline__ void search_tree(const TreeDesc &T, const float *q, KList<KC> &L) {
    if (T.root_cnt < 0) return;
    float rlo[DC], rhi[DC];
#pragma unroll
    for (int c = 0; c < DC; ++c) { rlo[c] = T.root_lo[c]; rhi[c] = T.root_hi[c]; }
    const float d_root = boxdist<DC>(q, rlo, rhi);
    if (d_root > L.kth()) return;
    if (T.root_cnt > 0) {
        scan_leaf<DC, KC>(T.bucket, T.root_ref, T.root_cnt, q, L);
        return;
    }
    int s_ref[KNN_STACK], s_cnt[KNN_STACK];
    float s_d[KNN_STACK];
    int sp = 0;
    s_ref[0] = T.root_ref; s_cnt[0] = 0; s_d[0] = d_root; sp = 1;
    constexpr int NW = node_w(DC);
    while (sp > 0) {
        --sp;
        int ref = s_ref[sp];
        int cnt = s_cnt[sp];
        if (s_d[sp] > L.kth()) continue;
        if (cnt > 0) {
            scan_leaf<DC, KC>(T.bucket, ref, cnt, q, L);
            continue;
        }
        for (;;) {
            float rec[4 * NW];
            const float4 *np = T.nodes + (size_t)ref * NW;
#pragma unroll
            for (int w = 0; w < NW; ++w) {
                float4 f = __ldg(np + w);
                rec[4 * w] = f.x; rec[4 * w + 1] = f.y; rec[4 * w + 2] = f.z; rec[4 * w + 3] = f.w;
            }
            const int *ri = reinterpret_cast<const int *>(rec + 4 * DC);
            const int r0 = ri[0], c0 = ri[1], r1 = ri[2], c1 = ri[3];
            const float d0 = boxdist<DC>(q, rec, rec + DC);
            const float d1 = boxdist<DC>(q, rec + 2 * DC, rec + 3 * DC);
            const bool sw = d1 < d0;
            const float dn = sw ? d1 : d0, df = sw ? d0 : d1;
            const int rn = sw ? r1 : r0, cn = sw ? c1 : c0;
            const int rf = sw ? r0 : r1, cf = sw ? c0 : c1;
            const float kth = L.kth();
            if (cf >= 0 && df <= kth && sp < KNN_STACK) {
                s_ref[sp] = rf; s_cnt[sp] = cf; s_d[sp] = df; ++sp;
            }
            if (cn >= 0 && dn <= kth) {
                if (cn > 0) {
                    scan_leaf<DC, KC>(T.bucket, rn, cn, q, L);
                    break;
                }
                ref = rn;
                continue;
            }
            break;
        }
    }
}

// queries: row-major m*dim (NULL when self_bucket is given).
// self_bucket: the tree's own bucket entries as queries (all-kNN); the
// output row is then the entry's id.
template <int DC, int KC>
__global__ void __launch_bounds__(KNN_THREADS) k_knn(const TreeDesc *__restrict__ trees, int ntrees,
                                                     const float *__restrict__ queries,
                                                     const float4 *__restrict__ self_bucket, int64_t m, int dim,
                                                     int k, int32_t *__restrict__ out_idx,
                                                     float *__restrict__ out_dist) {
    const int64_t qi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (qi >= m) return;
    float q[DC];
    int64_t row = qi;
    if (self_bucket) {
        unsigned qid;
        load_point<DC>(self_bucket, qi, q, qid);
        row = (int64_t)qid;
    } else {
#pragma unroll
        for (int c = 0; c < DC; ++c) q[c] = c < dim ? queries[qi * dim + c] : 0.f;
    }
    KList<KC> L;
    L.init(k);
    for (int t = 0; t < ntrees; ++t) search_tree<DC, KC>(trees[t], q, L);
    int32_t *oi = out_idx + row * k;
    float *od = out_dist + row * k;
#pragma unroll
    for (int j = 0; j < KC; ++j) {
        if (j >= KC - k) {
            const int o = j - (KC - k);
            oi[o] = L.id[j] == DEAD_ID ? -1 : (int32_t)L.id[j];
            od[o] = L.d[j];
        }
    }
}

}  // namespace pg

// Host launcher for one dimension class: picks the list capacity KC >= k.
#define PG_DEFINE_KNN_LAUNCH(DCN)                                                                          \
    namespace pg {                                                                                         \
    pg_status knn_launch_dc##DCN(const TreeDesc *trees, int ntrees, const float *queries,                  \
                                 const float4 *self_bucket, int64_t m, int dim, int k, int32_t *out_idx,    \
                                 float *out_dist, cudaStream_t s) {                                         \
        const int grid = ceil_div_i(m, KNN_THREADS);                                                       \
        KTimer kt("knn_traverse", s);                                                                      \
        switch (k_class(k)) {                                                                              \
            case 1: k_knn<DCN, 1><<<grid, KNN_THREADS, 0, s>>>(trees, ntrees, queries, self_bucket, m, dim, k, out_idx, out_dist); break; \
            case 2: k_knn<DCN, 2><<<grid, KNN_THREADS, 0, s>>>(trees, ntrees, queries, self_bucket, m, dim, k, out_idx, out_dist); break; \
            case 4: k_knn<DCN, 4><<<grid, KNN_THREADS, 0, s>>>(trees, ntrees, queries, self_bucket, m, dim, k, out_idx, out_dist); break; \
            case 8: k_knn<DCN, 8><<<grid, KNN_THREADS, 0, s>>>(trees, ntrees, queries, self_bucket, m, dim, k, out_idx, out_dist); break; \
            case 10: k_knn<DCN, 10><<<grid, KNN_THREADS, 0, s>>>(trees, ntrees, queries, self_bucket, m, dim, k, out_idx, out_dist); break; \
            case 16: k_knn<DCN, 16><<<grid, KNN_THREADS, 0, s>>>(trees, ntrees, queries, self_bucket, m, dim, k, out_idx, out_dist); break; \
            case 32: k_knn<DCN, 32><<<grid, KNN_THREADS, 0, s>>>(trees, ntrees, queries, self_bucket, m, dim, k, out_idx, out_dist); break; \
            case 64: k_knn<DCN, 64><<<grid, KNN_THREADS, 0, s>>>(trees, ntrees, queries, self_bucket, m, dim, k, out_idx, out_dist); break; \
            default: return fail(PG_EINVAL, "k out of range");                                             \
        }                                                                                                  \
        count_launch();                                                                                    \
        return check_launch("knn traverse");                                                               \
    }                                                                                                      \
    }
