// k-NN graph from the kd-tree's k-NN search (paper Section 4, geometric graph
// generators: the k-NN graph is generated with the kd-tree's k-NN search).
//
// Every point is joined to its k nearest OTHER points (the k smallest
// (squared distance, id) pairs over points with a different id).  Edges are
// undirected: an edge {i, j} exists when j is among i's k or i among j's k,
// and it is listed once as (u, v) with u < v; the list is sorted by (u, v).
//
// Steps: all-kNN with k + 1 (self included), then per point the k entries
// other than itself (if k + 1 points at distance 0 precede it, it is not in
// its list and the first k are kept); one (min, max) pair per entry; a
// stable LSD radix sort by v then by u; the first of every run of equal
// pairs is kept (flags + exclusive scan + compaction).
#include <algorithm>

#include "internal.h"
#include "sort.h"

namespace pg {

namespace {

constexpr int BT = 256;

inline int grid_of(int64_t n) { return std::max(1, ceil_div_i(n, BT)); }

// eu/ev: one (min, max) pair per (point, neighbour); padding (fewer than k
// other points) becomes (n, n), which sorts last and is dropped.
__global__ void k_graph_pairs(const int32_t *__restrict__ idx, int64_t n, int k, uint32_t *__restrict__ eu,
                              uint32_t *__restrict__ ev) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t *row = idx + i * (k + 1);
    bool self_seen = false;
    int o = 0;
    for (int j = 0; j <= k && o < k; ++j) {
        const int32_t t = row[j];
        if (!self_seen && t == (int32_t)i) {
            self_seen = true;
            continue;
        }
        uint32_t u = (uint32_t)n, v = (uint32_t)n;
        if (t >= 0) {
            u = (uint32_t)min((int64_t)t, i);
            v = (uint32_t)max((int64_t)t, i);
        }
        eu[i * k + o] = u;
        ev[i * k + o] = v;
        ++o;
    }
}

// keep the first of every run of equal (u, v); drop padding
__global__ void k_graph_flags(const uint32_t *__restrict__ su, const uint32_t *__restrict__ sv, int64_t P,
                              uint32_t n, int *__restrict__ flag) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= P) return;
    const uint32_t u = su[e], v = sv[e];
    flag[e] = u < n && (e == 0 || su[e - 1] != u || sv[e - 1] != v);
}

__global__ void k_graph_compact(const uint32_t *__restrict__ su, const uint32_t *__restrict__ sv,
                                const int *__restrict__ flag, const int *__restrict__ pos, int64_t P,
                                int32_t *__restrict__ out) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= P || !flag[e]) return;
    const int64_t p = pos[e];
    out[2 * p] = (int32_t)su[e];
    out[2 * p + 1] = (int32_t)sv[e];
}

int bits_for(int64_t n) {
    int b = 1;
    while (b < 32 && ((int64_t)1 << b) <= n) ++b;
    return b;
}

}  // namespace

}  // namespace pg

using namespace pg;

extern "C" pg_status pg_knn_graph(const pg_tree *tree, int k, int64_t capacity, int32_t *out_edges,
                                  int64_t *out_count, void *stream) {
    if (!tree || !out_count) return fail(PG_EINVAL, "pg_knn_graph: NULL argument");
    PG_TRY(tree_sync_meta(const_cast<pg_tree *>(tree)));
    if (k < 1 || k >= PG_MAX_K) return fail(PG_EINVAL, "pg_knn_graph: k must be in [1, 63]");
    if (capacity < 0) return fail(PG_EINVAL, "pg_knn_graph: capacity must be >= 0");
    *out_count = 0;
    const int64_t n = tree->n;
    if (n < 2) return PG_OK;
    const int64_t P = n * k;
    if (P >= ((int64_t)1 << 31)) return fail(PG_EINVAL, "pg_knn_graph: n * k must be < 2^31");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    Scratch knn, pairs, flags;
    PG_TRY(knn.alloc(sizeof(int32_t) * (size_t)(n * (k + 1)) * 2, s));
    int32_t *idx = knn.as<int32_t>();
    float *dist = reinterpret_cast<float *>(idx + n * (k + 1));
    PG_TRY(pg_knn(tree, nullptr, n, k + 1, idx, dist, stream));
    PG_TRY(pairs.alloc(sizeof(uint32_t) * (size_t)(4 * P), s));
    uint32_t *eu = pairs.as<uint32_t>(), *ev = eu + P, *tk = ev + P, *tv = tk + P;
    k_graph_pairs<<<grid_of(n), BT, 0, s>>>(idx, n, k, eu, ev);
    count_launch();
    knn.release();
    // lexicographic (u, v): stable sort by v, then stably by u
    const int bits = bits_for(n);
    uint32_t *sk = nullptr, *sv = nullptr;
    PG_TRY(radix_sort_pairs(ev, eu, false, tk, tv, P, bits, s, &sk, &sv));   // keys v, values u
    uint32_t *k2 = sv, *v2 = sk;                                            // keys u, values v
    uint32_t *t2k = (k2 == eu || k2 == ev) ? tk : eu, *t2v = (k2 == eu || k2 == ev) ? tv : ev;
    uint32_t *su = nullptr, *svv = nullptr;
    PG_TRY(radix_sort_pairs(k2, v2, false, t2k, t2v, P, bits, s, &su, &svv));
    PG_TRY(flags.alloc(sizeof(int) * (size_t)(2 * P + 1), s));
    int *flag = flags.as<int>(), *pos = flag + P;
    k_graph_flags<<<grid_of(P), BT, 0, s>>>(su, svv, P, (uint32_t)n, flag);
    count_launch();
    PG_TRY(exclusive_scan(flag, pos, P, s));
    int total = 0;
    PG_TRY(read_small(&total, pos + P, sizeof(int), s));
    *out_count = total;
    if (!out_edges) return PG_OK;
    if (capacity < total) return fail(PG_EINVAL, "pg_knn_graph: capacity is below the edge count");
    k_graph_compact<<<grid_of(P), BT, 0, s>>>(su, svv, flag, pos, P, out_edges);
    count_launch();
    return check_launch("knn graph");
}
