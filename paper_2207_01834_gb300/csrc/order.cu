// Query ordering for coherent warps: each query descends the tree by the
// split predicate to the leaf it lies in, and the queries are sorted stably by
// that leaf's bucket position.  Queries in one warp then share most of their
// search.  Only the processing order changes; every query still gets its own
// exact answer in its own output row.
#include <algorithm>

#include "internal.h"
#include "sort.h"

namespace pg {

namespace {

constexpr int BT = 256;

// The root comes from the tree's device descriptor, so the ordering needs no
// host-side copy of it (a leaf or empty root gives every query key 0).
template <int DC>
__global__ void k_locate(const float *__restrict__ queries, int64_t m, int dim, const TreeDesc *__restrict__ desc,
                         const int *__restrict__ split_dim, const float *__restrict__ split_val,
                         uint32_t *__restrict__ keys) {
    constexpr int NW = node_w(DC);
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const float4 *__restrict__ nodes = desc->nodes;
    int ref = desc->root_ref, cnt = desc->root_cnt;
    for (int guard = 0; cnt == 0 && guard <= PG_DEPTH_CAP; ++guard) {
        const int sd = split_dim[ref];
        const float x = queries[i * dim + sd];
        const int side = x < split_val[ref] ? 0 : 1;
        const int *ri = reinterpret_cast<const int *>(nodes + (size_t)ref * NW) + 4 * DC;
        const int nref = ri[2 * side], ncnt = ri[2 * side + 1];
        ref = nref;
        cnt = ncnt;
    }
    keys[i] = (uint32_t)max(ref, 0);
}

}  // namespace

pg_status query_order(const pg_tree *t, const float *queries, int64_t m, int dim, int32_t *order, cudaStream_t s,
                      int32_t *leaf_ref) {
    if (m <= 0) return PG_OK;
    Scratch sk, st;
    PG_TRY(sk.alloc(sizeof(uint32_t) * (size_t)m, s));
    PG_TRY(st.alloc(sizeof(uint32_t) * (size_t)(2 * m), s));
    uint32_t *keys = sk.as<uint32_t>();
    uint32_t *tk = st.as<uint32_t>(), *tv = tk + m;
    uint32_t *vals = reinterpret_cast<uint32_t *>(order);
    {
        const int grid = std::max(1, ceil_div_i(m, BT));
        switch (t->dc) {
#define PG_LOC(D) case D: k_locate<D><<<grid, BT, 0, s>>>(queries, m, dim, t->desc, t->split_dim, t->split_val, keys); break;
            PG_LOC(2) PG_LOC(3) PG_LOC(4) PG_LOC(5) PG_LOC(6) PG_LOC(7) PG_LOC(8) PG_LOC(12) PG_LOC(16)
#undef PG_LOC
            default: return fail(PG_EUNSUPPORTED, "dimension class");
        }
        count_launch();
    }
    int bits = 1;
    while (bits < 32 && ((int64_t)1 << bits) <= t->n) ++bits;
    uint32_t *sk_out, *sv_out;
    PG_TRY(radix_sort_pairs(keys, vals, true, tk, tv, m, bits, s, &sk_out, &sv_out));
    if (sv_out != vals) PG_CUDA(cudaMemcpyAsync(vals, sv_out, sizeof(uint32_t) * (size_t)m, cudaMemcpyDeviceToDevice, s));
    if (leaf_ref)
        PG_CUDA(cudaMemcpyAsync(leaf_ref, sk_out, sizeof(uint32_t) * (size_t)m, cudaMemcpyDeviceToDevice, s));
    return check_launch("query order");
}

}  // namespace pg
