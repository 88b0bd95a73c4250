// BDL-tree: a log-structured forest of static kd-trees (paper Section 5;
// Appendix A.2 Insert_L, A.3 Erase_L, A.4 kNN_L).
//
// Device state: every point ever inserted keeps its coordinates in a store
// indexed by its id, and `slot_of[id]` records where it lives (tree slot,
// buffer tree, or erased).  Trees are rebuilt from id lists gathered out of
// the store, so any set of ids can be turned into a tree with the same
// builder as pg_tree_build.  Id lists are produced by order-preserving stream
// compactions over slot_of, which makes every choice of "which points" depend
// on ids only, never on a tree's internal layout.
//
// Host state: the bitmask F of occupied slots, per-slot live counts and the
// buffer's live count.  The forest bookkeeping follows the paper's steps:
// Insert_L adds floor(|P|/X) (+1 on buffer overflow) to F and rebuilds the
// slots whose bit becomes set from the slots whose bit clears plus the batch;
// Erase_L tombstones points in every tree, then gathers the trees left below
// half capacity and reinserts their points with Insert_L.
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "internal.h"

namespace pg {
pg_status build_gather(const float *store, const int32_t *ids, int64_t n, int dim, int leaf, cudaStream_t s,
                       pg_tree *t);
}

using namespace pg;

namespace {

constexpr int8_t SLOT_DEAD = -1;
constexpr int8_t SLOT_BUF = -2;
constexpr int8_t SLOT_NONE = -3;   // transient: being reassigned
constexpr int BT = 256;
constexpr int MAX_SLOTS = 62;

__global__ void k_iota(int32_t *out, int64_t cnt, int64_t base) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < cnt) out[i] = (int32_t)(base + i);
}

__global__ void k_set_slot(const int32_t *ids, int64_t cnt, int8_t code, int8_t *slot_of) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < cnt) slot_of[ids[i]] = code;
}

__global__ void k_slot_flags(const int8_t *slot_of, int64_t n, unsigned long long mask, int want_buf, int *flags) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int v = slot_of[i];
    flags[i] = (v >= 0 && ((mask >> v) & 1ull)) || (want_buf && v == SLOT_BUF);
}

__global__ void k_compact(const int *flags, const int *pre, int64_t n, int32_t *out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && flags[i]) out[pre[i]] = (int32_t)i;
}

template <int DC>
__global__ void k_erase(const float *__restrict__ pts, int64_t cnt, int dim, float4 *bucket,
                        const float4 *__restrict__ nodes, const int *__restrict__ split_dim,
                        const float *__restrict__ split_val, int root_ref, int root_cnt, int8_t *slot_of,
                        int *erased) {
    constexpr int W = bucket_w(DC);
    constexpr int NW = node_w(DC);
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= cnt) return;
    float p[DC];
#pragma unroll
    for (int c = 0; c < DC; ++c) p[c] = c < dim ? pts[i * dim + c] : 0.f;
    int ref = root_ref, c = root_cnt;
    // Descend by the split predicate: an exact copy of a stored point follows
    // the same path the point took when the tree was built.
    for (int guard = 0; c == 0 && guard <= PG_DEPTH_CAP; ++guard) {
        const int sd = split_dim[ref];
        const int side = p[sd] < split_val[ref] ? 0 : 1;
        const int *ri = reinterpret_cast<const int *>(nodes + (size_t)ref * NW) + 4 * DC;
        const int nref = ri[2 * side], ncnt = ri[2 * side + 1];
        ref = nref;
        c = ncnt;
    }
    if (c <= 0) return;
    float *bf = reinterpret_cast<float *>(bucket);
    for (int e = ref; e < ref + c; ++e) {
        float *ent = bf + (size_t)e * 4 * W;
        unsigned *idw = reinterpret_cast<unsigned *>(ent + DC);
        const unsigned id = *reinterpret_cast<volatile unsigned *>(idw);
        if (id == DEAD_ID) continue;
        bool same = true;
        for (int d = 0; d < dim; ++d) same &= __float_as_uint(ent[d]) == __float_as_uint(p[d]);
        if (!same) continue;
        if (atomicCAS(idw, id, DEAD_ID) == id) {
            const float qnan = __int_as_float(0x7fc00000);
#pragma unroll
            for (int d = 0; d < DC; ++d) ent[d] = qnan;   // never closer than anything
            slot_of[id] = SLOT_DEAD;
            atomicAdd(erased, 1);
        }
    }
}

template <int DC>
__global__ void k_live_flags(const float4 *bucket, int64_t n, int *flags) {
    constexpr int W = bucket_w(DC);
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const unsigned id = __float_as_uint(reinterpret_cast<const float *>(bucket + i * W)[DC]);
    flags[i] = id != DEAD_ID;
}

// A child whose bucket range holds no live point is marked empty (cnt = -1)
// so that searches skip it: the GPU counterpart of collapsing emptied
// subtrees in Erase_S.
template <int DC>
__global__ void k_mark_dead(float4 *nodes, int num_nodes, const int2 *__restrict__ node_range,
                            const int *__restrict__ pre) {
    constexpr int NW = node_w(DC);
    int nd = blockIdx.x * blockDim.x + threadIdx.x;
    if (nd >= num_nodes) return;
    int *ri = reinterpret_cast<int *>(nodes + (size_t)nd * NW) + 4 * DC;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        const int ref = ri[2 * c], cnt = ri[2 * c + 1];
        if (cnt < 0) continue;
        int lo, hi;
        if (cnt > 0) { lo = ref; hi = ref + cnt; }
        else { const int2 r = node_range[ref]; lo = r.x; hi = r.y; }
        if (pre[hi] - pre[lo] == 0) ri[2 * c + 1] = -1;
    }
}

inline int grid_of(int64_t n) { return std::max(1, ceil_div_i(n, BT)); }

}  // namespace

struct pg_bdl {
    int dim = 0, dc = 2, leaf = 16;
    int64_t X = 1;
    cudaStream_t s = nullptr;
    float *store = nullptr;
    int8_t *slot_of = nullptr;
    int64_t cap = 0;
    int64_t next_id = 0;
    uint64_t F = 0;
    pg_tree *slot[64] = {};
    pg_tree *buffer = nullptr;
    int64_t buffer_live = 0;
    TreeDesc *forest = nullptr;
    int forest_cap = 0;
    int forest_n = 0;
    bool dirty = true;
};

namespace {

int64_t capacity(const pg_bdl *b, int i) { return b->X << i; }

pg_status bdl_reserve(pg_bdl *b, int64_t need) {
    if (need <= b->cap) return PG_OK;
    int64_t cap = std::max<int64_t>(need, std::max<int64_t>(1024, b->cap * 2));
    float *st;
    int8_t *so;
    PG_TRY(dalloc_n(&st, (size_t)cap * b->dim, b->s));
    if (dalloc_n(&so, (size_t)cap, b->s) != PG_OK) { dfree(st, b->s); return PG_ENOMEM; }
    if (b->next_id > 0) {
        PG_CUDA(cudaMemcpyAsync(st, b->store, sizeof(float) * b->dim * (size_t)b->next_id, cudaMemcpyDeviceToDevice, b->s));
        PG_CUDA(cudaMemcpyAsync(so, b->slot_of, (size_t)b->next_id, cudaMemcpyDeviceToDevice, b->s));
    }
    dfree(b->store, b->s);
    dfree(b->slot_of, b->s);
    b->store = st;
    b->slot_of = so;
    b->cap = cap;
    return PG_OK;
}

// Ids (ascending) whose slot is in `mask` (and the buffer if want_buf).
pg_status bdl_collect(pg_bdl *b, uint64_t mask, bool want_buf, Scratch &out, int64_t *count) {
    const int64_t n = b->next_id;
    Scratch flags, pre;
    PG_TRY(flags.alloc(sizeof(int) * (size_t)std::max<int64_t>(n, 1), b->s));
    PG_TRY(pre.alloc(sizeof(int) * (size_t)(n + 1), b->s));
    if (n > 0) {
        k_slot_flags<<<grid_of(n), BT, 0, b->s>>>(b->slot_of, n, (unsigned long long)mask, want_buf ? 1 : 0,
                                                  flags.as<int>());
        count_launch();
    }
    PG_TRY(exclusive_scan(flags.as<int>(), pre.as<int>(), n, b->s));
    int h = 0;
    PG_TRY(read_small(&h, pre.as<int>() + n, sizeof(int), b->s));
    PG_TRY(out.alloc(sizeof(int32_t) * (size_t)std::max(h, 1), b->s));
    if (h > 0) {
        k_compact<<<grid_of(n), BT, 0, b->s>>>(flags.as<int>(), pre.as<int>(), n, out.as<int32_t>());
        count_launch();
    }
    *count = h;
    return check_launch("bdl collect");
}

pg_status set_slot(pg_bdl *b, const int32_t *ids, int64_t cnt, int8_t code) {
    if (cnt <= 0) return PG_OK;
    k_set_slot<<<grid_of(cnt), BT, 0, b->s>>>(ids, cnt, code, b->slot_of);
    count_launch();
    return check_launch("bdl set slot");
}

pg_status new_tree(pg_bdl *b, const int32_t *ids, int64_t cnt, pg_tree **out) {
    pg_tree *t = new (std::nothrow) pg_tree();
    if (!t) return fail(PG_ENOMEM, "bdl: host allocation");
    pg_status st = build_gather(b->store, ids, cnt, b->dim, b->leaf, b->s, t);
    if (st != PG_OK) {
        tree_release(t);
        delete t;
        return st;
    }
    *out = t;
    return PG_OK;
}

void drop_tree(pg_tree *&t) {
    if (t) {
        tree_release(t);
        delete t;
        t = nullptr;
    }
}

// The trees an Insert_L creates, built before the forest changes.
struct InsertPlan {
    pg_tree *made[64] = {};
    pg_tree *buffer = nullptr;   // the rebuilt buffer tree (when buffer_changed)
    bool buffer_changed = false;
    int64_t buffer_live = 0;
    uint64_t F = 0, consumed = 0;
};

// Insert_L over an id list (device, in pool order) against the full-tree
// mask F0: every new tree, and the new buffer tree, is built here; the only
// state of the forest this changes is the slot code of ids.
pg_status insert_plan(pg_bdl *b, const int32_t *ids, int64_t cnt, uint64_t F0, InsertPlan &p) {
    const int64_t X = b->X;
    int64_t q = cnt / X;
    const int64_t r = cnt % X;
    const int64_t nbatch = cnt - r;
    PG_TRY(set_slot(b, ids, nbatch, SLOT_NONE));
    PG_TRY(set_slot(b, ids + nbatch, r, SLOT_BUF));
    p.buffer_changed = r > 0;
    // the buffer's members after the remainder joined, ascending ids
    Scratch bufids;
    int64_t nbuf = 0;
    if (r > 0) PG_TRY(bdl_collect(b, 0, true, bufids, &nbuf));
    else nbuf = b->buffer_live;
    bool overflow = nbuf >= X;
    // pool = batch ids, then (on overflow) the X smallest buffer ids
    Scratch pool;
    const int64_t npool = nbatch + (overflow ? X : 0);
    PG_TRY(pool.alloc(sizeof(int32_t) * (size_t)std::max<int64_t>(npool, 1), b->s));
    if (nbatch > 0) PG_CUDA(cudaMemcpyAsync(pool.as<int32_t>(), ids, sizeof(int32_t) * nbatch, cudaMemcpyDeviceToDevice, b->s));
    if (overflow) {
        if (r == 0) PG_TRY(bdl_collect(b, 0, true, bufids, &nbuf));
        PG_CUDA(cudaMemcpyAsync(pool.as<int32_t>() + nbatch, bufids.as<int32_t>(), sizeof(int32_t) * X,
                                cudaMemcpyDeviceToDevice, b->s));
        PG_TRY(set_slot(b, bufids.as<int32_t>(), X, SLOT_NONE));
        q += 1;
        p.buffer_changed = true;
    }
    const uint64_t Fn = F0 + (uint64_t)q;
    const uint64_t consumed = F0 & ~Fn;
    const uint64_t created = Fn & ~F0;
    if ((Fn >> MAX_SLOTS) != 0) return fail(PG_EINVAL, "bdl: forest would exceed 62 slots");
    uint64_t taken = 0;
    int64_t pos = 0;
    int top = -1;
    for (int j = 0; j < 64; ++j)
        if ((created >> j) & 1) top = j;
    for (int j = 0; j < 64; ++j) {
        if (!((created >> j) & 1)) continue;
        const uint64_t below = consumed & ~taken & ((j == 0) ? 0ull : ((1ull << j) - 1));
        taken |= below;
        Scratch cons;
        int64_t ncons = 0;
        if (below) PG_TRY(bdl_collect(b, below, false, cons, &ncons));
        const int64_t need = (j == top) ? (npool - pos) : (capacity(b, j) - ncons);
        if (need < 0 || pos + need > npool) return fail(PG_EINVAL, "bdl: inconsistent cascade");
        const int64_t total = ncons + need;
        Scratch members;
        PG_TRY(members.alloc(sizeof(int32_t) * (size_t)std::max<int64_t>(total, 1), b->s));
        if (ncons > 0)
            PG_CUDA(cudaMemcpyAsync(members.as<int32_t>(), cons.as<int32_t>(), sizeof(int32_t) * ncons,
                                    cudaMemcpyDeviceToDevice, b->s));
        if (need > 0)
            PG_CUDA(cudaMemcpyAsync(members.as<int32_t>() + ncons, pool.as<int32_t>() + pos, sizeof(int32_t) * need,
                                    cudaMemcpyDeviceToDevice, b->s));
        pos += need;
        PG_TRY(set_slot(b, members.as<int32_t>(), total, (int8_t)j));
        PG_TRY(new_tree(b, members.as<int32_t>(), total, &p.made[j]));
    }
    if (taken != consumed || pos != npool) return fail(PG_EINVAL, "bdl: inconsistent cascade");
    p.F = Fn;
    p.consumed = consumed;
    if (p.buffer_changed) {
        Scratch bids;
        PG_TRY(bdl_collect(b, 0, true, bids, &p.buffer_live));
        if (p.buffer_live > 0) PG_TRY(new_tree(b, bids.as<int32_t>(), p.buffer_live, &p.buffer));
    }
    return PG_OK;
}

// Insert_L, all or nothing.  `drop`: slots whose trees the caller has
// emptied (erase's under-full trees; their live ids are among ids), released
// with the consumed trees.  Until every new tree is built nothing but slot
// codes changes; on an error the new trees are released and the slot codes
// restored from a copy taken first, so the forest is as before the call.
pg_status insert_ids(pg_bdl *b, const int32_t *ids, int64_t cnt, uint64_t drop = 0) {
    if (cnt <= 0 && !drop) return PG_OK;
    const int64_t nid = b->next_id;
    Scratch saved;
    PG_TRY(saved.alloc((size_t)std::max<int64_t>(nid, 1), b->s));
    if (nid > 0) PG_CUDA(cudaMemcpyAsync(saved.p, b->slot_of, (size_t)nid, cudaMemcpyDeviceToDevice, b->s));
    InsertPlan p;
    p.F = b->F & ~drop;
    const pg_status st = cnt > 0 ? insert_plan(b, ids, cnt, b->F & ~drop, p) : PG_OK;
    if (st != PG_OK) {
        for (auto &t : p.made) drop_tree(t);
        drop_tree(p.buffer);
        if (nid > 0) cudaMemcpyAsync(b->slot_of, saved.p, (size_t)nid, cudaMemcpyDeviceToDevice, b->s);
        return st;   // (the message of the first error stands)
    }
    for (int i = 0; i < 64; ++i)
        if (((p.consumed | drop) >> i) & 1) drop_tree(b->slot[i]);
    for (int j = 0; j < 64; ++j)
        if (p.made[j]) b->slot[j] = p.made[j];
    b->F = p.F;
    if (p.buffer_changed) {
        drop_tree(b->buffer);
        b->buffer = p.buffer;
        b->buffer_live = p.buffer_live;
    }
    b->dirty = true;
    return PG_OK;
}

template <int DC>
pg_status erase_tree(pg_bdl *b, pg_tree *t, const float *pts, int64_t cnt, int *erased) {
    k_erase<DC><<<grid_of(cnt), BT, 0, b->s>>>(pts, cnt, b->dim, t->bucket, t->nodes, t->split_dim,
                                                 t->split_val, t->root_ref, t->root_cnt, b->slot_of, erased);
    count_launch();
    return check_launch("bdl erase");
}

template <int DC>
pg_status recount_tree(pg_bdl *b, pg_tree *t) {
    Scratch flags, pre;
    PG_TRY(flags.alloc(sizeof(int) * (size_t)t->n, b->s));
    PG_TRY(pre.alloc(sizeof(int) * (size_t)(t->n + 1), b->s));
    k_live_flags<DC><<<grid_of(t->n), BT, 0, b->s>>>(t->bucket, t->n, flags.as<int>());
    count_launch();
    PG_TRY(exclusive_scan(flags.as<int>(), pre.as<int>(), t->n, b->s));
    if (t->num_nodes > 0) {
        k_mark_dead<DC><<<grid_of(t->num_nodes), BT, 0, b->s>>>(t->nodes, t->num_nodes, t->node_range,
                                                                pre.as<int>());
        count_launch();
    }
    return check_launch("bdl recount");
}

#define PG_DC_DISPATCH(dc, EXPR)                                  \
    switch (dc) {                                                 \
        case 2: { constexpr int DCV = 2; EXPR; } break;           \
        case 3: { constexpr int DCV = 3; EXPR; } break;           \
        case 4: { constexpr int DCV = 4; EXPR; } break;           \
        case 5: { constexpr int DCV = 5; EXPR; } break;           \
        case 6: { constexpr int DCV = 6; EXPR; } break;           \
        case 7: { constexpr int DCV = 7; EXPR; } break;           \
        case 8: { constexpr int DCV = 8; EXPR; } break;           \
        case 12: { constexpr int DCV = 12; EXPR; } break;         \
        case 16: { constexpr int DCV = 16; EXPR; } break;         \
        default: return fail(PG_EUNSUPPORTED, "dimension class"); \
    }

pg_status erase_impl(pg_bdl *b, const float *pts, int64_t cnt) {
    if (cnt <= 0) return PG_OK;
    std::vector<pg_tree *> trees;
    std::vector<int> which;   // slot index, or -1 for the buffer
    for (int i = 0; i < 64; ++i)
        if (b->slot[i] && b->slot[i]->live > 0) { trees.push_back(b->slot[i]); which.push_back(i); }
    if (b->buffer && b->buffer_live > 0) { trees.push_back(b->buffer); which.push_back(-1); }
    if (trees.empty()) return PG_OK;
    Scratch cnts;
    PG_TRY(cnts.alloc(sizeof(int) * trees.size(), b->s));
    PG_CUDA(cudaMemsetAsync(cnts.p, 0, sizeof(int) * trees.size(), b->s));
    for (size_t t = 0; t < trees.size(); ++t) {
        pg_status st = PG_OK;
        PG_DC_DISPATCH(b->dc, st = erase_tree<DCV>(b, trees[t], pts, cnt, cnts.as<int>() + t));
        PG_TRY(st);
    }
    std::vector<int> erased(trees.size());
    PG_TRY(read_small(erased.data(), cnts.p, sizeof(int) * trees.size(), b->s));
    // the tombstones are in: count them everywhere first, so that a failure
    // below leaves every live count right (a tree not yet recounted only
    // keeps subtrees that hold no live point, which searches never match)
    uint64_t destroy = 0;
    for (size_t t = 0; t < trees.size(); ++t) {
        trees[t]->live -= erased[t];
        if (which[t] < 0) b->buffer_live -= erased[t];
        if (erased[t] > 0 && which[t] >= 0 && 2 * trees[t]->live < capacity(b, which[t]))
            destroy |= 1ull << which[t];
    }
    b->dirty = true;
    for (size_t t = 0; t < trees.size(); ++t) {
        if (erased[t] == 0) continue;
        pg_status st = PG_OK;
        PG_DC_DISPATCH(b->dc, st = recount_tree<DCV>(b, trees[t]));
        PG_TRY(st);
    }
    if (!destroy) return PG_OK;
    // the erase stands; if the reinsertion fails the under-full trees stay
    // (every query is still exact) and the error is returned
    Scratch R;
    int64_t nR = 0;
    PG_TRY(bdl_collect(b, destroy, false, R, &nR));
    return insert_ids(b, R.as<int32_t>(), nR, destroy);
}

pg_status refresh_forest(const pg_bdl *cb) {
    pg_bdl *b = const_cast<pg_bdl *>(cb);
    if (!b->dirty) return PG_OK;
    std::vector<TreeDesc> d;
    std::vector<std::pair<int64_t, pg_tree *>> order;
    for (int i = 0; i < 64; ++i)
        if (b->slot[i] && b->slot[i]->live > 0) order.push_back({b->slot[i]->live, b->slot[i]});
    // largest first (the first of equals in slot order: the tree pg_bdl_knn orders queries by)
    std::stable_sort(order.begin(), order.end(), [](auto &x, auto &y) { return x.first > y.first; });
    for (auto &o : order) d.push_back(tree_desc(o.second));
    if (b->buffer && b->buffer_live > 0) d.push_back(tree_desc(b->buffer));
    if ((int)d.size() > b->forest_cap) {
        dfree(b->forest, b->s);
        b->forest = nullptr;
        b->forest_cap = 0;
        PG_TRY(dalloc_n(&b->forest, std::max<size_t>(d.size(), 8), b->s));
        b->forest_cap = (int)std::max<size_t>(d.size(), 8);
    }
    if (!d.empty())
        PG_CUDA(cudaMemcpyAsync(b->forest, d.data(), sizeof(TreeDesc) * d.size(), cudaMemcpyHostToDevice, b->s));
    PG_CUDA(cudaStreamSynchronize(b->s));
    b->forest_n = (int)d.size();
    b->dirty = false;
    return PG_OK;
}

}  // namespace

extern "C" {

pg_status pg_bdl_create(int dim, int64_t X, int leaf, void *stream, pg_bdl **out) {
    if (out) *out = nullptr;
    if (!out) return fail(PG_EINVAL, "pg_bdl_create: out is NULL");
    if (dim < 1 || dim > PG_MAX_DIM) return fail(PG_EINVAL, "pg_bdl_create: dim must be in [1, 16]");
    if (X < 1 || X >= ((int64_t)1 << 31)) return fail(PG_EINVAL, "pg_bdl_create: buffer_size must be in [1, 2^31)");
    if (leaf < 1 || leaf > PG_MAX_LEAF) return fail(PG_EINVAL, "pg_bdl_create: leaf_size must be in [1, 256]");
    pg_bdl *b = new (std::nothrow) pg_bdl();
    if (!b) return fail(PG_ENOMEM, "pg_bdl_create: host allocation");
    b->dim = dim;
    b->dc = dim_class(dim);
    b->leaf = leaf;
    b->X = X;
    b->s = reinterpret_cast<cudaStream_t>(stream);
    *out = b;
    return PG_OK;
}

pg_status pg_bdl_insert(pg_bdl *b, const float *pts, int64_t cnt, int32_t *out_ids) {
    if (!b) return fail(PG_EINVAL, "pg_bdl_insert: forest is NULL");
    if (cnt < 0) return fail(PG_EINVAL, "pg_bdl_insert: cnt < 0");
    if (cnt > 0 && !pts) return fail(PG_EINVAL, "pg_bdl_insert: points is NULL");
    if (b->next_id + cnt >= ((int64_t)1 << 31)) return fail(PG_EINVAL, "pg_bdl_insert: more than 2^31-1 ids");
    if (cnt == 0) return PG_OK;
    PG_TRY(bdl_reserve(b, b->next_id + cnt));
    PG_CUDA(cudaMemcpyAsync(b->store + (size_t)b->next_id * b->dim, pts, sizeof(float) * b->dim * (size_t)cnt,
                            cudaMemcpyDeviceToDevice, b->s));
    Scratch ids;
    PG_TRY(ids.alloc(sizeof(int32_t) * (size_t)cnt, b->s));
    k_iota<<<grid_of(cnt), BT, 0, b->s>>>(ids.as<int32_t>(), cnt, b->next_id);
    count_launch();
    if (out_ids) PG_CUDA(cudaMemcpyAsync(out_ids, ids.p, sizeof(int32_t) * cnt, cudaMemcpyDeviceToDevice, b->s));
    const int64_t first = b->next_id;
    b->next_id += cnt;
    const pg_status st = insert_ids(b, ids.as<int32_t>(), cnt);
    if (st != PG_OK) b->next_id = first;   // the ids are handed out again by the next insert
    return st;
}

pg_status pg_bdl_erase(pg_bdl *b, const float *pts, int64_t cnt) {
    if (!b) return fail(PG_EINVAL, "pg_bdl_erase: forest is NULL");
    if (cnt < 0) return fail(PG_EINVAL, "pg_bdl_erase: cnt < 0");
    if (cnt > 0 && !pts) return fail(PG_EINVAL, "pg_bdl_erase: points is NULL");
    return erase_impl(b, pts, cnt);
}

pg_status pg_bdl_knn(const pg_bdl *b, const float *queries, int64_t m, int k, int32_t *out_idx, float *out_dist) {
    return pg_bdl_knn_ex(b, queries, m, k, PG_KNN_AUTO, out_idx, out_dist);
}

pg_status pg_bdl_knn_ex(const pg_bdl *b, const float *queries, int64_t m, int k, int variant, int32_t *out_idx,
                        float *out_dist) {
    if (!b) return fail(PG_EINVAL, "pg_bdl_knn: forest is NULL");
    if (!valid_variant(variant)) return fail(PG_EINVAL, "pg_bdl_knn: unknown traversal variant");
    if (k < 1 || k > PG_MAX_K) return fail(PG_EINVAL, "pg_bdl_knn: k must be in [1, 64]");
    if (m < 0 || m >= ((int64_t)1 << 31)) return fail(PG_EINVAL, "pg_bdl_knn: m must be in [0, 2^31)");
    if (m > 0 && (!queries || !out_idx || !out_dist)) return fail(PG_EINVAL, "pg_bdl_knn: NULL pointer");
    if (m == 0) return PG_OK;
    PG_TRY(refresh_forest(b));
    // order the queries by the leaves of the largest tree (the forest's first
    // descriptor), where the search then starts from each query's leaf
    const pg_tree *big = nullptr;
    for (int i = 0; i < 64; ++i)
        if (b->slot[i] && b->slot[i]->live > 0 && (!big || b->slot[i]->live > big->live)) big = b->slot[i];
    Scratch ord;
    const bool sorted = big && m >= kOrderMinQueries;
    if (sorted) {
        PG_TRY(ord.alloc(sizeof(int32_t) * (size_t)(2 * m), b->s));
        PG_TRY(query_order(big, queries, m, b->dim, ord.as<int32_t>(), b->s, ord.as<int32_t>() + m));
    }
    return knn_launch(b->forest, b->forest_n, b->dc, queries, nullptr, sorted ? ord.as<int32_t>() : nullptr,
                      sorted ? ord.as<int32_t>() + m : nullptr, m, b->dim, k, out_idx, out_dist, variant, b->s);
}

pg_status pg_bdl_size(const pg_bdl *b, int64_t *live) {
    if (!b || !live) return fail(PG_EINVAL, "pg_bdl_size: NULL argument");
    int64_t s = b->buffer_live;
    for (int i = 0; i < 64; ++i)
        if (b->slot[i]) s += b->slot[i]->live;
    *live = s;
    return PG_OK;
}

pg_status pg_bdl_structure(const pg_bdl *b, uint64_t *F, int64_t *slot_live, int64_t *buffer_live,
                           int64_t *next_id) {
    if (!b) return fail(PG_EINVAL, "pg_bdl_structure: forest is NULL");
    if (F) *F = b->F;
    if (slot_live)
        for (int i = 0; i < 64; ++i) slot_live[i] = b->slot[i] ? b->slot[i]->live : 0;
    if (buffer_live) *buffer_live = b->buffer_live;
    if (next_id) *next_id = b->next_id;
    return PG_OK;
}

pg_status pg_bdl_slot_of(const pg_bdl *b, int8_t *out) {
    if (!b || !out) return fail(PG_EINVAL, "pg_bdl_slot_of: NULL argument");
    if (b->next_id > 0) {
        PG_CUDA(cudaMemcpyAsync(out, b->slot_of, (size_t)b->next_id, cudaMemcpyDeviceToHost, b->s));
        PG_CUDA(cudaStreamSynchronize(b->s));
    }
    return PG_OK;
}

pg_status pg_bdl_free(pg_bdl *b) {
    if (!b) return PG_OK;
    for (int i = 0; i < 64; ++i) drop_tree(b->slot[i]);
    drop_tree(b->buffer);
    dfree(b->store, b->s);
    dfree(b->slot_of, b->s);
    dfree(b->forest, b->s);
    delete b;
    return PG_OK;
}

}  // extern "C"
