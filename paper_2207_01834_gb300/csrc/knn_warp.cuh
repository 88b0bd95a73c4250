// Warp-per-query exact k-NN traversal (paper App. A.1.3: every query is
// searched independently; here the 32 lanes of a warp search one query
// together).  Meant for higher dimensions, where a query visits many nodes
// and leaves and one lane per query leaves most lanes idle on divergence.
//
// The query's k-list is spread over the warp: lane j holds the j-th smallest
// (distance, id) key (and the (32+j)-th for lists of up to 64), so the k-th
// key is one shuffle away and an insertion is a ballot (insertion point) and
// a shuffle-up (shift) executed by all lanes at once.
//
// Leaves are scanned cooperatively: lane j takes point j of a 32-point chunk
// (one coalesced load per lane); the chunk's candidates that precede the k-th
// key are inserted one after the other, lowest lane first.
//
// Nodes are expanded 32 at a time: the warp keeps a stack of subtrees (tree
// node or leaf, with the box distance that was measured when it was pushed)
// in shared memory; each round the lanes pop up to 32 entries from the top,
// drop the ones farther than the k-th distance, expand the internal nodes
// (both children's tight boxes measured by the expanding lane, with the same
// rounded chain as the other traversals), push the internal children and
// collect the leaves, which are then scanned nearest first by box distance.
// All-kNN (and separate queries with a start leaf) first scans the query's
// own leaf and climbs the parent links, pushing the sibling subtree of every
// ancestor until the k-th ball lies inside the subtree searched so far; other
// queries start from each tree's root in turn (one k-list across a forest).
// Every pruning test is the query's own k-th distance, so the answer is the
// same exact k smallest pairs as the other traversals.
#pragma once

namespace pg {

constexpr int WQ_THREADS = 128;            // four warps, one query each at a time
constexpr int WQ_WARPS = WQ_THREADS / 32;
constexpr int WQ_STACK = 512;              // subtree stack entries per warp
// Rounds pop up to 32 entries while the stack holds at most WQ_WIDE_LIMIT;
// above it they pop one (depth first), which grows the stack by at most one
// entry per tree level.  A wide round adds at most 32 entries, so the stack
// never exceeds WQ_WIDE_LIMIT + 32 + PG_DEPTH_CAP + 1 < WQ_STACK.
constexpr int WQ_WIDE_LIMIT = WQ_STACK - 32 - PG_DEPTH_CAP - 16;
constexpr int WQ_LEAVES = 96;              // leaves collected by one round: 32 popped + 2 children of 32

static_assert(WQ_WIDE_LIMIT + 32 + PG_DEPTH_CAP + 1 < WQ_STACK, "warp traversal stack bound");

struct WqShared {
    int s_ref[WQ_WARPS][WQ_STACK];
    int s_cnt[WQ_WARPS][WQ_STACK];
    float s_d[WQ_WARPS][WQ_STACK];
    int l_ref[WQ_WARPS][WQ_LEAVES];
    int l_cnt[WQ_WARPS][WQ_LEAVES];
    float l_d[WQ_WARPS][WQ_LEAVES];
};

constexpr unsigned long long WQ_NONE = ~0ull;   // key of a lane outside the list

// The warp's k-list: slot s lives in lane s % 32, register s / 32 (slots
// below KC - k hold the key 0, which nothing precedes, so a capacity-KC list
// serves any k <= KC; slots >= KC hold a key above every real one).
template <int KC>
struct WarpList {
    static constexpr int NK = (KC + 31) / 32;   // keys per lane
    unsigned long long key[NK];
    unsigned long long kth;   // slot KC-1, the same in every lane

    __device__ __forceinline__ void init(int k, int lane) {
#pragma unroll
        for (int i = 0; i < NK; ++i) {
            const int s = i * 32 + lane;
            key[i] = s >= KC ? WQ_NONE : (s < KC - k ? 0ull : PAD_KEY);
        }
        kth = PAD_KEY;
    }
    __device__ __forceinline__ float kth_dist() const { return __uint_as_float((unsigned)(kth >> 32)); }
    // Insert kx (the same value in every lane) if it precedes the k-th key:
    // its slot is the number of keys not above it; the slots from there up
    // take their predecessor's key.
    __device__ __forceinline__ void insert(unsigned long long kx, int lane) {
        if (!(kx < kth)) return;   // warp-uniform
        int at = 0;
#pragma unroll
        for (int i = 0; i < NK; ++i) at += __popc(__ballot_sync(0xffffffffu, key[i] <= kx && i * 32 + lane < KC));
        unsigned long long prev[NK];
#pragma unroll
        for (int i = 0; i < NK; ++i) {
            const unsigned long long up = __shfl_up_sync(0xffffffffu, key[i], 1);
            const unsigned long long carry = __shfl_sync(0xffffffffu, key[i > 0 ? i - 1 : 0], 31);
            prev[i] = lane == 0 ? (i > 0 ? carry : key[0]) : up;
        }
#pragma unroll
        for (int i = 0; i < NK; ++i) {
            const int s = i * 32 + lane;
            if (s < KC) key[i] = s > at ? prev[i] : (s == at ? kx : key[i]);
        }
        kth = __shfl_sync(0xffffffffu, key[(KC - 1) / 32], (KC - 1) % 32);
    }
};

// Cooperative scan of bucket entries [ref, ref + cnt): lane j tests entries
// base + j and base + 32 + j of each 64-entry chunk (both loads in flight
// together); passing keys are inserted lowest entry first, each tested again
// against the k-th key at its turn.
template <int KC>
__device__ __forceinline__ void wq_insert_passing(unsigned long long kx, WarpList<KC> &L, int lane) {
    unsigned pass = __ballot_sync(0xffffffffu, kx < L.kth);
    while (pass) {
        const int src = __ffs(pass) - 1;
        pass &= pass - 1;
        L.insert(__shfl_sync(0xffffffffu, kx, src), lane);
    }
}

template <int DC, int KC>
__device__ __forceinline__ void wq_scan(const float4 *__restrict__ bucket, int ref, int cnt, const float *q,
                                        WarpList<KC> &L, int lane) {
    if (cnt <= 32) {   // one entry per lane
        unsigned long long k0 = WQ_NONE;
        if (lane < cnt) {
            float p0[DC];
            unsigned id0;
            load_point<DC>(bucket, ref + lane, p0, id0);
            k0 = pair_key(sqdist<DC>(q, p0), id0);
        }
        wq_insert_passing<KC>(k0, L, lane);
        return;
    }
    for (int base = 0; base < cnt; base += 64) {
        const bool ok0 = base + lane < cnt, ok1 = base + 32 + lane < cnt;
        float p0[DC], p1[DC];
        unsigned id0 = 0, id1 = 0;
        if (ok0) load_point<DC>(bucket, ref + base + lane, p0, id0);
        if (ok1) load_point<DC>(bucket, ref + base + 32 + lane, p1, id1);
        const unsigned long long k0 = ok0 ? pair_key(sqdist<DC>(q, p0), id0) : WQ_NONE;
        const unsigned long long k1 = ok1 ? pair_key(sqdist<DC>(q, p1), id1) : WQ_NONE;
        wq_insert_passing<KC>(k0, L, lane);
        if (base + 32 < cnt) wq_insert_passing<KC>(k1, L, lane);
    }
}

// Push `n_lanes` entries (one per lane with `want`) onto the warp's stack in
// lane order; sp is the same in every lane before and after.
__device__ __forceinline__ void wq_push(WqShared &S, int w, int &sp, bool want, int ref, int cnt, float d,
                                        unsigned below) {
    const unsigned m = __ballot_sync(0xffffffffu, want);
    if (want) {
        const int at = sp + __popc(m & below);
        S.s_ref[w][at] = ref;
        S.s_cnt[w][at] = cnt;
        S.s_d[w][at] = d;
    }
    sp += __popc(m);
}

__device__ __forceinline__ void wq_leaf(WqShared &S, int w, int &nl, bool want, int ref, int cnt, float d,
                                        unsigned below) {
    const unsigned m = __ballot_sync(0xffffffffu, want);
    if (want) {
        const int at = nl + __popc(m & below);
        S.l_ref[w][at] = ref;
        S.l_cnt[w][at] = cnt;
        S.l_d[w][at] = d;
    }
    nl += __popc(m);
}

// Search the subtrees on the warp's stack (all of one tree) until it is empty.
template <int DC, int KC>
__device__ __forceinline__ void wq_drain(WqShared &S, int w, int &sp, const TreeDesc &T, const float *q,
                                         WarpList<KC> &L, int lane) {
    constexpr int NW = node_w(DC);
    const unsigned below = (1u << lane) - 1u;
    while (sp > 0) {
        const int P = sp > WQ_WIDE_LIMIT ? 1 : min(32, sp);
        bool have = lane < P;
        int eref = 0, ecnt = 0;
        float ed = 0.f;
        if (have) {
            const int at = sp - 1 - lane;   // the top entry goes to lane 0
            eref = S.s_ref[w][at];
            ecnt = S.s_cnt[w][at];
            ed = S.s_d[w][at];
        }
        sp -= P;
        __syncwarp();
        const float kth = L.kth_dist();
        have = have && ed <= kth;
        // expand the popped internal nodes: near child first
        int rn = 0, cn = -1, rf = 0, cf = -1;
        float dn = 0.f, df = 0.f;
        if (have && ecnt == 0) {
            float rec[4 * NW];
            const float4 *np = T.nodes + (size_t)eref * NW;
#pragma unroll
            for (int x = 0; x < NW; ++x) {
                float4 f = __ldg(np + x);
                rec[4 * x] = f.x; rec[4 * x + 1] = f.y; rec[4 * x + 2] = f.z; rec[4 * x + 3] = f.w;
            }
            const int *ri = reinterpret_cast<const int *>(rec + 4 * DC);
            const float d0 = boxdist<DC>(q, rec, rec + DC);
            const float d1 = boxdist<DC>(q, rec + 2 * DC, rec + 3 * DC);
            const bool sw = d1 < d0;
            rn = sw ? ri[2] : ri[0]; cn = sw ? ri[3] : ri[1]; dn = sw ? d1 : d0;
            rf = sw ? ri[0] : ri[2]; cf = sw ? ri[1] : ri[3]; df = sw ? d0 : d1;
            if (!(dn <= kth)) cn = -1;
            if (!(df <= kth)) cf = -1;
        }
        // internal children onto the stack, far ones below near ones
        wq_push(S, w, sp, cf == 0, rf, 0, df, below);
        wq_push(S, w, sp, cn == 0, rn, 0, dn, below);
        // leaves of this round: popped ones and leaf children
        int nl = 0;
        wq_leaf(S, w, nl, have && ecnt > 0, eref, ecnt, ed, below);
        wq_leaf(S, w, nl, cn > 0, rn, cn, dn, below);
        wq_leaf(S, w, nl, cf > 0, rf, cf, df, below);
        __syncwarp();
        // scan them nearest first; stop at the first one beyond the k-th distance
        for (int t = 0; t < nl; ++t) {
            float best = __int_as_float(0x7f800000);
            int bi = -1;
            for (int i = lane; i < nl; i += 32) {
                const float d = S.l_d[w][i];
                if (d < best) { best = d; bi = i; }
            }
            const unsigned bb = __float_as_uint(best);
            const unsigned mn = __reduce_min_sync(0xffffffffu, bb);
            if (__uint_as_float(mn) > L.kth_dist()) break;   // every leaf left is farther (inf: all scanned)
            const int src = __ffs(__ballot_sync(0xffffffffu, bb == mn && bi >= 0)) - 1;
            const int li = __shfl_sync(0xffffffffu, bi, src);
            const int lref = S.l_ref[w][li], lcnt = S.l_cnt[w][li];
            __syncwarp();
            if (lane == 0) S.l_d[w][li] = __int_as_float(0x7f800000);
            __syncwarp();
            wq_scan<DC, KC>(T.bucket, lref, lcnt, q, L, lane);
        }
        __syncwarp();
    }
}

// One warp per query (position p of the processing order: bucket entry p for
// all-kNN, order[p] otherwise).  start_leaf as for k_knn_ww.
template <int DC, int KC>
__global__ void __launch_bounds__(WQ_THREADS) k_knn_warp(const TreeDesc *__restrict__ trees, int ntrees,
                                                         const float *__restrict__ queries,
                                                         const float4 *__restrict__ self_bucket,
                                                         const int32_t *__restrict__ order,
                                                         const int32_t *__restrict__ start_leaf, int64_t m,
                                                         int dim, int k, int32_t *__restrict__ out_idx,
                                                         float *__restrict__ out_dist) {
    constexpr int NW = node_w(DC);
    __shared__ WqShared S;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t pos = (int64_t)blockIdx.x * WQ_WARPS + w;
    if (pos >= m) return;   // warp-uniform
    const bool self = self_bucket != nullptr;
    float q[DC];
    int64_t row;
    if (self) {
        unsigned qid;
        load_point<DC>(self_bucket, pos, q, qid);
        row = (int64_t)qid;
    } else {
        row = order ? (int64_t)order[pos] : pos;
#pragma unroll
        for (int c = 0; c < DC; ++c) q[c] = c < dim ? __ldg(queries + row * dim + c) : 0.f;
    }
    WarpList<KC> L;
    L.init(k, lane);
    int sp = 0;
    const bool bottom = (self ? ntrees == 1 : start_leaf != nullptr) && trees[0].leaf_parent && trees[0].parent;
    if (bottom) {
        const TreeDesc &T = trees[0];
        const int64_t lp = self ? pos : (int64_t)start_leaf[pos];
        int up = __ldg(T.leaf_parent + lp);
        int lref = T.root_ref, lcnt = T.root_cnt;
        if (up >= 0) {
            const int2 rc = __ldg(reinterpret_cast<const int2 *>(
                reinterpret_cast<const float *>(T.nodes + (size_t)(up >> 1) * NW) + 4 * DC) + (up & 1));
            lref = rc.x;
            lcnt = rc.y;
        }
        if (lcnt > 0) wq_scan<DC, KC>(T.bucket, lref, lcnt, q, L, lane);
        // climb: every ancestor's other subtree goes on the stack, until the
        // k-th ball lies inside the subtree searched so far
        while (up >= 0) {
            const int pn = up >> 1, side = up & 1, other = 1 - side;
            const float *rec = reinterpret_cast<const float *>(T.nodes + (size_t)pn * NW);
            float lo[DC], hi[DC];
#pragma unroll
            for (int c = 0; c < DC; ++c) {
                lo[c] = __ldg(rec + side * 2 * DC + c);
                hi[c] = __ldg(rec + side * 2 * DC + DC + c);
            }
            if (ball_inside<DC>(q, lo, hi, dim, L.kth_dist())) break;
#pragma unroll
            for (int c = 0; c < DC; ++c) {
                lo[c] = __ldg(rec + other * 2 * DC + c);
                hi[c] = __ldg(rec + other * 2 * DC + DC + c);
            }
            const int2 rc = __ldg(reinterpret_cast<const int2 *>(rec + 4 * DC) + other);
            up = __ldg(T.parent + pn);
            const float ds = boxdist<DC>(q, lo, hi);
            if (rc.y >= 0 && ds <= L.kth_dist()) {
                if (lane == 0) {
                    S.s_ref[w][sp] = rc.x;
                    S.s_cnt[w][sp] = rc.y;
                    S.s_d[w][sp] = ds;
                }
                ++sp;
                if (sp > WQ_WIDE_LIMIT) {   // keep the bound of the stack: drain what is there
                    __syncwarp();
                    wq_drain<DC, KC>(S, w, sp, T, q, L, lane);
                }
            }
        }
        __syncwarp();
        wq_drain<DC, KC>(S, w, sp, T, q, L, lane);
    }
    {   // the other trees of a forest (all of them without a start leaf), each from its root
        for (int t = bottom ? 1 : 0; t < ntrees; ++t) {
            const TreeDesc &T = trees[t];
            if (T.root_cnt < 0) continue;
            float rlo[DC], rhi[DC];
#pragma unroll
            for (int c = 0; c < DC; ++c) { rlo[c] = T.root_lo[c]; rhi[c] = T.root_hi[c]; }
            const float dr = boxdist<DC>(q, rlo, rhi);
            if (!(dr <= L.kth_dist())) continue;
            if (lane == 0) {
                S.s_ref[w][0] = T.root_ref;
                S.s_cnt[w][0] = T.root_cnt;
                S.s_d[w][0] = dr;
            }
            sp = 1;
            __syncwarp();
            wq_drain<DC, KC>(S, w, sp, T, q, L, lane);
        }
    }
#pragma unroll
    for (int i = 0; i < WarpList<KC>::NK; ++i) {
        const int s = i * 32 + lane;
        if (s < KC && s >= KC - k) {
            const int o = s - (KC - k);
            const unsigned id = (unsigned)L.key[i];
            out_idx[row * k + o] = id == DEAD_ID ? -1 : (int32_t)id;
            out_dist[row * k + o] = __uint_as_float((unsigned)(L.key[i] >> 32));
        }
    }
}

template <int DC, int KC>
void launch_knn_warp(const TreeDesc *trees, int ntrees, const float *queries, const float4 *self_bucket,
                     const int32_t *order, const int32_t *start_leaf, int64_t m, int dim, int k, int32_t *out_idx,
                     float *out_dist, cudaStream_t s) {
    k_knn_warp<DC, KC><<<ceil_div_i(m, WQ_WARPS), WQ_THREADS, 0, s>>>(trees, ntrees, queries, self_bucket, order,
                                                                      start_leaf, m, dim, k, out_idx, out_dist);
}

}  // namespace pg
