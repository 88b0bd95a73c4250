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

// A (distance, id) pair is one 64-bit key: distances are >= 0, so their
// float bits order like unsigned integers, and (bits << 32 | id) orders
// exactly like (distance, id) lexicographically.  NaN (erased entries) sorts
// above +inf and is never taken.
__device__ __forceinline__ unsigned long long pair_key(float d, unsigned id) {
    return ((unsigned long long)__float_as_uint(d) << 32) | id;
}
constexpr unsigned long long PAD_KEY = (0x7f800000ull << 32) | 0xffffffffull;   // (+inf, no point)

template <int KC>
struct KList {
    unsigned long long key[KC];

    // Slots below KC-k hold the key 0, which never moves (nothing precedes
    // it), so a list of compile-time capacity KC serves any runtime k <= KC.
    __device__ __forceinline__ void init(int k) {
#pragma unroll
        for (int j = 0; j < KC; ++j) key[j] = j < KC - k ? 0ull : PAD_KEY;
    }
    __device__ __forceinline__ float kth() const { return __uint_as_float((unsigned)(key[KC - 1] >> 32)); }
    __device__ __forceinline__ unsigned long long kth_key() const { return key[KC - 1]; }
    __device__ __forceinline__ float dist(int j) const { return __uint_as_float((unsigned)(key[j] >> 32)); }
    __device__ __forceinline__ unsigned idx(int j) const { return (unsigned)key[j]; }

    // Insert (x, ix) if it precedes the current k-th pair.  Slot j takes slot
    // j-1 while the new key precedes it, else the new key once; each
    // comparison is made once and reused for the slot above.
    __device__ __forceinline__ void offer(float x, unsigned ix) {
        const unsigned long long kx = pair_key(x, ix);
        if (!(kx < key[KC - 1])) return;
        bool prev = true;
#pragma unroll
        for (int j = KC - 1; j > 0; --j) {
            const bool shift = kx < key[j - 1];
            key[j] = shift ? key[j - 1] : (prev ? kx : key[j]);
            prev = shift;
        }
        if (prev) key[0] = kx;
    }
    // Branch-free insertion executed by every lane of a warp; only lanes with
    // `ok` (and a pair that precedes the k-th) change their list.  Every
    // comparison reads the old list, so they are independent of each other.
    __device__ __forceinline__ void offer_pred(float x, unsigned ix, bool ok) {
        const unsigned long long kx = pair_key(x, ix);
        ok = ok && kx < key[KC - 1];
        bool prev = ok;   // x precedes slot j (old value)
#pragma unroll
        for (int j = KC - 1; j > 0; --j) {
            const bool shift = ok && kx < key[j - 1];
            const bool here = prev && !shift;
            key[j] = shift ? key[j - 1] : (here ? kx : key[j]);
            prev = shift;
        }
        if (prev) key[0] = kx;
    }
};

// The same k best pairs as a binary max-heap in shared memory, for large k:
// an insertion replaces the root (the k-th pair) and sifts the new key down,
// about log2(k) levels of two loads and one store instead of KC compare-and-
// select steps on registers, and the list costs no registers.  Slot j of
// thread t is word j * KNN_THREADS + t, so the 32 lanes of a warp always hit
// 32 different bank pairs, whatever slots they are at.  The root is also
// kept in a register (`top`) for the pruning tests.  Only the set of keys
// matters until the end, where a heapsort writes them out ascending: the
// answer is the same k smallest (distance, id) pairs as with KList.
template <int KC>
struct SmemHeap {
    static constexpr int LEVELS = KC >= 64 ? 7 : KC >= 32 ? 6 : KC >= 16 ? 5 : KC >= 8 ? 4 : KC >= 4 ? 3 : KC >= 2 ? 2 : 1;   // floor(log2 KC) + 1
    unsigned long long *h;
    unsigned long long top;
    int k;

    // base: KC * KNN_THREADS words of shared memory for the thread block
    __device__ __forceinline__ void init(unsigned long long *base, int k_) {
        h = base + threadIdx.x;
        k = k_;
        for (int j = 0; j < k; ++j) h[j * KNN_THREADS] = PAD_KEY;
        top = PAD_KEY;
    }
    __device__ __forceinline__ float kth() const { return __uint_as_float((unsigned)(top >> 32)); }
    __device__ __forceinline__ unsigned long long kth_key() const { return top; }

    // Sift key kx down from slot i of a heap of n slots; every lane of the
    // warp runs the same LEVELS steps, lanes without `act` change nothing.
    __device__ __forceinline__ void sift(unsigned long long kx, int i, int n, bool act) {
#pragma unroll
        for (int l = 0; l < LEVELS; ++l) {
            const int c = 2 * i + 1;
            const bool has = act && c < n;
            const unsigned long long a = has ? h[c * KNN_THREADS] : 0ull;
            const unsigned long long b = has && c + 1 < n ? h[(c + 1) * KNN_THREADS] : 0ull;
            const bool right = b > a;
            const unsigned long long m = right ? b : a;
            const bool down = has && m > kx;
            if (act) h[i * KNN_THREADS] = down ? m : kx;
            act = down;
            i = right ? c + 1 : c;
        }
    }
    __device__ __forceinline__ void offer_pred(float x, unsigned ix, bool ok) {
        const unsigned long long kx = pair_key(x, ix);
        ok = ok && kx < top;
        sift(kx, 0, k, ok);
        if (ok) top = h[0];
    }
    __device__ __forceinline__ void offer(float x, unsigned ix) {
        if (pair_key(x, ix) < top) offer_pred(x, ix, true);
    }
    // Heapsort: the largest goes last.  The heap ends in no particular state.
    __device__ __forceinline__ void write_sorted(int32_t *oi, float *od) {
        for (int n = k; n > 0; --n) {
            const unsigned long long r = h[0];
            oi[n - 1] = (unsigned)r == DEAD_ID ? -1 : (int32_t)(unsigned)r;
            od[n - 1] = __uint_as_float((unsigned)(r >> 32));
            if (n > 1) sift(h[(n - 1) * KNN_THREADS], 0, n - 1, true);
        }
    }
};

// NC: read through the non-coherent read-only path (data constant for the
// whole kernel); false for trees built earlier in the same kernel.
template <bool NC>
__device__ __forceinline__ float4 ld4(const float4 *p) { return NC ? __ldg(p) : *p; }
template <bool NC>
__device__ __forceinline__ float ld1(const float *p) { return NC ? __ldg(p) : *p; }

template <int DC, bool NC = true>
__device__ __forceinline__ void load_point(const float4 *__restrict__ bucket, int64_t i, float *p, unsigned &pid) {
    constexpr int W = bucket_w(DC);
    float v[4 * W];
#pragma unroll
    for (int w = 0; w < W; ++w) {
        float4 f = ld4<NC>(bucket + i * W + w);
        v[4 * w] = f.x; v[4 * w + 1] = f.y; v[4 * w + 2] = f.z; v[4 * w + 3] = f.w;
    }
#pragma unroll
    for (int c = 0; c < DC; ++c) p[c] = v[c];
    pid = __float_as_uint(v[DC]);
}

// True when every point within squared distance kth of q lies in the box
// [lo, hi] (the first `dim` coordinates; padding coordinates are zero for
// every point): q is inside and the squared gap to every face exceeds kth.
// A point outside the box lies beyond some face, and the rounded chain of
// sqdist is monotone in each term, so its distance is at least that face's
// squared gap: such a point cannot be within kth.
template <int DC>
__device__ __forceinline__ bool ball_inside(const float *q, const float *lo, const float *hi, int dim, float kth) {
    float g = fminf(__fsub_rn(q[0], lo[0]), __fsub_rn(hi[0], q[0]));
#pragma unroll
    for (int c = 1; c < DC; ++c)
        if (c < dim) g = fminf(g, fminf(__fsub_rn(q[c], lo[c]), __fsub_rn(hi[c], q[c])));
    return g > 0.f && __fmul_rn(g, g) > kth;
}

template <int DC, int KC, bool NC = true>
__device__ __forceinline__ void scan_leaf(const float4 *__restrict__ bucket, int ref, int cnt, const float *q,
                                          KList<KC> &L) {
    for (int i = ref; i < ref + cnt; ++i) {
        float p[DC];
        unsigned pid;
        load_point<DC, NC>(bucket, i, p, pid);
        const float d = sqdist<DC>(q, p);
        if (d <= L.kth()) L.offer(d, pid);   // cheap float test rejects most candidates
    }
}

template <int DC, int KC, bool NC = true>
__device__ __forceinline__ void search_tree(const TreeDesc &T, const float *q, KList<KC> &L) {
    if (T.root_cnt < 0) return;
    float rlo[DC], rhi[DC];
#pragma unroll
    for (int c = 0; c < DC; ++c) { rlo[c] = T.root_lo[c]; rhi[c] = T.root_hi[c]; }
    const float d_root = boxdist<DC>(q, rlo, rhi);
    if (d_root > L.kth()) return;
    if (T.root_cnt > 0) {
        scan_leaf<DC, KC, NC>(T.bucket, T.root_ref, T.root_cnt, q, L);
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
            scan_leaf<DC, KC, NC>(T.bucket, ref, cnt, q, L);
            continue;
        }
        for (;;) {
            float rec[4 * NW];
            const float4 *np = T.nodes + (size_t)ref * NW;
#pragma unroll
            for (int w = 0; w < NW; ++w) {
                float4 f = ld4<NC>(np + w);
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
                    scan_leaf<DC, KC, NC>(T.bucket, rn, cn, q, L);
                    break;
                }
                ref = rn;
                continue;
            }
            break;
        }
    }
}

// ---------------------------------------------------------------------------
// Thread-per-query traversal with postponed leaves ("while-while"): every lane
// walks nodes (one pop or node expansion per step) until it holds a leaf to
// scan or is finished; only when every lane of the warp is in that state do
// the lanes scan their leaves together, so leaf work, the bulk of the
// instructions, runs with the warp converged.  Candidates of a leaf chunk are
// first tested against the lane's k-th distance into a bit mask (a float
// compare: a candidate at exactly the k-th distance also passes, and the
// insertion's full (distance, id) compare decides it), and the insertions
// then run converged (as many rounds as the busiest lane needs).
// Each lane's pruning uses only its own k-th distance, so the answer is the
// same exact k-NN as the other variants.
template <int DC, int KC, bool NC = true, bool COUNT = false, class LT = KList<KC>>
__device__ __forceinline__ void scan_own_leaf_converged(const float4 *__restrict__ bucket, int lref, int lcnt,
                                                        const float *q, LT &L, unsigned &cand) {
    const int maxc = __reduce_max_sync(0xffffffffu, lcnt);
    for (int base = 0; base < maxc; base += 32) {
        const int n = min(32, maxc - base);
        unsigned mask = 0;
        const float kf = L.kth();
        for (int j = 0; j < n; ++j) {
            if (base + j < lcnt) {
                float p[DC];
                unsigned pid;
                load_point<DC, NC>(bucket, lref + base + j, p, pid);
                if (COUNT) ++cand;
                const float dd = sqdist<DC>(q, p);
                mask |= (dd <= kf ? 1u : 0u) << j;
            }
        }
        const int rounds = __reduce_max_sync(0xffffffffu, __popc(mask));
        for (int t = 0; t < rounds; ++t) {
            const bool act = mask != 0;
            const int j = act ? __ffs(mask) - 1 : 0;
            mask &= mask - 1;
            float p[DC];
            unsigned pid;
            load_point<DC, NC>(bucket, act ? lref + base + j : lref, p, pid);
            if (COUNT && act) ++cand;
            L.offer_pred(sqdist<DC>(q, p), pid, act);
        }
    }
}

// COUNT: also count, per lane, the node records and bucket entries it loads
// (the touched-bytes model of the traversal; a separate instantiation).
template <int DC, int KC, bool NC = true, bool COUNT = false, class LT = KList<KC>>
__device__ __forceinline__ void search_tree_ww(const TreeDesc &T, const float *q, bool valid, LT &L,
                                               unsigned &nrec, unsigned &cand) {
    constexpr int NW = node_w(DC);
    int s_ref[KNN_STACK], s_cnt[KNN_STACK];
    float s_d[KNN_STACK];
    int sp = 0, ref = -1, lref = 0, lcnt = 0;
    bool done = !valid || T.root_cnt < 0;
    if (!done) {
        float rlo[DC], rhi[DC];
#pragma unroll
        for (int c = 0; c < DC; ++c) { rlo[c] = T.root_lo[c]; rhi[c] = T.root_hi[c]; }
        const float dr = boxdist<DC>(q, rlo, rhi);
        if (dr > L.kth()) done = true;
        else if (T.root_cnt > 0) { lref = T.root_ref; lcnt = T.root_cnt; }
        else ref = T.root_ref;
    }
    for (;;) {
        // node phase: lanes without a pending leaf advance until they get one
        for (;;) {
            const bool need = !done && lcnt == 0;
            if (!__any_sync(0xffffffffu, need)) break;
            if (need) {
                if (ref < 0) {
                    if (sp == 0) {
                        done = true;
                    } else {
                        --sp;
                        if (s_d[sp] <= L.kth()) {
                            if (s_cnt[sp] > 0) { lref = s_ref[sp]; lcnt = s_cnt[sp]; }
                            else ref = s_ref[sp];
                        }
                    }
                }
                if (ref >= 0) {
                    if (COUNT) ++nrec;
                    float rec[4 * NW];
                    const float4 *np = T.nodes + (size_t)ref * NW;
#pragma unroll
                    for (int w = 0; w < NW; ++w) {
                        float4 f = ld4<NC>(np + w);
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
                    ref = -1;
                    if (cn >= 0 && dn <= kth) {
                        if (cn > 0) { lref = rn; lcnt = cn; }
                        else ref = rn;
                    }
                }
            }
        }
        if (!__any_sync(0xffffffffu, lcnt > 0)) break;
        // leaf phase, converged
        scan_own_leaf_converged<DC, KC, NC, COUNT>(T.bucket, lref, lcnt, q, L, cand);
        lcnt = 0;
    }
}

// All-kNN with postponed leaves, from the bottom: the query is bucket entry
// `pos`, so its own leaf is known and is queued first (it gives the lane a
// close k-th distance at once); the lane then climbs the parent links and, at
// each ancestor, searches only the other child's subtree (every point lies in
// the own leaf or in exactly one such sibling subtree, so the answer is the
// same exact k-NN).  Leaves found by the walk go to a queue of two: a lane
// that already holds a leaf keeps walking while some other lane of the warp
// still looks for one, so fewer lanes idle in the node phase.  A queued leaf
// is tested again against the k-th distance when it is taken.
template <int DC, int KC, bool COUNT = false, class LT = KList<KC>>
__device__ __forceinline__ void search_self_ww(const TreeDesc &T, int64_t pos, const float *q, int dim, bool valid,
                                               LT &L, unsigned &nrec, unsigned &cand) {
    constexpr int NW = node_w(DC);
    int s_ref[KNN_STACK], s_cnt[KNN_STACK];
    float s_d[KNN_STACK];
    int sp = 0, cur = -1, up = -1, qn = 0;
    int q0r = 0, q0c = 0, q1r = 0, q1c = 0;   // leaf queue: (ref, cnt, bound), entry 0 taken first
    float q0d = 0.f, q1d = 0.f;
    bool done = !valid;
    auto enqueue = [&](int r, int c, float d) {
        if (qn == 0) { q0r = r; q0c = c; q0d = d; }
        else { q1r = r; q1c = c; q1d = d; }
        ++qn;
    };
    if (valid) {
        const int code = __ldg(T.leaf_parent + pos);
        if (code < 0) {
            enqueue(T.root_ref, T.root_cnt, 0.f);
        } else {
            const int2 rc = __ldg(reinterpret_cast<const int2 *>(
                reinterpret_cast<const float *>(T.nodes + (size_t)(code >> 1) * NW) + 4 * DC) + (code & 1));
            enqueue(rc.x, rc.y, 0.f);
        }
        up = code;
    }
    for (;;) {
        // node phase: lanes with a free queue slot advance while some lane has no leaf
        for (;;) {
            if (!__any_sync(0xffffffffu, !done && qn == 0)) break;
            if (!done && qn < 2) {
                if (cur < 0) {
                    if (sp > 0) {
                        --sp;
                        if (s_d[sp] <= L.kth()) {
                            if (s_cnt[sp] > 0) enqueue(s_ref[sp], s_cnt[sp], s_d[sp]);
                            else cur = s_ref[sp];
                        }
                    } else if (up >= 0) {
                        // climb: the other child of the next ancestor, unless
                        // the k-th ball lies inside the subtree searched so far
                        const int pn = up >> 1, side = up & 1, other = 1 - side;
                        const float *rec = reinterpret_cast<const float *>(T.nodes + (size_t)pn * NW);
                        float lo[DC], hi[DC];
#pragma unroll
                        for (int c = 0; c < DC; ++c) {
                            lo[c] = __ldg(rec + side * 2 * DC + c);
                            hi[c] = __ldg(rec + side * 2 * DC + DC + c);
                        }
                        if (ball_inside<DC>(q, lo, hi, dim, L.kth())) {
                            up = -1;
                        } else {
#pragma unroll
                            for (int c = 0; c < DC; ++c) {
                                lo[c] = __ldg(rec + other * 2 * DC + c);
                                hi[c] = __ldg(rec + other * 2 * DC + DC + c);
                            }
                            const int2 rc = __ldg(reinterpret_cast<const int2 *>(rec + 4 * DC) + other);
                            up = __ldg(T.parent + pn);
                            const float ds = boxdist<DC>(q, lo, hi);
                            if (rc.y >= 0 && ds <= L.kth()) {
                                if (rc.y > 0) enqueue(rc.x, rc.y, ds);
                                else cur = rc.x;
                            }
                        }
                    } else {
                        done = true;
                    }
                }
                if (cur >= 0) {
                    if (COUNT) ++nrec;
                    float rec[4 * NW];
                    const float4 *np = T.nodes + (size_t)cur * NW;
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
                    cur = -1;
                    if (cn >= 0 && dn <= kth) {
                        if (cn > 0) enqueue(rn, cn, dn);
                        else cur = rn;
                    }
                }
            }
        }
        if (!__any_sync(0xffffffffu, qn > 0)) break;
        // leaf phase, converged: every lane takes its first queued leaf
        int lref = 0, lcnt = 0;
        if (qn > 0) {
            if (q0d <= L.kth()) { lref = q0r; lcnt = q0c; }
            q0r = q1r; q0c = q1c; q0d = q1d;
            --qn;
        }
        scan_own_leaf_converged<DC, KC, true, COUNT>(T.bucket, lref, lcnt, q, L, cand);
    }
}

// Where the postponed-leaf search of each query starts.  Each launch uses an
// instance compiled for its own case only (the counting instance decides at
// run time), since paths that are never taken still cost registers and
// scheduling in the ones that are.
enum WwMode : int {
    WW_ANY = 0,     // decided per launch: the cases below, by their conditions
    WW_TOP = 1,     // every tree from its root (forests; queries without a start leaf)
    WW_SELF = 2,    // all-kNN: the query is bucket entry pos of the single tree
    WW_START = 3,   // separate queries from start_leaf[pos] in tree 0, then the other trees from their roots
};

// The k-list of the postponed-leaf kernel: registers, or (HEAP) a max-heap in
// KC * KNN_THREADS words of dynamic shared memory.
template <bool HEAP, int KC>
struct WwList { using type = KList<KC>; };
template <int KC>
struct WwList<true, KC> { using type = SmemHeap<KC>; };

template <int DC, int KC, bool COUNT = false, int MODE = WW_ANY, bool HEAP = false>
__global__ void __launch_bounds__(KNN_THREADS) k_knn_ww(const TreeDesc *__restrict__ trees, int ntrees,
                                                        const float *__restrict__ queries,
                                                        const float4 *__restrict__ self_bucket,
                                                        const int32_t *__restrict__ order,
                                                        const int32_t *__restrict__ start_leaf, int64_t m, int dim,
                                                        int k, int32_t *__restrict__ out_idx,
                                                        float *__restrict__ out_dist,
                                                        unsigned long long *__restrict__ touch = nullptr) {
    const int64_t pos = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = pos < m;
    float q[DC];
    int64_t row = 0;
#pragma unroll
    for (int c = 0; c < DC; ++c) q[c] = 0.f;
    const bool self = MODE == WW_SELF || (MODE != WW_START && self_bucket != nullptr);
    if (valid) {
        if (self) {
            unsigned qid;
            load_point<DC>(self_bucket, pos, q, qid);
            row = (int64_t)qid;
        } else {
            row = order ? (int64_t)order[pos] : pos;
#pragma unroll
            for (int c = 0; c < DC; ++c) q[c] = c < dim ? queries[row * dim + c] : 0.f;
        }
    }
    typename WwList<HEAP, KC>::type L;
    if constexpr (HEAP) {
        extern __shared__ unsigned long long ww_heap[];
        L.init(ww_heap, k);
    } else {
        L.init(k);
    }
    unsigned nrec = 0, cand = 0;
    bool bottom = MODE == WW_SELF || MODE == WW_START;
    if (MODE == WW_ANY)
        bottom = (self ? ntrees == 1 : start_leaf != nullptr) && trees[0].leaf_parent && trees[0].parent;
    // from the start leaf in tree 0 (all-kNN: the query's own entry), then the
    // other trees of a forest from their roots with the k-list tree 0 left
    if (bottom)
        search_self_ww<DC, KC, COUNT>(trees[0], self ? pos : (valid ? (int64_t)start_leaf[pos] : 0), q, dim, valid,
                                      L, nrec, cand);
    for (int t = bottom ? 1 : 0; t < ntrees; ++t) search_tree_ww<DC, KC, true, COUNT>(trees[t], q, valid, L, nrec, cand);
    if (COUNT) {
        unsigned long long a = nrec, b = cand;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            b += __shfl_xor_sync(0xffffffffu, b, o);
        }
        if ((threadIdx.x & 31) == 0) {
            atomicAdd(touch, a);
            atomicAdd(touch + 1, b);
        }
    }
    if (!valid) return;
    int32_t *oi = out_idx + row * k;
    float *od = out_dist + row * k;
    if constexpr (HEAP) {
        L.write_sorted(oi, od);
    } else {
#pragma unroll
        for (int j = 0; j < KC; ++j) {
            if (j >= KC - k) {
                const int o = j - (KC - k);
                oi[o] = L.idx(j) == DEAD_ID ? -1 : (int32_t)L.idx(j);
                od[o] = L.dist(j);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Packet traversal: the 32 queries of a warp, adjacent in tree order (bucket
// order for all-kNN, leaf-sorted order for separate queries), share one walk
// through the tree.  A child is entered when ANY lane still needs it (its box
// is within that lane's k-th distance); every lane scans every entered leaf
// against broadcast loads of the leaf's points.  Control flow is warp-uniform,
// so no lane idles on divergence; lanes that did not need a leaf just fail
// the k-th-distance test.  Each lane's k-list is still exact: a lane skips a
// subtree only when its own box distance exceeds its own k-th distance.
// The stack lives in registers spread over the lanes (entry e in lane e%32).
constexpr int PKT_THREADS = 128;

struct PktStack {
    int ref0, ref1, cnt0, cnt1, box0, box1;   // box = 2*node + side, or -1 for a tree root
    int sp;
    __device__ __forceinline__ void push(int lane, int ref, int cnt, int box) {
        if (sp < 2 * 32) {
            if (lane == (sp & 31)) {
                if (sp < 32) { ref0 = ref; cnt0 = cnt; box0 = box; }
                else { ref1 = ref; cnt1 = cnt; box1 = box; }
            }
            ++sp;
        }
    }
    __device__ __forceinline__ void pop(int &ref, int &cnt, int &box) {
        --sp;
        const int src = sp & 31;
        const bool lo = sp < 32;
        ref = __shfl_sync(0xffffffffu, lo ? ref0 : ref1, src);
        cnt = __shfl_sync(0xffffffffu, lo ? cnt0 : cnt1, src);
        box = __shfl_sync(0xffffffffu, lo ? box0 : box1, src);
    }
};

// Scan bucket entries [ref, ref+cnt) for every lane of the warp, skipping the
// entries in [skip0, skip1) (already offered by the warm start).  Entries are
// taken 32 at a time: every lane first tests all of them against its current
// k-th pair and records the ones that pass in a bit mask; the insertions then
// run converged, as many rounds as the busiest lane needs, so a lane's
// insertion never stalls the other 31.
template <int DC, int KC, bool NC = true>
__device__ __forceinline__ void scan_leaf_packet(const float4 *__restrict__ bucket, int ref, int cnt,
                                                 const float *q, KList<KC> &L, int skip0 = 0, int skip1 = 0) {
    // the part not yet offered: up to two pieces around the contiguous window
    int r0 = ref, r1 = ref + cnt, r2 = 0, r3 = 0;
    if (skip1 > skip0 && skip0 < r1 && r0 < skip1) {
        const int e = r1;
        r1 = max(r0, min(r1, skip0));
        r2 = max(skip1, r0);
        r3 = e > skip1 ? e : r2;
    }
    for (int piece = 0; piece < 2; ++piece) {
        const int lo = piece ? r2 : r0, hi = piece ? r3 : r1;
    for (int base = lo; base < hi; base += 32) {
        const int n = min(32, hi - base);
        unsigned mask = 0;
        const unsigned long long kk = L.kth_key();
#pragma unroll 4
        for (int j = 0; j < n; ++j) {
            float p[DC];
            unsigned pid;
            load_point<DC, NC>(bucket, base + j, p, pid);
            const float dd = sqdist<DC>(q, p);
            mask |= (pair_key(dd, pid) < kk ? 1u : 0u) << j;
        }
        const int rounds = __reduce_max_sync(0xffffffffu, __popc(mask));
        for (int t = 0; t < rounds; ++t) {
            const bool act = mask != 0;
            const int j = act ? __ffs(mask) - 1 : 0;
            mask &= mask - 1;
            float p[DC];
            unsigned pid;
            load_point<DC, NC>(bucket, base + j, p, pid);
            L.offer_pred(sqdist<DC>(q, p), pid, act);
        }
    }
    }
}

template <int DC, int KC, bool NC = true>
__device__ __forceinline__ void search_tree_packet(const TreeDesc &T, const float *q, bool valid, int lane,
                                                   KList<KC> &L, int skip0 = 0, int skip1 = 0) {
    constexpr int NW = node_w(DC);
    const int root_cnt = T.root_cnt;
    if (root_cnt < 0) return;
    float rlo[DC], rhi[DC];
#pragma unroll
    for (int c = 0; c < DC; ++c) { rlo[c] = T.root_lo[c]; rhi[c] = T.root_hi[c]; }
    {
        const float dr = boxdist<DC>(q, rlo, rhi);
        if (!__any_sync(0xffffffffu, valid && dr <= L.kth())) return;
    }
    if (root_cnt > 0) {
        scan_leaf_packet<DC, KC, NC>(T.bucket, T.root_ref, root_cnt, q, L, skip0, skip1);
        return;
    }
    PktStack st;
    st.sp = 0;
    st.push(lane, T.root_ref, 0, -1);
    while (st.sp > 0) {
        int ref, cnt, box;
        st.pop(ref, cnt, box);
        float d;
        if (box < 0) {
            d = boxdist<DC>(q, rlo, rhi);
        } else {
            const float *rec = reinterpret_cast<const float *>(T.nodes + (size_t)(box >> 1) * NW);
            float lo[DC], hi[DC];
            const int off = (box & 1) * 2 * DC;
#pragma unroll
            for (int c = 0; c < DC; ++c) { lo[c] = ld1<NC>(rec + off + c); hi[c] = ld1<NC>(rec + off + DC + c); }
            d = boxdist<DC>(q, lo, hi);
        }
        if (!__any_sync(0xffffffffu, valid && d <= L.kth())) continue;
        if (cnt > 0) {
            scan_leaf_packet<DC, KC, NC>(T.bucket, ref, cnt, q, L, skip0, skip1);
            continue;
        }
        for (;;) {
            float rec[4 * NW];
            const float4 *np = T.nodes + (size_t)ref * NW;
#pragma unroll
            for (int w = 0; w < NW; ++w) {
                float4 f = ld4<NC>(np + w);
                rec[4 * w] = f.x; rec[4 * w + 1] = f.y; rec[4 * w + 2] = f.z; rec[4 * w + 3] = f.w;
            }
            const int *ri = reinterpret_cast<const int *>(rec + 4 * DC);
            const int r0 = ri[0], c0 = ri[1], r1 = ri[2], c1 = ri[3];
            const float d0 = boxdist<DC>(q, rec, rec + DC);
            const float d1 = boxdist<DC>(q, rec + 2 * DC, rec + 3 * DC);
            const float kth = L.kth();
            const bool n0 = valid && c0 >= 0 && d0 <= kth;
            const bool n1 = valid && c1 >= 0 && d1 <= kth;
            const unsigned b0 = __ballot_sync(0xffffffffu, n0);
            const unsigned b1 = __ballot_sync(0xffffffffu, n1);
            if (!(b0 | b1)) break;
            int first;
            if (b0 && b1) {
                // majority vote on which child is nearer among lanes that need it
                const int v0 = __popc(__ballot_sync(0xffffffffu, n0 && (!n1 || d0 <= d1)));
                const int v1 = __popc(__ballot_sync(0xffffffffu, n1 && (!n0 || d1 < d0)));
                first = v0 >= v1 ? 0 : 1;
                if (first == 0) st.push(lane, r1, c1, 2 * ref + 1);
                else st.push(lane, r0, c0, 2 * ref);
            } else {
                first = b0 ? 0 : 1;
            }
            const int rf = first ? r1 : r0, cf = first ? c1 : c0;
            if (cf > 0) {
                scan_leaf_packet<DC, KC, NC>(T.bucket, rf, cf, q, L, skip0, skip1);
                break;
            }
            ref = rf;
        }
    }
}

// Warp-coherent k-NN.  Processing position p = warp*32 + lane; with
// self_bucket the query is bucket entry p (all-kNN); otherwise it is query
// order[p] (or p when order is NULL).
template <int DC, int KC>
__global__ void __launch_bounds__(PKT_THREADS) k_knn_packet(const TreeDesc *__restrict__ trees, int ntrees,
                                                            const float *__restrict__ queries,
                                                            const float4 *__restrict__ self_bucket,
                                                            const int32_t *__restrict__ order, int64_t m, int dim,
                                                            int k, int32_t *__restrict__ out_idx,
                                                            float *__restrict__ out_dist) {
    const int lane = threadIdx.x & 31;
    const int64_t pos = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = pos < m;
    float q[DC];
    int64_t row = 0;
#pragma unroll
    for (int c = 0; c < DC; ++c) q[c] = 0.f;
    if (valid) {
        if (self_bucket) {
            unsigned qid;
            load_point<DC>(self_bucket, pos, q, qid);
            row = (int64_t)qid;
        } else {
            row = order ? (int64_t)order[pos] : pos;
#pragma unroll
            for (int c = 0; c < DC; ++c) q[c] = c < dim ? queries[row * dim + c] : 0.f;
        }
    }
    KList<KC> L;
    L.init(k);
    if (self_bucket) {
        // warm start: the warp's own bucket window (its queries and their
        // neighbours in tree order) gives every lane a close k-th distance
        // before the search; the search then skips that window.
        const int64_t w0 = pos - lane;
        const int64_t wl = max((int64_t)0, w0 - 16), wh = min(m, w0 + 48);
        scan_leaf_packet<DC, KC>(self_bucket, (int)wl, (int)(wh - wl), q, L);
        search_tree_packet<DC, KC>(trees[0], q, valid, lane, L, (int)wl, (int)wh);
    } else {
        for (int t = 0; t < ntrees; ++t) search_tree_packet<DC, KC>(trees[t], q, valid, lane, L);
    }
    if (!valid) return;
    int32_t *oi = out_idx + row * k;
    float *od = out_dist + row * k;
#pragma unroll
    for (int j = 0; j < KC; ++j) {
        if (j >= KC - k) {
            const int o = j - (KC - k);
            oi[o] = L.idx(j) == DEAD_ID ? -1 : (int32_t)L.idx(j);
            od[o] = L.dist(j);
        }
    }
}

// All-kNN from the bottom: a query that is itself bucket entry `pos` starts in
// its own leaf (which gives it a close k-th distance at once), then walks up
// the parent links; at every ancestor only the other child's subtree can hold
// points not seen yet, and it is searched top-down when its box is within the
// k-th distance.  Every point lies in the own leaf or in exactly one such
// sibling subtree, so the answer is the same exact k-NN, without the
// top-down descent from the root.
template <int DC, int KC>
__device__ __forceinline__ void search_self_up(const TreeDesc &T, int64_t pos, const float *q, int dim, KList<KC> &L) {
    constexpr int NW = node_w(DC);
    int code = __ldg(T.leaf_parent + pos);
    {
        int lref, lcnt;
        if (code < 0) { lref = T.root_ref; lcnt = T.root_cnt; }
        else {
            const int2 rc = __ldg(reinterpret_cast<const int2 *>(reinterpret_cast<const float *>(T.nodes + (size_t)(code >> 1) * NW) + 4 * DC) + (code & 1));
            lref = rc.x;
            lcnt = rc.y;
        }
        scan_leaf<DC, KC>(T.bucket, lref, lcnt, q, L);
    }
    int s_ref[KNN_STACK], s_cnt[KNN_STACK];
    float s_d[KNN_STACK];
    while (code >= 0) {
        const int pn = code >> 1, side = code & 1, other = 1 - side;
        const float *rec = reinterpret_cast<const float *>(T.nodes + (size_t)pn * NW);
        float lo[DC], hi[DC];
#pragma unroll
        for (int c = 0; c < DC; ++c) { lo[c] = __ldg(rec + side * 2 * DC + c); hi[c] = __ldg(rec + side * 2 * DC + DC + c); }
        // the k-th ball inside the subtree searched so far: nothing above can hold a neighbour
        if (ball_inside<DC>(q, lo, hi, dim, L.kth())) break;
#pragma unroll
        for (int c = 0; c < DC; ++c) { lo[c] = __ldg(rec + other * 2 * DC + c); hi[c] = __ldg(rec + other * 2 * DC + DC + c); }
        const int2 rc = __ldg(reinterpret_cast<const int2 *>(rec + 4 * DC) + other);
        code = __ldg(T.parent + pn);
        const float ds = boxdist<DC>(q, lo, hi);
        if (rc.y < 0 || ds > L.kth()) continue;
        if (rc.y > 0) {
            scan_leaf<DC, KC>(T.bucket, rc.x, rc.y, q, L);
            continue;
        }
        // top-down search of the sibling subtree
        int sp = 0;
        s_ref[0] = rc.x; s_cnt[0] = 0; s_d[0] = ds; sp = 1;
        while (sp > 0) {
            --sp;
            int ref = s_ref[sp];
            const int cnt = s_cnt[sp];
            if (s_d[sp] > L.kth()) continue;
            if (cnt > 0) {
                scan_leaf<DC, KC>(T.bucket, ref, cnt, q, L);
                continue;
            }
            for (;;) {
                float r[4 * NW];
                const float4 *np = T.nodes + (size_t)ref * NW;
#pragma unroll
                for (int w = 0; w < NW; ++w) {
                    float4 f = __ldg(np + w);
                    r[4 * w] = f.x; r[4 * w + 1] = f.y; r[4 * w + 2] = f.z; r[4 * w + 3] = f.w;
                }
                const int *ri = reinterpret_cast<const int *>(r + 4 * DC);
                const int r0 = ri[0], c0 = ri[1], r1 = ri[2], c1 = ri[3];
                const float d0 = boxdist<DC>(q, r, r + DC);
                const float d1 = boxdist<DC>(q, r + 2 * DC, r + 3 * DC);
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
    if (self_bucket && trees[0].leaf_parent && trees[0].parent) {
        search_self_up<DC, KC>(trees[0], qi, q, dim, L);
    } else {
        for (int t = 0; t < ntrees; ++t) search_tree<DC, KC>(trees[t], q, L);
    }
    int32_t *oi = out_idx + row * k;
    float *od = out_dist + row * k;
#pragma unroll
    for (int j = 0; j < KC; ++j) {
        if (j >= KC - k) {
            const int o = j - (KC - k);
            oi[o] = L.idx(j) == DEAD_ID ? -1 : (int32_t)L.idx(j);
            od[o] = L.dist(j);
        }
    }
}

// PG_KNN_POSTPONED_HEAP: the postponed-leaf kernel with its k-list as a
// shared-memory heap for list capacities from 16; smaller lists stay in
// registers (the PG_KNN_POSTPONED instances).
template <int DC, int KC, int MODE>
cudaError_t launch_knn_ww_mode(const TreeDesc *trees, int ntrees, const float *queries, const float4 *self_bucket,
                               const int32_t *order, const int32_t *start_leaf, int64_t m, int dim, int k,
                               int32_t *out_idx, float *out_dist, bool heap, cudaStream_t s) {
    constexpr bool CAN_HEAP = KC >= 16;
    if (CAN_HEAP && heap) {
        constexpr int smem = KC * KNN_THREADS * (int)sizeof(unsigned long long);
        const cudaError_t e = cudaFuncSetAttribute(k_knn_ww<DC, KC, false, MODE, CAN_HEAP>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        k_knn_ww<DC, KC, false, MODE, CAN_HEAP><<<ceil_div_i(m, KNN_THREADS), KNN_THREADS, smem, s>>>(
            trees, ntrees, queries, self_bucket, order, start_leaf, m, dim, k, out_idx, out_dist);
    } else {
        k_knn_ww<DC, KC, false, MODE><<<ceil_div_i(m, KNN_THREADS), KNN_THREADS, 0, s>>>(
            trees, ntrees, queries, self_bucket, order, start_leaf, m, dim, k, out_idx, out_dist);
    }
    return cudaSuccess;
}

// The start mode of a postponed-leaf launch: all-kNN from the own entry,
// separate queries from their start leaves, else every tree from its root.
template <int DC, int KC>
cudaError_t launch_knn_ww(const TreeDesc *trees, int ntrees, const float *queries, const float4 *self_bucket,
                          const int32_t *order, const int32_t *start_leaf, int64_t m, int dim, int k,
                          int32_t *out_idx, float *out_dist, bool heap, cudaStream_t s) {
    if (self_bucket)
        return launch_knn_ww_mode<DC, KC, WW_SELF>(trees, ntrees, queries, self_bucket, order, start_leaf, m, dim, k,
                                                   out_idx, out_dist, heap, s);
    if (start_leaf)
        return launch_knn_ww_mode<DC, KC, WW_START>(trees, ntrees, queries, self_bucket, order, start_leaf, m, dim,
                                                    k, out_idx, out_dist, heap, s);
    return launch_knn_ww_mode<DC, KC, WW_TOP>(trees, ntrees, queries, self_bucket, order, start_leaf, m, dim, k,
                                              out_idx, out_dist, heap, s);
}

}  // namespace pg

#include "knn_warp.cuh"

// Host launcher for one dimension class: picks the list capacity KC >= k and
// the traversal kernel for the resolved variant (PG_KNN_THREAD,
// PG_KNN_POSTPONED[_HEAP], PG_KNN_WARP, the counting instance, else warp
// packets).
#define PG_KNN_CASE(DCN, KCN)                                                                              \
    case KCN:                                                                                              \
        if (variant == PG_KNN_THREAD)                                                                      \
            k_knn<DCN, KCN><<<ceil_div_i(m, KNN_THREADS), KNN_THREADS, 0, s>>>(trees, ntrees, queries,      \
                                                                               self_bucket, m, dim, k,     \
                                                                               out_idx, out_dist);         \
        else if (variant == PG_KNN_POSTPONED || variant == PG_KNN_POSTPONED_HEAP) {                        \
            if (launch_knn_ww<DCN, KCN>(trees, ntrees, queries, self_bucket, order, start_leaf, m, dim, k,   \
                                        out_idx, out_dist, variant == PG_KNN_POSTPONED_HEAP, s) !=          \
                cudaSuccess)                                                                               \
                return fail(PG_ECUDA, "k-NN: shared-memory size of the heap traversal");                  \
        }                                                                                                  \
        else if (variant == PG_KNN_WARP)                                                                   \
            launch_knn_warp<DCN, KCN>(trees, ntrees, queries, self_bucket, order, start_leaf, m, dim, k,     \
                                      out_idx, out_dist, s);                                               \
        else if (variant == kKnnCountingInstance)                                                          \
            k_knn_ww<DCN, KCN, true><<<ceil_div_i(m, KNN_THREADS), KNN_THREADS, 0, s>>>(                   \
                trees, ntrees, queries, self_bucket, order, start_leaf, m, dim, k, out_idx, out_dist,      \
                touch);                                                                                    \
        else                                                                                               \
            k_knn_packet<DCN, KCN><<<ceil_div_i(m, PKT_THREADS), PKT_THREADS, 0, s>>>(                     \
                trees, ntrees, queries, self_bucket, order, m, dim, k, out_idx, out_dist);                 \
        break;

#define PG_DEFINE_KNN_LAUNCH(DCN)                                                                          \
    namespace pg {                                                                                         \
    pg_status knn_launch_dc##DCN(const TreeDesc *trees, int ntrees, const float *queries,                  \
                                 const float4 *self_bucket, const int32_t *order,                          \
                                 const int32_t *start_leaf, int64_t m, int dim,                            \
                                 int k, int32_t *out_idx, float *out_dist, int variant,                    \
                                 unsigned long long *touch, cudaStream_t s) {                              \
        KTimer kt("knn_traverse", s);                                                                      \
        switch (k_class(k)) {                                                                              \
            PG_KNN_CASE(DCN, 1)                                                                            \
            PG_KNN_CASE(DCN, 2)                                                                            \
            PG_KNN_CASE(DCN, 4)                                                                            \
            PG_KNN_CASE(DCN, 8)                                                                            \
            PG_KNN_CASE(DCN, 10)                                                                           \
            PG_KNN_CASE(DCN, 16)                                                                           \
            PG_KNN_CASE(DCN, 32)                                                                           \
            PG_KNN_CASE(DCN, 64)                                                                           \
            default: return fail(PG_EINVAL, "k out of range");                                             \
        }                                                                                                  \
        count_launch();                                                                                    \
        return check_launch("knn traverse");                                                               \
    }                                                                                                      \
    }
