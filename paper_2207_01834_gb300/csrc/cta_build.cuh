// kd-tree construction by ONE thread block over a contiguous range of points
// (paper Section 5 intro, spatial-median split of Section 6, recursive
// construction of Appendix A.1.1 done level by level).
//
// The block runs the same level-synchronous steps as the device-wide builder,
// with block barriers instead of kernel boundaries: classify segments, number
// the split nodes by a block-wide scan, link children into their parents, flag
// the points that go left, scan the flags, scatter stably, and reduce the
// children's tight boxes.  Everything lives in global scratch slices owned by
// this block, so many blocks can build many independent trees at once.
#pragma once

#include <climits>

#include "common.cuh"

namespace pg {

// Words of per-tree scratch a block needs for n points (see CtaScratch).
__host__ __device__ inline int64_t cta_seg_cap(int64_t n, int leaf) { return 2 * (n / (leaf + 1)) + 2; }
__host__ __device__ inline int64_t cta_scratch_words(int64_t n, int leaf, int dc) {
    const int64_t sc = cta_seg_cap(n, leaf);
    return 2 * (5 + 2 * (int64_t)dc) * sc + 4 * sc + 1 + 4 * n + 1;
}

struct CtaSegs {
    int *start, *end, *parent, *side, *depth, *lo, *hi;
};

template <int DC>
struct CtaScratch {
    CtaSegs a, b;
    int *split, *rank, *sdim;
    float *sval;
    int *seg_a, *seg_b, *flag, *pre;
    __device__ void carve(int *base, int64_t n, int leaf) {
        const int64_t sc = cta_seg_cap(n, leaf);
        int *p = base;
        auto segs = [&](CtaSegs &g) {
            g.start = p; p += sc; g.end = p; p += sc; g.parent = p; p += sc; g.side = p; p += sc;
            g.depth = p; p += sc; g.lo = p; p += sc * DC; g.hi = p; p += sc * DC;
        };
        segs(a);
        segs(b);
        split = p; p += sc;
        rank = p; p += sc + 1;
        sdim = p; p += sc;
        sval = reinterpret_cast<float *>(p); p += sc;
        seg_a = p; p += n;
        seg_b = p; p += n;
        flag = p; p += n;
        pre = p;
    }
};

// Block-wide exclusive scan of in[0..L) into out[0..L], out[L] = total, which
// is also returned to every thread.  s_w: 33 ints of shared memory.
template <int NT>
__device__ int cta_excl_scan(const int *in, int *out, int L, int *s_w) {
    constexpr int NWARP = NT / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int carry = 0;
    for (int base = 0; base < L; base += 4 * NT) {
        int v[4], loc[4], s = 0;
        const int i0 = base + 4 * threadIdx.x;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            v[j] = (i0 + j < L) ? in[i0 + j] : 0;
            loc[j] = s;
            s += v[j];
        }
        int x = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_w[warp] = x;
        __syncthreads();
        if (warp == 0) {
            int w = lane < NWARP ? s_w[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            if (lane < NWARP) s_w[lane] = w;
        }
        __syncthreads();
        const int off = carry + (warp ? s_w[warp - 1] : 0) + x - s;
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (i0 + j < L) out[i0 + j] = off + loc[j];
        carry += s_w[NWARP - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[L] = carry;
    __syncthreads();
    return carry;
}

// Build a kd-tree over bucket entries P[s0, s1) (already packed, any order)
// whose root sits at depth depth0 of an enclosing tree (the depth cap counts
// from the enclosing root).  When n_parent / leaf_parent are given, every new
// node and bucket entry records the code (2*parent node + side) of where it
// hangs; root_code is that code for the range's own root (-1: tree root).
// Q is a ping-pong buffer addressed by the same positions.  Nodes are written
// to node indices node_base .. node_base + (s1 - s0 - 2) (at most n-1 nodes).
// root_lo/root_hi: the range's tight box as order-preserving ints.
// root_slot >= 0: the root, if it splits, goes to that node slot instead.
// Returns the tree's root reference and node count (valid in thread 0 and,
// after the final barrier, in every thread).
template <int DC, int NT>
__device__ CtaTree cta_build_tree(float4 *P, float4 *Q, int s0, int s1, const int *root_lo, const int *root_hi,
                                  int *scratch, int leaf, int node_base, float4 *nodes, int *n_sdim,
                                  float *n_sval, int2 *n_range, int *s_w, int depth0 = 0,
                                  int *n_parent = nullptr, int *leaf_parent = nullptr, int root_code = -1,
                                  int root_slot = -1) {
    constexpr int W = bucket_w(DC);
    const int n = s1 - s0;
    CtaScratch<DC> sc;
    sc.carve(scratch, n, leaf);
    CtaSegs cur = sc.a, nxt = sc.b;
    int *seg_cur = sc.seg_a, *seg_nxt = sc.seg_b;
    const int lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        cur.start[0] = s0; cur.end[0] = s1; cur.parent[0] = -1; cur.side[0] = 0; cur.depth[0] = depth0;
    }
    if (threadIdx.x < DC) {
        cur.lo[threadIdx.x] = root_lo[threadIdx.x];
        cur.hi[threadIdx.x] = root_hi[threadIdx.x];
    }
    for (int i = threadIdx.x; i < n; i += NT) seg_cur[i] = 0;
    __syncthreads();
    float4 *cbuf = P, *obuf = Q;
    int S = 1, used = 0, level = 0;
    CtaTree res;
    res.root_ref = 0;
    res.root_cnt = n;
    // depth grows by one per level and nothing splits at the depth cap, so at
    // most PG_DEPTH_CAP + 1 levels run; the bound also holds on bad input
    for (int guard = 0; guard <= PG_DEPTH_CAP + 1; ++guard) {
        // classify
        for (int s = threadIdx.x; s < S; s += NT) {
            const int size = cur.end[s] - cur.start[s];
            int flag = 0, bd = 0;
            float bv = 0.f;
            if (size > leaf && cur.depth[s] < PG_DEPTH_CAP) {
                float best = 0.f;
#pragma unroll
                for (int c = 0; c < DC; ++c) {
                    const float e = __fsub_rn(o2f(cur.hi[s * DC + c]), o2f(cur.lo[s * DC + c]));
                    if (e > best) { best = e; bd = c; }
                }
                if (best > 0.f) {
                    const float l = o2f(cur.lo[s * DC + bd]), h = o2f(cur.hi[s * DC + bd]);
                    float mid = __fadd_rn(__fmul_rn(0.5f, l), __fmul_rn(0.5f, h));
                    if (!(mid > l)) mid = h;
                    if (mid > h) mid = h;
                    flag = 1;
                    bv = mid;
                }
            }
            sc.split[s] = flag;
            sc.sdim[s] = bd;
            sc.sval[s] = bv;
        }
        __syncthreads();
        const int T = cta_excl_scan<NT>(sc.split, sc.rank, S, s_w);
        // link
        for (int s = threadIdx.x; s < S; s += NT) {
            const int st = cur.start[s], size = cur.end[s] - st;
            const bool split = sc.split[s] != 0;
            const int node = (level == 0 && root_slot >= 0) ? root_slot : node_base + used + sc.rank[s];
            const int p = cur.parent[s];
            // where this segment hangs in the whole tree (parent node, side)
            const int code = p >= 0 ? 2 * p + cur.side[s] : root_code;
            if (split) {
                if (n_parent) n_parent[node] = code;
            } else if (leaf_parent) {
                for (int i = st; i < st + size; ++i) leaf_parent[i] = code;
            }
            if (p >= 0) {
                float *rec = reinterpret_cast<float *>(nodes + (size_t)p * node_w(DC));
                const int c = cur.side[s];
#pragma unroll
                for (int d = 0; d < DC; ++d) {
                    rec[c * 2 * DC + d] = o2f(cur.lo[s * DC + d]);
                    rec[c * 2 * DC + DC + d] = o2f(cur.hi[s * DC + d]);
                }
                int *ri = reinterpret_cast<int *>(rec + 4 * DC);
                ri[2 * c] = split ? node : st;
                ri[2 * c + 1] = split ? 0 : size;
            } else if (split) {
                res.root_ref = node;
                res.root_cnt = 0;
            } else {
                res.root_ref = st;
                res.root_cnt = size;
            }
            if (split) {
                n_sdim[node] = sc.sdim[s];
                n_sval[node] = sc.sval[s];
                n_range[node] = make_int2(st, st + size);
                const int r = sc.rank[s];
#pragma unroll
                for (int ch = 0; ch < 2; ++ch) {
                    const int x = 2 * r + ch;
                    nxt.parent[x] = node;
                    nxt.side[x] = ch;
                    nxt.depth[x] = cur.depth[s] + 1;
#pragma unroll
                    for (int d = 0; d < DC; ++d) {
                        nxt.lo[x * DC + d] = 0x7f800000;
                        nxt.hi[x * DC + d] = (int)0x807fffffu;
                    }
                }
            }
        }
        __syncthreads();
        if (T == 0) break;
        // flags
        const float *cf = reinterpret_cast<const float *>(cbuf);
        for (int i = threadIdx.x; i < n; i += NT) {
            const int s = seg_cur[i];
            int f = 0;
            if (s >= 0 && sc.split[s]) f = cf[(size_t)(s0 + i) * 4 * W + sc.sdim[s]] < sc.sval[s];
            sc.flag[i] = f;
        }
        __syncthreads();
        cta_excl_scan<NT>(sc.flag, sc.pre, n, s_w);
        // stable scatter + child boxes
        for (int base = 0; base < n; base += NT) {
            const int i = base + threadIdx.x;
            const bool valid = i < n;
            int child = -1;
            float4 v[W];
#pragma unroll
            for (int w = 0; w < W; ++w) v[w] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (valid) {
                const int g = s0 + i;
#pragma unroll
                for (int w = 0; w < W; ++w) v[w] = cbuf[(size_t)g * W + w];
                const int s = seg_cur[i];
                int dst = g;
                if (s >= 0 && sc.split[s]) {
                    const int st = cur.start[s], en = cur.end[s];
                    const int b0 = sc.pre[st - s0];
                    const int nl = sc.pre[en - s0] - b0;
                    const int r = sc.pre[i] - b0;
                    const int f = sc.flag[i];
                    const int rk = sc.rank[s];
                    if (f) { dst = st + r; child = 2 * rk; }
                    else { dst = st + nl + (g - st) - r; child = 2 * rk + 1; }
                    if (g == st) {
                        nxt.start[2 * rk] = st;
                        nxt.end[2 * rk] = st + nl;
                        nxt.start[2 * rk + 1] = st + nl;
                        nxt.end[2 * rk + 1] = en;
                    }
#pragma unroll
                    for (int w = 0; w < W; ++w) obuf[(size_t)dst * W + w] = v[w];
                    seg_nxt[dst - s0] = child;
                } else {
                    if (s >= 0 && cbuf != P) {
#pragma unroll
                        for (int w = 0; w < W; ++w) P[(size_t)g * W + w] = v[w];
                    }
                    seg_nxt[i] = -1;
                }
            }
            const float *vf = reinterpret_cast<const float *>(v);
            unsigned active = __ballot_sync(0xffffffffu, child >= 0);
            while (active) {
                const int leader = __ffs(active) - 1;
                const int key = __shfl_sync(0xffffffffu, child, leader);
                const bool mine = child == key;
                const unsigned grp = __ballot_sync(0xffffffffu, mine);
#pragma unroll
                for (int d = 0; d < DC; ++d) {
                    const int e = f2o(vf[d]);
                    const int a = __reduce_min_sync(0xffffffffu, mine ? e : INT_MAX);
                    const int b = __reduce_max_sync(0xffffffffu, mine ? e : INT_MIN);
                    if (lane == leader) {
                        atomicMin(&nxt.lo[key * DC + d], a);
                        atomicMax(&nxt.hi[key * DC + d], b);
                    }
                }
                active &= ~grp;
            }
        }
        __syncthreads();
        CtaSegs t = cur; cur = nxt; nxt = t;
        int *ts = seg_cur; seg_cur = seg_nxt; seg_nxt = ts;
        float4 *tb = cbuf; cbuf = obuf; obuf = tb;
        used += T;
        S = 2 * T;
        ++level;
    }
    // leaves of the last level still sit in the current buffer
    if (cbuf != P) {
        for (int i = threadIdx.x; i < n; i += NT) {
            if (seg_cur[i] >= 0) {
#pragma unroll
                for (int w = 0; w < W; ++w) P[(size_t)(s0 + i) * W + w] = cbuf[(size_t)(s0 + i) * W + w];
            }
        }
    }
    __syncthreads();
    res.nodes = used;
    res.depth = depth0 + level;
    return res;
}

}  // namespace pg
