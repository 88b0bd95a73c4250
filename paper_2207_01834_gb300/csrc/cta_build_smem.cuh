// kd-tree construction of a few thousand points by ONE thread block, held
// entirely in shared memory (paper Section 5 intro, spatial-median split of
// Section 6, recursive construction of Appendix A.1.1 done level by level).
//
// The points are loaded once; each level then partitions a 16-bit permutation
// of them, so a level touches shared memory only:
//   classify   one thread per segment: spatial-median split or leaf,
//   flags      one ballot word per 32 positions (point goes left),
//   scan       popcount prefix of the ballot words (and of the split flags,
//              which numbers the next level's segments),
//   link       one thread per segment: record the node, hang the segment in
//              its parent's record, set up the two children,
//   scatter    partition of the permutation (left points in order at the
//              front, right points from the back), children's tight boxes
//              by warp-aggregated shared-memory min/max.
// An internal node splitting [st, en) at m is stored in node slot
// node_base + (m - 1): the gaps between consecutive positions name the
// internal nodes uniquely, so the numbering is fixed by the tree alone and a
// range of n points needs at most n - 1 slots.  Splits and boxes are those
// of the level-synchronous builders (only the order of the points inside a
// leaf may differ, which no answer depends on).
#pragma once

#include <climits>

#include "common.cuh"

namespace pg {

__host__ __device__ inline int smem_seg_cap(int ns, int leaf) { return 2 * (ns / (leaf + 1)) + 2; }

__host__ __device__ inline size_t smem_al16(size_t x) { return (x + 15) & ~(size_t)15; }

// Shared-memory bytes for up to ns points and sc segments per level.
__host__ __device__ inline size_t smem_build_bytes(int ns, int sc, int dc) {
    const size_t nw = (size_t)ns / 32 + 1, sw = (size_t)sc / 32 + 1;
    size_t b = 0;
    b += smem_al16(sizeof(float4) * (size_t)ns * bucket_w(dc));   // points
    b += smem_al16(sizeof(uint16_t) * 4 * (size_t)ns);            // permutation, segment of each position (x2)
    b += smem_al16(sizeof(uint32_t) * nw);                        // flag ballots
    b += smem_al16(sizeof(int) * (nw + 1));                       // their prefix
    b += smem_al16(sizeof(uint16_t) * 4 * (size_t)sc);            // segment start, end (x2)
    b += smem_al16(sizeof(int) * 4 * (size_t)sc);                 // parent code, depth (x2)
    b += smem_al16(sizeof(int) * 2 * (size_t)sc * dc);            // tight boxes
    b += smem_al16(sizeof(int) * 2 * (size_t)sc);                 // split dimension, split value
    b += smem_al16(sizeof(int) * 2 * (size_t)sc);                 // left-count base, split rank
    b += smem_al16(sizeof(uint32_t) * sw);                        // split ballots
    b += smem_al16(sizeof(int) * (sw + 1));                       // their prefix
    return b;
}

// Largest point count (a multiple of 32) whose layout fits in `budget` bytes.
inline int smem_build_points(int dc, int leaf, size_t budget) {
    int lo = 0, hi = 65504 / 32;
    while (lo < hi) {
        const int mid = (lo + hi + 1) / 2;
        const int ns = mid * 32;
        if (smem_build_bytes(ns, smem_seg_cap(ns, leaf), dc) <= budget) lo = mid;
        else hi = mid - 1;
    }
    return lo * 32;
}

template <int DC>
struct SmemBuild {
    float4 *pts;
    uint16_t *perm, *seg;      // two buffers of ns each (current, next)
    uint32_t *word;
    int *wpre;
    uint16_t *st, *en;         // two tables of sc each
    int *code, *depth;
    int *lo, *hi;
    int *sdim;
    float *sval;
    int *sb0, *srk;            // per split segment: flags before its start, its rank
    uint32_t *sword;
    int *spre;
    __device__ void carve(unsigned char *base, int ns, int sc) {
        const size_t nw = (size_t)ns / 32 + 1, sw = (size_t)sc / 32 + 1;
        unsigned char *p = base;
        auto take = [&](size_t bytes) { unsigned char *q = p; p += smem_al16(bytes); return q; };
        pts = reinterpret_cast<float4 *>(take(sizeof(float4) * (size_t)ns * bucket_w(DC)));
        uint16_t *u = reinterpret_cast<uint16_t *>(take(sizeof(uint16_t) * 4 * (size_t)ns));
        perm = u; seg = u + 2 * ns;
        word = reinterpret_cast<uint32_t *>(take(sizeof(uint32_t) * nw));
        wpre = reinterpret_cast<int *>(take(sizeof(int) * (nw + 1)));
        u = reinterpret_cast<uint16_t *>(take(sizeof(uint16_t) * 4 * (size_t)sc));
        st = u; en = u + 2 * sc;
        int *q = reinterpret_cast<int *>(take(sizeof(int) * 4 * (size_t)sc));
        code = q; depth = q + 2 * sc;
        q = reinterpret_cast<int *>(take(sizeof(int) * 2 * (size_t)sc * DC));
        lo = q; hi = q + (size_t)sc * DC;
        q = reinterpret_cast<int *>(take(sizeof(int) * 2 * (size_t)sc));
        sdim = q; sval = reinterpret_cast<float *>(q + sc);
        q = reinterpret_cast<int *>(take(sizeof(int) * 2 * (size_t)sc));
        sb0 = q; srk = q + sc;
        sword = reinterpret_cast<uint32_t *>(take(sizeof(uint32_t) * sw));
        spre = reinterpret_cast<int *>(take(sizeof(int) * (sw + 1)));
    }
};

// Number of set ballot bits before bit x (x may equal the count of bits).
__device__ __forceinline__ int ballot_prefix(const uint32_t *w, const int *pre, int x) {
    return pre[x >> 5] + __popc(w[x >> 5] & ((1u << (x & 31)) - 1u));
}

// Exclusive prefix of the popcounts of w[0..count) into pre[0..count],
// pre[count] = total; run by one whole warp.
__device__ __forceinline__ void warp_popc_scan(const uint32_t *w, int *pre, int count) {
    const int lane = threadIdx.x & 31;
    int carry = 0;
    for (int b = 0; b < count; b += 32) {
        const int i = b + lane;
        const int v = i < count ? __popc(w[i]) : 0;
        int x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (i < count) pre[i] = carry + x - v;
        carry += __shfl_sync(0xffffffffu, x, 31);
    }
    if (lane == 0) pre[count] = carry;
}

// Build the tree of bucket entries P[s0, s1) (packed, any order; at most ns
// of them) in place.  Arguments as for cta_build_tree; smem holds
// smem_build_bytes(ns, sc, DC) bytes with sc = smem_seg_cap(ns, leaf).
// root_slot >= 0: the root, if it splits, goes to that node slot (outside
// node_base .. node_base + n - 2) instead of its split position.
template <int DC, int NT>
__device__ CtaTree cta_build_smem(float4 *P, int s0, int s1, const int *root_lo, const int *root_hi,
                                  unsigned char *smem, int ns, int sc, int leaf, int node_base, float4 *nodes,
                                  int *n_sdim, float *n_sval, int2 *n_range, int depth0 = 0,
                                  int *n_parent = nullptr, int *leaf_parent = nullptr, int root_code = -1,
                                  int root_slot = -1) {
    constexpr int W = bucket_w(DC);
    constexpr int NW = node_w(DC);
    constexpr uint16_t NONE = 0xffff;
    __shared__ int s_root[2];
    const int n = s1 - s0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    SmemBuild<DC> m;
    m.carve(smem, ns, sc);
    for (int i = threadIdx.x; i < n; i += NT) {
#pragma unroll
        for (int w = 0; w < W; ++w) m.pts[(size_t)i * W + w] = P[(size_t)(s0 + i) * W + w];
        m.perm[i] = (uint16_t)i;
        m.seg[i] = 0;
    }
    if (threadIdx.x == 0) {
        m.st[0] = 0; m.en[0] = (uint16_t)n; m.code[0] = root_code; m.depth[0] = depth0;
    }
    if (threadIdx.x < DC) {
        m.lo[threadIdx.x] = root_lo[threadIdx.x];
        m.hi[threadIdx.x] = root_hi[threadIdx.x];
    }
    __syncthreads();
    const float *pf = reinterpret_cast<const float *>(m.pts);
    const int nwords = (n >> 5) + 1;
    int S = 1, cur = 0, level = 0;
    // depth grows by one per level and nothing splits at the depth cap, so at
    // most PG_DEPTH_CAP + 1 levels run; the bound also holds on bad input
    for (int guard = 0; guard <= PG_DEPTH_CAP + 1; ++guard) {
        const int nxt = cur ^ 1;
        const int swords = (S >> 5) + 1;
        // this level's (c_) and the next level's (n_) buffers
        const uint16_t *c_perm = m.perm + cur * ns, *c_seg = m.seg + cur * ns;
        uint16_t *n_perm = m.perm + nxt * ns, *n_seg = m.seg + nxt * ns;
        const uint16_t *c_st = m.st + cur * sc, *c_en = m.en + cur * sc;
        uint16_t *n_st = m.st + nxt * sc, *n_en = m.en + nxt * sc;
        const int *c_code = m.code + cur * sc, *c_depth = m.depth + cur * sc;
        int *n_code = m.code + nxt * sc, *n_depth = m.depth + nxt * sc;
        // classify
        for (int b = 0; b < swords * 32; b += NT) {
            const int s = b + threadIdx.x;
            int flag = 0, bd = 0;
            float bv = 0.f;
            if (s < S) {
                const int size = c_en[s] - c_st[s];
                if (size > leaf && c_depth[s] < PG_DEPTH_CAP) {
                    float best = 0.f;
#pragma unroll
                    for (int c = 0; c < DC; ++c) {
                        const float e = __fsub_rn(o2f(m.hi[s * DC + c]), o2f(m.lo[s * DC + c]));
                        if (e > best) { best = e; bd = c; }
                    }
                    if (best > 0.f) {
                        const float l = o2f(m.lo[s * DC + bd]), h = o2f(m.hi[s * DC + bd]);
                        float mid = __fadd_rn(__fmul_rn(0.5f, l), __fmul_rn(0.5f, h));
                        if (!(mid > l)) mid = h;
                        if (mid > h) mid = h;
                        flag = 1;
                        bv = mid;
                    }
                }
                m.sdim[s] = bd;
                m.sval[s] = bv;
            }
            const unsigned bal = __ballot_sync(0xffffffffu, flag);
            if (lane == 0 && (s >> 5) < swords) m.sword[s >> 5] = bal;
        }
        __syncthreads();
        // flags: the point at position i goes left
        for (int b = 0; b < nwords * 32; b += NT) {
            const int i = b + threadIdx.x;
            int f = 0;
            if (i < n) {
                const int s = c_seg[i];
                if (s != NONE && ((m.sword[s >> 5] >> (s & 31)) & 1u))
                    f = pf[(size_t)c_perm[i] * 4 * W + m.sdim[s]] < m.sval[s];
            }
            const unsigned bal = __ballot_sync(0xffffffffu, f);
            if (lane == 0 && (i >> 5) < nwords) m.word[i >> 5] = bal;
        }
        __syncthreads();
        if (warp == 0) warp_popc_scan(m.word, m.wpre, nwords);
        else if (warp == 1) warp_popc_scan(m.sword, m.spre, swords);
        __syncthreads();
        const int T = m.spre[swords];
        // link
        for (int s = threadIdx.x; s < S; s += NT) {
            const int st = c_st[s], en = c_en[s], size = en - st;
            const bool split = (m.sword[s >> 5] >> (s & 31)) & 1u;
            const int code = c_code[s];
            int node = -1, nl = 0;
            int b0 = 0;
            if (split) {
                b0 = ballot_prefix(m.word, m.wpre, st);
                nl = ballot_prefix(m.word, m.wpre, en) - b0;
                node = (level == 0 && root_slot >= 0) ? root_slot : node_base + st + nl - 1;
            }
            if (level == 0) {
                s_root[0] = split ? node : s0 + st;
                s_root[1] = split ? 0 : size;
            } else {
                float *rec = reinterpret_cast<float *>(nodes + (size_t)(code >> 1) * NW);
                const int c = code & 1;
#pragma unroll
                for (int d = 0; d < DC; ++d) {
                    rec[c * 2 * DC + d] = o2f(m.lo[s * DC + d]);
                    rec[c * 2 * DC + DC + d] = o2f(m.hi[s * DC + d]);
                }
                int *ri = reinterpret_cast<int *>(rec + 4 * DC);
                ri[2 * c] = split ? node : s0 + st;
                ri[2 * c + 1] = split ? 0 : size;
            }
            if (split) {
                n_sdim[node] = m.sdim[s];
                n_sval[node] = m.sval[s];
                n_range[node] = make_int2(s0 + st, s0 + en);
                if (n_parent) n_parent[node] = code;
                const int r = ballot_prefix(m.sword, m.spre, s);
                m.sb0[s] = b0;
                m.srk[s] = r;
#pragma unroll
                for (int ch = 0; ch < 2; ++ch) {
                    const int x = 2 * r + ch;
                    n_st[x] = (uint16_t)(ch ? st + nl : st);
                    n_en[x] = (uint16_t)(ch ? en : st + nl);
                    n_code[x] = 2 * node + ch;
                    n_depth[x] = c_depth[s] + 1;
                }
            } else if (leaf_parent) {
                for (int i = st; i < en; ++i) leaf_parent[s0 + i] = code;
            }
        }
        __syncthreads();
        if (T == 0) break;
        for (int x = threadIdx.x; x < 2 * T * DC; x += NT) {
            m.lo[x] = 0x7f800000;
            m.hi[x] = (int)0x807fffffu;
        }
        __syncthreads();
        // stable scatter of the permutation + children's tight boxes
        for (int b = 0; b < n; b += NT) {
            const int i = b + threadIdx.x;
            int child = -1, pidx = 0;
            if (i < n) {
                pidx = c_perm[i];
                const int s = c_seg[i];
                int dst = i;
                if (s != NONE && ((m.sword[s >> 5] >> (s & 31)) & 1u)) {
                    // left points keep their order at the front, right points
                    // fill the segment from the back (no segment total needed)
                    const int st = c_st[s], en = c_en[s];
                    const int r = ballot_prefix(m.word, m.wpre, i) - m.sb0[s];
                    const int rk = m.srk[s];
                    if ((m.word[i >> 5] >> (i & 31)) & 1u) { dst = st + r; child = 2 * rk; }
                    else { dst = en - 1 - ((i - st) - r); child = 2 * rk + 1; }
                }
                n_perm[dst] = (uint16_t)pidx;
                n_seg[dst] = child >= 0 ? (uint16_t)child : NONE;
            }
            unsigned active = __ballot_sync(0xffffffffu, child >= 0);
            while (active) {
                const int leader = __ffs(active) - 1;
                const int key = __shfl_sync(0xffffffffu, child, leader);
                const bool mine = child == key;
                const unsigned grp = __ballot_sync(0xffffffffu, mine);
#pragma unroll
                for (int d = 0; d < DC; ++d) {
                    const int e = mine ? f2o(pf[(size_t)pidx * 4 * W + d]) : 0;
                    const int a = __reduce_min_sync(0xffffffffu, mine ? e : INT_MAX);
                    const int c = __reduce_max_sync(0xffffffffu, mine ? e : INT_MIN);
                    if (lane == leader) {
                        atomicMin(&m.lo[key * DC + d], a);
                        atomicMax(&m.hi[key * DC + d], c);
                    }
                }
                active &= ~grp;
            }
        }
        __syncthreads();
        cur = nxt;
        S = 2 * T;
        ++level;
    }
    for (int i = threadIdx.x; i < n; i += NT) {
        const int p = m.perm[cur * ns + i];
#pragma unroll
        for (int w = 0; w < W; ++w) P[(size_t)(s0 + i) * W + w] = m.pts[(size_t)p * W + w];
    }
    CtaTree res;
    res.root_ref = s_root[0];
    res.root_cnt = s_root[1];
    res.nodes = 0;
    res.depth = depth0 + level;
    __syncthreads();
    return res;
}

}  // namespace pg
