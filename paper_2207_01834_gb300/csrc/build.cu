// kd-tree construction on the GPU (paper Section 5 intro and Appendix A.1.1;
// spatial-median split of Section 6 "Construction").
//
// Level-synchronous top-down build.  At every level each active segment (a
// contiguous range of the point array holding one node's points) is
// classified as a leaf or split at the midpoint of its tight bounding box in
// its widest dimension.  All points of split segments are then partitioned:
// a segmented scan of the "goes left" flags (restarting at every segment
// start) gives each point its rank among the left-going points of its
// segment; left points keep their order at the front of the segment, right
// points fill it from the back.  The same pass reduces the two children's
// tight boxes (per tile in shared memory, then integer atomics on an
// order-preserving float encoding).  The node that a segment becomes is
// numbered by a scan over the level's split flags, so the layout is
// deterministic.  Segments small enough for one block's shared memory are
// finished there (cta_build_smem.cuh).
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>

#include "cta_build_smem.cuh"
#include "internal.h"
#include "sort.h"

namespace pg {

namespace {

constexpr int BT = 256;

struct Segs {
    int *start, *end, *parent, *side, *depth, *lo, *hi;
};

__device__ __forceinline__ float *rec_of(float4 *nodes, int node, int dc) {
    return reinterpret_cast<float *>(nodes + (size_t)node * node_w(dc));
}

__global__ void k_init_box(int *lo, int *hi, int count) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) {
        lo[i] = 0x7f800000;                 // f2o(+inf)
        hi[i] = (int)0x807fffffu;           // f2o(-inf)
    }
}

// Pack rows into bucket entries (coordinates zero padded to DC, id at word
// DC) and reduce the root box.
template <int DC>
__global__ void __launch_bounds__(BT) k_pack(const float *__restrict__ src, const int32_t *__restrict__ rows,
                                             const int32_t *__restrict__ ids, int64_t n, int dim,
                                             float4 *__restrict__ out, int *__restrict__ box_lo,
                                             int *__restrict__ box_hi) {
    constexpr int W = bucket_w(DC);
    float lo[DC], hi[DC];
#pragma unroll
    for (int c = 0; c < DC; ++c) { lo[c] = __int_as_float(0x7f800000); hi[c] = -lo[c]; }
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = rows ? (int64_t)rows[i] : i;
        float v[4 * W];
#pragma unroll
        for (int c = 0; c < 4 * W; ++c) v[c] = 0.f;
#pragma unroll
        for (int c = 0; c < DC; ++c)
            if (c < dim) v[c] = src[row * dim + c];
        v[DC] = __int_as_float(ids ? ids[i] : (int)i);
#pragma unroll
        for (int w = 0; w < W; ++w) out[i * W + w] = make_float4(v[4 * w], v[4 * w + 1], v[4 * w + 2], v[4 * w + 3]);
#pragma unroll
        for (int c = 0; c < DC; ++c) { lo[c] = fminf(lo[c], v[c]); hi[c] = fmaxf(hi[c], v[c]); }
    }
    __shared__ int s_lo[BT / 32][DC], s_hi[BT / 32][DC];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < DC; ++c) {
        int a = __reduce_min_sync(0xffffffffu, f2o(lo[c]));
        int b = __reduce_max_sync(0xffffffffu, f2o(hi[c]));
        if (lane == 0) { s_lo[warp][c] = a; s_hi[warp][c] = b; }
    }
    __syncthreads();
    if (threadIdx.x < DC) {
        int a = INT_MAX, b = INT_MIN;
        for (int w = 0; w < BT / 32; ++w) { a = min(a, s_lo[w][threadIdx.x]); b = max(b, s_hi[w][threadIdx.x]); }
        atomicMin(&box_lo[threadIdx.x], a);
        atomicMax(&box_hi[threadIdx.x], b);
    }
}

// Device-side control block of the level loop: the host enqueues levels with
// launch sizes from upper bounds and never waits on a count; kernels read the
// live values here and do nothing once the loop is done.
// Control block of a level loop: live segments, level nodes so far, finisher
// segments so far, done flag, levels that moved points, level count at the
// end, whether the root split, the next level's index (for a loop driven by
// the device), the finisher's next work item.
enum { CTL_S = 0, CTL_NB, CTL_FIN, CTL_DONE, CTL_SCATTERS, CTL_LEVELS, CTL_ROOT_SPLIT, CTL_CUR, CTL_FIN_NEXT, CTL_WORDS };

// Level partition in two passes over tiles of PT_ROWS x PT_THREADS points
// (position base + row * PT_THREADS + thread):
//   k_part_tiles  per tile, the number of "goes left" flags after the last
//                 segment start in the tile (or all of them, with no start),
//   k_part_carry  segmented exclusive scan of those over the tiles,
//   k_part        per point, the number r of left-going points before it in
//                 its segment; left points go to st + r in order, right
//                 points fill the segment from the end (en - 1 - (i - st - r)),
//                 so no segment total is needed before the move; the last
//                 point of a segment writes the two children's ranges.
// A segment start is a position whose segment differs from the previous one.
constexpr int PT_THREADS = 256, PT_ROWS = 8, PT_TILE = PT_THREADS * PT_ROWS, PT_WARPS = PT_THREADS / 32;
constexpr int kBoxSlots = 16;   // children whose boxes a tile reduces in shared memory

// Segmented count: `has` a segment start, `cnt` flags after the last start.
__device__ __forceinline__ unsigned seg_pack(bool has, int cnt) { return (has ? 0x80000000u : 0u) | (unsigned)cnt; }
__device__ __forceinline__ unsigned seg_combine(unsigned a, unsigned b) {   // a before b
    return (b & 0x80000000u) ? (a & 0x80000000u) | b : (a & 0x80000000u) + ((a & 0x7fffffffu) + b);
}

// Flags and segment starts of one tile; every warp-row's segmented count
// goes to rowsum[row * PT_WARPS + warp].
// PRE: the "goes left" flag of each position is given in pflag (object-median
// levels) instead of computed from the split value.
template <int DC, bool PRE = false>
__device__ __forceinline__ void tile_flags(int n, int base, const float *pf, const int *seg_of,
                                           const int *split_flag, const int *sdim, const float *sval,
                                           unsigned *fword, unsigned *rword, unsigned *rowsum,
                                           const int *pflag = nullptr) {
    constexpr int W = bucket_w(DC);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < PT_ROWS; ++j) {
        const int i = base + j * PT_THREADS + threadIdx.x;
        const bool valid = i < n;
        const int s = valid ? seg_of[i] : -1;
        int sp = __shfl_up_sync(0xffffffffu, s, 1);   // position i - 1 (same warp row)
        if (lane == 0) sp = (valid && i > 0) ? seg_of[i - 1] : -2;
        const bool start = valid && s != sp;
        int f = 0;
        if (valid && s >= 0 && split_flag[s]) f = PRE ? pflag[i] : pf[(size_t)i * 4 * W + sdim[s]] < sval[s];
        const unsigned F = __ballot_sync(0xffffffffu, f), R = __ballot_sync(0xffffffffu, start);
        if (lane == 0) {
            const unsigned keep = R ? ~((1u << (31 - __clz(R))) - 1u) : 0xffffffffu;
            rowsum[j * PT_WARPS + warp] = seg_pack(R != 0, __popc(F & keep));
            fword[j * PT_WARPS + warp] = F;
            rword[j * PT_WARPS + warp] = R;
        }
    }
}

// Per tile: the segmented count (tsum), and for each of its PT_ROWS *
// PT_WARPS warp-rows the flag ballot, the segment-start ballot and the
// segmented exclusive prefix inside the tile (twords, 3 words per warp-row),
// so that the move pass needs no flag of its own.
constexpr int PT_WR = PT_ROWS * PT_WARPS;   // warp-rows per tile
constexpr int PT_TW = 3 * PT_WR;            // stored words per tile

template <int DC, bool PRE = false>
__global__ void __launch_bounds__(PT_THREADS) k_part_tiles(int64_t n, const float4 *__restrict__ P,
                                                           const int *__restrict__ seg_of,
                                                           const int *__restrict__ split_flag,
                                                           const int *__restrict__ sdim,
                                                           const float *__restrict__ sval,
                                                           const int *__restrict__ T, unsigned *__restrict__ tsum,
                                                           unsigned *__restrict__ twords,
                                                           const int *__restrict__ pflag = nullptr) {
    pdl_wait();
    pdl_trigger();
    if (*T == 0) return;
    __shared__ unsigned rowsum[PT_WR], fword[PT_WR], rword[PT_WR];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    tile_flags<DC, PRE>((int)n, blockIdx.x * PT_TILE, reinterpret_cast<const float *>(P), seg_of, split_flag, sdim,
                        sval, fword, rword, rowsum, pflag);
    __syncthreads();
    unsigned *tw = twords + (size_t)blockIdx.x * PT_TW;
    if (warp == 0) {
        constexpr int PER = PT_WR / 32;
        unsigned loc = 0;
#pragma unroll
        for (int k = 0; k < PER; ++k) loc = seg_combine(loc, rowsum[lane * PER + k]);
        unsigned x = loc;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x = seg_combine(y, x);
        }
        unsigned in = __shfl_up_sync(0xffffffffu, x, 1);
        if (lane == 0) in = 0u;
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int e = lane * PER + k;
            tw[2 * PT_WR + e] = in;
            in = seg_combine(in, rowsum[e]);
        }
        if (lane == 31) tsum[blockIdx.x] = in;
    } else if (warp == 1) {
        for (int e = lane; e < PT_WR; e += 32) {
            tw[e] = fword[e];
            tw[PT_WR + e] = rword[e];
        }
    }
}

// Segmented exclusive scan over the tiles (one block).
__global__ void __launch_bounds__(1024) k_part_carry(unsigned *__restrict__ tsum, int ntiles, const int *__restrict__ T,
                                                     int *__restrict__ ctl, const int *__restrict__ fin_total, int level) {
    pdl_wait();
    pdl_trigger();
    // end of the level: advance the control block (nothing after this kernel
    // in the level reads it); level < 0: the index is kept in the block
    if (threadIdx.x == 0 && !ctl[CTL_DONE]) {
        if (level < 0) level = ctl[CTL_CUR]++;
        const int t = *T;
        ctl[CTL_NB] += t;
        ctl[CTL_FIN] += *fin_total;
        ctl[CTL_S] = 2 * t;
        if (level == 0) ctl[CTL_ROOT_SPLIT] = t > 0;
        if (t > 0) ctl[CTL_SCATTERS] += 1;
        else { ctl[CTL_DONE] = 1; ctl[CTL_LEVELS] = level; }
    }
    if (*T == 0) return;
    __shared__ unsigned wtot[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned carry = 0;
    for (int b0 = 0; b0 < ntiles; b0 += 1024) {
        const int t = b0 + threadIdx.x;
        const unsigned v = t < ntiles ? tsum[t] : 0u;
        unsigned x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x = seg_combine(y, x);
        }
        if (lane == 31) wtot[warp] = x;
        __syncthreads();
        if (warp == 0) {
            unsigned w = wtot[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w = seg_combine(y, w);
            }
            wtot[lane] = w;
        }
        __syncthreads();
        // exclusive: everything before this tile
        unsigned ex = __shfl_up_sync(0xffffffffu, x, 1);
        if (lane == 0) ex = 0u;
        if (warp > 0) ex = seg_combine(wtot[warp - 1], ex);
        ex = seg_combine(carry, ex);
        if (t < ntiles) tsum[t] = ex;
        carry = seg_combine(carry, wtot[31]);
        __syncthreads();
    }
}

// Decide, per segment, leaf or split; for a split pick the widest dimension
// of the tight box (lowest index on ties) and its midpoint.
template <int DC>
__device__ __forceinline__ void classify_seg(int s, bool live, const int *__restrict__ start,
                                             const int *__restrict__ end, const int *__restrict__ depth,
                                             const int *__restrict__ lo, const int *__restrict__ hi, int leaf,
                                             int depth_cap, int fin_threshold, int *__restrict__ split_flag,
                                             int *__restrict__ fin_flag, int *__restrict__ sdim,
                                             float *__restrict__ sval) {
    if (!live) {   // padding up to the launch bound (or loop over)
        split_flag[s] = 0;
        fin_flag[s] = 0;
        return;
    }
    const int size = end[s] - start[s];
    int flag = 0, bd = 0;
    float bv = 0.f;
    if (size > leaf && depth[s] < depth_cap) {
        float best = 0.f;
#pragma unroll
        for (int c = 0; c < DC; ++c) {
            float e = __fsub_rn(o2f(hi[s * DC + c]), o2f(lo[s * DC + c]));
            if (e > best) { best = e; bd = c; }
        }
        if (best > 0.f) {
            const float l = o2f(lo[s * DC + bd]), h = o2f(hi[s * DC + bd]);
            float mid = __fadd_rn(__fmul_rn(0.5f, l), __fmul_rn(0.5f, h));
            if (!(mid > l)) mid = h;
            if (mid > h) mid = h;
            flag = 1;
            bv = mid;
        }
    }
    // a segment small enough for one block is finished by the block-scope builder
    const int fin = flag && size <= fin_threshold;
    split_flag[s] = flag && !fin;
    fin_flag[s] = fin;
    sdim[s] = bd;
    sval[s] = bv;
}

template <int DC>
__global__ void k_classify(int S_max, const int *__restrict__ ctl, const int *__restrict__ start, const int *__restrict__ end,
                           const int *__restrict__ depth, const int *__restrict__ lo,
                           const int *__restrict__ hi, int leaf, int depth_cap, int fin_threshold,
                           int *__restrict__ split_flag, int *__restrict__ fin_flag, int *__restrict__ sdim,
                           float *__restrict__ sval) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S_max) return;
    classify_seg<DC>(s, !ctl[CTL_DONE] && s < ctl[CTL_S], start, end, depth, lo, hi, leaf, depth_cap,
                     fin_threshold, split_flag, fin_flag, sdim, sval);
}

// Write each segment into its parent's child slot (tight box + reference),
// record split nodes and prepare the next level's child segments.
template <int DC>
__device__ __forceinline__ void link_seg(int s, const int *__restrict__ ctl, const int *__restrict__ start, const int *__restrict__ end,
                       const int *__restrict__ parent, const int *__restrict__ side,
                       const int *__restrict__ depth, const int *__restrict__ lo, const int *__restrict__ hi,
                       const int *__restrict__ split_flag, const int *__restrict__ split_rank,
                       const int *__restrict__ sdim, const float *__restrict__ sval,
                       float4 *__restrict__ nodes, int *__restrict__ n_sdim, float *__restrict__ n_sval,
                       int2 *__restrict__ n_range, int *__restrict__ nx_parent, int *__restrict__ nx_side,
                       int *__restrict__ nx_depth, int *__restrict__ nx_lo, int *__restrict__ nx_hi,
                       const int *__restrict__ fin_flag, const int *__restrict__ fin_rank, Segs fin,
                       int *__restrict__ n_parent, int *__restrict__ roots, int fin_link) {
    const int node_base = ctl[CTL_NB], fin_base = ctl[CTL_FIN];
    const int st = start[s], size = end[s] - st;
    const int p = parent[s];
    const bool split = split_flag[s] != 0;
    const int node = node_base + split_rank[s];
    if (fin_flag[s]) {
        // handed to the block-scope builder, which links the subtree root
        const int f = fin_base + fin_rank[s];
        fin.start[f] = st;
        fin.end[f] = st + size;
        fin.parent[f] = p;
        fin.side[f] = side[s];
        fin.depth[f] = depth[s];
#pragma unroll
        for (int d = 0; d < DC; ++d) {
            fin.lo[f * DC + d] = lo[s * DC + d];
            fin.hi[f * DC + d] = hi[s * DC + d];
        }
        if (p >= 0) {
            float *rec = rec_of(nodes, p, DC);
            const int c = side[s];
#pragma unroll
            for (int d = 0; d < DC; ++d) {
                rec[c * 2 * DC + d] = o2f(lo[s * DC + d]);
                rec[c * 2 * DC + DC + d] = o2f(hi[s * DC + d]);
            }
            if (fin_link) {   // forest: the finisher puts the subtree root in slot en - 1
                int *ri = reinterpret_cast<int *>(rec + 4 * DC);
                ri[2 * c] = st + size - 1;
                ri[2 * c + 1] = 0;
            }
        } else if (p < -1) {
            roots[2 * (-p - 2)] = st + size - 1;
            roots[2 * (-p - 2) + 1] = 0;
        }
        return;
    }
    const int code = p >= 0 ? 2 * p + side[s] : -1;   // where this segment hangs
    if (split) n_parent[node] = code;
    if (p < -1) {   // root of tree -p-2 of a forest
        roots[2 * (-p - 2)] = split ? node : st;
        roots[2 * (-p - 2) + 1] = split ? 0 : size;
    }
    if (p >= 0) {
        float *rec = rec_of(nodes, p, DC);
        const int c = side[s];
#pragma unroll
        for (int d = 0; d < DC; ++d) {
            rec[c * 2 * DC + d] = o2f(lo[s * DC + d]);
            rec[c * 2 * DC + DC + d] = o2f(hi[s * DC + d]);
        }
        int *ri = reinterpret_cast<int *>(rec + 4 * DC);
        ri[2 * c] = split ? node : st;
        ri[2 * c + 1] = split ? 0 : size;
    }
    if (split) {
        n_sdim[node] = sdim[s];
        n_sval[node] = sval[s];
        n_range[node] = make_int2(st, st + size);
        const int r = split_rank[s];
#pragma unroll
        for (int ch = 0; ch < 2; ++ch) {
            const int x = 2 * r + ch;
            nx_parent[x] = node;
            nx_side[x] = ch;
            nx_depth[x] = depth[s] + 1;
#pragma unroll
            for (int d = 0; d < DC; ++d) {
                nx_lo[x * DC + d] = 0x7f800000;
                nx_hi[x * DC + d] = (int)0x807fffffu;
            }
        }
    }
}

template <int DC>
__global__ void k_link(int S_max, const int *__restrict__ ctl, const int *__restrict__ start, const int *__restrict__ end,
                       const int *__restrict__ parent, const int *__restrict__ side,
                       const int *__restrict__ depth, const int *__restrict__ lo, const int *__restrict__ hi,
                       const int *__restrict__ split_flag, const int *__restrict__ split_rank,
                       const int *__restrict__ sdim, const float *__restrict__ sval,
                       float4 *__restrict__ nodes, int *__restrict__ n_sdim, float *__restrict__ n_sval,
                       int2 *__restrict__ n_range, int *__restrict__ nx_parent, int *__restrict__ nx_side,
                       int *__restrict__ nx_depth, int *__restrict__ nx_lo, int *__restrict__ nx_hi,
                       const int *__restrict__ fin_flag, const int *__restrict__ fin_rank, Segs fin,
                       int *__restrict__ n_parent, int *__restrict__ roots, int fin_link) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S_max || ctl[CTL_DONE] || s >= ctl[CTL_S]) return;
    link_seg<DC>(s, ctl, start, end, parent, side, depth, lo, hi, split_flag, split_rank, sdim, sval, nodes, n_sdim, n_sval, n_range, nx_parent, nx_side, nx_depth, nx_lo, nx_hi, fin_flag, fin_rank, fin, n_parent, roots, fin_link);
}

// One block does a whole level's segment work when the level has at most
// kHeadMax segment slots: classify, the two exclusive scans (split and
// finisher flags, totals at index S_max) and link, with block barriers
// instead of eight kernel boundaries.
constexpr int HEAD_NT = 1024;
constexpr int kHeadMax = 16384;

// Exclusive scan of in[0, n) into out[0, n], out[n] = total, by one block.
__device__ void block_excl_scan(const int *in, int *out, int n, int *wsum) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int per = (n + HEAD_NT - 1) / HEAD_NT;
    const int i0 = min(n, threadIdx.x * per), i1 = min(n, i0 + per);
    int t = 0;
    for (int i = i0; i < i1; ++i) t += in[i];
    int x = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int w = wsum[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        wsum[lane] = w;
    }
    __syncthreads();
    int run = (warp ? wsum[warp - 1] : 0) + x - t;
    for (int i = i0; i < i1; ++i) {
        const int v = in[i];
        out[i] = run;
        run += v;
    }
    if (threadIdx.x == HEAD_NT - 1) out[n] = wsum[31];
    __syncthreads();
}

template <int DC>
__global__ void __launch_bounds__(HEAD_NT) k_level_head(
    int S_max, const int *__restrict__ ctl, const int *__restrict__ start, const int *__restrict__ end,
    const int *__restrict__ parent, const int *__restrict__ side, const int *__restrict__ depth,
    const int *__restrict__ lo, const int *__restrict__ hi, int leaf, int depth_cap, int fin_threshold,
    int *__restrict__ split_flag, int *__restrict__ split_rank, int *__restrict__ sdim, float *__restrict__ sval,
    float4 *__restrict__ nodes, int *__restrict__ n_sdim, float *__restrict__ n_sval, int2 *__restrict__ n_range,
    int *__restrict__ nx_parent, int *__restrict__ nx_side, int *__restrict__ nx_depth, int *__restrict__ nx_lo,
    int *__restrict__ nx_hi, int *__restrict__ fin_flag, int *__restrict__ fin_rank, Segs fin,
    int *__restrict__ n_parent, int *__restrict__ roots, int fin_link) {
    pdl_wait();
    pdl_trigger();
    __shared__ int wsum[32];
    const int S = ctl[CTL_DONE] ? 0 : min(ctl[CTL_S], S_max);
    for (int x = threadIdx.x; x < S_max; x += HEAD_NT)
        classify_seg<DC>(x, x < S, start, end, depth, lo, hi, leaf, depth_cap, fin_threshold, split_flag, fin_flag,
                         sdim, sval);
    __syncthreads();
    block_excl_scan(split_flag, split_rank, S_max, wsum);
    block_excl_scan(fin_flag, fin_rank, S_max, wsum);
    for (int x = threadIdx.x; x < S; x += HEAD_NT)
        link_seg<DC>(x, ctl, start, end, parent, side, depth, lo, hi, split_flag, split_rank, sdim, sval, nodes,
                     n_sdim, n_sval, n_range, nx_parent, nx_side, nx_depth, nx_lo, nx_hi, fin_flag, fin_rank, fin,
                     n_parent, roots, fin_link);
}

// Enqueue one level's segment work: the one-block head when the level has
// few enough segment slots, else classify + two device-wide scans + link.
// scan_ws (may be NULL) is workspace for the scans (scan_ws_words(S_max)).
template <int DC>
pg_status level_segments(int S_max, int *ctl, const Segs &cur, const Segs &nxt, int leaf, int thr, int *split_flag,
                         int *split_rank, int *sdim, float *sval, int *fin_flag, int *fin_rank, const Segs &fin,
                         float4 *nodes, int *n_sdim, float *n_sval, int2 *n_range, int *n_parent, int *roots,
                         int fin_link, int *scan_ws, cudaStream_t s, bool pdl = false) {
    if (S_max <= kHeadMax) {
        if (pdl) {
            PG_CUDA(launch_pdl(k_level_head<DC>, 1, HEAD_NT, 0, s, S_max, ctl, cur.start, cur.end, cur.parent,
                               cur.side, cur.depth, cur.lo, cur.hi, leaf, PG_DEPTH_CAP, thr, split_flag, split_rank,
                               sdim, sval, nodes, n_sdim, n_sval, n_range, nxt.parent, nxt.side, nxt.depth, nxt.lo,
                               nxt.hi, fin_flag, fin_rank, fin, n_parent, roots, fin_link));
        } else {
            k_level_head<DC><<<1, HEAD_NT, 0, s>>>(S_max, ctl, cur.start, cur.end, cur.parent, cur.side, cur.depth,
                                                   cur.lo, cur.hi, leaf, PG_DEPTH_CAP, thr, split_flag, split_rank,
                                                   sdim, sval, nodes, n_sdim, n_sval, n_range, nxt.parent, nxt.side,
                                                   nxt.depth, nxt.lo, nxt.hi, fin_flag, fin_rank, fin, n_parent,
                                                   roots, fin_link);
        }
        count_launch();
        return PG_OK;
    }
    const int gs = ceil_div_i(S_max, BT);
    k_classify<DC><<<gs, BT, 0, s>>>(S_max, ctl, cur.start, cur.end, cur.depth, cur.lo, cur.hi, leaf, PG_DEPTH_CAP,
                                     thr, split_flag, fin_flag, sdim, sval);
    count_launch();
    if (scan_ws) {
        PG_TRY(exclusive_scan_ws(split_flag, split_rank, S_max, scan_ws, s));
        PG_TRY(exclusive_scan_ws(fin_flag, fin_rank, S_max, scan_ws, s));
    } else {
        PG_TRY(exclusive_scan(split_flag, split_rank, S_max, s));
        PG_TRY(exclusive_scan(fin_flag, fin_rank, S_max, s));
    }
    k_link<DC><<<gs, BT, 0, s>>>(S_max, ctl, cur.start, cur.end, cur.parent, cur.side, cur.depth, cur.lo, cur.hi,
                                 split_flag, split_rank, sdim, sval, nodes, n_sdim, n_sval, n_range, nxt.parent,
                                 nxt.side, nxt.depth, nxt.lo, nxt.hi, fin_flag, fin_rank, fin, n_parent, roots,
                                 fin_link);
    count_launch();
    return PG_OK;
}

// Move every point of a split segment to its child range (see k_part_tiles)
// and reduce the children's tight boxes: per tile in shared memory (children
// of a tile are few and consecutive), then one global atomic per child and
// dimension; a child that finds its slot taken goes straight to global memory.
template <int DC>
__global__ void __launch_bounds__(PT_THREADS, DC <= 4 ? 8 : 4) k_part(int64_t n, const float4 *__restrict__ P, float4 *__restrict__ Q,
                                                     const int *__restrict__ seg_of, int *__restrict__ seg_of_nx,
                                                     const int *__restrict__ start, const int *__restrict__ end,
                                                     const int *__restrict__ split_flag,
                                                     const int *__restrict__ split_rank,
                                                     const unsigned *__restrict__ tcarry,
                                                     const unsigned *__restrict__ twords, int *__restrict__ nx_start,
                                                     int *__restrict__ nx_end, int *__restrict__ nx_lo,
                                                     int *__restrict__ nx_hi, const int *__restrict__ T) {
    pdl_wait();
    pdl_trigger();
    constexpr int W = bucket_w(DC);
    if (*T == 0) return;
    __shared__ int tag[kBoxSlots];
    __shared__ int b_lo[kBoxSlots * DC], b_hi[kBoxSlots * DC];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int base = blockIdx.x * PT_TILE;
    const int n32 = (int)n;
    if (threadIdx.x < kBoxSlots) tag[threadIdx.x] = -1;
    for (int x = threadIdx.x; x < kBoxSlots * DC; x += PT_THREADS) {
        b_lo[x] = 0x7f800000;
        b_hi[x] = (int)0x807fffffu;
    }
    __syncthreads();
    const unsigned *tw = twords + (size_t)blockIdx.x * PT_TW;
    const unsigned carry = tcarry[blockIdx.x];
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int j = 0; j < PT_ROWS; ++j) {
        const int i = base + j * PT_THREADS + threadIdx.x;
        const bool valid = i < n32;
        float4 v[W];
#pragma unroll
        for (int w = 0; w < W; ++w) v[w] = valid ? P[(size_t)i * W + w] : make_float4(0.f, 0.f, 0.f, 0.f);
        const int s = valid ? seg_of[i] : -1;
        const int e = j * PT_WARPS + warp;
        const unsigned F = tw[e], R = tw[PT_WR + e];
        const int f = (F >> lane) & 1u;
        const unsigned m = R & (lt | (1u << lane));
        int r;
        if (m) r = __popc(F & lt & ~((1u << (31 - __clz(m))) - 1u));
        else r = (int)(seg_combine(carry, tw[2 * PT_WR + e]) & 0x7fffffffu) + __popc(F & lt);
        int child = -1;
        if (valid) {
            int dst = i;
            if (s >= 0 && split_flag[s]) {
                const int st = start[s], en = end[s], rk = split_rank[s];
                if (f) { dst = st + r; child = 2 * rk; }
                else { dst = en - 1 - ((i - st) - r); child = 2 * rk + 1; }
                if (i == en - 1) {
                    const int nl = r + f;
                    nx_start[2 * rk] = st;
                    nx_end[2 * rk] = st + nl;
                    nx_start[2 * rk + 1] = st + nl;
                    nx_end[2 * rk + 1] = en;
                }
            }
#pragma unroll
            for (int w = 0; w < W; ++w) Q[(size_t)dst * W + w] = v[w];
            seg_of_nx[dst] = child;
        }
        const float *cf = reinterpret_cast<const float *>(v);
        unsigned active = __ballot_sync(0xffffffffu, child >= 0);
        while (active) {
            const int leader = __ffs(active) - 1;
            const int key = __shfl_sync(0xffffffffu, child, leader);
            const bool mine = child == key;
            const unsigned grp = __ballot_sync(0xffffffffu, mine);
            int slot = -1;
            if (lane == leader) {
                const int t = atomicCAS(&tag[key & (kBoxSlots - 1)], -1, key);
                if (t == -1 || t == key) slot = key & (kBoxSlots - 1);
            }
#pragma unroll
            for (int d = 0; d < DC; ++d) {
                const int e = f2o(cf[d]);
                const int a = __reduce_min_sync(0xffffffffu, mine ? e : INT_MAX);
                const int c = __reduce_max_sync(0xffffffffu, mine ? e : INT_MIN);
                if (lane == leader) {
                    if (slot >= 0) {
                        atomicMin(&b_lo[slot * DC + d], a);
                        atomicMax(&b_hi[slot * DC + d], c);
                    } else {
                        atomicMin(&nx_lo[key * DC + d], a);
                        atomicMax(&nx_hi[key * DC + d], c);
                    }
                }
            }
            active &= ~grp;
        }
    }
    __syncthreads();
    for (int x = threadIdx.x; x < kBoxSlots * DC; x += PT_THREADS) {
        const int key = tag[x / DC];
        if (key >= 0) {
            atomicMin(&nx_lo[key * DC + x % DC], b_lo[x]);
            atomicMax(&nx_hi[key * DC + x % DC], b_hi[x]);
        }
    }
}

// ---------------------------------------------------------------- object median
// Object-median levels (paper Section 4: kd-tree splits by spatial median or
// by object median): a split segment of c points sends its floor(c / 2)
// smallest points along the split dimension to the left child, ties by
// position.  The points of all split segments are put in (segment,
// coordinate, position) order by two stable radix sorts (coordinate first,
// then segment); a point's rank inside its segment's run decides its side,
// and the point of rank floor(c / 2) gives the node's split value.

// Once the loop is done (T == 0) the segment ids of later levels were never
// written, so they are not read: every key becomes the sentinel.
template <int DC>
__global__ void k_obj_keys(int n, const float4 *__restrict__ P, const int *__restrict__ seg_of,
                           const int *__restrict__ split_flag, const int *__restrict__ sdim,
                           const int *__restrict__ T, uint32_t sentinel, uint32_t *__restrict__ kc,
                           uint32_t *__restrict__ ks, uint32_t *__restrict__ val) {
    constexpr int W = bucket_w(DC);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int s = *T != 0 ? seg_of[i] : -1;
    const bool a = s >= 0 && split_flag[s];
    const float x = a ? reinterpret_cast<const float *>(P)[(size_t)i * 4 * W + sdim[s]] : 0.f;
    kc[i] = a ? ((uint32_t)f2o(x) ^ 0x80000000u) : 0xffffffffu;   // unsigned key in float order
    ks[i] = a ? (uint32_t)s : sentinel;
    val[i] = (uint32_t)i;
}

__global__ void k_obj_gather(int n, const uint32_t *__restrict__ ks, const uint32_t *__restrict__ pos,
                             uint32_t *__restrict__ out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) out[j] = ks[pos[j]];
}

__global__ void k_obj_first(int n, const uint32_t *__restrict__ sk, uint32_t sentinel, int *__restrict__ first) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const uint32_t s = sk[j];
    if (s != sentinel && (j == 0 || sk[j - 1] != s)) first[s] = j;
}

template <int DC>
__global__ void k_obj_flags(int n, const uint32_t *__restrict__ sk, const uint32_t *__restrict__ spos,
                            uint32_t sentinel, const int *__restrict__ first, const int *__restrict__ start,
                            const int *__restrict__ end, const int *__restrict__ split_rank,
                            const int *__restrict__ sdim, const float4 *__restrict__ P, const int *__restrict__ ctl,
                            int *__restrict__ pflag, float *__restrict__ n_sval) {
    constexpr int W = bucket_w(DC);
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const uint32_t s = sk[j];
    if (s == sentinel) return;
    const int rank = j - first[s];
    const int half = (end[s] - start[s]) / 2;
    const int i = (int)spos[j];
    pflag[i] = rank < half;
    if (rank == half)   // the first right point: the node's split value
        n_sval[ctl[CTL_NB] + split_rank[s]] = reinterpret_cast<const float *>(P)[(size_t)i * 4 * W + sdim[s]];
}

constexpr int FIN_NT = 512;                  // threads of a finisher block
constexpr size_t kFinSmemBudget = 72 * 1024;    // shared memory of a finisher block (three blocks per SM)

// Segments small enough for one block's shared memory are finished by the
// in-block builder; node slots are reserved by bucket position: segment
// [st, en) uses slots [nb + st, nb + en - 1).  Blocks take segments from the
// control block's work counter until all ctl[CTL_FIN] are done; the points
// are in P0 or P1 by the parity of the levels that moved them.
template <int DC>
__global__ void __launch_bounds__(FIN_NT, 3) k_finish(Segs fin, float4 *P0, float4 *P1, int leaf, int ns, int sc,
                                                      int *ctl, float4 *nodes, int *n_sdim, float *n_sval,
                                                      int2 *n_range, int *root_rec, int *depth_max, int *n_parent,
                                                      int *leaf_parent) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int f_take;
    float4 *P = (ctl[CTL_SCATTERS] & 1) ? P1 : P0;
    const int nb = ctl[CTL_NB], total = ctl[CTL_FIN];
    for (;;) {
        if (threadIdx.x == 0) f_take = atomicAdd(&ctl[CTL_FIN_NEXT], 1);
        __syncthreads();
        const int f = f_take;
        __syncthreads();
        if (f >= total) break;
        const int st = fin.start[f], en = fin.end[f];
        const CtaTree r = cta_build_smem<DC, FIN_NT>(P, st, en, fin.lo + (size_t)f * DC, fin.hi + (size_t)f * DC, smem, ns,
                                                     sc, leaf, nb + st, nodes, n_sdim, n_sval, n_range, fin.depth[f],
                                                     n_parent, leaf_parent,
                                                     fin.parent[f] >= 0 ? 2 * fin.parent[f] + fin.side[f] : -1);
        if (threadIdx.x == 0) {
            const int p = fin.parent[f];
            if (p >= 0) {
                int *ri = reinterpret_cast<int *>(nodes + (size_t)p * node_w(DC)) + 4 * DC;
                const int c = fin.side[f];
                ri[2 * c] = r.root_ref;
                ri[2 * c + 1] = r.root_cnt;
            } else {
                root_rec[0] = r.root_ref;
                root_rec[1] = r.root_cnt;
            }
            atomicMax(depth_max, r.depth);
        }
        __syncthreads();   // the block's shared memory is reused by its next segment
    }
}

// Every bucket entry records the code (2*node + side) of the leaf that holds
// it: one thread per level node (the first ctl[CTL_NB] slots) fills its leaf
// children's ranges (entries of a leaf root keep -1).
template <int DC>
__global__ void k_leaf_parents(const float4 *__restrict__ nodes, const int *__restrict__ ctl,
                               int *__restrict__ leaf_parent) {
    const int nb = ctl[CTL_NB];
    for (int nd = blockIdx.x * blockDim.x + threadIdx.x; nd < nb; nd += gridDim.x * blockDim.x) {
        const int *ri = reinterpret_cast<const int *>(nodes + (size_t)nd * node_w(DC)) + 4 * DC;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int ref = ri[2 * c], cnt = ri[2 * c + 1];
            for (int i = 0; i < cnt; ++i) leaf_parent[ref + i] = 2 * nd + c;
        }
    }
}

// The device-driven level loop (a build enqueued into a CUDA graph under
// stream capture) runs while no level has ended the loop and the depth cap
// is not passed.
__global__ void k_level_cond(cudaGraphConditionalHandle h, const int *__restrict__ ctl, int cap) {
    cudaGraphSetConditional(h, (!ctl[CTL_DONE] && ctl[CTL_CUR] <= cap) ? 1u : 0u);
}

// After a device-driven build: the final order is in P1 when an odd number
// of levels moved points; it is copied to P0, which becomes the bucket.
__global__ void k_copy_if_odd(const int *__restrict__ ctl, const float4 *__restrict__ P1, float4 *__restrict__ P0,
                              size_t words) {
    if (!(ctl[CTL_SCATTERS] & 1)) return;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < words; i += (size_t)gridDim.x * blockDim.x)
        P0[i] = P1[i];
}

// After a device-driven build: the tree descriptor (root from the control
// block and the finisher's root record, root box from the packed box) and the
// host-side metadata words the library reads back when it next needs them:
// root_ref, root_cnt, depth, level nodes, finisher segments, done, then the
// root box (DC lows, DC highs) as float bits.
template <int DC>
__global__ void k_tree_meta(const int *__restrict__ ctl, const int *__restrict__ rec, const int *__restrict__ box,
                            int n, const float4 *bucket, const float4 *nodes, const int *parent,
                            const int *leaf_parent, TreeDesc *desc, int *meta) {
    if (threadIdx.x != 0) return;
    const bool root_split = ctl[CTL_ROOT_SPLIT] != 0;
    const int fin_total = ctl[CTL_FIN];
    int root_ref = 0, root_cnt = root_split ? 0 : n;
    if (!root_split && fin_total > 0) { root_ref = rec[0]; root_cnt = rec[1]; }
    TreeDesc d;
    d.bucket = bucket;
    d.nodes = nodes;
    d.parent = parent;
    d.leaf_parent = leaf_parent;
    d.root_ref = root_ref;
    d.root_cnt = root_cnt;
    for (int c = 0; c < PG_MAX_DIM; ++c) {
        d.root_lo[c] = c < DC ? o2f(box[c]) : 0.f;
        d.root_hi[c] = c < DC ? o2f(box[DC + c]) : 0.f;
    }
    *desc = d;
    meta[0] = root_ref;
    meta[1] = root_cnt;
    meta[2] = max(ctl[CTL_LEVELS], fin_total > 0 ? rec[2] : 0);
    meta[3] = ctl[CTL_NB];
    meta[4] = fin_total;
    meta[5] = ctl[CTL_DONE];
    for (int c = 0; c < DC; ++c) {
        meta[8 + c] = __float_as_int(d.root_lo[c]);
        meta[8 + PG_MAX_DIM + c] = __float_as_int(d.root_hi[c]);
    }
}

// Level 0 of a single tree: one segment over all n points with the packed
// root box; the control block starts with one live segment.
template <int DC>
__global__ void k_level0_init(int n, const int *__restrict__ box, Segs cur, int *__restrict__ ctl) {
    const int t = threadIdx.x;
    if (t == 0) {
        cur.start[0] = 0;
        cur.end[0] = n;
        cur.parent[0] = -1;
        cur.side[0] = 0;
        cur.depth[0] = 0;
        for (int w = 0; w < CTL_WORDS; ++w) ctl[w] = 0;
        ctl[CTL_S] = 1;
    }
    if (t < DC) {
        cur.lo[t] = box[t];
        cur.hi[t] = box[DC + t];
    }
}

template <int DC>
struct Builder {
    // deferred: the stream is being captured into a CUDA graph, so nothing
    // may wait on the host; the level loop becomes a device-driven loop and
    // the tree's host-side metadata is read back when it is next needed.
    // lazy_meta (eager builds): the level loop still reads its end flag, but
    // the root record and descriptor are written by a kernel and the
    // host-side metadata is read back when it is next needed, as above.
    static pg_status run(float4 *packed, int *box, int64_t n, int leaf, int rule, cudaStream_t s, pg_tree *t,
                         bool deferred, bool lazy_meta = false);
};

pg_status grow_nodes(pg_tree *t, int need, cudaStream_t s) {
    if (need <= t->node_cap) return PG_OK;
    int cap = std::max(need, std::max(16, t->node_cap * 2));
    const int nw = node_w(t->dc);
    float4 *nodes = nullptr;
    int *sd = nullptr, *par = nullptr;
    float *sv = nullptr;
    int2 *rg = nullptr;
    pg_status st = dalloc_n(&nodes, (size_t)cap * nw, s);
    if (st == PG_OK) st = dalloc_n(&sd, cap, s);
    if (st == PG_OK) st = dalloc_n(&sv, cap, s);
    if (st == PG_OK) st = dalloc_n(&rg, cap, s);
    if (st == PG_OK) st = dalloc_n(&par, cap, s);
    if (st != PG_OK) {
        dfree(nodes, s); dfree(sd, s); dfree(sv, s); dfree(rg, s); dfree(par, s);
        return st;
    }
    if (t->num_nodes > 0) {
        PG_CUDA(cudaMemcpyAsync(nodes, t->nodes, sizeof(float4) * nw * (size_t)t->num_nodes, cudaMemcpyDeviceToDevice, s));
        PG_CUDA(cudaMemcpyAsync(sd, t->split_dim, sizeof(int) * (size_t)t->num_nodes, cudaMemcpyDeviceToDevice, s));
        PG_CUDA(cudaMemcpyAsync(sv, t->split_val, sizeof(float) * (size_t)t->num_nodes, cudaMemcpyDeviceToDevice, s));
        PG_CUDA(cudaMemcpyAsync(rg, t->node_range, sizeof(int2) * (size_t)t->num_nodes, cudaMemcpyDeviceToDevice, s));
        PG_CUDA(cudaMemcpyAsync(par, t->parent, sizeof(int) * (size_t)t->num_nodes, cudaMemcpyDeviceToDevice, s));
    }
    dfree(t->nodes, s);
    dfree(t->split_dim, s);
    dfree(t->split_val, s);
    dfree(t->node_range, s);
    dfree(t->parent, s);
    t->nodes = nodes;
    t->split_dim = sd;
    t->split_val = sv;
    t->node_range = rg;
    t->parent = par;
    t->node_cap = cap;
    return PG_OK;
}

template <int DC>
pg_status Builder<DC>::run(float4 *P0, int *box, int64_t n, int leaf, int rule, cudaStream_t s, pg_tree *t,
                           bool deferred, bool lazy_meta) {
    constexpr int W = bucket_w(DC);
    // Split segments hold more than `leaf` points and are disjoint, so a level
    // has at most 2*floor(n/(leaf+1)) segments.
    const int seg_cap = (int)std::max<int64_t>(2, 2 * (n / (leaf + 1)) + 2);

    Scratch sP1, sSeg0, sSeg1, sSegA, sSegB, sLvl, sBsum, sCtl;
    PG_TRY(sP1.alloc(sizeof(float4) * W * (size_t)n, s));
    PG_TRY(sSeg0.alloc(sizeof(int) * (size_t)n, s));
    PG_TRY(sSeg1.alloc(sizeof(int) * (size_t)n, s));
    const size_t seg_words = (size_t)seg_cap * (5 + 2 * DC);
    PG_TRY(sSegA.alloc(sizeof(int) * seg_words, s));
    PG_TRY(sSegB.alloc(sizeof(int) * seg_words, s));
    // per-level: split_flag, split_rank (+1), sdim, sval, fin_flag, fin_rank (+1)
    PG_TRY(sLvl.alloc(sizeof(int) * (size_t)(6 * seg_cap + 2), s));
    int *split_flag = sLvl.as<int>();
    int *split_rank = split_flag + seg_cap;
    int *sdim = split_rank + seg_cap + 1;
    float *sval = reinterpret_cast<float *>(sdim + seg_cap);
    int *fin_flag = sdim + 2 * seg_cap;
    int *fin_rank = fin_flag + seg_cap;
    const int ntiles = std::max(1, ceil_div_i(n, PT_TILE));
    PG_TRY(sBsum.alloc(sizeof(unsigned) * (size_t)ntiles * (1 + PT_TW), s));
    unsigned *tsum = sBsum.as<unsigned>(), *twords = tsum + ntiles;
    PG_TRY(sCtl.alloc(sizeof(int) * CTL_WORDS, s));
    int *ctl = sCtl.as<int>();
    // segments handed to the block-scope finisher (disjoint, > leaf points each)
    const int fin_cap = (int)(n / (leaf + 1) + 1);
    Scratch sFin;
    PG_TRY(sFin.alloc(sizeof(int) * (size_t)fin_cap * (5 + 2 * DC), s));
    Segs fin;
    {
        int *b = sFin.as<int>();
        fin.start = b; fin.end = b + fin_cap; fin.parent = b + 2 * fin_cap; fin.side = b + 3 * fin_cap;
        fin.depth = b + 4 * fin_cap; fin.lo = b + 5 * fin_cap; fin.hi = b + (5 + DC) * fin_cap;
    }
    auto carve = [&](Scratch &sc) {
        int *b = sc.as<int>();
        Segs g;
        g.start = b; g.end = b + seg_cap; g.parent = b + 2 * seg_cap; g.side = b + 3 * seg_cap;
        g.depth = b + 4 * seg_cap; g.lo = b + 5 * seg_cap; g.hi = b + (5 + DC) * seg_cap;
        return g;
    };
    Segs cur = carve(sSegA), nxt = carve(sSegB);

    float4 *P = P0, *Q = sP1.as<float4>();
    int *seg_of = sSeg0.as<int>(), *seg_of_nx = sSeg1.as<int>();
    PG_TRY(fill_words(seg_of, 0u, (size_t)n, s));   // all in segment 0
    if (!t->leaf_parent) PG_TRY(dalloc_n(&t->leaf_parent, (size_t)n, s));
    PG_TRY(fill_words(t->leaf_parent, 0xffffffffu, (size_t)n, s));   // a leaf root keeps -1
    // Segments of up to fin_max points are finished in one block's shared memory.
    // (object-median trees split every level on the device: no finisher)
    const int fin_max = rule == PG_SPLIT_OBJECT ? 0 : smem_build_points(DC, leaf, kFinSmemBudget);
    const int fin_sc = smem_seg_cap(fin_max, leaf);
    const size_t fin_smem = smem_build_bytes(fin_max, fin_sc, DC);
    // Node slots: every global split holds more than fin_max points (at most
    // n/(fin_max+1) per level), and finisher segment [st, en) reserves slots
    // [nb + st, nb + en) after the nb global nodes.  Unused slots stay
    // all-ones (cnt = -1).
    const int64_t slots = rule == PG_SPLIT_OBJECT ? n + 64 : (int64_t)(PG_DEPTH_CAP + 1) * (n / (fin_max + 1)) + 64 + n;
    if (slots >= ((int64_t)1 << 31)) return fail(PG_EINVAL, "tree build: too many node slots");
    PG_TRY(grow_nodes(t, (int)slots, s));
    PG_TRY(fill_words(t->nodes, 0xffffffffu, 4 * node_w(DC) * (size_t)slots, s));

    // level 0: one segment covering everything, box reduced by k_pack
    {
        k_level0_init<DC><<<1, 32, 0, s>>>((int)n, box, cur, ctl);
        count_launch();
    }
    // The host enqueues levels without waiting; it starts checking for the
    // end around the level where uniform data would stop.
    int est = 1;
    const int64_t unit = rule == PG_SPLIT_OBJECT ? (int64_t)leaf + 1 : fin_max;
    while ((unit << (est - 1)) < n && est < PG_DEPTH_CAP) ++est;
    // object-median scratch: keys, segment keys, positions, two temporaries, a
    // gathered copy, flags (n each) and the first sorted index of each segment
    Scratch sObj;
    uint32_t *okc = nullptr, *oks = nullptr, *ov = nullptr, *ot0 = nullptr, *ot1 = nullptr, *oks2 = nullptr;
    int *opflag = nullptr, *ofirst = nullptr;
    if (rule == PG_SPLIT_OBJECT) {
        PG_TRY(sObj.alloc(sizeof(uint32_t) * (size_t)(7 * n + seg_cap + 8), s));
        okc = sObj.as<uint32_t>(); oks = okc + n; ov = oks + n; ot0 = ov + n; ot1 = ot0 + n; oks2 = ot1 + n;
        opflag = reinterpret_cast<int *>(oks2 + n);
        ofirst = opflag + n;
    }
    if (deferred) {
        if (rule == PG_SPLIT_OBJECT || fin_max <= 0)
            return fail(PG_EUNSUPPORTED, "tree build under stream capture: spatial-median split only");
        // Every segment of a level list is a child of a segment with more
        // than fin_max points, so a fixed slot count bounds every level.
        const int S_fix = (int)std::min<int64_t>(seg_cap, 2 * (n / (fin_max + 1)) + 2);
        Scratch sScan;
        int *scan_ws = nullptr;
        if (S_fix > kHeadMax) {
            PG_TRY(sScan.alloc(sizeof(int) * (size_t)scan_ws_words(S_fix), s));
            scan_ws = sScan.as<int>();
        }
        // Graph being captured and its current dependencies: a WHILE node goes
        // after them, its body is captured from a side stream.
        cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
        cudaGraph_t graph = nullptr;
        const cudaGraphNode_t *deps = nullptr;
        const cudaGraphEdgeData *edges = nullptr;
        size_t ndeps = 0;
        PG_CUDA(cudaStreamGetCaptureInfo(s, &cst, nullptr, &graph, &deps, &edges, &ndeps));
        if (cst != cudaStreamCaptureStatusActive) return fail(PG_ECUDA, "tree build: stream capture not active");
        cudaGraphConditionalHandle cond;
        PG_CUDA(cudaGraphConditionalHandleCreate(&cond, graph, 1, cudaGraphCondAssignDefault));
        cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
        cp.conditional.handle = cond;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t loop_node;
        PG_CUDA(cudaGraphAddNode(&loop_node, graph, deps, edges, ndeps, &cp));
        cudaStream_t side;
        PG_CUDA(cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking));
        pg_status st = PG_OK;
        cudaError_t e = cudaStreamBeginCaptureToGraph(side, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                                      cudaStreamCaptureModeRelaxed);
        if (e == cudaSuccess) {
            // body: two levels (the ping-pong buffers swap roles), then the test
            float4 *Pa = P, *Pb = Q;
            int *sa = seg_of, *sb = seg_of_nx;
            Segs ca = cur, cb = nxt;
            const int *T = split_rank + S_fix;
            for (int half = 0; half < 2 && st == PG_OK; ++half) {
                st = level_segments<DC>(S_fix, ctl, ca, cb, leaf, fin_max, split_flag, split_rank, sdim, sval,
                                        fin_flag, fin_rank, fin, t->nodes, t->split_dim, t->split_val,
                                        t->node_range, t->parent, nullptr, 0, scan_ws, side);
                if (st != PG_OK) break;
                k_part_tiles<DC><<<ntiles, PT_THREADS, 0, side>>>(n, Pa, sa, split_flag, sdim, sval, T, tsum, twords);
                k_part_carry<<<1, 1024, 0, side>>>(tsum, ntiles, T, ctl, fin_rank + S_fix, -1);
                k_part<DC><<<ntiles, PT_THREADS, 0, side>>>(n, Pa, Pb, sa, sb, ca.start, ca.end, split_flag,
                                                            split_rank, tsum, twords, cb.start, cb.end, cb.lo, cb.hi,
                                                            T);
                for (int c = 0; c < 3; ++c) count_launch();
                std::swap(Pa, Pb);
                std::swap(sa, sb);
                std::swap(ca, cb);
            }
            k_level_cond<<<1, 1, 0, side>>>(cond, ctl, PG_DEPTH_CAP + 1);
            count_launch();
            e = cudaGetLastError();
            cudaGraph_t body_out = nullptr;
            const cudaError_t e2 = cudaStreamEndCapture(side, &body_out);
            if (e == cudaSuccess) e = e2;
        }
        cudaStreamDestroy(side);
        if (st != PG_OK) return st;
        PG_CUDA(e);
        PG_CUDA(cudaStreamUpdateCaptureDependencies(s, &loop_node, nullptr, 1, cudaStreamSetCaptureDependencies));
        // after the loop: finisher, leaf codes, final order into P0, descriptor
        Scratch sRec;
        PG_TRY(sRec.alloc(sizeof(int) * 3, s));
        int *rec = sRec.as<int>();
        PG_TRY(fill_words(rec, 0u, 3, s));
        PG_CUDA(cudaFuncSetAttribute(k_finish<DC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fin_smem));
        k_finish<DC><<<num_sms() * 3, FIN_NT, fin_smem, s>>>(fin, P0, sP1.as<float4>(), leaf, fin_max, fin_sc, ctl,
                                                              t->nodes, t->split_dim, t->split_val, t->node_range,
                                                              rec, rec + 2, t->parent, t->leaf_parent);
        k_leaf_parents<DC><<<num_sms() * 8, BT, 0, s>>>(t->nodes, ctl, t->leaf_parent);
        k_copy_if_odd<<<num_sms() * 8, BT, 0, s>>>(ctl, sP1.as<float4>(), P0, (size_t)W * n);
        for (int c = 0; c < 3; ++c) count_launch();
        PG_TRY(check_launch("build (device-driven) finish"));
        if (!t->desc) PG_TRY(dalloc_n(&t->desc, 1, s));
        if (!t->meta) PG_TRY(dalloc_n(&t->meta, (size_t)kTreeMetaWords, s));
        k_tree_meta<DC><<<1, 32, 0, s>>>(ctl, rec, box, (int)n, P0, t->nodes, t->parent, t->leaf_parent, t->desc,
                                         t->meta);
        count_launch();
        PG_TRY(check_launch("build (device-driven) descriptor"));
        t->bucket = P0;
        t->meta_pending = true;
        t->num_nodes = (int)std::min<int64_t>(slots, INT32_MAX);   // until read back: every reserved slot
        t->depth = -1;
        t->root_ref = -1;
        t->root_cnt = 0;
        return PG_OK;
    }
    int hctl[CTL_WORDS] = {0};
    int level = 0;
    // With a finisher, every segment of a level list is a child of a split
    // segment of more than fin_max points: that bounds the list, so the
    // one-block head serves every level of most builds.
    const int64_t S_bound = (rule == PG_SPLIT_SPATIAL && fin_max > 0)
                                ? std::min<int64_t>(seg_cap, 2 * (n / (fin_max + 1)) + 2) : seg_cap;
    // The end flag is read from the expected depth on, then every 2, then 4
    // levels (levels enqueued after the end do nothing).
    int next_check = est - 1, stride = 1;
    for (; level <= PG_DEPTH_CAP + 1; ++level) {
        const int S_max = (int)std::min<int64_t>((int64_t)1 << std::min(level, 30), S_bound);
        PG_TRY(level_segments<DC>(S_max, ctl, cur, nxt, leaf, fin_max, split_flag, split_rank, sdim, sval, fin_flag,
                                  fin_rank, fin, t->nodes, t->split_dim, t->split_val, t->node_range, t->parent,
                                  nullptr, 0, nullptr, s, rule != PG_SPLIT_OBJECT));
        const int *T = split_rank + S_max;
        if (rule == PG_SPLIT_OBJECT) {
            const int g = ceil_div_i(n, BT);
            const uint32_t sentinel = (uint32_t)S_max;
            int sbits = 1;
            while (sbits < 32 && ((int64_t)1 << sbits) <= (int64_t)S_max) ++sbits;
            k_obj_keys<DC><<<g, BT, 0, s>>>((int)n, P, seg_of, split_flag, sdim, T, sentinel, okc, oks, ov);
            count_launch();
            uint32_t *k1 = nullptr, *v1 = nullptr, *k2 = nullptr, *v2 = nullptr;
            PG_TRY(radix_sort_pairs(okc, ov, false, ot0, ot1, n, 32, s, &k1, &v1));
            k_obj_gather<<<g, BT, 0, s>>>((int)n, oks, v1, oks2);
            count_launch();
            // temporaries for the second sort: two buffers other than oks2 and v1
            uint32_t *cand[4] = {okc, ov, ot0, ot1}, *tmp[2];
            int nt = 0;
            for (uint32_t *c : cand)
                if (c != v1 && nt < 2) tmp[nt++] = c;
            PG_TRY(radix_sort_pairs(oks2, v1, false, tmp[0], tmp[1], n, sbits, s, &k2, &v2));
            k_obj_first<<<g, BT, 0, s>>>((int)n, k2, sentinel, ofirst);
            k_obj_flags<DC><<<g, BT, 0, s>>>((int)n, k2, v2, sentinel, ofirst, cur.start, cur.end, split_rank, sdim, P,
                                            ctl, opflag, t->split_val);
            k_part_tiles<DC, true><<<ntiles, PT_THREADS, 0, s>>>(n, P, seg_of, split_flag, sdim, sval, T, tsum,
                                                                 twords, opflag);
            k_part_carry<<<1, 1024, 0, s>>>(tsum, ntiles, T, ctl, fin_rank + S_max, level);
            k_part<DC><<<ntiles, PT_THREADS, 0, s>>>(n, P, Q, seg_of, seg_of_nx, cur.start, cur.end, split_flag,
                                                     split_rank, tsum, twords, nxt.start, nxt.end, nxt.lo, nxt.hi, T);
            for (int c = 0; c < 5; ++c) count_launch();
        } else {
            // one chain of dependent launches per level (head, tiles, carry,
            // move): each may be scheduled while the one before finishes
            PG_CUDA(launch_pdl(k_part_tiles<DC>, ntiles, PT_THREADS, 0, s, n, P, seg_of, split_flag, sdim, sval, T,
                               tsum, twords, nullptr));
            PG_CUDA(launch_pdl(k_part_carry, 1, 1024, 0, s, tsum, ntiles, T, ctl, fin_rank + S_max, level));
            count_launch();
            count_launch();
            KTimer kt("build_scatter", s);
            PG_CUDA(launch_pdl(k_part<DC>, ntiles, PT_THREADS, 0, s, n, P, Q, seg_of, seg_of_nx, cur.start, cur.end,
                               split_flag, split_rank, tsum, twords, nxt.start, nxt.end, nxt.lo, nxt.hi, T));
            count_launch();
        }
        PG_TRY(check_launch("build level"));
        std::swap(P, Q);
        std::swap(seg_of, seg_of_nx);
        std::swap(cur, nxt);
        if (level >= next_check || level == PG_DEPTH_CAP + 1) {
            PG_TRY(read_small(hctl, ctl, sizeof(hctl), s));
            if (hctl[CTL_DONE]) break;
            stride = std::min(2 * stride, 4);
            next_check = level + stride;
        }
    }
    if (!hctl[CTL_DONE]) return fail(PG_ECUDA, "tree build: level count exceeded the depth cap");
    const int nb = hctl[CTL_NB], fin_total = hctl[CTL_FIN];
    const bool root_split = hctl[CTL_ROOT_SPLIT] != 0;
    // the buffers alternate once per level that split something
    P = (hctl[CTL_SCATTERS] % 2 == 0) ? P0 : sP1.as<float4>();
    t->num_nodes = fin_total > 0 ? nb + (int)n : nb;
    t->depth = hctl[CTL_LEVELS];
    t->root_ref = 0;
    t->root_cnt = root_split ? 0 : (int)n;
    Scratch sRec;
    int *rec = nullptr;
    if (fin_total > 0 || lazy_meta) {
        PG_TRY(sRec.alloc(sizeof(int) * 3, s));
        rec = sRec.as<int>();
        PG_TRY(fill_words(rec, 0u, 3, s));
    }
    if (fin_total > 0) {
        PG_CUDA(cudaFuncSetAttribute(k_finish<DC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fin_smem));
        {
            KTimer kt("build_finish", s);
            k_finish<DC><<<std::min(fin_total, num_sms() * 3), FIN_NT, fin_smem, s>>>(
                fin, P0, sP1.as<float4>(), leaf, fin_max, fin_sc, ctl, t->nodes, t->split_dim, t->split_val,
                t->node_range, rec, rec + 2, t->parent, t->leaf_parent);
            count_launch();
        }
        PG_TRY(check_launch("build finish"));
        if (!lazy_meta) {
            int h[3];
            PG_TRY(read_small(h, rec, sizeof(int) * 3, s));
            t->depth = std::max(t->depth, h[2]);
            if (!root_split) {   // the whole tree was one finisher segment
                t->root_ref = h[0];
                t->root_cnt = h[1];
            }
        }
    }
    // leaves of finisher segments were recorded by the finisher; the level
    // nodes' leaf children are recorded here
    if (nb > 0) {
        k_leaf_parents<DC><<<ceil_div_i(nb, BT), BT, 0, s>>>(t->nodes, ctl, t->leaf_parent);
        count_launch();
    }
    // The final array becomes the bucket; the other ping-pong buffer is freed.
    if (P == P0) {
        t->bucket = P0;
    } else {
        t->bucket = P;
        sP1.p = nullptr;           // ownership moves to the tree
        dfree(P0, s);
    }
    if (lazy_meta) {
        if (!t->desc) PG_TRY(dalloc_n(&t->desc, 1, s));
        if (!t->meta) PG_TRY(dalloc_n(&t->meta, (size_t)kTreeMetaWords, s));
        k_tree_meta<DC><<<1, 32, 0, s>>>(ctl, rec, box, (int)n, t->bucket, t->nodes, t->parent, t->leaf_parent,
                                         t->desc, t->meta);
        count_launch();
        PG_TRY(check_launch("build descriptor"));
        t->meta_pending = true;
    }
    return PG_OK;
}

// ---------------------------------------------------------------- forest
// Many independent trees at once: level 0 holds one root segment per tree
// (parent code -(t+2) for tree t), and the same level kernels split all of
// them together.  A fixed number of levels is enqueued (no host wait, so the
// sequence can be captured in a graph); at the last level every segment that
// could still split is handed to the finisher list instead.  Finisher
// segment [st, en) owns node slots [st, en) and puts its root (always an
// internal node: the segment could split) in slot en - 1, so its parent is
// linked here; level nodes are numbered from node_off on.

template <int DC>
__global__ void k_forest_init(int ntrees, const int *__restrict__ t_start, const int *__restrict__ t_end,
                              const int *__restrict__ t_box, int node_off, Segs cur, int *__restrict__ ctl) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t == 0) {
        for (int w = 0; w < CTL_WORDS; ++w) ctl[w] = 0;
        ctl[CTL_S] = ntrees;
        ctl[CTL_NB] = node_off;
    }
    if (t >= ntrees) return;
    cur.start[t] = t_start[t];
    cur.end[t] = t_end[t];
    cur.parent[t] = -(t + 2);
    cur.side[t] = 0;
    cur.depth[t] = 0;
#pragma unroll
    for (int d = 0; d < DC; ++d) {
        cur.lo[t * DC + d] = t_box[t * 2 * DC + d];
        cur.hi[t * DC + d] = t_box[t * 2 * DC + DC + d];
    }
}

template <int DC>
pg_status forest_levels_impl(const ForestArgs &fa, cudaStream_t s) {
    const int seg_cap = fa.seg_cap, fin_cap = fa.fin_cap;
    auto carve = [&](int *b, int cap) {
        Segs g;
        g.start = b; g.end = b + cap; g.parent = b + 2 * cap; g.side = b + 3 * cap;
        g.depth = b + 4 * cap; g.lo = b + 5 * cap; g.hi = b + (5 + DC) * cap;
        return g;
    };
    Segs cur = carve(fa.seg_a, seg_cap), nxt = carve(fa.seg_b, seg_cap), fin = carve(fa.fin, fin_cap);
    int *split_flag = fa.lvl;
    int *split_rank = split_flag + seg_cap;
    int *sdim = split_rank + seg_cap + 1;
    float *sval = reinterpret_cast<float *>(sdim + seg_cap);
    int *fin_flag = sdim + 2 * seg_cap;
    int *fin_rank = fin_flag + seg_cap;
    float4 *P = fa.P, *Q = fa.Q;
    int *seg_of = fa.seg_of, *seg_of_nx = fa.seg_of_nx;
    const int ntiles = std::max(1, ceil_div_i(fa.n, PT_TILE));
    k_forest_init<DC><<<ceil_div_i(fa.ntrees, BT), BT, 0, s>>>(fa.ntrees, fa.t_start, fa.t_end, fa.t_box,
                                                               fa.node_off, cur, fa.ctl);
    count_launch();
    for (int level = 0; level < fa.levels; ++level) {
        const int S_max = (int)std::min<int64_t>((int64_t)fa.ntrees << std::min(level, 30), seg_cap);
        const int thr = level == fa.levels - 1 ? INT_MAX : fa.fin_max;
        PG_TRY(level_segments<DC>(S_max, fa.ctl, cur, nxt, fa.leaf, thr, split_flag, split_rank, sdim, sval, fin_flag,
                                  fin_rank, fin, fa.nodes, fa.n_sdim, fa.n_sval, fa.n_range, fa.n_parent, fa.roots, 1,
                                  fa.scan_ws, s));
        const int *T = split_rank + S_max;
        unsigned *twords = fa.tiles + ntiles;
        k_part_tiles<DC><<<ntiles, PT_THREADS, 0, s>>>(fa.n, P, seg_of, split_flag, sdim, sval, T, fa.tiles, twords);
        k_part_carry<<<1, 1024, 0, s>>>(fa.tiles, ntiles, T, fa.ctl, fin_rank + S_max, level);
        k_part<DC><<<ntiles, PT_THREADS, 0, s>>>(fa.n, P, Q, seg_of, seg_of_nx, cur.start, cur.end, split_flag,
                                                 split_rank, fa.tiles, twords, nxt.start, nxt.end, nxt.lo, nxt.hi,
                                                 T);
        count_launch();
        count_launch();
        count_launch();
        PG_TRY(check_launch("forest level"));
        std::swap(P, Q);
        std::swap(seg_of, seg_of_nx);
        std::swap(cur, nxt);
    }
    return PG_OK;
}

template <int DC>
pg_status pack_impl(const float *src, const int32_t *rows, const int32_t *ids, int64_t n, int dim, float4 *out,
                    int *box, cudaStream_t s) {
    k_init_box<<<1, 64, 0, s>>>(box, box + DC, DC);
    count_launch();
    if (n > 0) {
        const int grid = std::max(1, std::min(ceil_div_i(n, BT), num_sms() * 4));
        k_pack<DC><<<grid, BT, 0, s>>>(src, rows, ids, n, dim, out, box, box + DC);
        count_launch();
    }
    return check_launch("pack");
}

}  // namespace

int64_t forest_words(int dc, int seg_cap, int fin_cap, int64_t n) {
    const int64_t ntiles = std::max<int64_t>(1, (n + PT_TILE - 1) / PT_TILE);
    return 2 * (int64_t)seg_cap * (5 + 2 * dc) + 6 * (int64_t)seg_cap + 2 + (int64_t)fin_cap * (5 + 2 * dc) +
           ntiles * (1 + PT_TW) + CTL_WORDS + scan_ws_words(seg_cap) + 64;
}

void forest_carve(ForestArgs &fa, int *words, int dc) {
    int *p = words;
    fa.seg_a = p; p += (size_t)fa.seg_cap * (5 + 2 * dc);
    fa.seg_b = p; p += (size_t)fa.seg_cap * (5 + 2 * dc);
    fa.lvl = p; p += 6 * (size_t)fa.seg_cap + 2;
    fa.fin = p; p += (size_t)fa.fin_cap * (5 + 2 * dc);
    fa.tiles = reinterpret_cast<unsigned *>(p);
    p += std::max<int64_t>(1, (fa.n + PT_TILE - 1) / PT_TILE) * (1 + PT_TW);
    fa.ctl = p; p += CTL_WORDS;
    fa.scan_ws = p;
}

ForestCtl forest_ctl() { return ForestCtl{CTL_NB, CTL_FIN, CTL_SCATTERS}; }

pg_status forest_levels(int dc, const ForestArgs &fa, cudaStream_t s) {
    switch (dc) {
        case 2: return forest_levels_impl<2>(fa, s);
        case 3: return forest_levels_impl<3>(fa, s);
        case 4: return forest_levels_impl<4>(fa, s);
        case 5: return forest_levels_impl<5>(fa, s);
        case 6: return forest_levels_impl<6>(fa, s);
        case 7: return forest_levels_impl<7>(fa, s);
        case 8: return forest_levels_impl<8>(fa, s);
        case 12: return forest_levels_impl<12>(fa, s);
        case 16: return forest_levels_impl<16>(fa, s);
        default: return fail(PG_EUNSUPPORTED, "dimension class");
    }
}

#define PG_DC_SWITCH(dc, CALL)                                   \
    switch (dc) {                                                \
        case 2: { constexpr int DCV = 2; CALL; } break;          \
        case 3: { constexpr int DCV = 3; CALL; } break;          \
        case 4: { constexpr int DCV = 4; CALL; } break;          \
        case 5: { constexpr int DCV = 5; CALL; } break;          \
        case 6: { constexpr int DCV = 6; CALL; } break;          \
        case 7: { constexpr int DCV = 7; CALL; } break;          \
        case 8: { constexpr int DCV = 8; CALL; } break;          \
        case 12: { constexpr int DCV = 12; CALL; } break;        \
        case 16: { constexpr int DCV = 16; CALL; } break;        \
        default: return fail(PG_EUNSUPPORTED, "dimension class"); \
    }

// Packs and builds in one go (the packed array is allocated here).
static pg_status build_from(const float *src, const int32_t *rows, const int32_t *ids, int64_t n, int dim,
                            int leaf, int rule, cudaStream_t s, pg_tree *t, bool allow_deferred) {
    const int dc = dim_class(dim);
    t->n = n;
    t->dim = dim;
    t->dc = dc;
    t->leaf_size = leaf;
    t->stream = s;
    t->live = n;
    if (n == 0) {
        t->root_ref = -1;
        t->root_cnt = -1;
        t->num_nodes = 0;
        t->depth = 0;
        return tree_upload_desc(t);
    }
    const int W = bucket_w(dc);
    float4 *packed = nullptr;
    PG_TRY(dalloc_n(&packed, (size_t)W * n, s));
    Scratch box;
    if (box.alloc(sizeof(int) * 2 * PG_MAX_DIM, s) != PG_OK) {
        dfree(packed, s);
        return PG_ENOMEM;
    }
    // Under stream capture nothing may wait on the host: the build is
    // enqueued device-driven and its host-side metadata read back later.
    bool deferred = false;
    if (allow_deferred) {
        cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(s, &cst) != cudaSuccess) {
            dfree(packed, s);
            return cuda_fail(cudaGetLastError(), "cudaStreamIsCapturing");
        }
        deferred = cst == cudaStreamCaptureStatusActive;
    }
    pg_status st = PG_OK;
    PG_DC_SWITCH(dc, st = pack_impl<DCV>(src, rows, ids, n, dim, packed, box.as<int>(), s));
    if (st != PG_OK) { dfree(packed, s); return st; }
    if (deferred) {   // root box, descriptor and finite check stay on the device
        PG_DC_SWITCH(dc, st = Builder<DCV>::run(packed, box.as<int>(), n, leaf, rule, s, t, true));
        if (st != PG_OK && t->bucket != packed) dfree(packed, s);
        return st;
    }
    int hbox[2 * PG_MAX_DIM];
    PG_TRY(read_small(hbox, box.as<int>(), sizeof(int) * 2 * dc, s));
    for (int c = 0; c < PG_MAX_DIM; ++c) { t->root_lo[c] = 0.f; t->root_hi[c] = 0.f; }
    for (int c = 0; c < dc; ++c) {
        int a = hbox[c], b = hbox[dc + c];
        a = a >= 0 ? a : (a ^ 0x7fffffff);
        b = b >= 0 ? b : (b ^ 0x7fffffff);
        float fa, fb;
        memcpy(&fa, &a, 4);
        memcpy(&fb, &b, 4);
        t->root_lo[c] = fa;
        t->root_hi[c] = fb;
        if (!std::isfinite(fa) || !std::isfinite(fb)) {
            dfree(packed, s);
            return fail(PG_EINVAL, "points must have finite coordinates");
        }
    }
    // builds of pg_tree_build (allow_deferred) leave the root record and the
    // descriptor to a kernel: the host does not wait for the finisher
    PG_DC_SWITCH(dc, st = Builder<DCV>::run(packed, box.as<int>(), n, leaf, rule, s, t, false, allow_deferred));
    if (st != PG_OK) {
        if (t->bucket != packed) dfree(packed, s);
        return st;
    }
    return t->meta_pending ? PG_OK : tree_upload_desc(t);
}

pg_status build_rows(const float *pts, int64_t n, int dim, int leaf, int rule, cudaStream_t s, pg_tree *t) {
    return build_from(pts, nullptr, nullptr, n, dim, leaf, rule, s, t, true);
}

pg_status build_gather(const float *store, const int32_t *ids, int64_t n, int dim, int leaf, cudaStream_t s,
                       pg_tree *t) {
    return build_from(store, ids, ids, n, dim, leaf, PG_SPLIT_SPATIAL, s, t, false);
}

pg_status tree_sync_meta(pg_tree *t) {
    if (!t->meta_pending) return PG_OK;
    int h[kTreeMetaWords];
    PG_TRY(read_small(h, t->meta, sizeof(h), t->stream));
    if (!h[5]) return fail(PG_ECUDA, "tree build: level count exceeded the depth cap");
    t->root_ref = h[0];
    t->root_cnt = h[1];
    t->depth = h[2];
    t->num_nodes = h[4] > 0 ? h[3] + (int)t->n : h[3];
    for (int c = 0; c < PG_MAX_DIM; ++c) {
        const bool in = c < t->dc;
        int a = in ? h[8 + c] : 0, b = in ? h[8 + PG_MAX_DIM + c] : 0;
        memcpy(&t->root_lo[c], &a, 4);
        memcpy(&t->root_hi[c], &b, 4);
        if (in && (!std::isfinite(t->root_lo[c]) || !std::isfinite(t->root_hi[c])))
            return fail(PG_EINVAL, "points must have finite coordinates");
    }
    t->meta_pending = false;
    return PG_OK;
}

TreeDesc tree_desc(const pg_tree *t) {
    TreeDesc d;
    memset(&d, 0, sizeof(d));
    d.bucket = t->bucket;
    d.nodes = t->nodes;
    d.parent = t->parent;
    d.leaf_parent = t->leaf_parent;
    d.root_ref = t->root_ref;
    d.root_cnt = t->root_cnt;
    for (int c = 0; c < PG_MAX_DIM; ++c) { d.root_lo[c] = t->root_lo[c]; d.root_hi[c] = t->root_hi[c]; }
    return d;
}

pg_status tree_upload_desc(pg_tree *t) {
    if (!t->desc) PG_TRY(dalloc_n(&t->desc, 1, t->stream));
    TreeDesc d = tree_desc(t);
    static_assert(sizeof(TreeDesc) <= kStoreSmallBytes && sizeof(TreeDesc) % 4 == 0, "descriptor size");
    PG_TRY(store_small(t->desc, &d, sizeof(d), t->stream));
    cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
    PG_CUDA(cudaStreamIsCapturing(t->stream, &cst));
    if (cst == cudaStreamCaptureStatusNone) PG_CUDA(cudaStreamSynchronize(t->stream));
    return PG_OK;
}

void tree_release(pg_tree *t) {
    cudaStream_t s = t->stream;
    dfree(t->bucket, s);
    dfree(t->nodes, s);
    dfree(t->split_dim, s);
    dfree(t->split_val, s);
    dfree(t->node_range, s);
    dfree(t->parent, s);
    dfree(t->leaf_parent, s);
    dfree(t->desc, s);
    dfree(t->meta, s);
    t->meta = nullptr;
    t->meta_pending = false;
    t->bucket = nullptr;
    t->nodes = nullptr;
    t->split_dim = nullptr;
    t->split_val = nullptr;
    t->node_range = nullptr;
    t->parent = nullptr;
    t->leaf_parent = nullptr;
    t->desc = nullptr;
}

}  // namespace pg
