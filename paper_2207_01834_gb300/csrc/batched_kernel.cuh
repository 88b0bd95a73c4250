// Batched multi-cloud k-NN in one persistent launch (not in the paper; it
// batches the paper's per-tree build (Appendix A.1.1) and data-parallel k-NN
// (Appendix A.1.3) over many independent point clouds).
//
// Work queue: one item per cloud build (largest clouds first), then one item
// per chunk of NT queries of one (pair, direction).  Persistent blocks take
// items with an atomic counter.  A build item packs the cloud, builds its
// kd-tree with the block-scope builder and publishes a ready flag; a query
// item waits (bounded) for the flags of its two clouds, then runs the warp
// packet traversal with the source cloud's points in tree order as queries.
// Every build item precedes every query item in the queue and a block only
// waits after all builds have been taken by running blocks, so the waits
// always end; a wait that exceeds its bound sets a status word instead.
#pragma once

#include "cta_build.cuh"
#include "knn_kernel.cuh"

namespace pg {

struct BWork {
    int type;    // 0 build cloud `a`; 1 query chunk: pair a, direction b, first position c
    int a, b, c;
};

struct CloudMeta {
    long long scratch_off;   // ints into the scratch arena
    int off;                 // first bucket position (multiple of 8)
    int n;
    int node_base;           // first node index (multiple of 8)
    int row0;                // first row in the caller's array
    int src;                 // 0: array a, 1: array b
    int root_ref, root_cnt;
    float lo[PG_MAX_DIM], hi[PG_MAX_DIM];
};

struct BArgs {
    const float *a, *b;
    int32_t *idx_ab, *idx_ba;
    float *dist_ab, *dist_ba;
    long long wait_limit;    // spins (about 100 ns each) before a query gives up
    int skip_publish;        // test hook: builders never set their ready flag
};

constexpr int BATCH_NT = 256;
constexpr long long kWaitLimit = 20000000;   // default: x ~100 ns sleeps, about two seconds

__device__ __forceinline__ int ld_acquire(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

template <int DC, int KC>
__global__ void __launch_bounds__(BATCH_NT) k_batched(const BArgs *__restrict__ args, const BWork *__restrict__ items,
                                                      int nitems, int nbuild, int *counter, CloudMeta *meta,
                                                      int *ready, int *status, float4 *P, float4 *Q, float4 *nodes,
                                                      int *n_sdim, float *n_sval, int2 *n_range, int *scratch,
                                                      float *partial, int dim, int k, int leaf) {
    constexpr int NT = BATCH_NT;
    constexpr int W = bucket_w(DC);
    __shared__ int s_item;
    __shared__ int s_w[33];
    __shared__ int s_lo[PG_MAX_DIM], s_hi[PG_MAX_DIM];
    __shared__ TreeDesc s_desc;
    __shared__ float s_red[NT / 32];
    __shared__ int s_src_off, s_src_n, s_src_row0, s_fail;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const BArgs A = *args;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int it = s_item;
        __syncthreads();
        if (it >= nitems) break;
        const BWork w = items[it];
        if (w.type == 0) {
            // ---------------------------------------------------------- build
            const int c = w.a;
            const int off = meta[c].off, n = meta[c].n, row0 = meta[c].row0;
            const float *rows = (meta[c].src == 0 ? A.a : A.b) + (size_t)row0 * dim;
            float lo[DC], hi[DC];
#pragma unroll
            for (int d = 0; d < DC; ++d) { lo[d] = __int_as_float(0x7f800000); hi[d] = -lo[d]; }
            if (threadIdx.x < DC) { s_lo[threadIdx.x] = 0x7f800000; s_hi[threadIdx.x] = (int)0x807fffffu; }
            __syncthreads();
            for (int i = threadIdx.x; i < n; i += NT) {
                float v[4 * W];
#pragma unroll
                for (int x = 0; x < 4 * W; ++x) v[x] = 0.f;
#pragma unroll
                for (int d = 0; d < DC; ++d)
                    if (d < dim) v[d] = rows[(size_t)i * dim + d];
                v[DC] = __int_as_float(i);
#pragma unroll
                for (int x = 0; x < W; ++x)
                    P[(size_t)(off + i) * W + x] = make_float4(v[4 * x], v[4 * x + 1], v[4 * x + 2], v[4 * x + 3]);
#pragma unroll
                for (int d = 0; d < DC; ++d) { lo[d] = fminf(lo[d], v[d]); hi[d] = fmaxf(hi[d], v[d]); }
            }
#pragma unroll
            for (int d = 0; d < DC; ++d) {
                const int a = __reduce_min_sync(0xffffffffu, f2o(lo[d]));
                const int b = __reduce_max_sync(0xffffffffu, f2o(hi[d]));
                if (lane == 0) { atomicMin(&s_lo[d], a); atomicMax(&s_hi[d], b); }
            }
            __syncthreads();
            const CtaTree r = cta_build_tree<DC, NT>(P, Q, off, off + n, s_lo, s_hi, scratch + meta[c].scratch_off,
                                                     leaf, meta[c].node_base, nodes, n_sdim, n_sval, n_range, s_w);
            if (threadIdx.x == 0) {
                meta[c].root_ref = r.root_ref;
                meta[c].root_cnt = r.root_cnt;
#pragma unroll
                for (int d = 0; d < PG_MAX_DIM; ++d) {
                    meta[c].lo[d] = d < DC ? o2f(s_lo[d]) : 0.f;
                    meta[c].hi[d] = d < DC ? o2f(s_hi[d]) : 0.f;
                }
            }
            __threadfence();
            __syncthreads();
            if (threadIdx.x == 0 && !A.skip_publish) atomicExch(&ready[c], 1);
        } else {
            // ---------------------------------------------------------- query
            const int pair = w.a, dir = w.b, start = w.c;
            const int src = 2 * pair + dir, dst = 2 * pair + 1 - dir;
            if (threadIdx.x == 0) {
                int fail = 0;
                for (int cl = 0; cl < 2 && !fail; ++cl) {
                    const int *f = &ready[cl == 0 ? src : dst];
                    long long spins = 0;
                    while (ld_acquire(f) == 0) {
                        if (++spins > A.wait_limit) { fail = 1; break; }
                        __nanosleep(100);
                    }
                }
                s_fail = fail;
                if (fail) atomicExch(status, 1);
                const CloudMeta *md = meta + dst;
                s_desc.bucket = P;
                s_desc.nodes = nodes;
                s_desc.root_ref = __ldcg(&md->root_ref);
                s_desc.root_cnt = __ldcg(&md->root_cnt);
#pragma unroll
                for (int d = 0; d < PG_MAX_DIM; ++d) {
                    s_desc.root_lo[d] = __ldcg(&md->lo[d]);
                    s_desc.root_hi[d] = __ldcg(&md->hi[d]);
                }
                s_src_off = __ldcg(&meta[src].off);
                s_src_n = __ldcg(&meta[src].n);
                s_src_row0 = __ldcg(&meta[src].row0);
            }
            __syncthreads();
            float part = 0.f;
            if (!s_fail) {
                const int pos = start + threadIdx.x;
                const bool valid = pos < s_src_n;
                float q[DC];
                unsigned qid = 0;
#pragma unroll
                for (int d = 0; d < DC; ++d) q[d] = 0.f;
                if (valid) load_point<DC, false>(P, (int64_t)s_src_off + pos, q, qid);
                KList<KC> L;
                L.init(k);
                search_tree_packet<DC, KC, false>(s_desc, q, valid, lane, L);
                if (valid) {
                    const int64_t row = (int64_t)s_src_row0 + qid;
                    int32_t *oi = (dir == 0 ? A.idx_ab : A.idx_ba) + row * k;
                    float *od = dir == 0 ? A.dist_ab : A.dist_ba;
                    if (od) od += row * k;
#pragma unroll
                    for (int j = 0; j < KC; ++j) {
                        if (j >= KC - k) {
                            const int o = j - (KC - k);
                            const bool pad = L.idx(j) == DEAD_ID;
                            oi[o] = pad ? -1 : (int32_t)L.idx(j);
                            if (od) od[o] = L.dist(j);
                            if (!pad) part += L.dist(j);
                        }
                    }
                }
            }
            // fixed-order block sum of the chunk's distances
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
            if (lane == 0) s_red[warp] = part;
            __syncthreads();
            if (threadIdx.x == 0) {
                float t = 0.f;
                for (int x = 0; x < NT / 32; ++x) t += s_red[x];
                partial[it - nbuild] = t;
            }
            __syncthreads();
        }
    }
}

}  // namespace pg

#define PG_BATCHED_CASE(DCN, KCN)                                                                          \
    case KCN:                                                                                              \
        k_batched<DCN, KCN><<<grid, BATCH_NT, 0, s>>>(args, items, nitems, nbuild, counter, meta, ready,   \
                                                      status, P, Q, nodes, sdim, sval, range, scratch,     \
                                                      partial, dim, k, leaf);                              \
        break;

#define PG_DEFINE_BATCHED_LAUNCH(DCN)                                                                      \
    namespace pg {                                                                                         \
    pg_status batched_launch_dc##DCN(int grid, const BArgs *args, const BWork *items, int nitems,          \
                                     int nbuild, int *counter, CloudMeta *meta, int *ready, int *status,   \
                                     float4 *P, float4 *Q, float4 *nodes, int *sdim, float *sval,          \
                                     int2 *range, int *scratch, float *partial, int dim, int k, int leaf,  \
                                     cudaStream_t s) {                                                     \
        switch (k_class(k)) {                                                                              \
            PG_BATCHED_CASE(DCN, 1)                                                                        \
            PG_BATCHED_CASE(DCN, 2)                                                                        \
            PG_BATCHED_CASE(DCN, 4)                                                                        \
            PG_BATCHED_CASE(DCN, 8)                                                                        \
            PG_BATCHED_CASE(DCN, 10)                                                                       \
            PG_BATCHED_CASE(DCN, 16)                                                                       \
            PG_BATCHED_CASE(DCN, 32)                                                                       \
            PG_BATCHED_CASE(DCN, 64)                                                                       \
            default: return fail(PG_EINVAL, "k out of range");                                             \
        }                                                                                                  \
        count_launch();                                                                                    \
        return check_launch("batched persistent kernel");                                                  \
    }                                                                                                      \
    int batched_blocks_per_sm_dc##DCN(int k) {                                                             \
        int nb = 0;                                                                                        \
        switch (k_class(k)) {                                                                              \
            case 1: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batched<DCN, 1>, BATCH_NT, 0); break;   \
            case 2: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batched<DCN, 2>, BATCH_NT, 0); break;   \
            case 4: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batched<DCN, 4>, BATCH_NT, 0); break;   \
            case 8: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batched<DCN, 8>, BATCH_NT, 0); break;   \
            case 10: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batched<DCN, 10>, BATCH_NT, 0); break; \
            case 16: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batched<DCN, 16>, BATCH_NT, 0); break; \
            case 32: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batched<DCN, 32>, BATCH_NT, 0); break; \
            default: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batched<DCN, 64>, BATCH_NT, 0); break; \
        }                                                                                                  \
        return nb > 0 ? nb : 1;                                                                            \
    }                                                                                                      \
    }
