// Batched multi-cloud k-NN (not in the paper; it batches the paper's per-tree
// build (Appendix A.1.1) and data-parallel k-NN (Appendix A.1.3) over many
// independent point clouds).
//
// One forward pass, all of it in one CUDA graph:
//   pack       every cloud into bucket entries (cloud regions 128-byte
//              aligned) with its tight box,
//   levels     the device-wide level kernels split all clouds' trees at once
//              (build.cu, forest mode) down to segments one block can finish,
//   persistent one launch; blocks take work items from an atomic counter:
//              first the finisher segments (each built by one block, in
//              shared memory), then query chunks of NT points of one
//              (pair, direction).  A query chunk waits (bounded) until every
//              segment of its two clouds is finished, so queries of finished
//              clouds overlap the remaining builds.  Every finisher item
//              precedes every query item and a block only waits after all
//              finisher items have been taken by running blocks, so the waits
//              always end; a wait that exceeds its bound sets a status word.
#pragma once

#include "cta_build.cuh"
#include "cta_build_smem.cuh"
#include "knn_kernel.cuh"

namespace pg {

struct BWork {
    int pair, dir, start;   // query chunk: pair, direction (0: a -> b), first position
    int pad;
};

struct CloudMeta {
    int off;    // first bucket position (multiple of 8)
    int n;
    int row0;   // first row in the caller's array
    int src;    // 0: array a, 1: array b
};

// Per-call arguments (device memory, refreshed before each graph launch).
struct BArgs {
    const float *a, *b;
    int32_t *idx_ab, *idx_ba;
    float *dist_ab, *dist_ba;
    long long wait_limit;    // spins (about 100 ns each) before a query gives up
    int skip_publish;        // test hook: finished clouds are never published
};

// Everything else the kernels of one plan read (fixed per plan).
struct BDev {
    const BWork *items;
    int nquery;
    int *counter, *status;
    const int *ctl;
    int ctl_nb, ctl_fin, ctl_scat;
    const int *fin;          // finisher list: start, end, parent, side, depth, lo, hi
    int fin_cap;
    const CloudMeta *meta;
    const int *cl_start;     // first position per cloud (ascending)
    const int *cl_box;       // per cloud: DC lows, DC highs (order-preserving ints)
    int ncl;
    int *roots;              // per cloud: root reference, count
    int *pending, *ready;
    float4 *P, *Q;
    float4 *nodes;
    int *sdim;
    float *sval;
    int2 *range;
    int *parent;
    int *pool;               // scratch for segments larger than shared memory
    long long pool_cap;
    long long *pool_top;
    float *partial;
    int dim, k, leaf, ns, sc;
};

constexpr int BATCH_NT = 256;
constexpr long long kWaitLimit = 20000000;   // default: x ~100 ns sleeps, about two seconds

__device__ __forceinline__ int ld_acquire(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Cloud holding bucket position pos: the last c with cl_start[c] <= pos.
__device__ __forceinline__ int cloud_of(const int *cl_start, int ncl, int pos) {
    int lo = 0, hi = ncl;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (cl_start[mid] <= pos) lo = mid; else hi = mid;
    }
    return lo;
}

// Pack all clouds (positions [0, npoints)): entry = coordinates zero padded to
// DC, row within its cloud at word DC; gap positions get tree -1.  Cloud
// boxes by warp-aggregated atomics.
template <int DC>
__global__ void __launch_bounds__(256) k_bpack(const BArgs *__restrict__ args, const CloudMeta *__restrict__ meta,
                                               const int *__restrict__ cl_start, int ncl, int npoints, int dim,
                                               float4 *__restrict__ P, int *__restrict__ seg_of,
                                               int *__restrict__ cl_box) {
    constexpr int W = bucket_w(DC);
    const int lane = threadIdx.x & 31;
    const float *A = args->a, *B = args->b;
    for (int base = blockIdx.x * blockDim.x; base < npoints; base += gridDim.x * blockDim.x) {
        const int p = base + threadIdx.x;
        int c = -1;
        float v[4 * W];
#pragma unroll
        for (int x = 0; x < 4 * W; ++x) v[x] = 0.f;
        if (p < npoints) {
            const int cc = cloud_of(cl_start, ncl, p);
            const CloudMeta m = meta[cc];
            const int row = p - m.off;
            if (row < m.n) {
                c = cc;
                const float *src = (m.src == 0 ? A : B) + (size_t)(m.row0 + row) * dim;
#pragma unroll
                for (int d = 0; d < DC; ++d)
                    if (d < dim) v[d] = src[d];
                v[DC] = __int_as_float(row);
            }
#pragma unroll
            for (int x = 0; x < W; ++x)
                P[(size_t)p * W + x] = make_float4(v[4 * x], v[4 * x + 1], v[4 * x + 2], v[4 * x + 3]);
            seg_of[p] = c;
        }
        unsigned active = __ballot_sync(0xffffffffu, c >= 0);
        while (active) {
            const int leader = __ffs(active) - 1;
            const int key = __shfl_sync(0xffffffffu, c, leader);
            const bool mine = c == key;
            const unsigned grp = __ballot_sync(0xffffffffu, mine);
#pragma unroll
            for (int d = 0; d < DC; ++d) {
                const int e = f2o(v[d]);
                const int lo = __reduce_min_sync(0xffffffffu, mine ? e : INT_MAX);
                const int hi = __reduce_max_sync(0xffffffffu, mine ? e : INT_MIN);
                if (lane == leader) {
                    atomicMin(&cl_box[key * 2 * DC + d], lo);
                    atomicMax(&cl_box[key * 2 * DC + DC + d], hi);
                }
            }
            active &= ~grp;
        }
    }
}

template <int DC>
__global__ void k_bbox_init(int *cl_box, int ncl) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x < ncl * 2 * DC) cl_box[x] = (x % (2 * DC)) < DC ? 0x7f800000 : (int)0x807fffffu;
}

template <int DC, int KC>
__global__ void __launch_bounds__(BATCH_NT, KC <= 16 ? 4 : 2) k_batched(const BArgs *__restrict__ args, BDev D) {
    constexpr int NT = BATCH_NT;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_item;
    __shared__ int s_w[33];
    __shared__ long long s_pool;
    __shared__ TreeDesc s_desc;
    __shared__ float s_red[NT / 32];
    __shared__ int s_src_off, s_src_n, s_src_row0, s_fail;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const BArgs A = *args;
    // written by the level kernels that ran before this launch
    const int nfin = D.ctl[D.ctl_fin];
    const bool odd = D.ctl[D.ctl_scat] & 1;
    float4 *Pf = odd ? D.Q : D.P;   // buffer holding the final order
    float4 *Qf = odd ? D.P : D.Q;
    const int fc = D.fin_cap;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(D.counter, 1);
        __syncthreads();
        const int it = s_item;
        __syncthreads();
        if (it >= nfin + D.nquery) break;
        if (it < nfin) {
            // ------------------------------------------------- finisher segment
            const int st = D.fin[it], en = D.fin[fc + it];
            const int par = D.fin[2 * fc + it], side = D.fin[3 * fc + it], dep = D.fin[4 * fc + it];
            const int *lo = D.fin + 5 * fc + (size_t)it * DC;
            const int *hi = D.fin + (5 + DC) * (size_t)fc + (size_t)it * DC;
            const int code = par >= 0 ? 2 * par + side : -1;
            const int c = cloud_of(D.cl_start, D.ncl, st);
            if (en - st <= D.ns) {
                cta_build_smem<DC, NT>(Pf, st, en, lo, hi, smem, D.ns, D.sc, D.leaf, st, D.nodes, D.sdim, D.sval,
                                       D.range, dep, D.parent, nullptr, code, en - 1);
            } else {
                const long long words = (cta_scratch_words(en - st, D.leaf, DC) + 31) / 32 * 32;
                if (threadIdx.x == 0) s_pool = atomicAdd((unsigned long long *)D.pool_top, (unsigned long long)words);
                __syncthreads();
                if (s_pool + words <= D.pool_cap) {
                    cta_build_tree<DC, NT>(Pf, Qf, st, en, lo, hi, D.pool + s_pool, D.leaf, st, D.nodes, D.sdim,
                                           D.sval, D.range, s_w, dep, D.parent, nullptr, code, en - 1);
                } else if (threadIdx.x == 0) {
                    // out of scratch (the pool is sized so this cannot happen):
                    // the root becomes one leaf over the whole segment, still exact
                    int *ref = par >= 0 ? reinterpret_cast<int *>(D.nodes + (size_t)par * node_w(DC)) + 4 * DC + 2 * side
                                        : D.roots + 2 * c;
                    ref[0] = st;
                    ref[1] = en - st;
                    atomicExch(D.status, 2);
                }
            }
            __threadfence();
            __syncthreads();
            if (threadIdx.x == 0 && atomicSub(&D.pending[c], 1) == 1 && !A.skip_publish) atomicExch(&D.ready[c], 1);
        } else {
            // ------------------------------------------------------ query chunk
            const int q = it - nfin;
            const BWork w = D.items[q];
            const int src = 2 * w.pair + w.dir, dst = 2 * w.pair + 1 - w.dir;
            if (threadIdx.x == 0) {
                int fail = 0;
                for (int cl = 0; cl < 2 && !fail; ++cl) {
                    const int *f = &D.ready[cl == 0 ? src : dst];
                    long long spins = 0;
                    while (ld_acquire(f) == 0) {
                        if (++spins > A.wait_limit) { fail = 1; break; }
                        __nanosleep(100);
                    }
                }
                s_fail = fail;
                if (fail) atomicExch(D.status, 1);
                s_desc.bucket = Pf;
                s_desc.nodes = D.nodes;
                s_desc.parent = nullptr;
                s_desc.leaf_parent = nullptr;
                s_desc.root_ref = __ldcg(&D.roots[2 * dst]);
                s_desc.root_cnt = __ldcg(&D.roots[2 * dst + 1]);
#pragma unroll
                for (int d = 0; d < PG_MAX_DIM; ++d) {
                    s_desc.root_lo[d] = d < DC ? o2f(__ldcg(&D.cl_box[dst * 2 * DC + d])) : 0.f;
                    s_desc.root_hi[d] = d < DC ? o2f(__ldcg(&D.cl_box[dst * 2 * DC + DC + d])) : 0.f;
                }
                s_src_off = D.meta[src].off;
                s_src_n = D.meta[src].n;
                s_src_row0 = D.meta[src].row0;
            }
            __syncthreads();
            float part = 0.f;
            if (!s_fail) {
                const int pos = w.start + threadIdx.x;
                const bool valid = pos < s_src_n;
                float qp[DC];
                unsigned qid = 0;
#pragma unroll
                for (int d = 0; d < DC; ++d) qp[d] = 0.f;
                if (valid) load_point<DC, false>(Pf, (int64_t)s_src_off + pos, qp, qid);
                KList<KC> L;
                L.init(D.k);
                search_tree_packet<DC, KC, false>(s_desc, qp, valid, lane, L);
                if (valid) {
                    const int64_t row = (int64_t)s_src_row0 + qid;
                    int32_t *oi = (w.dir == 0 ? A.idx_ab : A.idx_ba) + row * D.k;
                    float *od = w.dir == 0 ? A.dist_ab : A.dist_ba;
                    if (od) od += row * D.k;
#pragma unroll
                    for (int j = 0; j < KC; ++j) {
                        if (j >= KC - D.k) {
                            const int o = j - (KC - D.k);
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
                D.partial[q] = t;
            }
            __syncthreads();
        }
    }
}

}  // namespace pg

#define PG_BATCHED_CASE(DCN, KCN)                                                                          \
    case KCN:                                                                                              \
        if (smem) cudaFuncSetAttribute(k_batched<DCN, KCN>, cudaFuncAttributeMaxDynamicSharedMemorySize,    \
                                       (int)smem);                                                         \
        if (grid <= 0) {                                                                                   \
            int nb = 0;                                                                                    \
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batched<DCN, KCN>, BATCH_NT, smem);      \
            return nb > 0 ? nb : 1;                                                                        \
        }                                                                                                  \
        k_batched<DCN, KCN><<<grid, BATCH_NT, smem, s>>>(args, D);                                          \
        break;

// batched_launch_dcN(grid > 0): launch the persistent kernel; grid <= 0: set
// its shared-memory limit and return the resident blocks per SM.
// batched_pack_dcN: box init + pack of one forward pass.
#define PG_DEFINE_BATCHED_LAUNCH(DCN)                                                                      \
    namespace pg {                                                                                         \
    int batched_launch_dc##DCN(int grid, size_t smem, const BArgs *args, const BDev &D, cudaStream_t s) {  \
        switch (k_class(D.k)) {                                                                            \
            PG_BATCHED_CASE(DCN, 1)                                                                        \
            PG_BATCHED_CASE(DCN, 2)                                                                        \
            PG_BATCHED_CASE(DCN, 4)                                                                        \
            PG_BATCHED_CASE(DCN, 8)                                                                        \
            PG_BATCHED_CASE(DCN, 10)                                                                       \
            PG_BATCHED_CASE(DCN, 16)                                                                       \
            PG_BATCHED_CASE(DCN, 32)                                                                       \
            PG_BATCHED_CASE(DCN, 64)                                                                       \
            default: return -1;                                                                            \
        }                                                                                                  \
        count_launch();                                                                                    \
        return 0;                                                                                          \
    }                                                                                                      \
    void batched_pack_dc##DCN(const BArgs *args, const CloudMeta *meta, const int *cl_start, int ncl,      \
                              int npoints, int dim, float4 *P, int *seg_of, int *cl_box, cudaStream_t s) { \
        k_bbox_init<DCN><<<ceil_div_i((int64_t)ncl * 2 * DCN, 256), 256, 0, s>>>(cl_box, ncl);            \
        const int grid = std::max(1, std::min(ceil_div_i(npoints, 256), num_sms() * 8));                  \
        k_bpack<DCN><<<grid, 256, 0, s>>>(args, meta, cl_start, ncl, npoints, dim, P, seg_of, cl_box);     \
        count_launch();                                                                                    \
        count_launch();                                                                                    \
    }                                                                                                      \
    }
