// Host side of the batched multi-cloud Chamfer path: plan (layout, work queue,
// scratch), a CUDA graph that replays {reset counters, persistent kernel,
// per-pair loss sums} per call, and the deterministic backward twin.
#include <algorithm>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <vector>

#include "batched_kernel.cuh"
#include "internal.h"
#include "sort.h"

namespace pg {

#define PG_BDECL(DCN)                                                                                      \
    int batched_launch_dc##DCN(int, size_t, const BArgs *, const BDev &, cudaStream_t);                    \
    void batched_pack_dc##DCN(const BArgs *, const CloudMeta *, const int *, int, int, int, float4 *, int *, \
                              int *, cudaStream_t);
PG_BDECL(2) PG_BDECL(3) PG_BDECL(4) PG_BDECL(5) PG_BDECL(6) PG_BDECL(7) PG_BDECL(8) PG_BDECL(12) PG_BDECL(16)
#undef PG_BDECL

namespace {

constexpr int BT = 256;

__global__ void k_pair_loss(const int *__restrict__ first, const float *__restrict__ partial, int npairs,
                            float *__restrict__ loss) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npairs) return;
    float t = 0.f;
    for (int x = first[i]; x < first[i + 1]; ++x) t += partial[x];
    loss[i] = t;
}

// row -> pair index by binary search over the pair offsets
__global__ void k_row_pair(const long long *__restrict__ off, int npairs, int64_t rows, int *__restrict__ pair) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    int lo = 0, hi = npairs;   // off[lo] <= r < off[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= r) lo = mid; else hi = mid;
    }
    pair[r] = lo;
}

// Sort keys of one direction: the global row of the neighbour in the other
// array (or `sentinel` for padding).
__global__ void k_bkeys(const int32_t *__restrict__ idx, int64_t rows, int k, const int *__restrict__ row_pair,
                        const long long *__restrict__ other_off, uint32_t sentinel, uint32_t *__restrict__ keys) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= rows * k) return;
    const int t = idx[p];
    const int pr = row_pair[p / k];
    const long long lim = other_off[pr + 1] - other_off[pr];
    keys[p] = (t >= 0 && t < lim) ? (uint32_t)(other_off[pr] + t) : sentinel;
}

__global__ void k_bbounds(const uint32_t *__restrict__ sk, int64_t P, uint32_t n, int *__restrict__ lo,
                          int *__restrict__ hi) {
    const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= P) return;
    const uint32_t key = sk[x];
    if (key >= n) return;
    if (x == 0 || sk[x - 1] != key) lo[key] = (int)x;
    if (x == P - 1 || sk[x + 1] != key) hi[key] = (int)(x + 1);
}

// Gradient of sum_i g_i loss_i for the rows of one array X (the other array
// is Y):  direct part from X's own k neighbours in Y, then the contributions
// of every Y row that selected this X row, in ascending (row, slot) order.
// A row selected more than kHeavy times (a hub) is split into chunks of
// kChunk entries: one warp sums a chunk (lane l takes entries l, l+32, ... in
// order, then a fixed butterfly), and the row adds its chunk sums in chunk
// order.  Every order is fixed, so the result is the same on every run, and
// no warp is held back by one hub.
constexpr int kHeavy = 64;
constexpr int kChunk = 256;

template <int DC>
__global__ void k_bgrad(const float *__restrict__ X, int64_t nx, const float *__restrict__ Y, int dim, int k,
                        const int32_t *__restrict__ idx_xy, const int *__restrict__ row_pair_x,
                        const int *__restrict__ row_pair_y, const long long *__restrict__ off_y,
                        const float *__restrict__ g, const uint32_t *__restrict__ sv_yx, const int *__restrict__ lo,
                        const int *__restrict__ hi, float *__restrict__ gx, int2 *__restrict__ heavy,
                        int *__restrict__ nheavy, int *__restrict__ chunk_row, int *__restrict__ nchunks) {
    const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= nx) return;
    float p[DC], acc[DC];
#pragma unroll
    for (int c = 0; c < DC; ++c) {
        p[c] = c < dim ? X[x * dim + c] : 0.f;
        acc[c] = 0.f;
    }
    const int pr = row_pair_x[x];
    const float w = 2.f * g[pr];
    const long long base = off_y[pr], lim = off_y[pr + 1] - base;
    for (int j = 0; j < k; ++j) {
        const int t = idx_xy[x * k + j];
        if (t < 0 || t >= lim) continue;
        const int64_t yr = base + t;
#pragma unroll
        for (int c = 0; c < DC; ++c)
            if (c < dim) acc[c] = __fmaf_rn(w, __fsub_rn(p[c], Y[yr * dim + c]), acc[c]);
    }
    const int e0 = lo[x], e1 = hi[x];
    if (e1 - e0 > kHeavy) {
        // list positions and chunk slots do not affect any sum
        const int nch = (e1 - e0 + kChunk - 1) / kChunk;
        const int first = atomicAdd(nchunks, nch);
        const int h = atomicAdd(nheavy, 1);
        heavy[h] = make_int2((int)x, first);
        for (int c = 0; c < nch; ++c) chunk_row[first + c] = h;
    } else {
        for (int e = e0; e < e1; ++e) {
            const uint32_t v = sv_yx[e];
            const int64_t yr = v / (uint32_t)k;
            const float wy = -2.f * g[row_pair_y[yr]];
#pragma unroll
            for (int c = 0; c < DC; ++c)
                if (c < dim) acc[c] = __fmaf_rn(wy, __fsub_rn(Y[yr * dim + c], p[c]), acc[c]);
        }
    }
#pragma unroll
    for (int c = 0; c < DC; ++c)
        if (c < dim) gx[x * dim + c] = acc[c];
}

// One warp per chunk of a hub row: the chunk's sum goes to part[slot].
template <int DC>
__global__ void k_bgrad_chunk(const float *__restrict__ X, const float *__restrict__ Y, int dim, int k,
                              const int *__restrict__ row_pair_y, const float *__restrict__ g,
                              const uint32_t *__restrict__ sv_yx, const int *__restrict__ lo,
                              const int *__restrict__ hi, const int2 *__restrict__ heavy,
                              const int *__restrict__ chunk_row, const int *__restrict__ nchunks,
                              float *__restrict__ part) {
    const int lane = threadIdx.x & 31;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int cnt = *nchunks;
    for (int64_t slot = wid; slot < cnt; slot += nw) {
        const int2 hr = heavy[chunk_row[slot]];
        const int64_t x = hr.x;
        const int e0 = lo[x] + (int)(slot - hr.y) * kChunk, e1 = min(hi[x], e0 + kChunk);
        float p[DC], acc[DC];
#pragma unroll
        for (int c = 0; c < DC; ++c) {
            p[c] = c < dim ? X[x * dim + c] : 0.f;
            acc[c] = 0.f;
        }
        for (int e = e0 + lane; e < e1; e += 32) {
            const uint32_t v = sv_yx[e];
            const int64_t yr = v / (uint32_t)k;
            const float wy = -2.f * g[row_pair_y[yr]];
#pragma unroll
            for (int c = 0; c < DC; ++c)
                if (c < dim) acc[c] = __fmaf_rn(wy, __fsub_rn(Y[yr * dim + c], p[c]), acc[c]);
        }
#pragma unroll
        for (int c = 0; c < DC; ++c) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc[c] = __fadd_rn(acc[c], __shfl_xor_sync(0xffffffffu, acc[c], o));
        }
        if (lane == 0) {
#pragma unroll
            for (int c = 0; c < DC; ++c) part[slot * DC + c] = acc[c];
        }
    }
}

// One thread per hub row: direct part (already in gx) + chunk sums in order.
template <int DC>
__global__ void k_bgrad_hubs(int dim, const int *__restrict__ lo, const int *__restrict__ hi,
                             const int2 *__restrict__ heavy, const int *__restrict__ nheavy,
                             const float *__restrict__ part, float *__restrict__ gx) {
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= *nheavy) return;
    const int2 hr = heavy[h];
    const int64_t x = hr.x;
    const int nch = (hi[x] - lo[x] + kChunk - 1) / kChunk;
    float acc[DC];
#pragma unroll
    for (int c = 0; c < DC; ++c) acc[c] = 0.f;
    for (int j = 0; j < nch; ++j) {
#pragma unroll
        for (int c = 0; c < DC; ++c) acc[c] = __fadd_rn(acc[c], part[(int64_t)(hr.y + j) * DC + c]);
    }
#pragma unroll
    for (int c = 0; c < DC; ++c)
        if (c < dim) gx[x * dim + c] = __fadd_rn(gx[x * dim + c], acc[c]);
}

inline int grid_of(int64_t n) { return std::max(1, ceil_div_i(n, BT)); }

constexpr size_t kBatchSmemBudget = 52 * 1024;    // finisher shared memory per block (leaves room for query occupancy)

__global__ void k_bpending(BDev D) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f < D.fin_cap && f < D.ctl[D.ctl_fin]) atomicAdd(&D.pending[cloud_of(D.cl_start, D.ncl, D.fin[f])], 1);
}
__global__ void k_bready(BDev D, const BArgs *__restrict__ args) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < D.ncl) D.ready[c] = (D.pending[c] == 0 && !args->skip_publish) ? 1 : 0;
}

struct Plan {
    int npairs = 0, dim = 0, k = 0, leaf = 0, dc = 2, ncl = 0;
    std::vector<long long> a_off, b_off;
    int64_t Na = 0, Nb = 0, npoints = 0;
    int nquery = 0, grid = 0, graph_kernels = 0;
    size_t smem = 0;
    cudaStream_t cap = nullptr;
    cudaGraphExec_t exec = nullptr;
    ForestArgs fa{};
    BDev D{};
    BArgs *args = nullptr;
    CloudMeta *meta = nullptr;
    int *cl_start = nullptr, *cl_end = nullptr, *cl_box = nullptr, *status = nullptr;
    int *first = nullptr;
    float *loss_dev = nullptr;
    std::vector<void *> owned;
    ~Plan() {
        if (exec) cudaGraphExecDestroy(exec);
        for (void *p : owned) cudaFree(p);
        if (cap) cudaStreamDestroy(cap);
    }
};

long long g_wait_limit = kWaitLimit;
int g_skip_publish = 0;

std::mutex g_plans_mu;
std::map<std::vector<long long>, std::unique_ptr<Plan>> g_plans;

template <class T>
pg_status plan_alloc(Plan &pl, T **p, size_t n) {
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, std::max<size_t>(n, 1) * sizeof(T));
    if (e != cudaSuccess) return cuda_fail(e, "batched plan allocation");
    pl.owned.push_back(q);
    *p = reinterpret_cast<T *>(q);
    return PG_OK;
}

#define PG_BSWITCH(dc, CALL)                                                                               \
    switch (dc) {                                                                                          \
        case 2: { CALL(2); } break;                                                                        \
        case 3: { CALL(3); } break;                                                                        \
        case 4: { CALL(4); } break;                                                                        \
        case 5: { CALL(5); } break;                                                                        \
        case 6: { CALL(6); } break;                                                                        \
        case 7: { CALL(7); } break;                                                                        \
        case 8: { CALL(8); } break;                                                                        \
        case 12: { CALL(12); } break;                                                                      \
        case 16: { CALL(16); } break;                                                                      \
        default: return fail(PG_EUNSUPPORTED, "dimension class");                                          \
    }

// Enqueue one forward pass (everything inside the captured graph).
pg_status enqueue_forward(Plan &pl, cudaStream_t s) {
    const BDev &D = pl.D;
    PG_CUDA(cudaMemsetAsync(D.pending, 0, sizeof(int) * (size_t)pl.ncl, s));
    PG_CUDA(cudaMemsetAsync(D.counter, 0, sizeof(int), s));
    PG_CUDA(cudaMemsetAsync(D.status, 0, sizeof(int), s));
    PG_CUDA(cudaMemsetAsync(D.pool_top, 0, sizeof(long long), s));
#define PG_PACK(DCN)                                                                                       \
    batched_pack_dc##DCN(pl.args, pl.meta, pl.cl_start, pl.ncl, (int)pl.npoints, pl.dim, pl.fa.P,            \
                         pl.fa.seg_of, pl.cl_box, s)
    PG_BSWITCH(pl.dc, PG_PACK)
#undef PG_PACK
    PG_TRY(forest_levels(pl.dc, pl.fa, s));
    k_bpending<<<grid_of(pl.fa.fin_cap), BT, 0, s>>>(D);
    k_bready<<<grid_of(pl.ncl), BT, 0, s>>>(D, pl.args);
    count_launch();
    count_launch();
    int r = 0;
#define PG_RUN(DCN) r = batched_launch_dc##DCN(pl.grid, pl.smem, pl.args, D, s)
    PG_BSWITCH(pl.dc, PG_RUN)
#undef PG_RUN
    if (r < 0) return fail(PG_EINVAL, "k out of range");
    PG_TRY(check_launch("batched persistent kernel"));
    k_pair_loss<<<grid_of(pl.npairs), BT, 0, s>>>(pl.first, D.partial, pl.npairs, pl.loss_dev);
    count_launch();
    return check_launch("batched loss");
}

pg_status make_plan(Plan &pl) {
    const int np = pl.npairs, dc = pl.dc;
    pl.ncl = 2 * np;
    std::vector<CloudMeta> meta(pl.ncl);
    std::vector<int> cl_start(pl.ncl), cl_end(pl.ncl);
    int64_t pos = 0, max_n = 1;
    for (int i = 0; i < np; ++i) {
        for (int side = 0; side < 2; ++side) {
            const int c = 2 * i + side;
            const std::vector<long long> &off = side == 0 ? pl.a_off : pl.b_off;
            const int64_t n = off[i + 1] - off[i];
            meta[c] = CloudMeta{(int)pos, (int)n, (int)off[i], side};
            cl_start[c] = (int)pos;
            cl_end[c] = (int)(pos + n);
            max_n = std::max(max_n, n);
            // 8-entry alignment keeps every cloud's buckets and finisher node
            // slots on their own 128-byte lines: a block never caches a line
            // that another cloud's finisher is still writing
            pos += (n + 7) / 8 * 8;
        }
    }
    pl.npoints = pos;
    // query work items: chunks of BATCH_NT points per (pair, direction)
    std::vector<BWork> items;
    std::vector<int> first(np + 1, 0);
    for (int i = 0; i < np; ++i) {
        first[i] = (int)items.size();
        for (int dir = 0; dir < 2; ++dir) {
            const int n = meta[2 * i + dir].n;
            for (int st = 0; st < n; st += BATCH_NT) items.push_back({i, dir, st, 0});
        }
    }
    first[np] = (int)items.size();
    pl.nquery = (int)items.size();
    // forest levels: enough for balanced splits of the largest cloud down to
    // one block's shared memory, plus a margin for clustered clouds
    const int ns = smem_build_points(dc, pl.leaf, kBatchSmemBudget);
    const int sc = smem_seg_cap(ns, pl.leaf);
    int levels = 1;
    while (((int64_t)ns << (levels - 1)) < max_n && levels < PG_DEPTH_CAP) ++levels;
    levels = std::min(levels + 6, PG_DEPTH_CAP + 1);
    ForestArgs &fa = pl.fa;
    fa.n = pl.npoints;
    fa.ntrees = pl.ncl;
    fa.leaf = pl.leaf;
    fa.fin_max = ns;
    fa.levels = levels;
    // level splits hold more than ns points each (at most npoints/(ns+1) per level)
    fa.seg_cap = (int)std::max<int64_t>(pl.ncl, 2 * (pl.npoints / (ns + 1)) + 2);
    fa.fin_cap = (int)(pl.npoints / (pl.leaf + 1) + pl.ncl + 1);
    fa.node_off = (int)pos;   // finisher segments own the slots of their positions
    const int64_t nnodes = pos + (int64_t)levels * (pl.npoints / (ns + 1) + 1) + 64;
    if (nnodes >= ((int64_t)1 << 31) || pl.npoints >= ((int64_t)1 << 31) - 64)
        return fail(PG_EINVAL, "batched: too many points");
    const int W4 = bucket_w(dc);
    PG_TRY(plan_alloc(pl, &fa.P, (size_t)pl.npoints * W4));
    PG_TRY(plan_alloc(pl, &fa.Q, (size_t)pl.npoints * W4));
    PG_TRY(plan_alloc(pl, &fa.seg_of, (size_t)pl.npoints));
    PG_TRY(plan_alloc(pl, &fa.seg_of_nx, (size_t)pl.npoints));
    PG_TRY(plan_alloc(pl, &fa.nodes, (size_t)nnodes * node_w(dc)));
    PG_TRY(plan_alloc(pl, &fa.n_sdim, (size_t)nnodes));
    PG_TRY(plan_alloc(pl, &fa.n_sval, (size_t)nnodes));
    PG_TRY(plan_alloc(pl, &fa.n_range, (size_t)nnodes));
    PG_TRY(plan_alloc(pl, &fa.n_parent, (size_t)nnodes));
    PG_TRY(plan_alloc(pl, &fa.roots, (size_t)(2 * pl.ncl)));
    int *fw = nullptr;
    PG_TRY(plan_alloc(pl, &fw, (size_t)forest_words(dc, fa.seg_cap, fa.fin_cap, fa.n)));
    forest_carve(fa, fw, dc);
    PG_TRY(plan_alloc(pl, &pl.cl_start, (size_t)pl.ncl));
    PG_TRY(plan_alloc(pl, &pl.cl_end, (size_t)pl.ncl));
    PG_TRY(plan_alloc(pl, &pl.cl_box, (size_t)pl.ncl * 2 * dc));
    fa.t_start = pl.cl_start;
    fa.t_end = pl.cl_end;
    fa.t_box = pl.cl_box;
    PG_TRY(plan_alloc(pl, &pl.meta, (size_t)pl.ncl));
    PG_TRY(plan_alloc(pl, &pl.args, 1));
    PG_TRY(plan_alloc(pl, &pl.first, (size_t)(np + 1)));
    PG_TRY(plan_alloc(pl, &pl.loss_dev, (size_t)np));
    BDev &D = pl.D;
    BWork *items_d = nullptr;
    PG_TRY(plan_alloc(pl, &items_d, (size_t)pl.nquery));
    D.items = items_d;
    D.nquery = pl.nquery;
    PG_TRY(plan_alloc(pl, &D.counter, 1));
    PG_TRY(plan_alloc(pl, &D.status, 1));
    pl.status = D.status;
    D.ctl = fa.ctl;
    const ForestCtl fcw = forest_ctl();
    D.ctl_nb = fcw.nb;
    D.ctl_fin = fcw.fin;
    D.ctl_scat = fcw.scatters;
    D.fin = fa.fin;
    D.fin_cap = fa.fin_cap;
    D.meta = pl.meta;
    D.cl_start = pl.cl_start;
    D.cl_box = pl.cl_box;
    D.ncl = pl.ncl;
    D.roots = fa.roots;
    PG_TRY(plan_alloc(pl, &D.pending, (size_t)pl.ncl));
    PG_TRY(plan_alloc(pl, &D.ready, (size_t)pl.ncl));
    D.P = fa.P;
    D.Q = fa.Q;
    D.nodes = fa.nodes;
    D.sdim = fa.n_sdim;
    D.sval = fa.n_sval;
    D.range = fa.n_range;
    D.parent = fa.n_parent;
    // scratch for finisher segments above ns points (only after the last
    // level): the sizes are disjoint parts of npoints, each above ns
    D.pool_cap = cta_scratch_words(pl.npoints, pl.leaf, dc) +
                 (pl.npoints / (ns + 1) + 1) * (cta_scratch_words(0, pl.leaf, dc) + 64);
    PG_TRY(plan_alloc(pl, &D.pool, (size_t)D.pool_cap));
    PG_TRY(plan_alloc(pl, &D.pool_top, 1));
    PG_TRY(plan_alloc(pl, &D.partial, (size_t)pl.nquery));
    D.dim = pl.dim;
    D.k = pl.k;
    D.leaf = pl.leaf;
    D.ns = ns;
    D.sc = sc;
    pl.smem = smem_build_bytes(ns, sc, dc);
    PG_CUDA(cudaMemcpy(pl.meta, meta.data(), sizeof(CloudMeta) * meta.size(), cudaMemcpyHostToDevice));
    PG_CUDA(cudaMemcpy(pl.cl_start, cl_start.data(), sizeof(int) * cl_start.size(), cudaMemcpyHostToDevice));
    PG_CUDA(cudaMemcpy(pl.cl_end, cl_end.data(), sizeof(int) * cl_end.size(), cudaMemcpyHostToDevice));
    PG_CUDA(cudaMemcpy(items_d, items.data(), sizeof(BWork) * items.size(), cudaMemcpyHostToDevice));
    PG_CUDA(cudaMemcpy(pl.first, first.data(), sizeof(int) * first.size(), cudaMemcpyHostToDevice));
    int per_sm = 0;
#define PG_OCC(DCN) per_sm = batched_launch_dc##DCN(0, pl.smem, pl.args, D, nullptr)
    PG_BSWITCH(dc, PG_OCC)
#undef PG_OCC
    if (per_sm <= 0) return fail(PG_EINVAL, "k out of range");
    pl.grid = num_sms() * per_sm;
    // capture the forward sequence once; calls only refresh the argument block
    PG_CUDA(cudaStreamCreateWithFlags(&pl.cap, cudaStreamNonBlocking));
    PG_CUDA(cudaStreamBeginCapture(pl.cap, cudaStreamCaptureModeThreadLocal));
    const uint64_t before = pg_launch_count();
    pg_status st = enqueue_forward(pl, pl.cap);
    pl.graph_kernels = (int)(pg_launch_count() - before);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(pl.cap, &graph);
    if (st != PG_OK) { if (graph) cudaGraphDestroy(graph); return st; }
    if (e != cudaSuccess) return cuda_fail(e, "batched graph capture");
    e = cudaGraphInstantiate(&pl.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "batched graph instantiate");
    return PG_OK;
}

// The caller holds g_plans_mu until it is done with the plan's buffers.
pg_status get_plan(const int64_t *a_off, const int64_t *b_off, int npairs, int dim, int k, int leaf, Plan **out) {
    std::vector<long long> key = {npairs, dim, k, leaf};
    for (int i = 0; i <= npairs; ++i) key.push_back(a_off[i]);
    for (int i = 0; i <= npairs; ++i) key.push_back(b_off[i]);
    auto it = g_plans.find(key);
    if (it != g_plans.end()) { *out = it->second.get(); return PG_OK; }
    std::unique_ptr<Plan> pl(new Plan());
    pl->npairs = npairs;
    pl->dim = dim;
    pl->k = k;
    pl->leaf = leaf;
    pl->dc = dim_class(dim);
    pl->a_off.assign(a_off, a_off + npairs + 1);
    pl->b_off.assign(b_off, b_off + npairs + 1);
    pl->Na = a_off[npairs];
    pl->Nb = b_off[npairs];
    PG_TRY(make_plan(*pl));
    if (g_plans.size() > 16) g_plans.clear();   // bound the cache
    *out = pl.get();
    g_plans[key] = std::move(pl);
    return PG_OK;
}

pg_status check_offsets(const int64_t *off, int npairs, const char *what) {
    if (off[0] != 0) return fail(PG_EINVAL, std::string("pg_batched_chamfer: ") + what + "[0] must be 0");
    for (int i = 0; i < npairs; ++i)
        if (off[i + 1] <= off[i]) return fail(PG_EINVAL, std::string("pg_batched_chamfer: every cloud needs >= 1 point (") + what + ")");
    if (off[npairs] >= ((int64_t)1 << 31)) return fail(PG_EINVAL, "pg_batched_chamfer: too many points");
    return PG_OK;
}

}  // namespace

}  // namespace pg

using namespace pg;

extern "C" pg_status pg_batched_chamfer(const float *a, const int64_t *a_off, const float *b, const int64_t *b_off,
                                        int npairs, int dim, int k, int leaf_size, float *loss, int32_t *idx_ab,
                                        int32_t *idx_ba, float *dist_ab, float *dist_ba, void *stream) {
    if (npairs < 1) return fail(PG_EINVAL, "pg_batched_chamfer: npairs must be >= 1");
    if (dim < 1 || dim > PG_MAX_DIM) return fail(PG_EINVAL, "pg_batched_chamfer: dim must be in [1, 16]");
    if (k < 1 || k > PG_MAX_K) return fail(PG_EINVAL, "pg_batched_chamfer: k must be in [1, 64]");
    if (leaf_size < 1 || leaf_size > PG_MAX_LEAF) return fail(PG_EINVAL, "pg_batched_chamfer: leaf_size must be in [1, 256]");
    if (!a || !b || !a_off || !b_off || !loss || !idx_ab || !idx_ba) return fail(PG_EINVAL, "pg_batched_chamfer: NULL argument");
    PG_TRY(check_offsets(a_off, npairs, "a_off"));
    PG_TRY(check_offsets(b_off, npairs, "b_off"));
    if ((a_off[npairs] + b_off[npairs]) * (int64_t)k >= ((int64_t)1 << 31))
        return fail(PG_EINVAL, "pg_batched_chamfer: (|a| + |b|) * k must be < 2^31");
    // A plan's argument block, loss and status buffers are shared by every
    // call with its shapes, and the cache may drop plans: the lock is held
    // until this call's stream has passed its last use of them (the status
    // read below synchronises it), so concurrent calls run one at a time.
    std::lock_guard<std::mutex> lk(g_plans_mu);
    Plan *pl = nullptr;
    PG_TRY(get_plan(a_off, b_off, npairs, dim, k, leaf_size, &pl));
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    BArgs args{a, b, idx_ab, idx_ba, dist_ab, dist_ba, g_wait_limit, g_skip_publish};
    PG_CUDA(cudaMemcpyAsync(pl->args, &args, sizeof(args), cudaMemcpyHostToDevice, s));
    PG_CUDA(cudaGraphLaunch(pl->exec, s));
    for (int i = 0; i < pl->graph_kernels; ++i) count_launch();   // the graph's kernel nodes
    PG_CUDA(cudaMemcpyAsync(loss, pl->loss_dev, sizeof(float) * npairs, cudaMemcpyDeviceToDevice, s));
    int st = 0;
    PG_TRY(read_small(&st, pl->status, sizeof(int), s));
    if (st == 1) return fail(PG_ETIMEOUT, "pg_batched_chamfer: a query waited too long for a tree");
    // st == 2: a finisher ran out of scratch and kept one leaf (results stay exact)
    return PG_OK;
}

extern "C" pg_status pg_debug_batched_faults(int skip_publish, long long wait_limit) {
    g_skip_publish = skip_publish ? 1 : 0;
    g_wait_limit = wait_limit > 0 ? wait_limit : kWaitLimit;
    return PG_OK;
}

extern "C" pg_status pg_batched_chamfer_backward(const float *a, const int64_t *a_off, const float *b,
                                                 const int64_t *b_off, int npairs, int dim, int k,
                                                 const int32_t *idx_ab, const int32_t *idx_ba,
                                                 const float *grad_loss, float *grad_a, float *grad_b,
                                                 void *stream) {
    if (npairs < 1) return fail(PG_EINVAL, "pg_batched_chamfer_backward: npairs must be >= 1");
    if (dim < 1 || dim > PG_MAX_DIM) return fail(PG_EINVAL, "pg_batched_chamfer_backward: dim must be in [1, 16]");
    if (k < 1 || k > PG_MAX_K) return fail(PG_EINVAL, "pg_batched_chamfer_backward: k must be in [1, 64]");
    if (!a || !b || !a_off || !b_off || !idx_ab || !idx_ba || !grad_loss || !grad_a || !grad_b)
        return fail(PG_EINVAL, "pg_batched_chamfer_backward: NULL argument");
    PG_TRY(check_offsets(a_off, npairs, "a_off"));
    PG_TRY(check_offsets(b_off, npairs, "b_off"));
    const int64_t Na = a_off[npairs], Nb = b_off[npairs];
    if ((Na + Nb) * (int64_t)k >= ((int64_t)1 << 31)) return fail(PG_EINVAL, "pg_batched_chamfer_backward: too many pairs");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    Scratch offs, rp, sc;
    PG_TRY(offs.alloc(sizeof(long long) * 2 * (npairs + 1), s));
    long long *aoff = offs.as<long long>(), *boff = aoff + npairs + 1;
    PG_CUDA(cudaMemcpyAsync(aoff, a_off, sizeof(long long) * (npairs + 1), cudaMemcpyHostToDevice, s));
    PG_CUDA(cudaMemcpyAsync(boff, b_off, sizeof(long long) * (npairs + 1), cudaMemcpyHostToDevice, s));
    PG_TRY(rp.alloc(sizeof(int) * (size_t)(Na + Nb), s));
    int *rpa = rp.as<int>(), *rpb = rpa + Na;
    k_row_pair<<<grid_of(Na), BT, 0, s>>>(aoff, npairs, Na, rpa);
    k_row_pair<<<grid_of(Nb), BT, 0, s>>>(boff, npairs, Nb, rpb);
    count_launch();
    count_launch();
    const int64_t Pab = Na * k, Pba = Nb * k, Pm = std::max(Pab, Pba);
    // keys, vals, two temporaries (for the larger direction) + bounds for a and b
    // hub rows hold more than kHeavy entries each: at most Pm/kHeavy of them,
    // and at most Pm/kChunk + Pm/kHeavy chunks
    const int64_t Nm = std::max(Na, Nb), Hm = Pm / kHeavy + 1, Cm = Pm / kChunk + Hm;
    PG_TRY(sc.alloc(sizeof(uint32_t) * (size_t)(4 * Pm) + sizeof(int) * (size_t)(2 * Nm + 2 * Hm + Cm + 2) +
                        sizeof(float) * (size_t)(Cm * dim_class(dim)) + 256, s));
    uint32_t *keys = sc.as<uint32_t>(), *vals = keys + Pm, *tk = vals + Pm, *tv = tk + Pm;
    int *lo = reinterpret_cast<int *>(tv + Pm), *hi = lo + Nm;
    int2 *heavy = reinterpret_cast<int2 *>(hi + Nm);
    int *chunk_row = reinterpret_cast<int *>(heavy + Hm);
    int *nheavy = chunk_row + Cm, *nchunks = nheavy + 1;
    float *part = reinterpret_cast<float *>(nchunks + 1);
    auto bits_for = [](int64_t n) { int b = 1; while (b < 32 && ((int64_t)1 << b) <= n) ++b; return b; };
    // grad_b: b rows' own neighbours in a (idx_ba) + a rows that selected them (idx_ab)
    for (int side = 0; side < 2; ++side) {
        const bool for_b = side == 0;
        const int64_t nx = for_b ? Nb : Na, ny = for_b ? Na : Nb;
        const int32_t *idx_yx = for_b ? idx_ab : idx_ba;    // Y rows selecting X rows
        const int *rpy = for_b ? rpa : rpb;
        const long long *offx = for_b ? boff : aoff;
        const int64_t P = ny * k;
        PG_CUDA(cudaMemsetAsync(lo, 0, sizeof(int) * (size_t)(2 * Nm), s));
        k_bkeys<<<grid_of(P), BT, 0, s>>>(idx_yx, ny, k, rpy, offx, (uint32_t)nx, keys);
        count_launch();
        uint32_t *sk, *sv;
        PG_TRY(radix_sort_pairs(keys, vals, true, tk, tv, P, bits_for(nx), s, &sk, &sv));
        k_bbounds<<<grid_of(P), BT, 0, s>>>(sk, P, (uint32_t)nx, lo, hi);
        count_launch();
        KTimer kt("batched_backward_grad", s);
        PG_CUDA(cudaMemsetAsync(nheavy, 0, sizeof(int) * 2, s));
        const float *Xp = for_b ? b : a, *Yp = for_b ? a : b;
        const int32_t *ixy = for_b ? idx_ba : idx_ab;
        const int *rpx = for_b ? rpb : rpa;
        const long long *offy = for_b ? aoff : boff;
        float *gxp = for_b ? grad_b : grad_a;
        int *hi_arr = hi;
        const int hgrid = num_sms() * 8;
        switch (dim_class(dim)) {
#define PG_BG(D)                                                                                            \
            case D:                                                                                         \
                k_bgrad<D><<<grid_of(nx), BT, 0, s>>>(Xp, nx, Yp, dim, k, ixy, rpx, rpy, offy, grad_loss, sv, lo, \
                                                      hi_arr, gxp, heavy, nheavy, chunk_row, nchunks);      \
                k_bgrad_chunk<D><<<hgrid, BT, 0, s>>>(Xp, Yp, dim, k, rpy, grad_loss, sv, lo, hi_arr, heavy, \
                                                      chunk_row, nchunks, part);                            \
                k_bgrad_hubs<D><<<grid_of(Hm), BT, 0, s>>>(dim, lo, hi_arr, heavy, nheavy, part, gxp);      \
                break;
            PG_BG(2) PG_BG(3) PG_BG(4) PG_BG(5) PG_BG(6) PG_BG(7) PG_BG(8) PG_BG(12) PG_BG(16)
#undef PG_BG
            default: return fail(PG_EUNSUPPORTED, "dimension class");
        }
        count_launch();
        count_launch();
        count_launch();
        PG_TRY(check_launch("batched backward"));
    }
    return PG_OK;
}
