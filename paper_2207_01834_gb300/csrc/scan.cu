// Device-wide exclusive prefix sum of int32 (reduce / scan-of-partials /
// down-sweep).  Used by the tree builder (stable partition offsets, segment
// numbering) and by stream compactions.
#include "internal.h"
#include "sort.h"

namespace pg {

namespace {

constexpr int kThreads = 256;
constexpr int kItems = 16;
constexpr int kTile = kThreads * kItems;
static_assert(kTile == kScanTileItems, "scan tile published in sort.h");

__device__ __forceinline__ int warp_incl_scan(int x) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

// Exclusive scan of one value per thread across the block; *total gets the sum.
__device__ __forceinline__ int block_excl_scan(int v, int *wsum, int *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    int x = warp_incl_scan(v);
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int w = lane < nw ? wsum[lane] : 0;
        w = warp_incl_scan(w);
        if (lane < nw) wsum[lane] = w;
    }
    __syncthreads();
    int off = warp ? wsum[warp - 1] : 0;
    *total = wsum[nw - 1];
    __syncthreads();
    return off + x - v;
}

__global__ void __launch_bounds__(kThreads) k_scan_reduce(const int *__restrict__ in, int64_t n,
                                                          int *__restrict__ bsum) {
    __shared__ int wsum[32];
    const int64_t base = (int64_t)blockIdx.x * kTile;
    int s = 0;
#pragma unroll 4
    for (int i = threadIdx.x; i < kTile; i += kThreads) {
        int64_t g = base + i;
        if (g < n) s += in[g];
    }
    int tot;
    block_excl_scan(s, wsum, &tot);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

// One block: exclusive scan of bsum[0..nb) in place, bsum[nb] = total.
__global__ void __launch_bounds__(1024) k_scan_top(int *__restrict__ bsum, int nb) {
    __shared__ int wsum[32];
    int carry = 0;
    for (int base = 0; base < nb; base += 1024) {
        int i = base + threadIdx.x;
        int v = i < nb ? bsum[i] : 0;
        int tot;
        int ex = block_excl_scan(v, wsum, &tot);
        if (i < nb) bsum[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) bsum[nb] = carry;
}

__global__ void __launch_bounds__(kThreads) k_scan_down(const int *__restrict__ in, int64_t n,
                                                        const int *__restrict__ bsum, int nb,
                                                        int *__restrict__ out) {
    __shared__ int tile[kTile];
    __shared__ int wsum[32];
    const int64_t base = (int64_t)blockIdx.x * kTile;
    for (int i = threadIdx.x; i < kTile; i += kThreads) {
        int64_t g = base + i;
        tile[i] = g < n ? in[g] : 0;
    }
    __syncthreads();
    int loc[kItems];
    int s = 0;
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
        loc[j] = s;
        s += tile[threadIdx.x * kItems + j];
    }
    int tot;
    int ex = block_excl_scan(s, wsum, &tot);
    const int off = bsum[blockIdx.x] + ex;
#pragma unroll
    for (int j = 0; j < kItems; ++j) tile[threadIdx.x * kItems + j] = off + loc[j];
    __syncthreads();
    for (int i = threadIdx.x; i < kTile; i += kThreads) {
        int64_t g = base + i;
        if (g < n) out[g] = tile[i];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = bsum[nb];
}

}  // namespace

pg_status exclusive_scan(const int *in, int *out, int64_t n, cudaStream_t s) {
    if (n <= 0) {
        PG_CUDA(cudaMemsetAsync(out, 0, sizeof(int), s));
        return PG_OK;
    }
    const int nb = ceil_div_i(n, kTile);
    Scratch bs;
    PG_TRY(bs.alloc(sizeof(int) * (size_t)(nb + 1), s));
    int *bsum = bs.as<int>();
    k_scan_reduce<<<nb, kThreads, 0, s>>>(in, n, bsum);
    count_launch();
    k_scan_top<<<1, 1024, 0, s>>>(bsum, nb);
    count_launch();
    k_scan_down<<<nb, kThreads, 0, s>>>(in, n, bsum, nb, out);
    count_launch();
    return check_launch("exclusive_scan");
}

// Same scan with caller-provided partial-sum workspace (scan_ws_words(n) ints):
// allocates nothing.
int64_t scan_ws_words(int64_t n) { return scan_ws_words_ce(n); }

pg_status exclusive_scan_ws(const int *in, int *out, int64_t n, int *ws, cudaStream_t s) {
    if (n <= 0) {
        PG_CUDA(cudaMemsetAsync(out, 0, sizeof(int), s));
        return PG_OK;
    }
    const int nb = ceil_div_i(n, kTile);
    k_scan_reduce<<<nb, kThreads, 0, s>>>(in, n, ws);
    count_launch();
    k_scan_top<<<1, 1024, 0, s>>>(ws, nb);
    count_launch();
    k_scan_down<<<nb, kThreads, 0, s>>>(in, n, ws, nb, out);
    count_launch();
    return check_launch("exclusive_scan_ws");
}

}  // namespace pg
