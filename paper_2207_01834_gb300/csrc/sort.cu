// Stable least-significant-digit radix sort of (uint32 key, uint32 value)
// pairs, 8 bits per pass.  Each pass: per-tile digit histograms, one
// device-wide exclusive scan over the digit-major histogram table, then a
// stable scatter in which every tile ranks its items in input order (warp
// match + popcount, then per-digit offsets across the tile's warps), puts
// them in that order in shared memory, and writes each digit's run to its
// global range with consecutive threads on consecutive addresses.
#include "internal.h"
#include "sort.h"

namespace pg {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kRounds = 8;                    // items per thread
constexpr int kTile = kThreads * kRounds;     // 2048 items per tile
constexpr int kRadix = 256;
static_assert(kThreads == kRadix, "one thread per digit in the scatter's tile scan");
static_assert(kTile == kRadixTileItems && kRadix == kRadixDigits, "tile constants published in sort.h");

__global__ void __launch_bounds__(kThreads) k_rs_hist(const uint32_t *__restrict__ keys, int64_t n, int shift,
                                                      int ntiles, int *__restrict__ ghist) {
    __shared__ int hist[kRadix];
    hist[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kTile;
#pragma unroll
    for (int r = 0; r < kRounds; ++r) {
        const int64_t i = base + r * kThreads + threadIdx.x;
        if (i < n) atomicAdd(&hist[(keys[i] >> shift) & 0xff], 1);
    }
    __syncthreads();
    ghist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = hist[threadIdx.x];
}

__global__ void __launch_bounds__(kThreads) k_rs_scatter(const uint32_t *__restrict__ keys,
                                                         const uint32_t *__restrict__ vals, int64_t n, int shift,
                                                         int ntiles, const int *__restrict__ goff,
                                                         uint32_t *__restrict__ okeys, uint32_t *__restrict__ ovals) {
    __shared__ int wcnt[kWarps][kRadix];
    __shared__ int toff[kRadix], lstart[kRadix], wsum[kWarps];
    __shared__ uint32_t sk[kTile], sv[kTile];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kWarps * kRadix; i += kThreads) (&wcnt[0][0])[i] = 0;
    toff[threadIdx.x] = goff[(int64_t)threadIdx.x * ntiles + blockIdx.x];
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)warp * (kTile / kWarps);
    const unsigned lt = (1u << lane) - 1u;
    uint32_t k_[kRounds], v_[kRounds];
    int d_[kRounds], rank[kRounds];
#pragma unroll
    for (int r = 0; r < kRounds; ++r) {
        const int64_t i = base + r * 32 + lane;
        const bool valid = i < n;
        k_[r] = valid ? keys[i] : 0u;
        v_[r] = valid ? (vals ? vals[i] : (uint32_t)i) : 0u;
        const int d = valid ? (int)((k_[r] >> shift) & 0xff) : kRadix;
        d_[r] = d;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int before = valid ? wcnt[warp][d] : 0;
        rank[r] = before + __popc(peers & lt);
        __syncwarp();
        if (valid && lane == __ffs(peers) - 1) wcnt[warp][d] = before + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    {
        // per digit (thread = digit): offsets of the warps' runs, the tile's
        // count, and the exclusive scan of the counts over the digits
        int run = 0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) {
            const int c = wcnt[w][threadIdx.x];
            wcnt[w][threadIdx.x] = run;
            run += c;
        }
        int x = run;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[warp] = x;
        __syncthreads();
        int before = 0;
        for (int w = 0; w < warp; ++w) before += wsum[w];
        lstart[threadIdx.x] = before + x - run;
    }
    __syncthreads();
    // the tile in stable digit order in shared memory
#pragma unroll
    for (int r = 0; r < kRounds; ++r) {
        const int d = d_[r];
        if (d < kRadix) {
            const int lp = lstart[d] + wcnt[warp][d] + rank[r];
            sk[lp] = k_[r];
            sv[lp] = v_[r];
        }
    }
    __syncthreads();
    // item j of the tile goes to its digit's global offset + its place in the run
    const int64_t tb = (int64_t)blockIdx.x * kTile;
    const int tn = (int)min((int64_t)kTile, n - tb);
    for (int j = threadIdx.x; j < tn; j += kThreads) {
        const uint32_t kk = sk[j];
        const int d = (int)((kk >> shift) & 0xff);
        const int pos = toff[d] + (j - lstart[d]);
        okeys[pos] = kk;
        ovals[pos] = sv[j];
    }
}

}  // namespace

pg_status radix_sort_pairs(uint32_t *keys, uint32_t *vals, bool iota_vals, uint32_t *tk, uint32_t *tv, int64_t n,
                           int bits, cudaStream_t s, uint32_t **out_keys, uint32_t **out_vals) {
    *out_keys = keys;
    *out_vals = vals;
    if (n <= 0) return PG_OK;
    if (n >= ((int64_t)1 << 31)) return fail(PG_EINVAL, "radix sort: too many items");
    const int ntiles = ceil_div_i(n, kTile);
    Scratch hist, off;
    PG_TRY(hist.alloc(sizeof(int) * (size_t)kRadix * ntiles, s));
    PG_TRY(off.alloc(sizeof(int) * ((size_t)kRadix * ntiles + 1), s));
    uint32_t *ik = keys, *iv = vals, *ok = tk, *ov = tv;
    const int passes = bits <= 8 ? 1 : (bits + 7) / 8;
    for (int p = 0; p < passes; ++p) {
        const int shift = 8 * p;
        k_rs_hist<<<ntiles, kThreads, 0, s>>>(ik, n, shift, ntiles, hist.as<int>());
        count_launch();
        PG_TRY(exclusive_scan(hist.as<int>(), off.as<int>(), (int64_t)kRadix * ntiles, s));
        k_rs_scatter<<<ntiles, kThreads, 0, s>>>(ik, (p == 0 && iota_vals) ? nullptr : iv, n, shift, ntiles,
                                                 off.as<int>(), ok, ov);
        count_launch();
        PG_TRY(check_launch("radix sort"));
        std::swap(ik, ok);
        std::swap(iv, ov);
    }
    *out_keys = ik;
    *out_vals = iv;
    return PG_OK;
}

// hist (cells) + offsets (cells + 1) + the offsets scan's partials
int64_t radix_ws_words(int64_t n) { return radix_ws_words_ce(n); }

pg_status radix_sort_pairs_ws(uint32_t *keys, uint32_t *vals, bool iota_vals, uint32_t *tk, uint32_t *tv,
                              int64_t n, int bits, int *ws, cudaStream_t s, uint32_t **out_keys,
                              uint32_t **out_vals) {
    *out_keys = keys;
    *out_vals = vals;
    if (n <= 0) return PG_OK;
    if (n >= ((int64_t)1 << 31)) return fail(PG_EINVAL, "radix sort: too many items");
    const int ntiles = ceil_div_i(n, kTile);
    const int64_t cells = (int64_t)kRadix * ntiles;
    int *hist = ws, *off = ws + cells, *scan_ws = off + cells + 1;
    uint32_t *ik = keys, *iv = vals, *ok = tk, *ov = tv;
    const int passes = bits <= 8 ? 1 : (bits + 7) / 8;
    for (int p = 0; p < passes; ++p) {
        const int shift = 8 * p;
        k_rs_hist<<<ntiles, kThreads, 0, s>>>(ik, n, shift, ntiles, hist);
        count_launch();
        PG_TRY(exclusive_scan_ws(hist, off, cells, scan_ws, s));
        k_rs_scatter<<<ntiles, kThreads, 0, s>>>(ik, (p == 0 && iota_vals) ? nullptr : iv, n, shift, ntiles, off,
                                                 ok, ov);
        count_launch();
        PG_TRY(check_launch("radix sort"));
        std::swap(ik, ok);
        std::swap(iv, ov);
    }
    *out_keys = ik;
    *out_vals = iv;
    return PG_OK;
}

}  // namespace pg
