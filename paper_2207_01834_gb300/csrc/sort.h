// Stable radix sort of (key, value) pairs (device memory, stream-ordered).
#pragma once

#include "common.cuh"

namespace pg {

// Tile sizes of the radix sort (items per tile, digits per pass) and of the
// device-wide scan (items per tile).  Workspace sizes follow from them; a
// caller that reserves workspace at compile time sizes it with the constexpr
// functions below, so a tile change cannot leave a reserve too small.
constexpr int kRadixTileItems = 2048;
constexpr int kRadixDigits = 256;
constexpr int kScanTileItems = 4096;

constexpr int64_t scan_ws_words_ce(int64_t n) { return n <= 0 ? 1 : (n + kScanTileItems - 1) / kScanTileItems + 1; }
constexpr int64_t radix_ws_words_ce(int64_t n) {
    return 2 * ((int64_t)kRadixDigits * (n > 0 ? (n + kRadixTileItems - 1) / kRadixTileItems : 1)) + 1 +
           scan_ws_words_ce((int64_t)kRadixDigits * (n > 0 ? (n + kRadixTileItems - 1) / kRadixTileItems : 1));
}

// Sorts n pairs by the low `bits` bits of the key, stably.  keys/vals hold the
// input (vals is ignored and the item index used instead when iota_vals);
// tk/tv are temporaries of n entries.  The sorted arrays end in whichever pair
// of buffers *out_keys/*out_vals point to.
pg_status radix_sort_pairs(uint32_t *keys, uint32_t *vals, bool iota_vals, uint32_t *tk, uint32_t *tv, int64_t n,
                           int bits, cudaStream_t s, uint32_t **out_keys, uint32_t **out_vals);

// Workspace variants that allocate nothing: `ws` must hold radix_ws_words(n)
// ints (scan_ws_words(n) for the scan).
int64_t scan_ws_words(int64_t n);
pg_status exclusive_scan_ws(const int *in, int *out, int64_t n, int *ws, cudaStream_t s);
int64_t radix_ws_words(int64_t n);
pg_status radix_sort_pairs_ws(uint32_t *keys, uint32_t *vals, bool iota_vals, uint32_t *tk, uint32_t *tv,
                              int64_t n, int bits, int *ws, cudaStream_t s, uint32_t **out_keys,
                              uint32_t **out_vals);

}  // namespace pg
