// Device-wide primitives written for this library (no vendor sort or scan):
// an exclusive prefix sum and a stable LSD radix sort of (key, value) pairs.
// ArborX 2.0 (section 2.6) sorts Morton codes and queries with the vendor
// libraries; here both sorts run on this radix sort.
#pragma once

#include "common.cuh"

namespace arbx {

// out[i] = sum_{j<i} in[j] for i in [0, n]; out[n] is the total.
// TIn/TOut: (int32_t, int64_t) or (uint32_t, uint32_t).
template <class TIn, class TOut>
arbx_status exclusive_scan(const TIn* in, TOut* out, int64_t n, cudaStream_t s);

// The int32 -> int64 scan of any size with its temporaries supplied by the
// caller: temp holds at least scan_temp_elems(n) int64 entries.  No device
// allocation (the launches can be captured in a graph).
int64_t scan_temp_elems(int64_t n);
arbx_status exclusive_scan_temp(const int32_t* in, int64_t* out, int64_t n, int64_t* temp, cudaStream_t s);

// The same int32 -> int64 scan with its temporaries supplied by the caller:
// totals and offs hold `cap` entries each, at least scan_prealloc_tiles(n) + 1;
// n <= scan_prealloc_max().  ARBX_ERR_CAPACITY when cap is too small.  No
// device allocation.
constexpr int SCAN_TILE_ELEMS = 2048;  // counts per scan tile (256 threads x 8)
inline int64_t scan_prealloc_tiles(int64_t n) { return (n + SCAN_TILE_ELEMS - 1) / SCAN_TILE_ELEMS; }
int64_t scan_prealloc_max();
arbx_status exclusive_scan_prealloc(const int32_t* in, int64_t* out, int64_t n, int64_t* totals, int64_t* offs,
                                    int64_t cap, cudaStream_t s);

// Stable sort of (keys, vals) by bits [begin_bit, end_bit) of the keys, in
// passes of 8 bits.  keys/vals and keys_alt/vals_alt are ping-pong buffers of n
// elements; *in_alt tells which pair holds the result.  K: uint32_t or uint64_t.
template <class K>
arbx_status radix_sort_pairs(K* keys, uint32_t* vals, K* keys_alt, uint32_t* vals_alt, int64_t n,
                             int begin_bit, int end_bit, bool* in_alt, cudaStream_t s);

}  // namespace arbx
