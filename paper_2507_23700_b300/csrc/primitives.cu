// Exclusive scan and stable LSD radix sort (see primitives.cuh).
#include "primitives.cuh"

#include <mutex>
#include <utility>
#include <vector>

namespace arbx {
namespace {

constexpr unsigned FULL = 0xffffffffu;

// ------------------------------------------------------------------ scan
//
// Three phases with no inter-block waiting: per-tile totals, a scan of the
// totals (recursive), then per-tile scans offset by the scanned totals.

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_IPT = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_IPT;
static_assert(SCAN_TILE == SCAN_TILE_ELEMS, "scan tile size exported in primitives.cuh");

template <class T>
__device__ __forceinline__ T warp_inclusive_scan(T v, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T u = __shfl_up_sync(FULL, v, o);
    if (lane >= o) v += u;
  }
  return v;
}

// Inclusive scan over the block (blockDim.x == SCAN_THREADS); *total receives the sum.
template <class T>
__device__ __forceinline__ T block_inclusive_scan(T v, T* s_warp, T* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T w = warp_inclusive_scan(v, lane);
  if (lane == 31) s_warp[warp] = w;
  __syncthreads();
  if (warp == 0) {
    T t = lane < (SCAN_THREADS / 32) ? s_warp[lane] : T(0);
    t = warp_inclusive_scan(t, lane);
    if (lane < (SCAN_THREADS / 32)) s_warp[lane] = t;
  }
  __syncthreads();
  T r = w + (warp > 0 ? s_warp[warp - 1] : T(0));
  *total = s_warp[SCAN_THREADS / 32 - 1];
  __syncthreads();
  return r;
}

template <class TIn, class TOut>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_tile_totals(const TIn* in, int64_t n, TOut* totals) {
  __shared__ TOut s_warp[SCAN_THREADS / 32];
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_IPT;
  TOut acc = 0;
#pragma unroll
  for (int k = 0; k < SCAN_IPT; ++k)
    if (base + k < n) acc += (TOut)in[base + k];
  TOut total;
  block_inclusive_scan(acc, s_warp, &total);
  if (threadIdx.x == 0) totals[blockIdx.x] = total;
}

template <class TIn, class TOut>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_tiles(const TIn* in, TOut* out, int64_t n,
                                                             const TOut* tile_offsets, bool write_total) {
  __shared__ TOut s_warp[SCAN_THREADS / 32];
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_IPT;
  TOut v[SCAN_IPT];
  TOut acc = 0;
#pragma unroll
  for (int k = 0; k < SCAN_IPT; ++k) {
    v[k] = (base + k < n) ? (TOut)in[base + k] : TOut(0);
    acc += v[k];
  }
  TOut total;
  TOut incl = block_inclusive_scan(acc, s_warp, &total);
  TOut run = incl - acc + (tile_offsets ? tile_offsets[blockIdx.x] : TOut(0));
#pragma unroll
  for (int k = 0; k < SCAN_IPT; ++k) {
    if (base + k < n) out[base + k] = run;
    run += v[k];
  }
  if (write_total && blockIdx.x == gridDim.x - 1 && threadIdx.x == SCAN_THREADS - 1) out[n] = run;
}

template <class TIn, class TOut>
arbx_status scan_impl(const TIn* in, TOut* out, int64_t n, bool write_total, cudaStream_t s) {
  if (n <= 0) {
    if (write_total) ARBX_CUDA(cudaMemsetAsync(out, 0, sizeof(TOut), s));
    return ARBX_OK;
  }
  const int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
  if (tiles == 1) {
    ARBX_LAUNCH("scan_tiles", s, k_scan_tiles<TIn, TOut><<<1, SCAN_THREADS, 0, s>>>(in, out, n, nullptr, write_total));
    return ARBX_OK;
  }
  DevTemp<TOut> totals(s), offs(s);
  ARBX_TRY(totals.alloc(tiles));
  ARBX_TRY(offs.alloc(tiles + 1));
  ARBX_LAUNCH("scan_tile_totals", s, k_scan_tile_totals<TIn, TOut><<<(unsigned)tiles, SCAN_THREADS, 0, s>>>(in, n, totals.p));
  ARBX_TRY((scan_impl<TOut, TOut>(totals.p, offs.p, tiles, false, s)));
  ARBX_LAUNCH("scan_tiles", s, k_scan_tiles<TIn, TOut><<<(unsigned)tiles, SCAN_THREADS, 0, s>>>(in, out, n, offs.p, write_total));
  return ARBX_OK;
}

// ------------------------------------------------------------------ radix sort
//
// LSD, 8-bit digits.  One kernel counts the digits of every pass in one read
// of the keys; then each pass is a single launch (k_rs_pass) that ranks a
// tile's keys stably, finds each digit's output start by a look-back over the
// earlier tiles' published counts (the decoupled look-back of Merrill and
// Garland's single-pass prefix scan, as in their Onesweep radix sort), and
// scatters through shared memory so that each digit's run is written
// contiguously.

constexpr int RS_THREADS = 256;  // one thread per digit in the per-tile steps
// Keys per thread of a radix-sort tile (8: the 64-bit-key scatter pass fits
// 77 registers, three blocks per SM; 10M keys, build sort + query order,
// measured with __match_any_sync ranking: 2.79 ms at 8, 3.20 at 12, 3.05 at
// 16; 2.19 ms at 8 with the ballot ranking and per-warp histograms).
#ifndef ARBX_RS_IPT
#define ARBX_RS_IPT 8
#endif
constexpr int RS_IPT = ARBX_RS_IPT;
constexpr int RS_TILE = RS_THREADS * RS_IPT;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RADIX = 256;

template <class K>
__device__ __forceinline__ uint32_t digit_of(K k, int shift) {
  return (uint32_t)(k >> shift) & 0xffu;
}

template <class K>
__global__ void __launch_bounds__(RS_THREADS) k_rs_upsweep(const K* keys, int64_t n, int shift, uint32_t num_tiles,
                                                           uint32_t* hist) {
  // per-warp digit counts (plain shared-memory atomics; warp-aggregating them
  // with __match_any_sync measured 2.2x slower), summed per digit at the end
  __shared__ uint32_t wc[RS_WARPS][RADIX];
  const int warp = threadIdx.x >> 5;
#pragma unroll
  for (int w = 0; w < RS_WARPS; ++w) wc[w][threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * RS_TILE;
#pragma unroll 4
  for (int k = 0; k < RS_IPT; ++k) {
    const int64_t i = base + (int64_t)k * RS_THREADS + threadIdx.x;
    if (i < n) atomicAdd(&wc[warp][digit_of(keys[i], shift)], 1u);
  }
  __syncthreads();
  uint32_t c = 0;
#pragma unroll
  for (int w = 0; w < RS_WARPS; ++w) c += wc[w][threadIdx.x];
  hist[(size_t)threadIdx.x * num_tiles + blockIdx.x] = c;
}

// Digit counts of every pass from one read of the keys: pass p counts the
// 8-bit digit at bit begin_bit + 8p.  Per-warp counts in shared memory (plain
// shared atomics), summed per block, then added to the global counts
// (ghist[p * 256 + digit], zeroed by the caller) once per block.
template <class K>
__global__ void __launch_bounds__(RS_THREADS) k_rs_hist(const K* __restrict__ keys, int64_t n, int begin_bit,
                                                        int npasses, uint32_t* __restrict__ ghist) {
  extern __shared__ __align__(16) unsigned char rs_smem[];
  uint32_t* wc = reinterpret_cast<uint32_t*>(rs_smem);  // [RS_WARPS][npasses][RADIX]
  const int warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < RS_WARPS * npasses * RADIX; i += RS_THREADS) wc[i] = 0;
  __syncthreads();
  uint32_t* mine = wc + warp * npasses * RADIX;
  for (int64_t i = (int64_t)blockIdx.x * RS_THREADS + threadIdx.x; i < n; i += (int64_t)gridDim.x * RS_THREADS) {
    const K k = keys[i];
    for (int p = 0; p < npasses; ++p) atomicAdd(&mine[p * RADIX + digit_of(k, begin_bit + 8 * p)], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < npasses * RADIX; i += RS_THREADS) {
    uint32_t c = 0;
#pragma unroll
    for (int w = 0; w < RS_WARPS; ++w) c += wc[w * npasses * RADIX + i];
    if (c) atomicAdd(&ghist[i], c);
  }
}

// Tile status words of the look-back: the flag above bit 32 (0: not yet
// published, 1: the tile's own digit count, 2: the count of every key of this
// digit in this and all earlier tiles), the count in the low 32 bits.
constexpr unsigned long long RS_AGG = 1ull << 32, RS_INCL = 2ull << 32, RS_COUNT = 0xffffffffull;
// Polls of a predecessor's status word before a pass gives up (far beyond any
// wait of a working pass; the pass then sets DEVERR_INTERNAL).
constexpr uint32_t RS_SPIN_LIMIT = 1u << 22;

__device__ __forceinline__ unsigned long long ld_relaxed(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// One stable counting pass on the digit at bit `shift`.  A block ranks a
// tile's keys stably (warp-private running counts, the lanes of equal digit
// found with one ballot per digit bit, in input order) and scatters them
// through shared memory so that each digit's run goes out contiguously.
// Where each of the tile's digits starts in the output comes either
// (LOOKBACK false) from the scan of all tiles' digit counts that k_rs_upsweep
// and exclusive_scan make before the launch (reduce-then-scan: four launches
// per pass), or (LOOKBACK true: one launch per pass) from a look-back over the
// earlier tiles: the block takes the next tile in launch order from
// `tile_counter`; a tile publishes its own digit counts at once and the
// running count once it knows it, and a successor sums the counts it meets,
// walking back until it meets a running count.  Tiles are numbered in the
// order their blocks started, so every tile waited on belongs to a block that
// is already running and waits only on earlier tiles.  The digit starts are
// then the exclusive scan of the pass's global digit counts (ghist, counted
// for every pass by one k_rs_hist launch) plus that look-back sum.  A
// look-back that runs out of polls (RS_SPIN_LIMIT) sets DEVERR_INTERNAL and
// uses the partial sum, which is never above the true one, so every write
// stays inside the output.
template <class K, bool LOOKBACK>
__global__ void __launch_bounds__(RS_THREADS) k_rs_pass(const K* __restrict__ keys_in, const uint32_t* __restrict__ vals_in,
                                                        K* __restrict__ keys_out, uint32_t* __restrict__ vals_out,
                                                        int64_t n, int shift, const uint32_t* __restrict__ starts,
                                                        uint32_t num_tiles, const uint32_t* __restrict__ ghist,
                                                        unsigned long long* __restrict__ status,
                                                        uint32_t* __restrict__ tile_counter,
                                                        uint32_t* __restrict__ err) {
  extern __shared__ __align__(16) unsigned char rs_smem[];
  K* s_keys = reinterpret_cast<K*>(rs_smem);
  uint32_t* s_vals = reinterpret_cast<uint32_t*>(s_keys + RS_TILE);
  uint32_t* s_wcnt = s_vals + RS_TILE;         // [RS_WARPS][RADIX]
  uint32_t* s_dstart = s_wcnt + RS_WARPS * RADIX;  // tile-local start of each digit
  uint32_t* s_gbase = s_dstart + RADIX;        // global start of each digit for this tile
  uint32_t* s_warp = s_gbase + RADIX;          // scan scratch (+ the tile number)

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (LOOKBACK && tid == 0) s_warp[RS_WARPS] = atomicAdd(tile_counter, 1u);
  for (int i = tid; i < RS_WARPS * RADIX; i += RS_THREADS) s_wcnt[i] = 0;
  __syncthreads();
  const uint32_t tile = LOOKBACK ? s_warp[RS_WARPS] : blockIdx.x;

  const int64_t tile_base = (int64_t)tile * RS_TILE;
  const int64_t wbase = tile_base + (int64_t)warp * 32 * RS_IPT;
  const unsigned lt = (1u << lane) - 1u;
  K key[RS_IPT];
  uint32_t val[RS_IPT];
  uint32_t rank[RS_IPT];
#pragma unroll
  for (int k = 0; k < RS_IPT; ++k) {
    const int64_t i = wbase + k * 32 + lane;
    const bool valid = i < n;
    key[k] = valid ? keys_in[i] : K(0);
    val[k] = valid ? vals_in[i] : 0u;
    const uint32_t d = valid ? digit_of(key[k], shift) : 256u;
    // lanes of the warp holding the same digit: eight ballots, one per digit
    // bit, within the valid lanes (7% faster here than __match_any_sync)
    unsigned peers = __ballot_sync(FULL, valid);
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const bool bit = (d >> b) & 1u;
      const unsigned m = __ballot_sync(FULL, bit);
      peers &= bit ? m : ~m;
    }
    const uint32_t old = valid ? s_wcnt[warp * RADIX + d] : 0u;
    __syncwarp();
    if (valid && lane == __ffs(peers) - 1) s_wcnt[warp * RADIX + d] = old + (uint32_t)__popc(peers);
    __syncwarp();
    rank[k] = valid ? old + (uint32_t)__popc(peers & lt) : 0xffffffffu;
  }
  __syncthreads();
  // Per digit (one per thread): exclusive prefix over the warps, tile count.
  uint32_t run = 0;
#pragma unroll
  for (int w = 0; w < RS_WARPS; ++w) {
    const uint32_t t = s_wcnt[w * RADIX + tid];
    s_wcnt[w * RADIX + tid] = run;
    run += t;
  }
  // publish this tile's count of digit tid (the running count at once for tile 0)
  unsigned long long* my_status = LOOKBACK ? status + (size_t)tile * RADIX + tid : nullptr;
  if (LOOKBACK) st_relaxed(my_status, (tile == 0 ? RS_INCL : RS_AGG) | run);
  // Exclusive scans of the tile's digit counts and (look-back) of the pass's global digit counts.
  const uint32_t gcount = LOOKBACK ? ghist[tid] : 0u;
  {
    uint32_t w = warp_inclusive_scan(run, lane);
    uint32_t gw = warp_inclusive_scan(gcount, lane);
    if (lane == 31) {
      s_warp[warp] = w;
      s_gbase[warp] = gw;  // per-warp totals of the global counts (s_gbase reused below)
    }
    __syncthreads();
    if (warp == 0) {
      uint32_t t = lane < RS_WARPS ? s_warp[lane] : 0u;
      uint32_t gt = lane < RS_WARPS ? s_gbase[lane] : 0u;
      t = warp_inclusive_scan(t, lane);
      gt = warp_inclusive_scan(gt, lane);
      if (lane < RS_WARPS) {
        s_warp[lane] = t;
        s_gbase[lane] = gt;
      }
    }
    __syncthreads();
    const uint32_t incl = w + (warp > 0 ? s_warp[warp - 1] : 0u);
    const uint32_t gincl = gw + (warp > 0 ? s_gbase[warp - 1] : 0u);
    s_dstart[tid] = incl - run;
    // look back over the earlier tiles for the keys of digit tid before this tile
    uint32_t before = 0;
    if (LOOKBACK && tile > 0) {
      int64_t t = (int64_t)tile - 1;
      uint32_t polls = 0;
      for (;;) {
        const unsigned long long v = ld_relaxed(status + (size_t)t * RADIX + tid);
        if ((v & ~RS_COUNT) == 0u) {
          if (++polls > RS_SPIN_LIMIT) {
            atomicOr(err, DEVERR_INTERNAL);
            break;
          }
          if (polls > 8) __nanosleep(64);
          continue;
        }
        before += (uint32_t)(v & RS_COUNT);
        if ((v & ~RS_COUNT) == RS_INCL || t == 0) break;
        --t;
      }
      st_relaxed(my_status, RS_INCL | (before + run));
    }
    __syncthreads();  // s_gbase's warp totals are read before it is overwritten
    s_gbase[tid] = LOOKBACK ? (gincl - gcount) + before : starts[(size_t)tid * num_tiles + blockIdx.x];
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < RS_IPT; ++k) {
    if (rank[k] != 0xffffffffu) {
      const uint32_t d = digit_of(key[k], shift);
      const uint32_t pos = s_dstart[d] + s_wcnt[warp * RADIX + d] + rank[k];
      s_keys[pos] = key[k];
      s_vals[pos] = val[k];
    }
  }
  __syncthreads();
  const int64_t rem = n - tile_base;
  const int count = rem < RS_TILE ? (int)rem : RS_TILE;
  for (int i = tid; i < count; i += RS_THREADS) {
    const K kk = s_keys[i];
    const uint32_t d = digit_of(kk, shift);
    const int64_t g = (int64_t)s_gbase[d] + (i - (int)s_dstart[d]);
    if (g < n) {
      keys_out[g] = kk;
      vals_out[g] = s_vals[i];
    }
  }
}

template <class K>
constexpr size_t rs_smem_bytes() {
  return RS_TILE * sizeof(K) + RS_TILE * sizeof(uint32_t) + RS_WARPS * RADIX * 4 + 2 * RADIX * 4 + 32 * 4;
}
constexpr int RS_MAX_PASSES = 8;
constexpr size_t rs_hist_smem_bytes(int npasses) { return (size_t)RS_WARPS * npasses * RADIX * 4; }

}  // namespace

template <class TIn, class TOut>
arbx_status exclusive_scan(const TIn* in, TOut* out, int64_t n, cudaStream_t s) {
  return scan_impl<TIn, TOut>(in, out, n, true, s);
}

template arbx_status exclusive_scan<int32_t, int64_t>(const int32_t*, int64_t*, int64_t, cudaStream_t);
template arbx_status exclusive_scan<uint32_t, uint32_t>(const uint32_t*, uint32_t*, int64_t, cudaStream_t);

int64_t scan_temp_elems(int64_t n) {
  int64_t total = 0;
  for (int64_t level = n; level > SCAN_TILE;) {
    const int64_t tiles = (level + SCAN_TILE - 1) / SCAN_TILE;
    total += 2 * tiles + 1;
    level = tiles;
  }
  return total;
}

arbx_status exclusive_scan_temp(const int32_t* in, int64_t* out, int64_t n, int64_t* temp, cudaStream_t s) {
  if (n <= 0) {
    ARBX_CUDA(cudaMemsetAsync(out, 0, sizeof(int64_t), s));
    return ARBX_OK;
  }
  const int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
  if (tiles == 1) {
    ARBX_LAUNCH("scan_tiles", s, k_scan_tiles<int32_t, int64_t><<<1, SCAN_THREADS, 0, s>>>(in, out, n, nullptr, true));
    return ARBX_OK;
  }
  // level 1: per-tile totals, then their exclusive scan (recursively, in the
  // rest of the temporary), then the per-tile scans offset by it
  int64_t* totals = temp;
  int64_t* offs = temp + tiles;
  int64_t* rest = offs + tiles + 1;
  ARBX_LAUNCH("scan_tile_totals", s,
              k_scan_tile_totals<int32_t, int64_t><<<(unsigned)tiles, SCAN_THREADS, 0, s>>>(in, n, totals));
  int64_t level = tiles;
  const int64_t* lin = totals;
  int64_t* lout = offs;
  // scan the int64 totals level by level (each level again by tiles)
  std::vector<std::pair<const int64_t*, int64_t*>> pending;
  std::vector<int64_t> sizes;
  while (level > SCAN_TILE) {
    const int64_t t2 = (level + SCAN_TILE - 1) / SCAN_TILE;
    int64_t* tot2 = rest;
    int64_t* off2 = rest + t2;
    rest = off2 + t2 + 1;
    ARBX_LAUNCH("scan_tile_totals", s,
                k_scan_tile_totals<int64_t, int64_t><<<(unsigned)t2, SCAN_THREADS, 0, s>>>(lin, level, tot2));
    pending.push_back({lin, lout});
    sizes.push_back(level);
    lin = tot2;
    lout = off2;
    level = t2;
  }
  ARBX_LAUNCH("scan_tiles", s, k_scan_tiles<int64_t, int64_t><<<1, SCAN_THREADS, 0, s>>>(lin, lout, level, nullptr, false));
  for (int i = (int)pending.size() - 1; i >= 0; --i) {
    const int64_t lv = sizes[i];
    const int64_t t2 = (lv + SCAN_TILE - 1) / SCAN_TILE;
    ARBX_LAUNCH("scan_tiles", s,
                k_scan_tiles<int64_t, int64_t><<<(unsigned)t2, SCAN_THREADS, 0, s>>>(pending[i].first, pending[i].second, lv,
                                                                                     lout, false));
    lout = pending[i].second;
  }
  ARBX_LAUNCH("scan_tiles", s,
              k_scan_tiles<int32_t, int64_t><<<(unsigned)tiles, SCAN_THREADS, 0, s>>>(in, out, n, offs, true));
  return ARBX_OK;
}

int64_t scan_prealloc_max() { return (int64_t)SCAN_TILE * SCAN_TILE; }

arbx_status exclusive_scan_prealloc(const int32_t* in, int64_t* out, int64_t n, int64_t* totals, int64_t* offs,
                                    int64_t cap, cudaStream_t s) {
  if (n <= 0) {
    ARBX_CUDA(cudaMemsetAsync(out, 0, sizeof(int64_t), s));
    return ARBX_OK;
  }
  if (n > scan_prealloc_max()) return ARBX_ERR_UNSUPPORTED;
  const int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
  if (tiles + 1 > cap) return ARBX_ERR_CAPACITY;
  if (tiles == 1) {
    ARBX_LAUNCH("scan_tiles", s, k_scan_tiles<int32_t, int64_t><<<1, SCAN_THREADS, 0, s>>>(in, out, n, nullptr, true));
    return ARBX_OK;
  }
  // tiles <= SCAN_TILE: the tile totals are scanned by one block
  ARBX_LAUNCH("scan_tile_totals", s,
              k_scan_tile_totals<int32_t, int64_t><<<(unsigned)tiles, SCAN_THREADS, 0, s>>>(in, n, totals));
  ARBX_LAUNCH("scan_tiles", s, k_scan_tiles<int64_t, int64_t><<<1, SCAN_THREADS, 0, s>>>(totals, offs, tiles, nullptr, false));
  ARBX_LAUNCH("scan_tiles", s,
              k_scan_tiles<int32_t, int64_t><<<(unsigned)tiles, SCAN_THREADS, 0, s>>>(in, out, n, offs, true));
  return ARBX_OK;
}

// Tiles of one resident wave of k_rs_pass blocks (three 256-thread blocks per
// SM for 64-bit keys): up to this many the single-launch look-back pass is
// used, above it the reduce-then-scan pass.  Measured, 10M 64-bit keys: 149
// us per look-back pass (the look-back waits on tiles of blocks that are
// still ranking) vs 103 us for the scattering launch of a reduce-then-scan
// pass; for small sorts the look-back pass saves three of four launches.
template <class K>
int64_t rs_lookback_max_tiles() {
  static int per_sm = 0;
  if (per_sm == 0) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_rs_pass<K, true>, RS_THREADS, rs_smem_bytes<K>()) !=
        cudaSuccess)
      b = 1;
    per_sm = std::max(1, b);
  }
  return (int64_t)per_sm * num_sms();
}

template <class K>
arbx_status radix_sort_pairs(K* keys, uint32_t* vals, K* keys_alt, uint32_t* vals_alt, int64_t n,
                             int begin_bit, int end_bit, bool* in_alt, cudaStream_t s) {
  *in_alt = false;
  if (n <= 1 || end_bit <= begin_bit) return ARBX_OK;
  if (n > (int64_t)INT32_MAX) return ARBX_ERR_UNSUPPORTED;  // 32-bit digit starts
  const int64_t tiles64 = (n + RS_TILE - 1) / RS_TILE;
  if (tiles64 * RADIX >= (int64_t(1) << 31)) return ARBX_ERR_UNSUPPORTED;
  const uint32_t tiles = (uint32_t)tiles64;
  const int npasses = (end_bit - begin_bit + 7) / 8;
  if (npasses > RS_MAX_PASSES) return ARBX_ERR_UNSUPPORTED;
  {
    // the attribute is per function and device; set it once (host threads share it)
    static std::mutex mu;
    static bool set_on[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    if (dev >= 0 && dev < 64 && !set_on[dev]) {
      ARBX_CUDA(cudaFuncSetAttribute(k_rs_pass<K, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)rs_smem_bytes<K>()));
      ARBX_CUDA(cudaFuncSetAttribute(k_rs_pass<K, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)rs_smem_bytes<K>()));
      ARBX_CUDA(cudaFuncSetAttribute(k_rs_hist<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)rs_hist_smem_bytes(RS_MAX_PASSES)));
      set_on[dev] = true;
    }
  }
  K* kin = keys;
  uint32_t* vin = vals;
  K* kout = keys_alt;
  uint32_t* vout = vals_alt;
  bool alt = false;
  if (tiles64 <= rs_lookback_max_tiles<K>()) {
    uint32_t* err = nullptr;
    ARBX_TRY(device_error_word(&err));
    // one zeroed block of 8-byte words: the status words of every pass's
    // tiles, then per pass its 256 global digit counts (pass p at p * 256,
    // contiguous for the histogram kernel) and its tile counter (32-bit)
    const size_t nstatus = (size_t)npasses * tiles * RADIX;
    const size_t nwords = nstatus + ((size_t)npasses * (RADIX + 1) + 1) / 2;
    DevTemp<unsigned long long> work(s);
    ARBX_TRY(work.alloc(nwords));
    ARBX_CUDA(cudaMemsetAsync(work.p, 0, nwords * sizeof(unsigned long long), s));
    unsigned long long* status = work.p;
    uint32_t* ghist = reinterpret_cast<uint32_t*>(work.p + nstatus);
    uint32_t* counters = ghist + (size_t)npasses * RADIX;
    const int hgrid = (int)std::min<int64_t>((n + RS_THREADS - 1) / RS_THREADS, (int64_t)2 * num_sms());
    ARBX_LAUNCH("radix_hist", s,
                k_rs_hist<K><<<hgrid, RS_THREADS, rs_hist_smem_bytes(npasses), s>>>(keys, n, begin_bit, npasses, ghist));
    for (int p = 0; p < npasses; ++p) {
      ARBX_LAUNCH("radix_pass", s,
                  (k_rs_pass<K, true><<<tiles, RS_THREADS, rs_smem_bytes<K>(), s>>>(
                      kin, vin, kout, vout, n, begin_bit + 8 * p, nullptr, tiles, ghist + (size_t)p * RADIX,
                      status + (size_t)p * tiles * RADIX, counters + p, err)));
      std::swap(kin, kout);
      std::swap(vin, vout);
      alt = !alt;
    }
    *in_alt = alt;
    return ARBX_OK;
  }
  DevTemp<uint32_t> hist(s), starts(s);
  ARBX_TRY(hist.alloc((size_t)tiles * RADIX));
  ARBX_TRY(starts.alloc((size_t)tiles * RADIX + 1));
  for (int shift = begin_bit; shift < end_bit; shift += 8) {
    ARBX_LAUNCH("radix_upsweep", s, k_rs_upsweep<K><<<tiles, RS_THREADS, 0, s>>>(kin, n, shift, tiles, hist.p));
    ARBX_TRY((exclusive_scan<uint32_t, uint32_t>(hist.p, starts.p, (int64_t)tiles * RADIX, s)));
    ARBX_LAUNCH("radix_downsweep", s,
                (k_rs_pass<K, false><<<tiles, RS_THREADS, rs_smem_bytes<K>(), s>>>(
                    kin, vin, kout, vout, n, shift, starts.p, tiles, nullptr, nullptr, nullptr, nullptr)));
    std::swap(kin, kout);
    std::swap(vin, vout);
    alt = !alt;
  }
  *in_alt = alt;
  return ARBX_OK;
}

template arbx_status radix_sort_pairs<uint32_t>(uint32_t*, uint32_t*, uint32_t*, uint32_t*, int64_t, int, int, bool*, cudaStream_t);
template arbx_status radix_sort_pairs<uint64_t>(uint64_t*, uint32_t*, uint64_t*, uint32_t*, int64_t, int, int, bool*, cudaStream_t);

}  // namespace arbx
