// Linear BVH construction (ArborX 2.0, section 2.6: 64-bit Morton codes,
// Apetrei's bottom-up construction in place of Karras', sorting of the codes).
//
// Pipeline, all on the caller's stream:
//   1. k_bounds / k_bounds_final  scene box of all primitives (exact min/max)
//                                 and a finiteness check of every coordinate
//   2. k_morton                   interleaved cell codes of the primitive
//                                 centroids in the scene box (64 bits: 21 per
//                                 axis in 3D, 32 in 2D, 10 in 6D)
//   3. radix_sort_pairs           (code, index) in code order, stable
//   4. k_gather                   primitives in sorted order
//   5. k_apetrei_chunks,          a climb from every leaf, handed off in shared
//      k_apetrei_global           memory inside chunks of sorted leaves and in
//                                 global memory across them; the hierarchy is
//                                 the binary radix tree of the sorted codes
//                                 (ties between equal codes broken by the
//                                 index, Karras 2012), built bottom-up with an
//                                 atomic handoff and box refit (Apetrei 2014)
//   6. k_top_levels               BFS copy of the top nodes for shared memory
//   7. k_quantize (optional)      16-bit child boxes relative to each node
//
// Node numbering: internal node g is the node whose split lies between sorted
// leaves g and g+1 (Apetrei's numbering); its children cover [l, g] and
// [g+1, r].  The root is the node covering [0, n-1], recorded by the thread
// that completes it.
#include <cstddef>
#include <mutex>

#include "build.cuh"
#include "primitives.cuh"

namespace arbx {
namespace {

constexpr int BUILD_THREADS = 256;

__device__ __forceinline__ bool finite_bits(float x) {
  return (__float_as_uint(x) & 0x7f800000u) != 0x7f800000u;
}

// Per-primitive bounding box.  Points: the point.  Boxes: lo, hi.
// Triangles: per-axis min/max of the three vertices.
template <int D, int KIND>
__device__ __forceinline__ void prim_box(const float* __restrict__ data, int64_t i, float* lo, float* hi) {
  if (KIND == ARBX_POINT) {
#pragma unroll
    for (int a = 0; a < D; ++a) lo[a] = hi[a] = data[i * D + a];
  } else if (KIND == ARBX_BOX) {
#pragma unroll
    for (int a = 0; a < D; ++a) {
      lo[a] = data[i * 2 * D + a];
      hi[a] = data[i * 2 * D + D + a];
    }
  } else {
    const float* t = data + i * 9;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      lo[a] = fminf(fminf(t[a], t[3 + a]), t[6 + a]);
      hi[a] = fmaxf(fmaxf(t[a], t[3 + a]), t[6 + a]);
    }
  }
}

template <int D, int KIND>
__device__ __forceinline__ bool prim_finite(const float* __restrict__ data, int64_t i) {
  constexpr int W = KIND == ARBX_POINT ? D : (KIND == ARBX_BOX ? 2 * D : 9);
  bool ok = true;
#pragma unroll
  for (int a = 0; a < W; ++a) ok = ok && finite_bits(data[i * W + a]);
  return ok;
}

// Grid-stride min/max; one partial box per block.
template <int D, int KIND>
__global__ void __launch_bounds__(BUILD_THREADS) k_bounds(const float* __restrict__ data, int64_t n,
                                                          float* __restrict__ partial, uint32_t* __restrict__ err) {
  __shared__ float s_lo[BUILD_THREADS / 32][D], s_hi[BUILD_THREADS / 32][D];
  float lo[D], hi[D];
#pragma unroll
  for (int a = 0; a < D; ++a) {
    lo[a] = __int_as_float(0x7f800000);
    hi[a] = -__int_as_float(0x7f800000);
  }
  bool ok = true;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    ok = ok && prim_finite<D, KIND>(data, i);
    float plo[D], phi[D];
    prim_box<D, KIND>(data, i, plo, phi);
#pragma unroll
    for (int a = 0; a < D; ++a) {
      lo[a] = fminf(lo[a], plo[a]);
      hi[a] = fmaxf(hi[a], phi[a]);
    }
  }
  if (!ok) atomicOr(err, DEVERR_NONFINITE);
#pragma unroll
  for (int a = 0; a < D; ++a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      lo[a] = fminf(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
      hi[a] = fmaxf(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
#pragma unroll
    for (int a = 0; a < D; ++a) { s_lo[warp][a] = lo[a]; s_hi[warp][a] = hi[a]; }
  }
  __syncthreads();
  if (threadIdx.x < D) {
    float l = s_lo[0][threadIdx.x], h = s_hi[0][threadIdx.x];
    for (int w = 1; w < BUILD_THREADS / 32; ++w) {
      l = fminf(l, s_lo[w][threadIdx.x]);
      h = fmaxf(h, s_hi[w][threadIdx.x]);
    }
    partial[blockIdx.x * 2 * D + threadIdx.x] = l;
    partial[blockIdx.x * 2 * D + D + threadIdx.x] = h;
  }
}

// The same for points whose coordinates start on a 16-byte boundary: the
// coordinates read as a flat float4 array in groups of G = D / gcd(4, D)
// float4s, in which float c of float4 j belongs to axis (4j + c) mod D; the
// floats after the last whole group are read one by one.  Each thread keeps
// G independent 16-byte loads in flight.
template <int D>
__global__ void __launch_bounds__(BUILD_THREADS) k_bounds_vec(const float* __restrict__ data, int64_t nfloats,
                                                              float* __restrict__ partial, uint32_t* __restrict__ err) {
  constexpr int G = D % 4 == 0 ? D / 4 : (D % 2 == 0 ? D / 2 : D);
  __shared__ float s_lo[BUILD_THREADS / 32][D], s_hi[BUILD_THREADS / 32][D];
  float lo[D], hi[D];
#pragma unroll
  for (int a = 0; a < D; ++a) {
    lo[a] = __int_as_float(0x7f800000);
    hi[a] = -__int_as_float(0x7f800000);
  }
  bool ok = true;
  const float4* __restrict__ d4 = reinterpret_cast<const float4*>(data);
  const int64_t ngroups = nfloats / (4 * G);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t gi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; gi < ngroups; gi += stride) {
    float4 v[G];
#pragma unroll
    for (int j = 0; j < G; ++j) v[j] = __ldg(d4 + gi * G + j);
#pragma unroll
    for (int j = 0; j < G; ++j) {
      const float f[4] = {v[j].x, v[j].y, v[j].z, v[j].w};
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int a = (4 * j + c) % D;
        ok = ok && finite_bits(f[c]);
        lo[a] = fminf(lo[a], f[c]);
        hi[a] = fmaxf(hi[a], f[c]);
      }
    }
  }
  for (int64_t f = ngroups * 4 * G + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < nfloats; f += stride) {
    const float x = data[f];
    const int a = (int)(f % D);
    ok = ok && finite_bits(x);
#pragma unroll
    for (int b = 0; b < D; ++b) {
      if (b == a) {
        lo[b] = fminf(lo[b], x);
        hi[b] = fmaxf(hi[b], x);
      }
    }
  }
  if (!ok) atomicOr(err, DEVERR_NONFINITE);
#pragma unroll
  for (int a = 0; a < D; ++a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      lo[a] = fminf(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
      hi[a] = fmaxf(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
#pragma unroll
    for (int a = 0; a < D; ++a) { s_lo[warp][a] = lo[a]; s_hi[warp][a] = hi[a]; }
  }
  __syncthreads();
  if (threadIdx.x < D) {
    float l = s_lo[0][threadIdx.x], h = s_hi[0][threadIdx.x];
    for (int w = 1; w < BUILD_THREADS / 32; ++w) {
      l = fminf(l, s_lo[w][threadIdx.x]);
      h = fmaxf(h, s_hi[w][threadIdx.x]);
    }
    partial[blockIdx.x * 2 * D + threadIdx.x] = l;
    partial[blockIdx.x * 2 * D + D + threadIdx.x] = h;
  }
}

// Reduce the partial boxes; write the scene box (lo, hi) and the Morton
// frame (lo, scale) with scale = 2^bits / extent (0 for a flat axis).
template <int D>
__global__ void k_bounds_final(const float* __restrict__ partial, int nparts, float* __restrict__ scene,
                               float* __restrict__ frame, int bits) {
  const int a = threadIdx.x;
  if (a >= D) return;
  float l = __int_as_float(0x7f800000), h = -__int_as_float(0x7f800000);
  for (int p = 0; p < nparts; ++p) {
    l = fminf(l, partial[p * 2 * D + a]);
    h = fmaxf(h, partial[p * 2 * D + D + a]);
  }
  scene[a] = l;
  scene[D + a] = h;
  const float ext = h - l;
  frame[a] = l;
  frame[D + a] = ext > 0.0f ? (float)(1ull << bits) / ext : 0.0f;
}

// Morton code of the primitive's box centre.  Only the tree's shape depends
// on these codes, never a result.
template <int D, int KIND>
__global__ void __launch_bounds__(BUILD_THREADS) k_morton(const float* __restrict__ data, int64_t n,
                                                          const float* __restrict__ frame, int bits,
                                                          uint64_t* __restrict__ keys, uint32_t* __restrict__ vals) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float lo[D], hi[D];
  prim_box<D, KIND>(data, i, lo, hi);
  const uint32_t cmax = (uint32_t)((1ull << bits) - 1);
  uint32_t cell[D];
#pragma unroll
  for (int a = 0; a < D; ++a) {
    const float c = KIND == ARBX_POINT ? lo[a] : 0.5f * (lo[a] + hi[a]);
    float u = (c - frame[a]) * frame[D + a];
    u = fmaxf(u, 0.0f);
    cell[a] = u >= (float)cmax ? cmax : (uint32_t)u;
  }
  uint64_t code = 0;
  for (int b = bits - 1; b >= 0; --b) {
#pragma unroll
    for (int a = 0; a < D; ++a) code = (code << 1) | ((cell[a] >> b) & 1u);
  }
  keys[i] = code;
  vals[i] = (uint32_t)i;
}

// Sorted primitive boxes (points: the coordinates; boxes: lo, hi) or, for
// triangles, sorted leaf records holding the vertices and input index.
template <int D, int KIND>
__global__ void __launch_bounds__(BUILD_THREADS) k_gather(const float* __restrict__ data, int64_t n,
                                                          const uint32_t* __restrict__ perm,
                                                          float* __restrict__ sorted_box, TriLeaf* __restrict__ leaves) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t j = perm[i];
  float lo[D], hi[D];
  prim_box<D, KIND>(data, j, lo, hi);
#pragma unroll
  for (int a = 0; a < D; ++a) {
    sorted_box[i * 2 * D + a] = lo[a];
    sorted_box[i * 2 * D + D + a] = hi[a];
  }
  if (KIND == ARBX_TRIANGLE) {
    TriLeaf L;
#pragma unroll
    for (int k = 0; k < 9; ++k) L.v[k] = data[j * 9 + k];
    L.orig = (int32_t)j;
    L.pad[0] = L.pad[1] = 0;
    leaves[i] = L;
  }
}

// delta(i) for 0 <= i < n-1: length of the common prefix of the augmented
// keys (code_i, i) and (code_{i+1}, i+1).
__device__ __forceinline__ int delta(const uint64_t* __restrict__ keys, int i) {
  const uint64_t a = keys[i], b = keys[i + 1];
  return a != b ? __clzll((long long)(a ^ b)) : 64 + __clz((int)((uint32_t)i ^ (uint32_t)(i + 1)));
}

// Apetrei's construction.  A climb starts at a leaf i with range [l, r] = [i, i].
// The parent of a node covering [l, r] is split r (the node is its left child)
// when l == 0 or r < n-1 and delta(r) > delta(l-1); otherwise it is split l-1
// (the node is its right child).  The child writes its box, code and input
// index into its half of the parent and exchanges its far range end into the
// parent's flag: the first arriver stops; the second takes the sibling's
// box, merges it with its own and climbs on.
//
// Two kernels.  k_apetrei_chunks: each block takes chunks of AP_CHUNK
// consecutive sorted leaves, and a node whose two children both lie inside the
// chunk (its range does) is handed off in shared memory: the chunk's keys,
// flags and the arriving children's boxes are kept there, so such a step waits
// on no global memory (each child still writes its half of the node there).
// (Keeping the chunk's whole nodes in shared memory and writing them out
// together at the chunk's end measured slower: 0.59 vs 0.53 ms at 10M.)  An arrival whose parent's split is at the chunk's edge,
// or that arrived first at a node whose other child never came (its subtree
// reaches outside the chunk), is written to a list.  k_apetrei_global takes
// the listed arrivals and completes the remaining nodes -- those whose range
// crosses a chunk boundary, a root path per boundary -- with the handoff in
// global memory (release: the half is visible first; acquire: the sibling's
// half is visible after; halves written and read as 8-byte pairs past L1).
// The tree does not depend on which arrival comes first.
constexpr int AP_CHUNK = 512;      // sorted leaves per chunk
constexpr int AP_THREADS = 256;    // k_apetrei_chunks block (8 warps of AP_CHUNK / 8 leaves)

// The listed arrivals: parent split g and the child's far range end v (its
// range is [v, g] when v <= g, the left child; [g+1, v] otherwise).
struct ApArrival {
  int32_t g, v;
};

template <int D>
constexpr size_t ap_smem_bytes() {
  return (size_t)(AP_CHUNK + 2) * sizeof(uint64_t) + (size_t)(AP_CHUNK - 1) * (sizeof(int32_t) + 4 * D * sizeof(float));
}

// Upper bound on the listed arrivals: only nodes whose range crosses a chunk
// boundary get them, at most two each; the nodes crossing one boundary lie on
// one root path, at most 97 deep (63-bit codes, 32-bit index tie-breaks).
inline int64_t ap_list_cap(int64_t n) {
  const int64_t chunks = (n + AP_CHUNK - 1) / AP_CHUNK;
  return std::min<int64_t>(2 * n, 2 * 97 * chunks + 2);
}

template <int D>
__device__ __forceinline__ void ap_write_half(Node<D>* p, bool left, const float* lo, const float* hi, int32_t code,
                                              int32_t orig) {
  static_assert(offsetof(Node<D>, lo1) == 2 * D * sizeof(float), "halves: lo0 hi0 | lo1 hi1");
  float box[2 * D];
#pragma unroll
  for (int a = 0; a < D; ++a) {
    box[a] = lo[a];
    box[D + a] = hi[a];
  }
  float2* mine = reinterpret_cast<float2*>(left ? p->lo0 : p->lo1);  // lo[D] then hi[D]
#pragma unroll
  for (int j = 0; j < D; ++j) __stcg(mine + j, make_float2(box[2 * j], box[2 * j + 1]));
  __stcg(&p->child[left ? 0 : 1], code);
  __stcg(&p->orig[left ? 0 : 1], orig);
}

template <int D>
__device__ __forceinline__ void ap_read_half(const Node<D>* p, bool left, float* lo, float* hi) {
  const float2* h = reinterpret_cast<const float2*>(left ? p->lo0 : p->lo1);
  float box[2 * D];
#pragma unroll
  for (int j = 0; j < D; ++j) {
    const float2 v = __ldcg(h + j);
    box[2 * j] = v.x;
    box[2 * j + 1] = v.y;
  }
#pragma unroll
  for (int a = 0; a < D; ++a) {
    lo[a] = box[a];
    hi[a] = box[D + a];
  }
}

__device__ __forceinline__ void ap_list(ApArrival* list, unsigned int* count, int64_t cap, int32_t g, int32_t v,
                                        uint32_t* err) {
  const unsigned int at = atomicAdd(count, 1u);
  if ((int64_t)at < cap) list[at] = ApArrival{g, v};
  else atomicOr(err, DEVERR_INTERNAL);
}

// Lane refill in both kernels: a warp owns a contiguous range of work items
// (leaves, listed arrivals) and a lane whose climb has ended takes the warp's
// next item in the same iteration, so a warp does not wait, batch by batch,
// for the longest of 32 climbs.  Every iteration of a busy lane is one
// arrival, so the loops end.
template <int D>
__global__ void __launch_bounds__(AP_THREADS) k_apetrei_chunks(const uint64_t* __restrict__ keys,
                                                              const uint32_t* __restrict__ perm,
                                                              const float* __restrict__ sorted_box, int n,
                                                              Node<D>* nodes, int32_t* __restrict__ root_out,
                                                              ApArrival* __restrict__ list, unsigned int* count,
                                                              int64_t cap, uint32_t* __restrict__ err) {
  extern __shared__ __align__(16) unsigned char ap_smem[];
  uint64_t* s_keys = reinterpret_cast<uint64_t*>(ap_smem);                   // keys[c0-1 .. c0+AP_CHUNK]
  int32_t* s_flag = reinterpret_cast<int32_t*>(s_keys + AP_CHUNK + 2);       // split g at g - c0
  float* s_box = reinterpret_cast<float*>(s_flag + AP_CHUNK - 1);           // [split][side][lo D, hi D]
  const unsigned FULL = 0xffffffffu;
  const int lane = (int)(threadIdx.x & 31u), warp = (int)(threadIdx.x >> 5);
  constexpr int PER_WARP = AP_CHUNK / (AP_THREADS / 32);
  const int64_t nchunks = ((int64_t)n + AP_CHUNK - 1) / AP_CHUNK;
  for (int64_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
    const int c0 = (int)(ch * AP_CHUNK);
    const int c1 = (int)std::min<int64_t>((int64_t)n, (int64_t)c0 + AP_CHUNK);  // leaves [c0, c1)
    for (int j = threadIdx.x; j < AP_CHUNK + 2; j += AP_THREADS) {
      const int64_t gj = (int64_t)c0 - 1 + j;
      if (gj >= 0 && gj < n) s_keys[j] = keys[gj];
    }
    for (int j = threadIdx.x; j < AP_CHUNK - 1; j += AP_THREADS) s_flag[j] = -1;
    __syncthreads();
    // delta(i) of the chunk's keys: i in [c0-1, c1-1], i+1 < n
    auto sdelta = [&](int i) {
      const uint64_t x = s_keys[i - c0 + 1], y = s_keys[i - c0 + 2];
      return x != y ? __clzll((long long)(x ^ y)) : 64 + __clz((int)((uint32_t)i ^ (uint32_t)(i + 1)));
    };
    const int w1 = std::min(c1, c0 + (warp + 1) * PER_WARP);
    int next = c0 + warp * PER_WARP;  // the warp's next unclaimed leaf (the same in every lane)
    bool busy = false;
    float lo[D], hi[D];
    int l = 0, r = 0;
    int32_t code = 0, orig = 0;
    for (;;) {
      const unsigned freem = __ballot_sync(FULL, !busy);
      if (freem != 0u && next < w1) {
        if (!busy) {
          const int i = next + __popc(freem & ((1u << lane) - 1u));
          if (i < w1) {
#pragma unroll
            for (int a = 0; a < D; ++a) {
              lo[a] = sorted_box[(int64_t)i * 2 * D + a];
              hi[a] = sorted_box[(int64_t)i * 2 * D + D + a];
            }
            l = r = i;
            code = ~(int32_t)i;
            orig = (int32_t)perm[i];
            busy = true;
          }
        }
        next += __popc(freem);
      }
      if (!__any_sync(FULL, busy)) break;
      if (!busy) continue;
      const bool left = (l == 0) || (r != n - 1 && sdelta(r) > sdelta(l - 1));
      const int g = left ? r : l - 1;
      ap_write_half(nodes + g, left, lo, hi, code, orig);
      // both leaves of split g in the chunk (c0 <= g and g + 1 < c1): the
      // sibling, if its range lies in the chunk too, arrives through shared memory
      if (left ? r >= c1 - 1 : l <= c0) {
        ap_list(list, count, cap, g, left ? l : r, err);
        busy = false;
        continue;
      }
      float* mine = s_box + ((size_t)(g - c0) * 2 + (left ? 0 : 1)) * 2 * D;
#pragma unroll
      for (int a = 0; a < D; ++a) {
        mine[a] = lo[a];
        mine[D + a] = hi[a];
      }
      __threadfence_block();
      const int other = atomicExch(s_flag + (g - c0), left ? l : r);
      __threadfence_block();
      if (other < 0) {  // first arriver: the sibling finishes this node (here or in k_apetrei_global)
        busy = false;
        continue;
      }
      s_flag[g - c0] = -2;  // both children arrived
      const float* sib = s_box + ((size_t)(g - c0) * 2 + (left ? 1 : 0)) * 2 * D;
#pragma unroll
      for (int a = 0; a < D; ++a) {
        lo[a] = fminf(lo[a], sib[a]);
        hi[a] = fmaxf(hi[a], sib[D + a]);
      }
      if (left) r = other; else l = other;
      code = g;
      orig = r;  // an internal child's orig slot holds its range end (stackless traversal)
      if (l == 0 && r == n - 1) {
        *root_out = g;
        busy = false;
      }
    }
    __syncthreads();
    // a first arrival whose sibling never came: the sibling's range reaches
    // outside the chunk, so the node is completed in global memory
    for (int j = threadIdx.x; j < c1 - c0 - 1; j += AP_THREADS) {
      const int v = s_flag[j];
      if (v >= 0) ap_list(list, count, cap, c0 + j, v, err);
    }
    __syncthreads();  // the shared arrays are reused by the next chunk
  }
}

template <int D>
__global__ void __launch_bounds__(BUILD_THREADS) k_apetrei_global(const uint64_t* __restrict__ keys, int n,
                                                                  const ApArrival* __restrict__ list,
                                                                  const unsigned int* __restrict__ count, int64_t cap,
                                                                  int32_t* __restrict__ flags, Node<D>* nodes,
                                                                  int32_t* __restrict__ root_out) {
  const unsigned FULL = 0xffffffffu;
  const int lane = (int)(threadIdx.x & 31u);
  const int64_t total = std::min<int64_t>((int64_t)*count, cap);
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
  const int64_t per_warp = (total + warps - 1) / warps;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t wend = std::min<int64_t>(total, (warp + 1) * per_warp);
  int64_t next = warp * per_warp;  // the warp's next unclaimed arrival (the same in every lane)
  bool busy = false, written = false, left = false;
  float lo[D], hi[D];
  int l = 0, r = 0, g = 0;
  int32_t code = 0, orig = 0;
  for (;;) {
    const unsigned freem = __ballot_sync(FULL, !busy);
    if (freem != 0u && next < wend) {
      if (!busy) {
        const int64_t i = next + __popc(freem & ((1u << lane) - 1u));
        if (i < wend) {
          // a listed arrival: its half of node g is written already
          const ApArrival e = list[i];
          g = e.g;
          left = e.v <= g;
          l = left ? e.v : g + 1;
          r = left ? g : e.v;
          ap_read_half(nodes + g, left, lo, hi);
          written = true;
          busy = true;
        }
      }
      next += __popc(freem);
    }
    if (!__any_sync(FULL, busy)) break;
    if (!busy) continue;
    if (!written) {
      left = (l == 0) || (r != n - 1 && delta(keys, r) > delta(keys, l - 1));
      g = left ? r : l - 1;
      ap_write_half(nodes + g, left, lo, hi, code, orig);
    }
    written = false;
    const int other = exch_acq_rel(flags + g, left ? l : r);
    if (other < 0) {  // first arriver: the sibling finishes this node
      busy = false;
      continue;
    }
    float slo[D], shi[D];
    ap_read_half(nodes + g, !left, slo, shi);
#pragma unroll
    for (int a = 0; a < D; ++a) {
      lo[a] = fminf(lo[a], slo[a]);
      hi[a] = fmaxf(hi[a], shi[a]);
    }
    if (left) r = other; else l = other;
    code = g;
    orig = r;
    if (l == 0 && r == n - 1) {
      *root_out = g;
      busy = false;
    }
  }
}

// One-leaf tree: a pseudo root whose first child is leaf 0 and whose second
// child is NULL_CHILD.
template <int D>
__global__ void k_single(const float* __restrict__ sorted_box, Node<D>* nodes, int32_t* root_out) {
  Node<D> nd;
#pragma unroll
  for (int a = 0; a < D; ++a) {
    nd.lo0[a] = sorted_box[a];
    nd.hi0[a] = sorted_box[D + a];
    nd.lo1[a] = __int_as_float(0x7f800000);
    nd.hi1[a] = -__int_as_float(0x7f800000);
  }
  nd.child[0] = ~0;
  nd.child[1] = NULL_CHILD;
  nd.orig[0] = 0;
  nd.orig[1] = -1;
  nodes[0] = nd;
  *root_out = 0;
}

// BFS copy of the top `cap` internal nodes, level by level with a block scan
// (deterministic order).  Children that made it into the copy are re-coded
// TOP_FLAG | local index.  One block of 1024 threads; cap <= 1023.
template <class NodeT>
__global__ void __launch_bounds__(1024) k_top_levels(const NodeT* __restrict__ nodes, const int32_t* __restrict__ root,
                                                     int cap, NodeT* __restrict__ top, int32_t* __restrict__ count_out) {
  __shared__ int32_t s_global[1024];  // global index of each copied node
  __shared__ int32_t s_scan[1024];
  __shared__ int32_t s_count;
  const int t = threadIdx.x;
  if (t == 0) {
    s_global[0] = *root;
    s_count = 1;
  }
  __syncthreads();
  int level_begin = 0, level_end = 1;
  while (level_begin < level_end) {
    const int me = level_begin + t;
    NodeT nd;
    int nint = 0;
    if (me < level_end) {
      nd = nodes[s_global[me]];
      nint = (nd.child[0] >= 0) + (nd.child[1] >= 0);
    }
    s_scan[t] = nint;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {  // inclusive scan
      const int v = t >= o ? s_scan[t - o] : 0;
      __syncthreads();
      s_scan[t] += v;
      __syncthreads();
    }
    const int base = s_count;
    if (me < level_end) {
      int slot = base + s_scan[t] - nint;
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        if (nd.child[c] >= 0) {
          if (slot < cap) {
            s_global[slot] = nd.child[c];
            nd.child[c] = TOP_FLAG | slot;
          }
          ++slot;
        }
      }
      top[me] = nd;
    }
    __syncthreads();
    const int total = s_scan[1023];
    __syncthreads();
    if (t == 0) s_count = min(cap, base + total);
    __syncthreads();
    level_begin = level_end;
    level_end = s_count;
  }
  if (t == 0) *count_out = s_count;
}

// 16-bit quantization of the child boxes of every internal node relative to
// the node's own box [L, H] (the union of its children):
//   step_a = 2^e_a, the smallest power of two with 65535 * step_a >= fl_up(H_a - L_a)
//   lo code = floor(fl_down(c_lo - L) / step), hi code = ceil(fl_up(c_hi - L) / step)
//   decode: lo = fl_down(L + q*step), hi = fl_up(L + q*step)   (q*step is exact: one
//   fused multiply-add with directed rounding)
// so decoded lo <= exact child lo and decoded hi >= exact child hi: culling
// stays conservative.  The encoder re-checks each code with the same decode
// used by the traversal.
__device__ __forceinline__ float q_decode_lo(float origin, int q, float step) {
  return __fmaf_rd((float)q, step, origin);
}
__device__ __forceinline__ float q_decode_hi(float origin, int q, float step) {
  return __fmaf_ru((float)q, step, origin);
}

__global__ void __launch_bounds__(BUILD_THREADS) k_quantize(const Node<3>* __restrict__ nodes, int64_t count,
                                                            QNode* __restrict__ qnodes, uint32_t* __restrict__ err) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= count) return;
  const Node<3> nd = nodes[g];
  QNode qn;
  const bool has1 = nd.child[1] != NULL_CHILD;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float L = has1 ? fminf(nd.lo0[a], nd.lo1[a]) : nd.lo0[a];
    const float H = has1 ? fmaxf(nd.hi0[a], nd.hi1[a]) : nd.hi0[a];
    const float ext = __fsub_ru(H, L);
    int e = -126;
    if (ext > 0.0f) {
      int E = ((__float_as_int(ext) >> 23) & 0xff) - 127;  // ext >= 2^E
      e = max(-126, E - 16);
      while (65535.0f * pow2f(e) < ext) ++e;
    }
    const float step = pow2f(e);
    qn.origin[a] = L;
    qn.exps[a] = (int8_t)max(-128, min(127, e));
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const float clo = c == 0 ? nd.lo0[a] : (has1 ? nd.lo1[a] : L);
      const float chi = c == 0 ? nd.hi0[a] : (has1 ? nd.hi1[a] : L);
      int ql = (int)floorf(__fmul_rn(__fsub_rd(clo, L), pow2f(-e)));
      int qh = (int)ceilf(__fmul_rn(__fsub_ru(chi, L), pow2f(-e)));
      ql = max(0, min(65535, ql));
      qh = max(0, min(65535, qh));
      while (ql > 0 && q_decode_lo(L, ql, step) > clo) --ql;
      while (qh < 65535 && q_decode_hi(L, qh, step) < chi) ++qh;
      if (q_decode_lo(L, ql, step) > clo || q_decode_hi(L, qh, step) < chi) atomicOr(err, DEVERR_INTERNAL);
      qn.q[c][0][a] = (uint16_t)ql;
      qn.q[c][1][a] = (uint16_t)qh;
    }
  }
  qn.pad = 0;
  qn.child[0] = nd.child[0];
  qn.child[1] = nd.child[1];
  qnodes[g] = qn;
}

// Parent-relative 16-bit nodes (PNode, see common.cuh), encoded top-down one
// tree level per launch.  A level is a list of (internal node, frame of its
// decoded box); encoding a node picks each child's tightest codes in that
// frame (starting from floor/ceil of the outward-rounded offsets, then moved
// outward until the decoded box holds the exact child box, checked with the
// decoder itself) and lists each internal child with the frame of its decoded
// box for the next level.  Codes 0 and 65535 always hold the child (the
// parent's decoded box holds its exact box, which holds the child's), so the
// searches end; a failed check is reported, not hidden.
__device__ __forceinline__ void p16_encode(float4 fr, const float* clo, const float* chi, uint16_t* qlo,
                                           uint16_t* qhi, float* dlo, float* dhi, uint32_t* err) {
  const float o[3] = {fr.x, fr.y, fr.z};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float step = p16_step(fr, a);
    const int e = (int)((__float_as_uint(fr.w) >> (8 * a)) & 0xffu) - 127;
    const float inv = pow2f(-e);
    const float fl = floorf(__fmul_rn(__fsub_rd(clo[a], o[a]), inv));
    const float fh = ceilf(__fmul_rn(__fsub_ru(chi[a], o[a]), inv));
    uint32_t ql = (uint32_t)fminf(fmaxf(fl, 0.0f), 65535.0f);
    uint32_t qh = (uint32_t)fminf(fmaxf(fh, 0.0f), 65535.0f);
    while (ql > 0u && p16_lo(o[a], ql, step) > clo[a]) --ql;
    while (qh < 65535u && p16_hi(o[a], qh, step) < chi[a]) ++qh;
    dlo[a] = p16_lo(o[a], ql, step);
    dhi[a] = p16_hi(o[a], qh, step);
    if (!(dlo[a] <= clo[a]) || !(dhi[a] >= chi[a])) atomicOr(err, DEVERR_INTERNAL);
    qlo[a] = (uint16_t)ql;
    qhi[a] = (uint16_t)qh;
  }
}

// The first level: the root with the frame of its exact box (kept by the
// tree as the decoded box of the root).
__global__ void k_pquant_root(const Node<3>* __restrict__ nodes, const int32_t* __restrict__ root,
                              int32_t* __restrict__ level_node, float4* __restrict__ level_frame,
                              int32_t* __restrict__ count, float4* __restrict__ rframe) {
  const Node<3> nd = nodes[*root];
  float lo[3], hi[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    lo[a] = fminf(nd.lo0[a], nd.lo1[a]);
    hi[a] = fmaxf(nd.hi0[a], nd.hi1[a]);
  }
  const float4 fr = p16_frame(lo, hi);
  level_node[0] = *root;
  level_frame[0] = fr;
  count[0] = 1;
  *rframe = fr;
}

__global__ void __launch_bounds__(BUILD_THREADS) k_pquant_level(
    const Node<3>* __restrict__ nodes, PNode* __restrict__ out, const int32_t* __restrict__ in_node,
    const float4* __restrict__ in_frame, const int32_t* __restrict__ in_count, int32_t* __restrict__ out_node,
    float4* __restrict__ out_frame, int32_t* __restrict__ out_count, uint32_t* __restrict__ err) {
  const int64_t cnt = *in_count;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t g = in_node[i];
    const float4 fr = in_frame[i];
    const Node<3> nd = nodes[g];
    PNode pn;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const float* clo = c == 0 ? nd.lo0 : nd.lo1;
      const float* chi = c == 0 ? nd.hi0 : nd.hi1;
      float dlo[3], dhi[3];
      p16_encode(fr, clo, chi, pn.q[c][0], pn.q[c][1], dlo, dhi, err);
      pn.child[c] = nd.child[c];
      if (nd.child[c] >= 0) {
        const int32_t slot = atomicAdd(out_count, 1);
        out_node[slot] = nd.child[c];
        out_frame[slot] = p16_frame(dlo, dhi);
      }
    }
    out[g] = pn;
  }
}

// Four-wide records (see Wide in common.cuh): record g holds the grandchildren
// of binary node g, each copied with its box, code and orig field from the
// binary node that holds it (for an internal entry orig is its range end).
template <int D>
__global__ void __launch_bounds__(BUILD_THREADS) k_widen(const Node<D>* __restrict__ nodes, int64_t count,
                                                         Wide<D>* __restrict__ wide) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= count) return;
  const Node<D> nd = load_node_global(nodes + g);
  Wide<D> w;
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    const int32_t code = nd.child[c];
    const float* clo = c == 0 ? nd.lo0 : nd.lo1;
    const float* chi = c == 0 ? nd.hi0 : nd.hi1;
    if (code >= 0) {
      const Node<D> ch = load_node_global(nodes + code);
#pragma unroll
      for (int a = 0; a < D; ++a) {
        w.lo[2 * c][a] = ch.lo0[a];
        w.hi[2 * c][a] = ch.hi0[a];
        w.lo[2 * c + 1][a] = ch.lo1[a];
        w.hi[2 * c + 1][a] = ch.hi1[a];
      }
      w.code[2 * c] = ch.child[0];
      w.code[2 * c + 1] = ch.child[1];
      w.aux[2 * c] = ch.orig[0];
      w.aux[2 * c + 1] = ch.orig[1];
    } else {
#pragma unroll
      for (int a = 0; a < D; ++a) {
        w.lo[2 * c][a] = clo[a];
        w.hi[2 * c][a] = chi[a];
        w.lo[2 * c + 1][a] = 0.0f;
        w.hi[2 * c + 1][a] = 0.0f;
      }
      w.code[2 * c] = code;  // a leaf, or NULL_CHILD (the one-leaf tree's second child)
      w.aux[2 * c] = nd.orig[c];
      w.code[2 * c + 1] = NULL_CHILD;
      w.aux[2 * c + 1] = 0;
    }
  }
  wide[g] = w;
}

// 63/64-bit codes (section 2.6).  (48-bit codes in 3D, 16 bits per axis,
// measured the same visit counts on the 10M mixture and a 0.3 ms shorter build
// -- two radix passes fewer -- but denser data needs the finer cells.)
template <int D>
int morton_bits() { return D == 2 ? 32 : (D == 3 ? 21 : 10); }

int div_up(int64_t a, int b) { return (int)((a + b - 1) / b); }

// Resident blocks per SM of the two Apetrei kernels, and the chunk kernel's
// shared-memory attribute (6D asks for more than 48 KB), once per device.
struct ApLaunch {
  int per_sm = 0, per_sm_g = 0;
};

template <int D>
arbx_status ap_launch_facts(ApLaunch* out) {
  constexpr int MAXDEV = 64;
  static std::mutex mu;
  static ApLaunch facts[MAXDEV];
  int dev = 0;
  ARBX_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(mu);
  ApLaunch f = dev >= 0 && dev < MAXDEV ? facts[dev] : ApLaunch{};
  if (f.per_sm == 0) {
    if (ap_smem_bytes<D>() > 48 * 1024)
      ARBX_CUDA(cudaFuncSetAttribute(k_apetrei_chunks<D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)ap_smem_bytes<D>()));
    int b = 0, bg = 0;
    ARBX_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_apetrei_chunks<D>, AP_THREADS, ap_smem_bytes<D>()));
    ARBX_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bg, k_apetrei_global<D>, BUILD_THREADS, 0));
    f.per_sm = std::max(1, b);
    f.per_sm_g = std::max(1, bg);
    if (dev >= 0 && dev < MAXDEV) facts[dev] = f;
  }
  *out = f;
  return ARBX_OK;
}

template <int D, int KIND>
arbx_status build_impl(const float* data, int64_t n, uint32_t flags, BuiltTree* out, cudaStream_t s) {
  uint32_t* err = nullptr;
  ARBX_TRY(device_error_word(&err));
  const int bits = morton_bits<D>();
  out->n = n;
  out->node_stride = (int32_t)sizeof(Node<D>);
  out->quantized = false;
  // 1. bounds
  const int nparts = (int)std::min<int64_t>(std::max<int64_t>(1, div_up(n, BUILD_THREADS)), 2 * num_sms());
  DevTemp<float> partial(s), frame(s);
  ARBX_TRY(partial.alloc((size_t)nparts * 2 * D));
  ARBX_TRY(frame.alloc(2 * D));
  ARBX_TRY(dev_alloc_t(&out->scene, 2 * D, s));
  if (KIND == ARBX_POINT && (reinterpret_cast<uintptr_t>(data) & 15) == 0) {
    ARBX_LAUNCH("bounds", s, k_bounds_vec<D><<<nparts, BUILD_THREADS, 0, s>>>(data, n * D, partial.p, err));
  } else {
    ARBX_LAUNCH("bounds", s, k_bounds<D, KIND><<<nparts, BUILD_THREADS, 0, s>>>(data, n, partial.p, err));
  }
  ARBX_LAUNCH("bounds_final", s, k_bounds_final<D><<<1, 32, 0, s>>>(partial.p, nparts, out->scene, frame.p, bits));
  // 2-3. Morton codes, sort
  DevTemp<uint64_t> keys(s), keys_alt(s);
  DevTemp<uint32_t> vals(s), vals_alt(s);
  ARBX_TRY(keys.alloc(n));
  ARBX_TRY(keys_alt.alloc(n));
  ARBX_TRY(vals.alloc(n));
  ARBX_TRY(vals_alt.alloc(n));
  ARBX_LAUNCH("morton", s, k_morton<D, KIND><<<div_up(n, BUILD_THREADS), BUILD_THREADS, 0, s>>>(data, n, frame.p, bits, keys.p, vals.p));
  bool alt = false;
  ARBX_TRY(radix_sort_pairs<uint64_t>(keys.p, vals.p, keys_alt.p, vals_alt.p, n, 0, D * bits, &alt, s));
  const uint64_t* skeys = alt ? keys_alt.p : keys.p;
  const uint32_t* perm = alt ? vals_alt.p : vals.p;
  // 4. gather
  DevTemp<float> sbox(s);
  ARBX_TRY(sbox.alloc((size_t)n * 2 * D));
  if (KIND == ARBX_TRIANGLE) ARBX_TRY(dev_alloc_t(&out->leaves, n, s));
  ARBX_LAUNCH("gather", s, k_gather<D, KIND><<<div_up(n, BUILD_THREADS), BUILD_THREADS, 0, s>>>(data, n, perm, sbox.p, out->leaves));
  // 5. hierarchy
  const int64_t nnodes = n > 1 ? n - 1 : 1;
  Node<D>* nodes = nullptr;
  ARBX_TRY(dev_alloc_t(&nodes, nnodes, s));
  out->nodes = nodes;
  out->nnodes = nnodes;
  DevTemp<int32_t> root(s);  // [root, nodes in the 255-copy, nodes in the 1023-copy]
  ARBX_TRY(root.alloc(3));
  if (n == 1) {
    ARBX_LAUNCH("single_leaf", s, k_single<D><<<1, 1, 0, s>>>(sbox.p, nodes, root.p));
  } else {
    DevTemp<int32_t> fl(s);
    ARBX_TRY(fl.alloc(n - 1));
    ARBX_CUDA(cudaMemsetAsync(fl.p, 0xff, (size_t)(n - 1) * sizeof(int32_t), s));
    ARBX_CUDA(cudaMemsetAsync(root.p, 0, sizeof(int32_t), s));
#if ARBX_CHECKED
    // an incomplete hierarchy then holds in-range codes only (the walk after
    // the build reports it)
    ARBX_CUDA(cudaMemsetAsync(nodes, 0, (size_t)nnodes * sizeof(Node<D>), s));
#endif
    DevTemp<ApArrival> alist(s);
    DevTemp<unsigned int> acount(s);
    const int64_t cap = ap_list_cap(n);
    ARBX_TRY(alist.alloc((size_t)cap));
    ARBX_TRY(acount.alloc(1));
    ARBX_CUDA(cudaMemsetAsync(acount.p, 0, sizeof(unsigned int), s));
    // resident blocks only, each over a sequence of chunks; then resident warps
    // over the listed arrivals
    ApLaunch lf;
    ARBX_TRY(ap_launch_facts<D>(&lf));
    const int64_t nchunks = (n + AP_CHUNK - 1) / AP_CHUNK;
    const int grid = (int)std::min<int64_t>(nchunks, (int64_t)lf.per_sm * num_sms());
    ARBX_LAUNCH("apetrei", s,
                k_apetrei_chunks<D><<<grid, AP_THREADS, ap_smem_bytes<D>(), s>>>(skeys, perm, sbox.p, (int)n, nodes, root.p,
                                                                                alist.p, acount.p, cap, err));
    if (nchunks > 1) {
      const int ggrid = (int)std::min<int64_t>(div_up(cap, BUILD_THREADS), (int64_t)lf.per_sm_g * num_sms());
      ARBX_LAUNCH("apetrei_global", s,
                  k_apetrei_global<D><<<ggrid, BUILD_THREADS, 0, s>>>(skeys, (int)n, alist.p, acount.p, cap, fl.p, nodes,
                                                                      root.p));
    }
  }
  // four-wide records for the nearest and counting traversals (point and box trees, on request)
  if (KIND != ARBX_TRIANGLE && (flags & ARBX_WIDE_NODES)) {
    Wide<D>* wide = nullptr;
    ARBX_TRY(dev_alloc_t(&wide, nnodes, s));
    out->wide = wide;
    ARBX_LAUNCH("widen", s, k_widen<D><<<div_up(nnodes, BUILD_THREADS), BUILD_THREADS, 0, s>>>(nodes, nnodes, wide));
  }
  // 7. quantized copy (3D triangle trees): parent-relative 32-byte nodes,
  // encoded top-down one level per launch (the level lists are read back every
  // eighth level to stop after the deepest; the radix tree of 63-bit codes with
  // index tie-breaks is at most 96 levels deep)
  DevTemp<float4> rframe(s);
  if ((flags & ARBX_QUANTIZED_NODES) && (flags & ARBX_PARENT_RELATIVE) && D == 3 && n > 1) {
    PNode* q = nullptr;
    ARBX_TRY(dev_alloc_t(&q, nnodes, s));
    out->pnodes = q;
    constexpr int MAX_LEVELS = 104;
    DevTemp<int32_t> lnode(s), counts(s);
    DevTemp<float4> lframe(s);
    ARBX_TRY(lnode.alloc((size_t)2 * nnodes));
    ARBX_TRY(lframe.alloc((size_t)2 * nnodes));
    ARBX_TRY(counts.alloc(MAX_LEVELS + 1));
    ARBX_TRY(rframe.alloc(1));
    ARBX_CUDA(cudaMemsetAsync(counts.p, 0, (MAX_LEVELS + 1) * sizeof(int32_t), s));
    const Node<3>* n3 = reinterpret_cast<const Node<3>*>(nodes);
    ARBX_LAUNCH("pquant_root", s, k_pquant_root<<<1, 1, 0, s>>>(n3, root.p, lnode.p, lframe.p, counts.p, rframe.p));
    const int grid = std::min(div_up(nnodes, BUILD_THREADS), 4 * num_sms());
    bool ended = false;
    for (int l = 0; l < MAX_LEVELS && !ended; ++l) {
      const int64_t in = (l & 1) ? nnodes : 0, o = (l & 1) ? 0 : nnodes;
      ARBX_LAUNCH("pquant_level", s, k_pquant_level<<<grid, BUILD_THREADS, 0, s>>>(
                                       n3, q, lnode.p + in, lframe.p + in, counts.p + l, lnode.p + o, lframe.p + o,
                                       counts.p + l + 1, err));
      if ((l & 7) == 7) {
        int32_t c = 0;
        ARBX_TRY(read_small(counts.p + l + 1, &c, sizeof(c), s));
        ended = c == 0;
      }
    }
    if (!ended) return ARBX_ERR_CUDA;  // deeper than the radix-tree bound: not a tree this build makes
    float4 fr;
    ARBX_TRY(read_small(rframe.p, &fr, sizeof(fr), s));
    out->rframe[0] = fr.x;
    out->rframe[1] = fr.y;
    out->rframe[2] = fr.z;
    out->rframe[3] = fr.w;
    out->quantized = true;
    out->prel = true;
    ARBX_TRY(dev_alloc_t(&out->leaf_orig, n, s));
    ARBX_CUDA(cudaMemcpyAsync(out->leaf_orig, perm, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
  } else if ((flags & ARBX_QUANTIZED_NODES) && D == 3 && n > 1) {
    QNode* q = nullptr;
    ARBX_TRY(dev_alloc_t(&q, nnodes, s));
    ARBX_LAUNCH("quantize", s, k_quantize<<<div_up(nnodes, BUILD_THREADS), BUILD_THREADS, 0, s>>>(
                                  reinterpret_cast<const Node<3>*>(nodes), nnodes, q, err));
    out->qnodes = q;
    out->quantized = true;
    // input index by sorted position: a leaf that needs no exact test needs no
    // 48-byte leaf record either (box queries whose box holds the decoded leaf box)
    ARBX_TRY(dev_alloc_t(&out->leaf_orig, n, s));
    ARBX_CUDA(cudaMemcpyAsync(out->leaf_orig, perm, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
  } else if (flags & ARBX_QUANTIZED_NODES) {
    // n == 1: the pseudo root keeps its float32 node
  }
  // 6. top levels for both node formats in use (caps 255 and 1023)
  for (int ci = 0; ci < 2; ++ci) {
    const int cap = ci == 0 ? 255 : 1023;
    if (out->prel) {
      PNode* top = nullptr;
      ARBX_TRY(dev_alloc_t(&top, cap, s));
      out->top[ci] = top;
      ARBX_LAUNCH("top_levels", s, k_top_levels<PNode><<<1, 1024, 0, s>>>(out->pnodes, root.p, cap, top, root.p + 1 + ci));
    } else if (out->quantized) {
      QNode* top = nullptr;
      ARBX_TRY(dev_alloc_t(&top, cap, s));
      out->top[ci] = top;
      ARBX_LAUNCH("top_levels", s, k_top_levels<QNode><<<1, 1024, 0, s>>>(out->qnodes, root.p, cap, top, root.p + 1 + ci));
    } else {
      Node<D>* top = nullptr;
      ARBX_TRY(dev_alloc_t(&top, cap, s));
      out->top[ci] = top;
      ARBX_LAUNCH("top_levels", s, k_top_levels<Node<D>><<<1, 1024, 0, s>>>(nodes, root.p, cap, top, root.p + 1 + ci));
    }
  }
  int32_t hv[3];
  ARBX_TRY(read_small(root.p, hv, sizeof(hv), s));
  ARBX_TRY(read_small(out->scene, out->scene_host, 2 * D * sizeof(float), s));
  out->root = hv[0];
  out->ntop[0] = hv[1];
  out->ntop[1] = hv[2];
  if (out->quantized) {
    // the 16-bit nodes replace the float32 ones
    dev_free(nodes, s);
    out->nodes = out->prel ? static_cast<void*>(out->pnodes) : static_cast<void*>(out->qnodes);
    out->node_stride = out->prel ? (int32_t)sizeof(PNode) : (int32_t)sizeof(QNode);
  }
  return ARBX_OK;
}

// ------------------------------------------------------------------ checked builds: tree validation
//
// A walk from the root, one level per launch: every internal record and every
// sorted leaf must be reached exactly once through codes that name existing
// records, in at most 104 levels (the radix tree is at most 96 deep).  Float32
// nodes also check that the box a parent keeps for an internal child holds
// that child's two boxes, and that their orig fields are input indices / range
// ends below n.  Any failure sets DEVERR_BOUNDS.

template <int D>
__device__ __forceinline__ void check_node_extra(const Node<D>* nodes, int64_t nint, int64_t n, const Node<D>& nd,
                                                 uint32_t* err) {
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    const int32_t code = nd.child[c];
    if (code == NULL_CHILD) continue;
    if (nd.orig[c] < 0 || nd.orig[c] >= n) atomicOr(err, DEVERR_BOUNDS | BAD_TREE);
    if (code >= 0 && code < nint) {
      const Node<D> ch = nodes[code];
      const float* blo = c == 0 ? nd.lo0 : nd.lo1;
      const float* bhi = c == 0 ? nd.hi0 : nd.hi1;
      bool ok = true;
#pragma unroll
      for (int a = 0; a < D; ++a) {
        ok = ok && blo[a] <= ch.lo0[a] && ch.hi0[a] <= bhi[a];
        if (ch.child[1] != NULL_CHILD) ok = ok && blo[a] <= ch.lo1[a] && ch.hi1[a] <= bhi[a];
      }
      if (!ok) atomicOr(err, DEVERR_BOUNDS | BAD_TREE);
    }
  }
}
template <class NodeT>
__device__ __forceinline__ void check_node_extra(const NodeT*, int64_t, int64_t, const NodeT&, uint32_t*) {}

template <class NodeT>
__global__ void __launch_bounds__(BUILD_THREADS) k_check_level(
    const NodeT* __restrict__ nodes, int64_t nint, int64_t n, const int32_t* __restrict__ in_list,
    const int32_t* __restrict__ in_count, int32_t* __restrict__ out_list, int32_t* __restrict__ out_count,
    int32_t* __restrict__ seen_int, int32_t* __restrict__ seen_leaf, uint32_t* __restrict__ err) {
  const int64_t cnt = min((int64_t)*in_count, nint);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t g = in_list[i];
    if (atomicAdd(seen_int + g, 1) != 0) {  // reached twice
      atomicOr(err, DEVERR_BOUNDS | BAD_TREE);
      continue;
    }
    const NodeT nd = nodes[g];
    check_node_extra(nodes, nint, n, nd, err);
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int32_t code = nd.child[c];
      if (code == NULL_CHILD) {
        if (!(n == 1 && c == 1)) atomicOr(err, DEVERR_BOUNDS | BAD_TREE);
      } else if (code >= 0) {
        if (code >= nint) {
          atomicOr(err, DEVERR_BOUNDS | BAD_TREE);
        } else {
          const int32_t slot = atomicAdd(out_count, 1);
          if (slot < nint) out_list[slot] = code;
          else atomicOr(err, DEVERR_BOUNDS | BAD_TREE);
        }
      } else {
        const int64_t pos = ~(int64_t)code;
        if (pos >= n || atomicAdd(seen_leaf + pos, 1) != 0) atomicOr(err, DEVERR_BOUNDS | BAD_TREE);
      }
    }
  }
}

// Every record and leaf reached once; the per-leaf input indices below n.
__global__ void k_check_seen(const int32_t* __restrict__ seen_int, int64_t nint, const int32_t* __restrict__ seen_leaf,
                             int64_t n, const TriLeaf* __restrict__ leaves, const int32_t* __restrict__ leaf_orig,
                             uint32_t* __restrict__ err) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nint && seen_int[i] != 1) atomicOr(err, DEVERR_BOUNDS | BAD_TREE);
  if (i < n) {
    if (seen_leaf[i] != 1) atomicOr(err, DEVERR_BOUNDS | BAD_TREE);
    if (leaves && (leaves[i].orig < 0 || leaves[i].orig >= n)) atomicOr(err, DEVERR_BOUNDS | BAD_TREE);
    if (leaf_orig && (leaf_orig[i] < 0 || leaf_orig[i] >= n)) atomicOr(err, DEVERR_BOUNDS | BAD_TREE);
  }
}

// Top-level copies: local codes below ntop, other codes as in the full array.
template <class NodeT>
__global__ void k_check_top(const NodeT* __restrict__ top, int32_t ntop, int64_t nint, int64_t n,
                            uint32_t* __restrict__ err) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ntop) return;
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    const int32_t code = top[i].child[c];
    if (code == NULL_CHILD) continue;
    const bool ok = code >= 0 ? ((code & TOP_FLAG) ? (code & ~TOP_FLAG) < ntop : code < nint) : ~(int64_t)code < n;
    if (!ok) atomicOr(err, DEVERR_BOUNDS | BAD_TREE);
  }
}

// Four-wide records: codes name records or sorted leaves, aux fields below n.
template <int D>
__global__ void k_check_wide(const Wide<D>* __restrict__ w, int64_t nint, int64_t n, uint32_t* __restrict__ err) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= nint) return;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int32_t code = w[g].code[c];
    if (code == NULL_CHILD) continue;
    const bool ok = (code >= 0 ? code < nint : ~(int64_t)code < n) && w[g].aux[c] >= 0 && w[g].aux[c] < n;
    if (!ok) atomicOr(err, DEVERR_BOUNDS | BAD_TREE);
  }
}

template <class NodeT, int D>
arbx_status validate_impl(const BuiltTree& b, cudaStream_t s) {
  uint32_t* err = nullptr;
  ARBX_TRY(device_error_word(&err));
  const int64_t nint = b.nnodes, n = b.n;
  const NodeT* nodes = static_cast<const NodeT*>(b.nodes);
  constexpr int MAX_LEVELS = 104;
  DevTemp<int32_t> lists(s), counts(s), seen(s);
  ARBX_TRY(lists.alloc((size_t)2 * nint));
  ARBX_TRY(counts.alloc(MAX_LEVELS + 1));
  ARBX_TRY(seen.alloc((size_t)(nint + n)));
  ARBX_CUDA(cudaMemsetAsync(counts.p, 0, (MAX_LEVELS + 1) * sizeof(int32_t), s));
  ARBX_CUDA(cudaMemsetAsync(seen.p, 0, (size_t)(nint + n) * sizeof(int32_t), s));
  const int32_t first[2] = {b.root, 1};
  ARBX_CUDA(cudaMemcpyAsync(lists.p, &first[0], sizeof(int32_t), cudaMemcpyHostToDevice, s));
  ARBX_CUDA(cudaMemcpyAsync(counts.p, &first[1], sizeof(int32_t), cudaMemcpyHostToDevice, s));
  const int grid = std::min(div_up(nint, BUILD_THREADS), 4 * num_sms());
  bool ended = false;
  for (int l = 0; l < MAX_LEVELS && !ended; ++l) {
    const int64_t in = (l & 1) ? nint : 0, o = (l & 1) ? 0 : nint;
    ARBX_LAUNCH("check_level", s, k_check_level<NodeT><<<grid, BUILD_THREADS, 0, s>>>(
                                      nodes, nint, n, lists.p + in, counts.p + l, lists.p + o, counts.p + l + 1,
                                      seen.p, seen.p + nint, err));
    if ((l & 7) == 7) {
      int32_t c = 0;
      ARBX_TRY(read_small(counts.p + l + 1, &c, sizeof(c), s));
      ended = c == 0;
    }
  }
  if (!ended) return ARBX_ERR_BOUNDS;
  ARBX_LAUNCH("check_seen", s, k_check_seen<<<div_up(std::max(nint, n), BUILD_THREADS), BUILD_THREADS, 0, s>>>(
                                   seen.p, nint, seen.p + nint, n, b.leaves, b.leaf_orig, err));
  for (int ci = 0; ci < 2; ++ci)
    if (b.top[ci] && b.ntop[ci] > 0)
      ARBX_LAUNCH("check_top", s, k_check_top<NodeT><<<div_up(b.ntop[ci], BUILD_THREADS), BUILD_THREADS, 0, s>>>(
                                      static_cast<const NodeT*>(b.top[ci]), b.ntop[ci], nint, n, err));
  if (b.wide)
    ARBX_LAUNCH("check_wide", s, k_check_wide<D><<<div_up(nint, BUILD_THREADS), BUILD_THREADS, 0, s>>>(
                                     static_cast<const Wide<D>*>(b.wide), nint, n, err));
  return ARBX_OK;
}

arbx_status validate_tree(int dim, const BuiltTree& b, cudaStream_t s) {
  if (b.n == 0) return ARBX_OK;
  if (b.prel) return validate_impl<PNode, 3>(b, s);
  if (b.quantized) return validate_impl<QNode, 3>(b, s);
  switch (dim) {
    case 2: return validate_impl<Node<2>, 2>(b, s);
    case 3: return validate_impl<Node<3>, 3>(b, s);
    case 6: return validate_impl<Node<6>, 6>(b, s);
  }
  return ARBX_ERR_UNSUPPORTED;
}

}  // namespace

arbx_status build_tree(int kind, int dim, const float* data, int64_t n, uint32_t flags, BuiltTree* out,
                       cudaStream_t s) {
  arbx_status st = ARBX_ERR_UNSUPPORTED;
  switch (kind * 16 + dim) {
    case ARBX_POINT * 16 + 2: st = build_impl<2, ARBX_POINT>(data, n, flags, out, s); break;
    case ARBX_POINT * 16 + 3: st = build_impl<3, ARBX_POINT>(data, n, flags, out, s); break;
    case ARBX_POINT * 16 + 6: st = build_impl<6, ARBX_POINT>(data, n, flags, out, s); break;
    case ARBX_BOX * 16 + 2: st = build_impl<2, ARBX_BOX>(data, n, flags, out, s); break;
    case ARBX_BOX * 16 + 3: st = build_impl<3, ARBX_BOX>(data, n, flags, out, s); break;
    case ARBX_BOX * 16 + 6: st = build_impl<6, ARBX_BOX>(data, n, flags, out, s); break;
    case ARBX_TRIANGLE * 16 + 3: st = build_impl<3, ARBX_TRIANGLE>(data, n, flags, out, s); break;
  }
  if (st == ARBX_OK && CHECKED) {
    st = check_stream(s);  // a rejected input (e.g. non-finite coordinates) is reported as such
    if (st == ARBX_OK) st = validate_tree(dim, *out, s);
  }
  return st;
}

}  // namespace arbx
