// Batches of independent trees ("forests"): thousands of point sets of
// different sizes and dimensions are built and queried together.
//
// Build (per dimension group D in {2, 3, 6}, all sets of that dimension at once):
//   k_f_bounds   one block per set: the set's box (exact min/max) and Morton
//                frame; finiteness check
//   k_f_morton   key = set index (12 bits) << 52 | Morton code of the point in
//                its set's box (52/D bits per axis)
//   radix sort   one sort of all keys: every set's points end up contiguous
//                and in Morton order inside the set
//   k_f_gather   points in sorted order
//   k_f_apetrei  Apetrei's bottom-up construction over the concatenation, run
//                with each set's own range [b, e] in place of [0, n-1]: a node
//                whose range reaches [b, e] is that set's root and stops, so
//                the pass yields one binary radix tree per set (a single-point
//                set gets a pseudo root, as in the single-tree build)
// Leaf indices stored in the nodes are set-local.
//
// Query (a batch object holds the per-set query layout, radii and the query
// order buffers, so the query calls only enqueue device work and can be
// captured in a CUDA graph):
//   k_f_query_codes + radix sort: each call orders every group's queries by
//   (set, Morton code in the set's frame), as the single-tree path orders its
//   queries (section 2.6, sorting in search);
//   one persistent kernel per predicate pulls chunks of 32 or 64 query slots
//   (the batch's tuning) from a global counter; each dimension group's slots
//   start on a 64-slot boundary, so a chunk (and the warp working on it) has
//   one dimension, dispatched to the D-templated traversal.  Lanes map slots
//   to (set, query) by binary search.
// Launch settings (block size, chunk size, query ordering per dimension
// group) are the batch's arbx_forest_tuning, chosen by arbx_forest_autotune
// by measurement; every setting gives the same bytes.
// Radius: count -> scan -> fill into caller buffers with a capacity guard
// (the total is written to device memory; a fill larger than the capacity is
// not written and is reported by that total).  Nearest: k best (d2, index)
// pairs per query, rows of stride k.
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "build.cuh"
#include "primitives.cuh"
#include "query.cuh"
#include "traverse.cuh"

namespace arbx {
namespace {

constexpr int F_THREADS = 256;
constexpr int F_MAX_CHUNK = 64;  // group slot ranges are padded to this
constexpr int SET_BITS = 12;
constexpr int MAX_GROUP_SETS = 1 << SET_BITS;
constexpr int GROUP_DIMS[3] = {2, 3, 6};

__device__ __forceinline__ bool f_finite(float x) { return (__float_as_uint(x) & 0x7f800000u) != 0x7f800000u; }

// Largest s in [0, ns) with base[s] <= i (empty sets are skipped over).
__device__ __forceinline__ int find_set(const int64_t* __restrict__ base, int ns, int64_t i) {
  int lo = 0, hi = ns;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(base + mid) <= i) lo = mid;
    else hi = mid;
  }
  return lo;
}

template <int D>
__global__ void __launch_bounds__(F_THREADS) k_f_bounds(const float* __restrict__ data, const int64_t* __restrict__ foff,
                                                        const int64_t* __restrict__ pbase, int ns,
                                                        float* __restrict__ frame, uint32_t* __restrict__ err) {
  const int s = blockIdx.x;
  if (s >= ns) return;
  const int64_t n = pbase[s + 1] - pbase[s];
  const float* p = data + foff[s];
  float lo[D], hi[D];
#pragma unroll
  for (int a = 0; a < D; ++a) {
    lo[a] = __int_as_float(0x7f800000);
    hi[a] = -__int_as_float(0x7f800000);
  }
  bool ok = true;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const float v = p[i * D + a];
      ok = ok && f_finite(v);
      lo[a] = fminf(lo[a], v);
      hi[a] = fmaxf(hi[a], v);
    }
  }
  if (!ok) atomicOr(err, DEVERR_NONFINITE);
  __shared__ float s_lo[F_THREADS / 32][D], s_hi[F_THREADS / 32][D];
#pragma unroll
  for (int a = 0; a < D; ++a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      lo[a] = fminf(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
      hi[a] = fmaxf(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
    }
  }
  if ((threadIdx.x & 31) == 0) {
#pragma unroll
    for (int a = 0; a < D; ++a) {
      s_lo[threadIdx.x >> 5][a] = lo[a];
      s_hi[threadIdx.x >> 5][a] = hi[a];
    }
  }
  __syncthreads();
  if (threadIdx.x < D) {
    const int a = threadIdx.x;
    float l = s_lo[0][a], h = s_hi[0][a];
    for (int w = 1; w < F_THREADS / 32; ++w) {
      l = fminf(l, s_lo[w][a]);
      h = fmaxf(h, s_hi[w][a]);
    }
    const float ext = h - l;
    frame[(int64_t)s * 2 * D + a] = l;
    frame[(int64_t)s * 2 * D + D + a] = ext > 0.0f ? (float)(1ull << (52 / D)) / ext : 0.0f;
  }
}

template <int D>
__global__ void __launch_bounds__(F_THREADS) k_f_morton(const float* __restrict__ data, const int64_t* __restrict__ foff,
                                                        const int64_t* __restrict__ pbase, int ns, int64_t npts,
                                                        const float* __restrict__ frame, uint64_t* __restrict__ keys,
                                                        uint32_t* __restrict__ vals) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npts) return;
  const int s = find_set(pbase, ns, i);
  const float* p = data + foff[s] + (i - pbase[s]) * D;
  constexpr int BITS = 52 / D;
  const uint32_t cmax = (1u << BITS) - 1u;
  uint32_t cell[D];
#pragma unroll
  for (int a = 0; a < D; ++a) {
    float u = (p[a] - frame[(int64_t)s * 2 * D + a]) * frame[(int64_t)s * 2 * D + D + a];
    u = fmaxf(u, 0.0f);
    cell[a] = u >= (float)cmax ? cmax : (uint32_t)u;
  }
  uint64_t code = 0;
  for (int b = BITS - 1; b >= 0; --b) {
#pragma unroll
    for (int a = 0; a < D; ++a) code = (code << 1) | ((cell[a] >> b) & 1u);
  }
  keys[i] = ((uint64_t)s << 52) | code;
  vals[i] = (uint32_t)i;
}

template <int D>
__global__ void __launch_bounds__(F_THREADS) k_f_gather(const float* __restrict__ data, const int64_t* __restrict__ foff,
                                                        const int64_t* __restrict__ pbase, int64_t npts,
                                                        const uint32_t* __restrict__ perm,
                                                        const uint64_t* __restrict__ skeys, float* __restrict__ spts) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npts) return;
  const int s = (int)(skeys[i] >> 52);
  const int64_t j = perm[i];
  const float* p = data + foff[s] + (j - pbase[s]) * D;
#pragma unroll
  for (int a = 0; a < D; ++a) spts[i * D + a] = p[a];
}

__device__ __forceinline__ int f_delta(const uint64_t* __restrict__ keys, int i) {
  const uint64_t a = keys[i], b = keys[i + 1];
  return a != b ? __clzll((long long)(a ^ b)) : 64 + __clz((int)((uint32_t)i ^ (uint32_t)(i + 1)));
}

template <int D>
__global__ void __launch_bounds__(F_THREADS) k_f_apetrei(const uint64_t* __restrict__ keys,
                                                         const uint32_t* __restrict__ perm,
                                                         const float* __restrict__ spts,
                                                         const int64_t* __restrict__ pbase, int npts,
                                                         int32_t* __restrict__ flags, Node<D>* nodes,
                                                         int32_t* __restrict__ roots) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npts) return;
  const int s = (int)(keys[i] >> 52);
  const int b = (int)pbase[s], e = (int)pbase[s + 1] - 1;
  float lo[D], hi[D];
#pragma unroll
  for (int a = 0; a < D; ++a) lo[a] = hi[a] = spts[(int64_t)i * D + a];
  if (b == e) {
    // one-point set: pseudo root in the free node slot at its split position e
    Node<D> nd;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      nd.lo0[a] = nd.hi0[a] = lo[a];
      nd.lo1[a] = __int_as_float(0x7f800000);
      nd.hi1[a] = -__int_as_float(0x7f800000);
    }
    nd.child[0] = ~i;
    nd.child[1] = NULL_CHILD;
    nd.orig[0] = 0;
    nd.orig[1] = -1;
    nodes[e] = nd;
    roots[s] = e;
    return;
  }
  int l = i, r = i;
  int32_t code = ~i;
  int32_t orig = (int32_t)perm[i] - b;
  for (;;) {
    const bool left = (l == b) || (r != e && f_delta(keys, r) > f_delta(keys, l - 1));
    const int g = left ? r : l - 1;
    Node<D>* p = nodes + g;
    float* mlo = left ? p->lo0 : p->lo1;
    float* mhi = left ? p->hi0 : p->hi1;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      __stcg(mlo + a, lo[a]);
      __stcg(mhi + a, hi[a]);
    }
    __stcg(&p->child[left ? 0 : 1], code);
    __stcg(&p->orig[left ? 0 : 1], orig);
    // release: this half is visible first; acquire: the sibling's half is visible after
    const int other = exch_acq_rel(flags + g, left ? l : r);
    if (other < 0) return;
    const float* slo = left ? p->lo1 : p->lo0;
    const float* shi = left ? p->hi1 : p->hi0;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      lo[a] = fminf(lo[a], __ldcg(slo + a));
      hi[a] = fmaxf(hi[a], __ldcg(shi + a));
    }
    if (left) r = other;
    else l = other;
    code = g;
    orig = -1;
    if (l == b && r == e) {
      roots[s] = g;
      return;
    }
  }
}

// ------------------------------------------------------------------ query

struct FGroup {
  const void* nodes;
  int64_t nnodes;        // records in nodes (checked builds bound every node code by it)
  int ns;
  const int64_t* qbase;  // [ns+1] group-local query prefix
  const int64_t* gq;     // [ns] first global query id of the set
  const int64_t* qfoff;  // [ns] float offset of the set's queries in the query buffer
  const int32_t* roots;  // [ns] root node (NULL_CHILD for an empty set)
  const float* r2;       // [ns] fl(r*r)
  const int32_t* npts;   // [ns] points of the set (kNN: valid results)
  int64_t slot_base;     // first slot of the group (multiple of F_MAX_CHUNK)
  int64_t m;             // queries of the group
  int64_t max_steps;     // cap on one traversal (4x the group's points + 1024)
  const uint32_t* perm;  // processing order of the group's queries (set, then Morton order inside the set)
};

struct FArgs {
  FGroup g[3];
  int ngroups;
  int dims[3];
  const float* qs;
  int64_t slots;  // padded slot count over all groups
  int32_t* counts;
  const int64_t* offsets;
  int32_t* out_idx;
  float* out_d2;
  int64_t capacity;
  int32_t* knn_idx;
  float* knn_d2;
  int k;
  uint32_t* err;
  unsigned long long* counter;
  int chunk;  // query slots per work item (32 or 64)
};

// Per lane: the set, global query id and query coordinates of a group slot.
template <int D>
__device__ __forceinline__ void lane_query(const FArgs& a, const FGroup& G, int64_t q, int& s, int64_t& gid,
                                           float (&x)[D]) {
  s = find_set(G.qbase, G.ns, q);
  const int64_t j = q - __ldg(G.qbase + s);
  gid = __ldg(G.gq + s) + j;
  const float* p = a.qs + __ldg(G.qfoff + s) + j * D;
#pragma unroll
  for (int c = 0; c < D; ++c) x[c] = p[c];
}

// Sort keys of a group's queries: the set's index in the group above a
// 48-bit Morton code of the query in the set's frame (the frame of its
// points, 52/D bits per axis, coarsened to 48 bits), so neighbouring queries
// of one set are processed together.
template <int D>
__global__ void __launch_bounds__(256) k_f_query_codes(const float* __restrict__ qs, FGroup G,
                                                       const float* __restrict__ frame, uint64_t* __restrict__ keys,
                                                       uint32_t* __restrict__ vals) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= G.m) return;
  const int s = find_set(G.qbase, G.ns, q);
  const int64_t j = q - __ldg(G.qbase + s);
  const float* p = qs + __ldg(G.qfoff + s) + j * D;
  constexpr int FB = 52 / D;                          // frame bits per axis
  constexpr int QB = D == 2 ? 24 : (D == 3 ? 16 : 8);  // code bits per axis
  const float coarsen = 1.0f / (float)(1u << (FB - QB));
  uint32_t cell[D];
#pragma unroll
  for (int a = 0; a < D; ++a) {
    float u = (p[a] - frame[(int64_t)s * 2 * D + a]) * frame[(int64_t)s * 2 * D + D + a] * coarsen;
    u = fminf(fmaxf(u, 0.0f), (float)((1u << QB) - 1u));  // NaN -> 0
    cell[a] = (uint32_t)u;
  }
  uint64_t code = 0;
  for (int b = QB - 1; b >= 0; --b) {
#pragma unroll
    for (int a = 0; a < D; ++a) code = (code << 1) | ((cell[a] >> b) & 1u);
  }
  keys[q] = ((uint64_t)s << 48) | code;
  vals[q] = (uint32_t)q;
}

template <int D, int MODE>
__device__ __forceinline__ void f_spatial_chunk(const FArgs& a, const FGroup& G, int64_t chunk) {
  const Node<D>* __restrict__ g = static_cast<const Node<D>*>(G.nodes);
  int32_t st[STACK_DEPTH];
  float sd[MODE == MODE_FILL ? STACK_DEPTH : 1];
  for (int64_t base = chunk; base < chunk + a.chunk; base += 32) {
    const int64_t slot = base - G.slot_base + (threadIdx.x & 31);
    bool active = slot < G.m;
    const int64_t q = active && G.perm ? checked_index((int64_t)G.perm[slot], G.m, a.err, BAD_ORDER) : slot;
    SpherePred<D> p;
    int64_t gid = 0, w = 0, wend = 0;
    int32_t cur = NULL_CHILD, cnt = 0;
    float cur_d2 = 0.0f;
    int sp = 0;
    if (active) {
      int s;
      lane_query<D>(a, G, q, s, gid, p.q);
      p.r2 = __ldg(G.r2 + s);
      cur = __ldg(G.roots + s);
      if (MODE == MODE_FILL) {
        w = a.offsets[gid];
        wend = a.offsets[gid + 1];
      }
      if (cur == NULL_CHILD) {
        if (MODE != MODE_FILL) a.counts[gid] = 0;
        active = false;
      }
    }
    int64_t steps = 0;
    while (__any_sync(0xffffffffu, active)) {
      if (active && ++steps > G.max_steps) {  // runaway traversal: stop and report
        atomicOr(a.err, DEVERR_INTERNAL);
        active = false;
      }
      if (active) {
        bool done = false;
        int32_t next = -1;
        if (MODE == MODE_FILL && cur < 0) {
          if (w < wend && w < a.capacity) {
            a.out_idx[w] = ~cur;
            a.out_d2[w] = cur_d2;
          }
          ++w;
        } else {
          const Kids<D> k = unpack(load_node_global(g + checked_index(cur, G.nnodes, a.err, BAD_NODE)));
          float d0 = 0.0f, d1 = 0.0f;
          const bool h0 = p.test(k.lo[0], k.hi[0], d0);
          const bool h1 = k.child[1] != NULL_CHILD && p.test(k.lo[1], k.hi[1], d1);
          const bool i0 = h0 && k.child[0] >= 0, i1 = h1 && k.child[1] >= 0;
          const bool l0 = h0 && k.child[0] < 0, l1 = h1 && k.child[1] < 0;
          if (MODE == MODE_FILL) {
            if (l0) {
              if (w < wend && w < a.capacity) {
                a.out_idx[w] = k.orig[0];
                a.out_d2[w] = d0;
              }
              ++w;
            }
            if (l1 && !i0) {
              if (w < wend && w < a.capacity) {
                a.out_idx[w] = k.orig[1];
                a.out_d2[w] = d1;
              }
              ++w;
            }
            if (i0 && (l1 || i1)) {
              if (sp < STACK_DEPTH) {
                st[sp] = l1 ? ~k.orig[1] : k.child[1];
                sd[sp] = d1;
                ++sp;
              } else {
                atomicOr(a.err, DEVERR_STACK);
                done = true;
              }
            }
          } else {
            cnt += (int32_t)l0 + (int32_t)l1;
            if (i0 && i1) {
              if (sp < STACK_DEPTH) {
                st[sp++] = k.child[1];
              } else {
                atomicOr(a.err, DEVERR_STACK);
                done = true;
              }
            }
          }
          next = i0 ? k.child[0] : (i1 ? k.child[1] : -1);
        }
        if (!done) {
          if (next >= 0) {
            cur = next;
          } else if (sp > 0) {
            --sp;
            cur = st[sp];
            if (MODE == MODE_FILL) cur_d2 = sd[sp];
          } else {
            done = true;
          }
        }
        if (done) {
          if (MODE != MODE_FILL) a.counts[gid] = cnt;
          active = false;
        }
      }
    }
  }
}

template <int D, int K>
__device__ __forceinline__ void f_knn_chunk(const FArgs& a, const FGroup& G, int64_t chunk) {
  const Node<D>* __restrict__ g = static_cast<const Node<D>*>(G.nodes);
  int32_t st[STACK_DEPTH];
  float sb[STACK_DEPTH];
  for (int64_t base = chunk; base < chunk + a.chunk; base += 32) {
    const int64_t slot = base - G.slot_base + (threadIdx.x & 31);
    bool active = slot < G.m;
    const int64_t q = active && G.perm ? checked_index((int64_t)G.perm[slot], G.m, a.err, BAD_ORDER) : slot;
    float x[D];
    RegList<K> h;
    h.init(nullptr);
    int64_t gid = 0;
    int32_t cur = NULL_CHILD;
    int sp = 0;
    if (active) {
      int s;
      lane_query<D>(a, G, q, s, gid, x);
      cur = __ldg(G.roots + s);
    }
    bool finished = !active;
    if (active && cur == NULL_CHILD) active = false;
    int64_t steps = 0;
    while (__any_sync(0xffffffffu, active)) {
      if (active && ++steps > G.max_steps) {  // runaway traversal: stop and report
        atomicOr(a.err, DEVERR_INTERNAL);
        active = false;
      }
      if (active) {
        const Kids<D> k = unpack(load_node_global<Node<D>, false>(g + checked_index(cur, G.nnodes, a.err, BAD_NODE)));  // 16-byte loads: see load_node_global
        const bool v1 = k.child[1] != NULL_CHILD;
        const float d0 = box_d2<D>(x, k.lo[0], k.hi[0]);
        const float d1 = v1 ? box_d2<D>(x, k.lo[1], k.hi[1]) : F_INF;
        h.insert2(k.child[0] < 0, d0, k.orig[0], v1 && k.child[1] < 0, d1, k.orig[1]);
        const float worst = h.worst_d();
        const bool g0 = k.child[0] >= 0 && d0 <= worst;
        const bool g1 = v1 && k.child[1] >= 0 && d1 <= worst;
        int32_t next = -1;
        bool done = false;
        if (g0 && g1) {
          const bool first1 = d1 < d0;
          next = first1 ? k.child[1] : k.child[0];
          if (sp < STACK_DEPTH) {
            st[sp] = first1 ? k.child[0] : k.child[1];
            sb[sp] = first1 ? d0 : d1;
            ++sp;
          } else {
            atomicOr(a.err, DEVERR_STACK);
            done = true;
          }
        } else if (g0) {
          next = k.child[0];
        } else if (g1) {
          next = k.child[1];
        }
        if (!done && next < 0) {
          while (sp > 0 && sb[sp - 1] > h.worst_d()) --sp;
          if (sp > 0) next = st[--sp];
          else done = true;
        }
        cur = next;
        if (done) active = false;
      }
    }
    if (!finished) {
      int32_t* oi = a.knn_idx + gid * a.k;
      float* od = a.knn_d2 ? a.knn_d2 + gid * a.k : nullptr;
      h.write(oi, od, a.k);
    }
  }
}

// Warp-collective: the first slot of the next chunk (uniform across the warp), or -1.
__device__ __forceinline__ int64_t next_chunk(const FArgs& a) {
  unsigned long long c = 0;
  if ((threadIdx.x & 31) == 0) c = atomicAdd(a.counter, (unsigned long long)a.chunk);
  c = __shfl_sync(0xffffffffu, c, 0);
  return (int64_t)c < a.slots ? (int64_t)c : -1;
}

__device__ __forceinline__ int group_of(const FArgs& a, int64_t c) {
  int gi = 0;
  for (int h = 1; h < a.ngroups; ++h)
    if (c >= a.g[h].slot_base) gi = h;
  return gi;
}

template <int MODE>
__global__ void __launch_bounds__(F_THREADS) k_forest_spatial(FArgs a) {
  for (;;) {
    const int64_t c = next_chunk(a);
    if (c < 0) break;
    const int gi = group_of(a, c);
    switch (a.dims[gi]) {
      case 2: f_spatial_chunk<2, MODE>(a, a.g[gi], c); break;
      case 3: f_spatial_chunk<3, MODE>(a, a.g[gi], c); break;
      default: f_spatial_chunk<6, MODE>(a, a.g[gi], c); break;
    }
  }
}

template <int K>
__global__ void __launch_bounds__(F_THREADS) k_forest_knn(FArgs a) {
  for (;;) {
    const int64_t c = next_chunk(a);
    if (c < 0) break;
    const int gi = group_of(a, c);
    switch (a.dims[gi]) {
      case 2: f_knn_chunk<2, K>(a, a.g[gi], c); break;
      case 3: f_knn_chunk<3, K>(a, a.g[gi], c); break;
      default: f_knn_chunk<6, K>(a, a.g[gi], c); break;
    }
  }
}

}  // namespace
}  // namespace arbx

// ------------------------------------------------------------------ host objects

struct ForestGroup {
  int dim = 0;
  std::vector<int32_t> sets;  // global set index of each group set
  int64_t npts = 0;
  void* nodes = nullptr;       // Node<dim>[max(npts, 1)]
  int32_t* roots = nullptr;    // [ns]
  int64_t* pbase = nullptr;    // [ns+1] group-local point prefix
  int32_t* npts_dev = nullptr; // [ns]
  float* frame = nullptr;      // [ns][2*dim]: each set's Morton frame (lo, cells per unit)
};

struct arbx_forest_t {
  int device = 0;
  int32_t nsets = 0;
  std::vector<int32_t> dims;
  std::vector<int64_t> counts;
  int64_t total_points = 0;
  ForestGroup groups[3];
};

struct arbx_forest_batch_t {
  arbx_forest_t* f = nullptr;
  int64_t total_queries = 0;
  int64_t slots = 0;
  // per group device arrays
  int64_t* qbase[3] = {};
  int64_t* gq[3] = {};
  int64_t* qfoff[3] = {};
  float* r2[3] = {};
  int64_t slot_base[3] = {};
  int64_t gm[3] = {};
  // query order per group: sort keys and values (ping-pong)
  uint64_t* qk[3] = {};
  uint64_t* qk_alt[3] = {};
  uint32_t* qv[3] = {};
  uint32_t* qv_alt[3] = {};
  arbx_forest_tuning tune{256, 32, {1, 1, 1}};
  // temporaries owned by the batch (no allocation in the query calls)
  int32_t* counts = nullptr;
  int64_t* scan_temp = nullptr;
  unsigned long long* counters = nullptr;  // [2]: spatial, nearest
  uint32_t* err = nullptr;
};

struct arbx_graph_t {
  int device = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace arbx {
namespace {

template <int D>
arbx_status build_group(ForestGroup& G, const float* data, const std::vector<int64_t>& foff_all,
                        const std::vector<int64_t>& counts, uint32_t* err, cudaStream_t s) {
  const int ns = (int)G.sets.size();
  std::vector<int64_t> pbase(ns + 1, 0), foff(ns);
  std::vector<int32_t> np(ns);
  for (int j = 0; j < ns; ++j) {
    pbase[j + 1] = pbase[j] + counts[G.sets[j]];
    foff[j] = foff_all[G.sets[j]];
    np[j] = (int32_t)counts[G.sets[j]];
  }
  G.npts = pbase[ns];
  if (G.npts >= (int64_t(1) << 31)) return ARBX_ERR_UNSUPPORTED;
  ARBX_TRY(dev_alloc_t(&G.pbase, ns + 1, s));
  ARBX_TRY(dev_alloc_t(&G.roots, ns, s));
  ARBX_TRY(dev_alloc_t(&G.npts_dev, ns, s));
  Node<D>* nodes = nullptr;
  ARBX_TRY(dev_alloc_t(&nodes, std::max<int64_t>(G.npts, 1), s));
  G.nodes = nodes;
  DevTemp<int64_t> foff_d(s);
  ARBX_TRY(foff_d.alloc(ns));
  ARBX_CUDA(cudaMemcpyAsync(G.pbase, pbase.data(), (ns + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  ARBX_CUDA(cudaMemcpyAsync(foff_d.p, foff.data(), ns * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  ARBX_CUDA(cudaMemcpyAsync(G.npts_dev, np.data(), ns * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  const int64_t n = G.npts;
  ARBX_TRY(dev_alloc_t(&G.frame, (size_t)ns * 2 * D, s));
  ARBX_LAUNCH("forest_bounds", s, k_f_bounds<D><<<ns, F_THREADS, 0, s>>>(data, foff_d.p, G.pbase, ns, G.frame, err));
  if (n == 0) return ARBX_OK;
  DevTemp<uint64_t> keys(s), keys_alt(s);
  DevTemp<uint32_t> vals(s), vals_alt(s);
  ARBX_TRY(keys.alloc(n));
  ARBX_TRY(keys_alt.alloc(n));
  ARBX_TRY(vals.alloc(n));
  ARBX_TRY(vals_alt.alloc(n));
  const unsigned grid = (unsigned)((n + F_THREADS - 1) / F_THREADS);
  ARBX_LAUNCH("forest_morton", s,
              k_f_morton<D><<<grid, F_THREADS, 0, s>>>(data, foff_d.p, G.pbase, ns, n, G.frame, keys.p, vals.p));
  bool alt = false;
  ARBX_TRY(radix_sort_pairs<uint64_t>(keys.p, vals.p, keys_alt.p, vals_alt.p, n, 0, 64, &alt, s));
  const uint64_t* skeys = alt ? keys_alt.p : keys.p;
  const uint32_t* perm = alt ? vals_alt.p : vals.p;
  DevTemp<float> spts(s);
  ARBX_TRY(spts.alloc((size_t)n * D));
  ARBX_LAUNCH("forest_gather", s,
              k_f_gather<D><<<grid, F_THREADS, 0, s>>>(data, foff_d.p, G.pbase, n, perm, skeys, spts.p));
  DevTemp<int32_t> flags(s);
  ARBX_TRY(flags.alloc(n));
  ARBX_CUDA(cudaMemsetAsync(flags.p, 0xff, (size_t)n * sizeof(int32_t), s));
  ARBX_LAUNCH("forest_apetrei", s,
              k_f_apetrei<D><<<grid, F_THREADS, 0, s>>>(skeys, perm, spts.p, G.pbase, (int)n, flags.p, nodes, G.roots));
  return ARBX_OK;
}

// Empty sets keep the root NULL_CHILD.
__global__ void k_f_empty_roots(const int64_t* pbase, int ns, int32_t* roots) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < ns && pbase[j + 1] == pbase[j]) roots[j] = NULL_CHILD;
}

void free_group(ForestGroup& G) {
  void* ptrs[] = {G.nodes, G.roots, G.pbase, G.npts_dev, G.frame};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  G = ForestGroup();
}

FArgs make_args(const arbx_forest_batch_t* b, const float* queries) {
  FArgs a;
  std::memset(&a, 0, sizeof(a));
  int ng = 0;
  for (int gi = 0; gi < 3; ++gi) {
    const ForestGroup& G = b->f->groups[gi];
    if (b->gm[gi] == 0) continue;
    FGroup& g = a.g[ng];
    g.nodes = G.nodes;
    g.nnodes = std::max<int64_t>(G.npts, 1);
    g.ns = (int)G.sets.size();
    g.qbase = b->qbase[gi];
    g.gq = b->gq[gi];
    g.qfoff = b->qfoff[gi];
    g.roots = G.roots;
    g.r2 = b->r2[gi];
    g.npts = G.npts_dev;
    g.slot_base = b->slot_base[gi];
    g.m = b->gm[gi];
    g.max_steps = 4 * G.npts + 1024;
    a.dims[ng] = G.dim;
    ++ng;
  }
  a.ngroups = ng;
  a.qs = queries;
  a.slots = b->slots;
  a.chunk = b->tune.chunk;
  a.err = b->err;
  return a;
}

// Processing order of every group's queries for one call (the queries may
// differ between calls): set-major, Morton order inside each set.
arbx_status order_queries(const arbx_forest_batch_t* b, FArgs& a, cudaStream_t s) {
  int ng = 0;
  for (int gi = 0; gi < 3; ++gi) {
    if (b->gm[gi] == 0) continue;
    FGroup& g = a.g[ng++];
    if (g.m < 2 || !b->qk[gi] || b->tune.sort_queries[gi] == 0) continue;
    const ForestGroup& G = b->f->groups[gi];
    const unsigned grid = (unsigned)((g.m + 255) / 256);
    switch (G.dim) {
      case 2: ARBX_LAUNCH("forest_query_codes", s, k_f_query_codes<2><<<grid, 256, 0, s>>>(a.qs, g, G.frame, b->qk[gi], b->qv[gi])); break;
      case 3: ARBX_LAUNCH("forest_query_codes", s, k_f_query_codes<3><<<grid, 256, 0, s>>>(a.qs, g, G.frame, b->qk[gi], b->qv[gi])); break;
      default: ARBX_LAUNCH("forest_query_codes", s, k_f_query_codes<6><<<grid, 256, 0, s>>>(a.qs, g, G.frame, b->qk[gi], b->qv[gi])); break;
    }
    int set_bits = 0;
    while ((1 << set_bits) < g.ns) ++set_bits;
    bool alt = false;
    ARBX_TRY(radix_sort_pairs<uint64_t>(b->qk[gi], b->qv[gi], b->qk_alt[gi], b->qv_alt[gi], g.m, 0, 48 + set_bits,
                                        &alt, s));
    g.perm = alt ? b->qv_alt[gi] : b->qv[gi];
  }
  return ARBX_OK;
}

int forest_grid(const void* kern, int block) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, block, 0);
  return std::max(1, per_sm) * num_sms();
}

bool is_capturing(cudaStream_t s) {
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s, &st);
  return st != cudaStreamCaptureStatusNone;
}

bool valid_tuning(const arbx_forest_tuning& t) {
  if (t.block != 128 && t.block != 256) return false;
  if (t.chunk != 32 && t.chunk != 64) return false;
  for (int gi = 0; gi < 3; ++gi)
    if (t.sort_queries[gi] != 0 && t.sort_queries[gi] != 1) return false;
  return true;
}

// Recorded forest settings, keyed by GPU model, the dimension groups present
// (bit gi for dims 2, 3, 6) and floor(log4) of the batch's query count; set
// by arbx_forest_autotune, applied to new batches with the same key.
struct FKey {
  std::string gpu;
  int dims_mask, mb;
  bool operator<(const FKey& o) const { return std::tie(gpu, dims_mask, mb) < std::tie(o.gpu, o.dims_mask, o.mb); }
};
std::mutex g_ftune_mu;
std::map<FKey, arbx_forest_tuning> g_ftune;

std::string device_name() {
  cudaDeviceProp prop;
  int d = 0;
  cudaGetDevice(&d);
  std::string n = cudaGetDeviceProperties(&prop, d) == cudaSuccess ? prop.name : "unknown";
  for (char& c : n)
    if (c == ' ') c = '_';
  return n;
}

FKey batch_key(const arbx_forest_batch_t* b) {
  int mask = 0;
  for (int gi = 0; gi < 3; ++gi)
    if (b->gm[gi] > 0) mask |= 1 << gi;
  int mb = 0;
  for (int64_t v = b->total_queries; v > 1; v >>= 2) ++mb;
  return FKey{device_name(), mask, mb};
}
}  // namespace

// Forest records in the autotune text file (lines starting with "forest").
void forest_records_save(FILE* f) {
  std::lock_guard<std::mutex> lk(g_ftune_mu);
  for (const auto& kv : g_ftune) {
    const arbx_forest_tuning& t = kv.second;
    std::fprintf(f, "forest %s %d %d %d %d %d %d %d\n", kv.first.gpu.c_str(), kv.first.dims_mask, kv.first.mb,
                 t.block, t.chunk, t.sort_queries[0], t.sort_queries[1], t.sort_queries[2]);
  }
}

bool forest_record_load(const char* line) {
  char gpu[256];
  FKey k;
  arbx_forest_tuning t{};
  if (std::sscanf(line, "forest %255s %d %d %d %d %d %d %d", gpu, &k.dims_mask, &k.mb, &t.block, &t.chunk,
                  &t.sort_queries[0], &t.sort_queries[1], &t.sort_queries[2]) != 8)
    return false;
  if (!valid_tuning(t)) return false;
  k.gpu = gpu;
  std::lock_guard<std::mutex> lk(g_ftune_mu);
  g_ftune[k] = t;
  return true;
}

void forest_records_clear() {
  std::lock_guard<std::mutex> lk(g_ftune_mu);
  g_ftune.clear();
}
}  // namespace arbx

using namespace arbx;

extern "C" {

arbx_status arbx_forest_build(arbx_forest* out, int32_t nsets, const int32_t* dims_host, const int64_t* counts_host,
                              const float* data_dev, arbx_stream stream) {
  if (!out || nsets <= 0 || !dims_host || !counts_host) return ARBX_ERR_INVALID;
  *out = nullptr;
  int64_t total = 0, floats = 0;
  int per_dim[3] = {0, 0, 0};
  for (int s = 0; s < nsets; ++s) {
    const int d = dims_host[s];
    const int gi = d == 2 ? 0 : d == 3 ? 1 : d == 6 ? 2 : -1;
    if (d < 1 || d > 10) return ARBX_ERR_INVALID;
    if (gi < 0) return ARBX_ERR_UNSUPPORTED;
    if (counts_host[s] < 0 || counts_host[s] > MAX_PRIMS) return ARBX_ERR_INVALID;
    if (++per_dim[gi] > MAX_GROUP_SETS) return ARBX_ERR_UNSUPPORTED;
    total += counts_host[s];
    floats += counts_host[s] * d;
  }
  if (floats > 0 && !data_dev) return ARBX_ERR_INVALID;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  uint32_t* err = nullptr;
  ARBX_TRY(device_error_word(&err));
  ARBX_TRY(check_stream(s));
  arbx_forest_t* f = new arbx_forest_t;
  cudaGetDevice(&f->device);
  f->nsets = nsets;
  f->dims.assign(dims_host, dims_host + nsets);
  f->counts.assign(counts_host, counts_host + nsets);
  f->total_points = total;
  std::vector<int64_t> foff(nsets);
  int64_t acc = 0;
  for (int s2 = 0; s2 < nsets; ++s2) {
    foff[s2] = acc;
    acc += counts_host[s2] * dims_host[s2];
  }
  arbx_status st = ARBX_OK;
  for (int gi = 0; gi < 3 && st == ARBX_OK; ++gi) {
    ForestGroup& G = f->groups[gi];
    G.dim = GROUP_DIMS[gi];
    for (int s2 = 0; s2 < nsets; ++s2)
      if (dims_host[s2] == G.dim) G.sets.push_back(s2);
    if (G.sets.empty()) continue;
    if (G.dim == 2) st = build_group<2>(G, data_dev, foff, f->counts, err, s);
    else if (G.dim == 3) st = build_group<3>(G, data_dev, foff, f->counts, err, s);
    else st = build_group<6>(G, data_dev, foff, f->counts, err, s);
    if (st == ARBX_OK) {
      const int ns = (int)G.sets.size();
      k_f_empty_roots<<<(ns + 255) / 256, 256, 0, s>>>(G.pbase, ns, G.roots);
      g_launches.fetch_add(1);
      if (cudaGetLastError() != cudaSuccess) st = ARBX_ERR_CUDA;
    }
  }
  if (st == ARBX_OK) st = check_stream(s);
  if (st != ARBX_OK) {
    arbx_forest_destroy(f);
    return st;
  }
  *out = f;
  return ARBX_OK;
}

arbx_status arbx_forest_destroy(arbx_forest f) {
  if (!f) return ARBX_OK;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(f->device);
  cudaDeviceSynchronize();
  for (auto& G : f->groups) free_group(G);
  cudaSetDevice(prev);
  delete f;
  return ARBX_OK;
}

arbx_status arbx_forest_info(arbx_forest f, int32_t* nsets_out, int64_t* points_out) {
  if (!f) return ARBX_ERR_INVALID;
  if (nsets_out) *nsets_out = f->nsets;
  if (points_out) *points_out = f->total_points;
  return ARBX_OK;
}

arbx_status arbx_forest_batch_create(arbx_forest_batch* out, arbx_forest f, const int64_t* qcounts_host,
                                     const float* radii_host, arbx_stream stream) {
  if (!out || !f || !qcounts_host) return ARBX_ERR_INVALID;
  *out = nullptr;
  for (int s = 0; s < f->nsets; ++s) {
    if (qcounts_host[s] < 0) return ARBX_ERR_INVALID;
    if (radii_host) {
      const float r = radii_host[s];
      if (!(r == r) || r - r != 0.0f || r < 0.0f) return ARBX_ERR_INVALID;
    }
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  arbx_forest_batch_t* b = new arbx_forest_batch_t;
  b->f = f;
  // global query ids: sets in input order; float offsets of each set's queries
  std::vector<int64_t> gq(f->nsets), qfoff(f->nsets);
  int64_t acc = 0, facc = 0;
  for (int s2 = 0; s2 < f->nsets; ++s2) {
    gq[s2] = acc;
    qfoff[s2] = facc;
    acc += qcounts_host[s2];
    facc += qcounts_host[s2] * f->dims[s2];
  }
  b->total_queries = acc;
  auto fail = [&](arbx_status st) {
    arbx_forest_batch_destroy(b);
    return st;
  };
  int64_t slot = 0;
  for (int gi = 0; gi < 3; ++gi) {
    const ForestGroup& G = f->groups[gi];
    const int ns = (int)G.sets.size();
    if (ns == 0) continue;
    std::vector<int64_t> qb(ns + 1, 0), g_gq(ns), g_qf(ns);
    std::vector<float> r2(ns);
    for (int j = 0; j < ns; ++j) {
      const int set = G.sets[j];
      qb[j + 1] = qb[j] + qcounts_host[set];
      g_gq[j] = gq[set];
      g_qf[j] = qfoff[set];
      const float r = radii_host ? radii_host[set] : 0.0f;
      r2[j] = r * r;  // fl(r*r), one IEEE multiply
    }
    b->gm[gi] = qb[ns];
    b->slot_base[gi] = slot;
    if (qb[ns] > 1) {
      arbx_status sa;
      if ((sa = dev_alloc_t(&b->qk[gi], qb[ns], s)) != ARBX_OK || (sa = dev_alloc_t(&b->qk_alt[gi], qb[ns], s)) != ARBX_OK ||
          (sa = dev_alloc_t(&b->qv[gi], qb[ns], s)) != ARBX_OK || (sa = dev_alloc_t(&b->qv_alt[gi], qb[ns], s)) != ARBX_OK)
        return fail(sa);
    }
    slot += (qb[ns] + F_MAX_CHUNK - 1) / F_MAX_CHUNK * F_MAX_CHUNK;
    arbx_status st;
    if ((st = dev_alloc_t(&b->qbase[gi], ns + 1, s)) != ARBX_OK || (st = dev_alloc_t(&b->gq[gi], ns, s)) != ARBX_OK ||
        (st = dev_alloc_t(&b->qfoff[gi], ns, s)) != ARBX_OK || (st = dev_alloc_t(&b->r2[gi], ns, s)) != ARBX_OK)
      return fail(st);
    if (cudaMemcpyAsync(b->qbase[gi], qb.data(), (ns + 1) * 8, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(b->gq[gi], g_gq.data(), ns * 8, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(b->qfoff[gi], g_qf.data(), ns * 8, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(b->r2[gi], r2.data(), ns * 4, cudaMemcpyHostToDevice, s) != cudaSuccess)
      return fail(ARBX_ERR_CUDA);
    if (cudaStreamSynchronize(s) != cudaSuccess) return fail(ARBX_ERR_CUDA);  // host vectors go out of scope
  }
  b->slots = slot;
  const int64_t m = b->total_queries;
  arbx_status st;
  if ((st = dev_alloc_t(&b->counts, std::max<int64_t>(m, 1), s)) != ARBX_OK ||
      (st = dev_alloc_t(&b->scan_temp, std::max<int64_t>(scan_temp_elems(m), 1), s)) != ARBX_OK ||
      (st = dev_alloc_t(&b->counters, 2, s)) != ARBX_OK)
    return fail(st);
  if ((st = device_error_word(&b->err)) != ARBX_OK) return fail(st);
  if (cudaStreamSynchronize(s) != cudaSuccess) return fail(ARBX_ERR_CUDA);
  {
    std::lock_guard<std::mutex> lk(g_ftune_mu);
    auto it = g_ftune.find(batch_key(b));
    if (it != g_ftune.end()) b->tune = it->second;
  }
  *out = b;
  return ARBX_OK;
}

arbx_status arbx_forest_batch_set_tuning(arbx_forest_batch b, const arbx_forest_tuning* tuning) {
  if (!b) return ARBX_ERR_INVALID;
  arbx_forest_tuning t{256, 32, {1, 1, 1}};
  if (tuning) {
    t = *tuning;
    if (t.block == 0) t.block = 256;
    if (t.chunk == 0) t.chunk = 32;
    for (int gi = 0; gi < 3; ++gi)
      if (t.sort_queries[gi] < 0) t.sort_queries[gi] = 1;
    if (!valid_tuning(t)) return ARBX_ERR_INVALID;
  }
  b->tune = t;
  return ARBX_OK;
}

arbx_status arbx_forest_batch_get_tuning(arbx_forest_batch b, arbx_forest_tuning* out) {
  if (!b || !out) return ARBX_ERR_INVALID;
  *out = b->tune;
  return ARBX_OK;
}

arbx_status arbx_forest_batch_destroy(arbx_forest_batch b) {
  if (!b) return ARBX_OK;
  cudaDeviceSynchronize();
  for (int gi = 0; gi < 3; ++gi) {
    void* ptrs[] = {b->qbase[gi], b->gq[gi], b->qfoff[gi], b->r2[gi], b->qk[gi], b->qk_alt[gi], b->qv[gi], b->qv_alt[gi]};
    for (void* p : ptrs)
      if (p) cudaFree(p);
  }
  void* ptrs[] = {b->counts, b->scan_temp, b->counters};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete b;
  return ARBX_OK;
}

arbx_status arbx_forest_batch_total(arbx_forest_batch b, int64_t* total_queries) {
  if (!b || !total_queries) return ARBX_ERR_INVALID;
  *total_queries = b->total_queries;
  return ARBX_OK;
}

arbx_status arbx_forest_query_radius(arbx_forest_batch b, const float* queries_dev, int64_t* offsets_dev,
                                     int32_t* indices_dev, float* d2_dev, int64_t capacity, int64_t* nnz_dev,
                                     arbx_stream stream) {
  if (!b || !offsets_dev || capacity < 0) return ARBX_ERR_INVALID;
  if (b->total_queries > 0 && !queries_dev) return ARBX_ERR_INVALID;
  if (capacity > 0 && (!indices_dev || !d2_dev)) return ARBX_ERR_INVALID;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int64_t m = b->total_queries;
  if (m == 0) {
    ARBX_CUDA(cudaMemsetAsync(offsets_dev, 0, sizeof(int64_t), s));
    if (nnz_dev) ARBX_CUDA(cudaMemsetAsync(nnz_dev, 0, sizeof(int64_t), s));
    return ARBX_OK;
  }
  FArgs a = make_args(b, queries_dev);
  ARBX_TRY(order_queries(b, a, s));
  a.counts = b->counts;
  a.counter = b->counters;
  const int block = b->tune.block;
  ARBX_CUDA(cudaMemsetAsync(b->counters, 0, sizeof(unsigned long long), s));
  {
    auto kern = k_forest_spatial<MODE_COUNT>;
    ARBX_LAUNCH("forest_count", s, kern<<<forest_grid((const void*)kern, block), block, 0, s>>>(a));
  }
  ARBX_TRY(exclusive_scan_temp(b->counts, offsets_dev, m, b->scan_temp, s));
  if (nnz_dev) ARBX_CUDA(cudaMemcpyAsync(nnz_dev, offsets_dev + m, sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
  if (capacity > 0) {
    a.offsets = offsets_dev;
    a.out_idx = indices_dev;
    a.out_d2 = d2_dev;
    a.capacity = capacity;
    ARBX_CUDA(cudaMemsetAsync(b->counters, 0, sizeof(unsigned long long), s));
    auto kern = k_forest_spatial<MODE_FILL>;
    ARBX_LAUNCH("forest_fill", s, kern<<<forest_grid((const void*)kern, block), block, 0, s>>>(a));
  }
  return ARBX_OK;
}

arbx_status arbx_forest_query_knn(arbx_forest_batch b, const float* queries_dev, int32_t k, int32_t* indices_dev,
                                  float* d2_dev, arbx_stream stream) {
  if (!b || k <= 0) return ARBX_ERR_INVALID;
  if (k > 32) return ARBX_ERR_UNSUPPORTED;
  if (b->total_queries > 0 && (!queries_dev || !indices_dev)) return ARBX_ERR_INVALID;
  if (b->total_queries == 0) return ARBX_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  FArgs a = make_args(b, queries_dev);
  ARBX_TRY(order_queries(b, a, s));
  a.knn_idx = indices_dev;
  a.knn_d2 = d2_dev;
  a.k = k;
  a.counter = b->counters + 1;
  ARBX_CUDA(cudaMemsetAsync(b->counters + 1, 0, sizeof(unsigned long long), s));
  const int block = b->tune.block;
  auto go = [&](auto kern) -> arbx_status {
    ARBX_LAUNCH("forest_knn", s, kern<<<forest_grid((const void*)kern, block), block, 0, s>>>(a));
    return ARBX_OK;
  };
  if (k <= 1) return go(k_forest_knn<1>);
  if (k <= 2) return go(k_forest_knn<2>);
  if (k <= 4) return go(k_forest_knn<4>);
  if (k <= 8) return go(k_forest_knn<8>);
  if (k <= 16) return go(k_forest_knn<16>);
  return go(k_forest_knn<32>);
}

arbx_status arbx_forest_autotune(arbx_forest_batch b, const float* queries_dev, int32_t k, arbx_forest_tuning* best_out,
                                 double* best_ms_out, arbx_stream stream) {
  if (!b || !best_out || k < 0 || k > 32) return ARBX_ERR_INVALID;
  if (b->total_queries > 0 && !queries_dev) return ARBX_ERR_INVALID;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int64_t m = b->total_queries;
  const arbx_forest_tuning keep = b->tune;
  *best_out = keep;
  if (best_ms_out) *best_ms_out = 0.0;
  if (m == 0) return ARBX_OK;
  // outputs of the timed calls: sized by one count pass under the current setting
  DevTemp<int64_t> offsets(s), nnz(s);
  ARBX_TRY(offsets.alloc(m + 1));
  ARBX_TRY(nnz.alloc(1));
  ARBX_TRY(arbx_forest_query_radius(b, queries_dev, offsets.p, nullptr, nullptr, 0, nnz.p, stream));
  int64_t total = 0;
  ARBX_TRY(read_small(nnz.p, &total, sizeof(total), s));
  DevTemp<int32_t> idx(s), kidx(s);
  DevTemp<float> d2(s), kd2(s);
  ARBX_TRY(idx.alloc(total));
  ARBX_TRY(d2.alloc(total));
  if (k > 0) {
    ARBX_TRY(kidx.alloc(m * k));
    ARBX_TRY(kd2.alloc(m * k));
  }
  cudaEvent_t e0, e1;
  ARBX_CUDA(cudaEventCreate(&e0));
  ARBX_CUDA(cudaEventCreate(&e1));
  // one candidate: the radius query (count, scan, fill) and the nearest query, as the graph runs them
  auto run = [&](const arbx_forest_tuning& t, float* ms) -> arbx_status {
    b->tune = t;
    for (int rep = 0; rep < 2; ++rep) {  // the first run warms up
      if (rep == 1) cudaEventRecord(e0, s);
      ARBX_TRY(arbx_forest_query_radius(b, queries_dev, offsets.p, idx.p, d2.p, total, nnz.p, stream));
      if (k > 0) ARBX_TRY(arbx_forest_query_knn(b, queries_dev, k, kidx.p, kd2.p, stream));
    }
    cudaEventRecord(e1, s);
    ARBX_CUDA(cudaEventSynchronize(e1));
    ARBX_CUDA(cudaEventElapsedTime(ms, e0, e1));
    return ARBX_OK;
  };
  // coordinate search: each dimension group's query ordering (the others
  // kept), then block size x chunk size
  arbx_forest_tuning best{256, 32, {1, 1, 1}};
  float best_ms = 0.0f;
  arbx_status st = run(best, &best_ms);
  for (int gi = 0; gi < 3 && st == ARBX_OK; ++gi) {
    if (b->gm[gi] == 0) continue;
    arbx_forest_tuning t = best;
    t.sort_queries[gi] = 0;
    float ms = 0.0f;
    if ((st = run(t, &ms)) == ARBX_OK && ms < best_ms) {
      best = t;
      best_ms = ms;
    }
  }
  for (int block : {128, 256}) {
    for (int chunk : {32, 64}) {
      if (st != ARBX_OK) break;
      if (block == best.block && chunk == best.chunk) continue;
      arbx_forest_tuning t = best;
      t.block = block;
      t.chunk = chunk;
      float ms = 0.0f;
      if ((st = run(t, &ms)) == ARBX_OK && ms < best_ms) {
        best = t;
        best_ms = ms;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st == ARBX_OK) st = check_stream(s);
  if (st != ARBX_OK) {
    b->tune = keep;
    return st;
  }
  b->tune = best;
  {
    std::lock_guard<std::mutex> lk(g_ftune_mu);
    g_ftune[batch_key(b)] = best;
  }
  *best_out = best;
  if (best_ms_out) *best_ms_out = best_ms;
  return ARBX_OK;
}

arbx_status arbx_forest_graph_create(arbx_graph* out, arbx_forest_batch b, const float* queries_dev,
                                     int64_t* offsets_dev, int32_t* indices_dev, float* d2_dev, int64_t capacity,
                                     int64_t* nnz_dev, int32_t k, int32_t* knn_idx_dev, float* knn_d2_dev,
                                     arbx_stream stream) {
  if (!out || !b || !stream) return ARBX_ERR_INVALID;  // capture needs a non-default stream
  *out = nullptr;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (is_capturing(s)) return ARBX_ERR_INVALID;
  ARBX_CUDA(cudaStreamSynchronize(s));
  arbx_graph_t* g = new arbx_graph_t;
  cudaGetDevice(&g->device);
  ARBX_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  arbx_status st = arbx_forest_query_radius(b, queries_dev, offsets_dev, indices_dev, d2_dev, capacity, nnz_dev, stream);
  if (st == ARBX_OK && k > 0) st = arbx_forest_query_knn(b, queries_dev, k, knn_idx_dev, knn_d2_dev, stream);
  cudaGraph_t graph = nullptr;
  const cudaError_t e = cudaStreamEndCapture(s, &graph);
  if (st == ARBX_OK && e != cudaSuccess) st = cuda_status(e, "cudaStreamEndCapture", __FILE__, __LINE__);
  if (st == ARBX_OK && cudaGraphInstantiate(&g->exec, graph, 0) != cudaSuccess) st = ARBX_ERR_CUDA;
  g->graph = graph;
  if (st != ARBX_OK) {
    arbx_graph_destroy(g);
    cudaGetLastError();
    return st;
  }
  *out = g;
  return ARBX_OK;
}

arbx_status arbx_graph_launch(arbx_graph g, arbx_stream stream) {
  if (!g) return ARBX_ERR_INVALID;
  ARBX_CUDA(cudaGraphLaunch(g->exec, reinterpret_cast<cudaStream_t>(stream)));
  return ARBX_OK;
}

arbx_status arbx_graph_destroy(arbx_graph g) {
  if (!g) return ARBX_OK;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  delete g;
  return ARBX_OK;
}

}  // extern "C"
