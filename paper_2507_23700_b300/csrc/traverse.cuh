// Device-side building blocks shared by the traversal kernels of query.cu
// (single trees) and forest.cu (batches of trees): node unpacking, the
// predicates, the warp work queue, the sorted k-best list and the ray tests.
#pragma once

#include "common.cuh"

namespace arbx {
namespace {

constexpr float F_INF = __builtin_huge_valf();

// ------------------------------------------------------------------ nodes

template <int D>
struct Kids {
  float lo[2][D];
  float hi[2][D];
  int32_t child[2];
  int32_t orig[2];
};

template <int D>
__device__ __forceinline__ Kids<D> unpack(const Node<D>& n) {
  Kids<D> k;
#pragma unroll
  for (int a = 0; a < D; ++a) {
    k.lo[0][a] = n.lo0[a];
    k.hi[0][a] = n.hi0[a];
    k.lo[1][a] = n.lo1[a];
    k.hi[1][a] = n.hi1[a];
  }
  k.child[0] = n.child[0];
  k.child[1] = n.child[1];
  k.orig[0] = n.orig[0];
  k.orig[1] = n.orig[1];
  return k;
}

// Decode the 16-bit child boxes (outward rounding; see k_quantize).
__device__ __forceinline__ Kids<3> unpack(const QNode& n) {
  Kids<3> k;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float step = pow2f(n.exps[a]);
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      k.lo[c][a] = __fmaf_rd((float)n.q[c][0][a], step, n.origin[a]);
      k.hi[c][a] = __fmaf_ru((float)n.q[c][1][a], step, n.origin[a]);
    }
  }
  k.child[0] = n.child[0];
  k.child[1] = n.child[1];
  k.orig[0] = k.orig[1] = -1;
  return k;
}

// Decode the parent-relative child boxes in the frame of the node's decoded box.
__device__ __forceinline__ Kids<3> unpack(const PNode& n, float4 fr) {
  Kids<3> k;
  const float o[3] = {fr.x, fr.y, fr.z};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float step = p16_step(fr, a);
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      k.lo[c][a] = p16_lo(o[a], n.q[c][0][a], step);
      k.hi[c][a] = p16_hi(o[a], n.q[c][1][a], step);
    }
  }
  k.child[0] = n.child[0];
  k.child[1] = n.child[1];
  k.orig[0] = k.orig[1] = -1;
  return k;
}

// The decoded-box frames a stack traversal carries: for parent-relative nodes
// one for the current node and one per stack entry (set when the entry's node
// is pushed, from the box its parent decoded); nothing for the formats whose
// records decode on their own.
template <class NodeT>
struct Frames {
  __device__ __forceinline__ void root(const TreeView&) {}
  template <class N>
  __device__ __forceinline__ auto open(const N& n) const { return unpack(n); }
  template <class K>
  __device__ __forceinline__ void go(const K&, int) {}
  template <class K>
  __device__ __forceinline__ void push(int, const K&, int) {}
  __device__ __forceinline__ void pop(int) {}
};

template <>
struct Frames<PNode> {
  float4 cur;
  float4 st[STACK_DEPTH];
  __device__ __forceinline__ void root(const TreeView& t) { cur = t.rframe; }
  __device__ __forceinline__ Kids<3> open(const PNode& n) const { return unpack(n, cur); }
  __device__ __forceinline__ void go(const Kids<3>& k, int c) { cur = p16_frame(k.lo[c], k.hi[c]); }
  __device__ __forceinline__ void push(int i, const Kids<3>& k, int c) { st[i] = p16_frame(k.lo[c], k.hi[c]); }
  __device__ __forceinline__ void pop(int i) { cur = st[i]; }
};

template <bool V8 = true, class NodeT>
__device__ __forceinline__ NodeT fetch(int32_t code, const TreeView& t, const NodeT* __restrict__ g,
                                       const NodeT* s) {
  if (code & TOP_FLAG) return load_node_shared(s + checked_index(code & ~TOP_FLAG, t.ntop, t.err, BAD_TOP));
  return load_node_global<NodeT, V8>(g + node_index(code, t));
}

// Copy the top-level nodes into shared memory (all threads of the block).
template <class NodeT>
__device__ __forceinline__ const NodeT* stage_top(const TreeView& t, float4* smem) {
  if (t.ntop > 0) {
    const float4* src = reinterpret_cast<const float4*>(t.top);
    const int nv = t.ntop * (int)(sizeof(NodeT) / 16);
    for (int i = threadIdx.x; i < nv; i += blockDim.x) smem[i] = __ldg(src + i);
  }
  __syncthreads();
  return reinterpret_cast<const NodeT*>(smem);
}

// ------------------------------------------------------------------ predicates

template <int D>
struct SpherePred {
  static constexpr bool LEAF_TEST = false;  // a leaf child's box is the primitive's own box
  static constexpr bool CONTAIN = true;
  float q[D];
  float r2;
  __device__ __forceinline__ bool test(const float* lo, const float* hi, float& d2) const {
    d2 = box_d2<D>(q, lo, hi);
    return d2 <= r2;
  }
  // The whole box lies within the radius: the d2 of its farthest corner (per
  // axis the larger of the two faces' terms, summed in dimension order) is <= r2.
  // A primitive box inside the box has a d2, computed as the leaf test computes
  // it, no larger than that bit for bit: the clamped coordinate lies between the
  // faces and fl-subtraction, squaring and fl-addition are monotone.  (Callers
  // test the box first, so a NaN query or radius never gets here.)
  __device__ __forceinline__ bool contains(const float* lo, const float* hi) const {
    float acc = fmaxf(sq_axis(q[0], lo[0]), sq_axis(q[0], hi[0]));
#pragma unroll
    for (int a = 1; a < D; ++a) acc = __fadd_rn(acc, fmaxf(sq_axis(q[a], lo[a]), sq_axis(q[a], hi[a])));
    return acc <= r2;
  }
  __device__ __forceinline__ void load(const float* __restrict__ qs, const float* __restrict__ radii, float r2u,
                                       int64_t i) {
#pragma unroll
    for (int a = 0; a < D; ++a) q[a] = qs[i * D + a];
    if (radii) {
      const float r = radii[i];
      r2 = __fmul_rn(r, r);
    } else {
      r2 = r2u;
    }
  }
};

template <int D>
struct BoxPred {
  static constexpr bool LEAF_TEST = false;
  static constexpr bool CONTAIN = true;
  float lo[D], hi[D];
  __device__ __forceinline__ bool test(const float* blo, const float* bhi, float& d2) const {
    d2 = 0.0f;
    return box_overlap<D>(lo, hi, blo, bhi);
  }
  // The box lies inside the query box, so every (non-inverted) primitive box
  // inside it overlaps the query box.
  __device__ __forceinline__ bool contains(const float* blo, const float* bhi) const {
    bool ok = true;
#pragma unroll
    for (int a = 0; a < D; ++a) ok = ok && (lo[a] <= blo[a]) && (bhi[a] <= hi[a]);
    return ok;
  }
  __device__ __forceinline__ void load(const float* __restrict__ qs, const float*, float, int64_t i) {
#pragma unroll
    for (int a = 0; a < D; ++a) {
      lo[a] = qs[i * 2 * D + a];
      hi[a] = qs[i * 2 * D + D + a];
    }
  }
};

// Exact leaf test of a triangle under a quantized (inflated) leaf box: the
// triangle's own bounding box from its leaf record.
template <class Pred>
__device__ __forceinline__ bool leaf_exact(const Pred& p, const TriLeaf* __restrict__ leaves, int32_t pos,
                                           int32_t& orig, float& d2) {
  const TriLeaf L = load_node_global(leaves + pos);
  float lo[3], hi[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    lo[a] = fminf(fminf(L.v[a], L.v[3 + a]), L.v[6 + a]);
    hi[a] = fmaxf(fmaxf(L.v[a], L.v[3 + a]), L.v[6 + a]);
  }
  orig = L.orig;
  return p.test(lo, hi, d2);
}

// Instrumented runs: add per-thread totals into stats[0..2] (warp-reduced).
__device__ __forceinline__ void add_stats(unsigned long long* stats, unsigned long long a, unsigned long long b,
                                          unsigned long long c) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
    c += __shfl_xor_sync(0xffffffffu, c, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(stats + 0, a);
    atomicAdd(stats + 1, b);
    atomicAdd(stats + 2, c);
  }
}

// ------------------------------------------------------------------ scheduling
//
// Traversal loops are warp-uniform: every lane of a warp runs the same
// iteration count (the loop ends when no lane of the warp has a query left),
// each iteration advances every active lane's traversal by one node, and lanes
// whose query is finished are refilled at the top of the next iteration.
// Divergent lanes therefore reconverge once per node step instead of running
// their traversals one after another.  Refills come from the warp's current
// chunk of CHUNK consecutive query slots (consecutive slots are neighbouring
// queries in Morton order, so a warp keeps working in one region); a warp
// takes its next chunk from a global counter, which balances the
// heavy-tailed per-query work across the GPU.

// One warp round per chunk: a heavy query's warp then holds one heavy round,
// not two, on the critical path (10M mixture, fill pass on 1M queries 7.4 ->
// 4.1 ms with 32 instead of 64; 10M queries 12.9 -> 12.8 ms).  A multiple of
// 32: the forest kernels walk a chunk in warp rounds.
constexpr int CHUNK = 32;

struct WarpQueue {
  int64_t next = 0, end = 0;
  bool exhausted = false;
};

// Warp-collective (all 32 lanes call it).  Lanes with !active receive the next
// slots of the warp's chunk; returns true for a lane that received one.  With
// chunk_perm, the i-th chunk handed out is chunk chunk_perm[i] of the slots.
__device__ __forceinline__ bool warp_refill(unsigned long long* counter, int64_t m, WarpQueue& q, bool active,
                                            int64_t& slot, const uint32_t* __restrict__ chunk_perm = nullptr) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  bool got = false;
  unsigned need = __ballot_sync(FULL, !active);
  while (need != 0u && !q.exhausted) {
    if (q.next >= q.end) {
      unsigned long long c = 0;
      if (lane == 0) c = atomicAdd(counter, (unsigned long long)CHUNK);
      c = __shfl_sync(FULL, c, 0);
      if ((int64_t)c >= m) {
        q.exhausted = true;
        break;
      }
      const int64_t base = chunk_perm ? (int64_t)chunk_perm[c / CHUNK] * CHUNK : (int64_t)c;
      q.next = base;
      q.end = min(base + CHUNK, m);
    }
    const int64_t avail = q.end - q.next;
    const int take = avail < (int64_t)__popc(need) ? (int)avail : __popc(need);
    const int rank = __popc(need & ((1u << lane) - 1u));
    if (((need >> lane) & 1u) && rank < take) {
      slot = q.next + rank;
      got = true;
    }
    q.next += take;
    need = __ballot_sync(FULL, !active && !got);
  }
  return got;
}

// Lane runs (nearest traversals): a warp of W walkers (32 lanes, or 32/L lane
// groups) takes W * RUN consecutive slots and answers them in RUN rounds of W
// adjacent slots, walker i taking slots i, W + i, 2W + i, ...  next() is
// warp-collective (called when no walker is busy): false when the work is
// exhausted; otherwise `slot` is the walker's slot of the round (possibly >= m
// in the last run) and `fresh` says that a new run started (the walker's
// previous query is not W slots back).
template <int RUN, int W = 32>
struct LaneRun {
  int64_t base = 0;
  int pos = RUN;
  __device__ __forceinline__ bool next(unsigned long long* counter, int64_t m, int walker, int64_t& slot,
                                       bool& fresh) {
    fresh = false;
    if (pos == RUN) {
      unsigned long long c = 0;
      if ((threadIdx.x & 31u) == 0) c = atomicAdd(counter, (unsigned long long)W * RUN);
      c = __shfl_sync(0xffffffffu, c, 0);
      if ((int64_t)c >= m) return false;
      base = (int64_t)c;
      pos = 0;
      fresh = true;
    }
    slot = base + (int64_t)pos * W + walker;
    ++pos;
    return true;
  }
};

// ------------------------------------------------------------------ stacks

// Per-thread stack of 64-bit entries for the nearest traversals (local memory).
// (Keeping the top 4, 8 or 16 entries in shared memory as a ring that spills
// its oldest entries here measured slower on the 10M mixture: kNN k=16 19.4 ms
// local, 22.3-23.6 ms with a ring.)
template <int DEPTH>
struct NNStack {
  unsigned long long e[DEPTH];
  int sp = 0;
  __device__ __forceinline__ void clear() { sp = 0; }
  __device__ __forceinline__ bool full() const { return sp >= DEPTH; }
  __device__ __forceinline__ void push(unsigned long long x) { e[sp++] = x; }  // !full()
  __device__ __forceinline__ unsigned long long pop() { return e[--sp]; }     // sp > 0
};

// A nearest-traversal stack entry: the node code above the bits of its box distance.
__device__ __forceinline__ unsigned long long nn_entry(int32_t code, float d) {
  return ((unsigned long long)(uint32_t)code << 32) | __float_as_uint(d);
}
__device__ __forceinline__ int32_t nn_code(unsigned long long e) { return (int32_t)(uint32_t)(e >> 32); }
__device__ __forceinline__ float nn_dist(unsigned long long e) { return __uint_as_float((uint32_t)e); }

// ------------------------------------------------------------------ fill staging

// Matches staged per lane before they are written (FILL mode).  A lane owns
// CAP slots of shared memory (plus a pad slot that keeps the flush reads free
// of bank conflicts).  flush() is warp-collective: once a lane has a sector's
// worth staged (8 entries of 4 bytes) it writes the entries up to the last
// 32-byte sector boundary its run reaches, and all of them when its query is
// finished, with consecutive lanes on consecutive addresses; the rest moves
// to the front of its slots.  Whole-sector stores keep the L2 from writing
// partial sectors back to DRAM (10M mixture: fill DRAM traffic 13.8 -> 9.2 GB).
constexpr int FILL_SECTOR = 8;  // entries per 32-byte sector

struct FillBuffer {
  static constexpr int CAP = 9;  // at most 7 entries stay after a flush, 2 more per step
  static constexpr int STRIDE = CAP + 1;
  int32_t* wi;  // this warp's index slots
  float* wd;    // this warp's distance slots
  int n = 0;    // entries staged by this lane

  static size_t bytes(int block) { return (size_t)block * STRIDE * (sizeof(int32_t) + sizeof(float)); }

  __device__ explicit FillBuffer(char* base) {
    int32_t* bi = reinterpret_cast<int32_t*>(base);
    float* bd = reinterpret_cast<float*>(base + (size_t)blockDim.x * STRIDE * sizeof(int32_t));
    const int w0 = (int)(threadIdx.x & ~31u) * STRIDE;
    wi = bi + w0;
    wd = bd + w0;
  }
  __device__ __forceinline__ static int slot(int lane, int i) { return lane * STRIDE + i; }
  // At most two pushes between flushes.
  __device__ __forceinline__ void push(int32_t j, float d) {
    const int me = slot((int)(threadIdx.x & 31u), n);
    wi[me] = j;
    wd[me] = d;
    ++n;
  }
  // Entries this lane writes now (see above).
  __device__ __forceinline__ int ready(bool finish, int64_t w) const {
    if (finish) return n;
    if (n < FILL_SECTOR) return 0;
    return (int)(((w + n) / FILL_SECTOR) * FILL_SECTOR - w);
  }
  // Write the ready entries of every lane at [w, w + cnt) (entries at or
  // beyond wend are dropped: the caller reports the mismatch), advance w and
  // keep the rest.  All 32 lanes must call it.
  __device__ __forceinline__ void flush(bool finish, int64_t& w, int64_t wend, int32_t* __restrict__ out_idx,
                                        float* __restrict__ out_d2) {
    const unsigned FULL = 0xffffffffu;
    const int cnt = ready(finish, w);
    unsigned m = __ballot_sync(FULL, cnt > 0);
    if (m == 0u) return;
    __syncwarp();
    const int lane = (int)(threadIdx.x & 31u);
    while (m != 0u) {
      const int j = __ffs(m) - 1;
      m &= m - 1u;
      const int cj = __shfl_sync(FULL, cnt, j);
      const int64_t wj = __shfl_sync(FULL, w, j);
      const int64_t ej = __shfl_sync(FULL, wend, j);
      if (lane < cj && wj + lane < ej) {
        out_idx[wj + lane] = wi[slot(j, lane)];
        if (out_d2) out_d2[wj + lane] = wd[slot(j, lane)];
      }
    }
    __syncwarp();
    if (cnt > 0) {
      for (int i = cnt; i < n; ++i) {
        wi[slot(lane, i - cnt)] = wi[slot(lane, i)];
        wd[slot(lane, i - cnt)] = wd[slot(lane, i)];
      }
      w += cnt;
      n -= cnt;
    }
    __syncwarp();
  }
};

// (d, j) < (hd, hj) lexicographically.
__device__ __forceinline__ bool lex_less(float d, int32_t j, float hd, int32_t hj) {
  return d < hd || (d == hd && j < hj);
}

// The k best (d2, index) pairs of one query: insert(d, j) keeps the pair if
// it beats the current k-th, worst_d() bounds pruning, write() stores the
// pairs in ascending order.  Unfilled entries are (+inf, INT32_MAX) and are
// written as index -1.  (A binary max-heap in shared memory measured slower
// for every k up to 32.)

// Sorted list in registers (small k).  A pair is one 64-bit key, the
// float32 bits of d2 above the index: for d2 >= +0 (squared distances) the
// bit patterns order like the values, so key order is the (d2, index) order
// and one integer compare replaces the lexicographic test; a NaN d2 sorts
// above +inf and is never kept.  Insertion shifts the larger keys up one slot
// from the top and stops at the new key's slot.

template <int K>
struct RegList {
  unsigned long long hk[K];
  // Resident 256-thread blocks per SM asked of the compiler (the register budget):
  // five for K <= 8 up to 3D (48 registers, no spill; 6D would spill), four up to
  // K = 16 (64 registers), two for K = 32.  10M mixture, 3D, measured with a
  // branch-free insertion: k=16 23.8 ms at 3 blocks, 22.4 at 4, spills at 5;
  // k=8 13.9 ms at 4, 13.0 at 5.
  template <int D>
  static constexpr int min_blocks() { return K <= 8 && D <= 3 ? 5 : K <= 16 ? 4 : 2; }
  static constexpr unsigned long long EMPTY = (0x7f800000ull << 32) | 0x7fffffffull;
  __device__ __forceinline__ static unsigned long long key(float d, int32_t j) {
    return ((unsigned long long)__float_as_uint(d) << 32) | (unsigned long long)(uint32_t)j;
  }
  __device__ __forceinline__ void init(char*) {
#pragma unroll
    for (int s = 0; s < K; ++s) hk[s] = EMPTY;
  }
  __device__ __forceinline__ void insert(float d, int32_t j) { insert_key(key(d, j)); }
  // The leaf children of one node (ok0 / ok1: child 0 / 1 is a leaf), smaller key
  // first: a warp whose lanes each hold one candidate, some in child 0 and some
  // in child 1, runs one insertion pass instead of two.  The list is the K
  // smallest keys seen, so the order of insertion does not change it.
  __device__ __forceinline__ void insert2(bool ok0, float d0, int32_t j0, bool ok1, float d1, int32_t j1) {
    const unsigned long long x0 = ok0 ? key(d0, j0) : EMPTY;
    const unsigned long long x1 = ok1 ? key(d1, j1) : EMPTY;
    const bool lt = x0 < x1;
    insert_key(lt ? x0 : x1);
    insert_key(lt ? x1 : x0);
  }
  // EMPTY is never inserted: it is not below the last entry.
  __device__ __forceinline__ void insert_key(unsigned long long x) {
    if (!(x < hk[K - 1])) return;
    // Top down, each slot takes its left neighbour while x is below that
    // neighbour; the first slot whose left neighbour is not above x takes x and
    // every slot under it keeps its key, so the chain stops there.  (A warp runs
    // only as deep as its deepest-landing lane: most keys that pass the test
    // land near the end; measured against the full branch-free chain on the 10M
    // mixture: k=16 22.1 -> 19.9 ms, k=32 56.9 -> 46.3, k=8 13.0 -> 12.7.)
    // (Written as a select per slot with a break: the list stays in registers.)
#pragma unroll
    for (int s = K - 1; s >= 0; --s) {
      if (s < K - 1 && !(x < hk[s])) break;
      const unsigned long long left = hk[s > 0 ? s - 1 : 0];
      hk[s] = s > 0 && x < left ? left : (x < hk[s] ? x : hk[s]);
    }
  }
  __device__ __forceinline__ float worst_d() const { return __uint_as_float((uint32_t)(hk[K - 1] >> 32)); }
  __device__ __forceinline__ void write(int32_t* oi, float* od, int kk) {
#pragma unroll
    for (int s = 0; s < K; ++s) {
      if (s < kk) {
        const int32_t j = (int32_t)(uint32_t)(hk[s] & 0xffffffffull);
        if (oi) oi[s] = j == INT32_MAX ? -1 : j;
        if (od) od[s] = __uint_as_float((uint32_t)(hk[s] >> 32));
      }
    }
  }
  static size_t smem_bytes(int) { return 0; }
};

// The k best keys of one query shared by the L lanes of a lane group (L
// consecutive lanes of a warp, L a power of two): the sorted list is split
// lane-major, group lane g holding ranks g*K/L .. (g+1)*K/L - 1, so each lane
// keeps K/L keys in registers.  Every lane of the group calls insert_key with
// the same key; a key below the list's last one takes its rank and every key
// at or above it moves up one rank, the key leaving a lane's top slot entering
// the next lane's bottom slot (one shuffle).  The result equals RegList<K>'s.
template <int K, int L>
struct GroupList {
  static_assert(L >= 2 && L <= 32 && (L & (L - 1)) == 0 && K % L == 0, "lane group shape");
  static constexpr int KL = K / L;
  static constexpr unsigned long long EMPTY = RegList<1>::EMPTY;
  unsigned long long hk[KL];
  __device__ __forceinline__ void init() {
#pragma unroll
    for (int s = 0; s < KL; ++s) hk[s] = EMPTY;
  }
  // The list's last key (held by the group's last lane).
  __device__ __forceinline__ unsigned long long last(unsigned gmask) const {
    return __shfl_sync(gmask, hk[KL - 1], L - 1, L);
  }
  __device__ __forceinline__ float worst_d(unsigned gmask) const {
    return __uint_as_float((uint32_t)(last(gmask) >> 32));
  }
  __device__ __forceinline__ void insert_key(unsigned long long x, unsigned gmask, int gl) {
    if (!(x < last(gmask))) return;  // the same decision in every lane of the group
    // the key below this lane's first slot: the previous lane's top key (none
    // below rank 0; 0 is not above any key, so rank 0 then takes x when x is
    // below it)
    unsigned long long left = __shfl_up_sync(gmask, hk[KL - 1], 1, L);
    if (gl == 0) left = 0ull;
#pragma unroll
    for (int s = KL - 1; s >= 0; --s) {
      const unsigned long long below = s > 0 ? hk[s - 1] : left;
      hk[s] = hk[s] < x ? hk[s] : (below < x ? x : below);
    }
  }
  // Columns gl*KL .. gl*KL + KL - 1 of the query's row (those below kk).
  __device__ __forceinline__ void write(int32_t* oi, float* od, int kk, int gl) const {
#pragma unroll
    for (int s = 0; s < KL; ++s) {
      const int c = gl * KL + s;
      if (c < kk) {
        const int32_t j = (int32_t)(uint32_t)(hk[s] & 0xffffffffull);
        if (oi) oi[c] = j == INT32_MAX ? -1 : j;
        if (od) od[c] = __uint_as_float((uint32_t)(hk[s] >> 32));
      }
    }
  }
};

// ------------------------------------------------------------------ rays

// Relative padding of every box for the ray slab test.  A Moller-Trumbore hit
// computed in float32 may lie a few ulps outside the exact triangle, so the
// traversal culls against boxes grown by PAD_REL * max(|lo|, |hi|, extent) per
// axis (rounded outward); the padding only costs traversal work.
constexpr float PAD_REL = 1.52587890625e-05f;  // 2^-16
// Far-distance widening of Ize (2013), "Robust BVH ray traversal": 1 + 2*gamma_3.
constexpr float FAR_WIDEN = 1.0f + 2.0f * (3.0f * 5.9604645e-08f) / (1.0f - 3.0f * 5.9604645e-08f);

struct Ray {
  float o[3], d[3], inv[3];
};

__device__ __forceinline__ bool slab(const Ray& r, const float* lo, const float* hi, float tlimit, float& tnear) {
  float tmin = 0.0f, tmax = tlimit;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float pad = __fmul_ru(PAD_REL, fmaxf(fmaxf(fabsf(lo[a]), fabsf(hi[a])), __fsub_ru(hi[a], lo[a])));
    const float L = __fsub_rd(lo[a], pad), H = __fadd_ru(hi[a], pad);
    const bool neg = (__float_as_uint(r.inv[a]) >> 31) != 0u;
    const float t0 = __fmul_rn(__fsub_rn(neg ? H : L, r.o[a]), r.inv[a]);
    const float t1 = __fmul_rn(__fsub_rn(neg ? L : H, r.o[a]), r.inv[a]);
    tmin = fmaxf(tmin, t0);  // NaN (0 * inf on a slab face) imposes no bound
    tmax = fminf(tmax, t1);
  }
  tnear = tmin;
  return tmin <= __fmul_ru(tmax, FAR_WIDEN);
}

// Moller & Trumbore (1997), two-sided, in the fixed operation order: e1 = v1-v0,
// e2 = v2-v0, p = d x e2, det = e1.p, miss if det == 0, inv = 1/det, s = o-v0,
// u = (s.p) inv, q = s x e1, v = (d.q) inv, t = (e2.q) inv; hit iff u >= 0,
// v >= 0, fl(u+v) <= 1, t >= 0.  Each cross component is fl(fl(a*b) - fl(c*d))
// and each dot product is summed x, y, z.
__device__ __forceinline__ bool moller_trumbore(const Ray& r, const float* v, float& t_out) {
  const float e1x = __fsub_rn(v[3], v[0]), e1y = __fsub_rn(v[4], v[1]), e1z = __fsub_rn(v[5], v[2]);
  const float e2x = __fsub_rn(v[6], v[0]), e2y = __fsub_rn(v[7], v[1]), e2z = __fsub_rn(v[8], v[2]);
  const float px = __fsub_rn(__fmul_rn(r.d[1], e2z), __fmul_rn(r.d[2], e2y));
  const float py = __fsub_rn(__fmul_rn(r.d[2], e2x), __fmul_rn(r.d[0], e2z));
  const float pz = __fsub_rn(__fmul_rn(r.d[0], e2y), __fmul_rn(r.d[1], e2x));
  const float det = __fadd_rn(__fadd_rn(__fmul_rn(e1x, px), __fmul_rn(e1y, py)), __fmul_rn(e1z, pz));
  if (det == 0.0f) return false;
  const float inv = __fdiv_rn(1.0f, det);
  const float sx = __fsub_rn(r.o[0], v[0]), sy = __fsub_rn(r.o[1], v[1]), sz = __fsub_rn(r.o[2], v[2]);
  const float u = __fmul_rn(__fadd_rn(__fadd_rn(__fmul_rn(sx, px), __fmul_rn(sy, py)), __fmul_rn(sz, pz)), inv);
  const float qx = __fsub_rn(__fmul_rn(sy, e1z), __fmul_rn(sz, e1y));
  const float qy = __fsub_rn(__fmul_rn(sz, e1x), __fmul_rn(sx, e1z));
  const float qz = __fsub_rn(__fmul_rn(sx, e1y), __fmul_rn(sy, e1x));
  const float vv = __fmul_rn(__fadd_rn(__fadd_rn(__fmul_rn(r.d[0], qx), __fmul_rn(r.d[1], qy)), __fmul_rn(r.d[2], qz)), inv);
  const float t = __fmul_rn(__fadd_rn(__fadd_rn(__fmul_rn(e2x, qx), __fmul_rn(e2y, qy)), __fmul_rn(e2z, qz)), inv);
  if (u >= 0.0f && vv >= 0.0f && __fadd_rn(u, vv) <= 1.0f && t >= 0.0f) {
    t_out = t;
    return true;
  }
  return false;
}

// intersect(ray) for the spatial traversal: child boxes by the padded slab
// test over t in [0, +inf), leaves by Moller-Trumbore (d receives t).
struct RayPred {
  static constexpr bool LEAF_TEST = true;
  static constexpr bool CONTAIN = false;
  __device__ __forceinline__ bool contains(const float*, const float*) const { return false; }
  Ray r;
  __device__ __forceinline__ bool test(const float* lo, const float* hi, float& d) const {
    float tn;
    d = 0.0f;
    return slab(r, lo, hi, F_INF, tn);
  }
  __device__ __forceinline__ void load(const float* __restrict__ qs, const float*, float, int64_t i) {
#pragma unroll
    for (int x = 0; x < 3; ++x) {
      r.o[x] = qs[i * 6 + x];
      r.d[x] = qs[i * 6 + 3 + x];
      r.inv[x] = __frcp_rn(r.d[x]);
    }
  }
  __device__ __forceinline__ bool leaf(const TriLeaf* __restrict__ leaves, int32_t pos, int32_t& orig,
                                       float& t) const {
    const TriLeaf L = load_node_global(leaves + pos);
    orig = L.orig;
    return moller_trumbore(r, L.v, t);
  }
};

// The test of a leaf child that needs its leaf record: the exact hit for
// rays, the triangle's own box under a quantized (inflated) child box.
template <class Pred>
__device__ __forceinline__ bool leaf_check(const Pred& p, const TriLeaf* __restrict__ leaves, int32_t pos,
                                           int32_t& orig, float& d) {
  if constexpr (Pred::LEAF_TEST) return p.leaf(leaves, pos, orig, d);
  else return leaf_exact(p, leaves, pos, orig, d);
}

// The k smallest (t, index) pairs in registers, ascending, compared as
// floats (so the t of a hit keeps its bits, -0.0 included); insertion as in
// RegList (shift from the top, stop at the new pair's slot).
template <int K>
struct LexList {
  float hd[K];
  int32_t hj[K];
  __device__ __forceinline__ void init() {
#pragma unroll
    for (int s = 0; s < K; ++s) {
      hd[s] = F_INF;
      hj[s] = INT32_MAX;
    }
  }
  __device__ __forceinline__ void insert(float d, int32_t j) {
    if (!lex_less(d, j, hd[K - 1], hj[K - 1])) return;
#pragma unroll
    for (int s = K - 1; s >= 0; --s) {
      const bool cs = lex_less(d, j, hd[s], hj[s]);
      if (s < K - 1 && !cs) break;
      const int l = s > 0 ? s - 1 : 0;
      const bool cp = s > 0 && lex_less(d, j, hd[l], hj[l]);
      const float nd = cp ? hd[l] : (cs ? d : hd[s]);
      const int32_t nj = cp ? hj[l] : (cs ? j : hj[s]);
      hd[s] = nd;
      hj[s] = nj;
    }
  }
};
}  // namespace
}  // namespace arbx
