// Batched traversal of the linear BVH.
//
// One thread owns one query at a time (queries are independent, so the
// per-query state needs no atomics: ArborX 2.0, section 2.2).  The grid is
// sized to the resident capacity of the GPU (each block stages the top tree
// levels into shared memory once) and warps pull chunks of consecutive query
// slots, in the given processing order (Morton order of the query centres when
// query sorting is on: section 2.6, sorting in search), from a work counter.
//
// Spatial predicates (section 2.1, intersects(Sphere) and intersects(Box))
// run a depth-first traversal with an explicit stack: both child boxes of a
// node are tested from the node record; matching leaves are emitted in
// left-to-right leaf order (a deferred right leaf waits on the stack while the
// left subtree is visited), so the fill pass writes each query's matches in a
// deterministic order independent of the launch shape.  The pure callbacks of
// section 2.2 are the count modes: COUNT, and COUNT_UP_TO, which stops the
// traversal once `limit` matches are found (FIRST_HIT is limit 1).
//
// Nearest predicates (section 2.1, nearest(point, k)) run a best-first depth
// first traversal: the nearer child first, the farther one pushed with its box
// distance; a subtree is pruned iff its box distance exceeds the current k-th
// distance (strict, so equal distances with lower indices are still found).
// The k best (d2, index) pairs live in registers, sorted.
//
// Ray nearest (section 2.5, nearest(ray, k)): slab tests on conservatively
// padded boxes, nearer child first, Moller-Trumbore on the leaves in a fixed
// operation order, the k smallest (t, index) kept.  Ray intersect and
// ordered_intersect run the spatial traversal with a ray predicate; the
// ordered form then sorts each query's hits by (t, index).
//
// DBSCAN (section 2.4) runs the spatial traversal per point with a union-find
// callback (FDBSCAN).
#include <mutex>
#include <type_traits>
#include <unordered_map>

#include "query.cuh"
#include "primitives.cuh"
#include "traverse.cuh"

namespace arbx {
namespace {




struct SpatialArgs {
  const float* qs;
  const float* radii;
  float r2u;
  const uint32_t* order;
  int64_t m;
  int32_t limit;
  int32_t* counts;
  const int64_t* offsets;
  int32_t* out_idx;
  float* out_d2;
  uint32_t* err;
  unsigned long long* stats;  // instrumented runs: [node fetches, leaf fetches, matches]
  unsigned long long* counter;  // warp work queue
  bool refill;                  // refill finished lanes at once (else when the whole warp is done)
  SingleStore single;           // MODE_SINGLE
  const uint32_t* chunk_perm = nullptr;  // order in which work chunks are handed out (null: in order)
  // COUNT / COUNT_UP_TO: a subtree whose box the predicate contains adds its
  // leaf count without being visited (off for trees of user boxes, which may be
  // inverted; see Pred::contains)
  bool contain = false;
  // instrumented sphere walks: per-query squared radii used as given (no
  // fl(r*r)), e.g. the final k-th distances of a nearest query
  const float* r2s = nullptr;
  int64_t nq = 0;  // queries in the data arrays when `order` lists a subset of them (0: m)
};

// Warp-collective flush of staged matches into single-pass storage.  Lanes
// with `want` append their staged run at logical position `pos` of query qi:
// positions below SINGLE_INLINE go to the query's inline slots, later ones to
// its chunks.  A run crosses at most one chunk boundary (a run holds at most
// 9 entries <=
// SINGLE_CHUNK), so a lane needs at most one new chunk per flush; the chunks
// of one flush are taken by one atomic per warp.
__device__ __forceinline__ void single_flush(FillBuffer& fb, bool want, int64_t qi, int64_t& pos, int& nch,
                                             int32_t& last_chunk, bool& ovf, const SingleStore& ss) {
  static_assert(9 <= SINGLE_CHUNK, "a staged run spans at most two chunks");
  const unsigned FULL = 0xffffffffu;
  const int lane = (int)(threadIdx.x & 31u);
  unsigned m = __ballot_sync(FULL, want);
  if (m == 0u) return;
  const int64_t cap = SINGLE_INLINE + (int64_t)nch * SINGLE_CHUNK;
  const bool need = want && !ovf && pos + fb.n > cap;
  const unsigned nm = __ballot_sync(FULL, need);
  const int32_t old_chunk = last_chunk;
  const int nch_before = nch;
  if (nm != 0u) {
    unsigned long long base = 0;
    const int leader = __ffs(nm) - 1;
    if (lane == leader) base = atomicAdd(ss.pool_counter, (unsigned long long)__popc(nm));
    base = __shfl_sync(FULL, base, leader);
    if (need) {
      const unsigned long long id = base + (unsigned long long)__popc(nm & ((1u << lane) - 1u));
      if ((int64_t)id < ss.pool_chunks) {
        if (nch == 0) ss.head[qi] = (int32_t)id;
        else ss.next[last_chunk] = (int32_t)id;
        last_chunk = (int32_t)id;
        ++nch;
      } else {
        ovf = true;
        const unsigned long long at = atomicAdd(ss.ovf_counter, 1ull);
        ss.ovf_list[at] = (int32_t)qi;
      }
    }
  }
  __syncwarp();
  unsigned wm = __ballot_sync(FULL, want && !ovf);
  while (wm != 0u) {
    const int j = __ffs(wm) - 1;
    wm &= wm - 1u;
    const int cnt = __shfl_sync(FULL, fb.n, j);
    const int64_t pj = __shfl_sync(FULL, pos, j);
    const int64_t qj = __shfl_sync(FULL, qi, j);
    const int32_t oc = __shfl_sync(FULL, old_chunk, j);
    const int32_t nc = __shfl_sync(FULL, last_chunk, j);
    const int nb = __shfl_sync(FULL, nch_before, j);
    if (lane < cnt) {
      const int64_t L = pj + lane;
      const int32_t vi = fb.wi[FillBuffer::slot(j, lane)];
      const float vd = fb.wd[FillBuffer::slot(j, lane)];
      int64_t at;
      int32_t* di;
      float* dd;
      if (L < SINGLE_INLINE) {
        at = qj * SINGLE_INLINE + L;
        di = ss.in_idx;
        dd = ss.in_d2;
      } else {
        const int64_t c = (L - SINGLE_INLINE) / SINGLE_CHUNK;
        const int32_t id = c == nb ? nc : oc;
        at = (int64_t)id * SINGLE_CHUNK + (L - SINGLE_INLINE) % SINGLE_CHUNK;
        di = ss.pool_idx;
        dd = ss.pool_d2;
      }
      di[at] = vi;
      if (dd) dd[at] = vd;
    }
  }
  __syncwarp();
  if (want) {
    pos += fb.n;
    fb.n = 0;
  }
}


// ------------------------------------------------------------------ spatial

// Cap on one query's traversal steps (a traversal takes fewer than 2n): a
// runaway query is stopped and reported instead of spinning.
__device__ __forceinline__ uint32_t step_limit(int64_t n) {
  const int64_t c = 4 * n + 1024;
  return c < (int64_t)0xffffffffu ? (uint32_t)c : 0xffffffffu;
}

template <int D, class NodeT, class Pred, int MODE, bool QUANT, bool STATS = false>
__global__ void __launch_bounds__(256) k_spatial(TreeView t, SpatialArgs a) {
  extern __shared__ float4 smem_top[];
  const NodeT* s_top = stage_top<NodeT>(t, smem_top);
  const NodeT* __restrict__ g = static_cast<const NodeT*>(t.nodes);
  // FILL: each lane's matches wait in shared memory (after the top levels)
  // and are written a sector at a time by the whole warp, so that one store
  // instruction covers consecutive addresses of one segment
  FillBuffer fb(reinterpret_cast<char*>(smem_top) + (size_t)t.ntop * sizeof(NodeT));
  constexpr bool EMIT = MODE == MODE_FILL || MODE == MODE_SINGLE;  // matches listed in leaf order
  int32_t st[STACK_DEPTH];
  float sd[EMIT ? STACK_DEPTH : 1];
  // counting modes: first sorted leaf position of the current node's range and
  // of each stacked (right) child's range (float32 nodes: quantized nodes do
  // not keep the range ends)
  constexpr bool RANGES = !EMIT && Pred::CONTAIN && !QUANT;
  int32_t sl[RANGES ? STACK_DEPTH : 1];
  int32_t first = 0;
  Frames<NodeT> fr;  // parent-relative nodes: the decoded boxes of the current and stacked nodes
  unsigned long long n_nodes = 0, n_leaves = 0, n_match = 0;
  WarpQueue wq;
  bool active = false, finished = false, faulted = false, ovf = false;
  int64_t slot = 0, qi = 0, w = 0, wend = 0;
  int nch = 0;
  int32_t last_chunk = -1;
  Pred p;
  int32_t cnt = 0, cur = 0;
  float cur_d2 = 0.0f;
  int sp = 0;
  uint32_t steps = 0;
  const uint32_t step_cap = step_limit(t.n);
  for (;;) {
    // new queries when the warp has none left (or, with lane refill, whenever
    // a lane is free); one vote per step while the warp is busy
    if (a.refill || __all_sync(0xffffffffu, !active)) {
    if (warp_refill(a.counter, a.m, wq, active, slot, a.chunk_perm)) {
      qi = query_at(a.order, slot, a.nq > 0 ? a.nq : a.m, a.err);
      p.load(a.qs, a.radii, a.r2u, qi);
      if constexpr (std::is_same<Pred, SpherePred<D>>::value) {
        if (STATS && a.r2s) p.r2 = a.r2s[qi];
      }
      cnt = 0;
      sp = 0;
      cur = t.root;
      fr.root(t);
      first = 0;
      steps = 0;
      faulted = false;
      if (MODE == MODE_FILL) {
        w = a.offsets[qi];
        wend = a.offsets[qi + 1];
      }
      if (MODE == MODE_SINGLE) {
        w = 0;
        nch = 0;
        last_chunk = -1;
        ovf = false;
      }
      active = true;
      if (MODE == MODE_COUNT_UP_TO && a.limit <= 0) {
        a.counts[qi] = 0;
        active = false;
      }
    }
    // done when no lane holds a query and the work queue is empty (a query
    // can finish at refill, e.g. count-up-to with limit 0)
    if (!__any_sync(0xffffffffu, active)) {
      if (wq.exhausted) break;
      continue;
    }
    }
    if (active && ++steps > step_cap) {
      // a traversal takes fewer than 2n steps: a runaway query is stopped and reported
      atomicOr(a.err, DEVERR_INTERNAL);
      active = false;
      finished = faulted = true;
    }
    if (active) {
    bool done = false;
    int32_t next = -1;
    if (EMIT && cur < 0) {
      // a right leaf deferred until its left sibling's subtree was listed
      fb.push(~cur, cur_d2);
    } else {
      const Kids<D> k = fr.open(fetch(cur, t, g, s_top));
      if (STATS) ++n_nodes;
      float d0 = 0.0f, d1 = 0.0f;
      int32_t o0 = k.orig[0], o1 = k.orig[1];
      bool h0 = p.test(k.lo[0], k.hi[0], d0);
      bool h1 = k.child[1] != NULL_CHILD && p.test(k.lo[1], k.hi[1], d1);
      constexpr bool LEAFREC = QUANT || Pred::LEAF_TEST;  // leaf children need their leaf record
      // box predicates on 16-bit nodes: a decoded leaf box (which holds the
      // triangle's exact box) inside the query box matches without the exact
      // test; only its input index is needed, and only when it is listed
      constexpr bool SETTLE = QUANT && !Pred::LEAF_TEST;
      bool s0 = false, s1 = false;
      if (SETTLE) {
        s0 = h0 && k.child[0] < 0 && p.contains(k.lo[0], k.hi[0]);
        s1 = h1 && k.child[1] < 0 && p.contains(k.lo[1], k.hi[1]);
        if (EMIT) {
          if (s0) o0 = __ldg(t.leaf_orig + leaf_index(~k.child[0], t));
          if (s1) o1 = __ldg(t.leaf_orig + leaf_index(~k.child[1], t));
        }
      }
      if (STATS && LEAFREC)
        n_leaves += (unsigned long long)((h0 && !s0 && k.child[0] < 0) + (h1 && !s1 && k.child[1] < 0));
      if (LEAFREC) {
        if (h0 && !s0 && k.child[0] < 0) h0 = leaf_check(p, t.leaves, leaf_index(~k.child[0], t), o0, d0);
        if (h1 && !s1 && k.child[1] < 0) h1 = leaf_check(p, t.leaves, leaf_index(~k.child[1], t), o1, d1);
      }
      const bool i0 = h0 && k.child[0] >= 0, i1 = h1 && k.child[1] >= 0;
      const bool l0 = h0 && k.child[0] < 0, l1 = h1 && k.child[1] < 0;
      if (EMIT) {
        if (l0) fb.push(o0, d0);
        if (l1 && !i0) fb.push(o1, d1);
        // push what must follow the left subtree: the right child (a leaf
        // entry ~index with its d2, or an internal node)
        if (i0 && (l1 || i1)) {
          if (sp < STACK_DEPTH) {
            st[sp] = l1 ? ~o1 : k.child[1];
            sd[sp] = d1;
            if (!l1) fr.push(sp, k, 1);
            ++sp;
          } else {
            atomicOr(a.err, DEVERR_STACK);
            done = faulted = true;
          }
        }
        next = i0 ? k.child[0] : (i1 ? k.child[1] : -1);
        if (next >= 0) fr.go(k, i0 ? 0 : 1);
      } else {
        cnt += (int32_t)l0 + (int32_t)l1;
        bool j0 = i0, j1 = i1;
        int32_t split = 0;
        if (RANGES) {
          // node ranges (Apetrei numbering): the node splits its range
          // [first, last] between sorted leaves `split` and split + 1; the left
          // child covers [first, split], the right child [split + 1, its range
          // end], and a left child's range end (or a left leaf's position) is
          // the split
          split = k.child[0] < 0 ? ~k.child[0] : k.orig[0];
          if (a.contain) {
            if (i0 && p.contains(k.lo[0], k.hi[0])) {
              cnt += split - first + 1;
              j0 = false;
            }
            if (i1 && p.contains(k.lo[1], k.hi[1])) {
              cnt += k.orig[1] - split;
              j1 = false;
            }
          }
        }
        if (MODE == MODE_COUNT_UP_TO && cnt >= a.limit) done = true;
        if (j0 && j1) {
          if (sp < STACK_DEPTH) {
            st[sp] = k.child[1];
            if (RANGES) sl[sp] = split + 1;
            fr.push(sp, k, 1);
            ++sp;
          } else {
            atomicOr(a.err, DEVERR_STACK);
            done = true;
          }
        }
        next = j0 ? k.child[0] : (j1 ? k.child[1] : -1);
        if (next >= 0) fr.go(k, j0 ? 0 : 1);
        if (RANGES && !j0 && j1) first = split + 1;
      }
    }
    if (!done) {
      if (next >= 0) {
        cur = next;
      } else if (sp > 0) {
        --sp;
        cur = st[sp];
        if (cur >= 0) fr.pop(sp);
        if (EMIT) cur_d2 = sd[sp];
        if (RANGES) first = sl[sp];
      } else {
        done = true;
      }
    }
    if (done) {
      if (EMIT) {
        finished = true;
      } else {
        a.counts[qi] = MODE == MODE_COUNT_UP_TO ? min(cnt, a.limit) : cnt;
      }
      if (STATS) n_match += (unsigned long long)cnt;
      active = false;
    }
    }  // active
    if (MODE == MODE_SINGLE) {
      single_flush(fb, fb.n >= FILL_SECTOR - 1 || (finished && fb.n > 0), qi, w, nch, last_chunk, ovf, a.single);
      if (finished) {
        a.counts[qi] = (int32_t)w;
        finished = false;
      }
    }
    if (MODE == MODE_FILL) {
      // warp-collective: write out full buffers and those of finished queries
      fb.flush(finished, w, wend, a.out_idx, a.out_d2);
      if (finished) {
        if (w != wend && !faulted) atomicOr(a.err, DEVERR_INTERNAL);
        finished = false;
      }
    }
  }
  if (STATS) add_stats(a.stats, n_nodes, n_leaves, n_match);
}

// ------------------------------------------------------------------ spatial, stackless

// Stackless variant of k_spatial (section 2.6: spatial search by a stackless
// algorithm).  In this node numbering the traversal needs no stored skip
// link: a subtree that covers sorted leaves [l, r] is followed, in depth-first
// left-to-right order, by the right child of internal node r (the node whose
// split lies between leaves r and r+1), and none follows when r = n - 1.  The
// build stores each internal child's range end r in the parent's orig slot
// of that child (a leaf child is its own range end), so a lane's whole state
// is one node index and one bit:
//   enter x:    test both child boxes of x; descend into a matching internal
//               left child, else emit a matching left leaf and go on with x's
//               right child from the same record;
//   right of y: re-fetch y, test only its right child box.
// After a right child (a matching leaf, a miss, or a subtree finished), the
// lane continues with "right of end(x)".  Matches come out in the same order
// as from k_spatial, so the results are the same bytes.
template <int D, class Pred, int MODE, bool STATS = false>
__global__ void __launch_bounds__(256) k_spatial_rope(TreeView t, SpatialArgs a) {
  extern __shared__ float4 smem_top[];
  const Node<D>* s_top = stage_top<Node<D>>(t, smem_top);
  const Node<D>* __restrict__ g = static_cast<const Node<D>*>(t.nodes);
  FillBuffer fb(reinterpret_cast<char*>(smem_top) + (size_t)t.ntop * sizeof(Node<D>));
  unsigned long long n_nodes = 0, n_match = 0;
  WarpQueue wq;
  bool active = false, right_only = false, finished = false;
  int64_t slot = 0, qi = 0, w = 0, wend = 0;
  Pred p;
  int32_t cnt = 0, cur = 0;
  int64_t steps = 0;
  const int32_t last = (int32_t)t.n - 1;
  for (;;) {
    if ((a.refill || __all_sync(0xffffffffu, !active)) && warp_refill(a.counter, a.m, wq, active, slot)) {
      qi = query_at(a.order, slot, a.nq > 0 ? a.nq : a.m, a.err);
      p.load(a.qs, a.radii, a.r2u, qi);
      cnt = 0;
      cur = t.root;
      right_only = false;
      steps = 0;
      if (MODE == MODE_FILL) {
        w = a.offsets[qi];
        wend = a.offsets[qi + 1];
      }
      active = true;
      if (MODE == MODE_COUNT_UP_TO && a.limit <= 0) {
        a.counts[qi] = 0;
        active = false;
      }
    }
    if (!__any_sync(0xffffffffu, active) && wq.exhausted) break;
    bool faulted = false;
    if (active && ++steps > 4 * t.n + 1024) {
      atomicOr(a.err, DEVERR_INTERNAL);
      active = false;
      finished = faulted = true;
    }
    if (active) {
      const Kids<D> k = unpack(fetch(cur, t, g, s_top));
      if (STATS) ++n_nodes;
      bool done = false;
      int32_t next = -1;  // >= 0: enter that node; < 0: continue with "right of end(cur)"
      float d0 = 0.0f, d1 = 0.0f;
      bool take_right = true;
      if (!right_only) {
        const bool h0 = p.test(k.lo[0], k.hi[0], d0);
        if (h0 && k.child[0] >= 0) {
          next = k.child[0];
          take_right = false;
        } else if (h0) {
          if (MODE == MODE_FILL) fb.push(k.orig[0], d0);
          ++cnt;
        }
      }
      if (take_right && k.child[1] != NULL_CHILD) {
        const bool h1 = p.test(k.lo[1], k.hi[1], d1);
        if (h1 && k.child[1] >= 0) {
          next = k.child[1];
        } else if (h1) {
          if (MODE == MODE_FILL) fb.push(k.orig[1], d1);
          ++cnt;
        }
      }
      if (MODE == MODE_COUNT_UP_TO && cnt >= a.limit) done = true;
      if (!done) {
        if (next >= 0) {
          cur = next;
          right_only = false;
        } else {
          // the right child of this node is finished: go on after its range
          const int32_t end = k.child[1] == NULL_CHILD ? last : (k.child[1] < 0 ? ~k.child[1] : k.orig[1]);
          if (end >= last) {
            done = true;
          } else {
            cur = end;
            right_only = true;
          }
        }
      }
      if (done) {
        if (MODE == MODE_FILL) {
          finished = true;
        } else {
          a.counts[qi] = MODE == MODE_COUNT_UP_TO ? min(cnt, a.limit) : cnt;
        }
        if (STATS) n_match += (unsigned long long)cnt;
        active = false;
      }
    }
    if (MODE == MODE_FILL) {
      fb.flush(finished, w, wend, a.out_idx, a.out_d2);
      if (finished) {
        if (w != wend && !faulted) atomicOr(a.err, DEVERR_INTERNAL);
        finished = false;
      }
    }
  }
  if (STATS) add_stats(a.stats, n_nodes, 0, n_match);
}

// ------------------------------------------------------------------ FDBSCAN

// DBSCAN (section 2.4) the FDBSCAN way: core points from a COUNT_UP_TO(minPts)
// pass, then one radius traversal per core point whose match callback merges
// the core neighbours that come before it in sorted leaf order (each core
// pair is merged once, from its later point) in a lock-free union-find, then
// one per non-core point that
// picks the smallest cluster label among its core neighbours.  The union
// hooks the larger root under the smaller (compare-and-swap), so every set's
// root is its smallest index and the labels do not depend on timing.

struct DbscanArgs {
  const float* qs;
  float r2;
  const uint32_t* order;
  int64_t m;
  const int32_t* counts;
  int32_t min_pts;
  int32_t* parent;
  int32_t* labels;
  uint32_t* err;
  unsigned long long* counter;
  bool refill;
  int64_t nq = 0;  // queries in the data arrays when `order` lists a subset of them (0: m)
  // union phase: sorted leaf position of each point (the queries are the
  // tree's own points); null: no pruning by position
  const int32_t* leaf_pos = nullptr;
};

// Every parent pointer points to a smaller index (roots point to
// themselves), so any ancestor of x is a valid parent for x: path halving may
// store the grandparent with a plain write even when another thread halves
// the same pointer at the same time.
__device__ __forceinline__ int32_t uf_find(int32_t* parent, int32_t x, int64_t limit, uint32_t* err) {
  for (int64_t it = 0; it < limit; ++it) {
    const int32_t p = *(volatile int32_t*)(parent + x);
    if (p == x) return x;
    const int32_t gp = *(volatile int32_t*)(parent + p);
    if (gp != p) *(volatile int32_t*)(parent + x) = gp;  // path halving
    x = gp;
  }
  atomicOr(err, DEVERR_INTERNAL);
  return x;
}

// Merge the sets of a and b; returns the root of the merged set as seen by
// this thread (an ancestor of both, possibly not the final root).
__device__ __forceinline__ int32_t uf_union(int32_t* parent, int32_t a, int32_t b, int64_t limit, uint32_t* err) {
  for (int64_t it = 0; it < limit; ++it) {
    a = uf_find(parent, a, limit, err);
    b = uf_find(parent, b, limit, err);
    if (a == b) return a;
    if (a < b) {
      const int32_t t = a;
      a = b;
      b = t;
    }
    // hook the larger root a under b; a failure means a got a parent meanwhile
    if (atomicCAS(parent + a, a, b) == a) return b;
  }
  atomicOr(err, DEVERR_INTERNAL);
  return b;
}

// PHASE 0: union over core points; PHASE 1: labels of non-core points (the
// core points' labels are written in between).
template <int D, int PHASE>
__global__ void __launch_bounds__(256) k_dbscan(TreeView t, DbscanArgs a) {
  extern __shared__ float4 smem_top[];
  const Node<D>* s_top = stage_top<Node<D>>(t, smem_top);
  const Node<D>* __restrict__ g = static_cast<const Node<D>*>(t.nodes);
  int32_t st[STACK_DEPTH];
  WarpQueue wq;
  bool active = false;
  int64_t slot = 0, qi = 0;
  SpherePred<D> p;
  int32_t cur = 0, best = -1;
  int32_t root_q = 0;  // union phase: an ancestor of the query's set (starts at the query)
  int32_t posq = INT32_MAX;  // union phase: the query's own sorted leaf position
  int sp = 0;
  int64_t steps = 0;
  const int64_t limit = t.n + 64;
  for (;;) {
    if ((a.refill || __all_sync(0xffffffffu, !active)) && warp_refill(a.counter, a.m, wq, active, slot)) {
      qi = query_at(a.order, slot, a.nq > 0 ? a.nq : a.m, a.err);
      const bool core = a.counts[qi] >= a.min_pts;
      active = PHASE == 0 ? core : !core;
      if (active) {
        p.load(a.qs, nullptr, a.r2, qi);
        sp = 0;
        cur = t.root;
        steps = 0;
        best = -1;
        root_q = (int32_t)qi;
        if (PHASE == 0 && a.leaf_pos) posq = a.leaf_pos[qi];
      }
    }
    if (!__any_sync(0xffffffffu, active) && wq.exhausted) break;
    if (active && ++steps > 4 * t.n + 1024) {
      atomicOr(a.err, DEVERR_INTERNAL);
      active = false;
    }
    if (active) {
      const Kids<D> k = unpack(fetch(cur, t, g, s_top));
      float d0 = 0.0f, d1 = 0.0f;
      const bool h0 = p.test(k.lo[0], k.hi[0], d0);
      bool h1 = k.child[1] != NULL_CHILD && p.test(k.lo[1], k.hi[1], d1);
      // Union phase: every core-core pair within eps needs one union, made
      // here by the point with the larger sorted leaf position, so a query
      // only looks at leaves before its own position.  A right child covers
      // positions from split + 1 on (split: the left child's range end, or the
      // left leaf's position) and is skipped when that is not before the
      // query's; a left child starts where its parent does, which is before.
      if (PHASE == 0 && a.leaf_pos) {
        const int32_t split = k.child[0] < 0 ? ~k.child[0] : k.orig[0];
        if (split >= posq - 1) h1 = false;
      }
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        if ((c == 0 ? h0 : h1) && k.child[c] < 0) {
          const int32_t j = k.orig[c];
          if (a.counts[j] >= a.min_pts) {
            if (PHASE == 0) {
              // most core neighbours already hang directly under the query's
              // root: one load decides, the union runs only otherwise
              const bool before = a.leaf_pos ? ~k.child[c] < posq : j < qi;
              if (before && *(volatile int32_t*)(a.parent + j) != root_q)
                root_q = uf_union(a.parent, root_q, j, limit, a.err);
            } else {
              const int32_t r = a.labels[j];  // core labels are final (previous launch)
              if (best < 0 || r < best) best = r;
            }
          }
        }
      }
      const bool i0 = h0 && k.child[0] >= 0, i1 = h1 && k.child[1] >= 0;
      bool done = false;
      if (i0 && i1) {
        if (sp < STACK_DEPTH) {
          st[sp++] = k.child[1];
        } else {
          atomicOr(a.err, DEVERR_STACK);
          done = true;
        }
      }
      if (!done) {
        if (i0 || i1) cur = i0 ? k.child[0] : k.child[1];
        else if (sp > 0) cur = st[--sp];
        else done = true;
      }
      if (done) {
        if (PHASE == 1) a.labels[qi] = best;
        active = false;
      }
    }
  }
}

// Sorted leaf position of every point of a point tree (the inverse of the
// build's sort permutation), read off the leaf children of the internal nodes.
template <int D>
__global__ void k_leaf_positions(const Node<D>* __restrict__ nodes, int64_t nnodes, int64_t n,
                                 int32_t* __restrict__ pos, uint32_t* err) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= nnodes) return;
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    const int32_t ch = nodes[g].child[c];
    if (ch < 0 && ch != NULL_CHILD) {
      const int32_t j = nodes[g].orig[c];
      if (j >= 0 && j < n) pos[j] = ~ch;
      else atomicOr(err, DEVERR_INTERNAL);
    }
  }
}

// Split the processing order into its core and non-core points, each part in
// the order's sequence (stable), so each phase's warps hold only queries
// that traverse.
__global__ void k_core_flags(const uint32_t* __restrict__ order, const int32_t* __restrict__ counts, int32_t min_pts,
                             int64_t n, int32_t* __restrict__ flags, uint32_t* err) {
  const int64_t slot = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (slot >= n) return;
  const int64_t q = query_at(order, slot, n, err);
  flags[slot] = counts[q] >= min_pts ? 1 : 0;
}

__global__ void k_split_order(const uint32_t* __restrict__ order, const int32_t* __restrict__ flags,
                              const int64_t* __restrict__ pos, int64_t n, int64_t ncore, uint32_t* __restrict__ out,
                              uint32_t* err) {
  const int64_t slot = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (slot >= n) return;
  const uint32_t q = (uint32_t)query_at(order, slot, n, err);
  out[flags[slot] ? pos[slot] : ncore + (slot - pos[slot])] = q;
}

__global__ void k_uf_init(int32_t* parent, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) parent[i] = (int32_t)i;
}

// Core points: the label is the root (the smallest index of the set); the
// clusters are counted at their roots.
__global__ void k_core_labels(int32_t* parent, const int32_t* __restrict__ counts, int32_t min_pts, int64_t n,
                              int32_t* __restrict__ labels, unsigned long long* clusters, uint32_t* err) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long c = 0;
  if (i < n && counts[i] >= min_pts) {
    const int32_t r = uf_find(parent, (int32_t)i, n + 64, err);
    labels[i] = r;
    c = r == i;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(clusters, c);
}

// ------------------------------------------------------------------ nearest

struct KnnArgs {
  const float* qs;
  const uint32_t* order;
  int64_t m;
  int kk;
  int32_t* out_idx;
  float* out_d2;
  uint32_t* err;
  unsigned long long* stats;
  unsigned long long* counter;
  bool refill;
  int64_t nq = 0;  // queries in the data arrays when `order` lists a subset of them (0: m)
};


// An upper bound on the k-th smallest float32 d2 of query q, from a query p
// whose k-th smallest d2 is pdk (p's k nearest points lie within
// sqrt(pdk) + |q - p| of q, triangle inequality).  Every term is rounded up
// and widened by 2^-18 relative (the float32 d2 of a pair is within 9 ulps of
// its exact value) plus 1e-37 absolute (underflow), so q's k-th float32 d2 is
// never above it; +inf when pdk is +inf (p found fewer than k points) or a
// coordinate is not finite.
template <int D>
__device__ __forceinline__ float knn_carry_bound(const float* p, float pdk, const float* q) {
  float s = 0.0f;
#pragma unroll
  for (int a = 0; a < D; ++a) {
    const float d = __fsub_ru(fmaxf(q[a], p[a]), fminf(q[a], p[a]));
    s = __fadd_ru(s, __fmul_ru(d, d));
  }
  const float r = __fadd_ru(__fsqrt_ru(__fadd_ru(__fmul_ru(pdk, 1.000004f), 1e-37f)), __fsqrt_ru(s));
  const float b = __fadd_ru(__fmul_ru(__fmul_ru(r, r), 1.000004f), 1e-37f);
  return b == b ? b : F_INF;  // NaN (a non-finite coordinate): no bound
}

// RUN > 1: a warp takes 32 * RUN consecutive slots of the processing order and
// answers them in RUN rounds of 32 adjacent slots (lane i: slots i, 32 + i,
// 64 + i, ...), so each of a lane's queries after the first starts with an
// upper bound on its k-th distance carried from the lane's previous query, 32
// positions earlier in the order (knn_carry_bound; any k real points bound it,
// so a query that stopped early still gives a valid one); nodes beyond the
// bound are pruned from the first step, before the list is full.  The list and
// the inclusive pruning rule are unchanged, so every point within the final
// k-th distance is still met: the same bytes.  (Runs of adjacent slots per
// lane -- a bound from the very next query, but lanes spread over 32 * RUN
// queries -- measured slower: k=16 17.4 vs 17.0 ms at RUN = 4 on the 10M
// mixture; runs of 16 or 32 rounds lose to the coarser work hand-out.)
template <int D, class Heap, bool STATS = false, int RUN = 1>
__global__ void __launch_bounds__(256, Heap::template min_blocks<D>()) k_knn(TreeView t, KnnArgs a) {
  extern __shared__ float4 smem_top[];
  const Node<D>* s_top = stage_top<Node<D>>(t, smem_top);
  char* heap_base = reinterpret_cast<char*>(smem_top) + (size_t)t.ntop * sizeof(Node<D>);
  const Node<D>* __restrict__ g = static_cast<const Node<D>*>(t.nodes);
  NNStack<STACK_DEPTH> st;  // (node code, bits of its box distance)
  unsigned long long n_nodes = 0;
  WarpQueue wq;
  bool active = false;
  int64_t slot = 0, qi = 0;
  float q[D];
  Heap h;
  uint32_t steps = 0;
  const uint32_t step_cap = step_limit(t.n);
  int32_t cur = 0;
  float bound = F_INF;        // carried upper bound on this query's k-th d2 (RUN > 1)
  float pq[RUN > 1 ? D : 1];  // the lane's previous query and its k-th d2
  float pdk = F_INF;
  LaneRun<RUN> run;
  for (;;) {
    if constexpr (RUN > 1) {
      // every lane's next query of its run, when the whole warp is done
      if (__all_sync(0xffffffffu, !active)) {
        bool fresh = false;
        if (!run.next(a.counter, a.m, (int)(threadIdx.x & 31u), slot, fresh)) break;
        if (fresh) pdk = F_INF;
        if (slot < a.m) {
          qi = query_at(a.order, slot, a.nq > 0 ? a.nq : a.m, a.err);
#pragma unroll
          for (int x = 0; x < D; ++x) q[x] = a.qs[qi * D + x];
          bound = pdk < F_INF ? knn_carry_bound<D>(pq, pdk, q) : F_INF;
          h.init(heap_base);
          st.clear();
          cur = t.root;
          steps = 0;
          active = true;
        }
        if (!__any_sync(0xffffffffu, active)) continue;
      }
    } else {
      // new queries when the warp has none left (or, with lane refill, whenever
      // a lane is free); one vote per step while the warp is busy
      if (a.refill || __all_sync(0xffffffffu, !active)) {
        if (warp_refill(a.counter, a.m, wq, active, slot)) {
          qi = query_at(a.order, slot, a.nq > 0 ? a.nq : a.m, a.err);
#pragma unroll
          for (int x = 0; x < D; ++x) q[x] = a.qs[qi * D + x];
          h.init(heap_base);
          st.clear();
          cur = t.root;
          steps = 0;
          active = true;
        }
        if (!__any_sync(0xffffffffu, active)) {
          if (wq.exhausted) break;
          continue;
        }
      }
    }
    if (active && ++steps > step_cap) {
      // a traversal takes fewer than 2n steps: a runaway query is stopped and reported
      atomicOr(a.err, DEVERR_INTERNAL);
      active = false;
    }
    if (active) {
      const Kids<D> k = unpack(fetch<false>(cur, t, g, s_top));
      if (STATS) ++n_nodes;
      const bool v1 = k.child[1] != NULL_CHILD;
      const float d0 = box_d2<D>(q, k.lo[0], k.hi[0]);
      const float d1 = v1 ? box_d2<D>(q, k.lo[1], k.hi[1]) : F_INF;
      h.insert2(k.child[0] < 0, d0, k.orig[0], v1 && k.child[1] < 0, d1, k.orig[1]);
      const float worst = RUN > 1 ? fminf(h.worst_d(), bound) : h.worst_d();
      const bool g0 = k.child[0] >= 0 && d0 <= worst;
      const bool g1 = v1 && k.child[1] >= 0 && d1 <= worst;
      bool done = false;
      int32_t next = -1;
      if (g0 && g1) {
        // nearer child first; the farther one waits with its box distance
        const bool first1 = d1 < d0;
        next = first1 ? k.child[1] : k.child[0];
        if (!st.full()) {
          st.push(nn_entry(first1 ? k.child[0] : k.child[1], first1 ? d0 : d1));
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
        // pop, discarding entries that can no longer hold a better pair
        const float worst_now = RUN > 1 ? fminf(h.worst_d(), bound) : h.worst_d();
        while (st.sp > 0) {
          const unsigned long long e = st.pop();
          if (nn_dist(e) <= worst_now) {
            next = nn_code(e);
            break;
          }
        }
        if (next < 0) done = true;
      }
      cur = next;
      if (done) {
        int32_t* oi = a.out_idx ? a.out_idx + qi * a.kk : nullptr;
        float* od = a.out_d2 ? a.out_d2 + qi * a.kk : nullptr;
        h.write(oi, od, a.kk);
        active = false;
        if constexpr (RUN > 1) {
#pragma unroll
          for (int x = 0; x < D; ++x) pq[x] = q[x];
          pdk = h.worst_d();
        }
      }
    }
  }
  if (STATS) add_stats(a.stats, n_nodes, 0ull, 0ull);
}

// nearest(point, k) with one traversal per warp ("packet"): the 32 lanes hold
// 32 neighbouring queries of the processing order and walk the union of the
// nodes they need together, one node per step for the whole warp, so every
// node record is one broadcast load.  Each lane tests the node's children
// against its own query and keeps its own k-best list.  A child is taken when
// some lane finds its box within that lane's current k-th distance -- so every
// lane still meets every node it needs, and the lists are exact -- the child
// more of those lanes find nearer first; the other is stacked with each
// lane's own box distance (a per-lane stack indexed by the warp's common depth,
// so its accesses are coalesced) and skipped at pop when no lane needs it any
// more.
template <int D, int K, bool STATS = false>
__global__ void __launch_bounds__(256, RegList<K>::template min_blocks<D>()) k_knn_packet(TreeView t, KnnArgs a) {
  using Heap = RegList<K>;
  const Node<D>* __restrict__ g = static_cast<const Node<D>*>(t.nodes);
  const unsigned FULL = 0xffffffffu;
  const int lane = (int)(threadIdx.x & 31u);
  int32_t sc[STACK_DEPTH];  // stacked node codes (the same in every lane)
  float sd[STACK_DEPTH];    // this lane's box distance of each stacked node
  unsigned long long n_nodes = 0;
  Heap h;
  float q[D];
  for (;;) {
    unsigned long long c = 0;
    if (lane == 0) c = atomicAdd(a.counter, 32ull);
    c = __shfl_sync(FULL, c, 0);
    if ((int64_t)c >= a.m) break;
    const int64_t slot = (int64_t)c + lane;
    const bool active = slot < a.m;
    const int64_t qi = active ? (query_at(a.order, slot, a.nq > 0 ? a.nq : a.m, a.err)) : 0;
#pragma unroll
    for (int x = 0; x < D; ++x) q[x] = active ? a.qs[qi * D + x] : __int_as_float(0x7fc00000);  // NaN: needs nothing
    h.init(nullptr);
    int sp = 0;
    int32_t cur = t.root;
    int64_t steps = 0;
    for (;;) {  // warp-uniform
      if (++steps > 4 * t.n + 1024) {
        if (lane == 0) atomicOr(a.err, DEVERR_INTERNAL);
        break;
      }
      const Kids<D> k = unpack(load_node_global(g + node_index(cur, t)));
      if (STATS && lane == 0) ++n_nodes;
      const bool v1 = k.child[1] != NULL_CHILD;
      const float d0 = box_d2<D>(q, k.lo[0], k.hi[0]);
      const float d1 = v1 ? box_d2<D>(q, k.lo[1], k.hi[1]) : F_INF;
      h.insert2(k.child[0] < 0, d0, k.orig[0], v1 && k.child[1] < 0, d1, k.orig[1]);
      const float worst = h.worst_d();
      const bool n0 = k.child[0] >= 0 && d0 <= worst;
      const bool n1 = v1 && k.child[1] >= 0 && d1 <= worst;
      const unsigned b0 = __ballot_sync(FULL, n0), b1 = __ballot_sync(FULL, n1);
      int32_t next = -1;
      bool fault = false;
      if (b0 != 0u && b1 != 0u) {
        const bool pref1 = n1 && (!n0 || d1 < d0);  // this lane would take child 1 first
        const int votes1 = __popc(__ballot_sync(FULL, (n0 || n1) && pref1));
        const int votes0 = __popc(__ballot_sync(FULL, (n0 || n1) && !pref1));
        const bool first1 = votes1 > votes0;
        next = first1 ? k.child[1] : k.child[0];
        if (sp < STACK_DEPTH) {
          sc[sp] = first1 ? k.child[0] : k.child[1];
          sd[sp] = first1 ? d0 : d1;
          ++sp;
        } else {
          if (lane == 0) atomicOr(a.err, DEVERR_STACK);
          fault = true;
        }
      } else if (b0 != 0u) {
        next = k.child[0];
      } else if (b1 != 0u) {
        next = k.child[1];
      }
      if (fault) break;
      if (next < 0) {
        while (sp > 0) {
          --sp;
          if (__any_sync(FULL, sd[sp] <= worst)) {
            next = sc[sp];
            break;
          }
        }
      }
      if (next < 0) break;
      cur = next;
    }
    if (active) h.write(a.out_idx ? a.out_idx + qi * a.kk : nullptr, a.out_d2 ? a.out_d2 + qi * a.kk : nullptr, a.kk);
  }
  if (STATS) add_stats(a.stats, n_nodes, 0ull, 0ull);
}

// Sort four (distance, code) pairs ascending by distance (five compare-exchanges).
__device__ __forceinline__ void sort4(float (&d)[4], int32_t (&c)[4]) {
  auto cx = [&](int i, int j) {
    const bool sw = d[j] < d[i];
    const float di = d[i], dj = d[j];
    const int32_t ci = c[i], cj = c[j];
    d[i] = sw ? dj : di;
    d[j] = sw ? di : dj;
    c[i] = sw ? cj : ci;
    c[j] = sw ? ci : cj;
  };
  cx(0, 1);
  cx(2, 3);
  cx(0, 2);
  cx(1, 3);
  cx(1, 2);
}

// nearest(point, k) over the four-wide records: each step opens one record
// (two binary levels), puts its leaf entries into the k-best list (smallest key
// first: once a key is refused, the larger ones are too), and continues with
// the nearest internal entry within the current k-th distance, the others
// pushed farthest first.  Same results as k_knn: the list is the k smallest
// (d2, index) keys of every leaf tested, and a pruned entry's box distance
// bounds every leaf below it (pruning is strict, as in k_knn).
template <int D, int K, bool STATS = false, int RUN = 1>
__global__ void __launch_bounds__(256, RegList<K>::template min_blocks<D>()) k_knn_wide(TreeView t, KnnArgs a) {
  using Heap = RegList<K>;
  const Wide<D>* __restrict__ w = static_cast<const Wide<D>*>(t.wide);
  NNStack<WIDE_STACK_DEPTH> st;  // (record, bits of its box distance)
  unsigned long long n_nodes = 0;
  WarpQueue wq;
  bool active = false;
  int64_t slot = 0, qi = 0;
  float q[D];
  Heap h;
  uint32_t steps = 0;
  const uint32_t step_cap = step_limit(t.n);
  int32_t cur = 0;
  float bound = F_INF;        // lane runs: carried upper bound on the k-th d2 (see k_knn)
  float pq[RUN > 1 ? D : 1];
  float pdk = F_INF;
  LaneRun<RUN> run;
  for (;;) {
    if constexpr (RUN > 1) {
      if (__all_sync(0xffffffffu, !active)) {
        bool fresh = false;
        if (!run.next(a.counter, a.m, (int)(threadIdx.x & 31u), slot, fresh)) break;
        if (fresh) pdk = F_INF;
        if (slot < a.m) {
          qi = query_at(a.order, slot, a.nq > 0 ? a.nq : a.m, a.err);
#pragma unroll
          for (int x = 0; x < D; ++x) q[x] = a.qs[qi * D + x];
          bound = pdk < F_INF ? knn_carry_bound<D>(pq, pdk, q) : F_INF;
          h.init(nullptr);
          st.clear();
          cur = t.root;
          steps = 0;
          active = true;
        }
        if (!__any_sync(0xffffffffu, active)) continue;
      }
    } else {
      if (a.refill || __all_sync(0xffffffffu, !active)) {
        if (warp_refill(a.counter, a.m, wq, active, slot)) {
          qi = query_at(a.order, slot, a.nq > 0 ? a.nq : a.m, a.err);
#pragma unroll
          for (int x = 0; x < D; ++x) q[x] = a.qs[qi * D + x];
          h.init(nullptr);
          st.clear();
          cur = t.root;
          steps = 0;
          active = true;
        }
        if (!__any_sync(0xffffffffu, active)) {
          if (wq.exhausted) break;
          continue;
        }
      }
    }
    if (active && ++steps > step_cap) {
      atomicOr(a.err, DEVERR_INTERNAL);
      active = false;
    }
    if (active) {
      const Wide<D> nd = load_node_global(w + node_index(cur, t));
      if (STATS) ++n_nodes;
      float d[4];
      unsigned long long x[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        d[c] = box_d2<D>(q, nd.lo[c], nd.hi[c]);
        const bool leaf = nd.code[c] < 0 && nd.code[c] != NULL_CHILD;
        x[c] = leaf ? Heap::key(d[c], nd.aux[c]) : Heap::EMPTY;
      }
      // leaf keys smallest first
      auto kx = [&](int i, int j) {
        const unsigned long long xi = x[i], xj = x[j];
        x[i] = xj < xi ? xj : xi;
        x[j] = xj < xi ? xi : xj;
      };
      kx(0, 1);
      kx(2, 3);
      kx(0, 2);
      kx(1, 3);
      kx(1, 2);
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        if (!(x[c] < h.hk[K - 1])) break;
        h.insert_key(x[c]);
      }
      const float worst = RUN > 1 ? fminf(h.worst_d(), bound) : h.worst_d();
      float dd[4];
      int32_t cc[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const bool go = nd.code[c] >= 0 && d[c] <= worst;
        dd[c] = go ? d[c] : F_INF;
        cc[c] = go ? nd.code[c] : -1;
      }
      sort4(dd, cc);
      bool done = false;
      int32_t next = cc[0];
#pragma unroll
      for (int c = 3; c >= 1; --c) {
        if (cc[c] >= 0) {
          if (next < 0) {
            next = cc[c];  // a passing entry sorted behind a refused one (box distance +inf)
          } else if (!st.full()) {
            st.push(nn_entry(cc[c], dd[c]));
          } else {
            atomicOr(a.err, DEVERR_STACK);
            done = true;
          }
        }
      }
      if (!done && next < 0) {
        const float worst_now = RUN > 1 ? fminf(h.worst_d(), bound) : h.worst_d();
        while (st.sp > 0) {
          const unsigned long long e = st.pop();
          if (nn_dist(e) <= worst_now) {
            next = nn_code(e);
            break;
          }
        }
        if (next < 0) done = true;
      }
      cur = next;
      if (done) {
        int32_t* oi = a.out_idx ? a.out_idx + qi * a.kk : nullptr;
        float* od = a.out_d2 ? a.out_d2 + qi * a.kk : nullptr;
        h.write(oi, od, a.kk);
        active = false;
        if constexpr (RUN > 1) {
#pragma unroll
          for (int x = 0; x < D; ++x) pq[x] = q[x];
          pdk = h.worst_d();
        }
      }
    }
  }
  if (STATS) add_stats(a.stats, n_nodes, 0ull, 0ull);
}

// The counting traversal (COUNT, COUNT_UP_TO; instrumented walks) over the
// four-wide records: each step opens one record, counts its leaf entries that
// pass, adds the leaf count of an internal entry whose box the predicate
// contains (when a.contain), and walks the other passing internal entries.
// The entries' ranges are consecutive from the record's range start, which
// is carried with each stacked entry, so a contained entry's leaf count is
// (its range end) - (its range start) + 1.
template <int D, class Pred, int MODE, bool STATS = false>
__global__ void __launch_bounds__(256) k_count_wide(TreeView t, SpatialArgs a) {
  const Wide<D>* __restrict__ w = static_cast<const Wide<D>*>(t.wide);
  int2 st[WIDE_STACK_DEPTH];  // (record, first sorted leaf of its range)
  unsigned long long n_nodes = 0, n_match = 0;
  WarpQueue wq;
  bool active = false;
  int64_t slot = 0, qi = 0;
  Pred p;
  int32_t cnt = 0, cur = 0, first = 0;
  int sp = 0;
  int64_t steps = 0;
  for (;;) {
    if ((a.refill || __all_sync(0xffffffffu, !active)) &&
        warp_refill(a.counter, a.m, wq, active, slot, a.chunk_perm)) {
      qi = query_at(a.order, slot, a.nq > 0 ? a.nq : a.m, a.err);
      p.load(a.qs, a.radii, a.r2u, qi);
      if constexpr (std::is_same<Pred, SpherePred<D>>::value) {
        if (STATS && a.r2s) p.r2 = a.r2s[qi];
      }
      cnt = 0;
      sp = 0;
      cur = t.root;
      first = 0;
      steps = 0;
      active = true;
      if (MODE == MODE_COUNT_UP_TO && a.limit <= 0) {
        a.counts[qi] = 0;
        active = false;
      }
    }
    if (!__any_sync(0xffffffffu, active) && wq.exhausted) break;
    if (active && ++steps > 4 * t.n + 1024) {
      atomicOr(a.err, DEVERR_INTERNAL);
      active = false;
    }
    if (active) {
      const Wide<D> nd = load_node_global(w + node_index(cur, t));
      if (STATS) ++n_nodes;
      bool done = false;
      int32_t next = -1, next_first = 0;
      int32_t start = first;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int32_t code = nd.code[c];
        if (code != NULL_CHILD) {
          const int32_t end = code < 0 ? ~code : nd.aux[c];
          float dd;
          if (p.test(nd.lo[c], nd.hi[c], dd)) {
            if (code < 0) {
              ++cnt;
            } else if (a.contain && p.contains(nd.lo[c], nd.hi[c])) {
              cnt += end - start + 1;
            } else if (next < 0) {
              next = code;
              next_first = start;
            } else if (sp < WIDE_STACK_DEPTH) {
              st[sp] = make_int2(code, start);
              ++sp;
            } else {
              atomicOr(a.err, DEVERR_STACK);
              done = true;
            }
          }
          start = end + 1;
        }
      }
      if (MODE == MODE_COUNT_UP_TO && cnt >= a.limit) done = true;
      if (!done) {
        if (next >= 0) {
          cur = next;
          first = next_first;
        } else if (sp > 0) {
          const int2 e = st[--sp];
          cur = e.x;
          first = e.y;
        } else {
          done = true;
        }
      }
      if (done) {
        a.counts[qi] = MODE == MODE_COUNT_UP_TO ? min(cnt, a.limit) : cnt;
        if (STATS) n_match += (unsigned long long)cnt;
        active = false;
      }
    }
  }
  if (STATS) add_stats(a.stats, n_nodes, 0ull, n_match);
}

// Resident 256-thread blocks per SM asked of the compiler for a lane-group
// kernel holding KL keys per lane (the same register budget as RegList<KL>).
template <int D, int KL>
constexpr int group_min_blocks() { return KL <= 8 && D <= 3 ? 5 : KL <= 16 ? 4 : 2; }

// nearest(point, k) with L lanes per query (L = 2 .. 32): the lanes of a group
// walk one query's traversal together -- the same node, the same decisions,
// the same best-first order as k_knn -- and share its sorted k-best list
// (GroupList: K/L keys per lane), so a lane holds fewer registers and a warp
// holds 32/L queries.  The group's stack is spread over its lanes too (entry
// e in lane e mod L), pushed by one lane and popped by one lane with a
// shuffle.  This also serves lists longer than a lane can hold (K up to 256).
template <int D, int K, int L, bool STATS = false, int RUN = 1>
__global__ void __launch_bounds__(256, group_min_blocks<D, K / L>()) k_knn_group(TreeView t, KnnArgs a) {
  constexpr int SD = STACK_DEPTH / L;  // this lane's share of the group's stack
  extern __shared__ float4 smem_top[];
  const Node<D>* s_top = stage_top<Node<D>>(t, smem_top);
  const Node<D>* __restrict__ g = static_cast<const Node<D>*>(t.nodes);
  const unsigned FULL = 0xffffffffu;
  const int lane = (int)(threadIdx.x & 31u);
  const int gl = lane & (L - 1);
  const int gbase = lane - gl;
  const unsigned gmask = L == 32 ? FULL : (((1u << L) - 1u) << gbase);
  unsigned long long st[SD];  // (node code << 32) | bits of its box distance
  unsigned long long n_nodes = 0;
  WarpQueue wq;
  bool active = false;  // the same in every lane of a group
  int64_t slot = 0, qi = 0;
  float q[D];
  GroupList<K, L> h;
  int sp = 0;
  int64_t steps = 0;
  int32_t cur = 0;
  float bound = F_INF;        // lane runs (per group): carried upper bound on the k-th d2 (see k_knn)
  float pq[RUN > 1 ? D : 1];
  float pdk = F_INF;
  LaneRun<RUN, 32 / L> run;
  for (;;) {
    if constexpr (RUN > 1) {
      if (__all_sync(FULL, !active)) {
        bool fresh = false;
        if (!run.next(a.counter, a.m, lane / L, slot, fresh)) break;
        if (fresh) pdk = F_INF;
        if (slot < a.m) {
          qi = query_at(a.order, slot, a.nq > 0 ? a.nq : a.m, a.err);
#pragma unroll
          for (int x = 0; x < D; ++x) q[x] = a.qs[qi * D + x];
          bound = pdk < F_INF ? knn_carry_bound<D>(pq, pdk, q) : F_INF;
          h.init();
          sp = 0;
          cur = t.root;
          steps = 0;
          active = true;
        }
        if (!__any_sync(FULL, active)) continue;
      }
    } else if (a.refill || __all_sync(FULL, !active)) {
      // the group's first lane asks for a slot for the group
      const bool got0 = warp_refill(a.counter, a.m, wq, active || gl != 0, slot);
      const bool got = __shfl_sync(FULL, got0, gbase);
      const int64_t gslot = __shfl_sync(FULL, slot, gbase);
      if (got) {
        slot = gslot;
        qi = query_at(a.order, slot, a.nq > 0 ? a.nq : a.m, a.err);
#pragma unroll
        for (int x = 0; x < D; ++x) q[x] = a.qs[qi * D + x];
        h.init();
        sp = 0;
        cur = t.root;
        steps = 0;
        active = true;
      }
    }
    if (RUN == 1 && !__any_sync(FULL, active) && wq.exhausted) break;
    if (active && ++steps > 4 * t.n + 1024) {
      if (gl == 0) atomicOr(a.err, DEVERR_INTERNAL);
      active = false;
    }
    if (active) {
      const Kids<D> k = unpack(fetch(cur, t, g, s_top));
      if (STATS && gl == 0) ++n_nodes;
      const bool v1 = k.child[1] != NULL_CHILD;
      const float d0 = box_d2<D>(q, k.lo[0], k.hi[0]);
      const float d1 = v1 ? box_d2<D>(q, k.lo[1], k.hi[1]) : F_INF;
      const unsigned long long x0 = k.child[0] < 0 ? RegList<1>::key(d0, k.orig[0]) : GroupList<K, L>::EMPTY;
      const unsigned long long x1 = v1 && k.child[1] < 0 ? RegList<1>::key(d1, k.orig[1]) : GroupList<K, L>::EMPTY;
      const bool lt = x0 < x1;
      h.insert_key(lt ? x0 : x1, gmask, gl);
      h.insert_key(lt ? x1 : x0, gmask, gl);
      const float worst = RUN > 1 ? fminf(h.worst_d(gmask), bound) : h.worst_d(gmask);
      const bool g0 = k.child[0] >= 0 && d0 <= worst;
      const bool g1 = v1 && k.child[1] >= 0 && d1 <= worst;
      bool done = false;
      int32_t next = -1;
      if (g0 && g1) {
        const bool first1 = d1 < d0;
        next = first1 ? k.child[1] : k.child[0];
        if (sp < SD * L) {
          if ((sp & (L - 1)) == gl)
            st[sp / L] = ((unsigned long long)(uint32_t)(first1 ? k.child[0] : k.child[1]) << 32) |
                         __float_as_uint(first1 ? d0 : d1);
          ++sp;
        } else {
          if (gl == 0) atomicOr(a.err, DEVERR_STACK);
          done = true;
        }
      } else if (g0) {
        next = k.child[0];
      } else if (g1) {
        next = k.child[1];
      }
      if (!done && next < 0) {
        // pop, discarding entries that can no longer hold a better pair
        while (sp > 0) {
          --sp;
          const int owner = sp & (L - 1);
          unsigned long long e = owner == gl ? st[sp / L] : 0ull;
          e = __shfl_sync(gmask, e, owner, L);
          if (__uint_as_float((uint32_t)e) <= worst) {
            next = (int32_t)(uint32_t)(e >> 32);
            break;
          }
        }
        if (next < 0) done = true;
      }
      cur = next;
      if (done) {
        h.write(a.out_idx ? a.out_idx + qi * a.kk : nullptr, a.out_d2 ? a.out_d2 + qi * a.kk : nullptr, a.kk, gl);
        active = false;
        if constexpr (RUN > 1) {
#pragma unroll
          for (int x = 0; x < D; ++x) pq[x] = q[x];
          pdk = h.worst_d(gmask);
        }
      }
    }
  }
  if (STATS) add_stats(a.stats, n_nodes, 0ull, 0ull);
}

struct RayArgs {
  const float* rays;
  const uint32_t* order;
  int64_t m;
  int kk;        // output columns: hit/t are [m][kk]
  int32_t* hit;
  float* t;
  uint32_t* err;
  unsigned long long* stats;
  unsigned long long* counter;
  bool refill;
  int64_t nq = 0;  // queries in the data arrays when `order` lists a subset of them (0: m)
};


// nearest(ray, k): the K smallest (t, index) hits; K = 1 is the first hit.
template <class NodeT, int K, bool STATS = false>
__global__ void __launch_bounds__(256) k_ray(TreeView t, RayArgs a) {
  extern __shared__ float4 smem_top[];
  const NodeT* s_top = stage_top<NodeT>(t, smem_top);
  const NodeT* __restrict__ g = static_cast<const NodeT*>(t.nodes);
  int32_t st[STACK_DEPTH];
  float stn[STACK_DEPTH];
  unsigned long long n_nodes = 0, n_leaves = 0, n_hits = 0;
  WarpQueue wq;
  bool active = false;
  int64_t slot = 0, qi = 0;
  Ray r;
  LexList<K> h;
  int sp = 0;
  uint32_t steps = 0;
  const uint32_t step_cap = step_limit(t.n);
  int32_t cur = 0;
  Frames<NodeT> fr;
  for (;;) {
    // new rays when the warp has none left (or, with lane refill, whenever a
    // lane is free); one vote per step while the warp is busy
    if (a.refill || __all_sync(0xffffffffu, !active)) {
      if (warp_refill(a.counter, a.m, wq, active, slot)) {
        qi = query_at(a.order, slot, a.nq > 0 ? a.nq : a.m, a.err);
#pragma unroll
        for (int x = 0; x < 3; ++x) {
          r.o[x] = a.rays[qi * 6 + x];
          r.d[x] = a.rays[qi * 6 + 3 + x];
          r.inv[x] = __frcp_rn(r.d[x]);
        }
        h.init();
        sp = 0;
        cur = t.root;
        fr.root(t);
        steps = 0;
        active = true;
      }
      if (!__any_sync(0xffffffffu, active)) {
        if (wq.exhausted) break;
        continue;
      }
    }
    if (active && ++steps > step_cap) {
      // a traversal takes fewer than 2n steps: a runaway query is stopped and reported
      atomicOr(a.err, DEVERR_INTERNAL);
      active = false;
    }
    if (active) {
      const Kids<3> k = fr.open(fetch(cur, t, g, s_top));
      if (STATS) ++n_nodes;
      float tn0 = F_INF, tn1 = F_INF;
      const bool v1 = k.child[1] != NULL_CHILD;
      const bool h0 = slab(r, k.lo[0], k.hi[0], h.hd[K - 1], tn0);
      const bool h1 = v1 && slab(r, k.lo[1], k.hi[1], h.hd[K - 1], tn1);
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        if ((c == 0 ? h0 : h1) && k.child[c] < 0) {
          const TriLeaf L = load_node_global(t.leaves + leaf_index(~k.child[c], t));
          if (STATS) ++n_leaves;
          float th;
          if (moller_trumbore(r, L.v, th)) h.insert(th, L.orig);
        }
      }
      const float worst = h.hd[K - 1];
      const bool g0 = h0 && k.child[0] >= 0 && tn0 <= worst;
      const bool g1 = h1 && k.child[1] >= 0 && tn1 <= worst;
      bool done = false;
      int32_t next = -1;
      if (g0 && g1) {
        const bool first1 = tn1 < tn0;
        next = first1 ? k.child[1] : k.child[0];
        fr.go(k, first1 ? 1 : 0);
        if (sp < STACK_DEPTH) {
          st[sp] = first1 ? k.child[0] : k.child[1];
          stn[sp] = first1 ? tn0 : tn1;
          fr.push(sp, k, first1 ? 0 : 1);
          ++sp;
        } else {
          atomicOr(a.err, DEVERR_STACK);
          done = true;
        }
      } else if (g0) {
        next = k.child[0];
        fr.go(k, 0);
      } else if (g1) {
        next = k.child[1];
        fr.go(k, 1);
      }
      if (!done && next < 0) {
        while (sp > 0 && stn[sp - 1] > h.hd[K - 1]) --sp;
        if (sp > 0) {
          next = st[--sp];
          fr.pop(sp);
        } else {
          done = true;
        }
      }
      cur = next;
      if (done) {
#pragma unroll
        for (int s = 0; s < K; ++s) {
          if (s < a.kk) {
            if (a.hit) a.hit[qi * a.kk + s] = h.hj[s] == INT32_MAX ? -1 : h.hj[s];
            if (a.t) a.t[qi * a.kk + s] = h.hd[s];
          }
          if (STATS) n_hits += h.hj[s] != INT32_MAX;
        }
        active = false;
      }
    }
  }
  if (STATS) add_stats(a.stats, n_nodes, n_leaves, n_hits);
}

// ------------------------------------------------------------------ ordering

// Morton code (30 bits at most) of each query's centre: the point, the box
// centre, or the ray origin.
template <int D, int PK>
__global__ void __launch_bounds__(256) k_query_codes(const float* __restrict__ qs, int64_t m,
                                                     const float* __restrict__ scene, int bits,
                                                     uint64_t* __restrict__ keys, uint32_t* __restrict__ vals) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const uint32_t cmax = (1u << bits) - 1u;
  uint32_t cell[D];
#pragma unroll
  for (int a = 0; a < D; ++a) {
    float c;
    if (PK == ARBX_BOX_PRED) c = 0.5f * (qs[i * 2 * D + a] + qs[i * 2 * D + D + a]);
    else if (PK == ARBX_RAY_NEAREST) c = qs[i * 6 + a];
    else c = qs[i * D + a];
    const float lo = scene[a], ext = scene[D + a] - scene[a];
    float u = ext > 0.0f ? (c - lo) * ((float)(1u << bits) / ext) : 0.0f;
    u = fminf(fmaxf(u, 0.0f), (float)cmax);  // NaN -> 0
    cell[a] = (uint32_t)u;
  }
  uint64_t code = 0;
  for (int b = bits - 1; b >= 0; --b) {
#pragma unroll
    for (int a = 0; a < D; ++a) code = (code << 1) | ((cell[a] >> b) & 1u);
  }
  keys[i] = code;
  vals[i] = (uint32_t)i;
}

// ------------------------------------------------------------------ launch

// Per-(kernel, device, block, shared bytes) launch facts, computed once and
// shared by every host thread (the serving runtime launches from several).
struct LaunchKey {
  const void* fn;
  int device, block;
  size_t smem;
  bool operator==(const LaunchKey& o) const {
    return fn == o.fn && device == o.device && block == o.block && smem == o.smem;
  }
};
struct LaunchKeyHash {
  size_t operator()(const LaunchKey& k) const {
    return std::hash<const void*>()(k.fn) ^ (size_t)k.device * 0x9e3779b97f4a7c15ull ^ (size_t)k.block << 20 ^ k.smem;
  }
};
std::mutex g_launch_mu;
std::unordered_map<LaunchKey, int, LaunchKeyHash> g_occupancy;
std::unordered_map<LaunchKey, bool, LaunchKeyHash> g_smem_set;

template <class Kernel>
arbx_status grid_for(Kernel k, const QueryPlan& p, size_t smem, int* grid) {
  int per_sm = p.grid_per_sm;
  if (per_sm <= 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    const LaunchKey key{(const void*)k, dev, p.block, smem};
    std::lock_guard<std::mutex> lk(g_launch_mu);
    auto it = g_occupancy.find(key);
    if (it == g_occupancy.end()) {
      ARBX_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, p.block, smem));
      it = g_occupancy.emplace(key, per_sm).first;
    }
    per_sm = it->second;
    if (per_sm <= 0) return ARBX_ERR_UNSUPPORTED;
  }
  const int64_t need = (p.m * (p.lanes > 1 ? p.lanes : 1) + p.block - 1) / p.block;
  *grid = (int)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)per_sm * num_sms()));
  return ARBX_OK;
}

// Allow the kernel the device's whole opt-in dynamic shared memory, once per
// (kernel, device).  The attribute is a per-kernel maximum: setting it to
// each launch's own size would let a smaller later launch lower the limit
// below a larger size already marked as set.
template <class Kernel>
arbx_status prepare(Kernel k, size_t smem) {
  if (smem <= 48 * 1024) return ARBX_OK;
  int dev = 0;
  cudaGetDevice(&dev);
  const LaunchKey key{(const void*)k, dev, 0, 0};
  std::lock_guard<std::mutex> lk(g_launch_mu);
  if (g_smem_set.count(key)) return ARBX_OK;
  const int optin = max_smem_optin();
  if ((size_t)optin < smem) return ARBX_ERR_UNSUPPORTED;
  ARBX_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
  g_smem_set.emplace(key, true);
  return ARBX_OK;
}

// Launch a traversal kernel whose Args carry a `counter` for the warp work
// queue (zeroed here, stream-ordered).
template <class Kernel, class Args>
arbx_status launch_traversal(const char* name, Kernel kern, const QueryPlan& p, size_t smem, Args a, cudaStream_t s) {
  ARBX_TRY(prepare(kern, smem));
  int grid = 0;
  ARBX_TRY(grid_for(kern, p, smem, &grid));
  DevTemp<unsigned long long> counter(s);
  ARBX_TRY(counter.alloc(1));
  ARBX_CUDA(cudaMemsetAsync(counter.p, 0, sizeof(unsigned long long), s));
  a.counter = counter.p;
  ARBX_LAUNCH(name, s, kern<<<grid, p.block, smem, s>>>(p.tv, a));
  return ARBX_OK;
}

const char* const SPATIAL_NAMES[4] = {"spatial_count", "spatial_count_up_to", "spatial_fill", "spatial_single"};

// The four-wide records serve a plan that asks for them when the tree has them
// and no top levels are staged (the wide kernels stage none).
bool use_wide(const QueryPlan& p) { return p.wide && p.tv.wide && p.tv.ntop == 0 && !p.stackless; }

template <int D, class Pred, int MODE, bool STATS = false>
arbx_status launch_count_wide(const QueryPlan& p, const SpatialArgs& a, cudaStream_t s) {
  return launch_traversal(STATS ? "stats" : SPATIAL_NAMES[MODE], k_count_wide<D, Pred, MODE, STATS>, p, 0, a, s);
}


template <int D, class NodeT, class Pred, int MODE, bool QUANT, bool STATS = false>
arbx_status launch_spatial(const QueryPlan& p, const SpatialArgs& a, cudaStream_t s) {
  const size_t smem = (size_t)p.tv.ntop * sizeof(NodeT) +
                      (MODE == MODE_FILL || MODE == MODE_SINGLE ? FillBuffer::bytes(p.block) : 0);
  return launch_traversal(STATS ? "stats" : SPATIAL_NAMES[MODE], k_spatial<D, NodeT, Pred, MODE, QUANT, STATS>, p,
                          smem, a, s);
}

const char* const ROPE_NAMES[3] = {"spatial_count_stackless", "spatial_count_up_to_stackless",
                                  "spatial_fill_stackless"};

template <int D, class Pred, int MODE, bool STATS = false>
arbx_status launch_rope(const QueryPlan& p, const SpatialArgs& a, cudaStream_t s) {
  const size_t smem = (size_t)p.tv.ntop * sizeof(Node<D>) + (MODE == MODE_FILL ? FillBuffer::bytes(p.block) : 0);
  return launch_traversal(STATS ? "stats" : ROPE_NAMES[MODE], k_spatial_rope<D, Pred, MODE, STATS>, p, smem, a, s);
}

template <int D, class Pred>
arbx_status spatial_mode(const QueryPlan& p, int mode, const SpatialArgs& a, cudaStream_t s) {
  if (p.stackless && mode != MODE_SINGLE) {  // the single pass has a stack traversal only
    switch (mode) {
      case MODE_COUNT: return launch_rope<D, Pred, MODE_COUNT>(p, a, s);
      case MODE_COUNT_UP_TO: return launch_rope<D, Pred, MODE_COUNT_UP_TO>(p, a, s);
      default: return launch_rope<D, Pred, MODE_FILL>(p, a, s);
    }
  }
  switch (mode) {
    case MODE_COUNT:
      if (use_wide(p)) return launch_count_wide<D, Pred, MODE_COUNT>(p, a, s);
      return launch_spatial<D, Node<D>, Pred, MODE_COUNT, false>(p, a, s);
    case MODE_COUNT_UP_TO:
      if (use_wide(p)) return launch_count_wide<D, Pred, MODE_COUNT_UP_TO>(p, a, s);
      return launch_spatial<D, Node<D>, Pred, MODE_COUNT_UP_TO, false>(p, a, s);
    case MODE_SINGLE: return launch_spatial<D, Node<D>, Pred, MODE_SINGLE, false>(p, a, s);
    default: return launch_spatial<D, Node<D>, Pred, MODE_FILL, false>(p, a, s);
  }
}

template <class NodeT>
arbx_status spatial_quantized(const QueryPlan& p, int mode, const SpatialArgs& a, cudaStream_t s) {
  switch (mode) {
    case MODE_COUNT: return launch_spatial<3, NodeT, BoxPred<3>, MODE_COUNT, true>(p, a, s);
    case MODE_COUNT_UP_TO: return launch_spatial<3, NodeT, BoxPred<3>, MODE_COUNT_UP_TO, true>(p, a, s);
    case MODE_SINGLE: return launch_spatial<3, NodeT, BoxPred<3>, MODE_SINGLE, true>(p, a, s);
    default: return launch_spatial<3, NodeT, BoxPred<3>, MODE_FILL, true>(p, a, s);
  }
}

template <int D, int K, bool STATS = false>
arbx_status launch_knn(const QueryPlan& p, const KnnArgs& a, cudaStream_t s) {
  using Heap = RegList<K>;
  const size_t smem = (size_t)p.tv.ntop * sizeof(Node<D>) + Heap::smem_bytes(p.block);
  const char* name = STATS ? "stats" : "knn";
  if (p.knn_run == 4) return launch_traversal(name, k_knn<D, Heap, STATS, 4>, p, smem, a, s);
  if (p.knn_run == 8) return launch_traversal(name, k_knn<D, Heap, STATS, 8>, p, smem, a, s);
  return launch_traversal(name, k_knn<D, Heap, STATS>, p, smem, a, s);
}

template <int D, int K, bool STATS = false>
arbx_status launch_knn_wide(const QueryPlan& p, const KnnArgs& a, cudaStream_t s) {
  const char* name = STATS ? "stats" : "knn";
  if (p.knn_run == 4) return launch_traversal(name, k_knn_wide<D, K, STATS, 4>, p, 0, a, s);
  if (p.knn_run == 8) return launch_traversal(name, k_knn_wide<D, K, STATS, 8>, p, 0, a, s);
  return launch_traversal(name, k_knn_wide<D, K, STATS>, p, 0, a, s);
}

template <int D, int K, int L, bool STATS = false>
arbx_status launch_knn_group(const QueryPlan& p, const KnnArgs& a, cudaStream_t s) {
  QueryPlan pl = p;
  pl.lanes = L;
  const char* name = STATS ? "stats" : "knn";
  const size_t smem = (size_t)p.tv.ntop * sizeof(Node<D>);
  if (p.knn_run == 4) return launch_traversal(name, k_knn_group<D, K, L, STATS, 4>, pl, smem, a, s);
  if (p.knn_run == 8) return launch_traversal(name, k_knn_group<D, K, L, STATS, 8>, pl, smem, a, s);
  return launch_traversal(name, k_knn_group<D, K, L, STATS>, pl, smem, a, s);
}

// One list size K (a power of two >= k): one lane per query (k_knn) or a lane
// group of L = p.lanes lanes (L <= K, 8 at most).
template <int D, int K, bool STATS = false>
arbx_status knn_lanes(const QueryPlan& p, const KnnArgs& a, cudaStream_t s) {
  const int L = p.lanes < K ? p.lanes : K;
  if (L <= 1 && p.packets && p.tv.ntop == 0)
    return launch_traversal(STATS ? "stats" : "knn", k_knn_packet<D, K, STATS>, p, 0, a, s);
  if (L <= 1 && use_wide(p)) return launch_knn_wide<D, K, STATS>(p, a, s);
  if (STATS || L <= 1) {
    // lane groups (k <= 32): their visits are counted on the one-lane walk
    // without lane runs
    if (L > 1 && p.knn_run != 1) {
      QueryPlan pl = p;
      pl.knn_run = 1;
      return launch_knn<D, K, STATS>(pl, a, s);
    }
    return launch_knn<D, K, STATS>(p, a, s);  // same node visits for every L
  }
  if constexpr (K >= 2) {
    if (L == 2) return launch_knn_group<D, K, 2>(p, a, s);
  }
  if constexpr (K >= 4) {
    if (L == 4) return launch_knn_group<D, K, 4>(p, a, s);
  }
  if constexpr (K >= 8) {
    if (L == 8) return launch_knn_group<D, K, 8>(p, a, s);
  }
  return ARBX_ERR_INVALID;
}

// Lists longer than 32 keys: groups of K/32, K/16 or K/8 lanes (p.lanes picks
// one of these; anything else takes K/16).  The node visits are the same for
// every group size, so instrumented runs use K/16.
template <int D, int K, bool STATS = false>
arbx_status knn_long(const QueryPlan& p, const KnnArgs& a, cudaStream_t s) {
  if (!STATS && p.lanes == K / 32) return launch_knn_group<D, K, K / 32>(p, a, s);
  if (!STATS && p.lanes == K / 8) return launch_knn_group<D, K, K / 8>(p, a, s);
  return launch_knn_group<D, K, K / 16, STATS>(p, a, s);
}

template <int D, bool STATS = false>
arbx_status knn_dim(const QueryPlan& p, int k, const KnnArgs& a, cudaStream_t s) {
  if (k <= 1) return knn_lanes<D, 1, STATS>(p, a, s);
  if (k <= 2) return knn_lanes<D, 2, STATS>(p, a, s);
  if (k <= 4) return knn_lanes<D, 4, STATS>(p, a, s);
  if (k <= 8) return knn_lanes<D, 8, STATS>(p, a, s);
  if (k <= 16) return knn_lanes<D, 16, STATS>(p, a, s);
  if (k <= 32) return knn_lanes<D, 32, STATS>(p, a, s);
  // longer lists: a lane group of K / KL lanes holding KL = 32, 16 or 8 keys
  // per lane (p.lanes asks for a group size; the default is 16 keys per lane)
  if (k <= 64) return knn_long<D, 64, STATS>(p, a, s);
  if (k <= 128) return knn_long<D, 128, STATS>(p, a, s);
  if (k <= KNN_MAX_K) return knn_long<D, 256, STATS>(p, a, s);
  return ARBX_ERR_UNSUPPORTED;
}

template <class NodeT, bool QUANT>
arbx_status ray_intersect_mode(const QueryPlan& p, int mode, const SpatialArgs& a, cudaStream_t s) {
  switch (mode) {
    case MODE_COUNT: return launch_spatial<3, NodeT, RayPred, MODE_COUNT, QUANT>(p, a, s);
    case MODE_COUNT_UP_TO: return launch_spatial<3, NodeT, RayPred, MODE_COUNT_UP_TO, QUANT>(p, a, s);
    case MODE_SINGLE: return launch_spatial<3, NodeT, RayPred, MODE_SINGLE, QUANT>(p, a, s);
    default: return launch_spatial<3, NodeT, RayPred, MODE_FILL, QUANT>(p, a, s);
  }
}

template <bool STATS>
arbx_status spatial_dispatch(const QueryPlan& p, int mode, const SpatialArgs& a, cudaStream_t s) {
  if (p.pred_kind == ARBX_RAY_INTERSECT || p.pred_kind == ARBX_RAY_ORDERED) {
    if (p.prim_kind != ARBX_TRIANGLE) return ARBX_ERR_UNSUPPORTED;
    if (p.prel)
      return STATS ? launch_spatial<3, PNode, RayPred, MODE_COUNT, true, true>(p, a, s)
                   : ray_intersect_mode<PNode, true>(p, mode, a, s);
    if (p.quantized)
      return STATS ? launch_spatial<3, QNode, RayPred, MODE_COUNT, true, true>(p, a, s)
                   : ray_intersect_mode<QNode, true>(p, mode, a, s);
    return STATS ? launch_spatial<3, Node<3>, RayPred, MODE_COUNT, false, true>(p, a, s)
                 : ray_intersect_mode<Node<3>, false>(p, mode, a, s);
  }
  if (p.quantized) {
    if (p.pred_kind != ARBX_BOX_PRED) return ARBX_ERR_UNSUPPORTED;
    if (p.prel) {
      if (STATS) return launch_spatial<3, PNode, BoxPred<3>, MODE_COUNT, true, true>(p, a, s);
      return spatial_quantized<PNode>(p, mode, a, s);
    }
    if (STATS) return launch_spatial<3, QNode, BoxPred<3>, MODE_COUNT, true, true>(p, a, s);
    return spatial_quantized<QNode>(p, mode, a, s);
  }
  if (p.pred_kind == ARBX_SPHERE) {
    if (p.prim_kind == ARBX_TRIANGLE) return ARBX_ERR_UNSUPPORTED;
    switch (p.dim) {
      case 2: return STATS ? (p.stackless ? launch_rope<2, SpherePred<2>, MODE_COUNT, true>(p, a, s)
                                         : launch_spatial<2, Node<2>, SpherePred<2>, MODE_COUNT, false, true>(p, a, s))
                           : spatial_mode<2, SpherePred<2>>(p, mode, a, s);
      case 3: return STATS ? (p.stackless ? launch_rope<3, SpherePred<3>, MODE_COUNT, true>(p, a, s)
                                         : launch_spatial<3, Node<3>, SpherePred<3>, MODE_COUNT, false, true>(p, a, s))
                           : spatial_mode<3, SpherePred<3>>(p, mode, a, s);
      case 6: return STATS ? (p.stackless ? launch_rope<6, SpherePred<6>, MODE_COUNT, true>(p, a, s)
                                         : launch_spatial<6, Node<6>, SpherePred<6>, MODE_COUNT, false, true>(p, a, s))
                           : spatial_mode<6, SpherePred<6>>(p, mode, a, s);
    }
  } else if (p.pred_kind == ARBX_BOX_PRED) {
    switch (p.dim) {
      case 2: return STATS ? (p.stackless ? launch_rope<2, BoxPred<2>, MODE_COUNT, true>(p, a, s)
                                         : launch_spatial<2, Node<2>, BoxPred<2>, MODE_COUNT, false, true>(p, a, s))
                           : spatial_mode<2, BoxPred<2>>(p, mode, a, s);
      case 3: return STATS ? (p.stackless ? launch_rope<3, BoxPred<3>, MODE_COUNT, true>(p, a, s)
                                         : launch_spatial<3, Node<3>, BoxPred<3>, MODE_COUNT, false, true>(p, a, s))
                           : spatial_mode<3, BoxPred<3>>(p, mode, a, s);
      case 6: return STATS ? (p.stackless ? launch_rope<6, BoxPred<6>, MODE_COUNT, true>(p, a, s)
                                         : launch_spatial<6, Node<6>, BoxPred<6>, MODE_COUNT, false, true>(p, a, s))
                           : spatial_mode<6, BoxPred<6>>(p, mode, a, s);
    }
  }
  return ARBX_ERR_UNSUPPORTED;
}

// Instrumented counting walk over the four-wide records (sphere or box predicates).
arbx_status count_wide_stats(const QueryPlan& p, const SpatialArgs& a, cudaStream_t s) {
  const bool sph = p.pred_kind == ARBX_SPHERE;
  switch (p.dim) {
    case 2: return sph ? launch_count_wide<2, SpherePred<2>, MODE_COUNT, true>(p, a, s)
                       : launch_count_wide<2, BoxPred<2>, MODE_COUNT, true>(p, a, s);
    case 3: return sph ? launch_count_wide<3, SpherePred<3>, MODE_COUNT, true>(p, a, s)
                       : launch_count_wide<3, BoxPred<3>, MODE_COUNT, true>(p, a, s);
    case 6: return sph ? launch_count_wide<6, SpherePred<6>, MODE_COUNT, true>(p, a, s)
                       : launch_count_wide<6, BoxPred<6>, MODE_COUNT, true>(p, a, s);
  }
  return ARBX_ERR_UNSUPPORTED;
}

template <bool STATS>
arbx_status knn_dispatch(const QueryPlan& p, int k, const KnnArgs& a, cudaStream_t s) {
  switch (p.dim) {
    case 2: return knn_dim<2, STATS>(p, k, a, s);
    case 3: return knn_dim<3, STATS>(p, k, a, s);
    case 6: return knn_dim<6, STATS>(p, k, a, s);
  }
  return ARBX_ERR_UNSUPPORTED;
}

template <class NodeT, int K, bool STATS>
arbx_status launch_ray(const QueryPlan& p, const RayArgs& a, cudaStream_t s) {
  const char* name = std::is_same<NodeT, QNode>::value   ? "ray_nearest_q16"
                     : std::is_same<NodeT, PNode>::value ? "ray_nearest_p16"
                                                         : "ray_nearest";
  return launch_traversal(STATS ? "stats" : name, k_ray<NodeT, K, STATS>, p,
                          (size_t)p.tv.ntop * sizeof(NodeT), a, s);
}

template <class NodeT, bool STATS>
arbx_status ray_k(const QueryPlan& p, int k, const RayArgs& a, cudaStream_t s) {
  if (k <= 1) return launch_ray<NodeT, 1, STATS>(p, a, s);
  if (k <= 2) return launch_ray<NodeT, 2, STATS>(p, a, s);
  if (k <= 4) return launch_ray<NodeT, 4, STATS>(p, a, s);
  if (k <= 8) return launch_ray<NodeT, 8, STATS>(p, a, s);
  if (k <= 16) return launch_ray<NodeT, 16, STATS>(p, a, s);
  return launch_ray<NodeT, 32, STATS>(p, a, s);
}

template <bool STATS>
arbx_status ray_dispatch(const QueryPlan& p, int k, const RayArgs& a, cudaStream_t s) {
  if (k > 32) return ARBX_ERR_UNSUPPORTED;
  if (p.prel) return ray_k<PNode, STATS>(p, k, a, s);
  if (p.quantized) return ray_k<QNode, STATS>(p, k, a, s);
  return ray_k<Node<3>, STATS>(p, k, a, s);
}

}  // namespace

namespace {

// Work classes of the fill pass's chunks (CHUNK consecutive slots of the
// processing order): the leading zeros of w = matches + 16 per query, i.e.
// 63 - floor(log2 w), so a stable sort by class hands out the heaviest chunks
// first and keeps the processing order inside a class.
__global__ void k_chunk_classes(const uint32_t* __restrict__ order, const int64_t* __restrict__ offsets, int64_t m,
                                int64_t nq, int64_t nchunks, uint32_t* __restrict__ keys, uint32_t* __restrict__ ids,
                                uint32_t* err) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nchunks) return;
  uint64_t w = 0;
  const int64_t end = min((c + 1) * (int64_t)CHUNK, m);
  for (int64_t slot = c * CHUNK; slot < end; ++slot) {
    const int64_t q = query_at(order, slot, nq, err);
    w += (uint64_t)(offsets[q + 1] - offsets[q]) + 16;
  }
  keys[c] = (uint32_t)__clzll((long long)w);
  ids[c] = (uint32_t)c;
}

}  // namespace

arbx_status run_spatial(const QueryPlan& p, int mode, int32_t limit, int32_t* counts, const int64_t* offsets,
                        int32_t* indices, float* d2, cudaStream_t s) {
  if (p.m == 0) return ARBX_OK;
  SpatialArgs a{p.qdata, p.radii, p.r2, p.order, p.m, limit, counts, offsets, indices, d2, nullptr, nullptr, nullptr,
                p.refill > 0};
  a.nq = p.nq > 0 ? p.nq : p.m;
  ARBX_TRY(device_error_word(&a.err));
  a.contain = (mode == MODE_COUNT || mode == MODE_COUNT_UP_TO) && p.prim_kind != ARBX_BOX;
  // fill pass: the match counts are known, so the heaviest chunks go first
  // (a heavy chunk handed out last leaves the GPU waiting on one warp)
  DevTemp<uint32_t> perm(s);
  const int64_t nchunks = (p.m + CHUNK - 1) / CHUNK;
  if (mode == MODE_FILL && nchunks >= 1024) {
    DevTemp<uint32_t> keys(s), keys_alt(s), ids_alt(s);
    ARBX_TRY(keys.alloc(nchunks));
    ARBX_TRY(keys_alt.alloc(nchunks));
    ARBX_TRY(ids_alt.alloc(nchunks));
    ARBX_TRY(perm.alloc(nchunks));
    ARBX_LAUNCH("chunk_classes", s, k_chunk_classes<<<(unsigned)((nchunks + 255) / 256), 256, 0, s>>>(
                                        p.order, offsets, p.m, a.nq, nchunks, keys.p, perm.p, a.err));
    bool alt = false;
    ARBX_TRY(radix_sort_pairs<uint32_t>(keys.p, perm.p, keys_alt.p, ids_alt.p, nchunks, 0, 8, &alt, s));
    if (alt)
      ARBX_CUDA(cudaMemcpyAsync(perm.p, ids_alt.p, (size_t)nchunks * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
    a.chunk_perm = perm.p;
  }
  return spatial_dispatch<false>(p, mode, a, s);
}

arbx_status run_spatial_single(const QueryPlan& p, const SingleStore& store, int32_t* counts, cudaStream_t s) {
  if (p.m == 0) return ARBX_OK;
  SpatialArgs a{p.qdata, p.radii, p.r2, p.order, p.m, 0, counts, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
                p.refill > 0, store};
  a.nq = p.nq > 0 ? p.nq : p.m;
  ARBX_TRY(device_error_word(&a.err));
  return spatial_dispatch<false>(p, MODE_SINGLE, a, s);
}

namespace {

// A warp takes 32 consecutive queries (whose CRS segments are adjacent):
// each lane copies its query's inline slots, then the warp copies the chunk
// chains of the lanes whose queries have more, one chunk per store.
__global__ void __launch_bounds__(256) k_single_compact(SingleStore ss, const int32_t* __restrict__ counts,
                                                        const int64_t* __restrict__ offsets, int64_t m,
                                                        const uint8_t* __restrict__ skip, int32_t* __restrict__ idx,
                                                        float* __restrict__ d2) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
  for (int64_t base = ((int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5)) * 32; base < m;
       base += warps * 32) {
    const int64_t q = base + lane;
    int64_t c = 0, o = 0;
    if (q < m && !(skip && skip[q])) {
      c = counts[q];
      o = offsets[q];
    }
    const int ni = c < SINGLE_INLINE ? (int)c : SINGLE_INLINE;
    for (int e = 0; e < ni; ++e) {
      idx[o + e] = ss.in_idx[q * SINGLE_INLINE + e];
      if (d2) d2[o + e] = ss.in_d2[q * SINGLE_INLINE + e];
    }
    unsigned big = __ballot_sync(FULL, c > SINGLE_INLINE);
    while (big != 0u) {
      const int j = __ffs(big) - 1;
      big &= big - 1u;
      const int64_t cj = __shfl_sync(FULL, c, j);
      const int64_t oj = __shfl_sync(FULL, o, j);
      const int64_t qj = base + j;
      int32_t id = ss.head[qj];
      for (int64_t e0 = SINGLE_INLINE; e0 < cj; e0 += SINGLE_CHUNK) {
        const int64_t e = e0 + lane;
        if (e < cj) {
          idx[oj + e] = ss.pool_idx[(int64_t)id * SINGLE_CHUNK + lane];
          if (d2) d2[oj + e] = ss.pool_d2[(int64_t)id * SINGLE_CHUNK + lane];
        }
        if (e0 + SINGLE_CHUNK < cj) id = ss.next[id];
      }
    }
  }
}

__global__ void k_mark(const int32_t* __restrict__ list, int64_t n, uint8_t* __restrict__ flags) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) flags[list[i]] = 1;
}

__global__ void k_chunks_needed(const uint32_t* __restrict__ sample, int64_t ns, const int32_t* __restrict__ counts,
                                unsigned long long* need) {
  unsigned long long v = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ns; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = counts[sample[i]];
    if (c > SINGLE_INLINE) v += (unsigned long long)((c - SINGLE_INLINE + SINGLE_CHUNK - 1) / SINGLE_CHUNK);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0 && v) atomicAdd(need, v);
}

}  // namespace

arbx_status single_compact(const SingleStore& store, const int32_t* counts, const int64_t* offsets, int64_t m,
                           uint64_t novf, int32_t* indices, float* d2, cudaStream_t s) {
  if (m == 0) return ARBX_OK;
  DevTemp<uint8_t> skip(s);
  if (novf > 0) {
    ARBX_TRY(skip.alloc(m));
    ARBX_CUDA(cudaMemsetAsync(skip.p, 0, (size_t)m, s));
    ARBX_LAUNCH("single_mark", s, k_mark<<<(unsigned)((novf + 255) / 256), 256, 0, s>>>(store.ovf_list, (int64_t)novf, skip.p));
  }
  const int64_t blocks = std::min<int64_t>((m + 255) / 256, (int64_t)num_sms() * 8);
  ARBX_LAUNCH("single_compact", s, k_single_compact<<<(unsigned)blocks, 256, 0, s>>>(store, counts, offsets, m,
                                                                                    novf ? skip.p : nullptr, indices, d2));
  return ARBX_OK;
}

arbx_status single_chunks_needed(const uint32_t* sample, int64_t ns, const int32_t* counts,
                                 unsigned long long* need_dev, cudaStream_t s) {
  if (ns == 0) return ARBX_OK;
  const int64_t blocks = std::min<int64_t>((ns + 255) / 256, (int64_t)num_sms() * 4);
  ARBX_LAUNCH("single_estimate", s, k_chunks_needed<<<(unsigned)blocks, 256, 0, s>>>(sample, ns, counts, need_dev));
  return ARBX_OK;
}

arbx_status run_dbscan(const QueryPlan& p, const int32_t* counts, int32_t min_pts, int32_t* labels,
                       int64_t* n_clusters, cudaStream_t s) {
  *n_clusters = 0;
  const int64_t n = p.m;
  if (n == 0) return ARBX_OK;
  if (p.prim_kind != ARBX_POINT || p.quantized || p.radii) return ARBX_ERR_UNSUPPORTED;
  DevTemp<int32_t> parent(s);
  DevTemp<unsigned long long> clusters(s);
  ARBX_TRY(parent.alloc(n));
  ARBX_TRY(clusters.alloc(1));
  ARBX_CUDA(cudaMemsetAsync(clusters.p, 0, sizeof(unsigned long long), s));
  const unsigned g = (unsigned)((n + 255) / 256);
  ARBX_LAUNCH("uf_init", s, k_uf_init<<<g, 256, 0, s>>>(parent.p, n));
  // core points first, then the others, each in processing order
  DevTemp<int32_t> flags(s);
  DevTemp<int64_t> pos(s);
  DevTemp<uint32_t> split(s);
  ARBX_TRY(flags.alloc(n));
  ARBX_TRY(pos.alloc(n + 1));
  ARBX_TRY(split.alloc(n));
  uint32_t* err = nullptr;
  ARBX_TRY(device_error_word(&err));
  ARBX_LAUNCH("core_flags", s, k_core_flags<<<g, 256, 0, s>>>(p.order, counts, min_pts, n, flags.p, err));
  ARBX_TRY((exclusive_scan<int32_t, int64_t>(flags.p, pos.p, n, s)));
  int64_t ncore = 0;
  ARBX_TRY(read_small(pos.p + n, &ncore, sizeof(ncore), s));
  ARBX_LAUNCH("split_order", s, k_split_order<<<g, 256, 0, s>>>(p.order, flags.p, pos.p, n, ncore, split.p, err));
  QueryPlan pc = p, pb = p;
  pc.order = split.p;
  pc.m = ncore;
  pb.order = split.p + ncore;
  pb.m = n - ncore;
  DbscanArgs a{p.qdata, p.r2, pc.order, pc.m, counts, min_pts, parent.p, labels, nullptr, nullptr, p.refill > 0};
  a.nq = n;  // the split orders list subsets of all n points
  ARBX_TRY(device_error_word(&a.err));
  // the union phase walks only the leaves before each query's own position
  DevTemp<int32_t> leaf_pos(s);
  ARBX_TRY(leaf_pos.alloc(n));
  {
    const int64_t nn = n > 1 ? n - 1 : 1;
    const unsigned gn = (unsigned)((nn + 255) / 256);
    switch (p.dim) {
      case 2: ARBX_LAUNCH("leaf_positions", s, k_leaf_positions<2><<<gn, 256, 0, s>>>(static_cast<const Node<2>*>(p.tv.nodes), nn, n, leaf_pos.p, a.err)); break;
      case 3: ARBX_LAUNCH("leaf_positions", s, k_leaf_positions<3><<<gn, 256, 0, s>>>(static_cast<const Node<3>*>(p.tv.nodes), nn, n, leaf_pos.p, a.err)); break;
      case 6: ARBX_LAUNCH("leaf_positions", s, k_leaf_positions<6><<<gn, 256, 0, s>>>(static_cast<const Node<6>*>(p.tv.nodes), nn, n, leaf_pos.p, a.err)); break;
      default: return ARBX_ERR_UNSUPPORTED;
    }
  }
  a.leaf_pos = leaf_pos.p;
  DbscanArgs b = a;
  b.order = pb.order;
  b.m = pb.m;
  auto both = [&](auto k0, auto k1, size_t smem) -> arbx_status {
    if (pc.m > 0) ARBX_TRY(launch_traversal("dbscan_union", k0, pc, smem, a, s));
    ARBX_LAUNCH("core_labels", s, k_core_labels<<<g, 256, 0, s>>>(parent.p, counts, min_pts, n, labels, clusters.p,
                                                                    a.err));
    if (pb.m > 0) ARBX_TRY(launch_traversal("dbscan_border", k1, pb, smem, b, s));
    return ARBX_OK;
  };
  switch (p.dim) {
    case 2: ARBX_TRY(both(k_dbscan<2, 0>, k_dbscan<2, 1>, (size_t)p.tv.ntop * sizeof(Node<2>))); break;
    case 3: ARBX_TRY(both(k_dbscan<3, 0>, k_dbscan<3, 1>, (size_t)p.tv.ntop * sizeof(Node<3>))); break;
    case 6: ARBX_TRY(both(k_dbscan<6, 0>, k_dbscan<6, 1>, (size_t)p.tv.ntop * sizeof(Node<6>))); break;
    default: return ARBX_ERR_UNSUPPORTED;
  }
  unsigned long long c = 0;
  ARBX_TRY(read_small(clusters.p, &c, sizeof(c), s));
  *n_clusters = (int64_t)c;
  return ARBX_OK;
}

arbx_status run_knn(const QueryPlan& p, int k, int kk, int32_t* indices, float* d2, cudaStream_t s) {
  if (p.m == 0 || kk == 0) return ARBX_OK;
  if (p.prim_kind == ARBX_TRIANGLE || k > KNN_MAX_K) return ARBX_ERR_UNSUPPORTED;
  KnnArgs a{p.qdata, p.order, p.m, kk, indices, d2, nullptr, nullptr, nullptr, p.refill > 0};
  a.nq = p.nq > 0 ? p.nq : p.m;
  ARBX_TRY(device_error_word(&a.err));
  return knn_dispatch<false>(p, k, a, s);
}

arbx_status run_ray(const QueryPlan& p, int k, int32_t* hit, float* t, cudaStream_t s) {
  if (p.m == 0) return ARBX_OK;
  if (p.prim_kind != ARBX_TRIANGLE) return ARBX_ERR_UNSUPPORTED;
  const int kk = k > 1 ? k : 1;
  RayArgs a{p.qdata, p.order, p.m, kk, hit, t, nullptr, nullptr, nullptr, p.refill > 0};
  a.nq = p.nq > 0 ? p.nq : p.m;
  ARBX_TRY(device_error_word(&a.err));
  return ray_dispatch<false>(p, kk, a, s);
}

namespace {

// (t, index) as one key: the bits of t with -0 mapped to +0 (t >= 0 here, so
// the bits order like the values) above the index.
__global__ void k_hit_keys(const int32_t* __restrict__ idx, const float* __restrict__ t, int64_t nnz,
                           unsigned long long* __restrict__ keys, uint32_t* __restrict__ vals) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nnz) return;
  const float te = t[e];
  const uint32_t tb = te == 0.0f ? 0u : __float_as_uint(te);
  keys[e] = ((unsigned long long)tb << 32) | (uint32_t)idx[e];
  vals[e] = (uint32_t)e;
}

__global__ void k_seg_of_pos(const int64_t* __restrict__ offsets, int64_t m, uint32_t* __restrict__ seg) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= m) return;
  for (int64_t e = offsets[q]; e < offsets[q + 1]; ++e) seg[e] = (uint32_t)q;
}

__global__ void k_seg_keys(const uint32_t* __restrict__ vals, const uint32_t* __restrict__ seg, int64_t nnz,
                           uint32_t* __restrict__ keys) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < nnz) keys[e] = seg[vals[e]];
}

__global__ void k_gather_hits(const uint32_t* __restrict__ vals, const int32_t* __restrict__ idx,
                              const float* __restrict__ t, int64_t nnz, int32_t* __restrict__ idx2,
                              float* __restrict__ t2) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nnz) return;
  idx2[e] = idx[vals[e]];
  t2[e] = t[vals[e]];
}

}  // namespace

// Two stable radix sorts: all hits by (t, index), then by segment, which
// keeps the (t, index) order inside every segment.
arbx_status sort_segments_by_t(const int64_t* offsets, int64_t m, int64_t nnz, int32_t* idx, float* t,
                               cudaStream_t s) {
  if (nnz <= 1 || m == 0) return ARBX_OK;
  if (nnz >= (int64_t(1) << 32)) return ARBX_ERR_UNSUPPORTED;
  const unsigned g = (unsigned)((nnz + 255) / 256);
  DevTemp<uint32_t> v(s), vb(s);
  ARBX_TRY(v.alloc(nnz));
  ARBX_TRY(vb.alloc(nnz));
  uint32_t* vals = v.p;
  uint32_t* vals_other = vb.p;
  {
    DevTemp<uint64_t> k64(s), k64b(s);
    ARBX_TRY(k64.alloc(nnz));
    ARBX_TRY(k64b.alloc(nnz));
    ARBX_LAUNCH("hit_keys", s, k_hit_keys<<<g, 256, 0, s>>>(idx, t, nnz,
                                                            reinterpret_cast<unsigned long long*>(k64.p), v.p));
    bool alt = false;
    ARBX_TRY(radix_sort_pairs<uint64_t>(k64.p, v.p, k64b.p, vb.p, nnz, 0, 63, &alt, s));
    if (alt) std::swap(vals, vals_other);
  }
  int bits = 1;
  while (bits < 32 && (int64_t(1) << bits) < m) ++bits;
  {
    DevTemp<uint32_t> seg(s), k32(s), k32b(s);
    ARBX_TRY(seg.alloc(nnz));
    ARBX_TRY(k32.alloc(nnz));
    ARBX_TRY(k32b.alloc(nnz));
    ARBX_LAUNCH("seg_of_pos", s, k_seg_of_pos<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(offsets, m, seg.p));
    ARBX_LAUNCH("seg_keys", s, k_seg_keys<<<g, 256, 0, s>>>(vals, seg.p, nnz, k32.p));
    bool alt2 = false;
    ARBX_TRY(radix_sort_pairs<uint32_t>(k32.p, vals, k32b.p, vals_other, nnz, 0, bits, &alt2, s));
    if (alt2) std::swap(vals, vals_other);
  }
  DevTemp<int32_t> idx2(s);
  DevTemp<float> t2(s);
  ARBX_TRY(idx2.alloc(nnz));
  ARBX_TRY(t2.alloc(nnz));
  ARBX_LAUNCH("gather_hits", s, k_gather_hits<<<g, 256, 0, s>>>(vals, idx, t, nnz, idx2.p, t2.p));
  ARBX_CUDA(cudaMemcpyAsync(idx, idx2.p, (size_t)nnz * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
  ARBX_CUDA(cudaMemcpyAsync(t, t2.p, (size_t)nnz * sizeof(float), cudaMemcpyDeviceToDevice, s));
  return ARBX_OK;
}

arbx_status run_stats(const QueryPlan& p, int k, unsigned long long* stats_dev, cudaStream_t s, bool counting,
                      const float* r2s) {
  if (p.m == 0) return ARBX_OK;
  if (p.pred_kind == ARBX_RAY_NEAREST) {
    if (p.prim_kind != ARBX_TRIANGLE) return ARBX_ERR_UNSUPPORTED;
    const int kk = k > 1 ? k : 1;
    RayArgs a{p.qdata, p.order, p.m, kk, nullptr, nullptr, nullptr, stats_dev, nullptr, p.refill > 0};
    a.nq = p.nq > 0 ? p.nq : p.m;
    ARBX_TRY(device_error_word(&a.err));
    return ray_dispatch<true>(p, kk, a, s);
  }
  if (p.pred_kind == ARBX_NEAREST) {
    if (p.prim_kind == ARBX_TRIANGLE || k > KNN_MAX_K || k < 1) return ARBX_ERR_UNSUPPORTED;
    KnnArgs a{p.qdata, p.order, p.m, 0, nullptr, nullptr, nullptr, stats_dev, nullptr, p.refill > 0};
    a.nq = p.nq > 0 ? p.nq : p.m;
    ARBX_TRY(device_error_word(&a.err));
    return knn_dispatch<true>(p, k, a, s);
  }
  DevTemp<int32_t> counts(s);
  ARBX_TRY(counts.alloc(p.m));
  SpatialArgs a{p.qdata, p.radii, p.r2, p.order, p.m, 0, counts.p, nullptr, nullptr, nullptr, nullptr, stats_dev,
                nullptr, p.refill > 0};
  a.nq = p.nq > 0 ? p.nq : p.m;
  a.contain = counting && p.prim_kind != ARBX_BOX;
  a.r2s = r2s;
  ARBX_TRY(device_error_word(&a.err));
  if (r2s) {
    // the plain walk (no contained-subtree rule): every record whose box passes is fetched
    if (p.pred_kind != ARBX_SPHERE || p.prim_kind == ARBX_TRIANGLE || p.quantized) return ARBX_ERR_UNSUPPORTED;
    QueryPlan ps = p;
    ps.stackless = false;
    a.contain = false;
    if (use_wide(ps)) return count_wide_stats(ps, a, s);
    return spatial_dispatch<true>(ps, MODE_COUNT, a, s);
  }
  // the counting walk over the records the count pass would use
  if (counting && use_wide(p) && (p.pred_kind == ARBX_SPHERE || p.pred_kind == ARBX_BOX_PRED))
    return count_wide_stats(p, a, s);
  return spatial_dispatch<true>(p, MODE_COUNT, a, s);
}

namespace {

// Launch with a work counter and error word supplied (and zeroed) by the
// caller: no device allocation on this path.
template <class Kernel>
arbx_status launch_prealloc(Kernel kern, const QueryPlan& p, size_t smem, const SpatialArgs& a, cudaStream_t s) {
  ARBX_TRY(prepare(kern, smem));
  int grid = 0;
  ARBX_TRY(grid_for(kern, p, smem, &grid));
  ARBX_LAUNCH("spatial_count", s, kern<<<grid, p.block, smem, s>>>(p.tv, a));
  return ARBX_OK;
}

template <int D>
arbx_status count_prealloc_dim(const QueryPlan& p, const SpatialArgs& a, cudaStream_t s) {
  const size_t smem = (size_t)p.tv.ntop * sizeof(Node<D>);
  if (p.pred_kind == ARBX_SPHERE)
    return launch_prealloc(k_spatial<D, Node<D>, SpherePred<D>, MODE_COUNT, false>, p, smem, a, s);
  return launch_prealloc(k_spatial<D, Node<D>, BoxPred<D>, MODE_COUNT, false>, p, smem, a, s);
}

}  // namespace

arbx_status run_spatial_count_prealloc(const QueryPlan& p, int32_t* counts, unsigned long long* counter,
                                       uint32_t* err, cudaStream_t s) {
  if (p.m == 0) return ARBX_OK;
  SpatialArgs a{p.qdata, p.radii, p.r2, p.order, p.m, 0, counts, nullptr, nullptr, nullptr, err, nullptr, counter,
                p.refill > 0};
  a.nq = p.nq > 0 ? p.nq : p.m;
  a.contain = p.prim_kind != ARBX_BOX;
  if (p.quantized) {
    if (p.pred_kind != ARBX_BOX_PRED) return ARBX_ERR_UNSUPPORTED;
    if (p.prel)
      return launch_prealloc(k_spatial<3, PNode, BoxPred<3>, MODE_COUNT, true>, p,
                             (size_t)p.tv.ntop * sizeof(PNode), a, s);
    return launch_prealloc(k_spatial<3, QNode, BoxPred<3>, MODE_COUNT, true>, p, (size_t)p.tv.ntop * sizeof(QNode),
                           a, s);
  }
  if (p.pred_kind == ARBX_SPHERE && p.prim_kind == ARBX_TRIANGLE) return ARBX_ERR_UNSUPPORTED;
  if (p.pred_kind != ARBX_SPHERE && p.pred_kind != ARBX_BOX_PRED) return ARBX_ERR_UNSUPPORTED;
  switch (p.dim) {
    case 2: return count_prealloc_dim<2>(p, a, s);
    case 3: return count_prealloc_dim<3>(p, a, s);
    case 6: return count_prealloc_dim<6>(p, a, s);
  }
  return ARBX_ERR_UNSUPPORTED;
}

arbx_status query_order(const QueryPlan& p, const float* scene_dev, uint32_t** order_out, cudaStream_t s,
                        uint32_t* into) {
  *order_out = nullptr;
  if (p.m <= 1) return ARBX_OK;
  const int D = p.dim;
  // 48-bit codes (six 8-bit sort passes): cells of 2^-16 of the scene in 3D,
  // fine enough to keep the queries of one dense cluster in space order too
  // (10M mixture: 30-bit codes count 10.45 ms, 63-bit 9.7 ms)
  const int bits = D == 2 ? 24 : (D == 3 ? 16 : 8);
  DevTemp<uint64_t> keys(s), keys_alt(s);
  DevTemp<uint32_t> vals_alt(s);
  uint32_t* vals = nullptr;
  ARBX_TRY(keys.alloc(p.m));
  ARBX_TRY(keys_alt.alloc(p.m));
  ARBX_TRY(vals_alt.alloc(p.m));
  if (into) vals = into;
  else ARBX_TRY(dev_alloc_t(&vals, p.m, s));
  auto release = [&]() {
    if (!into) dev_free(vals, s);
  };
  const int grid = (int)((p.m + 255) / 256);
  arbx_status st = ARBX_OK;
  auto go = [&](auto kern) -> arbx_status {
    ARBX_LAUNCH("query_codes", s, kern<<<grid, 256, 0, s>>>(p.qdata, p.m, scene_dev, bits, keys.p, vals));
    return ARBX_OK;
  };
  const int pk = p.pred_kind == ARBX_NEAREST ? ARBX_SPHERE
                 : (p.pred_kind == ARBX_RAY_INTERSECT || p.pred_kind == ARBX_RAY_ORDERED) ? ARBX_RAY_NEAREST
                                                                                          : p.pred_kind;
  switch (pk * 16 + D) {
    case ARBX_SPHERE * 16 + 2: st = go(k_query_codes<2, ARBX_SPHERE>); break;
    case ARBX_SPHERE * 16 + 3: st = go(k_query_codes<3, ARBX_SPHERE>); break;
    case ARBX_SPHERE * 16 + 6: st = go(k_query_codes<6, ARBX_SPHERE>); break;
    case ARBX_BOX_PRED * 16 + 2: st = go(k_query_codes<2, ARBX_BOX_PRED>); break;
    case ARBX_BOX_PRED * 16 + 3: st = go(k_query_codes<3, ARBX_BOX_PRED>); break;
    case ARBX_BOX_PRED * 16 + 6: st = go(k_query_codes<6, ARBX_BOX_PRED>); break;
    case ARBX_RAY_NEAREST * 16 + 3: st = go(k_query_codes<3, ARBX_RAY_NEAREST>); break;
    default: st = ARBX_ERR_UNSUPPORTED;
  }
  if (st != ARBX_OK) {
    release();
    return st;
  }
  bool alt = false;
  st = radix_sort_pairs<uint64_t>(keys.p, vals, keys_alt.p, vals_alt.p, p.m, 0, D * bits, &alt, s);
  if (st != ARBX_OK) {
    release();
    return st;
  }
  if (alt) ARBX_CUDA(cudaMemcpyAsync(vals, vals_alt.p, (size_t)p.m * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
  *order_out = vals;
  return ARBX_OK;
}

}  // namespace arbx
