// Batched queries against a built tree (see query.cu).
#pragma once

#include "common.cuh"

namespace arbx {

enum SpatialMode : int { MODE_COUNT = 0, MODE_COUNT_UP_TO = 1, MODE_FILL = 2, MODE_SINGLE = 3 };

// Single-pass storage (MODE_SINGLE): each query's matches, in leaf order, go
// to SINGLE_INLINE slots of its own and then to chunks of SINGLE_CHUNK slots
// taken from a shared pool and linked per query; counts[] receives the full
// match counts.  A query that finds the pool exhausted is appended to
// ovf_list and its later matches are dropped (it is re-run by the fill pass).
constexpr int SINGLE_INLINE = 8;
constexpr int SINGLE_CHUNK = 32;
struct SingleStore {
  int32_t* in_idx = nullptr;  // [m][SINGLE_INLINE]
  float* in_d2 = nullptr;     // same, or null
  int32_t* pool_idx = nullptr;  // [pool_chunks][SINGLE_CHUNK]
  float* pool_d2 = nullptr;
  int32_t* next = nullptr;      // [pool_chunks]: the query's next chunk
  int32_t* head = nullptr;      // [m]: the query's first chunk
  unsigned long long* pool_counter = nullptr;  // chunks taken (zeroed by the caller)
  int64_t pool_chunks = 0;
  int32_t* ovf_list = nullptr;                 // [m]
  unsigned long long* ovf_counter = nullptr;   // zeroed by the caller
};

struct QueryPlan {
  TreeView tv;
  int prim_kind = ARBX_POINT;
  int dim = 3;
  bool quantized = false;         // 16-bit nodes (QNode, or PNode when prel)
  bool prel = false;              // parent-relative 32-byte nodes
  int pred_kind = ARBX_SPHERE;
  const float* qdata = nullptr;
  const float* radii = nullptr;  // per-query radii or null
  float r2 = 0.0f;               // fl(r*r) for a uniform radius
  int64_t m = 0;
  const uint32_t* order = nullptr;  // query processing order (null = input order)
  int64_t nq = 0;                   // queries in qdata when `order` lists a subset of them (0: m)
  int block = 256;
  int grid_per_sm = 0;              // 0 = occupancy maximum
  int refill = -1;                  // lane refill: 1 on; 0 or -1 off (refill when the whole warp is done)
  bool stackless = false;           // spatial predicates on float32 nodes: k_spatial_rope
  bool single_pass = false;         // storage queries: one staged traversal (host-side choice)
  int lanes = 1;                    // nearest predicates: lanes per query (1, 2, 4, 8; longer lists fix their own)
  bool wide = false;                // nearest and counting traversals over the four-wide records (tv.wide)
  bool packets = false;             // one traversal per warp for its 32 queries
  int knn_run = 1;                  // nearest, one lane per query: adjacent queries per lane run (1, 4, 8)
};

// Largest k of nearest(point, k): lists up to 32 keys live in one lane's
// registers, longer ones are spread over a lane group (8 keys per lane).
constexpr int KNN_MAX_K = 256;

// Spatial predicates: MODE_COUNT / MODE_COUNT_UP_TO write counts[m]; MODE_FILL
// writes indices (and d2 when non-null) at the given offsets.
arbx_status run_spatial(const QueryPlan& p, int mode, int32_t limit, int32_t* counts, const int64_t* offsets,
                        int32_t* indices, float* d2, cudaStream_t s);

// MODE_SINGLE traversal into `store` (counts[m] receives every query's count).
arbx_status run_spatial_single(const QueryPlan& p, const SingleStore& store, int32_t* counts, cudaStream_t s);

// Copy single-pass storage into CRS at `offsets` (queries in the overflow
// list are skipped: their segments come from the fill pass).
arbx_status single_compact(const SingleStore& store, const int32_t* counts, const int64_t* offsets, int64_t m,
                           uint64_t n_overflow, int32_t* indices, float* d2, cudaStream_t s);

// Chunks a SingleStore needs for the queries listed in sample[0..ns) given
// their counts, summed into *need_dev (zeroed by the caller).
arbx_status single_chunks_needed(const uint32_t* sample, int64_t ns, const int32_t* counts,
                                 unsigned long long* need_dev, cudaStream_t s);

// FDBSCAN phases over a plan whose queries are the tree's own points and
// whose uniform radius is eps.  counts[i] = min(|N_eps(i)|, min_pts) (the
// COUNT_UP_TO pass); core iff counts[i] >= min_pts.  Writes labels[n] (the
// smallest core index of the cluster, border points the smallest label among
// their core neighbours, -1 for noise) and the number of clusters.
arbx_status run_dbscan(const QueryPlan& p, const int32_t* counts, int32_t min_pts, int32_t* labels,
                       int64_t* n_clusters, cudaStream_t s);

// Nearest: `kk` = min(k, n) results per query, row-major [m][kk].
arbx_status run_knn(const QueryPlan& p, int k, int kk, int32_t* indices, float* d2, cudaStream_t s);

// Ray nearest over a triangle tree: the max(1, k) first hits per ray, rows of
// hit[m][kk] / t[m][kk] (either nullable), padded with -1 / +inf.
arbx_status run_ray(const QueryPlan& p, int k, int32_t* hit, float* t, cudaStream_t s);

// Sort each CRS segment [offsets[i], offsets[i+1]) of (idx, t) ascending by
// (t, index), +0 and -0 equal (ordered_intersect); t keeps its bits.
arbx_status sort_segments_by_t(const int64_t* offsets, int64_t m, int64_t nnz, int32_t* idx, float* t,
                               cudaStream_t s);

// Instrumented traversal: adds [node records fetched, leaf records fetched,
// matches] over all queries into stats_dev (unsigned long long[3]).
// counting: spatial predicates walk the tree as the count pass does
// (contained subtrees counted whole)
// r2s (sphere predicates on point or box trees): per-query squared radii taken
// as given, walked without the contained-subtree rule
arbx_status run_stats(const QueryPlan& p, int k, unsigned long long* stats_dev, cudaStream_t s,
                      bool counting = false, const float* r2s = nullptr);

// COUNT pass of a spatial predicate with the work counter and error word
// supplied by the caller (both zeroed by the caller, stream-ordered); no device
// allocation happens on this path.
arbx_status run_spatial_count_prealloc(const QueryPlan& p, int32_t* counts, unsigned long long* counter,
                                       uint32_t* err, cudaStream_t s);

// Morton order of the query centres in the scene box (device array of m
// indices, allocated here and released with dev_free, or written into `into`
// when it is given).
arbx_status query_order(const QueryPlan& p, const float* scene_dev, uint32_t** order_out, cudaStream_t s,
                        uint32_t* into = nullptr);

}  // namespace arbx
