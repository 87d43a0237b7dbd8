// Batched queries against a built tree (see query.cu).
#pragma once

#include "common.cuh"

namespace arbx {

enum SpatialMode : int { MODE_COUNT = 0, MODE_COUNT_UP_TO = 1, MODE_FILL = 2 };

struct QueryPlan {
  TreeView tv;
  int prim_kind = ARBX_POINT;
  int dim = 3;
  bool quantized = false;
  int pred_kind = ARBX_SPHERE;
  const float* qdata = nullptr;
  const float* radii = nullptr;  // per-query radii or null
  float r2 = 0.0f;               // fl(r*r) for a uniform radius
  int64_t m = 0;
  const uint32_t* order = nullptr;  // query processing order (null = input order)
  int block = 256;
  int grid_per_sm = 0;              // 0 = occupancy maximum
  int refill = -1;                  // lane refill: 1 on; 0 or -1 off (refill when the whole warp is done)
  bool stackless = false;           // spatial predicates on float32 nodes: k_spatial_rope
};

// Spatial predicates: MODE_COUNT / MODE_COUNT_UP_TO write counts[m]; MODE_FILL
// writes indices (and d2 when non-null) at the given offsets.
arbx_status run_spatial(const QueryPlan& p, int mode, int32_t limit, int32_t* counts, const int64_t* offsets,
                        int32_t* indices, float* d2, cudaStream_t s);

// Nearest: `kk` = min(k, n) results per query, row-major [m][kk].
arbx_status run_knn(const QueryPlan& p, int k, int kk, int32_t* indices, float* d2, cudaStream_t s);

// Ray nearest hit over a triangle tree.
arbx_status run_ray(const QueryPlan& p, int32_t* hit, float* t, cudaStream_t s);

// Instrumented traversal: adds [node records fetched, leaf records fetched,
// matches] over all queries into stats_dev (unsigned long long[3]).
arbx_status run_stats(const QueryPlan& p, int k, unsigned long long* stats_dev, cudaStream_t s);

// COUNT pass of a spatial predicate with the work counter and error word
// supplied by the caller (both zeroed by the caller, stream-ordered); no device
// allocation happens on this path.
arbx_status run_spatial_count_prealloc(const QueryPlan& p, int32_t* counts, unsigned long long* counter,
                                       uint32_t* err, cudaStream_t s);

// Morton order of the query centres in the scene box (device array of m
// indices, allocated here; release with dev_free).
arbx_status query_order(const QueryPlan& p, const float* scene_dev, uint32_t** order_out, cudaStream_t s);

}  // namespace arbx
