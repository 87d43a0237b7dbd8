// CPU oracle for the linear-BVH search path: a plain all-pairs brute force.
//
// TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
// baseline leg of the benchmark load this library.  The product path never
// does: it has no CPU fallback.  Nothing here is shared with the CUDA sources
// (no headers, no helpers, no tables).
//
// What it computes (ArborX 2.0, section 2.1 "API v1/v2": a batch of spatial or
// nearest predicates answered with (offsets, indices) in compressed-sparse-row
// form; section 2.2: pure callbacks with early exit; section 2.5: ray nearest):
//
//   radius   R_i = { j : d2(q_i, p_j) <= fl(r_i * r_i) }, listed in ascending j
//   knn      the min(k, n) lexicographically smallest (d2(q_i, p_j), j), ascending
//   box      R_i = { j : for every axis a, lo_i[a] <= hi_j[a] and lo_j[a] <= hi_i[a] }
//            with (lo_j, hi_j) the exact per-axis min/max of primitive j
//   ray      min over j of (t_ij, j) among the Moller-Trumbore hits; miss -> (-1, +inf)
//   count    |R_i|;  count-up-to(n) min(|R_i|, n) stopping at the n-th match;
//            first-hit [|R_i| >= 1]
//
// Floating-point contract (the method is exact, so both sides must round
// identically): every operation is one IEEE binary32 operation, round to
// nearest even, never contracted (build flags -ffp-contract=off, no fast-math;
// x86-64 evaluates float in SSE registers with no excess precision), and
//   dx_a = fl(q_a - p_a),  d2 = fl(...fl(fl(dx_0*dx_0) + fl(dx_1*dx_1)) + ...)
// summed left to right in dimension order.
//
// Readings taken where the paper is silent: the radius boundary is inclusive
// (d2 <= r2) with r2 = fl(r*r); kNN ties go to the lower primitive index; k > n
// gives n results; count-up-to saturates at n; the Moller-Trumbore operation
// order is fixed below; the box predicate against triangles tests the
// triangle's axis-aligned bounding box.
//
// Parity status: every function here is pinned by CPU tests against
// hand-worked cases, closed forms, library routines (scipy) or invariants; see
// tests/test_oracle_pins.py.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <thread>
#include <vector>

namespace {

// Run body(i) for i in [0, m) on nthreads threads (0 = all hardware threads),
// handing out chunks of 16 queries from an atomic counter.
template <class F>
void parallel_for(int64_t m, int nthreads, F body) {
  if (nthreads <= 0) nthreads = (int)std::max(1u, std::thread::hardware_concurrency());
  if (m <= 0) return;
  std::atomic<int64_t> next{0};
  const int64_t chunk = 16;
  auto worker = [&]() {
    for (;;) {
      int64_t s = next.fetch_add(chunk);
      if (s >= m) return;
      int64_t e = std::min(m, s + chunk);
      for (int64_t i = s; i < e; ++i) body(i);
    }
  };
  if (nthreads == 1) { worker(); return; }
  std::vector<std::thread> ts;
  for (int t = 0; t < nthreads; ++t) ts.emplace_back(worker);
  for (auto& t : ts) t.join();
}

// Squared Euclidean distance in the fixed order: differences, squares, then a
// left-to-right sum in dimension order.
inline float sq_dist(const float* q, const float* p, int dim) {
  float dx = q[0] - p[0];
  float acc = dx * dx;
  for (int a = 1; a < dim; ++a) {
    float d = q[a] - p[a];
    float s = d * d;
    acc = acc + s;
  }
  return acc;
}

inline float radius_sq(const float* radii, float radius, int64_t i) {
  float r = radii ? radii[i] : radius;
  return r * r;
}

// Closed interval overlap between the query box (lo, hi: 2*dim floats) and the
// axis-aligned bounding box of primitive j.  For points the box is the point;
// for triangles it is the per-axis min/max of the three vertices.
inline bool box_hits_point(const float* qb, const float* p, int dim) {
  for (int a = 0; a < dim; ++a)
    if (!(qb[a] <= p[a] && p[a] <= qb[dim + a])) return false;
  return true;
}

inline bool box_hits_triangle(const float* qb, const float* t) {
  for (int a = 0; a < 3; ++a) {
    float lo = std::min(std::min(t[a], t[3 + a]), t[6 + a]);
    float hi = std::max(std::max(t[a], t[3 + a]), t[6 + a]);
    if (!(qb[a] <= hi && lo <= qb[3 + a])) return false;
  }
  return true;
}

// Moller & Trumbore (1997), "Fast, minimum storage ray/triangle intersection",
// two-sided, in a fixed operation order:
//   e1 = v1 - v0, e2 = v2 - v0, p = d x e2, det = e1 . p, miss if det == 0,
//   inv = 1/det, s = o - v0, u = (s . p) inv, qv = s x e1, v = (d . qv) inv,
//   t = (e2 . qv) inv, hit iff u >= 0, v >= 0, fl(u + v) <= 1, t >= 0.
// Each cross component is fl(fl(a*b) - fl(c*d)); each dot is summed x, y, z.
inline bool moller_trumbore(const float* o, const float* d, const float* tri, float* t_out) {
  const float* v0 = tri;
  const float* v1 = tri + 3;
  const float* v2 = tri + 6;
  float e1x = v1[0] - v0[0], e1y = v1[1] - v0[1], e1z = v1[2] - v0[2];
  float e2x = v2[0] - v0[0], e2y = v2[1] - v0[1], e2z = v2[2] - v0[2];
  float px = d[1] * e2z - d[2] * e2y;
  float py = d[2] * e2x - d[0] * e2z;
  float pz = d[0] * e2y - d[1] * e2x;
  float det = e1x * px + e1y * py;
  det = det + e1z * pz;
  if (det == 0.0f) return false;
  float inv = 1.0f / det;
  float sx = o[0] - v0[0], sy = o[1] - v0[1], sz = o[2] - v0[2];
  float su = sx * px + sy * py;
  su = su + sz * pz;
  float u = su * inv;
  float qx = sy * e1z - sz * e1y;
  float qy = sz * e1x - sx * e1z;
  float qz = sx * e1y - sy * e1x;
  float sv = d[0] * qx + d[1] * qy;
  sv = sv + d[2] * qz;
  float v = sv * inv;
  float st = e2x * qx + e2y * qy;
  st = st + e2z * qz;
  float t = st * inv;
  if (u >= 0.0f && v >= 0.0f && (u + v) <= 1.0f && t >= 0.0f) {
    *t_out = t;
    return true;
  }
  return false;
}

}  // namespace

extern "C" {

int oracle_abi_version() { return 1; }

float oracle_sq_dist(const float* q, const float* p, int dim) { return sq_dist(q, p, dim); }

int oracle_moller_trumbore(const float* ray6, const float* tri9, float* t) {
  return moller_trumbore(ray6, ray6 + 3, tri9, t) ? 1 : 0;
}

// |R_i| for the sphere predicate (inclusive radius).  radii may be null (then
// the uniform radius applies).
void oracle_radius_count(const float* pts, int64_t n, const float* qs, int64_t m, int dim,
                         const float* radii, float radius, int32_t* counts, int nthreads) {
  parallel_for(m, nthreads, [&](int64_t i) {
    const float* q = qs + i * dim;
    float r2 = radius_sq(radii, radius, i);
    int64_t c = 0;
    for (int64_t j = 0; j < n; ++j) c += (sq_dist(q, pts + j * dim, dim) <= r2) ? 1 : 0;
    counts[i] = (int32_t)c;
  });
}

// CRS fill: indices ascending in j, with their squared distances.
void oracle_radius_fill(const float* pts, int64_t n, const float* qs, int64_t m, int dim,
                        const float* radii, float radius, const int64_t* offsets,
                        int32_t* idx, float* d2, int nthreads) {
  parallel_for(m, nthreads, [&](int64_t i) {
    const float* q = qs + i * dim;
    float r2 = radius_sq(radii, radius, i);
    int64_t w = offsets[i];
    for (int64_t j = 0; j < n; ++j) {
      float e = sq_dist(q, pts + j * dim, dim);
      if (e <= r2) {
        idx[w] = (int32_t)j;
        if (d2) d2[w] = e;
        ++w;
      }
    }
  });
}

// Pure callback "count up to limit": the traversal of query i ends at the
// limit-th match, so the stored count saturates at limit.
void oracle_radius_count_up_to(const float* pts, int64_t n, const float* qs, int64_t m, int dim,
                               const float* radii, float radius, int32_t limit,
                               int32_t* out, int nthreads) {
  parallel_for(m, nthreads, [&](int64_t i) {
    const float* q = qs + i * dim;
    float r2 = radius_sq(radii, radius, i);
    int32_t c = 0;
    for (int64_t j = 0; j < n && c < limit; ++j)
      if (sq_dist(q, pts + j * dim, dim) <= r2) ++c;
    out[i] = c;
  });
}

// k nearest by (d2, j) lexicographic order, ascending; min(k, n) per query.
void oracle_knn(const float* pts, int64_t n, const float* qs, int64_t m, int dim, int k,
                int32_t* idx, float* d2, int nthreads) {
  const int64_t kk = std::min<int64_t>(k, n);
  if (kk <= 0) return;
  parallel_for(m, nthreads, [&](int64_t i) {
    const float* q = qs + i * dim;
    std::vector<float> bd(kk, std::numeric_limits<float>::infinity());
    std::vector<int64_t> bj(kk, std::numeric_limits<int64_t>::max());
    for (int64_t j = 0; j < n; ++j) {
      float e = sq_dist(q, pts + j * dim, dim);
      // accept iff (e, j) < (worst d2, worst j)
      if (e < bd[kk - 1] || (e == bd[kk - 1] && j < bj[kk - 1])) {
        int64_t s = kk - 1;
        while (s > 0 && (e < bd[s - 1] || (e == bd[s - 1] && j < bj[s - 1]))) {
          bd[s] = bd[s - 1];
          bj[s] = bj[s - 1];
          --s;
        }
        bd[s] = e;
        bj[s] = j;
      }
    }
    for (int64_t s = 0; s < kk; ++s) {
      idx[i * kk + s] = (int32_t)bj[s];
      if (d2) d2[i * kk + s] = bd[s];
    }
  });
}

// Box predicate.  kind 0: points float[n][dim]; kind 2: triangles float[n][3][3]
// (dim must be 3).  Query boxes are float[m][2*dim] (lo then hi).
void oracle_box_count(const float* prims, int64_t n, int kind, const float* boxes, int64_t m,
                      int dim, int32_t* counts, int nthreads) {
  parallel_for(m, nthreads, [&](int64_t i) {
    const float* qb = boxes + i * 2 * dim;
    int64_t c = 0;
    for (int64_t j = 0; j < n; ++j)
      c += (kind == 2 ? box_hits_triangle(qb, prims + j * 9) : box_hits_point(qb, prims + j * dim, dim)) ? 1 : 0;
    counts[i] = (int32_t)c;
  });
}

void oracle_box_fill(const float* prims, int64_t n, int kind, const float* boxes, int64_t m,
                     int dim, const int64_t* offsets, int32_t* idx, int nthreads) {
  parallel_for(m, nthreads, [&](int64_t i) {
    const float* qb = boxes + i * 2 * dim;
    int64_t w = offsets[i];
    for (int64_t j = 0; j < n; ++j)
      if (kind == 2 ? box_hits_triangle(qb, prims + j * 9) : box_hits_point(qb, prims + j * dim, dim))
        idx[w++] = (int32_t)j;
  });
}

// Ray nearest hit over triangles float[n][3][3]; rays float[m][6] (origin, dir).
void oracle_ray_nearest(const float* tris, int64_t n, const float* rays, int64_t m,
                        int32_t* hit, float* t_out, int nthreads) {
  parallel_for(m, nthreads, [&](int64_t i) {
    const float* o = rays + i * 6;
    const float* d = o + 3;
    // smallest (t, j) lexicographically; "no hit yet" compares above every index
    const int64_t none = std::numeric_limits<int64_t>::max();
    float best_t = std::numeric_limits<float>::infinity();
    int64_t best_j = none;
    for (int64_t j = 0; j < n; ++j) {
      float t;
      if (moller_trumbore(o, d, tris + j * 9, &t)) {
        if (t < best_t || (t == best_t && j < best_j)) {
          best_t = t;
          best_j = j;
        }
      }
    }
    hit[i] = best_j == none ? -1 : (int32_t)best_j;
    t_out[i] = best_t;
  });
}

// All Moller-Trumbore hits of each ray, ascending (t, j): the ordered-intersect
// predicate; the plain intersect predicate is the same set.
void oracle_ray_all_count(const float* tris, int64_t n, const float* rays, int64_t m,
                          int32_t* counts, int nthreads) {
  parallel_for(m, nthreads, [&](int64_t i) {
    const float* o = rays + i * 6;
    int64_t c = 0;
    for (int64_t j = 0; j < n; ++j) {
      float t;
      c += moller_trumbore(o, o + 3, tris + j * 9, &t) ? 1 : 0;
    }
    counts[i] = (int32_t)c;
  });
}

void oracle_ray_all_fill(const float* tris, int64_t n, const float* rays, int64_t m,
                         const int64_t* offsets, int32_t* idx, float* t_out, int nthreads) {
  parallel_for(m, nthreads, [&](int64_t i) {
    const float* o = rays + i * 6;
    std::vector<std::pair<float, int64_t>> hits;
    for (int64_t j = 0; j < n; ++j) {
      float t;
      if (moller_trumbore(o, o + 3, tris + j * 9, &t)) hits.emplace_back(t, j);
    }
    std::sort(hits.begin(), hits.end());
    int64_t w = offsets[i];
    for (auto& h : hits) {
      idx[w] = (int32_t)h.second;
      t_out[w] = h.first;
      ++w;
    }
  });
}

// DBSCAN (Ester et al. 1996; section 2.4), by the definition: the
// eps-neighbourhood of p is every point q with d2(p, q) <= fl(eps * eps),
// p included; p is a core point when its neighbourhood has at least min_pts
// points; clusters are the connected components of core points under the
// neighbour relation; a non-core point with a core neighbour is a border point
// of that neighbour's cluster.  Labels (a reading: the paper fixes only -1 for
// noise): a cluster's label is the smallest index of its core points; a
// border point takes the smallest label among the clusters of its core
// neighbours; noise is -1.  Returns the number of clusters.
int64_t oracle_dbscan(const float* pts, int64_t n, int dim, float eps, int32_t min_pts, int32_t* labels,
                      int nthreads) {
  const float r2 = eps * eps;
  std::vector<int32_t> count(n);
  parallel_for(n, nthreads, [&](int64_t i) {
    int64_t c = 0;
    for (int64_t j = 0; j < n; ++j) c += sq_dist(pts + i * dim, pts + j * dim, dim) <= r2 ? 1 : 0;
    count[i] = (int32_t)c;
  });
  std::vector<char> core(n);
  for (int64_t i = 0; i < n; ++i) core[i] = count[i] >= min_pts;
  // union-find over core-core neighbour pairs; the root of a set is its
  // smallest index
  std::vector<int64_t> parent(n);
  for (int64_t i = 0; i < n; ++i) parent[i] = i;
  auto find = [&](int64_t x) {
    while (parent[x] != x) x = parent[x];
    return x;
  };
  for (int64_t i = 0; i < n; ++i) {
    if (!core[i]) continue;
    for (int64_t j = i + 1; j < n; ++j) {
      if (!core[j] || sq_dist(pts + i * dim, pts + j * dim, dim) > r2) continue;
      int64_t a = find(i), b = find(j);
      if (a == b) continue;
      if (a < b) parent[b] = a;
      else parent[a] = b;
    }
  }
  int64_t clusters = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (core[i]) {
      labels[i] = (int32_t)find(i);
      clusters += labels[i] == i ? 1 : 0;
    }
  }
  parallel_for(n, nthreads, [&](int64_t i) {
    if (core[i]) return;
    int32_t best = -1;
    for (int64_t j = 0; j < n; ++j) {
      if (!core[j] || sq_dist(pts + i * dim, pts + j * dim, dim) > r2) continue;
      const int32_t l = labels[j];
      if (best < 0 || l < best) best = l;
    }
    labels[i] = best;
  });
  return clusters;
}

}  // extern "C"
