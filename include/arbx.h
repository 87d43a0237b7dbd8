/*
 * arbx.h -- C ABI of a B300-native linear-BVH geometric search library.
 *
 * The library follows the problem statement of ArborX 2.0 (section 2.1, "New
 * interface (API v2)"): build a search index over a set of primitives on an
 * execution space, then answer a batch of predicates against it, returning
 * either the matches in compressed-sparse-row form (offsets, indices) -- the
 * "storage query" (3) and the API v1 form -- or the result of a fixed callback
 * run on every match -- the "pure callback" query (1) of section 2.2, with the
 * early-exit control of the count-up-to-N example.  Index metadata follows the
 * size()/empty()/bounds() members of both API versions.
 *
 * The index is a linear BVH (section 2.6: 64-bit Morton codes, Apetrei's
 * bottom-up construction, vendor-free sorting) built by CUDA kernels for
 * sm_103a.  Every result is exact: neighbour sets and float32 squared
 * distances equal a brute-force search that rounds every operation the same way.
 *
 * Conventions for every entry point
 *  - Pointers named *_dev are device pointers; all others are host pointers.
 *  - Input device buffers are borrowed for the duration of the stream-ordered
 *    work of the call; the tree copies what it keeps.
 *  - Every call runs on the given stream (NULL = the legacy default stream).
 *    Calls that must read a device-computed size (arbx_build, arbx_query_crs)
 *    synchronise the stream before returning; the others are asynchronous and
 *    their results are valid after the stream is synchronised.
 *  - Errors are returned as arbx_status codes; no call aborts the process.
 *    Argument errors are detected on the host before any launch.  Errors found
 *    by kernels (a traversal stack overflow, non-finite primitive
 *    coordinates) set a per-device error word that the next synchronising call
 *    of this library (or arbx_stream_check) returns and clears; the word is
 *    shared by all streams of the device.
 *  - Trees are immutable after arbx_build; any number of queries may run on
 *    the same tree concurrently on different streams (section 2.1, execution
 *    spaces).
 *  - Layouts are row-major float32: points float[n][dim]; boxes float[n][2*dim]
 *    (lo[dim] then hi[dim]); triangles float[n][3][3] (three xyz vertices);
 *    rays float[m][6] (origin xyz, direction xyz).
 */
#ifndef ARBX_H
#define ARBX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t; NULL selects the legacy default stream. */
typedef struct CUstream_st* arbx_stream;

typedef int32_t arbx_status;
#define ARBX_OK                 0
#define ARBX_ERR_INVALID        1  /* bad argument (null pointer, dim, k, radius, kind) */
#define ARBX_ERR_OOM            2  /* device allocation failed */
#define ARBX_ERR_CUDA           3  /* a CUDA runtime call or launch failed */
#define ARBX_ERR_TIMEOUT        4  /* a bounded device wait ran out (reserved for persistent kernels) */
#define ARBX_ERR_STACK_OVERFLOW 5  /* a traversal stack overflowed (cannot happen for valid trees) */
#define ARBX_ERR_UNSUPPORTED    6  /* valid request outside what is built (e.g. k > 256, dim not 2/3/6) */
#define ARBX_ERR_NONFINITE      7  /* a primitive coordinate is NaN or infinite */
#define ARBX_ERR_CAPACITY       8  /* a caller-provided output buffer is too small */
#define ARBX_ERR_BOUNDS         9  /* checked library only: an index read from device memory (a query
                                      order entry, a node or leaf code) lies outside its array, or a
                                      built tree failed its structural check */

/* Primitive kinds (ArborX 2.0, section 1: points, boxes, triangles). */
#define ARBX_POINT    0
#define ARBX_BOX      1
#define ARBX_TRIANGLE 2

/* Predicate kinds.
 *  ARBX_SPHERE      intersects(Sphere(center, r)): d2 <= fl(r*r), inclusive
 *                   (section 2.1 spatial query: a point and a radius).
 *  ARBX_BOX_PRED    intersects(Box): closed overlap with the primitive's
 *                   axis-aligned bounding box (section 2.1).
 *  ARBX_NEAREST     nearest(point, k): the min(k, n) smallest (d2, index)
 *                   pairs, ties by lower index (section 2.1 nearest query).
 *  ARBX_RAY_NEAREST nearest(ray, k): the first k triangle hits, smallest
 *                   (t, index) first (section 2.5; k <= 1 means 1, k <= 32).
 *  ARBX_RAY_INTERSECT intersect(ray): every triangle hit, in left-to-right
 *                   leaf order, with its t (section 2.5).
 *  ARBX_RAY_ORDERED ordered_intersect(ray): every triangle hit, ascending by
 *                   (t, index), the order a ray meets them (section 2.5).
 * Ray predicates: data_dev holds (origin xyz, direction xyz) per ray, dim 3,
 * on triangle trees; a hit is a two-sided Moller-Trumbore intersection with
 * t >= 0 (t may be -0.0; +0 and -0 compare equal in the (t, index) order). */
#define ARBX_SPHERE        0
#define ARBX_BOX_PRED      1
#define ARBX_NEAREST       2
#define ARBX_RAY_NEAREST   3
#define ARBX_RAY_INTERSECT 4
#define ARBX_RAY_ORDERED   5

/* Fixed pure callbacks (section 2.2). */
#define ARBX_CB_COUNT       0  /* out[i] = |R_i| */
#define ARBX_CB_COUNT_UP_TO 1  /* out[i] = min(|R_i|, limit); traversal stops at the limit-th match */
#define ARBX_CB_FIRST_HIT   2  /* out[i] = [|R_i| >= 1]; stops at the first match */

/* Build flags. */
#define ARBX_QUANTIZED_NODES 1u  /* 16-bit child boxes relative to the parent, rounded outward (triangles):
                                   48-byte nodes that keep their own float32 box origin */
#define ARBX_WIDE_NODES      2u  /* also build four-wide records (points, boxes; see arbx_tuning.wide_nodes) */
#define ARBX_PARENT_RELATIVE 4u  /* with ARBX_QUANTIZED_NODES: 32-byte nodes whose child boxes are coded
                                   relative to the node's own box as decoded from its parent's record
                                   (the root's is its exact box); the traversal carries each node's
                                   decoded box on its stack.  Without ARBX_QUANTIZED_NODES:
                                   ARBX_ERR_INVALID. */

typedef struct arbx_tree_t* arbx_tree;

typedef struct {
  int32_t kind;      /* ARBX_POINT, ARBX_BOX or ARBX_TRIANGLE */
  int32_t dim;       /* 2, 3 or 6 for points and boxes; 3 for triangles */
  int64_t n;         /* number of primitives, 0 <= n < 2^30 */
  const float* data_dev;
  uint32_t flags;    /* ARBX_QUANTIZED_NODES, ARBX_WIDE_NODES, ARBX_PARENT_RELATIVE */
} arbx_primitives;

typedef struct {
  int32_t kind;          /* ARBX_SPHERE, ARBX_BOX_PRED, ARBX_NEAREST, ARBX_RAY_* */
  int32_t dim;           /* must equal the tree's dim */
  int64_t m;             /* number of queries, m < 2^31 */
  const float* data_dev; /* centers float[m][dim] | boxes float[m][2*dim] | rays float[m][6] */
  const float* radii_dev;/* ARBX_SPHERE: per-query radii float[m], or NULL to use `radius` */
  float radius;          /* ARBX_SPHERE uniform radius, finite and >= 0 */
  int32_t k;             /* ARBX_NEAREST: 1 <= k <= 256; ARBX_RAY_NEAREST: k <= 32 */
  /* Nullable processing order: a permutation of 0..m-1 (device uint32[m]), for
   * example from arbx_query_order, used instead of sorting the queries again
   * when the call sorts queries (tuning sort_queries; by default whenever an
   * order is given); lets several calls over the same queries share one sort
   * (section 2.6, sorting in search).  Results are written at the original query index, so they are
   * the same bytes with or without it; a buffer that is not a permutation of
   * 0..m-1 gives undefined results (the checked library, libarbx_checked.so,
   * verifies it first and returns ARBX_ERR_BOUNDS without querying).
   * Borrowed for the call. */
  const uint32_t* order_dev;
} arbx_predicates;

/* Compressed-sparse-row result (section 2.1, API v1 "indices and offsets").
 * Query i's matches are indices[offsets[i] .. offsets[i+1]).  Offsets are
 * int64 (the paper's views are int; batches here can exceed 2^31 matches).
 * Order within a query: left-to-right leaf (Morton) order for spatial
 * predicates, ascending (d2, index) for nearest.  d2 holds the float32 squared
 * distance of each match (NULL when not requested, or for box predicates).
 * Buffers returned by arbx_query_crs are owned by the library: release them
 * with arbx_crs_free. */
typedef struct {
  int64_t m;
  int64_t nnz;
  int64_t* offsets_dev;  /* int64[m+1] */
  int32_t* indices_dev;  /* int32[nnz] */
  float* d2_dev;         /* float[nnz] or NULL */
} arbx_crs;

/* Launch tuning; NULL selects the defaults.  Every setting gives identical
 * output bytes; only speed changes.
 *  block        threads per block (64..256, multiple of 32; 0 = default 256)
 *  sort_queries 1 = process queries in Morton order of their centres
 *               (section 2.6: sorting in search), 0 = input order, -1 = default
 *               (by batch size, measured: nearest from 32768 queries,
 *               callbacks and counts from 131072, CRS storage from 524288,
 *               rays always; a caller's pred->order_dev is always used)
 *  top_levels   number of top tree nodes staged in shared memory per block
 *               (0, 255 or 1023; -1 = default: 0 for spatial and nearest
 *               predicates, 255 for rays)
 *  grid_per_sm  resident blocks per SM for the persistent query grid (0 = default)
 *  warp_refill  1 = a lane that finishes its query takes the next one at once;
 *               0 = a warp takes a new group of queries only when all its
 *               lanes are done (keeps neighbouring queries in step);
 *               -1 = default (0)
 *  stackless    spatial predicates on float32 nodes: 1 = stackless traversal
 *               (section 2.6: spatial search by a stackless algorithm; a lane
 *               continues after a subtree covering sorted leaves [l, r] with
 *               the right child of internal node r, no stack), 0 = traversal
 *               with a per-thread stack, -1 = default (0).  Ignored for
 *               nearest, ray and quantized-node queries.
 *  single_pass  arbx_query_crs with spatial predicates: 1 = one traversal
 *               that stages each query's matches (8 slots per query, then
 *               32-slot chunks from a pool sized from a sampled count pass)
 *               followed by a copy into the CRS, queries that outgrow the
 *               pool re-run by the fill pass; 0 = count -> scan -> fill;
 *               -1 = default (0: on a B300 the staging writes and their copy
 *               cost about as much as the second traversal they replace).
 *               Same bytes either way.
 *  lanes_per_query  nearest predicates with k <= 32: 1 = one lane walks a
 *               query with its k-best list in its registers; 2, 4 or 8 = a
 *               group of that many lanes walks one query together, each lane
 *               holding K/L of the list (K = k rounded up to a power of two;
 *               groups larger than K use K lanes); 0 or -1 = default (1).
 *               k > 32: K/32, K/16 or K/8 lanes (32, 16 or 8 keys per lane;
 *               any other value, the default, gives K/16).  Same bytes
 *               either way.
 *  wide_nodes   trees built with ARBX_WIDE_NODES: 1 = the nearest traversal (one lane
 *               per query) and the counting traversals (COUNT, COUNT_UP_TO,
 *               FIRST_HIT, the count pass of the storage query) open
 *               four-wide records -- a binary node's four grandchildren with
 *               their boxes, built with the tree (about 0.45 ms more per 10M
 *               points, twice the node memory) -- so one step descends two
 *               levels; 0 = binary nodes; -1 = default (on for nearest
 *               predicates with 16 < k <= 32, where it measured faster, off
 *               otherwise).  Applies when no top levels are staged and the
 *               traversal is not stackless.  Same bytes either way.
 *  warp_packets nearest predicates, one lane per query, no staged top levels:
 *               1 = the 32 lanes of a warp (32 neighbouring queries of the
 *               processing order) walk one traversal together -- the union of
 *               the nodes they need, one broadcast node load per step, each
 *               lane testing its own query and keeping its own list; 0 = one
 *               traversal per lane; -1 = default (0).  Same bytes either way.
 *  query_runs   nearest predicates without warp packets (one lane per query on
 *               binary or four-wide records, or lane groups): R = 4 or 8 = a
 *               warp of W walkers (32 lanes, or 32/L groups) takes W*R
 *               consecutive queries of the processing order and answers them
 *               in R rounds of W adjacent ones, each walker starting each of
 *               its queries after the first with an upper bound on its k-th
 *               distance carried from its previous one (triangle inequality,
 *               rounded up), so far subtrees are pruned before its list is
 *               full (warp_refill does not apply to them); 1 = one query per
 *               walker, handed out a warp's worth at a time; 0 or -1 = default (in 2D
 *               and 3D 8 for k = 1, else 4; 1 in 6D, where the bound is
 *               loose, and with warp_refill = 1; measured fastest).  Same
 *               bytes either way. */
typedef struct {
  int32_t block;
  int32_t sort_queries;
  int32_t top_levels;
  int32_t grid_per_sm;
  int32_t warp_refill;
  int32_t stackless;
  int32_t single_pass;
  int32_t lanes_per_query;
  int32_t wide_nodes;
  int32_t warp_packets;
  int32_t query_runs;
} arbx_tuning;

/* Human-readable text for a status code (static storage). */
const char* arbx_status_string(arbx_status s);

/* Library ABI version (increments on incompatible changes; 3: arbx_tuning
 * gained query_runs). */
int32_t arbx_abi_version(void);

/* Build variant of the loaded library: ARBX_LIB_CHECKED for the checked
 * library (libarbx_checked.so: the same entry points, results and layouts;
 * every index a kernel reads from device memory is range-checked before it
 * addresses anything -- a bad one is recorded and replaced by 0, and the call
 * returns ARBX_ERR_BOUNDS --, each built tree is walked from its root on the
 * device (every record and leaf reached once, codes in range, float32 parent
 * boxes holding their children) and a caller's query order is checked to be a
 * permutation before any traversal).  0 for the regular library. */
#define ARBX_LIB_CHECKED 1u
uint32_t arbx_library_flags(void);

/* Build a BVH over prim->n primitives (section 2.1: BVH(space, values);
 * section 2.6: Morton codes, sort, Apetrei construction).  *out receives a
 * new tree (or NULL on error).  n == 0 gives an empty tree; n == 1 a tree
 * whose root is its only leaf.  Non-finite coordinates give
 * ARBX_ERR_NONFINITE.  Synchronises the stream before returning. */
arbx_status arbx_build(arbx_tree* out, const arbx_primitives* prim, arbx_stream stream);

/* size(), empty() and bounds() of section 2.1.  size_out (nullable) receives
 * n; dim_out (nullable) the dimension; bounds_out (nullable, host float[2*dim])
 * the scene box lo then hi (for n == 0: +inf then -inf). */
arbx_status arbx_tree_info(arbx_tree tree, int64_t* size_out, int32_t* dim_out, float* bounds_out);

/* Release a tree and its device memory (the caller must not have work
 * using it in flight). NULL is accepted. */
arbx_status arbx_tree_destroy(arbx_tree tree);

/* Storage query (section 2.1, query form (3) and API v1): all matches of each
 * predicate as CRS with library-allocated buffers.  want_d2 != 0 also returns
 * squared distances (sphere and nearest predicates) or the hit distances t
 * (ray predicates; for ARBX_RAY_NEAREST a row holds the hits found, at most
 * k).  Synchronises the stream once (to size the output) and again at the
 * end. */
arbx_status arbx_query_crs(arbx_tree tree, const arbx_predicates* pred, int32_t want_d2,
                           const arbx_tuning* tuning, arbx_crs* out, arbx_stream stream);

/* Storage query whose results go to host memory, for result sets larger
 * than the device can hold (section 2.1 notes that results may not fit in
 * memory; this is the storing form for that case).  A count pass over all
 * queries gives the global int64 offsets, written to offsets_host (int64[m+1];
 * *nnz_out, nullable, receives offsets[m]); then the queries are filled in
 * consecutive ranges whose results fit the chunk budget -- chunk_bytes, or
 * when 0 half of the device memory available at the call less 1 GiB -- each
 * range's segment copied to indices_host[offsets[lo] ..] (and d2_host, when
 * want_d2 and non-NULL: d2 for spheres, t for rays) before the next range
 * reuses the device buffers.  A single query larger than the budget is filled
 * on its own.  The bytes are those of arbx_query_crs.  Spatial and ray
 * intersect predicates.  capacity: entries of indices_host (and d2_host);
 * when nnz exceeds it the offsets are written and ARBX_ERR_CAPACITY returned
 * before any fill.  Host buffers may be pageable or pinned.  Synchronous. */
arbx_status arbx_query_crs_host(arbx_tree tree, const arbx_predicates* pred, int32_t want_d2,
                                const arbx_tuning* tuning, int64_t* offsets_host, int32_t* indices_host,
                                float* d2_host, int64_t capacity, int64_t chunk_bytes, int64_t* nnz_out,
                                arbx_stream stream);

/* Release the buffers of a CRS returned by arbx_query_crs (stream-ordered on
 * `stream`) and zero the struct. */
arbx_status arbx_crs_free(arbx_crs* crs, arbx_stream stream);

/* Pure-callback query (section 2.2, query form (1)): runs the fixed callback
 * `cb` on every match and stores nothing else.  out_dev: caller-owned device
 * int32[m].  limit: the N of ARBX_CB_COUNT_UP_TO (>= 0; ignored otherwise).
 * Spatial predicates (ARBX_SPHERE, ARBX_BOX_PRED) and the ray intersect
 * predicates (ARBX_RAY_INTERSECT, ARBX_RAY_ORDERED: hits are counted).
 * Asynchronous. */
arbx_status arbx_query_callback(arbx_tree tree, const arbx_predicates* pred, int32_t cb,
                                int32_t limit, int32_t* out_dev, const arbx_tuning* tuning,
                                arbx_stream stream);

/* Two-phase storage query into caller-owned buffers.  Phase 1 writes
 * offsets_dev[0..m] (int64, exclusive scan of the per-query counts; the total
 * is offsets_dev[m]).  Phase 2 fills indices_dev[offsets[i]..offsets[i+1])
 * (and d2_dev when non-NULL: squared distances, or t for rays) given those
 * offsets.  Spatial and ray intersect predicates (ARBX_RAY_ORDERED sorts
 * each segment by (t, index) after the fill, with temporaries of its own).
 * Both are asynchronous; phase 2 must see the same predicates and tree. */
arbx_status arbx_query_offsets(arbx_tree tree, const arbx_predicates* pred,
                               const arbx_tuning* tuning, int64_t* offsets_dev, arbx_stream stream);
arbx_status arbx_query_fill(arbx_tree tree, const arbx_predicates* pred, const arbx_tuning* tuning,
                            const int64_t* offsets_dev, int32_t* indices_dev, float* d2_dev,
                            arbx_stream stream);

/* Nearest query into caller-owned buffers (section 2.1, nearest(point, k)):
 * indices_dev int32[m][kk] and d2_dev float[m][kk] (nullable) with
 * kk = min(k, n), each row ascending by (d2, index).  1 <= k <= 256 (a list of
 * up to 32 keys is held by one lane, a longer one by a lane group; see
 * arbx_tuning.lanes_per_query).  Asynchronous. */
arbx_status arbx_query_knn(arbx_tree tree, const arbx_predicates* pred, const arbx_tuning* tuning,
                           int32_t* indices_dev, float* d2_dev, arbx_stream stream);

/* Ray nearest-hit query (section 2.5, nearest(ray, k)) on a triangle tree:
 * hit_dev int32[m][kk] (triangle indices, -1 past the last hit) and t_dev
 * float[m][kk] (+inf past the last hit) with kk = max(1, pred->k), each row
 * the kk smallest (t, index) over Moller-Trumbore hits with t >= 0.
 * pred->kind must be ARBX_RAY_NEAREST.  Asynchronous. */
arbx_status arbx_query_ray_nearest(arbx_tree tree, const arbx_predicates* pred,
                                   const arbx_tuning* tuning, int32_t* hit_dev, float* t_dev,
                                   arbx_stream stream);

/* Instrumented traversal, for measurement only: runs the traversal of `pred`
 * with counters and no output, and writes to stats_host (int64[3]) the totals
 * over all queries of [internal node records fetched, leaf records fetched
 * (triangle leaves; point leaves live inside their parent node), matches].
 * Multiplied by the record sizes these give the algorithmic bytes the
 * traversal moves.  For nearest predicates only the node count is filled.
 * Synchronous. */
arbx_status arbx_query_stats(arbx_tree tree, const arbx_predicates* pred, const arbx_tuning* tuning,
                             int64_t* stats_host, arbx_stream stream);

/* The visit counters of a sphere walk whose squared radii are given per query
 * (r2_dev: device float[m], used as is, no fl(r*r)): [node records fetched,
 * 0, matches], walking every record whose box distance is <= r2 (no
 * contained-subtree rule), over the records the nearest traversal of the same
 * tuning opens (four-wide records with wide_nodes on, else binary nodes).
 * Given the final k-th squared distances of a nearest query (the last column
 * of its d2 rows; +inf when k > n), the count is the set any exact best-first
 * search over those records must open -- the records whose box lies within
 * the k-th distance (section 2.1 nearest predicates) -- the algorithmic node
 * traffic of that query.  pred: ARBX_SPHERE on a point or box tree (radius
 * and radii_dev are ignored).  Synchronous. */
arbx_status arbx_query_stats_r2(arbx_tree tree, const arbx_predicates* pred, const arbx_tuning* tuning,
                                const float* r2_dev, int64_t* stats_host, arbx_stream stream);

/* The processing order the library would use for these predicates: the
 * queries sorted by the Morton code of their centre (point, box centre, ray
 * origin) in the tree's scene box (section 2.6, sorting in search), written to
 * order_dev (caller-owned device uint32[m]).  Pass it as pred->order_dev to
 * later calls over the same queries to sort them once.  Asynchronous. */
arbx_status arbx_query_order(arbx_tree tree, const arbx_predicates* pred, uint32_t* order_dev,
                             arbx_stream stream);

/* The same counters for the counting traversal of a spatial predicate (ARBX_SPHERE
 * or ARBX_BOX_PRED), as arbx_query_count, arbx_query_count_up_to and the count
 * pass of arbx_query_crs walk the tree: on trees of points or triangles, an
 * internal child whose box lies wholly inside the predicate's region adds its
 * leaf count without being visited.  Matches are the count pass's total (equal
 * to arbx_query_stats's).  Other predicate kinds: ARBX_ERR_INVALID.  Synchronous. */
arbx_status arbx_query_count_stats(arbx_tree tree, const arbx_predicates* pred, const arbx_tuning* tuning,
                                   int64_t* stats_host, arbx_stream stream);

/* ---------------------------------------------------------------- forests
 * Batches of independent point sets, each with its own BVH (the per-set form
 * of section 2.1's BVH), built and queried together: one batched build per
 * dimension, one persistent kernel per predicate over all sets.  Set s holds
 * counts[s] points of dims[s] floats (dims 2, 3 or 6, at most 4096 sets per
 * dimension); the sets are packed one after another in data_dev.  Indices in
 * results are set-local.  arbx_forest_build synchronises the stream. */
typedef struct arbx_forest_t* arbx_forest;
typedef struct arbx_forest_batch_t* arbx_forest_batch;
typedef struct arbx_graph_t* arbx_graph;

arbx_status arbx_forest_build(arbx_forest* out, int32_t nsets, const int32_t* dims_host, const int64_t* counts_host,
                              const float* data_dev, arbx_stream stream);
arbx_status arbx_forest_destroy(arbx_forest f);
arbx_status arbx_forest_info(arbx_forest f, int32_t* nsets_out, int64_t* points_out);

/* A query batch for a forest: set s gets qcounts_host[s] queries (packed set
 * after set in the query buffer, dims[s] floats each; global query ids follow
 * that order) and radius radii_host[s] (nullable: no radius queries).  The
 * batch uploads this layout and owns every temporary, so the query calls
 * below only enqueue device work.  Synchronous. */
arbx_status arbx_forest_batch_create(arbx_forest_batch* out, arbx_forest f, const int64_t* qcounts_host,
                                     const float* radii_host, arbx_stream stream);
arbx_status arbx_forest_batch_destroy(arbx_forest_batch b);
arbx_status arbx_forest_batch_total(arbx_forest_batch b, int64_t* total_queries);

/* Radius storage query over all sets: offsets_dev int64[M+1] over the global
 * query ids (count, then scan), then the fill of indices_dev/d2_dev (capacity
 * entries each; capacity 0 skips the fill).  nnz_dev (nullable, device int64)
 * receives offsets[M]; when it exceeds the capacity the fill wrote only the
 * entries below the capacity and must be re-run with larger buffers.
 * Asynchronous; allocates nothing (the batch holds the temporaries). */
arbx_status arbx_forest_query_radius(arbx_forest_batch b, const float* queries_dev, int64_t* offsets_dev,
                                     int32_t* indices_dev, float* d2_dev, int64_t capacity, int64_t* nnz_dev,
                                     arbx_stream stream);
/* Nearest query over all sets: rows of stride k in indices_dev int32[M][k] and
 * d2_dev float[M][k] (nullable), ascending (d2, index); entries beyond the
 * set's size are (-1, +inf).  1 <= k <= 32.  Asynchronous. */
arbx_status arbx_forest_query_knn(arbx_forest_batch b, const float* queries_dev, int32_t k, int32_t* indices_dev,
                                  float* d2_dev, arbx_stream stream);
/* Capture the radius query (count, scan, fill) and, when k > 0, the nearest
 * query of a batch into one executable CUDA graph on `stream` (a non-default
 * stream); arbx_graph_launch replays the whole sequence with one launch. */
arbx_status arbx_forest_graph_create(arbx_graph* out, arbx_forest_batch b, const float* queries_dev,
                                     int64_t* offsets_dev, int32_t* indices_dev, float* d2_dev, int64_t capacity,
                                     int64_t* nnz_dev, int32_t k, int32_t* knn_idx_dev, float* knn_d2_dev,
                                     arbx_stream stream);
arbx_status arbx_graph_launch(arbx_graph g, arbx_stream stream);

/* Launch settings of a batch's query kernels (the batched form of
 * arbx_tuning; every setting gives the same bytes, only speed changes):
 *  block            threads per block of the persistent query kernels: 128 or
 *                   256 (0 = 256)
 *  chunk            query slots a warp takes from the work counter at a time:
 *                   32 or 64 (0 = 32)
 *  sort_queries[g]  dimension group g (dims 2, 3, 6): 1 = each call orders the
 *                   group's queries set by set in Morton order of the set's
 *                   frame (section 2.6, sorting in search), 0 = input order,
 *                   -1 = default (1)
 * A new batch takes the setting recorded by arbx_forest_autotune for its key
 * (GPU model, dimension groups present, floor(log4) of its query count), else
 * the defaults.  A graph captured by arbx_forest_graph_create keeps the
 * setting the batch had at capture. */
typedef struct {
  int32_t block;
  int32_t chunk;
  int32_t sort_queries[3];
} arbx_forest_tuning;

/* Set (NULL: the defaults) or read a batch's launch settings.  Invalid
 * values give ARBX_ERR_INVALID and leave the batch unchanged. */
arbx_status arbx_forest_batch_set_tuning(arbx_forest_batch b, const arbx_forest_tuning* tuning);
arbx_status arbx_forest_batch_get_tuning(arbx_forest_batch b, arbx_forest_tuning* out);

/* Launch-setting search for a batch: times the radius query (count, scan,
 * fill) plus, when k > 0, the nearest query (k <= 32) on the batch's own
 * queries with CUDA events (second of two runs), first trying each dimension
 * group's query ordering off, then block 128/256 x chunk 32/64, and keeps the
 * fastest: it becomes the batch's setting, is written to *best_out (and its
 * time in ms to *best_ms_out, nullable), and is recorded for new batches with
 * the same key (arbx_autotune_save / _load / _clear cover these records too,
 * as lines starting with "forest").  Allocates temporaries for the outputs.
 * Synchronous. */
arbx_status arbx_forest_autotune(arbx_forest_batch b, const float* queries_dev, int32_t k,
                                 arbx_forest_tuning* best_out, double* best_ms_out, arbx_stream stream);
arbx_status arbx_graph_destroy(arbx_graph g);

/* ---------------------------------------------------------------- serving
 * A request loop over resident trees (section 2.1: queries on execution
 * spaces run concurrently).  `slots` worker threads, each with its own CUDA
 * stream, take requests from one FIFO queue; the queue head starts when a slot
 * is free and its device-memory estimate fits beside the running requests'
 * reservations within min(hbm_budget_bytes, the device memory available when
 * the server is created) and also fits the device memory available at that
 * moment (cudaMemGetInfo's free memory plus the unused part of the default
 * stream-ordered pool, less a 1 GiB reserve); a radius request reserves its
 * output after its count pass.  Requests that arrive while others run are
 * admitted as slots and memory free up and their work overlaps on the device.
 * When every running request waits for memory the oldest proceeds anyway (no
 * deadlock); an allocation that then fails ends that request with
 * ARBX_ERR_OOM and the server keeps serving.  Results stay in device memory
 * until arbx_server_release. */
typedef struct arbx_server_t* arbx_server;

typedef struct {
  int32_t tree_id;
  int32_t kind;          /* ARBX_SPHERE or ARBX_NEAREST; with a callback also ARBX_BOX_PRED */
  int32_t callback;      /* -1: storage query; ARBX_CB_COUNT / _COUNT_UP_TO / _FIRST_HIT: counts */
  int32_t limit;         /* ARBX_CB_COUNT_UP_TO limit */
  int32_t k;             /* ARBX_NEAREST */
  float radius;          /* ARBX_SPHERE */
  int64_t m;
  const float* queries_dev;  /* borrowed until the request completes */
  double arrival_s;      /* arrival time on the server clock (arbx_server_now); < 0: at submission */
} arbx_request;

typedef struct {
  arbx_status status;
  int64_t m;
  int64_t nnz;
  int64_t* offsets_dev;  /* storage queries: CRS (nearest: rows of min(k, n)) */
  int32_t* indices_dev;
  float* d2_dev;
  int32_t* counts_dev;   /* callback requests: int32[m] */
  double latency_s;      /* completion of the device work minus arrival */
} arbx_result;

arbx_status arbx_server_create(arbx_server* out, int32_t slots, int64_t hbm_budget_bytes);
/* The server takes ownership of the tree (destroyed with the server). */
arbx_status arbx_server_add_tree(arbx_server s, arbx_tree tree, int32_t* tree_id);
/* Seconds since the server was created (the clock of arrival_s). */
double arbx_server_now(arbx_server s);
arbx_status arbx_server_submit(arbx_server s, const arbx_request* req, uint64_t* ticket);
/* Wait for a request (timeout_us < 0: no limit; ARBX_ERR_TIMEOUT when it
 * runs out) and take its result; returns the request's status. */
arbx_status arbx_server_wait(arbx_server s, uint64_t ticket, int64_t timeout_us, arbx_result* out);
/* Free the device buffers of a result. */
arbx_status arbx_server_release(arbx_server s, arbx_result* r);
/* Latency percentiles (seconds) and throughput (queries from the first
 * arrival to the last completion) of the requests completed since creation
 * or the last reset. */
arbx_status arbx_server_stats(arbx_server s, double* p50_s, double* p99_s, double* mqps, int64_t* completed);
arbx_status arbx_server_reset_stats(arbx_server s);
/* Finish queued and running requests, then free everything. */
arbx_status arbx_server_destroy(arbx_server s);

/* The paper has no counterpart to this entry point.  It is arbx_query_offsets
 * for callers that cannot allocate device memory while it runs: a process whose
 * device memory belongs to another allocator or budget, a latency-critical path
 * where an allocation could synchronise the device, or work captured into a
 * CUDA graph in a mode that forbids allocation.  It allocates nothing: its
 * per-query counts, scan temporaries, work counter and error word live in a
 * fixed device array built into the library (about 4 MiB, held by every GPU
 * that loads the library until the process exits).
 *  - Limit: pred->m <= ARBX_NOALLOC_MAX_QUERIES, else ARBX_ERR_CAPACITY.
 *    Spatial predicates only (ARBX_SPHERE, ARBX_BOX_PRED).
 *  - offsets_dev: caller-owned device int64[m+1], written as by
 *    arbx_query_offsets (same bytes; queries are processed in input order).
 *  - error_dev: nullable caller-owned device uint32; receives 0, or nonzero
 *    when a kernel detected a fault (a traversal stack overflow, which a tree
 *    built by arbx_build cannot produce).
 *  - Asynchronous on `stream`.  The first call on a device looks up the
 *    array's device address (a CUDA runtime query) and caches it; make that
 *    first call before any stream capture.
 *  - Every call on a device uses the same array: calls whose work overlaps on
 *    the GPU (other streams or threads) race and must be serialised.  Each call
 *    clears what must start at zero and overwrites the rest. */
#define ARBX_NOALLOC_MAX_QUERIES (1 << 20)
arbx_status arbx_query_offsets_noalloc(arbx_tree tree, const arbx_predicates* pred, int64_t* offsets_dev,
                                       uint32_t* error_dev, arbx_stream stream);

/* Synchronise `stream` and return (and clear) the device error word. */
arbx_status arbx_stream_check(arbx_stream stream);

/* Copy the tree's internal arrays to host memory for inspection.  Each
 * (buffer, capacity-in-bytes) pair is optional (NULL skips it); bytes_out
 * (nullable, int64[5]) receives [node bytes, leaf bytes, node stride, leaf
 * stride, root index].  Internal node g is the node whose split lies between
 * sorted leaves g and g+1.  Synchronous. */
arbx_status arbx_tree_export(arbx_tree tree, void* nodes_host, int64_t nodes_cap,
                             void* leaves_host, int64_t leaves_cap, int64_t* bytes_out);

/* Kernel instrumentation.  arbx_profile_enable(1) makes every subsequent
 * launch of this library record CUDA events on its stream; arbx_profile_read
 * synchronises the recorded events and writes, for up to `cap` kernel names,
 * the name (host char[cap][64]), launch count and total device milliseconds,
 * returning the number of names in *count_out; arbx_profile_reset clears the
 * record.  arbx_launch_count returns the number of kernels this library has
 * launched since load. */
arbx_status arbx_profile_enable(int32_t on);
arbx_status arbx_profile_read(char* names_host, int64_t* launches_host, double* ms_host,
                              int32_t cap, int32_t* count_out);
arbx_status arbx_profile_reset(void);
int64_t arbx_launch_count(void);

/* Device memory: the library allocates from the current device's default
 * stream-ordered pool and keeps up to ARBX_POOL_RELEASE_GB (environment,
 * default 32) GiB of freed blocks cached for later calls.  arbx_memory_trim
 * synchronises the device and returns cached blocks to the driver until at
 * most keep_bytes remain reserved (0: all unused blocks). */
arbx_status arbx_memory_trim(int64_t keep_bytes);

/* Fault injection on the host, for tests: after `after` more successful
 * device allocations by the library, the next `count` allocations fail with
 * ARBX_ERR_OOM (count 0 turns it off).  Every entry point must then return an
 * error status, leave no work in flight that uses freed memory, and work
 * again once allocations succeed. */
arbx_status arbx_debug_fail_allocs(int64_t after, int64_t count);

/* DBSCAN (section 2.4: ArborX::dbscan(exec, points, eps, minPts)), the
 * FDBSCAN way: a BVH over the points, a COUNT_UP_TO(min_pts) pass for the core
 * points (a point's eps-neighbourhood, d2 <= fl(eps*eps) with the library's
 * distance contract, includes the point itself), one radius traversal per core
 * point that merges core neighbours in a lock-free union-find, and one per
 * non-core point for border labels.
 *  - points_dev: device float[n][dim], dim 2, 3 or 6; eps finite >= 0;
 *    min_pts <= 1 makes every point core.
 *  - labels_dev: device int32[n] (caller-owned): -1 for noise; otherwise the
 *    smallest index of a core point of the cluster (the paper fixes only -1;
 *    this choice makes labels independent of timing).  A border point takes
 *    the smallest label among its core neighbours' clusters.
 *  - n_clusters_out: nullable host int64, the number of clusters.
 *  - Synchronises the stream; builds and frees its own tree. */
arbx_status arbx_dbscan(const float* points_dev, int64_t n, int32_t dim, float eps, int32_t min_pts,
                        int32_t* labels_dev, int64_t* n_clusters_out, arbx_stream stream);

/* Launch-setting search.  The paper's queries run on an execution space whose
 * launch shape the backend picks (section 2.1, "Lack of execution spaces");
 * here block size, query ordering, staged top levels and lane refill (the
 * fields of arbx_tuning) are chosen by measurement.
 * arbx_autotune runs each candidate setting (block 128/256, query sort off/on,
 * top levels 0/255/1023, refill off/on, for spatial predicates on float32
 * nodes stackless off/on, for nearest predicates lanes per query 1/2/4/8 (at
 * most the list size; k > 32: K/32, K/16, K/8), wide nodes off/on where they
 * apply (no staged top levels, not stackless, one lane per query), warp packets
 * off/on for nearest predicates; grid_per_sm 0; single_pass is not
 * searched and keeps its default; pred->order_dev is ignored) twice on the
 * first min(pred->m, sample) predicates (sample <= 0: 2^20) of `pred` --
 * ordering plus the storage query's count, scan and fill passes for spatial
 * predicates, the k-nearest kernel for ARBX_NEAREST, the nearest-hit kernel
 * for rays -- times the second run with CUDA events on `stream`, times the
 * four fastest three more times each, writes the one with the smallest median
 * to *best_out (and that median in ms to *best_ms_out, nullable), and records it for the key (GPU model,
 * predicate kind, dim, k, floor(log2 n), floor(log4 m), node format).  Every
 * later query call given tuning == NULL whose key has a record uses it.
 * Synchronous; allocates temporaries for the sample's outputs.  Results of
 * every query are the same bytes under every setting; only time differs.
 * arbx_autotune_save / _load write / merge the records as a text file (one
 * line per key; lines with an invalid setting are skipped); ARBX_ERR_INVALID
 * when the file cannot be opened.  arbx_autotune_clear drops every record. */
arbx_status arbx_autotune(arbx_tree tree, const arbx_predicates* pred, int64_t sample, arbx_tuning* best_out,
                          double* best_ms_out, arbx_stream stream);
arbx_status arbx_autotune_save(const char* path);
arbx_status arbx_autotune_load(const char* path);
arbx_status arbx_autotune_clear(void);

#ifdef __cplusplus
}
#endif

#endif /* ARBX_H */
