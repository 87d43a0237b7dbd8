// Internal declarations shared by the CUDA translation units of libarbx.
//
// Exactness contract (ArborX 2.0 returns exact neighbour sets; this library
// additionally returns bit-exact float32 squared distances): every distance
// is formed as dx_a = fl(q_a - p_a), s_a = fl(dx_a * dx_a) and a left-to-right
// fl-sum over the axes, with the _rn intrinsics so that no multiply-add is
// ever contracted (the files are also compiled with -fmad=false).
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <cstdio>

#include "arbx.h"

// Checked build (compiled with -DARBX_CHECKED=1 into libarbx_checked.so): every
// index a kernel reads from device memory -- a node or leaf code, a query
// order entry -- is range-checked before it addresses anything; a bad one is
// recorded in the error word (ARBX_ERR_BOUNDS) and replaced by 0, so no access
// leaves its array.  Trees are validated on the device after each build and a
// caller's query order before each query.  The regular build compiles the
// checks away.
#ifndef ARBX_CHECKED
#define ARBX_CHECKED 0
#endif

namespace arbx {

constexpr bool CHECKED = ARBX_CHECKED != 0;

// ------------------------------------------------------------------ status

arbx_status cuda_status(cudaError_t e, const char* what, const char* file, int line);

#define ARBX_CUDA(expr)                                                         \
  do {                                                                          \
    cudaError_t _e = (expr);                                                    \
    if (_e != cudaSuccess) return ::arbx::cuda_status(_e, #expr, __FILE__, __LINE__); \
  } while (0)

#define ARBX_TRY(expr)                       \
  do {                                       \
    arbx_status _s = (expr);                 \
    if (_s != ARBX_OK) return _s;            \
  } while (0)

// Bits of the per-device error word written by kernels.
enum : uint32_t {
  DEVERR_STACK = 1u,
  DEVERR_NONFINITE = 2u,
  DEVERR_TIMEOUT = 4u,
  DEVERR_INTERNAL = 8u,  // a build invariant failed (e.g. a quantized box does not contain its child)
  DEVERR_BOUNDS = 16u,   // checked builds: an index read from device memory was out of range
  // with DEVERR_BOUNDS, which kind of index it was
  BAD_ORDER = 1u << 8,   // a query order entry
  BAD_NODE = 1u << 9,    // an internal node code
  BAD_TOP = 1u << 10,    // a code into the staged top levels
  BAD_LEAF = 1u << 11,   // a sorted leaf position
  BAD_TREE = 1u << 12,   // the structural walk of a built tree
};

// i itself in regular builds; in checked builds i when it lies in [0, n),
// else 0 with DEVERR_BOUNDS recorded in *err.
__device__ __forceinline__ int64_t checked_index(int64_t i, int64_t n, uint32_t* err, uint32_t what = 0) {
  if constexpr (CHECKED) {
    if ((uint64_t)i >= (uint64_t)n) {
      atomicOr(err, DEVERR_BOUNDS | what);
      return 0;
    }
  }
  return i;
}

// Query at position `slot` of a processing order (null: input order).
__device__ __forceinline__ int64_t query_at(const uint32_t* __restrict__ order, int64_t slot, int64_t m,
                                            uint32_t* err) {
  return order ? checked_index((int64_t)order[slot], m, err, BAD_ORDER) : slot;
}

// Device error word of the current device (allocated on first use).
arbx_status device_error_word(uint32_t** out);
// Synchronise `s`, then read and clear the error word of the current device.
arbx_status check_stream(cudaStream_t s);

// ------------------------------------------------------------------ launches

extern std::atomic<int64_t> g_launches;
void prof_begin(const char* name, cudaStream_t s, void** token);
void prof_end(void* token, cudaStream_t s);

// Launch wrapper: counts the launch, records profiling events when enabled,
// and converts a launch error into a status.
#define ARBX_LAUNCH(name, stream, ...)                                          \
  do {                                                                          \
    void* _tok = nullptr;                                                       \
    ::arbx::prof_begin(name, stream, &_tok);                                    \
    __VA_ARGS__;                                                                \
    ::arbx::prof_end(_tok, stream);                                             \
    ::arbx::g_launches.fetch_add(1, std::memory_order_relaxed);                 \
    ARBX_CUDA(cudaGetLastError());                                              \
  } while (0)

// Stream-ordered device allocation from the device's default memory pool.
arbx_status dev_alloc(void** p, size_t bytes, cudaStream_t s);
void dev_free(void* p, cudaStream_t s);

template <class T>
arbx_status dev_alloc_t(T** p, size_t count, cudaStream_t s) {
  return dev_alloc(reinterpret_cast<void**>(p), count * sizeof(T), s);
}

// Scoped stream-ordered temporary.
template <class T>
struct DevTemp {
  T* p = nullptr;
  cudaStream_t s = nullptr;
  explicit DevTemp(cudaStream_t st) : s(st) {}
  ~DevTemp() { if (p) dev_free(p, s); }
  arbx_status alloc(size_t count) { return dev_alloc_t(&p, count ? count : 1, s); }
  DevTemp(const DevTemp&) = delete;
  DevTemp& operator=(const DevTemp&) = delete;
};

int num_sms();
int max_smem_optin();

// Read `bytes` (<= 256) of device memory into host memory, stream-ordered on
// s, then synchronise s.  A one-thread kernel writes the bytes into mapped
// pinned host memory, so the read does not wait behind large copies queued
// on the copy engines by other streams.
arbx_status read_small(const void* dev_src, void* host_dst, size_t bytes, cudaStream_t s);

// Forest launch-setting records in the autotune text file (forest.cu): write
// them as "forest ..." lines, parse one such line (false if it is not a valid
// forest record), drop them all.
void forest_records_save(FILE* f);
bool forest_record_load(const char* line);
void forest_records_clear();

// ------------------------------------------------------------------ geometry

// One squared axis difference, rounded at every step.
__device__ __forceinline__ float sq_axis(float q, float p) {
  float d = __fsub_rn(q, p);
  return __fmul_rn(d, d);
}

// Squared distance from q to the closed box [lo, hi], with the same operation
// order as the point distance.  Culling soundness: for any p in the box, the
// clamped coordinate c = min(max(q, lo), hi) lies between q and p, so
// |q - c| <= |q - p| exactly; rounding, squaring and fl-addition are monotone,
// hence box_d2(q, box) <= d2(q, p) bitwise and a box that fails d2 <= r2 (or
// exceeds the current k-th distance) holds no match.  For a degenerate box
// [p, p] the clamp returns p and box_d2 equals d2(q, p) bit for bit.
template <int D>
__device__ __forceinline__ float box_d2(const float* q, const float* lo, const float* hi) {
  float acc = sq_axis(q[0], fminf(fmaxf(q[0], lo[0]), hi[0]));
#pragma unroll
  for (int a = 1; a < D; ++a) acc = __fadd_rn(acc, sq_axis(q[a], fminf(fmaxf(q[a], lo[a]), hi[a])));
  return acc;
}

// Closed overlap of two boxes.
template <int D>
__device__ __forceinline__ bool box_overlap(const float* alo, const float* ahi, const float* blo,
                                            const float* bhi) {
  bool ok = true;
#pragma unroll
  for (int a = 0; a < D; ++a) ok = ok && (alo[a] <= bhi[a]) && (blo[a] <= ahi[a]);
  return ok;
}

// ------------------------------------------------------------------ layouts

// Child code: c >= 0 is an internal node (numbered by its split position, see
// build.cu); c < 0 is a leaf at sorted position ~c.  NULL_CHILD marks the missing second child of the
// one-leaf tree.  Codes with TOP_FLAG refer to the shared-memory copy of the
// top levels (local index in the low bits).
constexpr int32_t NULL_CHILD = INT32_MIN;
constexpr int32_t TOP_FLAG = 1 << 30;
constexpr int64_t MAX_PRIMS = (int64_t(1) << 30) - 1;
constexpr int STACK_DEPTH = 128;  // > 96 = the radix-tree depth bound for 64+32-bit keys

// Internal node with float32 child boxes.  For a leaf child the box is the
// primitive's exact bounding box (the point itself for points) and orig[c]
// is the primitive's input index, so point leaves need no separate record;
// for an internal child orig[c] is the last sorted leaf of that child's
// subtree (its range end, used by the stackless traversal).
// Size 16*D + 16 bytes: 48 (2D), 64 (3D), 112 (6D).
template <int D>
struct alignas(16) Node {
  float lo0[D], hi0[D], lo1[D], hi1[D];
  int32_t child[2];
  int32_t orig[2];
};
static_assert(sizeof(Node<2>) == 48 && sizeof(Node<3>) == 64 && sizeof(Node<6>) == 112, "node size");

// Four-wide node: the grandchildren of binary node g in left-to-right order
// (an internal child of g contributes its two children, a leaf child itself;
// empty slots have code NULL_CHILD).  code[c] >= 0 is internal node code[c],
// whose own four-wide record is wide[code[c]]; code[c] < 0 is the leaf at
// sorted position ~code[c].  aux[c] is the leaf's input index, or for an
// internal entry the last sorted leaf of its subtree (its range end; the
// entries' ranges are consecutive, so a traversal that knows where g's range
// starts knows every entry's leaf count).  A traversal over these records
// opens one record per two binary levels.  Size 32*D + 32 bytes: 96 (2D),
// 128 (3D), 224 (6D).
template <int D>
struct alignas(16) Wide {
  float lo[4][D];
  float hi[4][D];
  int32_t code[4];
  int32_t aux[4];
};
static_assert(sizeof(Wide<2>) == 96 && sizeof(Wide<3>) == 128 && sizeof(Wide<6>) == 224, "wide node size");
// Stack bound of a traversal over four-wide records: at most three entries
// pushed per record, at most 48 records on a root-to-leaf path of the radix tree.
constexpr int WIDE_STACK_DEPTH = 160;

// Triangle leaf record in sorted order: vertices and input index (48 bytes).
struct alignas(16) TriLeaf {
  float v[9];
  int32_t orig;
  int32_t pad[2];
};
static_assert(sizeof(TriLeaf) == 48, "leaf size");

// Quantized internal node (3D): the node stores its own box origin (exact
// float32 lo) and a power-of-two step per axis (2^exps[a]); the two child
// boxes are 16-bit multiples of the step relative to the origin, decoded with
// downward rounding for lo and upward rounding for hi so that every decoded
// child box contains the exact child box (see k_quantize).  48 bytes.
struct alignas(16) QNode {
  float origin[3];
  int8_t exps[3];
  uint8_t pad;
  uint16_t q[2][2][3];  // [child][lo/hi][axis]
  int32_t child[2];
};
static_assert(sizeof(QNode) == 48, "qnode size");

__device__ __forceinline__ float pow2f(int e) {
  // 2^e for e in [-126, 127] (normal range), built from the exponent field.
  return __int_as_float((e + 127) << 23);
}

// Parent-relative 16-bit node (3D): the two child boxes as 16-bit multiples of
// a power-of-two step per axis, relative to this node's DECODED box -- the box
// its parent's record decodes for it (the root's is the exact root box, kept in
// the tree).  The node stores no box of its own, so a traversal carries each
// node's decoded box (its "frame": lo per axis and the three step exponents)
// from the parent, on its stack beside the node code.  32 bytes.
//   frame of a decoded box [lo, hi]:  origin = lo, step_a = 2^e_a with e_a the
//     smallest exponent in [-126, 127] such that 65535 * 2^e_a >= fl_up(hi_a - lo_a)
//   child box:  lo = fl_down(origin + q_lo * step), hi = fl_up(origin + q_hi * step)
// (q * step is exact; one rounding of the exact sum).  The encoder picks the tightest codes whose decoded box
// contains the exact child box, checked with these same functions, so culling
// stays conservative at every level even though the error of a level is
// measured from the decoded, not the exact, box of its parent.
struct alignas(16) PNode {
  uint16_t q[2][2][3];  // [child][lo/hi][axis]
  int32_t child[2];
};
static_assert(sizeof(PNode) == 32, "pnode size");

// The smallest e in [-126, 127] with 65535 * 2^e >= ext, from the bits of
// ext: for ext = 2^E * (1 + f / 2^23), 65535 * 2^(E-16) < ext always and
// 65535 * 2^(E-15) = 2^E * (2 - 2^-15) < ext exactly when f > 2^23 - 2^8,
// i.e. when adding 0xff to the bits carries into the exponent field, so
// e = E - 15 + carry, at least -126 (zero, subnormal and negative ext give
// -126; +inf gives 113, whose largest codes decode to +inf, still
// conservative).  Returned as the float32 exponent field of 2^e (e + 127).
__device__ __forceinline__ uint32_t p16_exp_field(float ext) {
  const int v = ((__float_as_int(ext) + 0xff) >> 23) - 15;
  return (uint32_t)max(1, v);
}

// Frame of the decoded box [lo, hi]: (lo_x, lo_y, lo_z, the three exponent
// fields of the steps in bytes 0..2 of w).
__device__ __forceinline__ float4 p16_frame(const float* lo, const float* hi) {
  uint32_t packed = 0;
#pragma unroll
  for (int a = 0; a < 3; ++a) packed |= p16_exp_field(__fsub_ru(hi[a], lo[a])) << (8 * a);
  return make_float4(lo[0], lo[1], lo[2], __uint_as_float(packed));
}

__device__ __forceinline__ float p16_step(float4 f, int a) {
  return __uint_as_float(((__float_as_uint(f.w) >> (8 * a)) & 0xffu) << 23);
}

// origin + q * step rounded down / up, as one fused multiply-add: q * step is
// exact (16-bit q, power-of-two step), so this is the directed rounding of
// the exact sum.
__device__ __forceinline__ float p16_lo(float origin, uint32_t q, float step) {
  return __fmaf_rd((float)q, step, origin);
}
__device__ __forceinline__ float p16_hi(float origin, uint32_t q, float step) {
  return __fmaf_ru((float)q, step, origin);
}

// Load a node of T (a multiple of 16 bytes) with read-only vector loads:
// 32-byte loads (ld.global.nc.v8) when T is a multiple of 32 bytes and the
// record starts on a 32-byte boundary (node arrays come from the allocator's
// aligned blocks; the check keeps any other pointer on the 16-byte path),
// else 16-byte loads.
// (V8 = false keeps 16-byte loads: the one-lane kNN kernel measured faster
// with them -- 19.2 vs 19.8 ms for k=16 at 10M, the wider loads cost it a
// register spill -- while the count and fill passes gain: count 7.6 -> 6.3 ms,
// radius storage query 20.7 -> 18.1 ms.)
template <class T, bool V8 = true>
__device__ __forceinline__ T load_node_global(const T* p) {
  static_assert(sizeof(T) % 16 == 0, "16-byte multiple");
  constexpr int NV = sizeof(T) / 16;
  union { float4 v[NV]; float f[4 * NV]; T t; } u;
  if constexpr (V8 && sizeof(T) % 32 == 0) {
    if ((reinterpret_cast<uintptr_t>(p) & 31u) == 0u) {
      const float* f = reinterpret_cast<const float*>(p);
#pragma unroll
      for (int i = 0; i < NV / 2; ++i) {
        asm volatile("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                     : "=f"(u.f[8 * i]), "=f"(u.f[8 * i + 1]), "=f"(u.f[8 * i + 2]), "=f"(u.f[8 * i + 3]),
                       "=f"(u.f[8 * i + 4]), "=f"(u.f[8 * i + 5]), "=f"(u.f[8 * i + 6]), "=f"(u.f[8 * i + 7])
                     : "l"(f + 8 * i));
      }
      return u.t;
    }
  }
  const float4* s = reinterpret_cast<const float4*>(p);
#pragma unroll
  for (int i = 0; i < NV; ++i) u.v[i] = __ldg(s + i);
  return u.t;
}

template <class T>
__device__ __forceinline__ T load_node_shared(const T* p) {
  constexpr int NV = sizeof(T) / 16;
  union { float4 v[NV]; T t; } u;
  const float4* s = reinterpret_cast<const float4*>(p);
#pragma unroll
  for (int i = 0; i < NV; ++i) u.v[i] = s[i];
  return u.t;
}

// ------------------------------------------------------------------ tree

// Device-side view of a tree handed to kernels by value.
struct TreeView {
  const void* nodes;     // Node<D>[n-1] (or QNode[n-1]); for n == 1 one pseudo node
  const void* top;       // top-level copy in BFS order (global memory), ntop nodes
  const TriLeaf* leaves; // triangles: sorted leaf records
  const void* wide;      // Wide<D>[nnodes] (point and box trees), or null
  const int32_t* leaf_orig;  // quantized triangle trees: input index of each sorted leaf
  int64_t n;
  int32_t ntop;
  int32_t root;          // code of the root internal node (0, or TOP_FLAG|0)
  float4 rframe;         // PNode trees: frame (see p16_frame) of the root's exact box
  uint32_t* err = nullptr;  // device error word (checked builds report bad indices here)
};

// Internal records of a tree over n primitives (one pseudo node for n == 1).
__device__ __forceinline__ int64_t internal_count(const TreeView& t) { return t.n > 1 ? t.n - 1 : 1; }

// Checked positions in a tree's arrays: an internal node code (no TOP_FLAG),
// a sorted leaf position.
__device__ __forceinline__ int64_t node_index(int32_t code, const TreeView& t) {
  return checked_index(code, internal_count(t), t.err, BAD_NODE);
}
__device__ __forceinline__ int64_t leaf_index(int32_t pos, const TreeView& t) {
  return checked_index(pos, t.n, t.err, BAD_LEAF);
}

}  // namespace arbx
