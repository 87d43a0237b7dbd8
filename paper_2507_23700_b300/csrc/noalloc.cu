// arbx_query_offsets_noalloc: the offsets phase of the storage query for
// callers that cannot allocate device memory.
//
// Who needs it: code that must not call cudaMalloc (or any allocator) while it
// runs -- for example a process whose device memory is entirely owned by
// another allocator or memory budget, a latency-critical path where an
// allocation could synchronise the device, or code running while the device
// is being captured into a CUDA graph in a mode that forbids allocation.  The
// regular entry point (arbx_query_offsets) allocates its per-query counts and
// scan temporaries from the stream-ordered pool; this one keeps them in a
// fixed device array that is part of the library image instead.
//
// The scratch array below is a file-scope __device__ array, so every GPU that
// loads libarbx holds it (about 4 MiB) until the process exits.  It is shared
// by every call on a device and keeps the last call's contents; each call
// clears what must start at zero (the work counter and the error word) and
// overwrites the rest.  Two calls whose work overlaps on the GPU (different
// streams, or different host threads) race on the array: serialise them.
//
// Host code cannot use the array's name as a device address (in host code it
// names a host-side stand-in), so the first call on each device looks the
// address up with cudaGetSymbolAddress while that device is current and caches
// it.  That first call on a device therefore makes a CUDA runtime query and
// should come before any stream capture.
#include <mutex>

#include "primitives.cuh"
#include "query.cuh"
#include "tree.cuh"

namespace {

constexpr int64_t NOALLOC_MAX_Q = ARBX_NOALLOC_MAX_QUERIES;
constexpr size_t HEADER_BYTES = 256;                       // [0,8) work counter, [8,12) error word
constexpr size_t COUNTS_BYTES = (size_t)NOALLOC_MAX_Q * 4;  // int32 count per query
constexpr int64_t MAX_TILES = (NOALLOC_MAX_Q + arbx::SCAN_TILE_ELEMS - 1) / arbx::SCAN_TILE_ELEMS;
constexpr size_t TILE_BYTES = (((size_t)(MAX_TILES + 1) * 8 + 255) / 256) * 256;
constexpr int64_t TILE_CAP = (int64_t)(TILE_BYTES / 8);  // entries of each scan temporary
constexpr size_t SCRATCH_BYTES = HEADER_BYTES + COUNTS_BYTES + 2 * TILE_BYTES;

static __device__ __align__(256) unsigned char g_noalloc_scratch[SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
unsigned char* g_scratch_addr[MAX_DEVICES] = {};

// Device address of the scratch array on the current device (looked up once).
arbx_status scratch_address(int dev, unsigned char** out) {
  if (dev < 0 || dev >= MAX_DEVICES) return ARBX_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return arbx::cuda_status(e, "cudaGetSymbolAddress", __FILE__, __LINE__);
    g_scratch_addr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_scratch_addr[dev];
  return ARBX_OK;
}

bool finite_nonneg(float x) { return x == x && x - x == 0.0f && x >= 0.0f; }

}  // namespace

extern "C" arbx_status arbx_query_offsets_noalloc(arbx_tree tree, const arbx_predicates* pred, int64_t* offsets_dev,
                                                  uint32_t* error_dev, arbx_stream stream) {
  using namespace arbx;
  if (!tree || !pred || !offsets_dev) return ARBX_ERR_INVALID;
  if (pred->kind != ARBX_SPHERE && pred->kind != ARBX_BOX_PRED) return ARBX_ERR_INVALID;
  if (pred->dim != tree->dim) return ARBX_ERR_INVALID;
  if (pred->m < 0) return ARBX_ERR_INVALID;
  if (pred->m > NOALLOC_MAX_Q) return ARBX_ERR_CAPACITY;  // beyond the fixed scratch array
  if (pred->m > 0 && !pred->data_dev) return ARBX_ERR_INVALID;
  if (pred->kind == ARBX_SPHERE && !pred->radii_dev && !finite_nonneg(pred->radius)) return ARBX_ERR_INVALID;
  if (pred->kind == ARBX_SPHERE && tree->kind == ARBX_TRIANGLE) return ARBX_ERR_UNSUPPORTED;
  // 16-bit nodes answer box predicates only; refused before any device work
  if (tree->bt.quantized && pred->kind != ARBX_BOX_PRED) return ARBX_ERR_UNSUPPORTED;

  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != tree->device) ARBX_CUDA(cudaSetDevice(tree->device));
  struct Restore {
    int d;
    ~Restore() {
      int cur = -1;
      cudaGetDevice(&cur);
      if (d >= 0 && cur != d) cudaSetDevice(d);
    }
  } restore{prev};

  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int64_t m = pred->m;
  if (tree->n == 0 || m == 0) {
    ARBX_CUDA(cudaMemsetAsync(offsets_dev, 0, (size_t)(m + 1) * sizeof(int64_t), s));
    if (error_dev) ARBX_CUDA(cudaMemsetAsync(error_dev, 0, sizeof(uint32_t), s));
    return ARBX_OK;
  }

  unsigned char* base = nullptr;
  ARBX_TRY(scratch_address(tree->device, &base));
  auto* counter = reinterpret_cast<unsigned long long*>(base);
  auto* err = reinterpret_cast<uint32_t*>(base + 8);
  auto* counts = reinterpret_cast<int32_t*>(base + HEADER_BYTES);
  auto* totals = reinterpret_cast<int64_t*>(base + HEADER_BYTES + COUNTS_BYTES);
  auto* offs = reinterpret_cast<int64_t*>(base + HEADER_BYTES + COUNTS_BYTES + TILE_BYTES);

  // Queries run in input order (the Morton ordering of the regular path needs
  // sort buffers); the results are the same bytes.
  const BuiltTree& b = tree->bt;
  QueryPlan p;
  p.prim_kind = tree->kind;
  p.dim = tree->dim;
  p.quantized = b.quantized;
  p.prel = b.prel;
  p.pred_kind = pred->kind;
  p.qdata = pred->data_dev;
  p.radii = pred->kind == ARBX_SPHERE ? pred->radii_dev : nullptr;
  p.r2 = pred->radius * pred->radius;
  p.m = m;
  p.tv.nodes = b.nodes;
  p.tv.leaves = b.leaves;
  p.tv.wide = nullptr;  // the binary traversal (its kernel is the one this path instantiates)
  p.tv.leaf_orig = b.leaf_orig;
  p.tv.n = b.n;
  p.tv.rframe = make_float4(b.rframe[0], b.rframe[1], b.rframe[2], b.rframe[3]);
  p.tv.err = err;
  // no staged top levels: the regular path's default for spatial predicates
  // (staging the top 1023 nodes measured slower on the 10M mixture)
  p.tv.ntop = 0;
  p.tv.top = nullptr;
  p.tv.root = b.root;

  ARBX_CUDA(cudaMemsetAsync(base, 0, 16, s));  // work counter and error word start at zero
  ARBX_TRY(run_spatial_count_prealloc(p, counts, counter, err, s));
  ARBX_TRY(exclusive_scan_prealloc(counts, offsets_dev, m, totals, offs, TILE_CAP, s));
  if (error_dev) ARBX_CUDA(cudaMemcpyAsync(error_dev, err, sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
  return ARBX_OK;
}
