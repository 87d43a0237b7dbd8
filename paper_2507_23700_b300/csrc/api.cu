// The C ABI of libarbx (declared and documented in include/arbx.h): argument
// checks, tree handles, stream-ordered memory, the count -> scan -> fill
// storage query, the device error word and kernel instrumentation.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <unordered_map>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "build.cuh"
#include "primitives.cuh"
#include "query.cuh"
#include "tree.cuh"

namespace arbx {

std::atomic<int64_t> g_launches{0};

namespace {

constexpr int MAX_DEVICES = 64;

// NVTX range around each public entry point (visible in Nsight Systems /
// Compute timelines; free when no tool is attached).
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
  Range(const Range&) = delete;
  Range& operator=(const Range&) = delete;
};

bool log_enabled() {
  static const bool on = [] {
    const char* v = std::getenv("ARBX_LOG");
    return v && *v && std::strcmp(v, "0") != 0;
  }();
  return on;
}

std::mutex g_dev_mu;
uint32_t* g_err_word[MAX_DEVICES] = {};
int g_sms[MAX_DEVICES] = {};
bool g_pool_ready[MAX_DEVICES] = {};

int current_device() {
  int d = 0;
  cudaGetDevice(&d);
  return d;
}

// ------------------------------------------------------------------ profiler

struct ProfRecord {
  const char* name;
  cudaEvent_t start, stop;
};

std::mutex g_prof_mu;
std::atomic<bool> g_prof_on{false};
std::vector<ProfRecord> g_prof_pending;
std::vector<cudaEvent_t> g_prof_free_events;
struct ProfTotal {
  int64_t launches = 0;
  double ms = 0.0;
};
std::vector<std::pair<std::string, ProfTotal>> g_prof_totals;

cudaEvent_t prof_event() {
  if (!g_prof_free_events.empty()) {
    cudaEvent_t e = g_prof_free_events.back();
    g_prof_free_events.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

void prof_collect_locked() {
  for (auto& r : g_prof_pending) {
    cudaEventSynchronize(r.stop);
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, r.start, r.stop);
    bool found = false;
    for (auto& t : g_prof_totals) {
      if (t.first == r.name) {
        t.second.launches += 1;
        t.second.ms += ms;
        found = true;
        break;
      }
    }
    if (!found) {
      ProfTotal pt;
      pt.launches = 1;
      pt.ms = ms;
      g_prof_totals.emplace_back(r.name, pt);
    }
    g_prof_free_events.push_back(r.start);
    g_prof_free_events.push_back(r.stop);
  }
  g_prof_pending.clear();
}

}  // namespace

arbx_status cuda_status(cudaError_t e, const char* what, const char* file, int line) {
  if (log_enabled()) std::fprintf(stderr, "arbx: %s failed: %s (%s:%d)\n", what, cudaGetErrorString(e), file, line);
  cudaGetLastError();  // clear a sticky-free error so later calls are not affected
  return e == cudaErrorMemoryAllocation ? ARBX_ERR_OOM : ARBX_ERR_CUDA;
}

void prof_begin(const char* name, cudaStream_t s, void** token) {
  *token = nullptr;
  if (!g_prof_on.load(std::memory_order_relaxed)) return;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;  // no timing in graphs
  std::lock_guard<std::mutex> lk(g_prof_mu);
  ProfRecord* r = new ProfRecord{name, prof_event(), prof_event()};
  cudaEventRecord(r->start, s);
  *token = r;
}

void prof_end(void* token, cudaStream_t s) {
  if (!token) return;
  ProfRecord* r = static_cast<ProfRecord*>(token);
  std::lock_guard<std::mutex> lk(g_prof_mu);
  cudaEventRecord(r->stop, s);
  g_prof_pending.push_back(*r);
  delete r;
}

arbx_status device_error_word(uint32_t** out) {
  const int d = current_device();
  if (d < 0 || d >= MAX_DEVICES) return ARBX_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lk(g_dev_mu);
  if (!g_err_word[d]) {
    uint32_t* p = nullptr;
    ARBX_CUDA(cudaMalloc(&p, sizeof(uint32_t)));
    ARBX_CUDA(cudaMemset(p, 0, sizeof(uint32_t)));
    ARBX_CUDA(cudaDeviceSynchronize());
    g_err_word[d] = p;
  }
  *out = g_err_word[d];
  return ARBX_OK;
}

// Mapped pinned host slots for read_small: 1024 slots of 256 bytes per
// device, handed out round robin (a slot is in use only for the duration of
// one synchronous read).
constexpr int SMALL_SLOTS = 1024;
constexpr size_t SMALL_BYTES = 256;
struct SmallSlots {
  unsigned char* host = nullptr;
  unsigned char* dev = nullptr;
  std::atomic<uint32_t> next{0};
};
SmallSlots g_small[MAX_DEVICES];

__global__ void k_read_small(const unsigned char* __restrict__ src, volatile unsigned char* dst, int bytes) {
  for (int i = threadIdx.x; i < bytes; i += blockDim.x) dst[i] = src[i];
  __threadfence_system();
}

arbx_status read_small(const void* dev_src, void* host_dst, size_t bytes, cudaStream_t s) {
  if (bytes > SMALL_BYTES) return ARBX_ERR_INVALID;
  const int d = current_device();
  if (d < 0 || d >= MAX_DEVICES) return ARBX_ERR_UNSUPPORTED;
  SmallSlots& sl = g_small[d];
  {
    std::lock_guard<std::mutex> lk(g_dev_mu);
    if (!sl.host) {
      void* h = nullptr;
      ARBX_CUDA(cudaHostAlloc(&h, SMALL_SLOTS * SMALL_BYTES, cudaHostAllocMapped | cudaHostAllocPortable));
      void* dp = nullptr;
      ARBX_CUDA(cudaHostGetDevicePointer(&dp, h, 0));
      sl.host = static_cast<unsigned char*>(h);
      sl.dev = static_cast<unsigned char*>(dp);
    }
  }
  const uint32_t slot = sl.next.fetch_add(1) % SMALL_SLOTS;
  ARBX_LAUNCH("read_small", s, k_read_small<<<1, 64, 0, s>>>(static_cast<const unsigned char*>(dev_src),
                                                             sl.dev + slot * SMALL_BYTES, (int)bytes));
  ARBX_CUDA(cudaStreamSynchronize(s));
  std::memcpy(host_dst, (const void*)(sl.host + slot * SMALL_BYTES), bytes);
  return ARBX_OK;
}

arbx_status check_stream(cudaStream_t s) {
  uint32_t* w = nullptr;
  ARBX_TRY(device_error_word(&w));
  uint32_t v = 0;
  ARBX_TRY(read_small(w, &v, sizeof(v), s));
  if (v == 0) return ARBX_OK;
  ARBX_CUDA(cudaMemsetAsync(w, 0, sizeof(uint32_t), s));
  ARBX_CUDA(cudaStreamSynchronize(s));
  if (v & DEVERR_BOUNDS) {
    if (log_enabled())
      std::fprintf(stderr, "arbx: index out of range:%s%s%s%s%s\n", (v & BAD_ORDER) ? " query order" : "",
                   (v & BAD_NODE) ? " node code" : "", (v & BAD_TOP) ? " top-level code" : "",
                   (v & BAD_LEAF) ? " leaf position" : "", (v & BAD_TREE) ? " tree structure" : "");
    return ARBX_ERR_BOUNDS;
  }
  if (v & DEVERR_STACK) return ARBX_ERR_STACK_OVERFLOW;
  if (v & DEVERR_NONFINITE) return ARBX_ERR_NONFINITE;
  if (v & DEVERR_TIMEOUT) return ARBX_ERR_TIMEOUT;
  return ARBX_ERR_CUDA;
}

int num_sms() {
  const int d = current_device();
  if (d >= 0 && d < MAX_DEVICES && g_sms[d] > 0) return g_sms[d];
  int v = 0;
  cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, d);
  if (v <= 0) v = 1;
  if (d >= 0 && d < MAX_DEVICES) g_sms[d] = v;
  return v;
}

int max_smem_optin() {
  int v = 0;
  cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, current_device());
  return v;
}

// Host-side fault injection (tests): after `g_fail_after` more successful
// device allocations, the next `g_fail_count` ones report ARBX_ERR_OOM.
std::atomic<int64_t> g_fail_after{-1};
std::atomic<int64_t> g_fail_count{0};

arbx_status dev_alloc(void** p, size_t bytes, cudaStream_t s) {
  *p = nullptr;
  if (g_fail_count.load(std::memory_order_relaxed) > 0) {
    if (g_fail_after.fetch_sub(1) <= 0) {
      if (g_fail_count.fetch_sub(1) > 0) return ARBX_ERR_OOM;
    }
  }
  const int d = current_device();
  if (d >= 0 && d < MAX_DEVICES && !g_pool_ready[d]) {
    // Keep freed blocks in the device's default pool instead of returning
    // them to the driver at every synchronisation.
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, d) == cudaSuccess) {
      // up to ARBX_POOL_RELEASE_GB (default 32) GiB of freed blocks stay
      // cached for the next call (mapping new device memory costs about a
      // millisecond per GB); beyond that they go back to the driver at the
      // next synchronisation (other allocators share the GPU);
      // arbx_memory_trim releases the cache
      uint64_t thr = uint64_t(32) << 30;
      if (const char* v = std::getenv("ARBX_POOL_RELEASE_GB")) thr = uint64_t(std::strtoull(v, nullptr, 10)) << 30;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    g_pool_ready[d] = true;
  }
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMallocAsync(p, bytes, s);
  if (e != cudaSuccess) {
    *p = nullptr;
    return cuda_status(e, "cudaMallocAsync", __FILE__, __LINE__);
  }
  return ARBX_OK;
}

void dev_free(void* p, cudaStream_t s) {
  if (p) cudaFreeAsync(p, s);
}

namespace {

// ------------------------------------------------------------------ helpers

__global__ void k_iota_offsets(int64_t* off, int64_t m, int64_t kk) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i <= m) off[i] = i * kk;
}

// Ray nearest rows of kk hits (padded with -1 after the last hit): hits per
// row, and the rows compacted into CRS order.
__global__ void k_hit_counts(const int32_t* hit, int64_t m, int kk, int32_t* counts) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  int32_t c = 0;
  for (int s = 0; s < kk; ++s) c += hit[i * kk + s] >= 0 ? 1 : 0;
  counts[i] = c;
}

__global__ void k_hit_compact(const int32_t* hit, const float* t, int64_t m, int kk, const int64_t* off,
                              int32_t* idx, float* d2) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  int64_t w = off[i];
  for (int s = 0; s < kk; ++s) {
    if (hit[i * kk + s] < 0) break;
    idx[w] = hit[i * kk + s];
    if (d2) d2[w] = t[i * kk + s];
    ++w;
  }
}

bool finite_f(float x) { return x == x && x - x == 0.0f; }

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int d) {
    cudaGetDevice(&prev);
    if (prev != d) cudaSetDevice(d);
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

bool is_ray_all(int kind) { return kind == ARBX_RAY_INTERSECT || kind == ARBX_RAY_ORDERED; }
// predicates answered by the count / fill traversal
bool is_spatial(int kind) { return kind == ARBX_SPHERE || kind == ARBX_BOX_PRED || is_ray_all(kind); }
// the value stored beside each match: d2 for spheres, t for rays
bool has_value(int kind) { return kind == ARBX_SPHERE || is_ray_all(kind); }

arbx_status check_pred(const arbx_tree_t* t, const arbx_predicates* p) {
  if (!t || !p) return ARBX_ERR_INVALID;
  if (p->m < 0 || p->m >= (int64_t(1) << 31)) return ARBX_ERR_INVALID;
  if (p->m > 0 && !p->data_dev) return ARBX_ERR_INVALID;
  switch (p->kind) {
    case ARBX_SPHERE:
      if (p->dim != t->dim) return ARBX_ERR_INVALID;
      if (!p->radii_dev && (!finite_f(p->radius) || p->radius < 0.0f)) return ARBX_ERR_INVALID;
      if (t->kind == ARBX_TRIANGLE) return ARBX_ERR_UNSUPPORTED;
      break;
    case ARBX_BOX_PRED:
      if (p->dim != t->dim) return ARBX_ERR_INVALID;
      break;
    case ARBX_NEAREST:
      if (p->dim != t->dim || p->k <= 0) return ARBX_ERR_INVALID;
      if (p->k > KNN_MAX_K || t->kind == ARBX_TRIANGLE) return ARBX_ERR_UNSUPPORTED;
      break;
    case ARBX_RAY_NEAREST:
      if (p->dim != 3) return ARBX_ERR_INVALID;
      if (t->kind != ARBX_TRIANGLE || p->k > 32) return ARBX_ERR_UNSUPPORTED;
      break;
    case ARBX_RAY_INTERSECT:
    case ARBX_RAY_ORDERED:
      if (p->dim != 3) return ARBX_ERR_INVALID;
      if (t->kind != ARBX_TRIANGLE) return ARBX_ERR_UNSUPPORTED;
      break;
    default:
      return ARBX_ERR_INVALID;
  }
  return ARBX_OK;
}

struct Tuning {
  int block = 256;
  int sort_queries = -1;  // -1: by batch size (see make_plan)
  int top_levels = -1;  // -1: by predicate (spatial and nearest 0, ray 255)
  int grid_per_sm = 0;
  int warp_refill = -1;
  int stackless = 0;
  int single_pass = 0;
  int lanes = 1;        // nearest predicates: lanes per query
  int wide = -1;        // nearest and counting traversals over the four-wide records (-1: by predicate)
  int packets = -1;     // one traversal per warp for its 32 queries (-1: off)
  int runs = 0;         // nearest: adjacent queries per lane run (0: by k)
};

arbx_status read_tuning(const arbx_tuning* tu, Tuning* out) {
  Tuning t;
  if (tu) {
    if (tu->block != 0) {
      if (tu->block < 64 || tu->block > 256 || tu->block % 32) return ARBX_ERR_INVALID;
      t.block = tu->block;
    }
    if (tu->sort_queries >= 0) t.sort_queries = tu->sort_queries ? 1 : 0;
    if (tu->top_levels >= 0) {
      if (tu->top_levels != 0 && tu->top_levels != 255 && tu->top_levels != 1023) return ARBX_ERR_INVALID;
      t.top_levels = tu->top_levels;
    }
    if (tu->grid_per_sm < 0 || tu->grid_per_sm > 64) return ARBX_ERR_INVALID;
    t.grid_per_sm = tu->grid_per_sm;
    if (tu->warp_refill > 1) return ARBX_ERR_INVALID;
    t.warp_refill = tu->warp_refill < 0 ? -1 : tu->warp_refill;
    if (tu->stackless > 1) return ARBX_ERR_INVALID;
    t.stackless = tu->stackless > 0 ? 1 : 0;
    if (tu->single_pass > 1) return ARBX_ERR_INVALID;
    if (tu->single_pass >= 0) t.single_pass = tu->single_pass;
    if (tu->lanes_per_query > 0) {
      const int L = tu->lanes_per_query;
      if (L != 1 && L != 2 && L != 4 && L != 8 && L != 16 && L != 32) return ARBX_ERR_INVALID;
      t.lanes = L;
    }
    if (tu->wide_nodes > 1) return ARBX_ERR_INVALID;
    if (tu->wide_nodes >= 0) t.wide = tu->wide_nodes;
    if (tu->warp_packets > 1) return ARBX_ERR_INVALID;
    if (tu->warp_packets >= 0) t.packets = tu->warp_packets;
    if (tu->query_runs > 0) {
      if (tu->query_runs != 1 && tu->query_runs != 4 && tu->query_runs != 8) return ARBX_ERR_INVALID;
      t.runs = tu->query_runs;
    }
  }
  *out = t;
  return ARBX_OK;
}

// What a plan's traversal produces: counts or per-query rows, or CRS storage
// (whose write pattern changes the best default query ordering).
enum class PlanUse { Traversal, Storage };

// A plan plus the query order it owns.
struct Planned {
  QueryPlan p;
  cudaStream_t s = nullptr;
  bool own_order = false;  // the order was sorted here (not the caller's)
  ~Planned() {
    if (p.order && own_order) dev_free(const_cast<uint32_t*>(p.order), s);
  }
};

// ------------------------------------------------------------------ autotuned settings
//
// Keyed by GPU model, predicate kind, dimension, k, node format and the
// binary orders of magnitude of n and m (a factor of 4 for m).  Filled by
// arbx_autotune or loaded from a file; consulted when a query passes no tuning.
struct TuneKey {
  std::string gpu;
  int kind, dim, k, nb, mb, quantized;
  bool operator<(const TuneKey& o) const {
    return std::tie(gpu, kind, dim, k, nb, mb, quantized) < std::tie(o.gpu, o.kind, o.dim, o.k, o.nb, o.mb, o.quantized);
  }
};
std::mutex g_tune_mu;
std::map<TuneKey, arbx_tuning> g_tune;

std::string gpu_name() {
  cudaDeviceProp prop;
  int d = current_device();
  std::string s = cudaGetDeviceProperties(&prop, d) == cudaSuccess ? prop.name : "unknown";
  for (char& c : s)
    if (c == ' ') c = '_';
  return s;
}

int log_bucket(int64_t v, int base_log2) {
  int b = 0;
  while (v > 1) {
    v >>= base_log2;
    ++b;
  }
  return b;
}

TuneKey tune_key(const arbx_tree_t* t, const arbx_predicates* pr) {
  return TuneKey{gpu_name(), pr->kind, t->dim, pr->kind == ARBX_NEAREST ? pr->k : 0, log_bucket(t->n, 1),
                 log_bucket(pr->m, 2), t->bt.prel ? 2 : (t->bt.quantized ? 1 : 0)};
}

bool tuned_for(const arbx_tree_t* t, const arbx_predicates* pr, arbx_tuning* out) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  if (g_tune.empty()) return false;
  auto it = g_tune.find(tune_key(t, pr));
  if (it == g_tune.end()) return false;
  *out = it->second;
  return true;
}

// Checked builds: a caller's order[0..m) must be a permutation of 0..m-1 (one
// bit per query marks the entries seen).
__global__ void k_check_perm(const uint32_t* __restrict__ order, int64_t m, uint32_t* __restrict__ bits,
                             uint32_t* __restrict__ err) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const uint32_t q = order[i];
  if ((int64_t)q >= m) {
    atomicOr(err, DEVERR_BOUNDS | BAD_ORDER);
    return;
  }
  const uint32_t bit = 1u << (q & 31u);
  if (atomicOr(bits + (q >> 5), bit) & bit) atomicOr(err, DEVERR_BOUNDS | BAD_ORDER);
}

// Reports ARBX_ERR_BOUNDS (synchronously) before anything reads the order.
arbx_status check_permutation(const uint32_t* order, int64_t m, cudaStream_t s) {
  uint32_t* err = nullptr;
  ARBX_TRY(device_error_word(&err));
  DevTemp<uint32_t> bits(s);
  const int64_t words = (m + 31) / 32;
  ARBX_TRY(bits.alloc(words));
  ARBX_CUDA(cudaMemsetAsync(bits.p, 0, (size_t)words * sizeof(uint32_t), s));
  ARBX_LAUNCH("check_perm", s, k_check_perm<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(order, m, bits.p, err));
  return check_stream(s);
}

// Smallest batch that the default query ordering sorts.  Measured on the 10M
// mixture with prefixes of its query stream (ms sorted / in input order):
//   count    64k 1.18 / 0.79, 256k 1.11 / 1.21, 1M 1.41 / 3.14
//   kNN k=16 16k 1.29 / 1.27, 64k 1.39 / 1.53, 1M 2.82 / 4.41
//   CRS      256k 4.63 / 3.36, 1M 5.28 / 8.41 (small sorted batches scatter a
//            warp's 32 output segments, input order keeps them adjacent)
// Rays are always sorted (their origins order them well at every size).
int64_t sort_threshold(int kind, PlanUse use) {
  if (kind == ARBX_RAY_NEAREST || is_ray_all(kind)) return 2;
  if (kind == ARBX_NEAREST) return 32768;
  return use == PlanUse::Storage ? 524288 : 131072;
}

arbx_status make_plan(const arbx_tree_t* t, const arbx_predicates* pr, const arbx_tuning* tu, cudaStream_t s,
                      Planned* out, PlanUse use = PlanUse::Traversal) {
  arbx_tuning auto_tu;
  if (!tu && tuned_for(t, pr, &auto_tu)) tu = &auto_tu;
  Tuning tn;
  ARBX_TRY(read_tuning(tu, &tn));
  QueryPlan& p = out->p;
  out->s = s;
  const BuiltTree& b = t->bt;
  p.prim_kind = t->kind;
  p.dim = t->dim;
  p.quantized = b.quantized;
  p.prel = b.prel;
  p.pred_kind = pr->kind;
  p.qdata = pr->data_dev;
  p.radii = pr->kind == ARBX_SPHERE ? pr->radii_dev : nullptr;
  p.r2 = pr->radius * pr->radius;  // fl(r*r), one IEEE multiply
  p.m = pr->m;
  p.block = tn.block;
  p.grid_per_sm = tn.grid_per_sm;
  p.refill = tn.warp_refill;
  p.stackless = tn.stackless == 1 && !p.quantized && (pr->kind == ARBX_SPHERE || pr->kind == ARBX_BOX_PRED);
  p.single_pass = tn.single_pass == 1;
  p.lanes = tn.lanes;
  // Warp packets are off by default: on the 10M mixture they beat one lane per
  // query only at k = 1 (5.7 vs 7.1 ms), and lane runs beat both there (4.6 ms);
  // for k = 8..32 the union of a warp's 32 visit sets is about four times one
  // query's (k=16: 22.6 vs 20.4 ms)
  p.packets = tn.packets == 1;
  // Lane runs, measured on the 10M 3D mixture (k=16: 19.2 ms one query per
  // lane, 17.0 / 17.3 with runs of 4 / 8; k=8: 12.2, 10.2 / 10.3; k=1 without
  // packets: 6.3, 4.6 / 4.4; k=2: 8.6, 5.9 with 4; k=32 on four-wide records:
  // 42.9, 36.0 / 35.7; lane groups on 2M queries: k=64 33.9, 32.1 / 33.7,
  // k=256 263.6, 243.1 / 244.0) and 4M uniform 2D points (k=16: 3.9, 3.6
  // with 4).  In 6D they lose (4M uniform, k=16: 59.3 ms, 64.0 with 4): the
  // triangle-inequality bound is loose there.
  int run = 1;
  if (pr->kind == ARBX_NEAREST && t->dim <= 3 && tn.warp_refill != 1) run = pr->k == 1 ? 8 : 4;
  p.knn_run = tn.runs > 0 ? tn.runs : run;
  // Default measured on B300 with the 10M mixture: the four-wide records pay
  // only for nearest lists of 17..32 keys (k=32 42.7 ms vs 47.4 binary; k=16
  // 21.8 vs 19.4, k=8 15.2 vs 12.4, count pass 7.8 vs 7.6: the records halve
  // the steps, not the node bytes or the box tests a query needs)
  p.wide = tn.wide == 1 || (tn.wide < 0 && pr->kind == ARBX_NEAREST && pr->k > 16 && pr->k <= 32);
  p.tv.nodes = b.nodes;
  p.tv.leaves = b.leaves;
  p.tv.wide = b.wide;
  p.tv.leaf_orig = b.leaf_orig;
  p.tv.n = b.n;
  p.tv.rframe = make_float4(b.rframe[0], b.rframe[1], b.rframe[2], b.rframe[3]);
  ARBX_TRY(device_error_word(&p.tv.err));
  // Defaults measured on B300 with the 10M-point mixture: spatial and nearest
  // passes run fastest without staged top levels (the shared memory is worth
  // more as L1 for the node records: fill 20.2 ms with 1023 staged nodes, 14.7
  // without); ray traversals keep 255.
  int top = tn.top_levels;
  if (top < 0) top = pr->kind == ARBX_RAY_NEAREST || is_ray_all(pr->kind) ? 255 : 0;
  const int ci = top == 1023 ? 1 : 0;
  p.tv.ntop = top == 0 ? 0 : b.ntop[ci];
  p.tv.top = b.top[ci];
  p.tv.root = p.tv.ntop > 0 ? (TOP_FLAG | 0) : b.root;
  // a caller's order is used unless sorting is switched off; otherwise the
  // default sorts batches from sort_threshold up
  const bool sort = pr->m > 1 && (tn.sort_queries == 1 || (tn.sort_queries < 0 &&
                                                            (pr->order_dev || pr->m >= sort_threshold(pr->kind, use))));
  if (sort) {
    if (pr->order_dev) {
      if (CHECKED) ARBX_TRY(check_permutation(pr->order_dev, pr->m, s));
      p.order = pr->order_dev;  // the caller's order (e.g. from arbx_query_order), shared between calls
    } else {
      uint32_t* order = nullptr;
      ARBX_TRY(query_order(p, b.scene, &order, s));
      p.order = order;
      out->own_order = true;
    }
  }
  return ARBX_OK;
}

arbx_status zero_counts(int32_t* out, int64_t m, cudaStream_t s) {
  if (m > 0) ARBX_CUDA(cudaMemsetAsync(out, 0, (size_t)m * sizeof(int32_t), s));
  return ARBX_OK;
}


__global__ void k_stride_sample(uint32_t* list, int64_t ns, int64_t m) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < ns) list[i] = (uint32_t)(i * m / ns);
}

// Storage query in one traversal (tuning single_pass): a count pass over a
// strided sample of the queries sizes the chunk pool, the MODE_SINGLE
// traversal stages every query's matches in leaf order, a scan of the counts
// gives the offsets, and a copy writes the CRS; queries that found the pool
// exhausted are listed by the traversal and re-run by the fill pass.
arbx_status storage_single(const QueryPlan& plan, bool want_d2, arbx_crs* r, cudaStream_t s) {
  const int64_t m = plan.m;
  constexpr int64_t SAMPLE = 16384;
  const int64_t ns = std::min<int64_t>(m, SAMPLE);
  DevTemp<int32_t> counts(s);
  ARBX_TRY(counts.alloc(m));
  DevTemp<unsigned long long> ctr(s);  // [need, pool chunks taken, overflowed queries]
  ARBX_TRY(ctr.alloc(3));
  ARBX_CUDA(cudaMemsetAsync(ctr.p, 0, 3 * sizeof(unsigned long long), s));
  {
    DevTemp<uint32_t> sample(s);
    ARBX_TRY(sample.alloc(ns));
    ARBX_LAUNCH("stride_sample", s, k_stride_sample<<<(unsigned)((ns + 255) / 256), 256, 0, s>>>(sample.p, ns, m));
    QueryPlan ps = plan;
    ps.order = sample.p;
    ps.nq = m;
    ps.m = ns;
    ARBX_TRY(run_spatial(ps, MODE_COUNT, 0, counts.p, nullptr, nullptr, nullptr, s));
    ARBX_TRY(single_chunks_needed(sample.p, ns, counts.p, ctr.p, s));
  }
  unsigned long long need = 0;
  ARBX_TRY(read_small(ctr.p, &need, sizeof(need), s));
  // the sample mean scaled to all queries, plus a margin; an underestimate
  // only sends the queries that do not fit to the fill pass
  const double est = (double)need * (double)m / (double)ns;
  const int64_t chunks = std::min<int64_t>((int64_t)(est * 1.25) + 1024 + m / 256, INT32_MAX);
  SingleStore ss;
  DevTemp<int32_t> in_idx(s), pool_idx(s), next(s), head(s), ovf(s);
  DevTemp<float> in_d2(s), pool_d2(s);
  ARBX_TRY(in_idx.alloc((size_t)m * SINGLE_INLINE));
  ARBX_TRY(pool_idx.alloc((size_t)chunks * SINGLE_CHUNK));
  if (want_d2) {
    ARBX_TRY(in_d2.alloc((size_t)m * SINGLE_INLINE));
    ARBX_TRY(pool_d2.alloc((size_t)chunks * SINGLE_CHUNK));
  }
  ARBX_TRY(next.alloc(chunks));
  ARBX_TRY(head.alloc(m));
  ARBX_TRY(ovf.alloc(m));
  ss.in_idx = in_idx.p;
  ss.in_d2 = want_d2 ? in_d2.p : nullptr;
  ss.pool_idx = pool_idx.p;
  ss.pool_d2 = want_d2 ? pool_d2.p : nullptr;
  ss.next = next.p;
  ss.head = head.p;
  ss.pool_counter = ctr.p + 1;
  ss.pool_chunks = chunks;
  ss.ovf_list = ovf.p;
  ss.ovf_counter = ctr.p + 2;
  ARBX_TRY(run_spatial_single(plan, ss, counts.p, s));
  ARBX_TRY((exclusive_scan<int32_t, int64_t>(counts.p, r->offsets_dev, m, s)));
  ARBX_TRY(read_small(r->offsets_dev + m, &r->nnz, sizeof(int64_t), s));
  unsigned long long novf = 0;
  ARBX_TRY(read_small(ctr.p + 2, &novf, sizeof(novf), s));
  ARBX_TRY(dev_alloc_t(&r->indices_dev, r->nnz, s));
  if (want_d2) ARBX_TRY(dev_alloc_t(&r->d2_dev, r->nnz, s));
  ARBX_TRY(single_compact(ss, counts.p, r->offsets_dev, m, novf, r->indices_dev, r->d2_dev, s));
  if (novf > 0) {
    QueryPlan pf = plan;
    pf.order = reinterpret_cast<const uint32_t*>(ovf.p);
    pf.nq = m;
    pf.m = (int64_t)novf;
    ARBX_TRY(run_spatial(pf, MODE_FILL, 0, nullptr, r->offsets_dev, r->indices_dev, r->d2_dev, s));
  }
  if (log_enabled() && novf > 0)
    std::fprintf(stderr, "arbx: single pass: %llu of %lld queries re-run (pool %lld chunks, est %.0f)\n", novf,
                 (long long)m, (long long)chunks, est);
  return ARBX_OK;
}

}  // namespace
}  // namespace arbx

namespace arbx {
// arbx_query_stats / arbx_query_count_stats
arbx_status query_stats(arbx_tree tree, const arbx_predicates* pred, const arbx_tuning* tuning, int64_t* stats_host,
                        arbx_stream stream, bool counting, const float* r2s = nullptr) {
  ARBX_TRY(check_pred(tree, pred));
  if (!stats_host) return ARBX_ERR_INVALID;
  if (counting && pred->kind != ARBX_SPHERE && pred->kind != ARBX_BOX_PRED) return ARBX_ERR_INVALID;
  DeviceGuard g(tree->device);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  stats_host[0] = stats_host[1] = stats_host[2] = 0;
  if (tree->n == 0 || pred->m == 0) return ARBX_OK;
  Planned pl;
  ARBX_TRY(make_plan(tree, pred, tuning, s, &pl));
  DevTemp<unsigned long long> st(s);
  ARBX_TRY(st.alloc(3));
  ARBX_CUDA(cudaMemsetAsync(st.p, 0, 3 * sizeof(unsigned long long), s));
  ARBX_TRY(run_stats(pl.p, pred->k, st.p, s, counting, r2s));
  unsigned long long h[3] = {0, 0, 0};
  ARBX_TRY(read_small(st.p, h, sizeof(h), s));
  ARBX_TRY(check_stream(s));
  for (int i = 0; i < 3; ++i) stats_host[i] = (int64_t)h[i];
  return ARBX_OK;
}
}  // namespace arbx

using namespace arbx;

extern "C" {

const char* arbx_status_string(arbx_status s) {
  switch (s) {
    case ARBX_OK: return "ok";
    case ARBX_ERR_INVALID: return "invalid argument";
    case ARBX_ERR_OOM: return "out of device memory";
    case ARBX_ERR_CUDA: return "CUDA error";
    case ARBX_ERR_TIMEOUT: return "device wait timed out";
    case ARBX_ERR_STACK_OVERFLOW: return "traversal stack overflow";
    case ARBX_ERR_UNSUPPORTED: return "unsupported request";
    case ARBX_ERR_NONFINITE: return "non-finite primitive coordinate";
    case ARBX_ERR_CAPACITY: return "output buffer too small";
    case ARBX_ERR_BOUNDS: return "index out of range (checked library)";
    default: return "unknown status";
  }
}

int32_t arbx_abi_version(void) { return 3; }

uint32_t arbx_library_flags(void) { return CHECKED ? ARBX_LIB_CHECKED : 0u; }

arbx_status arbx_build(arbx_tree* out, const arbx_primitives* prim, arbx_stream stream) {
  Range nvtx("arbx_build");
  if (!out || !prim) return ARBX_ERR_INVALID;
  *out = nullptr;
  if (prim->n < 0 || prim->n > MAX_PRIMS) return ARBX_ERR_INVALID;
  if (prim->n > 0 && !prim->data_dev) return ARBX_ERR_INVALID;
  if (prim->kind != ARBX_POINT && prim->kind != ARBX_BOX && prim->kind != ARBX_TRIANGLE) return ARBX_ERR_INVALID;
  if (prim->dim < 1 || prim->dim > 10) return ARBX_ERR_INVALID;
  if (prim->kind == ARBX_TRIANGLE && prim->dim != 3) return ARBX_ERR_INVALID;
  if (prim->dim != 2 && prim->dim != 3 && prim->dim != 6) return ARBX_ERR_UNSUPPORTED;
  if (prim->flags & ~(ARBX_QUANTIZED_NODES | ARBX_WIDE_NODES | ARBX_PARENT_RELATIVE)) return ARBX_ERR_INVALID;
  if ((prim->flags & ARBX_PARENT_RELATIVE) && !(prim->flags & ARBX_QUANTIZED_NODES)) return ARBX_ERR_INVALID;
  if ((prim->flags & ARBX_QUANTIZED_NODES) && prim->kind != ARBX_TRIANGLE) return ARBX_ERR_UNSUPPORTED;
  if ((prim->flags & ARBX_WIDE_NODES) && prim->kind == ARBX_TRIANGLE) return ARBX_ERR_UNSUPPORTED;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  arbx_tree_t* t = new arbx_tree_t;
  cudaGetDevice(&t->device);
  t->kind = prim->kind;
  t->dim = prim->dim;
  t->n = prim->n;
  t->flags = prim->flags;
  for (int a = 0; a < 2 * t->dim; ++a) t->bt.scene_host[a] = a < t->dim ? __builtin_huge_valf() : -__builtin_huge_valf();
  if (prim->n > 0) {
    arbx_status st = check_stream(s);  // surface earlier device errors before this build
    if (st == ARBX_OK) st = build_tree(prim->kind, prim->dim, prim->data_dev, prim->n, prim->flags, &t->bt, s);
    if (st == ARBX_OK) st = check_stream(s);
    if (st != ARBX_OK) {
      arbx_tree_destroy(t);
      return st;
    }
  }
  *out = t;
  return ARBX_OK;
}

arbx_status arbx_tree_info(arbx_tree tree, int64_t* size_out, int32_t* dim_out, float* bounds_out) {
  if (!tree) return ARBX_ERR_INVALID;
  if (size_out) *size_out = tree->n;
  if (dim_out) *dim_out = tree->dim;
  if (bounds_out) std::memcpy(bounds_out, tree->bt.scene_host, 2 * tree->dim * sizeof(float));
  return ARBX_OK;
}

arbx_status arbx_tree_destroy(arbx_tree tree) {
  if (!tree) return ARBX_OK;
  DeviceGuard g(tree->device);
  BuiltTree& b = tree->bt;
  // (qnodes or pnodes is a separate block only when a quantized build stopped early)
  void* ptrs[] = {b.nodes,  b.leaves, b.top[0], b.top[1], b.scene, b.qnodes != b.nodes ? b.qnodes : nullptr,
                  b.pnodes != b.nodes ? b.pnodes : nullptr, b.wide, b.leaf_orig};
  bool any = false;
  for (void* p : ptrs) any = any || p;
  // the caller has no work on the tree in flight; the device-wide sync makes
  // that certain, then the blocks go back to the stream-ordered pool
  if (any) cudaDeviceSynchronize();
  for (void* p : ptrs)
    if (p) cudaFreeAsync(p, 0);
  delete tree;
  return ARBX_OK;
}

arbx_status arbx_query_callback(arbx_tree tree, const arbx_predicates* pred, int32_t cb, int32_t limit,
                                int32_t* out_dev, const arbx_tuning* tuning, arbx_stream stream) {
  Range nvtx("arbx_query_callback");
  ARBX_TRY(check_pred(tree, pred));
  if (!is_spatial(pred->kind)) return ARBX_ERR_INVALID;
  if (cb != ARBX_CB_COUNT && cb != ARBX_CB_COUNT_UP_TO && cb != ARBX_CB_FIRST_HIT) return ARBX_ERR_INVALID;
  if (cb == ARBX_CB_COUNT_UP_TO && limit < 0) return ARBX_ERR_INVALID;
  if (pred->m > 0 && !out_dev) return ARBX_ERR_INVALID;
  DeviceGuard g(tree->device);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (pred->m == 0) return ARBX_OK;
  if (tree->n == 0) return zero_counts(out_dev, pred->m, s);
  Planned pl;
  ARBX_TRY(make_plan(tree, pred, tuning, s, &pl));
  const int mode = cb == ARBX_CB_COUNT ? MODE_COUNT : MODE_COUNT_UP_TO;
  const int32_t lim = cb == ARBX_CB_FIRST_HIT ? 1 : limit;
  return run_spatial(pl.p, mode, lim, out_dev, nullptr, nullptr, nullptr, s);
}

arbx_status arbx_query_offsets(arbx_tree tree, const arbx_predicates* pred, const arbx_tuning* tuning,
                               int64_t* offsets_dev, arbx_stream stream) {
  Range nvtx("arbx_query_offsets");
  ARBX_TRY(check_pred(tree, pred));
  if (!is_spatial(pred->kind)) return ARBX_ERR_INVALID;
  if (!offsets_dev) return ARBX_ERR_INVALID;
  DeviceGuard g(tree->device);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int64_t m = pred->m;
  if (tree->n == 0 || m == 0) {
    ARBX_CUDA(cudaMemsetAsync(offsets_dev, 0, (size_t)(m + 1) * sizeof(int64_t), s));
    return ARBX_OK;
  }
  Planned pl;
  ARBX_TRY(make_plan(tree, pred, tuning, s, &pl));
  DevTemp<int32_t> counts(s);
  ARBX_TRY(counts.alloc(m));
  ARBX_TRY(run_spatial(pl.p, MODE_COUNT, 0, counts.p, nullptr, nullptr, nullptr, s));
  return exclusive_scan<int32_t, int64_t>(counts.p, offsets_dev, m, s);
}

arbx_status arbx_query_fill(arbx_tree tree, const arbx_predicates* pred, const arbx_tuning* tuning,
                            const int64_t* offsets_dev, int32_t* indices_dev, float* d2_dev, arbx_stream stream) {
  Range nvtx("arbx_query_fill");
  ARBX_TRY(check_pred(tree, pred));
  if (!is_spatial(pred->kind)) return ARBX_ERR_INVALID;
  if (!offsets_dev) return ARBX_ERR_INVALID;
  DeviceGuard g(tree->device);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (tree->n == 0 || pred->m == 0) return ARBX_OK;
  Planned pl;
  ARBX_TRY(make_plan(tree, pred, tuning, s, &pl, PlanUse::Storage));
  if (pred->kind != ARBX_RAY_ORDERED)
    return run_spatial(pl.p, MODE_FILL, 0, nullptr, offsets_dev, indices_dev, has_value(pred->kind) ? d2_dev : nullptr,
                       s);
  // ordered_intersect: fill (with t, in a temporary when the caller wants
  // none), then sort every segment by (t, index)
  int64_t nnz = 0;
  ARBX_TRY(read_small(offsets_dev + pred->m, &nnz, sizeof(nnz), s));
  DevTemp<float> tt(s);
  float* t = d2_dev;
  if (!t) {
    ARBX_TRY(tt.alloc(nnz));
    t = tt.p;
  }
  ARBX_TRY(run_spatial(pl.p, MODE_FILL, 0, nullptr, offsets_dev, indices_dev, t, s));
  return sort_segments_by_t(offsets_dev, pred->m, nnz, indices_dev, t, s);
}

arbx_status arbx_query_knn(arbx_tree tree, const arbx_predicates* pred, const arbx_tuning* tuning,
                           int32_t* indices_dev, float* d2_dev, arbx_stream stream) {
  Range nvtx("arbx_query_knn");
  ARBX_TRY(check_pred(tree, pred));
  if (pred->kind != ARBX_NEAREST) return ARBX_ERR_INVALID;
  const int64_t kk = std::min<int64_t>(pred->k, tree->n);
  if (pred->m > 0 && kk > 0 && !indices_dev) return ARBX_ERR_INVALID;
  DeviceGuard g(tree->device);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (kk == 0 || pred->m == 0) return ARBX_OK;
  Planned pl;
  ARBX_TRY(make_plan(tree, pred, tuning, s, &pl));
  return run_knn(pl.p, pred->k, (int)kk, indices_dev, d2_dev, s);
}

arbx_status arbx_query_ray_nearest(arbx_tree tree, const arbx_predicates* pred, const arbx_tuning* tuning,
                                   int32_t* hit_dev, float* t_dev, arbx_stream stream) {
  Range nvtx("arbx_query_ray_nearest");
  ARBX_TRY(check_pred(tree, pred));
  if (pred->kind != ARBX_RAY_NEAREST) return ARBX_ERR_INVALID;
  if (pred->m > 0 && (!hit_dev || !t_dev)) return ARBX_ERR_INVALID;
  DeviceGuard g(tree->device);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (pred->m == 0) return ARBX_OK;
  const int64_t kk = pred->k > 1 ? pred->k : 1;
  if (tree->n == 0) {
    ARBX_CUDA(cudaMemsetAsync(hit_dev, 0xff, (size_t)(pred->m * kk) * sizeof(int32_t), s));
    std::vector<float> inf((size_t)(pred->m * kk), __builtin_huge_valf());
    ARBX_CUDA(cudaMemcpyAsync(t_dev, inf.data(), inf.size() * sizeof(float), cudaMemcpyHostToDevice, s));
    ARBX_CUDA(cudaStreamSynchronize(s));
    return ARBX_OK;
  }
  Planned pl;
  ARBX_TRY(make_plan(tree, pred, tuning, s, &pl));
  return run_ray(pl.p, (int)kk, hit_dev, t_dev, s);
}


arbx_status arbx_query_crs(arbx_tree tree, const arbx_predicates* pred, int32_t want_d2, const arbx_tuning* tuning,
                           arbx_crs* out, arbx_stream stream) {
  Range nvtx("arbx_query_crs");
  if (!out) return ARBX_ERR_INVALID;
  std::memset(out, 0, sizeof(*out));
  ARBX_TRY(check_pred(tree, pred));
  DeviceGuard g(tree->device);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int64_t m = pred->m;
  arbx_crs r;
  std::memset(&r, 0, sizeof(r));
  r.m = m;
  auto fail = [&](arbx_status st) {
    arbx_crs_free(&r, stream);
    return st;
  };
  arbx_status st = dev_alloc_t(&r.offsets_dev, m + 1, s);
  if (st != ARBX_OK) return fail(st);
  if (pred->kind == ARBX_NEAREST) {
    const int64_t kk = std::min<int64_t>(pred->k, tree->n);
    r.nnz = m * kk;
    ARBX_LAUNCH("iota_offsets", s, k_iota_offsets<<<(unsigned)((m + 256) / 256), 256, 0, s>>>(r.offsets_dev, m, kk));
    if ((st = dev_alloc_t(&r.indices_dev, r.nnz, s)) != ARBX_OK) return fail(st);
    if (want_d2 && (st = dev_alloc_t(&r.d2_dev, r.nnz, s)) != ARBX_OK) return fail(st);
    if ((st = arbx_query_knn(tree, pred, tuning, r.indices_dev, r.d2_dev, stream)) != ARBX_OK) return fail(st);
  } else if (pred->kind == ARBX_RAY_NEAREST) {
    // rows of kk hits (padded with -1), compacted to the hits found
    const int64_t kk = pred->k > 1 ? pred->k : 1;
    DevTemp<int32_t> hit(s), counts(s);
    DevTemp<float> t(s);
    if ((st = hit.alloc(m * kk)) != ARBX_OK || (st = t.alloc(m * kk)) != ARBX_OK || (st = counts.alloc(m)) != ARBX_OK)
      return fail(st);
    if ((st = arbx_query_ray_nearest(tree, pred, tuning, hit.p, t.p, stream)) != ARBX_OK) return fail(st);
    const unsigned grid = (unsigned)((m + 255) / 256);
    if (m > 0) ARBX_LAUNCH("hit_counts", s, k_hit_counts<<<grid, 256, 0, s>>>(hit.p, m, (int)kk, counts.p));
    if ((st = exclusive_scan<int32_t, int64_t>(counts.p, r.offsets_dev, m, s)) != ARBX_OK) return fail(st);
    if ((st = read_small(r.offsets_dev + m, &r.nnz, sizeof(int64_t), s)) != ARBX_OK) return fail(st);
    if ((st = dev_alloc_t(&r.indices_dev, r.nnz, s)) != ARBX_OK) return fail(st);
    if (want_d2 && (st = dev_alloc_t(&r.d2_dev, r.nnz, s)) != ARBX_OK) return fail(st);
    if (m > 0)
      ARBX_LAUNCH("hit_compact", s, k_hit_compact<<<grid, 256, 0, s>>>(hit.p, t.p, m, (int)kk, r.offsets_dev,
                                                                        r.indices_dev, r.d2_dev));
  } else if (tree->n == 0 || m == 0) {
    ARBX_CUDA(cudaMemsetAsync(r.offsets_dev, 0, (size_t)(m + 1) * sizeof(int64_t), s));
  } else {
    Planned pl;
    if ((st = make_plan(tree, pred, tuning, s, &pl, PlanUse::Storage)) != ARBX_OK) return fail(st);
    if (pl.p.single_pass) {
      st = storage_single(pl.p, has_value(pred->kind) && (want_d2 || pred->kind == ARBX_RAY_ORDERED), &r, s);
      if (st == ARBX_OK && pred->kind == ARBX_RAY_ORDERED)
        st = sort_segments_by_t(r.offsets_dev, m, r.nnz, r.indices_dev, r.d2_dev, s);
      if (st == ARBX_OK && pred->kind == ARBX_RAY_ORDERED && !want_d2) {
        dev_free(r.d2_dev, s);
        r.d2_dev = nullptr;
      }
      if (st == ARBX_OK) {
        if ((st = check_stream(s)) != ARBX_OK) return fail(st);
        *out = r;
        return ARBX_OK;
      }
      if (st != ARBX_ERR_OOM) return fail(st);
      // the staging did not fit: the two-pass form needs less memory
      dev_free(r.indices_dev, s);
      dev_free(r.d2_dev, s);
      r.indices_dev = nullptr;
      r.d2_dev = nullptr;
      r.nnz = 0;
    }
    // count -> scan -> fill, sharing one query order
    {
      DevTemp<int32_t> counts(s);
      if ((st = counts.alloc(m)) != ARBX_OK) return fail(st);
      if ((st = run_spatial(pl.p, MODE_COUNT, 0, counts.p, nullptr, nullptr, nullptr, s)) != ARBX_OK) return fail(st);
      if ((st = exclusive_scan<int32_t, int64_t>(counts.p, r.offsets_dev, m, s)) != ARBX_OK) return fail(st);
    }
    if ((st = read_small(r.offsets_dev + m, &r.nnz, sizeof(int64_t), s)) != ARBX_OK) return fail(st);
    if ((st = dev_alloc_t(&r.indices_dev, r.nnz, s)) != ARBX_OK) return fail(st);
    // ordered_intersect sorts by t, so it computes t even when not returned
    const bool value = has_value(pred->kind) && (want_d2 || pred->kind == ARBX_RAY_ORDERED);
    if (value && (st = dev_alloc_t(&r.d2_dev, r.nnz, s)) != ARBX_OK) return fail(st);
    if ((st = run_spatial(pl.p, MODE_FILL, 0, nullptr, r.offsets_dev, r.indices_dev, r.d2_dev, s)) != ARBX_OK) return fail(st);
    if (pred->kind == ARBX_RAY_ORDERED) {
      if ((st = sort_segments_by_t(r.offsets_dev, m, r.nnz, r.indices_dev, r.d2_dev, s)) != ARBX_OK) return fail(st);
      if (!want_d2) {
        dev_free(r.d2_dev, s);
        r.d2_dev = nullptr;
      }
    }
  }
  if ((st = check_stream(s)) != ARBX_OK) return fail(st);
  *out = r;
  return ARBX_OK;
}

// Device memory a new allocation can take now: free memory plus the unused
// part of the stream-ordered pool the library allocates from.
int64_t available_device_bytes() {
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int64_t slack = 0;
  int dev = 0;
  cudaMemPool_t pool;
  if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t res = 0, used = 0;
    if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &res) == cudaSuccess &&
        cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used) == cudaSuccess && res > used)
      slack = (int64_t)(res - used);
  }
  return (int64_t)fr + slack;
}

__global__ void k_chunk_offsets(const int64_t* __restrict__ off, int64_t lo, int64_t mc, int64_t* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i <= mc) out[i] = off[lo + i] - off[lo];
}

arbx_status arbx_query_crs_host(arbx_tree tree, const arbx_predicates* pred, int32_t want_d2,
                                const arbx_tuning* tuning, int64_t* offsets_host, int32_t* indices_host,
                                float* d2_host, int64_t capacity, int64_t chunk_bytes, int64_t* nnz_out,
                                arbx_stream stream) {
  Range nvtx("arbx_query_crs_host");
  ARBX_TRY(check_pred(tree, pred));
  if (!is_spatial(pred->kind)) return ARBX_ERR_INVALID;
  if (!offsets_host || capacity < 0 || chunk_bytes < 0) return ARBX_ERR_INVALID;
  if (capacity > 0 && !indices_host) return ARBX_ERR_INVALID;
  DeviceGuard g(tree->device);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int64_t m = pred->m;
  if (nnz_out) *nnz_out = 0;
  if (tree->n == 0 || m == 0) {
    for (int64_t i = 0; i <= m; ++i) offsets_host[i] = 0;
    return ARBX_OK;
  }
  // 1. counts and global offsets over all queries (one query order)
  DevTemp<int64_t> off(s);
  ARBX_TRY(off.alloc(m + 1));
  {
    Planned pl;
    ARBX_TRY(make_plan(tree, pred, tuning, s, &pl));
    DevTemp<int32_t> counts(s);
    ARBX_TRY(counts.alloc(m));
    ARBX_TRY(run_spatial(pl.p, MODE_COUNT, 0, counts.p, nullptr, nullptr, nullptr, s));
    ARBX_TRY((exclusive_scan<int32_t, int64_t>(counts.p, off.p, m, s)));
  }
  ARBX_CUDA(cudaMemcpyAsync(offsets_host, off.p, (size_t)(m + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  ARBX_TRY(check_stream(s));
  const int64_t nnz = offsets_host[m];
  if (nnz_out) *nnz_out = nnz;
  if (nnz > capacity) return ARBX_ERR_CAPACITY;
  if (nnz == 0) return ARBX_OK;
  // 2. query ranges whose results fit the chunk budget, filled and copied one after another
  const bool value = has_value(pred->kind) && (want_d2 || pred->kind == ARBX_RAY_ORDERED);
  const int64_t per_entry = value ? 8 : 4;
  int64_t budget = chunk_bytes > 0 ? chunk_bytes : std::max<int64_t>((available_device_bytes() - (int64_t(1) << 30)) / 2, 0);
  int64_t cap_entries = std::max<int64_t>(budget / per_entry, 1);
  cap_entries = std::min(cap_entries, nnz);
  int64_t widest = 0;  // the largest single query
  for (int64_t i = 0; i < m; ++i) widest = std::max(widest, offsets_host[i + 1] - offsets_host[i]);
  const int64_t buf_entries = std::max(cap_entries, widest);
  DevTemp<int32_t> cidx(s);
  DevTemp<float> cd2(s);
  DevTemp<int64_t> coff(s);
  ARBX_TRY(cidx.alloc(buf_entries));
  if (value) ARBX_TRY(cd2.alloc(buf_entries));
  const int stride = pred->kind == ARBX_BOX_PRED ? 2 * pred->dim : (is_ray_all(pred->kind) ? 6 : pred->dim);
  int64_t lo = 0;
  while (lo < m) {
    // the longest range [lo, hi) whose entries fit; at least one query
    int64_t a = lo + 1, b = m;
    while (a < b) {
      const int64_t mid = (a + b + 1) / 2;
      if (offsets_host[mid] - offsets_host[lo] <= cap_entries) a = mid;
      else b = mid - 1;
    }
    const int64_t hi = a;
    const int64_t mc = hi - lo;
    const int64_t ne = offsets_host[hi] - offsets_host[lo];
    if (ne > 0) {
      arbx_predicates sub = *pred;
      sub.m = mc;
      sub.data_dev = pred->data_dev + lo * stride;
      sub.radii_dev = pred->radii_dev ? pred->radii_dev + lo : nullptr;
      sub.order_dev = nullptr;  // a caller's order covers all m queries
      Planned pl;
      ARBX_TRY(make_plan(tree, &sub, tuning, s, &pl, PlanUse::Storage));
      ARBX_TRY(coff.alloc(mc + 1));
      ARBX_LAUNCH("chunk_offsets", s,
                  k_chunk_offsets<<<(unsigned)((mc + 256) / 256), 256, 0, s>>>(off.p, lo, mc, coff.p));
      ARBX_TRY(run_spatial(pl.p, MODE_FILL, 0, nullptr, coff.p, cidx.p, value ? cd2.p : nullptr, s));
      if (pred->kind == ARBX_RAY_ORDERED) ARBX_TRY(sort_segments_by_t(coff.p, mc, ne, cidx.p, cd2.p, s));
      const int64_t at = offsets_host[lo];
      ARBX_CUDA(cudaMemcpyAsync(indices_host + at, cidx.p, (size_t)ne * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
      if (want_d2 && d2_host && value)
        ARBX_CUDA(cudaMemcpyAsync(d2_host + at, cd2.p, (size_t)ne * sizeof(float), cudaMemcpyDeviceToHost, s));
      ARBX_TRY(check_stream(s));  // the buffers are reused by the next range
      dev_free(coff.p, s);
      coff.p = nullptr;
    }
    lo = hi;
  }
  return ARBX_OK;
}

arbx_status arbx_crs_free(arbx_crs* crs, arbx_stream stream) {
  if (!crs) return ARBX_ERR_INVALID;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  dev_free(crs->offsets_dev, s);
  dev_free(crs->indices_dev, s);
  dev_free(crs->d2_dev, s);
  std::memset(crs, 0, sizeof(*crs));
  return ARBX_OK;
}


arbx_status arbx_query_stats(arbx_tree tree, const arbx_predicates* pred, const arbx_tuning* tuning,
                             int64_t* stats_host, arbx_stream stream) {
  Range nvtx("arbx_query_stats");
  return arbx::query_stats(tree, pred, tuning, stats_host, stream, false);
}

arbx_status arbx_query_count_stats(arbx_tree tree, const arbx_predicates* pred, const arbx_tuning* tuning,
                                   int64_t* stats_host, arbx_stream stream) {
  Range nvtx("arbx_query_count_stats");
  return arbx::query_stats(tree, pred, tuning, stats_host, stream, true);
}

arbx_status arbx_query_stats_r2(arbx_tree tree, const arbx_predicates* pred, const arbx_tuning* tuning,
                                const float* r2_dev, int64_t* stats_host, arbx_stream stream) {
  Range nvtx("arbx_query_stats_r2");
  if (!pred || pred->kind != ARBX_SPHERE || (pred->m > 0 && !r2_dev)) return ARBX_ERR_INVALID;
  if (tree && tree->kind == ARBX_TRIANGLE) return ARBX_ERR_UNSUPPORTED;
  arbx_predicates p = *pred;
  p.radii_dev = nullptr;
  p.radius = 0.0f;  // unused: every query's squared radius comes from r2_dev
  return arbx::query_stats(tree, &p, tuning, stats_host, stream, false, r2_dev);
}

arbx_status arbx_query_order(arbx_tree tree, const arbx_predicates* pred, uint32_t* order_dev, arbx_stream stream) {
  Range nvtx("arbx_query_order");
  ARBX_TRY(check_pred(tree, pred));
  if (pred->m > 0 && !order_dev) return ARBX_ERR_INVALID;
  DeviceGuard g(tree->device);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (pred->m == 0) return ARBX_OK;
  if (pred->m == 1 || tree->n == 0) {
    // nothing to sort by (one query, or an empty tree with no scene box): input order
    ARBX_LAUNCH("stride_sample", s,
                k_stride_sample<<<(unsigned)((pred->m + 255) / 256), 256, 0, s>>>(order_dev, pred->m, pred->m));
    return ARBX_OK;
  }
  arbx_tuning tu{0, 0, -1, 0, -1, -1, -1, 0, -1, -1, 0};  // the plan itself sorts nothing
  Planned pl;
  arbx_predicates p = *pred;
  p.order_dev = nullptr;
  ARBX_TRY(make_plan(tree, &p, &tu, s, &pl));
  uint32_t* order = nullptr;
  return query_order(pl.p, tree->bt.scene, &order, s, order_dev);
}

arbx_status arbx_stream_check(arbx_stream stream) { return check_stream(reinterpret_cast<cudaStream_t>(stream)); }

arbx_status arbx_tree_export(arbx_tree tree, void* nodes_host, int64_t nodes_cap, void* leaves_host,
                             int64_t leaves_cap, int64_t* bytes_out) {
  if (!tree) return ARBX_ERR_INVALID;
  DeviceGuard g(tree->device);
  const BuiltTree& b = tree->bt;
  const int64_t nb = b.nnodes * b.node_stride;
  const int64_t lb = b.leaves ? b.n * (int64_t)sizeof(TriLeaf) : 0;
  if (bytes_out) {
    bytes_out[0] = nb;
    bytes_out[1] = lb;
    bytes_out[2] = b.node_stride;
    bytes_out[3] = b.leaves ? (int64_t)sizeof(TriLeaf) : 0;
    bytes_out[4] = b.root;
  }
  ARBX_CUDA(cudaDeviceSynchronize());
  if (nodes_host && b.nodes) {
    if (nodes_cap < nb) return ARBX_ERR_CAPACITY;
    ARBX_CUDA(cudaMemcpy(nodes_host, b.nodes, (size_t)nb, cudaMemcpyDeviceToHost));
  }
  if (leaves_host && b.leaves) {
    if (leaves_cap < lb) return ARBX_ERR_CAPACITY;
    ARBX_CUDA(cudaMemcpy(leaves_host, b.leaves, (size_t)lb, cudaMemcpyDeviceToHost));
  }
  return ARBX_OK;
}

arbx_status arbx_profile_enable(int32_t on) {
  g_prof_on.store(on != 0);
  return ARBX_OK;
}

arbx_status arbx_profile_read(char* names_host, int64_t* launches_host, double* ms_host, int32_t cap,
                              int32_t* count_out) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  prof_collect_locked();
  const int32_t nt = (int32_t)g_prof_totals.size();
  for (int32_t i = 0; i < nt && i < cap; ++i) {
    if (names_host) {
      std::strncpy(names_host + 64 * i, g_prof_totals[i].first.c_str(), 63);
      names_host[64 * i + 63] = 0;
    }
    if (launches_host) launches_host[i] = g_prof_totals[i].second.launches;
    if (ms_host) ms_host[i] = g_prof_totals[i].second.ms;
  }
  if (count_out) *count_out = nt;
  return ARBX_OK;
}

arbx_status arbx_profile_reset(void) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  prof_collect_locked();
  g_prof_totals.clear();
  return ARBX_OK;
}

int64_t arbx_launch_count(void) { return g_launches.load(); }

arbx_status arbx_debug_fail_allocs(int64_t after, int64_t count) {
  if (after < 0 || count < 0) return ARBX_ERR_INVALID;
  g_fail_count.store(0);
  g_fail_after.store(after);
  g_fail_count.store(count);
  return ARBX_OK;
}

arbx_status arbx_memory_trim(int64_t keep_bytes) {
  if (keep_bytes < 0) return ARBX_ERR_INVALID;
  cudaMemPool_t pool;
  ARBX_CUDA(cudaDeviceGetDefaultMemPool(&pool, current_device()));
  ARBX_CUDA(cudaDeviceSynchronize());
  ARBX_CUDA(cudaMemPoolTrimTo(pool, (size_t)keep_bytes));
  return ARBX_OK;
}

arbx_status arbx_dbscan(const float* points_dev, int64_t n, int32_t dim, float eps, int32_t min_pts,
                        int32_t* labels_dev, int64_t* n_clusters_out, arbx_stream stream) {
  Range nvtx("arbx_dbscan");
  if (n < 0 || n > MAX_PRIMS || (n > 0 && (!points_dev || !labels_dev))) return ARBX_ERR_INVALID;
  if (!finite_f(eps) || eps < 0.0f) return ARBX_ERR_INVALID;
  if (dim != 2 && dim != 3 && dim != 6) return dim >= 1 && dim <= 10 ? ARBX_ERR_UNSUPPORTED : ARBX_ERR_INVALID;
  if (n_clusters_out) *n_clusters_out = 0;
  if (n == 0) return ARBX_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  arbx_primitives prim{ARBX_POINT, dim, n, points_dev, 0u};
  arbx_tree tree = nullptr;
  ARBX_TRY(arbx_build(&tree, &prim, stream));
  struct Guard {
    arbx_tree t;
    ~Guard() { arbx_tree_destroy(t); }
  } guard{tree};
  DeviceGuard g(tree->device);
  arbx_predicates pred{ARBX_SPHERE, dim, n, points_dev, nullptr, eps, 0};
  Planned pl;
  ARBX_TRY(make_plan(tree, &pred, nullptr, s, &pl));
  // core points: the neighbourhood (the point included) holds min_pts points;
  // the count stops there
  const int32_t lim = min_pts > 1 ? min_pts : 1;
  DevTemp<int32_t> counts(s);
  ARBX_TRY(counts.alloc(n));
  ARBX_TRY(run_spatial(pl.p, MODE_COUNT_UP_TO, lim, counts.p, nullptr, nullptr, nullptr, s));
  int64_t nc = 0;
  ARBX_TRY(run_dbscan(pl.p, counts.p, lim, labels_dev, &nc, s));
  ARBX_TRY(check_stream(s));
  if (n_clusters_out) *n_clusters_out = nc;
  return ARBX_OK;
}

arbx_status arbx_autotune(arbx_tree tree, const arbx_predicates* pred, int64_t sample, arbx_tuning* best_out,
                          double* best_ms_out, arbx_stream stream) {
  Range nvtx("arbx_autotune");
  ARBX_TRY(check_pred(tree, pred));
  if (!best_out) return ARBX_ERR_INVALID;
  DeviceGuard g(tree->device);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  arbx_predicates p = *pred;
  p.m = std::min<int64_t>(pred->m, sample > 0 ? sample : (int64_t(1) << 20));
  p.order_dev = nullptr;  // a caller's order covers all m queries, not the sample
  if (tree->n == 0 || p.m == 0) {
    *best_out = arbx_tuning{0, -1, -1, 0, -1, -1, -1, 0, -1, -1, 0};
    if (best_ms_out) *best_ms_out = 0.0;
    return ARBX_OK;
  }
  const int64_t kk = p.kind == ARBX_NEAREST ? std::min<int64_t>(p.k, tree->n)
                     : p.kind == ARBX_RAY_NEAREST ? std::max<int64_t>(p.k, 1) : 1;
  DevTemp<int32_t> out_i(s);
  DevTemp<float> out_f(s);
  ARBX_TRY(out_i.alloc(p.m * kk));
  ARBX_TRY(out_f.alloc(p.m * kk));
  // spatial and ray-intersect predicates are timed as the storage query they
  // mostly serve: count -> scan -> fill into buffers sized once here
  const bool storage = is_spatial(p.kind);
  DevTemp<int64_t> offsets(s);
  DevTemp<int32_t> fill_i(s);
  DevTemp<float> fill_d2(s);
  if (storage) {
    ARBX_TRY(offsets.alloc(p.m + 1));
    Planned pl;
    ARBX_TRY(make_plan(tree, &p, nullptr, s, &pl));
    ARBX_TRY(run_spatial(pl.p, MODE_COUNT, 0, out_i.p, nullptr, nullptr, nullptr, s));
    ARBX_TRY((exclusive_scan<int32_t, int64_t>(out_i.p, offsets.p, p.m, s)));
    int64_t nnz = 0;
    ARBX_TRY(read_small(offsets.p + p.m, &nnz, sizeof(nnz), s));
    ARBX_TRY(fill_i.alloc(nnz));
    if (has_value(p.kind)) ARBX_TRY(fill_d2.alloc(nnz));
  }
  cudaEvent_t e0, e1;
  ARBX_CUDA(cudaEventCreate(&e0));
  ARBX_CUDA(cudaEventCreate(&e1));
  // one candidate: plan (including the query sort when on) + the traversal(s)
  auto run = [&](const arbx_tuning& tu) -> arbx_status {
    Planned pl;
    ARBX_TRY(make_plan(tree, &p, &tu, s, &pl));
    if (p.kind == ARBX_NEAREST) return run_knn(pl.p, p.k, (int)kk, out_i.p, out_f.p, s);
    if (p.kind == ARBX_RAY_NEAREST) return run_ray(pl.p, (int)kk, out_i.p, out_f.p, s);
    ARBX_TRY(run_spatial(pl.p, MODE_COUNT, 0, out_i.p, nullptr, nullptr, nullptr, s));
    ARBX_TRY((exclusive_scan<int32_t, int64_t>(out_i.p, offsets.p, p.m, s)));
    return run_spatial(pl.p, MODE_FILL, 0, nullptr, offsets.p, fill_i.p, fill_d2.p, s);
  };
  arbx_tuning best{0, -1, -1, 0, -1, -1, -1, 0, -1, -1, 0};
  double best_ms = 1e300;
  arbx_status st = ARBX_OK;
  const bool spatial = (p.kind == ARBX_SPHERE || p.kind == ARBX_BOX_PRED) && !tree->bt.quantized;  // stackless applies
  // lanes per query: nearest predicates whose list fits one lane (k <= 32),
  // groups of up to min(8, K) lanes, K the list size (k rounded up to a power of two)
  int min_lanes = 1, max_lanes = 1;
  if (p.kind == ARBX_NEAREST) {
    int K = 1;
    while (K < p.k) K <<= 1;
    if (K <= 32) {
      max_lanes = std::min(8, K);
    } else {  // lists over lane groups of 32, 16 or 8 keys per lane
      min_lanes = K / 32;
      max_lanes = K / 8;
    }
  }
  // four-wide records: nearest and counting traversals of point and box trees,
  // with no staged top levels (the wide kernels stage none)
  const bool widen = tree->bt.wide && (p.kind == ARBX_NEAREST || p.kind == ARBX_SPHERE || p.kind == ARBX_BOX_PRED);
  std::vector<arbx_tuning> cands;
  for (int block : {128, 256})
    for (int sort : {0, 1})
      for (int top : {0, 255, 1023})
        for (int refill : {0, 1})
          for (int sl = 0; sl <= (spatial ? 1 : 0); ++sl)
            for (int L = min_lanes; L <= max_lanes; L <<= 1)
              for (int wd = 0; wd <= (widen && top == 0 && sl == 0 && L == 1 ? 1 : 0); ++wd)
                for (int pk = 0; pk <= (p.kind == ARBX_NEAREST && top == 0 && L == 1 && wd == 0 && refill == 0 ? 1 : 0);
                     ++pk)
                  for (int run : {1, 4, 8}) {
                    // lane runs: nearest, no packets; they hand out work their own
                    // way, so lane refill pairs with runs of 1 only
                    const bool runs_apply = p.kind == ARBX_NEAREST && pk == 0;
                    if (run > 1 && (!runs_apply || refill == 1)) continue;
                    cands.push_back(arbx_tuning{block, sort, top, 0, refill, sl, 0, L, wd, pk, runs_apply ? run : 0});
                  }
  // every candidate: a warm-up run and one timed run; then the four fastest
  // again, three timed runs each, the median deciding (candidates within a
  // few percent of each other would otherwise be picked by timing noise)
  auto time_once = [&](const arbx_tuning& tu, float* ms) -> arbx_status {
    cudaEventRecord(e0, s);
    ARBX_TRY(run(tu));
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(ms, e0, e1);
    return ARBX_OK;
  };
  std::vector<std::pair<float, size_t>> first;
  for (size_t ci = 0; ci < cands.size() && st == ARBX_OK; ++ci) {
    float ms = 0.0f;
    if ((st = run(cands[ci])) != ARBX_OK) break;  // warm-up
    if ((st = time_once(cands[ci], &ms)) != ARBX_OK) break;
    first.emplace_back(ms, ci);
  }
  std::sort(first.begin(), first.end());
  for (size_t r = 0; r < first.size() && r < 4 && st == ARBX_OK; ++r) {
    float t3[3];
    for (int rep = 0; rep < 3 && st == ARBX_OK; ++rep) st = time_once(cands[first[r].second], &t3[rep]);
    if (st != ARBX_OK) break;
    std::sort(t3, t3 + 3);
    if (t3[1] < best_ms) {
      best_ms = t3[1];
      best = cands[first[r].second];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st == ARBX_OK) st = check_stream(s);
  if (st != ARBX_OK) return st;
  best.single_pass = -1;  // not searched: the storage form stays the default
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[tune_key(tree, pred)] = best;
  }
  *best_out = best;
  if (best_ms_out) *best_ms_out = best_ms;
  return ARBX_OK;
}

arbx_status arbx_autotune_save(const char* path) {
  if (!path) return ARBX_ERR_INVALID;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  FILE* f = std::fopen(path, "w");
  if (!f) return ARBX_ERR_INVALID;
  std::fprintf(f, "# gpu kind dim k n_bucket m_bucket quantized block sort_queries top_levels grid_per_sm warp_refill "
               "stackless lanes_per_query wide_nodes warp_packets query_runs\n");
  for (const auto& kv : g_tune) {
    const TuneKey& k = kv.first;
    const arbx_tuning& t = kv.second;
    std::fprintf(f, "%s %d %d %d %d %d %d %d %d %d %d %d %d %d %d %d %d\n", k.gpu.c_str(), k.kind, k.dim, k.k, k.nb,
                 k.mb, k.quantized, t.block, t.sort_queries, t.top_levels, t.grid_per_sm, t.warp_refill, t.stackless,
                 t.lanes_per_query, t.wide_nodes, t.warp_packets, t.query_runs);
  }
  forest_records_save(f);
  std::fclose(f);
  return ARBX_OK;
}

arbx_status arbx_autotune_load(const char* path) {
  if (!path) return ARBX_ERR_INVALID;
  FILE* f = std::fopen(path, "r");
  if (!f) return ARBX_ERR_INVALID;
  char line[512];
  std::lock_guard<std::mutex> lk(g_tune_mu);
  while (std::fgets(line, sizeof(line), f)) {
    if (line[0] == '#') continue;
    if (std::strncmp(line, "forest ", 7) == 0) {
      forest_record_load(line);  // an invalid forest line is skipped
      continue;
    }
    char gpu[256];
    TuneKey k;
    arbx_tuning t{0, -1, -1, 0, -1, -1, -1, 0, -1, -1, 0};
    // 17 fields; shorter lines of 13 to 16 (no lanes_per_query / wide_nodes / warp_packets / query_runs) keep
    // the defaults
    if (std::sscanf(line, "%255s %d %d %d %d %d %d %d %d %d %d %d %d %d %d %d %d", gpu, &k.kind, &k.dim, &k.k, &k.nb,
                    &k.mb, &k.quantized, &t.block, &t.sort_queries, &t.top_levels, &t.grid_per_sm, &t.warp_refill,
                    &t.stackless, &t.lanes_per_query, &t.wide_nodes, &t.warp_packets, &t.query_runs) >= 13) {
      k.gpu = gpu;
      Tuning check;
      if (read_tuning(&t, &check) == ARBX_OK) g_tune[k] = t;
    }
  }
  std::fclose(f);
  return ARBX_OK;
}

arbx_status arbx_autotune_clear(void) {
  forest_records_clear();
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune.clear();
  return ARBX_OK;
}

}  // extern "C"
