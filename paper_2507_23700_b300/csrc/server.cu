// Serving runtime: trees stay resident on the device while a stream of query
// requests of mixed size and kind is admitted and executed with overlap
// (continuous batching: a request that arrives while others run starts as soon
// as a slot and enough device memory are free).
//
// Structure: S slots, each a worker thread with its own CUDA stream.  Workers
// take requests from one FIFO queue.  The queue head is admitted when its
// memory estimate (query order, counts, offsets, and for nearest queries the
// k results per query) fits next to the reservations of the requests already
// running within the budget -- the caller's budget, capped by the device
// memory that was available when the server was created -- and also fits the
// device memory available at that moment (free memory plus the unused part of
// the stream-ordered pool, read at admission, less a reserve).  A radius
// request reserves its output (8 bytes per match) after its count pass; if
// that does not fit it waits for memory, and when every running request is
// waiting the oldest proceeds over budget, so the server never deadlocks (an
// allocation that then fails ends that request with ARBX_ERR_OOM; the server
// keeps serving).  Work on different slots overlaps on the GPU.
// Results stay in device memory until the client releases them.  Latency is
// measured from the request's arrival time to the end of its device work.
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "tree.cuh"

namespace {

using Clock = std::chrono::steady_clock;

bool server_log() {
  static const bool on = [] {
    const char* v = std::getenv("ARBX_LOG");
    return v && *v && std::strcmp(v, "0") != 0;
  }();
  return on;
}

#define SLOG(...)                                 \
  do {                                            \
    if (server_log()) {                           \
      std::fprintf(stderr, "arbx server: " __VA_ARGS__); \
      std::fputc('\n', stderr);                  \
    }                                             \
  } while (0)

constexpr double MEMORY_WAIT_LIMIT_S = 300.0;  // a request waits this long for memory, then runs anyway
constexpr int64_t HBM_RESERVE = int64_t(1) << 30;  // device memory left to other work at admission

// Device memory a new reservation can take now on the current device: free
// memory plus what the default stream-ordered pool (the library's allocator)
// holds unused, less HBM_RESERVE.  INT64_MAX when it cannot be read.
int64_t device_available() {
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
    cudaGetLastError();
    return INT64_MAX;
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
  return (int64_t)fr + slack - HBM_RESERVE;
}

struct Ticket {
  arbx_request req;
  double arrival = 0.0;
  double done_at = 0.0;
  bool done = false;
  bool waiting_memory = false;
  int64_t reserved = 0;
  arbx_result res;
};

}  // namespace

struct arbx_server_t {
  int device = 0;
  int64_t budget = 0;  // min(caller's budget, device memory available at creation)
  Clock::time_point t0;
  std::vector<arbx_tree> trees;
  std::vector<std::thread> workers;
  std::vector<cudaStream_t> streams;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<uint64_t> queue;
  std::unordered_map<uint64_t, Ticket> tickets;
  uint64_t next_ticket = 1;
  int64_t reserved = 0;
  int running = 0;
  int waiting = 0;
  bool stop = false;
  // statistics
  std::vector<double> latencies;
  int64_t queries_done = 0;
  double first_arrival = -1.0, last_done = 0.0;

  double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
  // a reservation of `bytes` fits the budget beside the running ones and the
  // device memory available now (called with mu held, on a worker thread
  // whose current device is the server's)
  bool fits(int64_t bytes) const { return reserved + bytes <= budget && bytes <= device_available(); }
};

namespace {

int64_t estimate_bytes(const arbx_request& r, int64_t n) {
  const int64_t m = r.m;
  int64_t b = m * 16 + 4096;  // query order keys/values
  if (r.callback >= 0) return b + m * 4;
  if (r.kind == ARBX_NEAREST) return b + m * std::min<int64_t>(r.k, n) * 8 + (m + 1) * 8;
  return b + m * 4 + (m + 1) * 8;  // counts + offsets; matches reserved after the count pass
}

// Run one request on `s`.  Called without the server lock.
arbx_status run_request(arbx_server_t* sv, Ticket& tk, cudaStream_t s, uint64_t id) {
  const arbx_request& r = tk.req;
  arbx_tree t = sv->trees[r.tree_id];
  arbx_predicates p;
  std::memset(&p, 0, sizeof(p));
  p.kind = r.kind;
  p.dim = t->dim;
  p.m = r.m;
  p.data_dev = r.queries_dev;
  p.radius = r.radius;
  p.k = r.k;
  arbx_result& out = tk.res;
  out.m = r.m;
  arbx_stream st = reinterpret_cast<arbx_stream>(s);
  if (r.callback >= 0) {
    if (arbx::dev_alloc_t(&out.counts_dev, std::max<int64_t>(r.m, 1), s) != ARBX_OK) return ARBX_ERR_OOM;
    ARBX_TRY(arbx_query_callback(t, &p, r.callback, r.limit, out.counts_dev, nullptr, st));
    return arbx_stream_check(st);
  }
  if (r.kind == ARBX_NEAREST) {
    arbx_crs crs;
    ARBX_TRY(arbx_query_crs(t, &p, 1, nullptr, &crs, st));
    out.nnz = crs.nnz;
    out.offsets_dev = crs.offsets_dev;
    out.indices_dev = crs.indices_dev;
    out.d2_dev = crs.d2_dev;
    return ARBX_OK;
  }
  // radius: offsets, then reserve the matches, then fill
  if (arbx::dev_alloc_t(&out.offsets_dev, r.m + 1, s) != ARBX_OK) return ARBX_ERR_OOM;
  ARBX_TRY(arbx_query_offsets(t, &p, nullptr, out.offsets_dev, st));
  int64_t nnz = 0;
  ARBX_TRY(arbx::read_small(out.offsets_dev + r.m, &nnz, sizeof(int64_t), s));
  ARBX_TRY(arbx_stream_check(st));
  out.nnz = nnz;
  const int64_t extra = nnz * 8;
  {
    std::unique_lock<std::mutex> lk(sv->mu);
    tk.waiting_memory = true;
    ++sv->waiting;
    // this may make every running request a waiter, which lets the oldest
    // waiter go ahead: wake the others so they re-check
    sv->cv.notify_all();
    SLOG("ticket %llu waits for %lld bytes (reserved %lld, budget %lld)", (unsigned long long)id,
         (long long)extra, (long long)sv->reserved, (long long)sv->budget);
    sv->cv.wait_for(lk, std::chrono::duration<double>(MEMORY_WAIT_LIMIT_S), [&] {
      if (sv->fits(extra)) return true;
      // everyone running is waiting for memory: the oldest goes ahead
      if (sv->waiting == sv->running) {
        for (const auto& kv : sv->tickets)
          if (kv.second.waiting_memory && kv.first < id) return false;
        return true;
      }
      return false;
    });
    --sv->waiting;
    tk.waiting_memory = false;
    sv->reserved += extra;
    tk.reserved += extra;
  }
  if (arbx::dev_alloc_t(&out.indices_dev, std::max<int64_t>(nnz, 1), s) != ARBX_OK ||
      arbx::dev_alloc_t(&out.d2_dev, std::max<int64_t>(nnz, 1), s) != ARBX_OK)
    return ARBX_ERR_OOM;
  ARBX_TRY(arbx_query_fill(t, &p, nullptr, out.offsets_dev, out.indices_dev, out.d2_dev, st));
  return arbx_stream_check(st);
}

void worker(arbx_server_t* sv, int slot) {
  cudaSetDevice(sv->device);
  cudaStream_t s = sv->streams[slot];
  for (;;) {
    uint64_t id = 0;
    Ticket* tk = nullptr;
    {
      std::unique_lock<std::mutex> lk(sv->mu);
      sv->cv.wait(lk, [&] {
        if (sv->stop) return true;
        if (sv->queue.empty()) return false;
        Ticket& head = sv->tickets[sv->queue.front()];
        const int64_t est = estimate_bytes(head.req, sv->trees[head.req.tree_id]->n);
        return sv->running == 0 || sv->fits(est);
      });
      if (sv->stop && sv->queue.empty()) return;
      id = sv->queue.front();
      sv->queue.pop_front();
      tk = &sv->tickets[id];
      tk->reserved = estimate_bytes(tk->req, sv->trees[tk->req.tree_id]->n);
      sv->reserved += tk->reserved;
      ++sv->running;
      SLOG("slot %d starts ticket %llu (tree %d, kind %d, callback %d, m %lld)", slot, (unsigned long long)id,
           tk->req.tree_id, tk->req.kind, tk->req.callback, (long long)tk->req.m);
    }
    const arbx_status st = run_request(sv, *tk, s, id);
    cudaStreamSynchronize(s);
    SLOG("slot %d finished ticket %llu status %d", slot, (unsigned long long)id, (int)st);
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      tk->res.status = st;
      tk->done_at = sv->now();
      tk->res.latency_s = tk->done_at - tk->arrival;
      tk->done = true;
      sv->reserved -= tk->reserved;
      --sv->running;
      if (st == ARBX_OK) {
        sv->latencies.push_back(tk->res.latency_s);
        sv->queries_done += tk->req.m;
        if (sv->first_arrival < 0 || tk->arrival < sv->first_arrival) sv->first_arrival = tk->arrival;
        sv->last_done = std::max(sv->last_done, tk->done_at);
      }
    }
    sv->cv.notify_all();
  }
}

double percentile(std::vector<double> v, double q) {
  if (v.empty()) return 0.0;
  std::sort(v.begin(), v.end());
  const double pos = q * (double)(v.size() - 1);
  const size_t i = (size_t)pos;
  const double f = pos - (double)i;
  return i + 1 < v.size() ? v[i] * (1.0 - f) + v[i + 1] * f : v[i];
}

}  // namespace

extern "C" {

arbx_status arbx_server_create(arbx_server* out, int32_t slots, int64_t hbm_budget_bytes) {
  if (!out || slots < 1 || slots > 64 || hbm_budget_bytes <= 0) return ARBX_ERR_INVALID;
  *out = nullptr;
  arbx_server_t* sv = new arbx_server_t;
  cudaGetDevice(&sv->device);
  sv->budget = std::min<int64_t>(hbm_budget_bytes, std::max<int64_t>(device_available(), 0));
  sv->t0 = Clock::now();
  for (int i = 0; i < slots; ++i) {
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
      for (cudaStream_t x : sv->streams) cudaStreamDestroy(x);
      delete sv;
      return ARBX_ERR_CUDA;
    }
    sv->streams.push_back(s);
  }
  for (int i = 0; i < slots; ++i) sv->workers.emplace_back(worker, sv, i);
  *out = sv;
  return ARBX_OK;
}

arbx_status arbx_server_add_tree(arbx_server sv, arbx_tree t, int32_t* tree_id) {
  if (!sv || !t || !tree_id) return ARBX_ERR_INVALID;
  std::lock_guard<std::mutex> lk(sv->mu);
  sv->trees.push_back(t);
  *tree_id = (int32_t)sv->trees.size() - 1;
  return ARBX_OK;
}

double arbx_server_now(arbx_server sv) { return sv ? sv->now() : 0.0; }

arbx_status arbx_server_submit(arbx_server sv, const arbx_request* req, uint64_t* ticket) {
  if (!sv || !req || !ticket) return ARBX_ERR_INVALID;
  if (req->tree_id < 0 || req->m < 0) return ARBX_ERR_INVALID;
  if (req->m > 0 && !req->queries_dev) return ARBX_ERR_INVALID;
  if (req->callback >= 0 && req->kind != ARBX_SPHERE && req->kind != ARBX_BOX_PRED) return ARBX_ERR_INVALID;
  if (req->callback < 0 && req->kind != ARBX_SPHERE && req->kind != ARBX_NEAREST) return ARBX_ERR_INVALID;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    if (req->tree_id >= (int32_t)sv->trees.size()) return ARBX_ERR_INVALID;
    const uint64_t id = sv->next_ticket++;
    Ticket& tk = sv->tickets[id];
    tk.req = *req;
    tk.arrival = req->arrival_s >= 0.0 ? req->arrival_s : sv->now();
    std::memset(&tk.res, 0, sizeof(tk.res));
    sv->queue.push_back(id);
    *ticket = id;
  }
  sv->cv.notify_all();
  return ARBX_OK;
}

arbx_status arbx_server_wait(arbx_server sv, uint64_t ticket, int64_t timeout_us, arbx_result* out) {
  if (!sv || !out) return ARBX_ERR_INVALID;
  std::unique_lock<std::mutex> lk(sv->mu);
  if (sv->tickets.find(ticket) == sv->tickets.end()) return ARBX_ERR_INVALID;
  // look the ticket up again on every wake-up: submissions from other threads
  // may rehash the map (element references stay valid, iterators do not)
  const auto pred = [&] { return sv->tickets.find(ticket)->second.done; };
  if (timeout_us < 0) {
    sv->cv.wait(lk, pred);
  } else if (!sv->cv.wait_for(lk, std::chrono::microseconds(timeout_us), pred)) {
    return ARBX_ERR_TIMEOUT;
  }
  auto it = sv->tickets.find(ticket);
  *out = it->second.res;
  const arbx_status st = it->second.res.status;
  sv->tickets.erase(it);  // the result buffers now belong to the caller
  return st;
}

arbx_status arbx_server_release(arbx_server sv, arbx_result* r) {
  if (!sv || !r) return ARBX_ERR_INVALID;
  void* ptrs[] = {r->offsets_dev, r->indices_dev, r->d2_dev, r->counts_dev};
  for (void* p : ptrs)
    if (p) cudaFreeAsync(p, sv->streams[0]);
  cudaStreamSynchronize(sv->streams[0]);
  std::memset(r, 0, sizeof(*r));
  return ARBX_OK;
}

arbx_status arbx_server_stats(arbx_server sv, double* p50_s, double* p99_s, double* mqps, int64_t* completed) {
  if (!sv) return ARBX_ERR_INVALID;
  std::lock_guard<std::mutex> lk(sv->mu);
  if (p50_s) *p50_s = percentile(sv->latencies, 0.50);
  if (p99_s) *p99_s = percentile(sv->latencies, 0.99);
  const double span = sv->last_done - sv->first_arrival;
  if (mqps) *mqps = span > 0 ? (double)sv->queries_done / span / 1e6 : 0.0;
  if (completed) *completed = (int64_t)sv->latencies.size();
  return ARBX_OK;
}

arbx_status arbx_server_reset_stats(arbx_server sv) {
  if (!sv) return ARBX_ERR_INVALID;
  std::lock_guard<std::mutex> lk(sv->mu);
  sv->latencies.clear();
  sv->queries_done = 0;
  sv->first_arrival = -1.0;
  sv->last_done = 0.0;
  return ARBX_OK;
}

arbx_status arbx_server_destroy(arbx_server sv) {
  if (!sv) return ARBX_OK;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
  }
  sv->cv.notify_all();
  for (auto& w : sv->workers) w.join();
  for (cudaStream_t s : sv->streams) cudaStreamDestroy(s);
  for (arbx_tree t : sv->trees) arbx_tree_destroy(t);
  delete sv;
  return ARBX_OK;
}

}  // extern "C"
