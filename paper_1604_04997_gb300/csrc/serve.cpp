// Serving runtime: continuous batching of autotuner queries over resident tables and
// weights (Sec. 6.1 uses the model to pick configurations; a tuner asks many small
// questions, so they are batched).
//
//   submit   validates a query on the host and queues it (FIFO), returning a ticket.
//   worker   forms a batch: at once if no batch is in flight, otherwise once the oldest
//            queued query is batch_interval_us old, max_batch_queries are queued or the
//            batches in flight have finished; it admits queries in FIFO order
//            while their bytes fit the free part of the memory region; packs them into
//            pinned staging memory and launches copy-in, the two kernels and copy-out on
//            the next of n_streams streams.
//   reaper   polls the batches in flight, copies each finished query's topk into the
//            caller's buffers, releases its region and completes its ticket.
//   poll     waits (bounded by timeout_us) for a ticket.
//
// Memory: one device region and one pinned host region of the same size
// (min(budget, 1 GiB)); a batch occupies the same offsets in both.  A query whose bytes
// exceed the region can never run and is refused with PM_ERR_BUSY.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "kernels.h"
#include "pm.h"
#include "pm_internal.h"
#include "pm_table.h"
#include "trace.h"

using Clock = std::chrono::steady_clock;

namespace {

constexpr size_t REGION_MAX = size_t(1) << 30;
constexpr size_t ALIGN = 256;
constexpr int EVAL_CTA = 128;   // candidates per k_serve_eval CTA

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Byte layout of one batch inside its region (offsets relative to the batch start).
// [points N*32][cand_off N*4][queries nq*24][blocks nb*8][status nq*4][out_idx nq*64][out_t nq*128][keys N*8]
// Copy-in covers [0, out_idx); copy-out covers [status, keys).
struct Layout {
  size_t points, cand_off, queries, blocks, status, out_idx, out_t, keys, total;
  Layout(int64_t N, int nq, int64_t nb) {
    points = 0;
    cand_off = points + (size_t)N * 32;
    queries = align_up(cand_off + (size_t)N * 4, 8);
    blocks = queries + (size_t)nq * sizeof(pmd::SQuery);
    status = align_up(blocks + (size_t)nb * 8, 8);
    out_idx = status + (size_t)nq * 4;
    out_t = align_up(out_idx + (size_t)nq * pmd::SV_MAX_TOPK * 4, 8);
    keys = out_t + (size_t)nq * pmd::SV_MAX_TOPK * 8;
    total = align_up(keys + (size_t)N * 8, ALIGN);
  }
};

size_t query_bytes(int64_t n) {
  // standalone layout of one query: an upper bound of its share in any batch
  return Layout(n, 1, (n + EVAL_CTA - 1) / EVAL_CTA).total;
}

// First-fit allocator over [0, cap).
struct Region {
  size_t cap = 0;
  std::map<size_t, size_t> free_;   // offset -> size
  void reset(size_t c) { cap = c; free_.clear(); free_[0] = c; }
  bool alloc(size_t bytes, size_t *off) {
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes, o = it->first + bytes;
        free_.erase(it);
        if (rest) free_[o] = rest;
        return true;
      }
    }
    return false;
  }
  size_t largest() const {
    size_t m = 0;
    for (const auto &kv : free_) m = std::max(m, kv.second);
    return m;
  }
  void release(size_t off, size_t bytes) {
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) { it->second += nx->second; free_.erase(nx); }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) { pv->second += it->second; free_.erase(it); }
    }
  }
};

struct Pending {
  uint64_t ticket;
  pm_query q;
  Clock::time_point t_submit;
};

struct Batch {
  std::vector<Pending> qs;
  size_t off = 0, bytes = 0;
  Layout lay{0, 0, 0};
  int stream = 0;
  cudaEvent_t done = nullptr;
  pm_status launch_error = PM_OK;
};

struct TicketState {
  bool done = false;
  pm_status result = PM_OK;
};

}  // namespace

struct ServeState {
  pm_ctx *ctx = nullptr;
  pm_serve_config cfg{};
  std::thread worker, reaper;
  std::mutex m;
  std::condition_variable cv_work;    // queue changed / stop / space freed
  std::condition_variable cv_done;    // a ticket completed
  std::condition_variable cv_flight;  // a batch was launched / worker finished
  std::deque<Pending> queue;
  std::unordered_map<uint64_t, TicketState> tickets;
  std::deque<Batch *> flight;
  uint64_t next_ticket = 1;
  bool running = false, stopping = false, worker_done = false;
  Region region;
  uint8_t *d_region = nullptr, *h_region = nullptr;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> free_events;
  int next_stream = 0;
  // statistics: every latency since the last reset, or (past LAT_CAP of them) a
  // uniform sample of LAT_CAP, kept by reservoir sampling
  std::vector<float> lat_us;
  uint64_t lat_seen = 0, lat_rng = 0;
  double lat_max = 0, lat_sum = 0;   // exact over every latency since the last reset
  uint64_t n_batches = 0, n_queries = 0, n_cand = 0;
  uint64_t n_rejected = 0, h2d_bytes = 0, d2h_bytes = 0;
};

constexpr size_t LAT_CAP = size_t(1) << 22;

// splitmix64 (Steele, Lea and Flood, 2014): a counter-based 64-bit generator
static uint64_t splitmix64(uint64_t &state) {
  uint64_t z = (state += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Record one latency: the first LAT_CAP are kept; the i-th after that (0-based
// count i of all seen) replaces a random kept one with probability LAT_CAP / (i + 1),
// which keeps a uniform sample of all seen (reservoir sampling, Vitter's Algorithm R).
static void record_latency(ServeState *S, float us) {
  if (S->lat_us.size() < LAT_CAP) {
    S->lat_us.push_back(us);
  } else {
    const uint64_t k = splitmix64(S->lat_rng) % (S->lat_seen + 1);
    if (k < LAT_CAP) S->lat_us[(size_t)k] = us;
  }
  S->lat_seen++;
  S->lat_max = std::max(S->lat_max, (double)us);
  S->lat_sum += us;
}

static pm_status cu_err(cudaError_t e, const char *what) {
  return pm_set_error(PM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// Pack the batch into the pinned region and launch it.  Called by the worker without
// the serve lock; holds ctx->mu while it reads table offsets and the arena pointer, so
// a concurrent pm_compile_counts cannot move the arena under a launch.
static pm_status launch_batch(ServeState *S, Batch *B) {
  PM_TRACE("pm_serve_batch");
  pm_ctx *c = S->ctx;
  uint8_t *h = S->h_region + B->off;
  uint8_t *d = S->d_region + B->off;
  const Layout &L = B->lay;
  auto *hq = (pmd::SQuery *)(h + L.queries);
  auto *hb = (int2 *)(h + L.blocks);
  auto *hp = (int64_t *)(h + L.points);
  auto *ho = (uint32_t *)(h + L.cand_off);
  int64_t begin = 0, nb = 0;
  std::lock_guard<std::mutex> lk(c->mu);
  for (size_t j = 0; j < B->qs.size(); j++) {
    const pm_query &q = B->qs[j].q;
    hq[j] = pmd::SQuery{begin, (int32_t)q.n_cand, q.model, q.topk, 0};
    std::memcpy(hp + begin * 4, q.h_points, (size_t)q.n_cand * 32);
    for (int64_t i = 0; i < q.n_cand; i++) ho[begin + i] = (uint32_t)c->dev_off[q.h_tables[i]];
    for (int64_t ch = 0; ch * EVAL_CTA < q.n_cand; ch++) hb[nb++] = make_int2((int)j, (int)ch);
    begin += q.n_cand;
  }
  std::memset(h + L.status, 0, B->qs.size() * 4);
  cudaStream_t st = S->streams[B->stream];
  cudaError_t e;
  if ((e = cudaSetDevice(c->device)) != cudaSuccess) return cu_err(e, "cudaSetDevice");
  if ((e = cudaMemcpyAsync(d, h, L.out_idx, cudaMemcpyHostToDevice, st)) != cudaSuccess)
    return cu_err(e, "copy-in");
  pmd::ServeArgs a;
  a.arena = c->arena;
  a.queries = (const pmd::SQuery *)(d + L.queries);
  a.n_queries = (int)B->qs.size();
  a.blocks = (const int2 *)(d + L.blocks);
  a.cand_off = (const uint32_t *)(d + L.cand_off);
  a.points = (const int64_t *)(d + L.points);
  a.models = c->d_models;
  a.keys = (int64_t *)(d + L.keys);
  a.q_status = (int32_t *)(d + L.status);
  a.out_idx = (int32_t *)(d + L.out_idx);
  a.out_t = (double *)(d + L.out_t);
  if ((e = pmd::launch_serve(a, (int)nb, st)) != cudaSuccess) return cu_err(e, "serve kernels");
  if ((e = cudaMemcpyAsync(h + L.status, d + L.status, L.keys - L.status, cudaMemcpyDeviceToHost, st)) !=
      cudaSuccess)
    return cu_err(e, "copy-out");
  if ((e = cudaEventRecord(B->done, st)) != cudaSuccess) return cu_err(e, "event");
  return PM_OK;
}

static void worker_loop(ServeState *S) {
  cudaSetDevice(S->ctx->device);
  const auto interval = std::chrono::microseconds(S->cfg.batch_interval_us);
  std::unique_lock<std::mutex> lk(S->m);
  while (true) {
    S->cv_work.wait(lk, [&] { return S->stopping || !S->queue.empty(); });
    if (S->queue.empty()) break;   // stopping and drained
    // batching window: an idle GPU takes the queue at once; a busy one lets queries
    // gather until the oldest has waited batch_interval_us or the GPU drains
    const auto deadline = S->queue.front().t_submit + interval;
    while (!S->stopping && !S->flight.empty() && (int)S->queue.size() < S->cfg.max_batch_queries &&
           Clock::now() < deadline)
      S->cv_work.wait_until(lk, deadline);
    // admission: FIFO while the batch fits the largest free block; needs a free event
    if (S->free_events.empty()) {
      S->cv_work.wait_for(lk, std::chrono::milliseconds(10));
      continue;
    }
    const size_t largest = S->region.largest();
    int take = 0;
    int64_t N = 0, nb = 0;
    size_t bytes = 0;
    for (const Pending &p : S->queue) {
      if (take >= S->cfg.max_batch_queries) break;
      const int64_t n2 = N + p.q.n_cand, nb2 = nb + (p.q.n_cand + EVAL_CTA - 1) / EVAL_CTA;
      const Layout L(n2, take + 1, nb2);
      if (L.total > largest) break;
      N = n2;
      nb = nb2;
      bytes = L.total;
      take++;
    }
    if (take == 0) {   // the oldest query waits for a batch in flight to release memory
      S->cv_work.wait_for(lk, std::chrono::milliseconds(10));
      continue;
    }
    Batch *B = new Batch();
    size_t off = 0;
    S->region.alloc(bytes, &off);   // fits: bytes <= largest free block
    for (int j = 0; j < take; j++) {
      B->qs.push_back(S->queue.front());
      S->queue.pop_front();
    }
    B->off = off;
    B->bytes = bytes;
    B->lay = Layout(N, (int)B->qs.size(), nb);
    B->stream = S->next_stream;
    S->next_stream = (S->next_stream + 1) % (int)S->streams.size();
    B->done = S->free_events.back();
    S->free_events.pop_back();
    lk.unlock();
    const pm_status rc = launch_batch(S, B);
    // a partly enqueued batch still owns its region until its stream drains
    if (rc != PM_OK) cudaStreamSynchronize(S->streams[B->stream]);
    B->launch_error = rc;
    lk.lock();
    S->flight.push_back(B);
    S->n_batches++;
    if (rc == PM_OK) {
      S->h2d_bytes += B->lay.out_idx;                  // the batch's copy-in
      S->d2h_bytes += B->lay.keys - B->lay.status;     // and copy-out
    }
    S->cv_flight.notify_all();
  }
  S->worker_done = true;
  S->cv_flight.notify_all();
}

static void finish_batch(ServeState *S, Batch *B) {
  // results -> caller buffers (outside the serve lock)
  const Layout &L = B->lay;
  const uint8_t *h = S->h_region + B->off;
  std::vector<pm_status> res(B->qs.size(), B->launch_error);
  if (B->launch_error == PM_OK) {
    const int32_t *st = (const int32_t *)(h + L.status);
    const int32_t *oi = (const int32_t *)(h + L.out_idx);
    const double *ot = (const double *)(h + L.out_t);
    for (size_t j = 0; j < B->qs.size(); j++) {
      const pm_query &q = B->qs[j].q;
      std::memcpy(q.h_top_idx, oi + j * pmd::SV_MAX_TOPK, (size_t)q.topk * 4);
      std::memcpy(q.h_top_t, ot + j * pmd::SV_MAX_TOPK, (size_t)q.topk * 8);
      if (st[j] & pmd::ST_OUT_OF_BOX) res[j] = PM_ERR_OUT_OF_BOX;
      else if (st[j] & pmd::ST_BAD_TABLE) res[j] = PM_ERR_INVALID_ARG;
    }
  }
  const auto now = Clock::now();
  std::lock_guard<std::mutex> lk(S->m);
  for (size_t j = 0; j < B->qs.size(); j++) {
    auto it = S->tickets.find(B->qs[j].ticket);
    if (it != S->tickets.end()) { it->second.done = true; it->second.result = res[j]; }
    record_latency(S, (float)std::chrono::duration<double, std::micro>(now - B->qs[j].t_submit).count());
    S->n_queries++;
    S->n_cand += (uint64_t)B->qs[j].q.n_cand;
  }
  S->region.release(B->off, B->bytes);
  if (B->done) S->free_events.push_back(B->done);
  delete B;
  S->cv_done.notify_all();
  S->cv_work.notify_all();
}

static void reaper_loop(ServeState *S) {
  cudaSetDevice(S->ctx->device);
  std::unique_lock<std::mutex> lk(S->m);
  while (true) {
    S->cv_flight.wait(lk, [&] { return !S->flight.empty() || S->worker_done; });
    if (S->flight.empty()) break;   // worker finished and nothing in flight
    std::vector<Batch *> snap(S->flight.begin(), S->flight.end());
    lk.unlock();
    std::vector<Batch *> ready;
    for (Batch *B : snap) {
      if (B->launch_error != PM_OK) { ready.push_back(B); continue; }
      const cudaError_t e = cudaEventQuery(B->done);
      if (e == cudaSuccess) ready.push_back(B);
      else if (e != cudaErrorNotReady) { B->launch_error = cu_err(e, "batch"); ready.push_back(B); }
    }
    if (ready.empty()) {
      std::this_thread::yield();
      lk.lock();
      continue;
    }
    lk.lock();
    for (Batch *B : ready) S->flight.erase(std::find(S->flight.begin(), S->flight.end(), B));
    lk.unlock();
    for (Batch *B : ready) finish_batch(S, B);
    lk.lock();
  }
}

static void release_resources(ServeState *S) {
  if (S->ctx->device >= 0) cudaSetDevice(S->ctx->device);
  for (cudaStream_t s : S->streams) { cudaStreamSynchronize(s); cudaStreamDestroy(s); }
  S->streams.clear();
  for (cudaEvent_t e : S->free_events) cudaEventDestroy(e);
  S->free_events.clear();
  if (S->d_region) cudaFree(S->d_region);
  if (S->h_region) cudaFreeHost(S->h_region);
  S->d_region = S->h_region = nullptr;
}

extern "C" pm_status pm_serve_set_weights(pm_ctx *c, const double *h_W, int32_t n_models) {
  pm_status g = ctx_device_guard(c);
  if (g) return g;
  if (!h_W || n_models <= 0) return pm_set_error(PM_ERR_INVALID_ARG, "need weights and n_models >= 1");
  if (c->serve && c->serve->running) return pm_set_error(PM_ERR_BUSY, "weights are fixed while serving");
  for (int64_t i = 0; i < (int64_t)n_models * 32; i++)
    if (!std::isfinite(h_W[i])) return pm_set_error(PM_ERR_INVALID_ARG, "weights must be finite");
  double *d = nullptr;
  cudaError_t e = cudaMalloc(&d, (size_t)n_models * 32 * 8);
  if (e != cudaSuccess) return cu_err(e, "cudaMalloc");
  e = cudaMemcpy(d, h_W, (size_t)n_models * 32 * 8, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) { cudaFree(d); return cu_err(e, "cudaMemcpy"); }
  if (c->d_models) cudaFree(c->d_models);
  c->d_models = d;
  c->n_models = n_models;
  return PM_OK;
}

extern "C" pm_status pm_serve_start(pm_ctx *c, const pm_serve_config *cfg) {
  PM_TRACE("pm_serve_start");
  pm_status g = ctx_device_guard(c);
  if (g) return g;
  if (!cfg) return pm_set_error(PM_ERR_INVALID_ARG, "null config");
  if (cfg->batch_interval_us < 0 || cfg->batch_interval_us > 1000000 || cfg->n_streams < 1 || cfg->n_streams > 16 ||
      cfg->max_batch_queries < 1 || cfg->max_batch_queries > 1024)
    return pm_set_error(PM_ERR_INVALID_ARG, "config: interval 0..1e6 us, 1..16 streams, 1..1024 queries per batch");
  if (!c->d_models) return pm_set_error(PM_ERR_INVALID_ARG, "pm_serve_set_weights first");
  if (c->serve && c->serve->running) return pm_set_error(PM_ERR_BUSY, "already serving");
  if (c->serve) { delete c->serve; c->serve = nullptr; }
  auto *S = new ServeState();
  S->ctx = c;
  S->cfg = *cfg;
  const size_t cap = std::min(c->budget, REGION_MAX) / ALIGN * ALIGN;
  cudaError_t e = cudaMalloc(&S->d_region, cap);
  if (e == cudaSuccess) e = cudaMallocHost(&S->h_region, cap);
  for (int i = 0; e == cudaSuccess && i < cfg->n_streams; i++) {
    cudaStream_t s;
    e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) S->streams.push_back(s);
  }
  // one event per batch that can be in flight at once (regions hold >= 1 query each)
  for (int i = 0; e == cudaSuccess && i < 64; i++) {
    cudaEvent_t ev;
    e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) S->free_events.push_back(ev);
  }
  if (e != cudaSuccess) {
    release_resources(S);
    delete S;
    return cu_err(e, "serve setup");
  }
  S->region.reset(cap);
  S->running = true;
  c->serve = S;
  S->worker = std::thread(worker_loop, S);
  S->reaper = std::thread(reaper_loop, S);
  return PM_OK;
}

extern "C" pm_status pm_serve_submit(pm_ctx *c, const pm_query *q, uint64_t *ticket) {
  if (!c || !q || !ticket) return pm_set_error(PM_ERR_INVALID_ARG, "null argument");
  ServeState *S = c->serve;
  if (!S || !S->running) return pm_set_error(PM_ERR_INVALID_ARG, "serve loop not started");
  if (q->model < 0 || q->model >= c->n_models) return pm_set_error(PM_ERR_INVALID_ARG, "no such model");
  if (q->topk < 1 || q->topk > PM_MAX_TOPK) return pm_set_error(PM_ERR_INVALID_ARG, "topk must be 1..16");
  if (q->n_cand < 0 || q->n_cand > (int64_t(1) << 30)) return pm_set_error(PM_ERR_INVALID_ARG, "bad n_cand");
  if (!q->h_top_idx || !q->h_top_t || (q->n_cand > 0 && (!q->h_tables || !q->h_points)))
    return pm_set_error(PM_ERR_INVALID_ARG, "null buffer");
  if (query_bytes(q->n_cand) > S->region.cap) {
    {
      std::lock_guard<std::mutex> lk(S->m);
      S->n_rejected++;
    }
    return pm_set_error(PM_ERR_BUSY, "query can never fit the memory budget");
  }
  {
    std::lock_guard<std::mutex> lk(c->mu);
    const int32_t nt = (int32_t)c->tables.size();
    for (int64_t i = 0; i < q->n_cand; i++) {
      const int32_t id = q->h_tables[i];
      if (id < 0 || id >= nt) return pm_set_error(PM_ERR_INVALID_ARG, "no such table");
      const std::vector<uint32_t> &T = c->tables[id];
      if (T[pmt::H_K] != 32 || c->dev_off[id] < 0) return pm_set_error(PM_ERR_INVALID_ARG, "serve needs PM_LAYOUT_32 tables");
    }
  }
  std::lock_guard<std::mutex> lk(S->m);
  if (S->stopping) return pm_set_error(PM_ERR_INVALID_ARG, "serve loop is stopping");
  const uint64_t t = S->next_ticket++;
  if (q->n_cand == 0) {
    for (int j = 0; j < q->topk; j++) { q->h_top_idx[j] = -1; q->h_top_t[j] = HUGE_VAL; }
    S->tickets[t] = TicketState{true, PM_OK};
  } else {
    S->tickets[t] = TicketState{};
    S->queue.push_back(Pending{t, *q, Clock::now()});
    S->cv_work.notify_all();
  }
  *ticket = t;
  return PM_OK;
}

extern "C" pm_status pm_serve_poll(pm_ctx *c, uint64_t ticket, int32_t timeout_us) {
  if (!c) return pm_set_error(PM_ERR_INVALID_ARG, "null context");
  ServeState *S = c->serve;
  if (!S) return pm_set_error(PM_ERR_NOT_FOUND, "no such ticket");
  std::unique_lock<std::mutex> lk(S->m);
  auto it = S->tickets.find(ticket);
  if (it == S->tickets.end()) return pm_set_error(PM_ERR_NOT_FOUND, "no such ticket");
  if (!it->second.done && timeout_us > 0)
    S->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), [&] { return it->second.done; });
  if (!it->second.done) return PM_PENDING;
  const pm_status r = it->second.result;
  S->tickets.erase(it);
  if (r < 0) return pm_set_error(r, r == PM_ERR_OUT_OF_BOX ? "a candidate point lies outside its table's box"
                                                          : "the query's batch failed");
  return PM_OK;
}

extern "C" pm_status pm_serve_stats(pm_ctx *c, int32_t reset, pm_serve_stats_t *out) {
  if (!c || !out) return pm_set_error(PM_ERR_INVALID_ARG, "null argument");
  std::memset(out, 0, sizeof(*out));
  ServeState *S = c->serve;
  if (!S) return PM_OK;
  // copy (or take) the record under the lock; the percentiles are found after it is
  // released, so that a stats call does not hold up admission or the completion thread
  std::vector<float> v;
  uint64_t seen;
  double mx, sum;
  {
    std::lock_guard<std::mutex> lk(S->m);
    out->n_queries = (int64_t)S->n_queries;
    out->n_batches = (int64_t)S->n_batches;
    out->n_candidates = (int64_t)S->n_cand;
    out->n_rejected = (int64_t)S->n_rejected;
    out->h2d_bytes = (int64_t)S->h2d_bytes;
    out->d2h_bytes = (int64_t)S->d2h_bytes;
    seen = S->lat_seen;
    mx = S->lat_max;
    sum = S->lat_sum;
    if (reset) {
      v.swap(S->lat_us);
      S->lat_seen = 0;
      S->lat_max = S->lat_sum = 0;
      S->n_queries = S->n_batches = S->n_cand = 0;
      S->n_rejected = S->h2d_bytes = S->d2h_bytes = 0;
    } else {
      v = S->lat_us;
    }
  }
  if (!v.empty()) {
    auto pct = [&](double p) {
      const size_t i = std::min(v.size() - 1, (size_t)(p * (double)(v.size() - 1) + 0.5));
      std::nth_element(v.begin(), v.begin() + (std::ptrdiff_t)i, v.end());
      return (double)v[i];
    };
    out->p50_us = pct(0.50);
    out->p99_us = pct(0.99);
    out->max_us = mx;
    out->mean_us = sum / (double)seen;
  }
  return PM_OK;
}

void serve_destroy(pm_ctx *c) {
  pm_serve_stop(c);
  delete c->serve;
  c->serve = nullptr;
  if (c->d_models) cudaFree(c->d_models);
  c->d_models = nullptr;
}

extern "C" pm_status pm_serve_stop(pm_ctx *c) {
  PM_TRACE("pm_serve_stop");
  if (!c) return pm_set_error(PM_ERR_INVALID_ARG, "null context");
  ServeState *S = c->serve;
  if (!S || !S->running) return PM_OK;
  {
    std::lock_guard<std::mutex> lk(S->m);
    S->stopping = true;
    S->cv_work.notify_all();
  }
  S->worker.join();   // drains the queue
  S->reaper.join();   // finishes every batch in flight
  release_resources(S);
  std::lock_guard<std::mutex> lk(S->m);
  S->running = false;
  S->stopping = false;
  return PM_OK;
}
