// Serving: continuous batching of partition requests under a device-memory
// budget.
//
// A server owns a pool of worker threads, each with its own CUDA stream.
// Submitted requests wait in FIFO order; the head is admitted as soon as a
// worker is free, its footprint (tp_footprint_bytes) fits in what is left of
// the budget, and, for a request on a resident graph, no other request is
// using that graph (a graph caches per-level state while it is partitioned).
// Admitted requests run concurrently on the device; each one's memory is
// returned to the budget when it finishes, which admits the next. A
// request's thread may allocate at most its footprint: one that would need
// more fails before allocating and goes back to the head of the queue with
// the whole budget as its footprint, so it runs again alone (a request whose
// footprint exceeds the budget is admitted that way from the start; it fails
// only if it would really need more than the budget). The device therefore
// never holds more than the budget for requests. Every
// request runs the unchanged single-graph path (upload, optional
// compression, tp_partition, copy back), so its result does not depend on
// what else is in flight.
#include <stdlib.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <new>
#include <system_error>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "tp_internal.cuh"

namespace tp {
tp_graph *from_csr(int64_t n, const int64_t *xadj, const int32_t *adj, const int64_t *vwgt,
                   const int64_t *ewgt, int host, cudaStream_t s);
tp_graph *compress(const tp_graph *c, cudaStream_t s);
void partition(tp_graph *g0, int32_t k, int64_t eps_ppm, const tp_params &p, int32_t *d_part,
               tp_stats *st, cudaStream_t s);
}  // namespace tp

using namespace tp;
using Clock = std::chrono::steady_clock;

namespace {

struct Request {
  tp_request r;
  uint64_t ticket = 0;
  int32_t retries = 0;
  int64_t need = 0;  // admitted footprint (bytes)
  int state = 0;     // 0 queued, 1 running, 2 done
  bool waited = false;  // a waiter holds this request (a ticket is waited once)
  tp_status status = TP_OK;
  tp_stats stats{};
  int64_t peak = 0;
  Clock::time_point t_submit, t_start, t_done;
};

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

}  // namespace

struct tp_server {
  int64_t budget = 0, in_use = 0, peak_in_use = 0;
  double footprint_scale = 1.0;  // diagnostics: TP_FOOTPRINT_SCALE scales every footprint
  int32_t max_running = 0, running = 0;
  tp_params params{};
  int device = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<uint64_t> queue;
  std::unordered_map<uint64_t, std::unique_ptr<Request>> reqs;
  std::unordered_set<const tp_graph *> busy;
  std::vector<std::thread> workers;
  uint64_t next_ticket = 1;
  bool stopping = false;

  // The queue head, if it can start now (caller holds mu).
  Request *admissible() {
    if (queue.empty() || running >= max_running) return nullptr;
    Request *q = reqs[queue.front()].get();
    if (in_use + q->need > budget) return nullptr;
    if (q->r.graph && busy.count(q->r.graph)) return nullptr;
    return q;
  }

  void run(Request *q, cudaStream_t s) {
    const tp_request &r = q->r;
    const int64_t mark = mem_mark();
    mem_cap(q->need);  // the admitted footprint, enforced
    q->status = guard([&] {
      std::unique_ptr<tp_graph> up, zp;
      const tp_graph *g = r.graph;
      if (!g) {
        up.reset(from_csr(r.n, r.xadj, r.adj, nullptr, nullptr, 1, s));
        g = up.get();
        if (r.compress) {
          zp.reset(compress(up.get(), s));
          up.reset();
          g = zp.get();
        }
      }
      Buf<int32_t> part(std::max<int64_t>(g->n, 1), s);
      partition(const_cast<tp_graph *>(g), r.k, (int64_t)llround(r.eps * 1e6), params, part.get(),
                &q->stats, s);
      if (g->n)
        TP_CUDA(cudaMemcpyAsync(r.part, part.get(), g->n * sizeof(int32_t),
                                cudaMemcpyDeviceToHost, s));
      TP_CUDA(cudaStreamSynchronize(s));
    });
    if (q->status != TP_OK) cudaStreamSynchronize(s);  // its buffers were freed on s
    mem_cap(-1);
    q->peak = mem_peak_since(mark);
  }

  void worker() {
    cudaStream_t s = nullptr;
    const bool ok = cudaSetDevice(device) == cudaSuccess &&
                    cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess;
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
      Request *q = nullptr;
      cv_work.wait(lk, [&] { return (q = admissible()) != nullptr || (stopping && queue.empty()); });
      if (!q) break;
      queue.pop_front();
      q->state = 1;
      q->t_start = Clock::now();
      in_use += q->need;
      peak_in_use = std::max(peak_in_use, in_use);
      ++running;
      if (q->r.graph) busy.insert(q->r.graph);
      cv_work.notify_all();  // the next head may fit as well
      lk.unlock();
      if (ok) run(q, s);
      else q->status = TP_ERR_CUDA;
      lk.lock();
      in_use -= q->need;
      --running;
      if (q->r.graph) busy.erase(q->r.graph);
      if (q->status == TP_ERR_BUDGET && q->need < budget && q->retries == 0) {
        // outgrew its footprint: again, alone, with the whole budget
        q->need = budget;
        q->retries = 1;
        q->state = 0;
        queue.push_front(q->ticket);
        cv_work.notify_all();
        continue;
      }
      q->t_done = Clock::now();
      q->state = 2;
      cv_done.notify_all();
      cv_work.notify_all();
    }
    lk.unlock();
    if (s) cudaStreamDestroy(s);
  }
};

extern "C" {

// Device bytes of one request, phase by phase from the library's
// allocations (bytes per vertex n / adjacency entry m / block k), for any graph whose hierarchy stays inside this
// envelope: the coarse levels together hold at most n vertices and 2 m
// adjacency entries (each level has fewer entries than the one below; R-MAT
// scale 26 coarse levels hold 0.05 n and 1.5 m, random geometric graphs
// about 0.1 n and 0.3 m), any level may be made of hubs entirely, and the
// coarsest graph has at most min(n, 4 c_lim k) vertices.
//   upload   CSR 8n + 4m; with compression the stream (<= 10n + 5m + the
//            chunk tables), its offsets and the encoder's scratch 16n
//   part     4n (the request's result)
//   levels   coarse CSR 16n + 12m per level; per level a map 4n and a tier
//            cache 5n + 0.05m  -> within the envelope 30n + 24m
//   cluster  C, map, cluster weights 16n; LP workspace 62n, 8n more for the
//            records of a compressed level; two-hop packing 88n; hub rating
//            tables 14 bytes per slot, fewer than 4 slots per hub neighbour: 56m
//   contract flags, ranks, offsets 24n + coarse weights 8n; keys and their
//            radix buffer 16m (weights unpackable into keys: 32m); coarse
//            CSR 12m while the keys live
//   initial  T attempts x 53 bytes per coarsest vertex + 40 + its CSR 12m
//   refine   two partition arrays 8n, LP workspace 50n, hub tables 56m;
//            block weights and per-block approval state 36k (counted apart)
// The server admits a request by this figure and caps what its thread may
// allocate at it; a request that would exceed it fails before allocating
// and runs again alone with the whole budget.
static int64_t footprint_model(int64_t n, int64_t m, int32_t k, bool upload, bool compress,
                               int32_t c_lim, int32_t T) {
  const double N = (double)n, M = (double)m, K = (double)k;
  double in = 0;
  if (upload) in = 8 * (N + 1) + 4 * (M + 4) + 64 + (compress ? (10 * N + 5.004 * M) + 16 * N : 0);
  const double levels = 30 * N + 24 * M;
  const double cluster = 174 * N + 56 * M;
  const double contract = 32 * N + std::max(32 * M, 16 * M + 12 * M + 8 * N);
  const double nc = std::min(N, 4.0 * c_lim * K);
  const double initial = (53.0 * T + 40) * nc + 12 * std::min(M, nc * nc) + 12 * nc;
  const double refine = 58 * N + 56 * M;
  const double work = std::max(std::max(cluster, contract), std::max(initial, refine));
  const double total = in + 4 * N + levels + work + 36 * K + (double)((int64_t)64 << 20);
  return total >= 9.0e18 ? INT64_MAX : (int64_t)total;
}

int64_t tp_footprint_bytes(int64_t n, int64_t m2, int32_t k, int32_t upload, int32_t compress) {
  if (n < 0 || m2 < 0 || k < 1) return -1;
  tp_params d;
  tp_params_default(&d);
  return footprint_model(n, m2, k, upload != 0, compress != 0, d.c_lim, d.ip_attempts);
}

tp_status tp_server_create(int64_t budget_bytes, int32_t workers, const tp_params *p,
                           tp_server **out) {
  if (!out || budget_bytes <= 0 || workers < 1 || workers > 256) return TP_ERR_INVALID;
  *out = nullptr;
  tp_params q;
  if (p) q = *p;
  else tp_params_default(&q);
  if (q.cluster_rounds < 0 || q.refine_rounds < 0 || q.sub_rounds < 1 || q.c_lim < 1 ||
      q.ip_attempts < 1 || q.max_levels < 1 || q.max_levels > 64)
    return TP_ERR_INVALID;
  auto *sv = new tp_server();
  sv->budget = budget_bytes;
  sv->max_running = workers;
  if (const char *f = getenv("TP_FOOTPRINT_SCALE")) {
    const double v = atof(f);
    if (v > 0) sv->footprint_scale = v;
  }
  sv->params = q;
  if (cudaGetDevice(&sv->device) != cudaSuccess) {
    delete sv;
    return TP_ERR_CUDA;
  }
  try {
    for (int32_t i = 0; i < workers; ++i) sv->workers.emplace_back([sv] { sv->worker(); });
  } catch (const std::system_error &) {
    tp_server_destroy(sv);  // stops and joins the workers already started
    return TP_ERR_OOM;
  }
  *out = sv;
  return TP_OK;
}

tp_status tp_server_submit(tp_server *sv, const tp_request *req, uint64_t *ticket) {
  if (!sv || !req || !ticket || req->k < 1 || !(req->eps >= 0.0 && req->eps < 1.0))
    return TP_ERR_INVALID;
  const tp_request &r = *req;
  int64_t n = r.graph ? r.graph->n : r.n;
  int64_t m2 = r.graph ? r.graph->m2 : (r.xadj && r.n >= 0 ? r.xadj[r.n] : -1);
  if (n < 0 || m2 < 0 || (n > 0 && !r.part) || (!r.graph && (!r.xadj || (m2 > 0 && !r.adj))))
    return TP_ERR_INVALID;
  std::unique_ptr<Request> q;
  try {
    q = std::make_unique<Request>();
  } catch (const std::bad_alloc &) {
    return TP_ERR_OOM;
  }
  q->r = r;
  q->need = (int64_t)(sv->footprint_scale *
                      (double)footprint_model(n, m2, r.k, !r.graph, !r.graph && r.compress,
                                              sv->params.c_lim, std::max(1, sv->params.ip_attempts)));
  // a footprint beyond the budget: the request runs alone, capped at the budget
  if (q->need > sv->budget) q->need = sv->budget;
  q->t_submit = Clock::now();
  std::lock_guard<std::mutex> lk(sv->mu);
  if (sv->stopping) return TP_ERR_INVALID;
  const uint64_t t = sv->next_ticket;
  q->ticket = t;
  try {
    sv->reqs.emplace(t, std::move(q));
    try {
      sv->queue.push_back(t);
    } catch (const std::bad_alloc &) {
      sv->reqs.erase(t);
      throw;
    }
  } catch (const std::bad_alloc &) {
    return TP_ERR_OOM;
  }
  ++sv->next_ticket;
  *ticket = t;
  sv->cv_work.notify_all();
  return TP_OK;
}

tp_status tp_server_wait(tp_server *sv, uint64_t ticket, tp_stats *stats, tp_request_info *info) {
  if (!sv) return TP_ERR_INVALID;
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->reqs.find(ticket);
  if (it == sv->reqs.end()) return TP_ERR_INVALID;
  Request *q = it->second.get();
  if (q->waited) return TP_ERR_INVALID;  // another thread is already waiting on it
  q->waited = true;
  sv->cv_done.wait(lk, [&] { return q->state == 2; });
  if (stats) *stats = q->stats;
  if (info) {
    info->queued_ms = ms_between(q->t_submit, q->t_start);
    info->run_ms = ms_between(q->t_start, q->t_done);
    info->total_ms = ms_between(q->t_submit, q->t_done);
    info->footprint_bytes = q->need;
    info->peak_bytes = q->peak;
    info->retries = q->retries;
  }
  tp_status st = q->status;
  sv->reqs.erase(it);
  return st;
}

int64_t tp_server_peak_in_use(tp_server *sv) {
  if (!sv) return -1;
  std::lock_guard<std::mutex> lk(sv->mu);
  return sv->peak_in_use;
}

void tp_server_destroy(tp_server *sv) {
  if (!sv) return;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stopping = true;
    sv->cv_work.notify_all();
  }
  for (std::thread &t : sv->workers) t.join();
  delete sv;
}

}  // extern "C"
