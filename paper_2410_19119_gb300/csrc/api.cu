// extern "C" entry points declared in include/terapart.h.
#include <math.h>

#include <algorithm>
#include <atomic>
#include <memory>
#include <mutex>
#include <system_error>
#include <thread>
#include <vector>

#include "tp_internal.cuh"

namespace tp {
tp_graph *from_csr(int64_t n, const int64_t *xadj, const int32_t *adj, const int64_t *vwgt,
                   const int64_t *ewgt, int host, cudaStream_t s);
tp_graph *compress(const tp_graph *c, cudaStream_t s);
tp_graph *decompress(const tp_graph *z, cudaStream_t s);
tp_graph *from_compressed(int64_t n, uint64_t nbytes, const uint8_t *bytes, const uint64_t *off,
                          int host, cudaStream_t s);
void export_csr(const tp_graph *g, int64_t *xadj, int32_t *adj, int64_t *vw, int64_t *ew,
                cudaStream_t s);
void export_compressed(const tp_graph *g, uint8_t *bytes, uint64_t *off, cudaStream_t s);
void partition(tp_graph *g0, int32_t k, int64_t eps_ppm, const tp_params &p, int32_t *d_part,
               tp_stats *st, cudaStream_t s);
uint64_t encode_ex(const tp_graph *g, bool intervals, bool weights, uint64_t *d_off,
                   uint8_t *d_bytes, cudaStream_t s);
tp_graph *decode_ex(int64_t n, uint64_t nbytes, const uint8_t *d_bytes, const uint64_t *d_off,
                    bool intervals, bool weighted, cudaStream_t s);
void partition_union(const std::vector<const tp_graph *> &gs, const std::vector<int32_t> &idx,
                     const int32_t *k, int64_t eps_ppm, const tp_params &p,
                     int32_t *const *d_part, tp_stats *stats, cudaStream_t s);

namespace {
void pool_setup_once() {
  int dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) {
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
      uint64_t thr = UINT64_MAX;  // keep freed blocks cached in this process
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
  }
}

void pool_setup() {
  static std::once_flag once;
  std::call_once(once, pool_setup_once);
}

bool params_ok(const tp_params &p) {
  return p.cluster_rounds >= 0 && p.refine_rounds >= 0 && p.sub_rounds >= 1 && p.c_lim >= 1 &&
         p.ip_attempts >= 1 && p.max_levels >= 1 && p.max_levels <= 64;
}

tp_params resolve(const tp_params *p) {
  tp_params q;
  if (p) q = *p;
  else tp_params_default(&q);
  TP_REQUIRE(params_ok(q), TP_ERR_INVALID);
  return q;
}

int64_t eps_ppm_of(double eps) { return (int64_t)llround(eps * 1e6); }
}  // namespace
}  // namespace tp

using namespace tp;

extern "C" {

void tp_params_default(tp_params *p) {
  p->seed = 1;
  p->cluster_rounds = 5;
  p->refine_rounds = 5;
  p->sub_rounds = 8;
  p->c_lim = 160;
  p->ip_attempts = 8;
  p->two_hop = 1;
  p->max_levels = 64;
  p->tier_lane = 32;
  p->tier_small = 64;
  p->tier_mid = 512;
  p->warps_per_block = 8;
  p->use_graphs = 1;
  p->graph_n = 1 << 19;
  p->table_slack = 2;
}

const char *tp_status_string(tp_status s) {
  switch (s) {
  case TP_OK: return "ok";
  case TP_ERR_INVALID: return "invalid argument or graph";
  case TP_ERR_OOM: return "out of device memory";
  case TP_ERR_CUDA: return "CUDA runtime error";
  case TP_ERR_CORRUPT: return "corrupt compressed graph";
  case TP_ERR_TIMEOUT: return "device wait timed out";
  case TP_ERR_BUDGET: return "memory budget exceeded";
  }
  return "unknown status";
}

tp_status tp_set_allocator(void *(*alloc)(size_t, void *, void *),
                           void (*free_fn)(void *, size_t, void *, void *), void *ctx);

tp_status tp_graph_from_csr(int64_t n, const int64_t *xadj, const int32_t *adj,
                            const int64_t *vwgt, const int64_t *ewgt, int host_ptrs, void *stream,
                            tp_graph **out) {
  if (!out) return TP_ERR_INVALID;
  *out = nullptr;
  return guard([&] {
    pool_setup();
    *out = from_csr(n, xadj, adj, vwgt, ewgt, host_ptrs, (cudaStream_t)stream);
  });
}

tp_status tp_graph_compress(const tp_graph *csr, void *stream, tp_graph **out) {
  if (!csr || !out) return TP_ERR_INVALID;
  *out = nullptr;
  return guard([&] { *out = compress(csr, (cudaStream_t)stream); });
}

tp_status tp_graph_from_compressed(int64_t n, uint64_t nbytes, const uint8_t *bytes,
                                   const uint64_t *off, int host_ptrs, void *stream,
                                   tp_graph **out) {
  if (!out) return TP_ERR_INVALID;
  *out = nullptr;
  return guard([&] {
    pool_setup();
    *out = from_compressed(n, nbytes, bytes, off, host_ptrs, (cudaStream_t)stream);
  });
}

tp_status tp_encode_ex(const tp_graph *g, int32_t intervals, int32_t weights, uint64_t *d_off,
                       uint8_t *d_bytes, uint64_t *nbytes, void *stream) {
  if (!g || !d_off || !nbytes) return TP_ERR_INVALID;
  return guard([&] {
    *nbytes = encode_ex(g, intervals != 0, weights != 0, d_off, d_bytes, (cudaStream_t)stream);
  });
}

tp_status tp_graph_from_stream_ex(int64_t n, uint64_t nbytes, const uint8_t *d_bytes,
                                  const uint64_t *d_off, int32_t intervals, int32_t weighted,
                                  void *stream, tp_graph **out) {
  if (!out) return TP_ERR_INVALID;
  *out = nullptr;
  return guard([&] {
    pool_setup();
    *out = decode_ex(n, nbytes, d_bytes, d_off, intervals != 0, weighted != 0,
                     (cudaStream_t)stream);
  });
}

tp_status tp_graph_decompress(const tp_graph *g, void *stream, tp_graph **out_csr) {
  if (!g || !out_csr) return TP_ERR_INVALID;
  *out_csr = nullptr;
  return guard([&] { *out_csr = decompress(g, (cudaStream_t)stream); });
}

tp_status tp_graph_info(const tp_graph *g, int64_t *n, int64_t *m2, int *compressed,
                        size_t *bytes, size_t *stream_bytes) {
  if (!g) return TP_ERR_INVALID;
  if (stream_bytes) *stream_bytes = g->compressed ? g->nbytes : 0;
  if (n) *n = g->n;
  if (m2) *m2 = g->m2;
  if (compressed) *compressed = g->compressed;
  if (bytes) {
    if (g->compressed)
      *bytes = g->nbytes + (g->n + 1) * (g->off_is64 ? 8 : 4);
    else
      *bytes = (g->n + 1) * 8 + g->m2 * 4 + (g->unit_vw ? 0 : g->n * 8) +
               (g->unit_ew ? 0 : g->m2 * 8);
  }
  return TP_OK;
}

tp_status tp_graph_export_csr(const tp_graph *g, int64_t *d_xadj, int32_t *d_adj, int64_t *d_vw,
                              int64_t *d_ew, void *stream) {
  if (!g) return TP_ERR_INVALID;
  return guard([&] { export_csr(g, d_xadj, d_adj, d_vw, d_ew, (cudaStream_t)stream); });
}

tp_status tp_graph_export_compressed(const tp_graph *g, uint8_t *d_bytes, uint64_t *d_off,
                                     void *stream) {
  if (!g) return TP_ERR_INVALID;
  return guard([&] { export_compressed(g, d_bytes, d_off, (cudaStream_t)stream); });
}

tp_status tp_graph_check(const tp_graph *g, void *stream) {
  if (!g) return TP_ERR_INVALID;
  tp_status st = TP_OK;
  tp_status r = guard([&] {
    cudaStream_t s = (cudaStream_t)stream;
    int32_t e = read_scalar(g->err.get(), s);
    if (e) TP_CUDA(cudaMemsetAsync(g->err.get(), 0, sizeof(int32_t), s));
    TP_CUDA(cudaStreamSynchronize(s));
    st = (tp_status)e;
  });
  return r != TP_OK ? r : st;
}

void tp_graph_destroy(tp_graph *g) {
  if (!g) return;
  cudaDeviceSynchronize();  // nothing may still run on g, on any stream
  g->rehome();
  delete g;
}

tp_status tp_lp_subround(const tp_graph *g, int32_t *d_label, int64_t *d_lw, int64_t nlabels,
                         int64_t cap, uint64_t round_key, int32_t S, int32_t s, void *stream) {
  if (!g || S < 1 || s < 0 || s >= S || nlabels < 1) return TP_ERR_INVALID;
  return guard([&] {
    cudaStream_t st = (cudaStream_t)stream;
    tp_params p;
    tp_params_default(&p);
    LpWork w;
    w.init(g->n, nlabels, st);
    LpState state{d_label, d_lw, nlabels, cap};
    lp_subround(const_cast<tp_graph *>(g), state, w, round_key, S, s, p, st);
    TP_CUDA(cudaStreamSynchronize(st));
  });
}

tp_status tp_lp_cluster(const tp_graph *g, int64_t max_cluster_weight, const tp_params *p,
                        int32_t level, int32_t *d_cluster, void *stream) {
  if (!g || max_cluster_weight < 1 || (g->n && !d_cluster)) return TP_ERR_INVALID;
  return guard([&] {
    tp_params q = resolve(p);
    lp_cluster(const_cast<tp_graph *>(g), max_cluster_weight, q, level, d_cluster,
               (cudaStream_t)stream);
  });
}

tp_status tp_contract(const tp_graph *g, const int32_t *d_cluster, void *stream,
                      tp_graph **coarse, int32_t *d_map) {
  if (!g || !coarse || (g->n && !d_cluster)) return TP_ERR_INVALID;
  *coarse = nullptr;
  return guard([&] { *coarse = contract(g, d_cluster, d_map, (cudaStream_t)stream); });
}

tp_status tp_initial_partition(const tp_graph *g, int32_t k, int64_t l_max, const tp_params *p,
                               int32_t *d_part, void *stream) {
  if (!g || k < 1 || (g->n && !d_part)) return TP_ERR_INVALID;
  return guard([&] {
    tp_params q = resolve(p);
    initial_partition(g, k, l_max, q, d_part, (cudaStream_t)stream);
    TP_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  });
}

tp_status tp_lp_refine(const tp_graph *g, int32_t k, int64_t l_max, const tp_params *p,
                       int32_t level, int32_t *d_part, void *stream) {
  if (!g || k < 1 || (g->n && !d_part)) return TP_ERR_INVALID;
  return guard([&] {
    tp_params q = resolve(p);
    cudaStream_t s = (cudaStream_t)stream;
    Buf<int64_t> B(k, s);
    block_weights(g, d_part, k, B.get(), s);
    lp_refine(const_cast<tp_graph *>(g), k, l_max, q, level, d_part, B.get(), s);
  });
}

tp_status tp_rebalance(const tp_graph *g, int32_t k, int64_t l_max, int32_t *d_part,
                       int *balanced, void *stream) {
  if (!g || k < 1 || (g->n && !d_part)) return TP_ERR_INVALID;
  return guard([&] {
    cudaStream_t s = (cudaStream_t)stream;
    tp_params q;
    tp_params_default(&q);
    Buf<int64_t> B(k, s);
    block_weights(g, d_part, k, B.get(), s);
    int ok = 1;
    rebalance_moves(const_cast<tp_graph *>(g), k, l_max, d_part, B.get(), &ok, q, s);
    TP_CUDA(cudaStreamSynchronize(s));
    if (balanced) *balanced = ok;
  });
}

tp_status tp_metrics(const tp_graph *g, const int32_t *d_part, int32_t k, int64_t *cut,
                     int64_t *h_block_weights, void *stream) {
  if (!g || k < 1 || (g->n && !d_part)) return TP_ERR_INVALID;
  return guard([&] {
    cudaStream_t s = (cudaStream_t)stream;
    if (h_block_weights) {
      Buf<int64_t> B(k, s);
      block_weights(g, d_part, k, B.get(), s);
      TP_CUDA(cudaMemcpyAsync(h_block_weights, B.get(), k * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    }
    int64_t c = edge_cut(g, d_part, s);
    if (cut) *cut = c;
  });
}

tp_status tp_partition(const tp_graph *g, int32_t k, double eps, const tp_params *p,
                       int32_t *d_part, tp_stats *stats, void *stream) {
  if (!g || k < 1 || !(eps >= 0.0 && eps < 1.0) || (g->n && !d_part)) return TP_ERR_INVALID;
  return guard([&] {
    tp_params q = resolve(p);
    partition(const_cast<tp_graph *>(g), k, eps_ppm_of(eps), q, d_part, stats,
              (cudaStream_t)stream);
  });
}

// Batched mode: the graphs are partitioned together, one union graph per
// level (batch.cu), so kernels are launched per level rather than per graph
// and every graph's result equals tp_partition of that graph alone. Graphs
// with k = 1 or no vertices are trivial; compressed inputs are decompressed
// first (the result does not depend on the representation). Large batches
// are cut into groups (in input order) that bound a union's size; up to
// `concurrency` groups run at once, each on a stream of its own worker.
tp_status tp_partition_batch(int32_t count, tp_graph *const *graphs, const int32_t *k, double eps,
                             const tp_params *p, int32_t *const *d_part, tp_stats *stats,
                             tp_status *status, int32_t concurrency) {
  if (count < 0 || concurrency < 1 || !(eps >= 0.0 && eps < 1.0)) return TP_ERR_INVALID;
  if (count == 0) return TP_OK;
  if (!graphs || !k || !d_part) return TP_ERR_INVALID;
  for (int32_t i = 0; i < count; ++i)
    if (!graphs[i] || k[i] < 1 || (graphs[i]->n && !d_part[i])) return TP_ERR_INVALID;
  {  // a graph caches per-level state while it is partitioned: no handle twice
    std::vector<tp_graph *> sorted(graphs, graphs + count);
    std::sort(sorted.begin(), sorted.end());
    if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end()) return TP_ERR_INVALID;
  }
  tp_params q;
  try {
    q = resolve(p);
  } catch (const Error &e) {
    return e.code;
  }
  const int64_t eps_ppm = eps_ppm_of(eps);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return TP_ERR_CUDA;
  std::vector<tp_status> st((size_t)count, TP_OK);
  // groups of non-trivial graphs in input order, each a union of bounded size
  // (graphs of a union are one grid row each: at most 2^15 per group)
  constexpr int64_t kGroupN = (int64_t)1 << 28, kGroupM = (int64_t)1 << 30, kGroupG = 1 << 15;
  std::vector<std::vector<int32_t>> groups;
  std::vector<int32_t> trivial;
  {
    int64_t gn = 0, gm = 0;
    for (int32_t i = 0; i < count; ++i) {
      const tp_graph *g = graphs[i];
      if (k[i] == 1 || g->n == 0) {
        trivial.push_back(i);
        continue;
      }
      if (groups.empty() || gn + g->n > kGroupN || gm + g->m2 > kGroupM ||
          (int64_t)groups.back().size() == kGroupG) {
        groups.emplace_back();
        gn = gm = 0;
      }
      groups.back().push_back(i);
      gn += g->n;
      gm += g->m2;
    }
  }
  std::vector<const tp_graph *> gs(graphs, graphs + count);
  std::atomic<int32_t> next{0};
  const int32_t ngroups = (int32_t)groups.size();
  auto worker = [&](bool first) {
    cudaStream_t s = nullptr;
    if (cudaSetDevice(dev) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
      (void)cudaGetLastError();
      for (int32_t t; (t = next.fetch_add(1)) < ngroups;)
        for (int32_t i : groups[(size_t)t]) st[(size_t)i] = TP_ERR_CUDA;
      return;
    }
    if (first) {  // trivial graphs: every vertex in block 0
      for (int32_t i : trivial) {
        st[(size_t)i] = guard([&] {
          const tp_graph *g = graphs[i];
          if (g->n) TP_CUDA(cudaMemsetAsync(d_part[i], 0, g->n * sizeof(int32_t), s));
          if (stats) {
            tp_stats &S = stats[i];
            S = tp_stats{};
            S.l_max = block_cap(g->total_vw, k[i], eps_ppm);
            S.u_max = cluster_cap(g->total_vw, k[i], eps_ppm);
            S.levels = 1;
            S.level_n[0] = g->n;
            S.level_m2[0] = g->m2;
            S.max_block_weight = k[i] == 1 ? g->total_vw : 0;
            S.balanced = S.max_block_weight <= S.l_max;
            const int64_t perfect = (g->total_vw + k[i] - 1) / k[i];
            S.imbalance = perfect > 0 ? (double)S.max_block_weight / (double)perfect - 1.0 : 0.0;
          }
        });
      }
    }
    for (int32_t t; (t = next.fetch_add(1)) < ngroups;) {
      const std::vector<int32_t> &grp = groups[(size_t)t];
      tp_status r = guard([&] {
        std::vector<const tp_graph *> local = gs;
        std::vector<std::unique_ptr<tp_graph>> tmp;  // CSR copies of compressed inputs
        for (int32_t i : grp)
          if (graphs[i]->compressed) {
            tmp.emplace_back(decompress(graphs[i], s));
            local[(size_t)i] = tmp.back().get();
          }
        partition_union(local, grp, k, eps_ppm, q, d_part, stats, s);
        TP_CUDA(cudaStreamSynchronize(s));
      });
      for (int32_t i : grp) st[(size_t)i] = r;
    }
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
  };
  const int32_t nthreads = std::max(1, std::min(concurrency, std::min(ngroups, 64)));
  std::vector<std::thread> pool;
  for (int32_t t = 1; t < nthreads; ++t) {
    try {
      pool.emplace_back(worker, false);
    } catch (const std::system_error &) {
      break;  // fewer threads: the shared counter still hands out every group
    }
  }
  worker(true);
  for (std::thread &t : pool) t.join();
  tp_status first = TP_OK;
  for (int32_t i = 0; i < count; ++i) {
    if (status) status[i] = st[(size_t)i];
    if (first == TP_OK) first = st[(size_t)i];
  }
  return first;
}

}  // extern "C"
