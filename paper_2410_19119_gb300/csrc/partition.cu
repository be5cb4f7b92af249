// Multilevel driver (Section "The Multilevel Scheme" of the paper), the
// balance constraint and metrics of the problem statement (Section
// "Introduction"), and projection between levels.
#include <algorithm>
#include <memory>
#include <vector>

#include "decode.cuh"

namespace tp {

int64_t cluster_cap(int64_t W, int32_t k, int64_t eps_ppm) {
  __int128 num = (__int128)eps_ppm * W;
  int64_t u = (int64_t)(num / ((__int128)1000000 * k));
  return u < 1 ? 1 : u;
}

int64_t block_cap(int64_t W, int32_t k, int64_t eps_ppm) {
  int64_t perfect = (W + k - 1) / k;
  return (int64_t)(((__int128)(1000000 + eps_ppm) * perfect) / 1000000);
}

namespace {

constexpr int kHistMax = 4096;

__global__ void k_block_weights(const int32_t *part, const int64_t *vw, int64_t n, int32_t k,
                                int64_t *B) {
  extern __shared__ int64_t hist[];
  const bool local = k <= kHistMax;
  if (local)
    for (int b = threadIdx.x; b < k; b += blockDim.x) hist[b] = 0;
  __syncthreads();
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n;
       u += (int64_t)gridDim.x * blockDim.x) {
    int64_t w = vw ? vw[u] : 1;
    if (local) atomicAdd((unsigned long long *)&hist[part[u]], (unsigned long long)w);
    else atomicAdd((unsigned long long *)&B[part[u]], (unsigned long long)w);
  }
  __syncthreads();
  if (local)
    for (int b = threadIdx.x; b < k; b += blockDim.x)
      if (hist[b]) atomicAdd((unsigned long long *)&B[b], (unsigned long long)hist[b]);
}

// Edge cut contributions of low-degree vertices, one thread per vertex.
template <bool COMP>
__global__ void k_cut_thread(GView g, const uint8_t *tier, const int32_t *part,
                             unsigned long long *out) {
  int64_t acc = 0;
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < g.n;
       u += (int64_t)gridDim.x * blockDim.x) {
    const uint8_t t = tier[u];
    if (t != TIER_LANE && t != TIER_SMALL) continue;
    const int32_t pu = part[u];
    thread_neighbours<COMP>(g, u, [&](int32_t v, int64_t w) {
      if (part[v] != pu) acc += w;
    });
  }
  acc = warp_sum(acc);
  if (lane_id() == 0 && acc) atomicAdd(out, (unsigned long long)acc);
}

// Edge cut contributions of the other vertices, one warp per vertex.
template <bool COMP>
__global__ void k_cut(GView g, const uint8_t *tier, const int32_t *part, unsigned long long *out) {
  int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  int64_t acc = 0;
  for (int64_t u = warp; u < g.n; u += nw) {
    if (tier[u] == TIER_LANE || tier[u] == TIER_SMALL) continue;
    int32_t pu = part[u];
    warp_neighbours<COMP>(g, u, -1, [&](bool has, int32_t v, int64_t w, int64_t) {
      if (has && part[v] != pu) acc += w;
    });
  }
  acc = warp_sum(acc);
  if (lane_id() == 0 && acc) atomicAdd(out, (unsigned long long)acc);
}

__global__ void k_project(const int32_t *coarse, const int32_t *map, int64_t n, int32_t *fine) {
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n;
       u += (int64_t)gridDim.x * blockDim.x)
    fine[u] = coarse[map[u]];
}

}  // namespace

void block_weights(const tp_graph *g, const int32_t *part, int32_t k, int64_t *d_B,
                   cudaStream_t s) {
  TP_CUDA(cudaMemsetAsync(d_B, 0, (size_t)k * sizeof(int64_t), s));
  if (g->n == 0) return;
  size_t sm = k <= kHistMax ? (size_t)k * sizeof(int64_t) : 0;
  launch(k_block_weights, grid_for(g->n, 256, num_sms() * 4), 256, sm, s, part, g->unit_vw ? nullptr : g->vw.get(), g->n, k, d_B);
  TP_LAUNCH_CHECK();
}

int64_t edge_cut(const tp_graph *g, const int32_t *part, cudaStream_t s) {
  Buf<unsigned long long> acc(1, s);
  TP_CUDA(cudaMemsetAsync(acc.get(), 0, sizeof(unsigned long long), s));
  if (g->n) {
    if (!g->tiers.built) {
      tp_params dp;
      tp_params_default(&dp);
      build_tiers(const_cast<tp_graph *>(g), dp, s);
    }
    const TierCache &T = g->tiers;
    const uint8_t *tier = T.tier.get();
    unsigned tb = grid_for(g->n, 256);
    if (g->compressed) launch(k_cut_thread<true>, tb, 256, 0, s, view(g), tier, part, acc.get());
    else launch(k_cut_thread<false>, tb, 256, 0, s, view(g), tier, part, acc.get());
    if (T.n_mid + T.n_mid2 + T.n_big0 + T.n_big1 + T.n_big + T.n_big2 + T.n_huge > 0) {
      unsigned b = grid_for(g->n * 32, 256);
      if (g->compressed) launch(k_cut<true>, b, 256, 0, s, view(g), tier, part, acc.get());
      else launch(k_cut<false>, b, 256, 0, s, view(g), tier, part, acc.get());
    }
    TP_LAUNCH_CHECK();
  }
  return (int64_t)(read_scalar(acc.get(), s) / 2);
}

void project(const int32_t *coarse_part, const int32_t *map, int64_t n, int32_t *fine_part,
             cudaStream_t s) {
  if (n == 0) return;
  launch(k_project, grid_for(n, 256), 256, 0, s, coarse_part, map, n, fine_part);
  TP_LAUNCH_CHECK();
}

struct EventTimer {
  cudaEvent_t a{}, b{};
  cudaStream_t s;
  explicit EventTimer(cudaStream_t st) : s(st) {
    TP_CUDA(cudaEventCreate(&a));
    TP_CUDA(cudaEventCreate(&b));
  }
  void start() { TP_CUDA(cudaEventRecord(a, s)); }
  void stop() { TP_CUDA(cudaEventRecord(b, s)); }
  double ms() {
    TP_CUDA(cudaEventSynchronize(b));
    float m = 0;
    TP_CUDA(cudaEventElapsedTime(&m, a, b));
    return m;
  }
  ~EventTimer() {
    cudaEventDestroy(a);
    cudaEventDestroy(b);
  }
};

void partition(tp_graph *g0, int32_t k, int64_t eps_ppm, const tp_params &p, int32_t *d_part,
               tp_stats *st, cudaStream_t s) {
  tp_stats local{};
  tp_stats &S = st ? *st : local;
  S = tp_stats{};
  const int64_t mark = mem_mark();
  const int64_t W = g0->total_vw;
  const int64_t U = cluster_cap(W, k, eps_ppm);
  const int64_t l_max = block_cap(W, k, eps_ppm);
  S.l_max = l_max;
  S.u_max = U;
  S.level_n[0] = g0->n;
  S.level_m2[0] = g0->m2;
  std::vector<tp_graph *> levels{g0};
  std::vector<Buf<int32_t>> maps;
  EventTimer t_all(s), t_phase(s), t_lp(s);
  struct Cleanup {
    std::vector<tp_graph *> &lv;
    ~Cleanup() {
      for (size_t i = 1; i < lv.size(); ++i) delete lv[i];
    }
  } cleanup{levels};
  const int32_t max_levels = std::max(1, std::min(p.max_levels, 64));
  t_phase.start();
  if (k > 1) {
    while (levels.back()->n > (int64_t)p.c_lim * k && (int32_t)levels.size() < max_levels) {
      tp_graph *g = levels.back();
      const int32_t level = (int32_t)levels.size() - 1;
      Buf<int32_t> C(g->n, s), map(g->n, s);
      if (level == 0) lp_cluster(g, U, p, level, C.get(), s, t_lp.a, t_lp.b);
      else lp_cluster(g, U, p, level, C.get(), s);
      tp_graph *cg = contract(g, C.get(), map.get(), s);
      if (20 * cg->n > 19 * g->n) {
        delete cg;
        break;
      }
      levels.push_back(cg);
      maps.push_back(std::move(map));
      mem_trace_dump(level == 0 ? "after contracting level 0" : "after contracting a level");
      S.level_n[levels.size() - 1] = cg->n;
      S.level_m2[levels.size() - 1] = cg->m2;
    }
  }
  t_phase.stop();
  S.ms_coarsen = t_phase.ms();
  if (levels.size() > 1) S.ms_lp_level0 = t_lp.ms();
  S.levels = (int32_t)levels.size();
  const int32_t L = S.levels - 1;
  Buf<int64_t> B(std::max(k, 1), s);
  Buf<int32_t> cur(std::max<int64_t>(levels[L]->n, 1), s);
  t_phase.start();
  // a compressed input that is not coarsened at all is partitioned as CSR
  std::unique_ptr<tp_graph> ip_csr(levels[L]->compressed ? decompress(levels[L], s) : nullptr);
  initial_partition(ip_csr ? ip_csr.get() : levels[L], k, l_max, p, cur.get(), s);
  ip_csr.reset();
  t_phase.stop();
  S.ms_initial = t_phase.ms();
  mem_trace_dump("after initial partitioning");
  t_phase.start();
  for (int32_t l = L; l >= 0; --l) {
    tp_graph *g = levels[l];
    if (l < L) {
      Buf<int32_t> fine(std::max<int64_t>(g->n, 1), s);
      project(cur.get(), maps[l].get(), g->n, fine.get(), s);
      cur = std::move(fine);
    }
    if (k > 1 && g->n) {
      block_weights(g, cur.get(), k, B.get(), s);
      int balanced = 1;
      rebalance_moves(g, k, l_max, cur.get(), B.get(), &balanced, p, s);
      lp_refine(g, k, l_max, p, l, cur.get(), B.get(), s);
    }
  }
  t_phase.stop();
  S.ms_uncoarsen = t_phase.ms();
  if (g0->n)
    TP_CUDA(cudaMemcpyAsync(d_part, cur.get(), g0->n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
  // statistics of the final partition
  block_weights(g0, d_part, k, B.get(), s);
  std::vector<int64_t> hB(k);
  TP_CUDA(cudaMemcpyAsync(hB.data(), B.get(), k * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  S.cut = edge_cut(g0, d_part, s);  // synchronises
  int64_t mx = 0;
  for (int64_t b : hB) mx = std::max(mx, b);
  S.max_block_weight = mx;
  S.balanced = mx <= l_max;
  int64_t perfect = (W + k - 1) / k;
  S.imbalance = perfect > 0 ? (double)mx / (double)perfect - 1.0 : 0.0;
  S.peak_bytes = mem_peak_since(mark);
  mem_trace_dump("tp_partition");
  int32_t e = read_scalar(g0->err.get(), s);
  TP_REQUIRE(e == 0, (tp_status)e);
}

}  // namespace tp
