// Cluster contraction (Section "Contraction" of the paper): every cluster
// becomes a coarse vertex, w'(a,b) sums the weights of the fine edges between
// clusters a and b, intra-cluster edges vanish.
//
// GPU form: coarse ids are ranks of the non-empty labels (mark + exclusive
// scan, so ids are deterministic where the paper's atomic counters are not);
// every inter-cluster adjacency entry is emitted as the key a*n' + b at a
// position fixed by a scan of per-vertex (per-chunk for hubs) counts, sorted
// with the library's LSD radix sort, and duplicate keys are reduced into the
// canonical coarse CSR (neighbours ascending, int64 weights).
#include <algorithm>

#include "decode.cuh"

namespace tp {

namespace {

__global__ void k_mark(const int32_t *C, int64_t n, int32_t *flag) {
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n;
       u += (int64_t)gridDim.x * blockDim.x)
    flag[C[u]] = 1;
}

__global__ void k_map(const int32_t *C, const int64_t *rank, const int64_t *vw, int64_t n,
                      int32_t *map, int64_t *cvw) {
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n;
       u += (int64_t)gridDim.x * blockDim.x) {
    int32_t a = (int32_t)rank[C[u]];
    map[u] = a;
    atomicAdd((unsigned long long *)&cvw[a], (unsigned long long)(vw ? vw[u] : 1));
  }
}

// Batched graphs: coarse offset of every graph (the rank of its first vertex).
__global__ void k_seg_rank(const int64_t *rank, const int64_t *voff, int64_t nseg, int64_t *coff) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= nseg;
       i += (int64_t)gridDim.x * blockDim.x)
    coff[i] = rank[voff[i]];
}

__device__ __forceinline__ bool thread_tier(uint8_t t) { return t == TIER_LANE || t == TIER_SMALL; }

// Per-vertex count of inter-cluster entries, one thread per low-degree vertex.
template <bool COMP>
__global__ void k_count_thread(GView g, const uint8_t *tier, const int32_t *map, int64_t *cnt) {
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < g.n;
       u += (int64_t)gridDim.x * blockDim.x) {
    if (!thread_tier(tier[u])) continue;
    const int32_t a = map[u];
    int64_t c = 0;
    thread_neighbours<COMP>(g, u, [&](int32_t v, int64_t) { c += map[v] != a; });
    cnt[u] = c;
  }
}

// Per-vertex count of inter-cluster entries, one warp per medium vertex
// (hubs are counted per chunk below).
template <bool COMP>
__global__ void k_count(GView g, const uint8_t *tier, const int32_t *map, int64_t *cnt) {
  int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t u = warp; u < g.n; u += nw) {
    if (thread_tier(tier[u])) continue;
    int64_t c = 0;
    if (tier[u] != TIER_HUGE) {
      int32_t a = map[u];
      warp_neighbours<COMP>(g, u, -1, [&](bool has, int32_t v, int64_t, int64_t) {
        c += __popc(__ballot_sync(kFull, has && map[v] != a));
      });
    }
    if (lane_id() == 0) cnt[u] = c;
  }
}

__device__ __forceinline__ int64_t find_item(const int64_t *start, int64_t cnt, int64_t item) {
  int64_t lo = 0, hi = cnt - 1;
  while (lo < hi) {
    int64_t mid = (lo + hi + 1) / 2;
    if (start[mid] <= item) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

template <bool COMP>
__global__ void k_count_chunks(GView g, const int32_t *huge, int64_t n_huge,
                               const int64_t *chunk_start, int64_t n_items, const int32_t *map,
                               int64_t *cnt) {
  int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t it = warp; it < n_items; it += nw) {
    int64_t i = find_item(chunk_start, n_huge, it);
    int64_t u = huge[i];
    int32_t a = map[u];
    int64_t c = 0;
    warp_neighbours<COMP>(g, u, it - chunk_start[i], [&](bool has, int32_t v, int64_t, int64_t) {
      c += __popc(__ballot_sync(kFull, has && map[v] != a));
    });
    if (lane_id() == 0) cnt[it] = c;
  }
}

template <bool COMP>
__device__ __forceinline__ void emit(const GView &g, int64_t u, int64_t chunk, const int32_t *map,
                                     int64_t nc, int64_t pos, uint64_t *keys, uint64_t *vals) {
  int32_t a = map[u];
  warp_neighbours<COMP>(g, u, chunk, [&](bool has, int32_t v, int64_t w, int64_t) {
    int32_t b = has ? map[v] : a;
    bool keep = has && b != a;
    unsigned m = __ballot_sync(kFull, keep);
    if (keep) {
      int64_t at = pos + __popc(m & lanemask_lt());
      keys[at] = (uint64_t)a * (uint64_t)nc + (uint64_t)b;
      if (vals) vals[at] = (uint64_t)w;
    }
    pos += __popc(m);
  });
}

template <bool COMP>
__global__ void k_emit_thread(GView g, const uint8_t *tier, const int32_t *map, int64_t nc,
                              const int64_t *off, uint64_t *keys, uint64_t *vals) {
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < g.n;
       u += (int64_t)gridDim.x * blockDim.x) {
    if (!thread_tier(tier[u])) continue;
    const int32_t a = map[u];
    int64_t pos = off[u];
    thread_neighbours<COMP>(g, u, [&](int32_t v, int64_t w) {
      const int32_t b = map[v];
      if (b == a) return;
      keys[pos] = (uint64_t)a * (uint64_t)nc + (uint64_t)b;
      if (vals) vals[pos] = (uint64_t)w;
      ++pos;
    });
  }
}

template <bool COMP>
__global__ void k_emit(GView g, const uint8_t *tier, const int32_t *map, int64_t nc,
                       const int64_t *off, uint64_t *keys, uint64_t *vals) {
  int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t u = warp; u < g.n; u += nw)
    if (!thread_tier(tier[u]) && tier[u] != TIER_HUGE)
      emit<COMP>(g, u, -1, map, nc, off[u], keys, vals);
}

template <bool COMP>
__global__ void k_emit_chunks(GView g, const int32_t *huge, int64_t n_huge,
                              const int64_t *chunk_start, int64_t n_items, const int32_t *map,
                              int64_t nc, int64_t base, const int64_t *off, uint64_t *keys,
                              uint64_t *vals) {
  int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t it = warp; it < n_items; it += nw) {
    int64_t i = find_item(chunk_start, n_huge, it);
    emit<COMP>(g, huge[i], it - chunk_start[i], map, nc, base + off[it], keys, vals);
  }
}

__global__ void k_heads(const uint64_t *keys, int64_t m, int32_t *flag) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x)
    flag[i] = i == 0 || keys[i] != keys[i - 1];
}

__global__ void k_reduce(const uint64_t *keys, const uint64_t *vals, const int64_t *idx, int64_t m,
                         int64_t nc, int32_t *adj, int64_t *ew, int64_t *deg) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x) {
    int64_t j = idx[i + 1] - 1;  // heads in [0, i] minus one: this key's output slot
    uint64_t k = keys[i];
    bool head = i == 0 || k != keys[i - 1];
    if (head) {
      adj[j] = (int32_t)(k % (uint64_t)nc);
      atomicAdd((unsigned long long *)&deg[k / (uint64_t)nc], 1ull);
    }
    atomicAdd((unsigned long long *)&ew[j], vals ? vals[i] : 1ull);
  }
}

}  // namespace

tp_graph *contract(const tp_graph *g, const int32_t *C, int32_t *d_map, cudaStream_t s,
                   const int64_t *seg_voff, int64_t nseg, int64_t *seg_coff) {
  int64_t n = g->n;
  tp_graph *cg = new_graph();
  try {
    cg->err.alloc(1, s);
    TP_CUDA(cudaMemsetAsync(cg->err.get(), 0, sizeof(int32_t), s));
    cg->unit_vw = 0;
    cg->unit_ew = 0;
    if (n == 0) {
      cg->xadj.alloc(1, s);
      TP_CUDA(cudaMemsetAsync(cg->xadj.get(), 0, 8, s));
      TP_CUDA(cudaStreamSynchronize(s));
      return cg;
    }
    Buf<int32_t> flag(n, s);
    TP_CUDA(cudaMemsetAsync(flag.get(), 0, n * sizeof(int32_t), s));
    launch(k_mark, grid_for(n, 256), 256, 0, s, C, n, flag.get());
    TP_LAUNCH_CHECK();
    Buf<int64_t> rank(n + 1, s);
    exclusive_scan_i32_to_i64(flag.get(), rank.get(), n, s);
    if (seg_voff) {
      launch(k_seg_rank, grid_for(nseg + 1, 256), 256, 0, s, rank.get(), seg_voff, nseg, seg_coff);
      TP_LAUNCH_CHECK();
    }
    int64_t nc = read_scalar(rank.get() + n, s);
    cg->n = nc;
    Buf<int32_t> own_map;
    int32_t *map = d_map;
    if (!map) {
      own_map.alloc(n, s);
      map = own_map.get();
    }
    cg->vw.alloc(nc, s);
    TP_CUDA(cudaMemsetAsync(cg->vw.get(), 0, nc * sizeof(int64_t), s));
    launch(k_map, grid_for(n, 256), 256, 0, s, C, rank.get(), g->unit_vw ? nullptr : g->vw.get(), n,
                                             map, cg->vw.get());
    TP_LAUNCH_CHECK();
    cg->total_vw = g->total_vw;

    // inter-cluster entries: counts, offsets, emission
    tp_params dp;
    tp_params_default(&dp);
    if (!g->tiers.built) build_tiers(const_cast<tp_graph *>(g), dp, s);
    const TierCache &T = g->tiers;
    GView v = view(g);
    const bool comp = g->compressed;
    Buf<int64_t> off(n + 1, s);
    unsigned wb = grid_for(n * 32, 256);
    unsigned tb = grid_for(n, 256);
    const bool warp_work = T.n_mid + T.n_big + T.n_big2 > 0;
    if (comp) launch(k_count_thread<true>, tb, 256, 0, s, v, T.tier.get(), map, off.get());
    else launch(k_count_thread<false>, tb, 256, 0, s, v, T.tier.get(), map, off.get());
    if (warp_work || T.n_huge) {  // the warp kernel also zeroes the hub entries
      if (comp) launch(k_count<true>, wb, 256, 0, s, v, T.tier.get(), map, off.get());
      else launch(k_count<false>, wb, 256, 0, s, v, T.tier.get(), map, off.get());
    }
    TP_LAUNCH_CHECK();
    exclusive_scan_i64(off.get(), off.get(), n, s);
    int64_t m_small = read_scalar(off.get() + n, s);
    int64_t m_huge = 0;
    Buf<int64_t> hoff;
    if (T.n_huge) {
      hoff.alloc(T.n_huge_chunks + 1, s);
      unsigned hb = grid_for(T.n_huge_chunks * 32, 256);
      if (comp)
        launch(k_count_chunks<true>, hb, 256, 0, s, v, T.huge.get(), T.n_huge, T.huge_chunk_start.get(),
                                                T.n_huge_chunks, map, hoff.get());
      else
        launch(k_count_chunks<false>, hb, 256, 0, s, v, T.huge.get(), T.n_huge, T.huge_chunk_start.get(),
                                                 T.n_huge_chunks, map, hoff.get());
      TP_LAUNCH_CHECK();
      exclusive_scan_i64(hoff.get(), hoff.get(), T.n_huge_chunks, s);
      m_huge = read_scalar(hoff.get() + T.n_huge_chunks, s);
    }
    int64_t m = m_small + m_huge;
    const bool weighted = !g->unit_ew;
    Buf<uint64_t> keys(std::max<int64_t>(m, 1), s), vals;
    if (weighted) vals.alloc(std::max<int64_t>(m, 1), s);
    if (comp)
      launch(k_emit_thread<true>, tb, 256, 0, s, v, T.tier.get(), map, nc, off.get(), keys.get(), vals.get());
    else
      launch(k_emit_thread<false>, tb, 256, 0, s, v, T.tier.get(), map, nc, off.get(), keys.get(), vals.get());
    if (warp_work) {
      if (comp) launch(k_emit<true>, wb, 256, 0, s, v, T.tier.get(), map, nc, off.get(), keys.get(), vals.get());
      else launch(k_emit<false>, wb, 256, 0, s, v, T.tier.get(), map, nc, off.get(), keys.get(), vals.get());
    }
    TP_LAUNCH_CHECK();
    if (T.n_huge) {
      unsigned hb = grid_for(T.n_huge_chunks * 32, 256);
      if (comp)
        launch(k_emit_chunks<true>, hb, 256, 0, s, v, T.huge.get(), T.n_huge, T.huge_chunk_start.get(),
                                               T.n_huge_chunks, map, nc, m_small, hoff.get(),
                                               keys.get(), vals.get());
      else
        launch(k_emit_chunks<false>, hb, 256, 0, s, v, T.huge.get(), T.n_huge, T.huge_chunk_start.get(),
                                                T.n_huge_chunks, map, nc, m_small, hoff.get(),
                                                keys.get(), vals.get());
      TP_LAUNCH_CHECK();
    }
    off.release();
    hoff.release();
    radix_sort_pairs(keys.get(), vals.get(), m, bits_for((uint64_t)nc * (uint64_t)nc - 1), s);
    Buf<int32_t> hf(std::max<int64_t>(m, 1), s);
    Buf<int64_t> idx(m + 1, s);
    if (m) {
      launch(k_heads, grid_for(m, 256), 256, 0, s, keys.get(), m, hf.get());
      TP_LAUNCH_CHECK();
    }
    exclusive_scan_i32_to_i64(hf.get(), idx.get(), m, s);
    int64_t m2 = read_scalar(idx.get() + m, s);
    cg->m2 = m2;
    cg->adj.alloc(m2 + kAdjPad, s);
    TP_CUDA(cudaMemsetAsync(cg->adj.get() + m2, 0, kAdjPad * sizeof(int32_t), s));
    cg->ew.alloc(m2, s);
    cg->xadj.alloc(nc + 1, s);
    if (m2) TP_CUDA(cudaMemsetAsync(cg->ew.get(), 0, m2 * sizeof(int64_t), s));
    TP_CUDA(cudaMemsetAsync(cg->xadj.get(), 0, (nc + 1) * sizeof(int64_t), s));
    if (m) {
      launch(k_reduce, grid_for(m, 256), 256, 0, s, keys.get(), weighted ? vals.get() : nullptr,
                                                  idx.get(), m, nc, cg->adj.get(), cg->ew.get(),
                                                  cg->xadj.get());
      TP_LAUNCH_CHECK();
    }
    exclusive_scan_i64(cg->xadj.get(), cg->xadj.get(), nc, s);
    cg->max_ew = max_i64(cg->ew.get(), m2, s);  // synchronises
  } catch (...) {
    delete cg;
    throw;
  }
  return cg;
}

}  // namespace tp
