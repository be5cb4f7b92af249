// Cluster contraction (Section "Contraction" of the paper): every cluster
// becomes a coarse vertex, w'(a,b) sums the weights of the fine edges between
// clusters a and b, intra-cluster edges vanish.
//
// GPU form: coarse ids are ranks of the non-empty labels (mark + exclusive
// scan, so ids are deterministic where the paper's atomic counters are not);
// every inter-cluster adjacency entry is emitted as the key a*n' + b at a
// position fixed by a scan of per-vertex (per-chunk for hubs) counts, sorted
// with the library's LSD radix sort, and duplicate keys are reduced into the
// canonical coarse CSR (neighbours ascending, int64 weights). Memory (the
// paper's third peak): a fine edge weight rides in the low bits of its key
// when both fit 64 bits, so weighted levels sort no separate values, and the
// reduction numbers the runs tile by tile (a count per 4096 entries) instead
// of through per-entry head flags and prefix sums.
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

// Sort key of an inter-cluster entry: a * n' + b, with the fine edge weight
// in the low wbits bits (wbits = 0: weights apart, in vals, or unit).
__device__ __forceinline__ uint64_t entry_key(int32_t a, int32_t b, int64_t nc, int64_t w,
                                              int wbits) {
  const uint64_t k = (uint64_t)a * (uint64_t)nc + (uint64_t)b;
  return wbits ? (k << wbits) | (uint64_t)w : k;
}

template <bool COMP>
__device__ __forceinline__ void emit(const GView &g, int64_t u, int64_t chunk, const int32_t *map,
                                     int64_t nc, int wbits, int64_t pos, uint64_t *keys,
                                     uint64_t *vals) {
  int32_t a = map[u];
  warp_neighbours<COMP>(g, u, chunk, [&](bool has, int32_t v, int64_t w, int64_t) {
    int32_t b = has ? map[v] : a;
    bool keep = has && b != a;
    unsigned m = __ballot_sync(kFull, keep);
    if (keep) {
      int64_t at = pos + __popc(m & lanemask_lt());
      keys[at] = entry_key(a, b, nc, w, wbits);
      if (vals) vals[at] = (uint64_t)w;
    }
    pos += __popc(m);
  });
}

template <bool COMP>
__global__ void k_emit_thread(GView g, const uint8_t *tier, const int32_t *map, int64_t nc,
                              int wbits, const int64_t *off, uint64_t *keys, uint64_t *vals) {
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < g.n;
       u += (int64_t)gridDim.x * blockDim.x) {
    if (!thread_tier(tier[u])) continue;
    const int32_t a = map[u];
    int64_t pos = off[u];
    thread_neighbours<COMP>(g, u, [&](int32_t v, int64_t w) {
      const int32_t b = map[v];
      if (b == a) return;
      keys[pos] = entry_key(a, b, nc, w, wbits);
      if (vals) vals[pos] = (uint64_t)w;
      ++pos;
    });
  }
}

template <bool COMP>
__global__ void k_emit(GView g, const uint8_t *tier, const int32_t *map, int64_t nc, int wbits,
                       const int64_t *off, uint64_t *keys, uint64_t *vals) {
  int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t u = warp; u < g.n; u += nw)
    if (!thread_tier(tier[u]) && tier[u] != TIER_HUGE)
      emit<COMP>(g, u, -1, map, nc, wbits, off[u], keys, vals);
}

template <bool COMP>
__global__ void k_emit_chunks(GView g, const int32_t *huge, int64_t n_huge,
                              const int64_t *chunk_start, int64_t n_items, const int32_t *map,
                              int64_t nc, int wbits, int64_t base, const int64_t *off,
                              uint64_t *keys, uint64_t *vals) {
  int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t it = warp; it < n_items; it += nw) {
    int64_t i = find_item(chunk_start, n_huge, it);
    emit<COMP>(g, huge[i], it - chunk_start[i], map, nc, wbits, base + off[it], keys, vals);
  }
}

// Run-length reduction of the sorted entries, 4096 per tile. Pass 1: runs
// starting in every tile.
constexpr int kRleThreads = 256;
constexpr int64_t kRleTile = 4096;

__device__ __forceinline__ bool run_head(const uint64_t *keys, int64_t i, int wbits) {
  return i == 0 || (keys[i] >> wbits) != (keys[i - 1] >> wbits);
}

__global__ void __launch_bounds__(kRleThreads) k_rle_count(const uint64_t *keys, int64_t m,
                                                           int wbits, int64_t ntiles,
                                                           int64_t *tcnt) {
  __shared__ int32_t red[kRleThreads / 32];
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t b = t * kRleTile, e = min(b + kRleTile, m);
    int32_t c = 0;
    for (int64_t i = b + threadIdx.x; i < e; i += kRleThreads) c += run_head(keys, i, wbits);
    c = warp_sum(c);
    if (lane_id() == 0) red[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
      int32_t tot = 0;
      for (int w = 0; w < kRleThreads / 32; ++w) tot += red[w];
      tcnt[t] = tot;
    }
    __syncthreads();
  }
}

// Pass 2: every entry adds its weight to its run's slot (the runs before it,
// from the tile's offset plus a block scan); a run's first entry also writes
// the neighbour and counts the coarse vertex's degree.
__global__ void __launch_bounds__(kRleThreads) k_rle_write(const uint64_t *keys,
                                                           const uint64_t *vals, int64_t m,
                                                           int64_t nc, int wbits, int64_t ntiles,
                                                           const int64_t *toff, int32_t *adj,
                                                           int64_t *ew, int64_t *deg) {
  __shared__ int32_t ws[kRleThreads / 32];
  const uint64_t wmask = wbits ? ((uint64_t)1 << wbits) - 1 : 0;
  const int lane = lane_id(), w = threadIdx.x >> 5;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    int64_t base = toff[t];  // runs started before this step
    const int64_t b = t * kRleTile, e = min(b + kRleTile, m);
    for (int64_t i0 = b; i0 < e; i0 += kRleThreads) {
      const int64_t i = i0 + threadIdx.x;
      const bool in = i < e;
      const int32_t h = in && run_head(keys, i, wbits);
      // block-wide inclusive scan of the head flags
      const unsigned bal = __ballot_sync(kFull, h);
      const int32_t winc = __popc(bal & (lanemask_lt() | (1u << lane)));
      if (lane == 31) ws[w] = winc;
      __syncthreads();
      int32_t before = 0, total = 0;
      for (int q = 0; q < kRleThreads / 32; ++q) {
        const int32_t c = ws[q];
        before += q < w ? c : 0;
        total += c;
      }
      if (in) {
        const int64_t slot = base + before + winc - 1;
        const uint64_t k = keys[i];
        const uint64_t key = k >> wbits;
        const uint64_t wt = wbits ? (k & wmask) : (vals ? vals[i] : 1ull);
        if (h) {
          adj[slot] = (int32_t)(key % (uint64_t)nc);
          atomicAdd((unsigned long long *)&deg[key / (uint64_t)nc], 1ull);
        }
        atomicAdd((unsigned long long *)&ew[slot], (unsigned long long)wt);
      }
      base += total;
      __syncthreads();  // ws is rewritten by the next step
    }
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
    const bool warp_work = T.n_mid + T.n_mid2 + T.n_big0 + T.n_big1 + T.n_big + T.n_big2 > 0;
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
    // weights ride in the keys' low bits when the pair fits 64 bits
    const int kbits = bits_for((uint64_t)nc * (uint64_t)nc - 1);
    const int wbits = weighted && kbits + bits_for((uint64_t)g->max_ew) <= 64
                          ? bits_for((uint64_t)g->max_ew)
                          : 0;
    Buf<uint64_t> keys(std::max<int64_t>(m, 1), s), vals;
    if (weighted && !wbits) vals.alloc(std::max<int64_t>(m, 1), s);
    if (comp)
      launch(k_emit_thread<true>, tb, 256, 0, s, v, T.tier.get(), map, nc, wbits, off.get(), keys.get(), vals.get());
    else
      launch(k_emit_thread<false>, tb, 256, 0, s, v, T.tier.get(), map, nc, wbits, off.get(), keys.get(), vals.get());
    if (warp_work) {
      if (comp) launch(k_emit<true>, wb, 256, 0, s, v, T.tier.get(), map, nc, wbits, off.get(), keys.get(), vals.get());
      else launch(k_emit<false>, wb, 256, 0, s, v, T.tier.get(), map, nc, wbits, off.get(), keys.get(), vals.get());
    }
    TP_LAUNCH_CHECK();
    if (T.n_huge) {
      unsigned hb = grid_for(T.n_huge_chunks * 32, 256);
      if (comp)
        launch(k_emit_chunks<true>, hb, 256, 0, s, v, T.huge.get(), T.n_huge, T.huge_chunk_start.get(),
                                               T.n_huge_chunks, map, nc, wbits, m_small, hoff.get(),
                                               keys.get(), vals.get());
      else
        launch(k_emit_chunks<false>, hb, 256, 0, s, v, T.huge.get(), T.n_huge, T.huge_chunk_start.get(),
                                                T.n_huge_chunks, map, nc, wbits, m_small, hoff.get(),
                                                keys.get(), vals.get());
      TP_LAUNCH_CHECK();
    }
    off.release();
    hoff.release();
    radix_sort_pairs(keys.get(), vals.get(), m, kbits, s, wbits);
    // runs per tile, their offsets, then the coarse CSR
    const int64_t ntiles = (m + kRleTile - 1) / kRleTile;
    Buf<int64_t> toff(ntiles + 1, s);
    const unsigned rb = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ntiles, (int64_t)num_sms() * 16));
    if (ntiles) {
      launch(k_rle_count, rb, kRleThreads, 0, s, keys.get(), m, wbits, ntiles, toff.get());
      TP_LAUNCH_CHECK();
    }
    exclusive_scan_i64(toff.get(), toff.get(), ntiles, s);
    int64_t m2 = read_scalar(toff.get() + ntiles, s);
    cg->m2 = m2;
    cg->adj.alloc(m2 + kAdjPad, s);
    TP_CUDA(cudaMemsetAsync(cg->adj.get() + m2, 0, kAdjPad * sizeof(int32_t), s));
    cg->ew.alloc(m2, s);
    cg->xadj.alloc(nc + 1, s);
    if (m2) TP_CUDA(cudaMemsetAsync(cg->ew.get(), 0, m2 * sizeof(int64_t), s));
    TP_CUDA(cudaMemsetAsync(cg->xadj.get(), 0, (nc + 1) * sizeof(int64_t), s));
    if (ntiles) {
      launch(k_rle_write, rb, kRleThreads, 0, s, keys.get(), vals.get(), m, nc, wbits, ntiles,
             toff.get(), cg->adj.get(), cg->ew.get(), cg->xadj.get());
      TP_LAUNCH_CHECK();
    }
    keys.release();
    vals.release();
    exclusive_scan_i64(cg->xadj.get(), cg->xadj.get(), nc, s);
    cg->max_ew = max_i64(cg->ew.get(), m2, s);  // synchronises
  } catch (...) {
    delete cg;
    throw;
  }
  return cg;
}

}  // namespace tp
