// Size-constrained label propagation on the GPU (Algorithm 1 of the paper,
// made synchronous and deterministic), its two-hop packing and rebalancing.
//
// Rating (Section "Rating Maps", Algorithm 2): a vertex's ratings R[C[v]] +=
// w(u,v) accumulate in a hash table. The paper's split into a first phase
// with small per-thread tables and a second phase for "bumped" high-degree
// vertices becomes five degree tiers, each a different kernel:
//   lane  (deg <= tier_lane):  one lane per vertex, labels sorted in
//          registers (no table at all);
//   small (deg <= tier_small): one warp per vertex, shared table of up to
//          128 slots;
//   mid   (deg <= tier_mid):   one warp per vertex, shared table of up to
//          1024 slots (both warp tiers fill and scan only the least power of
//          two >= table_slack * degree slots, at least 32);
//   big   (deg <= 10000):      one block per vertex, shared table of 8192 or
//          16384 slots;
//   huge  (deg > 10000):       one block per chunk of 1000 neighbours (the
//          compressed format's independently decodable chunks) aggregates in
//          a shared table and flushes into the vertex's global table with
//          atomics (the paper's "hash tables as flush buffers" against
//          contention); blocks then scan that table in segments and one
//          block per vertex combines the segments' results.
// The tier only decides where the sums are formed; integer sums commute and
// the argmax uses a total order, so the result is tier-independent.
//
// Approval: movers add their weight to in_w[target] with atomics. Targets
// whose weight plus in_w fits approve every mover; for the others one block
// per target runs a weighted radix select over the key (gain desc, vertex
// asc) and approves exactly the longest fitting prefix.
#include <algorithm>
#include <type_traits>
#include <mutex>

#include "decode.cuh"

namespace tp {

namespace {

enum Mode { M_LP = 0, M_FAV = 1, M_REBAL = 2 };

constexpr int kSmallLog = 7;   // 128 slots
constexpr int kMidSmallLog = 9;  // 512 slots: mid tier, degree <= kMidSplit = 256
constexpr int kMidLog = 10;    // 1024 slots: mid tier, degree <= 512
constexpr int kHugeLog = 11;   // 2048 slots: one 1000-neighbour chunk of a hub
constexpr int kMidWarps = 4;

struct RateCtx {
  GView g;
  const uint8_t *tier;
  const int32_t *label;
  const int64_t *lw;
  int64_t cap;
  uint64_t rk;
  const uint64_t *rk_dev;  // if set, the round key is read here (replayed round graphs)
  int32_t S, s;
  int32_t slack;  // warp tiers: table slots per neighbour (power of two)
  // M_LP outputs
  int32_t *mv_u, *mv_t, *mv_o;
  int64_t *mv_g;
  int64_t *in_w;
  unsigned long long *counters;
  // M_FAV output
  int32_t *fav;
  // M_REBAL (batched graphs: rb_best and blk_of hold one entry per graph)
  int32_t blk, k;
  int64_t *rb_loss;
  int32_t *rb_t;
  long long *rb_best;
  const int32_t *blk_of;
  // batched graphs (seg.gid == null: one graph)
  SegLp seg;
  // lists and global tables
  const int32_t *list;
  int64_t list_n;
  int32_t *tkeys;
  int64_t *tvals;
  int32_t *tlist, *tcount;  // filled slots per huge table
  const int64_t *toff;
  const int32_t *tcap;
  int64_t tbase;  // slot offset of this tier's tables inside tkeys/tvals
  const int64_t *chunk_start;
  int64_t n_chunks;
  const int64_t *seg_start;  // huge tables: prefix of segment counts
  int64_t n_segs;
  // lane tier in LP mode: this round's buckets (null: hash every vertex);
  // sub-round s holds bucket[bucket_off[s * nb] .. bucket_off[(s + 1) * nb])
  const int32_t *bucket;
  const int64_t *bucket_off;
  int64_t bucket_nb;
  // per listed vertex: record start << 8 | record length (compressed graphs)
  const uint64_t *bucket_rec;
  // this round's sub-round + 1 of every vertex (null: hash on the fly)
  const uint8_t *sub_byte;
  // bucket mode of the warp/block tiers: this tier's list positions grouped
  // by sub-round (null: scan the whole list and test each vertex)
  const int32_t *bpos;
  const int64_t *boff;  // this tier's S + 1 offsets into bpos
  // huge tier in bucket mode: prefix of chunk / segment counts over bpos and
  // the items (hub position << 32 | chunk or segment index)
  const int64_t *hc_pre, *hs_pre, *hc_item, *hs_item;
  // all tiers' buckets (rate_tiers slices them per tier)
  const int32_t *tb_pos;
  const int64_t *tb_off;
  int64_t tb_base[LpWork::kTiers];
};

// Range of list entries (bucket mode: of bpos) a tier kernel walks.
__device__ __forceinline__ void tier_range(const RateCtx &c, int64_t &b, int64_t &e) {
  if (c.bpos) b = c.boff[c.s], e = c.boff[c.s + 1];
  else b = 0, e = c.list_n;
}
// List position of entry k and whether its vertex is active this sub-round.
template <int MODE>
__device__ __forceinline__ bool tier_entry(const RateCtx &c, int64_t k, int64_t &pos, int64_t &u);

__device__ __forceinline__ int64_t node_w(const GView &g, int64_t u) { return g.vw ? g.vw[u] : 1; }

__device__ __forceinline__ uint64_t rk_of(const RateCtx &c) { return c.rk_dev ? *c.rk_dev : c.rk; }

// Batched graphs: u's number inside its own graph, its cap, and the
// favourite key of a vertex without favourite (one per graph).
__device__ __forceinline__ int64_t local_id(const RateCtx &c, int64_t u) {
  return c.seg.gid ? u - c.seg.vb[c.seg.gid[u]] : u;
}
__device__ __forceinline__ int64_t cap_of(const RateCtx &c, int64_t u) {
  return c.seg.gid ? c.seg.cap[c.seg.gid[u]] : c.cap;
}
__device__ __forceinline__ int32_t no_fav(const RateCtx &c, int64_t u) {
  return (int32_t)(c.g.n + (c.seg.gid ? c.seg.gid[u] : 0));
}

template <int MODE>
__device__ __forceinline__ bool active(const RateCtx &c, int64_t u) {
  if (MODE == M_LP)
    return c.sub_byte ? c.sub_byte[u] == c.s + 1
                      : sub_round_of(hstep(rk_of(c), (uint64_t)local_id(c, u)), c.S) == c.s;
  if (MODE == M_FAV) return c.label[u] == u && c.lw[u] == node_w(c.g, u);
  return c.label[u] == (c.blk_of ? c.blk_of[c.seg.gid[u]] : c.blk);
}

template <int MODE>
__device__ __forceinline__ bool tier_entry(const RateCtx &c, int64_t k, int64_t &pos, int64_t &u) {
  pos = c.bpos ? c.bpos[k] : k;
  u = c.list[pos];
  return c.bpos ? true : active<MODE>(c, u);
}

// The tie order of vertex u: tie_of(k, x) is the tie hash of label x as u's
// graph numbers it (its label base folded into the additive constant, so
// (x - base) + gamma costs one add, as x + gamma does for one graph).
struct TieKey {
  uint64_t hv, add;
};
__device__ __forceinline__ uint32_t tie_of(const TieKey &k, int32_t x) {
  return (uint32_t)(mix64(k.hv ^ ((uint64_t)(int64_t)x + k.add)) >> 32);
}
template <int MODE>
__device__ __forceinline__ TieKey tie_key(const RateCtx &c, int64_t u) {
  if (MODE == M_REBAL) return TieKey{0, 0};
  int64_t vb = 0, lb = 0;
  if (c.seg.gid) {
    const int32_t g = c.seg.gid[u];
    vb = c.seg.vb[g];
    lb = c.seg.lb[g];
  }
  return TieKey{hstep(hstep(rk_of(c), (uint64_t)(u - vb)), kTagTie), kGamma - (uint64_t)lb};
}
// The lane tier decides batched graphs at compile time (SEG), so the one-graph
// kernels carry no per-graph lookups in their tight register budget.
template <bool SEG>
__device__ __forceinline__ int64_t lane_cap(const RateCtx &c, int64_t u) {
  return SEG ? c.seg.cap[c.seg.gid[u]] : c.cap;
}
template <int MODE, bool SEG>
__device__ __forceinline__ TieKey lane_tie_key(const RateCtx &c, int64_t u) {
  if (SEG) return tie_key<MODE>(c, u);
  return TieKey{hstep(hstep(rk_of(c), (uint64_t)u), kTagTie), kGamma};
}

__device__ __forceinline__ uint32_t slot_of(int32_t x, int logcap) {
  return ((uint32_t)x * 0x9E3779B1u) >> (32 - logcap);
}

// Adds w to the rating of label x (open addressing, linear probing); V is
// int64_t, or uint32_t where ratings are counts (unit weights).
template <class V>
__device__ __forceinline__ void tbl_add(int32_t *keys, V *vals, int logcap, int32_t x, int64_t w,
                                        int32_t *err) {
  uint32_t mask = (1u << logcap) - 1u, h = slot_of(x, logcap);
  for (uint32_t probe = 0; probe <= mask; ++probe, h = (h + 1) & mask) {
    int32_t k = *(volatile int32_t *)&keys[h];
    if (k == -1) {
      int32_t prev = atomicCAS(&keys[h], -1, x);
      k = prev == -1 ? x : prev;
    }
    if (k == x) {
      if constexpr (sizeof(V) == 8) atomicAdd((unsigned long long *)&vals[h], (unsigned long long)w);
      else atomicAdd((unsigned int *)&vals[h], (unsigned int)w);
      return;
    }
  }
  latch_error(err, TP_ERR_CORRUPT);  // more distinct labels than the degree allows
}

struct Best {
  int64_t r;
  uint32_t t;
  int32_t x;
  int64_t rown;
  __device__ __forceinline__ void init() { r = -1, t = 0xffffffffu, x = INT32_MAX, rown = 0; }
};

__device__ __forceinline__ void warp_reduce_best(Best &b) {
  warp_best(b.r, b.t, b.x);
  b.rown = warp_max(b.rown);
}

// Per-warp buffer of mover records, flushed with one atomic per 32 movers.
struct MoverBuf {
  int32_t *u, *t, *o;
  int64_t *gain;
  int cnt;
};

__device__ __forceinline__ void flush_movers(const RateCtx &c, MoverBuf &mb) {
  __syncwarp();
  if (mb.cnt == 0) return;
  unsigned long long base = 0;
  if (lane_id() == 0) base = atomicAdd(c.counters, (unsigned long long)mb.cnt);
  base = __shfl_sync(kFull, base, 0);
  int l = lane_id();
  if (l < mb.cnt) {
    c.mv_u[base + l] = mb.u[l];
    c.mv_t[base + l] = mb.t[l];
    c.mv_o[base + l] = mb.o[l];
    c.mv_g[base + l] = mb.gain[l];
  }
  mb.cnt = 0;
  __syncwarp();
}

// Acts on the (warp-uniform) decision for vertex u.
template <int MODE>
__device__ __forceinline__ void finalize_warp(const RateCtx &c, const Best &b, int64_t u, int64_t cu,
                                              MoverBuf *mb) {
  int lane = lane_id();
  if (MODE == M_LP) {
    if (b.r > b.rown) {
      if (lane == 0) {
        mb->u[mb->cnt] = (int32_t)u;
        mb->t[mb->cnt] = b.x;
        mb->o[mb->cnt] = c.label[u];
        mb->gain[mb->cnt] = b.r - b.rown;
        atomicAdd((unsigned long long *)&c.in_w[b.x], (unsigned long long)cu);
      }
      if (++mb->cnt == 32) flush_movers(c, *mb);
    }
  } else if (MODE == M_FAV) {
    if (lane == 0) c.fav[u] = b.r > 0 ? b.x : no_fav(c, u);
  } else {
    // the graph's blocks are lb .. lb + k - 1 (one graph: 0 .. k - 1)
    int32_t blk = c.blk, k = c.k, lb = 0;
    long long *best = c.rb_best;
    if (c.seg.gid) {
      const int32_t g = c.seg.gid[u];
      blk = c.blk_of[g], k = c.seg.k[g], lb = (int32_t)c.seg.lb[g];
      best += g;
    }
    const int64_t cap = cap_of(c, u);
    int32_t tz = -1;
    if (b.r <= 0) {  // no admissible neighbouring block: smallest admissible block
      for (int32_t base = 0; base < k && tz < 0; base += 32) {
        int32_t t = lb + base + lane;
        bool ok = base + lane < k && t != blk && c.lw[t] + cu <= cap;
        unsigned m = __ballot_sync(kFull, ok);
        if (m) tz = lb + base + __ffs(m) - 1;
      }
    }
    if (lane == 0) {
      int32_t tt = b.r > 0 ? b.x : tz;
      c.rb_t[u] = tt;
      if (tt >= 0) {
        int64_t loss = b.rown - (b.r > 0 ? b.r : 0);
        c.rb_loss[u] = loss;
        atomicMin(best, (long long)loss);
      }
    }
  }
}

// Rates vertex u with one warp; the table must be empty on entry and is
// empty again on exit. The scan takes two passes: the top rating among the
// other labels (and the own rating), then the tie order among the labels at
// that rating only, so tie hashes are formed for tied candidates alone; in
// LP mode a vertex whose top rating does not beat its own cannot move and
// skips the second pass.
template <bool COMP, int MODE, class V>
__device__ void rate_vertex_warp(const RateCtx &c, int64_t u, int32_t *keys, V *vals, int logcap,
                                 MoverBuf *mb) {
  const int lane = lane_id();
  const int32_t own = c.label[u];
  const int64_t cu = node_w(c.g, u), capu = cap_of(c, u);
  // every lane adds its neighbour's label to the table (shared-memory
  // atomics are far cheaper than grouping equal labels across lanes first)
  warp_neighbours<COMP>(c.g, u, -1, [&](bool has, int32_t v, int64_t w, int64_t) {
    if (has) tbl_add<V>(keys, vals, logcap, c.label[v], w, c.g.err);
  });
  __syncwarp();
  __threadfence_block();
  const int cap = 1 << logcap;
  int64_t rmax = -1, rown = 0;
  for (int i = lane; i < cap; i += 32) {
    const int32_t x = keys[i];
    if (x < 0) continue;
    const int64_t R = (int64_t)vals[i];
    if (x == own) rown = R;
    else rmax = R > rmax ? R : rmax;
  }
  rmax = warp_max(rmax);
  rown = warp_max(rown);
  Best b;
  b.init();
  b.rown = rown;
  if (rmax >= 0 && (MODE != M_LP || rmax > rown)) {
    const TieKey hv = tie_key<MODE>(c, u);
    // the best label ignoring the cap: the top-rated one first in tie order
    for (int i = lane; i < cap; i += 32) {
      const int32_t x = keys[i];
      if (x < 0 || x == own || (int64_t)vals[i] != rmax) continue;
      const uint32_t t = MODE == M_REBAL ? 0u : tie_of(hv, x);
      if (better(rmax, t, x, b.r, b.t, b.x)) b.r = rmax, b.t = t, b.x = x;
    }
    warp_best(b.r, b.t, b.x);
    // the winner is full: the best admissible label instead (for a move it
    // must also improve on the own rating)
    if (MODE != M_FAV && b.x != INT32_MAX && c.lw[b.x] + cu > capu) {
      b.init();
      for (int i = lane; i < cap; i += 32) {
        const int32_t x = keys[i];
        if (x < 0 || x == own) continue;
        const int64_t R = (int64_t)vals[i];
        if (MODE == M_LP && R <= rown) continue;
        const uint32_t t = MODE == M_REBAL ? 0u : tie_of(hv, x);
        if (better(R, t, x, b.r, b.t, b.x) && c.lw[x] + cu <= capu) b.r = R, b.t = t, b.x = x;
      }
      warp_best(b.r, b.t, b.x);
      b.rown = rown;
    }
  }
  for (int i = lane; i < cap; i += 32) keys[i] = -1, vals[i] = 0;
  __syncwarp();
  finalize_warp<MODE>(c, b, u, cu, mb);
}

// Warp tiers: the table of a degree-d vertex uses the first 2^lc slots,
// the least power of two >= slack * d (at least 32, at most 2^maxlog); only
// those are scanned and cleared.
__device__ __forceinline__ int table_log(const RateCtx &c, int64_t d, int maxlog) {
  int lc = 5;
  while (lc < maxlog && ((int64_t)1 << lc) < c.slack * d) ++lc;
  return lc;
}

// Shared memory per warp: table keys + values, then the mover buffer.
template <int LOG, class V = int64_t>
struct WarpSmem {
  int32_t keys[1 << LOG];
  V vals[1 << LOG];
  int32_t mu[32], mt[32], mo[32];
  int64_t mg[32];
};

template <int LOG, class V>
__device__ __forceinline__ void init_table(WarpSmem<LOG, V> &w) {
  for (int i = lane_id(); i < (1 << LOG); i += 32) w.keys[i] = -1, w.vals[i] = 0;
  __syncwarp();
}

// Small tier: one warp per listed vertex (c.list), or, in rebalancing mode
// (c.list == nullptr), every vertex of the small and lane tiers, filtered in
// 32-vertex slabs.
template <bool COMP, int MODE>
__global__ void k_rate_small(RateCtx c) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  WarpSmem<kSmallLog> &ws = reinterpret_cast<WarpSmem<kSmallLog> *>(smem_raw)[threadIdx.x >> 5];
  init_table(ws);
  MoverBuf mb{ws.mu, ws.mt, ws.mo, ws.mg, 0};
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  if (c.list) {
    int64_t kb, ke;
    tier_range(c, kb, ke);
    for (int64_t k = kb + gw; k < ke; k += nw) {
      int64_t i, u;
      if (tier_entry<MODE>(c, k, i, u)) {
        const int64_t d = COMP ? zip_nbr(c.g, u).deg : c.g.xadj[u + 1] - c.g.xadj[u];
        rate_vertex_warp<COMP, MODE>(c, u, ws.keys, ws.vals, table_log(c, d, kSmallLog), &mb);
      }
    }
  } else {
    for (int64_t base = gw * 32; base < c.g.n; base += nw * 32) {
      int64_t u = base + lane_id();
      bool act = u < c.g.n && (c.tier[u] == TIER_SMALL || c.tier[u] == TIER_LANE) &&
                 active<MODE>(c, u);
      unsigned am = __ballot_sync(kFull, act);
      while (am) {
        int j = __ffs(am) - 1;
        am &= am - 1;
        const int64_t v = base + j;
        const int64_t d = COMP ? zip_nbr(c.g, v).deg : c.g.xadj[v + 1] - c.g.xadj[v];
        rate_vertex_warp<COMP, MODE>(c, v, ws.keys, ws.vals, table_log(c, d, kSmallLog), &mb);
      }
    }
  }
  if (MODE == M_LP) flush_movers(c, mb);
}

// ---------------------------------------------------------------- lane tier
// Low-degree vertices, one lane per vertex, so a warp keeps 32
// neighbourhoods in flight. Each warp step:
//   1. takes a window of up to 128 active vertices (this sub-round's bucket
//      list, or a scan of 256-vertex slabs) and rates it as four batches of
//      32 in list order;
//   2. per batch, every lane loads its compressed record at once (five
//      16-byte groups; the next batch's records are prefetched to L2
//      meanwhile) and decodes it a 32-bit word at a time into its column of
//      shared memory; the gaps are then summed into neighbour ids while the
//      label gathers are issued, all of them before the first is used (CSR:
//      the adjacency entries directly);
//   3. the labels are sorted with Batcher's odd-even merge network of 16 or
//      32 elements (picked per batch), so equal labels form runs whose
//      lengths (summed weights) are the ratings;
//   4. only the candidates tied at the top rating are hashed for the tie
//      order; the cap is checked for the winner only, with a scan over all
//      admissible candidates when the winner is full;
//   5. the window's movers are collected in shared memory and written out
//      with one atomic per window.
constexpr int kLaneWarps = 8;
constexpr int kLaneBlocksPerSM = 3;
constexpr int kLaneWin = 128;             // vertices per warp step
constexpr int kLaneQueue = kLaneWin + 32;  // slab scans append 32 at a time

struct LaneCand {
  int32_t r;
  uint32_t t;
  int32_t x;
};

__device__ __forceinline__ bool lane_better(const LaneCand &a, const LaneCand &b) {
  return better(a.r, a.t, a.x, b.r, b.t, b.x);
}

__device__ __forceinline__ void prefetch_l2(const void *p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// Decodes u's compressed record into its shared-memory column: the raw
// values (first the signed first neighbour, then the gaps) go to
// col[i * 32]; returns the degree. The record's first 80 bytes are
// loaded at once as five 16-byte groups from its 16-byte aligned start, so
// no load waits on another (a longer record, up to 165 bytes at degree 32
// with five-byte gaps, loads its further groups as the decoder reaches
// them), and consumed a 32-bit word at a time. Bytes
// before the record are turned into value ends and, like the header, are
// written to slot 0, which the first neighbour then overwrites; bytes after
// it are turned into continuation bytes, so they end no value.
template <bool LONG>
__device__ __forceinline__ int lane_decode(const GView &g, uint64_t b, uint64_t e, uint32_t *col) {
  constexpr int G = 5;  // 80-byte window
  const uint64_t ws = b & ~(uint64_t)15;
  const int p0 = (int)(b - ws), endp = (int)(e - ws);
  const uint4 *src = reinterpret_cast<const uint4 *>(g.bytes + ws);
  uint4 q[G];
#pragma unroll
  for (int j = 0; j < G; ++j) q[j] = 16 * j < endp ? __ldcs(src + j) : make_uint4(0, 0, 0, 0);
  int fi = 0;         // words of q[0] already taken
  int nextg = G;      // next 16-byte group to load (records longer than the window)
  auto pop = [&]() -> uint32_t {
    const uint32_t w = fi == 0 ? q[0].x : fi == 1 ? q[0].y : fi == 2 ? q[0].z : q[0].w;
    if (++fi == 4) {
#pragma unroll
      for (int j = 0; j + 1 < G; ++j) q[j] = q[j + 1];
      if (LONG) {
        q[G - 1] = 16 * nextg < endp ? __ldcs(src + nextg) : make_uint4(0, 0, 0, 0);
        ++nextg;
      }
      fi = 0;
    }
    return w;
  };
  int wi = p0 >> 2;
  for (int j = 0; j < wi; ++j) pop();
  // leading bytes of the first word: forced value ends
  uint32_t lead = 0x80808080u & ((1u << (8 * (p0 & 3))) - 1u);
  int idx = -1 - (p0 & 3);  // value index; < 0 for the leading bytes and the header
  uint32_t acc = 0;
  int accb = 0;
  for (; 4 * wi < endp; ++wi) {
    uint32_t w = pop() & ~lead;
    lead = 0;
    const int vhi = endp - 4 * wi;  // bytes of this word inside the record
    if (vhi < 4) w |= 0x80808080u & ~((1u << (8 * vhi)) - 1u);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const uint32_t by = (w >> (8 * j)) & 0xffu;
      acc |= (by & 0x7fu) << accb;
      accb += 7;
      if (!(by & 0x80u)) {
        col[max(idx, 0) * 32] = acc;
        ++idx;
        acc = 0;
        accb = 0;
      }
    }
  }
  return min(max(idx, 0), kLaneMaxDeg);
}

// Record range of a compressed lane-tier vertex: from the bucket list when
// it carries the ranges (coalesced with the vertex ids), else the offsets.
__device__ __forceinline__ void lane_record(const GView &g, const uint64_t *rec, int64_t pos,
                                            int32_t u, uint64_t &b, uint64_t &e) {
  if (rec) {
    const uint64_t r = rec[pos];
    b = r >> 8;
    e = b + (r & 255u);
  } else {
    b = off_at(g, u);
    e = off_at(g, u + 1);
  }
}

template <bool COMP>
__device__ __forceinline__ void lane_prefetch(const GView &g, const uint64_t *rec, int64_t pos,
                                              int64_t u) {
  if (COMP) {
    uint64_t b, e;
    lane_record(g, rec, pos, (int32_t)u, b, e);
    prefetch_l2(g.bytes + b);
    prefetch_l2(g.bytes + e);
  } else {
    const int64_t b = g.xadj[u], e = g.xadj[u + 1];
    if (e > b) {
      prefetch_l2(g.adj + b);
      prefetch_l2(g.adj + e - 1);
    }
  }
}

// Batcher's odd-even merge sort of a[0..N), ascending (N a power of two;
// 63 comparators for 16 elements, 191 for 32), registers only. The network
// is generated by template recursion so every index is a constant.
template <class T>
__device__ __forceinline__ void cmp_swap(T &x, T &y) {
  const T lo = min(x, y), hi = max(x, y);
  x = lo;
  y = hi;
}

// Merges the two sorted halves of the subsequence a[LO], a[LO + R], ...
template <int LO, int N, int R, class T>
__device__ __forceinline__ void oem_merge(T (&a)[kLaneMaxDeg]) {
  constexpr int M = 2 * R;
  if constexpr (M < N) {
    oem_merge<LO, N, M>(a);
    oem_merge<LO + R, N, M>(a);
#pragma unroll
    for (int i = LO + R; i + R < LO + N; i += M) cmp_swap(a[i], a[i + R]);
  } else {
    cmp_swap(a[LO], a[LO + R]);
  }
}

template <int LO, int N, class T>
__device__ __forceinline__ void oem_sort_range(T (&a)[kLaneMaxDeg]) {
  if constexpr (N > 1) {
    oem_sort_range<LO, N / 2>(a);
    oem_sort_range<LO + N / 2, N / 2>(a);
    oem_merge<LO, N, 1>(a);
  }
}

template <int N, class T>
__device__ __forceinline__ void oem_sort(T (&a)[kLaneMaxDeg]) {
  oem_sort_range<0, N>(a);
}

// Mover records of one warp's window, written out with one atomic per window.
struct LaneMovers {
  int32_t u[kLaneWin], t[kLaneWin], o[kLaneWin], g[kLaneWin];
};

// Emits the favourite (two-hop mode) or queues the move of this lane's
// vertex in the warp's buffer (nmv records so far, warp-uniform).
template <int MODE, class Movers>
__device__ __forceinline__ void emit_lane(const RateCtx &c, bool has, int32_t u, int32_t own,
                                          int32_t rown, int64_t cu, const LaneCand &best,
                                          Movers &mb, int &nmv) {
  if (MODE == M_FAV) {
    if (has) c.fav[u] = best.r > 0 ? best.x : no_fav(c, u);
  } else {
    const bool mv = has && best.r > rown;
    const unsigned mm = __ballot_sync(kFull, mv);
    if (mv) {
      const int at = nmv + __popc(mm & lanemask_lt());
      mb.u[at] = u;
      mb.t[at] = best.x;
      mb.o[at] = own;
      mb.g[at] = best.r - rown;
      atomicAdd((unsigned long long *)&c.in_w[best.x], (unsigned long long)cu);
    }
    nmv += __popc(mm);
  }
}

// Rates one batch: this lane's vertex u with deg neighbours (compressed:
// already decoded into the column; CSR: adjacency from xadj[u]) and emits
// the favourite, or queues the move in the warp's window buffer (nmv
// records so far, warp-uniform). N >= the largest degree of the batch.
template <bool COMP, int MODE, bool W, int N, bool SEG>
__device__ __forceinline__ void lane_batch(const RateCtx &c, bool has, int32_t u, int deg,
                                           uint32_t *col, uint32_t *wcol, uint8_t *cnt,
                                           LaneMovers &mb, int &nmv) {
  const int32_t own = has ? c.label[u] : -1;
  int32_t rown = 0, rmax = 0;
  int32_t *ccol = reinterpret_cast<int32_t *>(col);
  if constexpr (W) {  // weighted levels are CSR; candidates listed in the column
    // label << 32 | weight; padding: label INT32_MAX, weight 0
    constexpr uint64_t kPad = (uint64_t)INT32_MAX << 32;
    const int64_t b = has ? c.g.xadj[u] : 0;
    uint64_t a[kLaneMaxDeg];
#pragma unroll
    for (int i = 0; i < N; ++i)
      a[i] = i < deg ? ((uint64_t)(uint32_t)__ldg(c.label + __ldcs(c.g.adj + b + i)) << 32) |
                           (uint32_t)__ldcs(c.g.ew + b + i)
                     : kPad;
    oem_sort<N>(a);
    int ncand = 0;
    uint32_t run = 0;
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const int32_t x = (int32_t)(a[i] >> 32);
      run += (uint32_t)a[i];
      const bool end = i + 1 == N || (int32_t)(a[i + 1] >> 32) != x;
      const bool real = end && x != INT32_MAX;
      const bool cand = real && x != own;
      ccol[ncand * 32] = x;
      wcol[ncand * 32] = run;
      rown = real && !cand ? (int32_t)run : rown;
      rmax = cand ? max(rmax, (int32_t)run) : rmax;
      ncand += cand;
      run = end ? 0u : run;
    }
    const int64_t cu = has ? node_w(c.g, u) : 1;
    LaneCand best{-1, 0xffffffffu, INT32_MAX};
    if (MODE == M_FAV ? rmax > 0 : rmax > rown) {
      const TieKey hv = lane_tie_key<MODE, SEG>(c, u);
      const int64_t capu = lane_cap<SEG>(c, u);
      // the best candidate overall is tied at the top rating
      LaneCand b1{-1, 0xffffffffu, INT32_MAX};
      for (int k = 0; k < ncand; ++k) {
        if ((int32_t)wcol[k * 32] != rmax) continue;
        const int32_t x = ccol[k * 32];
        const LaneCand cand{rmax, tie_of(hv, x), x};
        if (lane_better(cand, b1)) b1 = cand;
      }
      if (MODE == M_FAV || c.lw[b1.x] + cu <= capu) {
        best = b1;
      } else {
        // the winner is full: the best admissible candidate that improves
        for (int k = 0; k < ncand; ++k) {
          const int32_t r = (int32_t)wcol[k * 32];
          const int32_t x = ccol[k * 32];
          if (r <= rown || x == b1.x) continue;
          const LaneCand cand{r, tie_of(hv, x), x};
          if (lane_better(cand, best) && c.lw[x] + cu <= capu) best = cand;
        }
      }
    }
    emit_lane<MODE>(c, has, u, own, rown, cu, best, mb, nmv);
  } else if constexpr (COMP) {
    // compressed, unit weights: the sorted runs become a list of (label,
    // rating) candidates in the lane's column; the decoder already keeps the
    // ALU pipe busy, and listing takes fewer instructions than walking the
    // runs when many labels tie (the first rounds)
    int32_t a[kLaneMaxDeg];
    {
      // raw values -> neighbour ids (first: signed offset from u, then gaps)
      const uint32_t nmax = (uint32_t)(c.g.n - 1);
      int32_t prev = u;
#pragma unroll
      for (int i = 0; i < N; ++i) {
        const uint32_t v = col[i * 32];
        int32_t x = i == 0 ? ((v & 1u) ? u - (int32_t)(v >> 1) : u + (int32_t)(v >> 1))
                           : prev + (int32_t)v;
        // streams are validated on creation; the clamp only keeps a
        // corrupted one from reading out of bounds
        x = (int32_t)min((uint32_t)x, nmax);
        prev = x;
        a[i] = i < deg ? __ldg(c.label + x) : INT32_MAX;
      }
    }
    oem_sort<N>(a);
    // branch-free run scan: every position writes slot ncand, which only
    // advances past a candidate (later writes overwrite the others)
    int ncand = 0, start = 0;
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const bool end = i + 1 == N || a[i + 1] != a[i];
      const int32_t run = i + 1 - start;
      const bool real = end && a[i] != INT32_MAX;
      const bool cand = real && a[i] != own;
      ccol[ncand * 32] = a[i];
      cnt[ncand * 32] = (uint8_t)run;
      rown = real && !cand ? run : rown;
      rmax = cand ? max(rmax, run) : rmax;
      ncand += cand;
      start = end ? i + 1 : start;
    }
    const int64_t cu = has ? node_w(c.g, u) : 1;
    LaneCand best{-1, 0xffffffffu, INT32_MAX};
    if (MODE == M_FAV ? rmax > 0 : rmax > rown) {
      const TieKey hv = lane_tie_key<MODE, SEG>(c, u);
      const int64_t capu = lane_cap<SEG>(c, u);
      // the best candidate overall is tied at the top rating
      LaneCand b1{-1, 0xffffffffu, INT32_MAX};
      for (int k = 0; k < ncand; ++k) {
        if ((int32_t)cnt[k * 32] != rmax) continue;
        const int32_t x = ccol[k * 32];
        const LaneCand cand{rmax, tie_of(hv, x), x};
        if (lane_better(cand, b1)) b1 = cand;
      }
      if (MODE == M_FAV || c.lw[b1.x] + cu <= capu) {
        best = b1;
      } else {
        // the winner is full: the best admissible candidate that improves
        for (int k = 0; k < ncand; ++k) {
          const int32_t r = (int32_t)cnt[k * 32];
          const int32_t x = ccol[k * 32];
          if (r <= rown || x == b1.x) continue;
          const LaneCand cand{r, tie_of(hv, x), x};
          if (lane_better(cand, best) && c.lw[x] + cu <= capu) best = cand;
        }
      }
    }
    emit_lane<MODE>(c, has, u, own, rown, cu, best, mb, nmv);
  } else {
    // CSR, unit weights: the labels are sorted with the own label as padding (its
    // count is corrected below), then one register pass finds the own
    // rating, the top rating among other labels, how many labels share it
    // and the first two of them
    int32_t a[kLaneMaxDeg];
    {
      const int64_t b = has ? c.g.xadj[u] : 0;
#pragma unroll
      for (int i = 0; i < N; ++i) a[i] = i < deg ? __ldg(c.label + __ldcs(c.g.adj + b + i)) : own;
    }
    oem_sort<N>(a);
    int start = 0, ntop = 0;
    int32_t x1 = 0, x2 = 0;
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const bool end = i + 1 == N || a[i + 1] != a[i];
      const int32_t run = i + 1 - start;
      const bool isown = a[i] == own;
      rown = end && isown ? run : rown;
      const bool cand = end && !isown;
      const bool gt = cand && run > rmax, eq = cand && run == rmax;
      x2 = eq && ntop == 1 ? a[i] : x2;
      x1 = gt ? a[i] : x1;
      ntop = gt ? 1 : ntop + (eq ? 1 : 0);
      rmax = gt ? run : rmax;
      start = end ? i + 1 : start;
    }
    rown -= N - deg;  // the padding counted as own label
    const int64_t cu = has ? node_w(c.g, u) : 1;
    const bool go = MODE == M_FAV ? rmax > 0 : rmax > rown;
    TieKey hv{0, 0};
    bool have_hv = false;
    LaneCand b1{rmax, 0u, x1};
    if (go && ntop >= 2) {
      hv = lane_tie_key<MODE, SEG>(c, u);
      have_hv = true;
      const LaneCand c1{rmax, tie_of(hv, x1), x1}, c2{rmax, tie_of(hv, x2), x2};
      b1 = lane_better(c1, c2) ? c1 : c2;
    }
    const bool many = go && ntop >= 3;
    bool full = false;
    const int64_t capu = go && MODE != M_FAV ? lane_cap<SEG>(c, u) : 0;
    if (go && MODE != M_FAV) full = c.lw[b1.x] + cu > capu;
    // rare: three or more labels tied at the top, or the winner is full;
    // the sorted labels go to this lane's column and the runs are walked
    if (__any_sync(kFull, many || full)) {
#pragma unroll
      for (int i = 0; i < N; ++i) ccol[i * 32] = a[i];
      if (many || full) {
        if (!have_hv) hv = lane_tie_key<MODE, SEG>(c, u);
        const int own_run = rown + (N - deg);  // the own label's entries, padding included
        LaneCand bb{-1, 0xffffffffu, INT32_MAX};
        for (int i = 0; i < N;) {
          const int32_t x = ccol[i * 32];
          if (x == own) {
            i += own_run;
            continue;
          }
          int j = i + 1;
          while (j < N && ccol[j * 32] == x) ++j;
          const int32_t r = j - i;
          i = j;
          if (many && !full) {  // the best of the top-tied labels
            if (r != rmax) continue;
          } else {  // the best admissible label that improves
            if (r <= rown) continue;
          }
          const LaneCand cand{r, tie_of(hv, x), x};
          if (lane_better(cand, bb) && (!full || MODE == M_FAV || c.lw[x] + cu <= capu))
            bb = cand;
        }
        if (!full) {
          b1 = bb;
          if (MODE != M_FAV) full = c.lw[b1.x] + cu > capu;
          if (full) {  // the top-tied winner is full: look again for an admissible one
            bb = LaneCand{-1, 0xffffffffu, INT32_MAX};
            for (int i = 0; i < N;) {
              const int32_t x = ccol[i * 32];
              if (x == own) {
                i += own_run;
                continue;
              }
              int j = i + 1;
              while (j < N && ccol[j * 32] == x) ++j;
              const int32_t r = j - i;
              i = j;
              if (r <= rown) continue;
              const LaneCand cand{r, tie_of(hv, x), x};
              if (lane_better(cand, bb) && c.lw[x] + cu <= capu) bb = cand;
            }
          }
        }
        if (full) b1 = bb;
      }
    }
    LaneCand best{-1, 0xffffffffu, INT32_MAX};
    if (go) best = b1;
    emit_lane<MODE>(c, has, u, own, rown, cu, best, mb, nmv);
    return;
  }
}

template <bool W>
__host__ __device__ constexpr int lane_warps() { return W ? 4 : kLaneWarps; }

// LONG: some compressed records exceed the 80-byte window (skewed graphs);
// a separate instantiation keeps the common kernel free of that path.
template <bool COMP, int MODE, bool W, bool LONG = false, bool SEG = false>
__global__ void __launch_bounds__(lane_warps<W>() * 32, W ? 1 : kLaneBlocksPerSM)
    k_rate_lane(RateCtx c) {
  static_assert(!(COMP && W), "weighted levels are CSR");
  constexpr int WARPS = lane_warps<W>();
  // per lane: staged record words, then candidate labels
  __shared__ uint32_t lab_all[WARPS][kLaneMaxDeg][32];
  __shared__ uint32_t aux_all[WARPS][W ? kLaneMaxDeg : 1][32];  // candidate ratings (weighted)
  __shared__ uint8_t cnt_all[WARPS][COMP && !W ? kLaneMaxDeg : 1][32];  // candidate ratings
  __shared__ int32_t queue_all[WARPS][kLaneQueue];
  __shared__ LaneMovers movers_all[WARPS];
  const int lane = lane_id(), w = threadIdx.x >> 5;
  uint32_t *col = &lab_all[w][0][lane];
  uint32_t *wcol = &aux_all[w][0][lane];
  int32_t *queue = queue_all[w];
  LaneMovers &mb = movers_all[w];
  uint8_t *cnt = &cnt_all[w][0][lane];
  // warps and list positions fit 32 bits (lists hold < 2^31 vertex ids)
  const int32_t gw = (int32_t)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int32_t nw = (int32_t)((gridDim.x * blockDim.x) >> 5);
  // bucket mode: this sub-round's lane-tier vertices come as a list
  const bool list_mode = MODE == M_LP && c.bucket != nullptr;
  int32_t bcount = 0, bnext = gw * kLaneWin;
  const int32_t *blist = c.bucket;
  const uint64_t *brec = COMP ? c.bucket_rec : nullptr;
  int64_t base = (int64_t)gw * 256;
  int j8 = 0, pending = 0;  // slab scan position; queued vertices (warp-uniform)
  if (list_mode) {
    const int64_t bstart = c.bucket_off[(int64_t)c.s * c.bucket_nb];
    bcount = (int32_t)(c.bucket_off[(int64_t)(c.s + 1) * c.bucket_nb] - bstart);
    blist += bstart;
    if (brec) brec += bstart;
    base = c.g.n;  // no slab scan
  }
  for (;;) {
    int take, wstart = 0;
    if (list_mode) {
      if (bnext >= bcount) break;
      wstart = bnext;
      take = bcount - bnext < kLaneWin ? bcount - bnext : kLaneWin;
      // never step past the end (keeps bnext below 2^31)
      bnext = bcount - bnext > nw * kLaneWin ? bnext + nw * kLaneWin : bcount;
    } else {
      // fill the queue, 32 vertices of the current 256-vertex slab at a time
      while (pending < kLaneWin && base < c.g.n) {
        const int64_t v = base + 32 * j8 + lane;
        const bool act = v < c.g.n && c.tier[v] == TIER_LANE && active<MODE>(c, v);
        const unsigned m = __ballot_sync(kFull, act);
        if (act) queue[pending + __popc(m & lanemask_lt())] = (int32_t)v;
        pending += __popc(m);
        if (++j8 == 8) j8 = 0, base += (int64_t)nw * 256;
      }
      if (pending == 0) break;
      __syncwarp();
      take = pending < kLaneWin ? pending : kLaneWin;
    }
    // batches of 32 in list order: vertices close in the list are close in
    // the graph, so a batch's records and label gathers share cache lines
    // (grouping a window by degree instead was measured slower)
    const int32_t *win = list_mode ? blist + wstart : queue;
    const uint64_t *wrec = list_mode && brec ? brec + wstart : nullptr;
    int nmv = 0;  // movers of this window so far (warp-uniform)
    for (int q = 0; q < take; q += 32) {
      const bool has = q + lane < take;
      const int32_t u = has ? win[q + lane] : 0;
      if (q + 32 + lane < take) lane_prefetch<COMP>(c.g, wrec, q + 32 + lane, win[q + 32 + lane]);
      int deg = 0;
      if (has) {
        if (COMP) {
          uint64_t rb, re;
          lane_record(c.g, wrec, q + lane, u, rb, re);
          // records beyond the 80-byte window (rare except on skewed graphs)
          // take the decoder that loads further groups
          if (LONG && __any_sync(__activemask(), (re - (rb & ~(uint64_t)15)) > 80))
            deg = lane_decode<true>(c.g, rb, re, col);
          else
            deg = lane_decode<false>(c.g, rb, re, col);
        } else {
          deg = min((int)(c.g.xadj[u + 1] - c.g.xadj[u]), kLaneMaxDeg);
        }
      }
      const unsigned maxdeg = __reduce_max_sync(kFull, (unsigned)deg);
      if (maxdeg <= 16) lane_batch<COMP, MODE, W, 16, SEG>(c, has, u, deg, col, wcol, cnt, mb, nmv);
      else lane_batch<COMP, MODE, W, kLaneMaxDeg, SEG>(c, has, u, deg, col, wcol, cnt, mb, nmv);
    }
    __syncwarp();
    if (nmv) {  // the window's movers, coalesced
      unsigned long long basep = 0;
      if (lane == 0) basep = atomicAdd(c.counters, (unsigned long long)nmv);
      basep = __shfl_sync(kFull, basep, 0);
      for (int i = lane; i < nmv; i += 32) {
        c.mv_u[basep + i] = mb.u[i];
        c.mv_t[basep + i] = mb.t[i];
        c.mv_o[basep + i] = mb.o[i];
        c.mv_g[basep + i] = mb.g[i];
      }
      __syncwarp();
    }
    if (!list_mode) {  // slab scans: move the vertices beyond the window to the front
      const int left = pending - take;
      const int32_t t = lane < left ? queue[take + lane] : 0;
      __syncwarp();
      if (lane < left) queue[lane] = t;
      __syncwarp();
      pending = left;
    }
  }
}

// Mid tier: one warp per listed vertex, its table of up to 2^LOG slots in
// shared memory (V: uint32_t counts at unit weights, int64_t sums otherwise;
// the smaller tables leave room for more warps per SM).
template <bool COMP, int MODE, int LOG, class V>
__global__ void k_rate_list(RateCtx c) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int32_t mu[kMidWarps][32], mt[kMidWarps][32], mo[kMidWarps][32];
  __shared__ int64_t mg[kMidWarps][32];
  const int w = threadIdx.x >> 5;
  WarpSmem<LOG, V> &ws = reinterpret_cast<WarpSmem<LOG, V> *>(smem_raw)[w];
  init_table(ws);
  MoverBuf mb{mu[w], mt[w], mo[w], mg[w], 0};
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  int64_t kb, ke;
  tier_range(c, kb, ke);
  for (int64_t k = kb + gw; k < ke; k += nw) {
    int64_t i, u;
    if (!tier_entry<MODE>(c, k, i, u)) continue;
    const int64_t d = COMP ? zip_nbr(c.g, u).deg : c.g.xadj[u + 1] - c.g.xadj[u];
    rate_vertex_warp<COMP, MODE, V>(c, u, ws.keys, ws.vals, table_log(c, d, LOG), &mb);
  }
  if (MODE == M_LP) flush_movers(c, mb);
}

// ---------------------------------------------------------------- big tier
// One block per listed vertex: its ratings are summed in a shared-memory
// hash table of 2^logc >= 1.5 deg slots (keys, then 32-bit counts for unit
// weights or 64-bit sums), so no rating touches global memory. A compressed
// neighbourhood (one chunk below the chunking threshold) is decoded by the
// whole block: every thread takes a slice of the record's bytes, assembles
// the values whose last byte lies in its slice (reading back into the
// previous slice for the first bytes of a value), and two block scans give
// each value its index and the sum of the gaps before it.
constexpr int kBlockThreads = 256;
constexpr int kBlockTinyLog = 11;   // 2048 slots: degrees up to kBigTinySplit = 1024
constexpr int kBlockMidLog = 12;    // 4096 slots: degrees up to kBigMidSplit = 2048
constexpr int kBlockSmallLog = 13;  // 8192 slots: degrees up to kBigSplit = 4096
constexpr int kBlockBigLog = 14;    // 16384 slots: degrees up to 10000
// Record staging and decoded values for a compressed vertex of degree <= dmax:
// at most 5 bytes per neighbour (+ alignment slack), 4 bytes per value.
__host__ __device__ constexpr size_t block_stage_bytes(int64_t dmax) {
  return ((size_t)(5 * dmax + 64) + 15) & ~(size_t)15;
}
__host__ __device__ constexpr size_t block_vbuf_bytes(int64_t dmax) { return (size_t)4 * dmax; }
__host__ __device__ constexpr int64_t block_max_deg(int lg) {
  return lg == kBlockTinyLog    ? kBigTinySplit
         : lg == kBlockMidLog   ? kBigMidSplit
         : lg == kBlockSmallLog ? kBigSplit
                                : kChunkThreshold;
}

// Block-wide exclusive sum of one int64 per thread; returns this thread's
// prefix and sets total. red holds kBlockThreads / 32 + 1 entries.
__device__ __forceinline__ int64_t block_excl_sum(int64_t v, int64_t *red, int64_t &total) {
  const int lane = lane_id(), w = threadIdx.x >> 5;
  const int64_t inc = warp_incl_scan(v);
  if (lane == 31) red[w] = inc;
  __syncthreads();
  if (w == 0) {
    const int64_t x = lane < kBlockThreads / 32 ? red[lane] : 0;
    const int64_t xi = warp_incl_scan(x);
    if (lane < kBlockThreads / 32) red[lane] = xi - x;
    if (lane == kBlockThreads / 32 - 1) red[kBlockThreads / 32] = xi;
  }
  __syncthreads();
  const int64_t r = red[w] + inc - v;
  total = red[kBlockThreads / 32];
  __syncthreads();
  return r;
}

// Block-wide exclusive sum of one uint32 per thread (same contract as
// block_excl_sum).
__device__ __forceinline__ uint32_t block_excl_sum32(uint32_t v, int64_t *red, uint32_t &total) {
  int64_t t;
  const int64_t r = block_excl_sum((int64_t)v, red, t);
  total = (uint32_t)t;
  return (uint32_t)r;
}

// Decodes one chunk [cb, ce) of u's neighbourhood (count values: the first
// a signed offset from u, then gaps) with the whole block and calls f(v)
// for every neighbour. The chunk's bytes are copied into shared memory
// (stage: at least ce - cb + 32 bytes, 16-byte aligned) with 16-byte loads;
// then (1) every thread counts the value ends (bytes without the
// continuation bit) in its slice of the bytes, (2) a block scan gives each
// thread the index of its first value and every thread writes the values
// ending in its slice to vbuf (count entries), each assembled without
// branches from its last byte and up to four preceding continuation bytes,
// (3) a block scan over the values turns them into neighbour ids, and (4)
// f(count) is called by every thread once the ids are in vbuf.
template <class F>
__device__ __forceinline__ void block_decode_range(const GView &g, int64_t u, uint64_t cb,
                                                   uint64_t ce, int64_t count, uint8_t *stage,
                                                   uint32_t *vbuf, int64_t *red, F &&f) {
  const uint64_t ws = cb & ~(uint64_t)15;
  const int off = (int)(cb - ws), L = (int)(ce - cb);
  const int ngroups = (off + L + 15) >> 4;
  const uint4 *src = reinterpret_cast<const uint4 *>(g.bytes + ws);
  for (int k = threadIdx.x; k < ngroups; k += kBlockThreads)
    reinterpret_cast<uint4 *>(stage)[k] = __ldcs(src + k);
  __syncthreads();
  const uint8_t *by = stage + off;
  const int K = (L + kBlockThreads - 1) / kBlockThreads;
  const int lo = min((int)threadIdx.x * K, L), hi = min((int)(threadIdx.x + 1) * K, L);
  uint32_t ends = 0;
  for (int p = lo; p < hi; ++p) ends += !(by[p] & 0x80u);
  uint32_t nval;
  uint32_t idx = block_excl_sum32(ends, red, nval);
  const int cnt = (int)min((int64_t)nval, count);
  if (threadIdx.x == 0 && (int64_t)nval != count) latch_error(g.err, TP_ERR_CORRUPT);
  // the four bytes before the slice (continuation bytes of a value ending in it)
  uint32_t win = 0;  // byte p-1 in bits 0..7, p-2 in 8..15, ...
#pragma unroll
  for (int d = 4; d >= 1; --d) win = (win << 8) | (lo - d >= 0 ? by[lo - d] : 0u);
  for (int p = lo; p < hi; ++p) {
    const uint32_t b0 = by[p];
    // continuation bytes directly before p: k = 0..4
    const uint32_t stop = ~win & 0x80808080u;
    const int k = stop ? (__ffs(stop) - 8) >> 3 : 4;
    // payloads of bytes p-1 .. p-4 packed 7 bits apart, p-1 lowest
    uint32_t pk = (win & 0x7fu) | ((win >> 1) & 0x3f80u) | ((win >> 2) & 0x1fc000u) |
                  ((win >> 3) & 0xfe00000u);
    // value = bytes p-k .. p, earliest byte lowest: reverse the k packed payloads
    uint32_t v = b0 & 0x7fu;
#pragma unroll
    for (int d = 0; d < 4; ++d) {
      const bool take = d < k;
      v = take ? (v << 7) | (pk & 0x7fu) : v;
      pk >>= 7;
    }
    if (!(b0 & 0x80u)) {
      if ((int)idx < cnt) vbuf[idx] = v;
      ++idx;
    }
    win = (win << 8) | b0;
  }
  __syncthreads();
  // ids: id_0 = u + signed offset, id_i = id_(i-1) + gap_i
  const int P = (cnt + kBlockThreads - 1) / kBlockThreads;
  const int a0 = min((int)threadIdx.x * P, cnt), a1 = min((int)(threadIdx.x + 1) * P, cnt);
  uint32_t part = 0;
  for (int i = max(a0, 1); i < a1; ++i) part += vbuf[i];
  uint32_t gtot;
  uint32_t run = block_excl_sum32(part, red, gtot);
  const uint32_t c0 = vbuf[0];
  const int64_t id0 = (c0 & 1u) ? u - (int64_t)(c0 >> 1) : u + (int64_t)(c0 >> 1);
  __syncthreads();  // vbuf[0] read by every thread before it is overwritten
  const int64_t nmax = g.n - 1;
  for (int i = a0; i < a1; ++i) {
    if (i > 0) run += vbuf[i];
    // streams are validated on creation; the clamp only keeps a corrupted
    // one from reading out of bounds
    vbuf[i] = (uint32_t)min(max(id0 + (int64_t)run, (int64_t)0), nmax);
  }
  __syncthreads();
  f(cnt);  // the ids are in vbuf[0 .. cnt)
  __syncthreads();  // stage and vbuf are reused
}

template <class V>
__device__ __forceinline__ void blk_add(int32_t *keys, V *vals, int logc, int32_t x, V w,
                                        int32_t *err) {
  const uint32_t mask = (1u << logc) - 1u;
  uint32_t h = slot_of(x, logc);
  for (uint32_t probe = 0; probe <= mask; ++probe, h = (h + 1) & mask) {
    int32_t k = keys[h];
    if (k == -1) {
      const int32_t prev = atomicCAS(&keys[h], -1, x);
      k = prev == -1 ? x : prev;
    }
    if (k == x) {
      atomicAdd(&vals[h], w);
      return;
    }
  }
  latch_error(err, TP_ERR_CORRUPT);
}

// Block-wide maxima of two values; the results are in every thread.
__device__ __forceinline__ void block_max2(int64_t &a, int64_t &b, int64_t *red) {
  a = warp_max(a);
  b = warp_max(b);
  const int lane = lane_id(), w = threadIdx.x >> 5;
  __shared__ int64_t rb[kBlockThreads / 32];
  if (lane == 0) red[w] = a, rb[w] = b;
  __syncthreads();
  int64_t x = lane < kBlockThreads / 32 ? red[lane] : INT64_MIN;
  int64_t y = lane < kBlockThreads / 32 ? rb[lane] : INT64_MIN;
  a = warp_max(x);
  b = warp_max(y);
  __syncthreads();
}

// Block-wide best (rating order) and own rating; the result is in every thread.
__device__ __forceinline__ void block_reduce_best(Best &b, Best *wb) {
  warp_reduce_best(b);
  const int lane = lane_id(), w = threadIdx.x >> 5;
  if (lane == 0) wb[w] = b;
  __syncthreads();
  b = lane < kBlockThreads / 32 ? wb[lane] : Best{-1, 0xffffffffu, INT32_MAX, 0};
  warp_reduce_best(b);
  __syncthreads();
}

template <bool COMP, int MODE, bool WT>
__global__ void __launch_bounds__(kBlockThreads) k_rate_block(RateCtx c, int maxlog) {
  using V = typename std::conditional<WT, unsigned long long, uint32_t>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  int32_t *keys = reinterpret_cast<int32_t *>(smem_raw);
  V *vals = reinterpret_cast<V *>(smem_raw + sizeof(int32_t) * ((size_t)1 << maxlog));
  // compressed: the record's bytes (at most 5 per neighbour, + alignment),
  // then its decoded values
  uint8_t *stage = reinterpret_cast<uint8_t *>(vals + ((size_t)1 << maxlog));
  uint32_t *vbuf = reinterpret_cast<uint32_t *>(stage + block_stage_bytes(block_max_deg(maxlog)));
  __shared__ int64_t red[kBlockThreads / 32 + 1];
  __shared__ Best wb[kBlockThreads / 32];
  __shared__ int32_t mu[32], mt[32], mo[32];
  __shared__ int64_t mg[32];
  const int tid = threadIdx.x;
  int64_t kb, ke;
  tier_range(c, kb, ke);
  for (int64_t k = kb + blockIdx.x; k < ke; k += gridDim.x) {
    int64_t i, u;
    if (!tier_entry<MODE>(c, k, i, u)) continue;  // uniform over the block
    const int64_t d = COMP ? zip_nbr(c.g, u).deg : c.g.xadj[u + 1] - c.g.xadj[u];
    int logc = 5;
    while (logc < maxlog && ((int64_t)1 << logc) < d + d / 2) ++logc;
    const int cap = 1 << logc;
    for (int k = tid; k < cap; k += kBlockThreads) keys[k] = -1, vals[k] = 0;
    __syncthreads();
    if (COMP) {
      const ZipNbr z = zip_nbr(c.g, u);  // one chunk: the big tier is below the chunking threshold
      block_decode_range(c.g, u, z.data, z.end, z.deg, stage, vbuf, red, [&](int cnt) {
        for (int e = tid; e < cnt; e += kBlockThreads)
          blk_add<V>(keys, vals, logc, c.label[vbuf[e]], (V)1, c.g.err);
      });
    } else {
      const int64_t b = c.g.xadj[u];
      for (int64_t e = tid; e < d; e += kBlockThreads) {
        const int32_t v = __ldcs(c.g.adj + b + e);
        blk_add<V>(keys, vals, logc, c.label[v], (V)(c.g.ew ? __ldcs(c.g.ew + b + e) : 1),
                   c.g.err);
      }
    }
    __syncthreads();
    // the top rating among the other labels and the own rating, then the tie
    // order among the top-rated labels only (as in the warp tiers)
    const int32_t own = c.label[u];
    const int64_t cu = node_w(c.g, u), capu = cap_of(c, u);
    int64_t rmax = -1, rown = 0;
    for (int k = tid; k < cap; k += kBlockThreads) {
      const int32_t x = keys[k];
      if (x < 0) continue;
      const int64_t R = (int64_t)vals[k];
      if (x == own) rown = R;
      else rmax = R > rmax ? R : rmax;
    }
    block_max2(rmax, rown, red);
    Best b;
    b.init();
    b.rown = rown;
    const bool rate = rmax >= 0 && (MODE != M_LP || rmax > rown);  // uniform over the block
    const TieKey hv = rate ? tie_key<MODE>(c, u) : TieKey{0, 0};
    if (rate) {
      for (int k = tid; k < cap; k += kBlockThreads) {
        const int32_t x = keys[k];
        if (x < 0 || x == own || (int64_t)vals[k] != rmax) continue;
        const uint32_t t = MODE == M_REBAL ? 0u : tie_of(hv, x);
        if (better(rmax, t, x, b.r, b.t, b.x)) b.r = rmax, b.t = t, b.x = x;
      }
      block_reduce_best(b, wb);
    }
    // the winner is full: the best admissible label instead (it must improve
    // on the own rating to matter)
    if (rate && MODE != M_FAV && b.x != INT32_MAX && c.lw[b.x] + cu > capu) {
      const int64_t rown = b.rown;
      b.init();
      for (int k = tid; k < cap; k += kBlockThreads) {
        const int32_t x = keys[k];
        if (x < 0 || x == own) continue;
        const int64_t R = (int64_t)vals[k];
        if (MODE == M_LP && R <= rown) continue;
        const uint32_t t = MODE == M_REBAL ? 0u : tie_of(hv, x);
        if (better(R, t, x, b.r, b.t, b.x) && c.lw[x] + cu <= capu) b.r = R, b.t = t, b.x = x;
      }
      block_reduce_best(b, wb);
      b.rown = rown;
    }
    if (tid < 32) {
      MoverBuf mb{mu, mt, mo, mg, 0};
      finalize_warp<MODE>(c, b, u, cu, &mb);
      if (MODE == M_LP) flush_movers(c, mb);
    }
    __syncthreads();
  }
}

// Huge tier, phase 1: one block per (vertex, chunk of 1000 neighbours; the
// compressed format's independently decodable chunks) sums the chunk's
// ratings in a shared-memory table and adds them into the vertex's global
// table (the paper's rating maps as flush buffers against contention).
constexpr int kHugeStage = (5 * kChunkSize + 64 + 15) & ~15;  // one chunk's bytes + alignment
template <bool COMP, int MODE>
__global__ void __launch_bounds__(kBlockThreads) k_rate_huge_chunks(RateCtx c) {
  __shared__ int32_t keys[1 << kHugeLog];
  __shared__ unsigned long long vals[1 << kHugeLog];
  __shared__ __align__(16) uint8_t stage[COMP ? kHugeStage : 16];
  __shared__ uint32_t vbuf[COMP ? kChunkSize : 1];
  __shared__ int64_t red[kBlockThreads / 32 + 1];
  __shared__ int64_t s_vi;
  __shared__ int32_t claimed[1 << kHugeLog];
  __shared__ int32_t s_nclaim, s_base;
  const int tid = threadIdx.x;
  for (int k = tid; k < (1 << kHugeLog); k += kBlockThreads) keys[k] = -1, vals[k] = 0;
  __syncthreads();
  // bucket mode: this sub-round's chunk items; else every chunk, skipping
  // inactive hubs (the hub of an item found by binary search)
  const int64_t ib = c.bpos ? c.hc_pre[c.boff[c.s]] : 0;
  const int64_t ie = c.bpos ? c.hc_pre[c.boff[c.s + 1]] : c.n_chunks;
  for (int64_t item = ib + blockIdx.x; item < ie; item += gridDim.x) {
    int64_t i, j;
    if (c.bpos) {
      const int64_t it = c.hc_item[item];
      i = it >> 32;
      j = it & 0xffffffffLL;
    } else {
      if (tid == 0) {  // vertex index: last i with chunk_start[i] <= item
        int64_t lo = 0, hi = c.list_n - 1;
        while (lo < hi) {
          const int64_t mid = (lo + hi + 1) / 2;
          if (c.chunk_start[mid] <= item) lo = mid;
          else hi = mid - 1;
        }
        s_vi = lo;
      }
      __syncthreads();
      i = s_vi;
      j = item - c.chunk_start[i];
      __syncthreads();  // s_vi is rewritten by the next item
    }
    const int64_t u = c.list[i];
    if (!c.bpos && !active<MODE>(c, u)) continue;  // uniform over the block
    if (COMP) {
      const ZipNbr z = zip_nbr(c.g, u);
      uint64_t cb, ce;
      int64_t cnt;
      zip_chunk(c.g, z, j, cb, ce, cnt);
      block_decode_range(c.g, u, cb, ce, cnt, stage, vbuf, red, [&](int n) {
        for (int e = tid; e < n; e += kBlockThreads)
          blk_add<unsigned long long>(keys, vals, kHugeLog, c.label[vbuf[e]], 1ull, c.g.err);
      });
    } else {
      const int64_t b = c.g.xadj[u] + j * kChunkSize;
      const int64_t e = min(b + kChunkSize, c.g.xadj[u + 1]);
      for (int64_t q = b + tid; q < e; q += kBlockThreads) {
        const int32_t v = __ldcs(c.g.adj + q);
        blk_add<unsigned long long>(keys, vals, kHugeLog, c.label[v],
                                    (unsigned long long)(c.g.ew ? __ldcs(c.g.ew + q) : 1), c.g.err);
      }
    }
    __syncthreads();
    int32_t *tk = c.tkeys + c.tbase + c.toff[i];
    int64_t *tv = c.tvals + c.tbase + c.toff[i];
    int32_t *tl = c.tlist + (c.tbase + c.toff[i]) / 2;
    const int lc = c.tcap[i];
    if (tid == 0) s_nclaim = 0;
    __syncthreads();
    // every thread inserts its kFlush shared slots together: each probe
    // step issues all pending key loads, then all claims (atomicCAS), so a
    // thread waits for one round trip per step instead of one per label
    constexpr int kFlush = (1 << kHugeLog) / kBlockThreads;
    {
      const uint32_t mask = (1u << lc) - 1u;
      int32_t lab[kFlush];
      int64_t w[kFlush];
      uint32_t h[kFlush], probes[kFlush];
      bool pend[kFlush];
#pragma unroll
      for (int q = 0; q < kFlush; ++q) {
        const int k = tid + q * kBlockThreads;
        lab[q] = keys[k];
        w[q] = (int64_t)vals[k];
        keys[k] = -1;
        vals[k] = 0;
        pend[q] = lab[q] >= 0;
        h[q] = pend[q] ? slot_of(lab[q], lc) : 0;
        probes[q] = 0;
      }
      for (;;) {
        bool any = false;
#pragma unroll
        for (int q = 0; q < kFlush; ++q) any |= pend[q];
        if (!any) break;
        int32_t cur[kFlush], prev[kFlush];
#pragma unroll
        for (int q = 0; q < kFlush; ++q) cur[q] = pend[q] ? *(volatile int32_t *)&tk[h[q]] : 0;
#pragma unroll
        for (int q = 0; q < kFlush; ++q)
          prev[q] = pend[q] && cur[q] == -1 ? atomicCAS(&tk[h[q]], -1, lab[q]) : 0;
#pragma unroll
        for (int q = 0; q < kFlush; ++q) {
          if (!pend[q]) continue;
          const int32_t kk = cur[q] == -1 ? (prev[q] == -1 ? lab[q] : prev[q]) : cur[q];
          if (kk == lab[q]) {
            atomicAdd((unsigned long long *)&tv[h[q]], (unsigned long long)w[q]);
            if (cur[q] == -1 && prev[q] == -1) claimed[atomicAdd(&s_nclaim, 1)] = (int32_t)h[q];
            pend[q] = false;
          } else if (++probes[q] > mask) {
            latch_error(c.g.err, TP_ERR_CORRUPT);  // more distinct labels than the table holds
            pend[q] = false;
          } else {
            h[q] = (h[q] + 1) & mask;
          }
        }
      }
    }
    __syncthreads();
    // the slots this chunk filled join the hub's list with one counter update
    if (tid == 0 && s_nclaim) s_base = atomicAdd(c.tcount + i, s_nclaim);
    __syncthreads();
    for (int j = tid; j < s_nclaim; j += kBlockThreads) tl[s_base + j] = claimed[j];
    __syncthreads();
  }
}

// Huge tier, phase 2: one block per vertex scans its global table.
static_assert(2 * sizeof(Best) == kSegBestBytes, "segment results are two Best records");

// Huge tier, phase 2: every (vertex, segment of 4096 table slots) is scanned
// by its own block for its best label ignoring the cap (with the own
// rating) and for its best admissible label; it then clears its slots.
// Admissibility is checked only for a label that beats the thread's best
// admissible one so far, so few label weights are read.
template <int MODE>
__global__ void __launch_bounds__(kBlockThreads) k_rate_huge_scan(RateCtx c, Best *seg_best) {
  __shared__ Best wb[kBlockThreads / 32];
  __shared__ int64_t s_vi;
  const int64_t ib = c.bpos ? c.hs_pre[c.boff[c.s]] : 0;
  const int64_t ie = c.bpos ? c.hs_pre[c.boff[c.s + 1]] : c.n_segs;
  for (int64_t item = ib + blockIdx.x; item < ie; item += gridDim.x) {
    int64_t i, sg;
    if (c.bpos) {
      const int64_t it = c.hs_item[item];
      i = it >> 32;
      sg = it & 0xffffffffLL;
    } else {
      if (threadIdx.x == 0) {  // vertex index: last i with seg_start[i] <= item
        int64_t lo = 0, hi = c.list_n - 1;
        while (lo < hi) {
          const int64_t mid = (lo + hi + 1) / 2;
          if (c.seg_start[mid] <= item) lo = mid;
          else hi = mid - 1;
        }
        s_vi = lo;
      }
      __syncthreads();
      i = s_vi;
      sg = item - c.seg_start[i];
      __syncthreads();
    }
    const int64_t u = c.list[i];
    if (!c.bpos && !active<MODE>(c, u)) continue;
    const int32_t own = c.label[u];
    const int64_t cu = node_w(c.g, u), capu = cap_of(c, u);
    const TieKey hv = tie_key<MODE>(c, u);
    // a table filled to an eighth or more is read in slot order (8192 slots
    // per segment); a sparser one through its list of filled slots (4096
    // list entries per segment)
    const int64_t filled = c.tcount[i], cap = (int64_t)1 << c.tcap[i];
    const bool dense = 8 * filled >= cap;
    const int64_t s0 = sg << kSegLog;
    const int64_t s1 = dense ? min(2 * (s0 + ((int64_t)1 << kSegLog)), cap)
                             : min(s0 + ((int64_t)1 << kSegLog), filled);
    int32_t *tk = c.tkeys + c.tbase + c.toff[i];
    int64_t *tv = c.tvals + c.tbase + c.toff[i];
    const int32_t *tl = c.tlist + (c.tbase + c.toff[i]) / 2;
    Best b, a;
    b.init();
    a.init();
    // kScanBatch slots per thread and step, every load of a step issued
    // before the first is used (list entries, then keys, then values), so a
    // thread waits for one round trip per step instead of one per slot
    constexpr int kScanBatch = 8;
    for (int64_t j0 = (dense ? 2 * s0 : s0) + threadIdx.x; j0 < s1;
         j0 += (int64_t)kBlockThreads * kScanBatch) {
      int32_t sl[kScanBatch], xs[kScanBatch];
      int64_t Rs[kScanBatch];
#pragma unroll
      for (int q = 0; q < kScanBatch; ++q) {
        const int64_t j = j0 + (int64_t)q * kBlockThreads;
        sl[q] = j < s1 ? (dense ? (int32_t)j : tl[j]) : -1;
      }
#pragma unroll
      for (int q = 0; q < kScanBatch; ++q) xs[q] = sl[q] >= 0 ? tk[sl[q]] : -1;
#pragma unroll
      for (int q = 0; q < kScanBatch; ++q) Rs[q] = xs[q] >= 0 ? tv[sl[q]] : 0;
#pragma unroll
      for (int q = 0; q < kScanBatch; ++q) {
        const int32_t x = xs[q];
        if (x < 0) continue;
        const int64_t R = Rs[q];
        tk[sl[q]] = -1;
        tv[sl[q]] = 0;
        if (x == own) {
          b.rown = R;
          continue;
        }
        const uint32_t t = MODE == M_REBAL ? 0u : tie_of(hv, x);
        if (better(R, t, x, b.r, b.t, b.x)) b.r = R, b.t = t, b.x = x;
        if (MODE != M_FAV && better(R, t, x, a.r, a.t, a.x) && c.lw[x] + cu <= capu)
          a.r = R, a.t = t, a.x = x;
      }
    }
    block_reduce_best(b, wb);
    if (MODE != M_FAV) block_reduce_best(a, wb);
    if (threadIdx.x == 0) {  // the hub's segment sg, where the decision reads it
      const int64_t q = c.seg_start[i] + sg;
      seg_best[2 * q] = b;
      seg_best[2 * q + 1] = a;
    }
  }
}

// Huge tier, phase 3: one block per vertex combines its segments: the best
// label if it is admissible, else the best admissible one; then it acts on
// the decision.
template <int MODE>
__global__ void __launch_bounds__(kBlockThreads) k_rate_huge_decide(RateCtx c, const Best *seg_best) {
  __shared__ Best wb[kBlockThreads / 32];
  __shared__ int32_t mu[32], mt[32], mo[32];
  __shared__ int64_t mg[32];
  int64_t kb, ke;
  tier_range(c, kb, ke);
  for (int64_t k = kb + blockIdx.x; k < ke; k += gridDim.x) {
    int64_t i, u;
    if (!tier_entry<MODE>(c, k, i, u)) continue;
    const int64_t cu = node_w(c.g, u);
    Best b, a;
    b.init();
    a.init();
    for (int64_t q = c.seg_start[i] + threadIdx.x; q < c.seg_start[i + 1]; q += kBlockThreads) {
      const Best o = seg_best[2 * q], oa = seg_best[2 * q + 1];
      if (better(o.r, o.t, o.x, b.r, b.t, b.x)) b.r = o.r, b.t = o.t, b.x = o.x;
      b.rown = max(b.rown, o.rown);
      if (better(oa.r, oa.t, oa.x, a.r, a.t, a.x)) a.r = oa.r, a.t = oa.t, a.x = oa.x;
    }
    block_reduce_best(b, wb);
    block_reduce_best(a, wb);
    if (MODE != M_FAV && b.x != INT32_MAX && c.lw[b.x] + cu > cap_of(c, u)) {
      // the winner is full: the best admissible label (for a move it must
      // also improve on the own rating, which finalize_warp checks)
      a.rown = b.rown;
      b = a;
    }
    if (threadIdx.x == 0) c.tcount[i] = 0;  // the segments cleared the table
    if (threadIdx.x < 32) {
      MoverBuf mb{mu, mt, mo, mg, 0};
      finalize_warp<MODE>(c, b, u, cu, &mb);
      if (MODE == M_LP) flush_movers(c, mb);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- approval
struct ApproveCtx {
  const int32_t *mv_u, *mv_t, *mv_o;
  const int64_t *mv_g;
  int8_t *mv_ok;
  int64_t *in_w;
  int32_t *ccnt, *cfill, *cseg, *ctarget;
  int64_t *cbase;
  unsigned long long *counters;  // [0] movers [1] contested targets [2] contested pool
  int32_t *label;
  int64_t *lw;
  int64_t cap;
  const int64_t *vw;
  // batched graphs: graph of every label and every graph's cap (null: one graph)
  const int32_t *lgid;
  const int64_t *gcap;
};

__device__ __forceinline__ int64_t vwt(const ApproveCtx &a, int64_t u) { return a.vw ? a.vw[u] : 1; }
__device__ __forceinline__ int64_t target_cap(const ApproveCtx &a, int32_t t) {
  return a.lgid ? a.gcap[a.lgid[t]] : a.cap;
}

// A: targets that fit take every mover; the others become contested and
// count their movers (the first one also lists the target).
__global__ void k_approve_fit(ApproveCtx a) {
  int64_t nm = (int64_t)a.counters[0];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nm;
       i += (int64_t)gridDim.x * blockDim.x) {
    int32_t t = a.mv_t[i];
    bool fits = a.lw[t] + a.in_w[t] <= target_cap(a, t);
    a.mv_ok[i] = fits;
    if (!fits && atomicAdd(&a.ccnt[t], 1) == 0) {
      unsigned long long j = atomicAdd(&a.counters[1], 1ull);
      a.ctarget[j] = t;
    }
  }
}

// A2: every contested target reserves its segment of the contested list.
__global__ void k_approve_alloc(ApproveCtx a) {
  int64_t nt = (int64_t)a.counters[1];
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nt;
       j += (int64_t)gridDim.x * blockDim.x) {
    int32_t t = a.ctarget[j];
    a.cbase[t] = (int64_t)atomicAdd(&a.counters[2], (unsigned long long)a.ccnt[t]);
  }
}

// B: contested movers are grouped by target.
__global__ void k_approve_scatter(ApproveCtx a) {
  int64_t nm = (int64_t)a.counters[0];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nm;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (a.mv_ok[i]) continue;
    int32_t t = a.mv_t[i];
    a.cseg[a.cbase[t] + atomicAdd(&a.cfill[t], 1)] = (int32_t)i;
  }
}

// Weighted radix select over 96-bit keys (hi = ~gain, lo = vertex): finds the
// first key whose inclusive weight prefix exceeds rem and returns it in
// (khi, klo). Every thread of the block must call it. Called only when the
// keys' total weight exceeds rem, so every pass selects a byte some remaining
// key carries: bytes on which all keys agree are taken without a pass.
template <class Item>
__device__ void block_select(int64_t cnt, int64_t rem, Item item, uint64_t &khi, uint32_t &klo) {
  __shared__ int64_t hist[256];
  __shared__ uint64_t fhi, mhi;
  __shared__ uint32_t flo, mlo;
  __shared__ int64_t cum;
  __shared__ unsigned long long and_hi, or_hi;
  __shared__ unsigned and_lo, or_lo;
  if (threadIdx.x == 0) {
    fhi = 0, mhi = 0, flo = 0, mlo = 0, cum = 0;
    and_hi = ~0ull, or_hi = 0, and_lo = ~0u, or_lo = 0;
  }
  __syncthreads();
  {  // bytes on which every key agrees need no histogram pass
    unsigned long long ah = ~0ull, oh = 0;
    unsigned al = ~0u, ol = 0;
    for (int64_t q = threadIdx.x; q < cnt; q += blockDim.x) {
      uint64_t hi;
      uint32_t lo;
      int64_t w;
      item(q, hi, lo, w);
      ah &= hi, oh |= hi, al &= lo, ol |= lo;
    }
    atomicAnd(&and_hi, ah), atomicOr(&or_hi, oh), atomicAnd(&and_lo, al), atomicOr(&or_lo, ol);
    __syncthreads();
  }
  for (int pass = 0; pass < 12; ++pass) {
    const bool in_hi = pass < 8;
    const int shift = in_hi ? 56 - 8 * pass : 24 - 8 * (pass - 8);
    const unsigned same = in_hi ? (unsigned)(((and_hi ^ or_hi) >> shift) & 255u)
                                : ((and_lo ^ or_lo) >> shift) & 255u;
    if (same == 0) {  // all keys carry this byte: it is the selected key's byte too
      if (threadIdx.x == 0) {
        if (in_hi) fhi |= ((uint64_t)and_hi >> shift & 255u) << shift, mhi |= 255ull << shift;
        else flo |= ((and_lo >> shift) & 255u) << shift, mlo |= 255u << shift;
      }
      __syncthreads();
      continue;
    }
    for (int b = threadIdx.x; b < 256; b += blockDim.x) hist[b] = 0;
    __syncthreads();
    for (int64_t q = threadIdx.x; q < cnt; q += blockDim.x) {
      uint64_t hi;
      uint32_t lo;
      int64_t w;
      item(q, hi, lo, w);
      if ((hi & mhi) != fhi || (lo & mlo) != flo) continue;
      uint32_t d = in_hi ? (uint32_t)(hi >> shift) & 255u : (lo >> shift) & 255u;
      atomicAdd((unsigned long long *)&hist[d], (unsigned long long)w);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int64_t run = cum;
      int b = 0;
      for (; b < 255; ++b) {
        if (run + hist[b] > rem) break;
        run += hist[b];
      }
      cum = run;
      if (in_hi) {
        fhi |= (uint64_t)b << shift;
        mhi |= 255ull << shift;
      } else {
        flo |= (uint32_t)b << shift;
        mlo |= 255u << shift;
      }
    }
    __syncthreads();
  }
  khi = fhi;
  klo = flo;
  __syncthreads();
}

// C: one block per contested target approves the longest fitting prefix in
// (gain desc, vertex asc) order.
__global__ void k_approve_contested(ApproveCtx a) {
  int64_t nt = (int64_t)a.counters[1];
  for (int64_t j = blockIdx.x; j < nt; j += gridDim.x) {
    int32_t t = a.ctarget[j];
    int64_t base = a.cbase[t], cnt = a.ccnt[t];
    int64_t rem = target_cap(a, t) - a.lw[t];
    __syncthreads();  // every thread has read ccnt before it is reset below
    if (threadIdx.x == 0) a.ccnt[t] = 0, a.cfill[t] = 0;
    auto item = [&](int64_t q, uint64_t &hi, uint32_t &lo, int64_t &w) {
      int32_t i = a.cseg[base + q];
      hi = ~(uint64_t)a.mv_g[i];
      lo = (uint32_t)a.mv_u[i];
      w = vwt(a, a.mv_u[i]);
    };
    if (rem < 0) continue;  // nothing can enter (mv_ok already 0)
    uint64_t khi;
    uint32_t klo;
    block_select(cnt, rem, item, khi, klo);
    for (int64_t q = threadIdx.x; q < cnt; q += blockDim.x) {
      uint64_t hi;
      uint32_t lo;
      int64_t w;
      item(q, hi, lo, w);
      if (hi < khi || (hi == khi && lo < klo)) a.mv_ok[a.cseg[base + q]] = 1;
    }
  }
}

// D: apply approved moves and reset the per-target counters. The grid covers
// the largest possible mover count, so every mover has its own thread and
// the dependent loads of different movers overlap.
__global__ void k_apply(ApproveCtx a) {
  int64_t nm = (int64_t)a.counters[0];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nm;
       i += (int64_t)gridDim.x * blockDim.x) {
    int32_t t = a.mv_t[i];
    if (a.mv_ok[i]) {
      int32_t u = a.mv_u[i];
      int64_t w = vwt(a, u);
      int32_t own = a.mv_o[i];  // labels change only here, so this is still u's label
      a.label[u] = t;
      atomicAdd((unsigned long long *)&a.lw[t], (unsigned long long)w);
      atomicAdd((unsigned long long *)&a.lw[own], (unsigned long long)(-w));
    }
    a.in_w[t] = 0;
  }
}

__global__ void k_init_singletons(const int64_t *vw, int64_t n, int32_t *label, int64_t *lw) {
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n;
       u += (int64_t)gridDim.x * blockDim.x) {
    label[u] = (int32_t)u;
    lw[u] = vw ? vw[u] : 1;
  }
}

// ---------------------------------------------------------------- tier dispatch
// Algorithmic bytes one round of rating must move for the vertices of one
// tier (level 0, unit weights): the tier's share of the adjacency stream and
// its offsets, one 4-byte label gather per adjacency entry, the own label
// and one 8-byte label-weight read per vertex.
double tier_round_bytes(const tp_graph *g, int64_t n_t, int64_t e_t) {
  double adj = g->compressed
                   ? (double)g->nbytes * (g->m2 ? (double)e_t / (double)g->m2 : 0.0) +
                         (double)n_t * (g->off_is64 ? 8.0 : 4.0)
                   : 4.0 * (double)e_t + 8.0 * (double)n_t;
  return adj + 4.0 * (double)e_t + 12.0 * (double)n_t;
}

template <int MODE>
void rate_tiers(tp_graph *g, RateCtx c, const tp_params &p, cudaStream_t s) {
  build_tiers(g, p, s);
  ensure_hub_tables(g, s);
  TierCache &T = g->tiers;
  c.g = view(g);
  c.tier = T.tier.get();
  {  // table slots per neighbour: a power of two in 1..8
    const int32_t sl = std::max(1, std::min(8, p.table_slack));
    c.slack = 1;
    while (c.slack < sl) c.slack <<= 1;
  }
  c.tkeys = T.tkeys.get();
  c.tvals = T.tvals.get();
  c.tlist = T.tlist.get();
  c.tcount = T.tcount.get();
  const int sms = num_sms();
  const bool comp = g->compressed;
  const bool prof = MODE == M_LP && prof_active();
  // bucket mode (M_LP with this round's tier buckets): tier t walks its
  // sub-round's positions only
  auto bucketed = [&](RateCtx &m, int t) {
    if (MODE == M_LP && c.tb_pos) {
      m.bpos = c.tb_pos + c.tb_base[t];
      m.boff = c.tb_off + (int64_t)t * (c.S + 1);
    } else {
      m.bpos = nullptr;
      m.boff = nullptr;
    }
  };
  const double per_launch = MODE == M_LP && c.S > 0 ? 1.0 / c.S : 0.0;
  const int64_t n_lane = MODE == M_REBAL ? 0 : T.count[TIER_LANE];
  const int64_t n_small = T.count[TIER_SMALL] + (MODE == M_REBAL ? T.count[TIER_LANE] : 0);
  if (n_lane > 0) {
    if (prof) prof_begin(PF_RATE_LANE, s);
    constexpr int LM = MODE == M_REBAL ? M_LP : MODE;
    if (g->unit_ew) {
      unsigned blocks = (unsigned)std::min<int64_t>(
          (g->n + 256 * kLaneWarps - 1) / (256 * kLaneWarps), (int64_t)sms * kLaneBlocksPerSM);
      // batched graphs are CSR unions
      if (comp && T.lane_long) launch(k_rate_lane<true, LM, false, true>, blocks, 32 * kLaneWarps, 0, s, c);
      else if (comp) launch(k_rate_lane<true, LM, false>, blocks, 32 * kLaneWarps, 0, s, c);
      else if (c.seg.gid) launch(k_rate_lane<false, LM, false, false, true>, blocks, 32 * kLaneWarps, 0, s, c);
      else launch(k_rate_lane<false, LM, false>, blocks, 32 * kLaneWarps, 0, s, c);
    } else {  // weighted levels are CSR
      constexpr int WW = lane_warps<true>();
      unsigned blocks =
          (unsigned)std::min<int64_t>((g->n + 256 * WW - 1) / (256 * WW), (int64_t)sms * 16);
      if (c.seg.gid) launch(k_rate_lane<false, LM, true, false, true>, blocks, 32 * WW, 0, s, c);
      else launch(k_rate_lane<false, LM, true>, blocks, 32 * WW, 0, s, c);
    }
    TP_LAUNCH_CHECK();
    if (prof) prof_end(PF_RATE_LANE, s, per_launch * tier_round_bytes(g, n_lane, T.edges[TIER_LANE]));
  }
  if (n_small > 0) {
    if (prof) prof_begin(PF_RATE_SMALL, s);
    int wpb = p.warps_per_block >= 1 && p.warps_per_block <= 16 ? p.warps_per_block : 8;
    size_t sm = sizeof(WarpSmem<kSmallLog>) * wpb;
    RateCtx m = c;
    int64_t items = g->n;
    if (MODE != M_REBAL) {
      m.list = T.small.get();
      m.list_n = T.n_small;
      items = T.n_small;
      bucketed(m, 0);
    } else {
      m.list = nullptr;
    }
    const int64_t per_warp = MODE != M_REBAL ? 1 : 32;  // list entries / vertices per warp step
    unsigned blocks = (unsigned)std::min<int64_t>((items + per_warp * wpb - 1) / (per_warp * wpb),
                                                  (int64_t)sms * 16);
    if (comp) launch(k_rate_small<true, MODE>, blocks, 32 * wpb, sm, s, m);
    else launch(k_rate_small<false, MODE>, blocks, 32 * wpb, sm, s, m);
    TP_LAUNCH_CHECK();
    if (prof) prof_end(PF_RATE_SMALL, s, per_launch * tier_round_bytes(g, T.count[TIER_SMALL], T.edges[TIER_SMALL]));
  }
  if (T.n_mid + T.n_mid2 > 0) {
    if (prof) prof_begin(PF_RATE_MID, s);
    // counts in 32 bits at unit weights (compressed levels have unit weights)
    const bool unit = g->unit_ew != 0;
    auto run = [&](const int32_t *list, int64_t cnt, int t, bool big_tables) {
      if (!cnt) return;
      RateCtx m = c;
      m.list = list;
      m.list_n = cnt;
      bucketed(m, t);
      const unsigned blocks =
          (unsigned)std::min<int64_t>((cnt + kMidWarps - 1) / kMidWarps, (int64_t)sms * 16);
#define TP_MID(LG, V)                                                                         \
  do {                                                                                        \
    const size_t sm = sizeof(WarpSmem<LG, V>) * kMidWarps;                                    \
    if (comp) launch(k_rate_list<true, MODE, LG, V>, blocks, 32 * kMidWarps, sm, s, m);      \
    else launch(k_rate_list<false, MODE, LG, V>, blocks, 32 * kMidWarps, sm, s, m);          \
  } while (0)
      if (big_tables) {
        if (unit) TP_MID(kMidLog, uint32_t);
        else TP_MID(kMidLog, int64_t);
      } else {
        if (unit) TP_MID(kMidSmallLog, uint32_t);
        else TP_MID(kMidSmallLog, int64_t);
      }
#undef TP_MID
      TP_LAUNCH_CHECK();
    };
    run(T.mid.get(), T.n_mid, 1, false);
    run(T.mid2.get(), T.n_mid2, 2, true);
    if (prof) prof_end(PF_RATE_MID, s, per_launch * tier_round_bytes(g, T.n_mid + T.n_mid2, T.edges[TIER_MID]));
  }
  if (T.n_big0 + T.n_big1 + T.n_big + T.n_big2 > 0) {
    if (prof) prof_begin(PF_RATE_BIG, s);
    const bool wt = !g->unit_ew;
    auto run = [&](const int32_t *list, int64_t cnt, int maxlog, int t) {
      if (!cnt) return;
      RateCtx m = c;
      m.list = list;
      m.list_n = cnt;
      bucketed(m, t);
      const size_t sm = ((size_t)1 << maxlog) * (sizeof(int32_t) + (wt ? 8 : 4)) +
                        (comp ? block_stage_bytes(block_max_deg(maxlog)) +
                                    block_vbuf_bytes(block_max_deg(maxlog))
                              : 0);
      const int per_sm = std::max(1, (int)((size_t)(228 * 1024) / (sm + 2048)));
      const unsigned blocks = (unsigned)std::min<int64_t>(cnt, (int64_t)sms * per_sm);
#define TP_BLK(CM, WW) launch(k_rate_block<CM, MODE, WW>, blocks, kBlockThreads, sm, s, m, maxlog)
      if (comp) TP_BLK(true, false);
      else if (wt) TP_BLK(false, true);
      else TP_BLK(false, false);
#undef TP_BLK
      TP_LAUNCH_CHECK();
    };
    run(T.big0.get(), T.n_big0, kBlockTinyLog, 3);
    run(T.big1.get(), T.n_big1, kBlockMidLog, 4);
    run(T.big.get(), T.n_big, kBlockSmallLog, 5);
    run(T.big2.get(), T.n_big2, kBlockBigLog, 6);
    if (prof) prof_end(PF_RATE_BIG, s, per_launch * tier_round_bytes(g, T.n_big0 + T.n_big1 + T.n_big + T.n_big2, T.edges[TIER_BIG]));
  }
  if (T.n_huge > 0) {
    if (prof) prof_begin(PF_RATE_HUGE, s);
    RateCtx m = c;
    m.list = T.huge.get();
    m.list_n = T.n_huge;
    bucketed(m, 7);
    m.toff = T.huge_toff.get();
    m.tcap = T.huge_tcap.get();
    m.tbase = 0;
    m.chunk_start = T.huge_chunk_start.get();
    m.n_chunks = T.n_huge_chunks;
    const unsigned blocks = (unsigned)std::max<int64_t>(
        1, std::min<int64_t>(T.n_huge_chunks, (int64_t)sms * 6));
    if (comp) launch(k_rate_huge_chunks<true, MODE>, blocks, kBlockThreads, 0, s, m);
    else launch(k_rate_huge_chunks<false, MODE>, blocks, kBlockThreads, 0, s, m);
    TP_LAUNCH_CHECK();
    m.seg_start = T.huge_seg_start.get();
    m.n_segs = T.n_huge_segs;
    Best *seg_best = reinterpret_cast<Best *>(T.huge_seg_best.get());
    const unsigned sb = (unsigned)std::max<int64_t>(1, std::min<int64_t>(T.n_huge_segs, (int64_t)sms * 8));
    launch(k_rate_huge_scan<MODE>, sb, kBlockThreads, 0, s, m, seg_best);
    const unsigned db = (unsigned)std::max<int64_t>(1, std::min<int64_t>(T.n_huge, (int64_t)sms * 4));
    launch(k_rate_huge_decide<MODE>, db, kBlockThreads, 0, s, m, (const Best *)seg_best);
    TP_LAUNCH_CHECK();
    if (prof) prof_end(PF_RATE_HUGE, s, per_launch * tier_round_bytes(g, T.n_huge, T.edges[TIER_HUGE]));
  }
}

template <class K>
void set_smem_limits(K kernel, size_t bytes) {
  TP_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
}

void configure_kernels_once() {
  size_t small16 = sizeof(WarpSmem<kSmallLog>) * 16;
#define TP_CFG_MID(M, LG, V)                                                       \
  set_smem_limits(k_rate_list<true, M, LG, V>, sizeof(WarpSmem<LG, V>) * kMidWarps); \
  set_smem_limits(k_rate_list<false, M, LG, V>, sizeof(WarpSmem<LG, V>) * kMidWarps);
#define TP_CFG_MODE(M)                                              \
  set_smem_limits(k_rate_small<true, M>, small16);                  \
  set_smem_limits(k_rate_small<false, M>, small16);                 \
  TP_CFG_MID(M, kMidSmallLog, uint32_t)                             \
  TP_CFG_MID(M, kMidSmallLog, int64_t)                              \
  TP_CFG_MID(M, kMidLog, uint32_t)                                  \
  TP_CFG_MID(M, kMidLog, int64_t)

  TP_CFG_MODE(M_LP)
  TP_CFG_MODE(M_FAV)
  TP_CFG_MODE(M_REBAL)
#undef TP_CFG_MODE
#undef TP_CFG_MID
  // the largest dynamic shared memory: weighted CSR with 16384 slots, or
  // compressed with 16384 slots and the record staging
  const size_t blk = std::max(((size_t)1 << kBlockBigLog) * (sizeof(int32_t) + 8),
                              ((size_t)1 << kBlockBigLog) * (sizeof(int32_t) + 4) +
                                  block_stage_bytes(kChunkThreshold) +
                                  block_vbuf_bytes(kChunkThreshold));
#define TP_CFG_BLOCK(M)                                   \
  set_smem_limits(k_rate_block<true, M, false>, blk);     \
  set_smem_limits(k_rate_block<false, M, false>, blk);    \
  set_smem_limits(k_rate_block<false, M, true>, blk);
  TP_CFG_BLOCK(M_LP)
  TP_CFG_BLOCK(M_FAV)
  TP_CFG_BLOCK(M_REBAL)
#undef TP_CFG_BLOCK
}

void configure_kernels() {
  static std::once_flag once;
  std::call_once(once, configure_kernels_once);
}

ApproveCtx approve_ctx(tp_graph *g, const LpState &st, LpWork &w) {
  ApproveCtx a;
  a.mv_u = w.mv_u.get();
  a.mv_o = w.mv_o.get();
  a.mv_t = w.mv_t.get();
  a.mv_g = w.mv_g.get();
  a.mv_ok = w.mv_ok.get();
  a.in_w = w.in_w.get();
  a.ccnt = w.ccnt.get();
  a.cfill = w.cfill.get();
  a.cseg = w.cseg.get();
  a.ctarget = w.ctarget.get();
  a.cbase = w.cbase.get();
  a.counters = (unsigned long long *)w.counters.get();
  a.label = st.label;
  a.lw = st.lw;
  a.cap = st.cap;
  a.vw = g->unit_vw ? nullptr : g->vw.get();
  a.lgid = st.seg.gid ? st.seg.lgid : nullptr;
  a.gcap = st.seg.cap;
  return a;
}

// A3: the lane-tier vertices of one round grouped by sub-round, in ascending
// vertex order inside every sub-round. Block b owns vertices
// [b * kBucketSpan, (b + 1) * kBucketSpan); pass 0 writes its count per
// sub-round to cnt[s * nblocks + b], an exclusive scan turns the counts into
// offsets, pass 1 writes every vertex at its offset plus its rank inside the
// block (chunks of 32 vertices in order, ballot ranks inside a chunk).
constexpr int kBucketSpan = 2048;
constexpr int kBucketChunks = kBucketSpan / 32;

// Pass 0 hashes every vertex once and keeps its sub-round + 1 in sub_byte
// (every rating tier tests it instead of hashing again) and counts the lane
// tier; pass 1 lists the lane tier. Lanes of a 32-vertex chunk with the
// same sub-round are grouped with one match instruction.
// With offsets (compressed graphs), pass 1 also stores each listed vertex's
// record start << 8 | record length in rec (lane-tier records are <= 65 bytes).
// Batched graphs (gid non-null): a vertex hashes its number inside its graph.
__global__ void __launch_bounds__(256) k_bucket(const uint8_t *tier, int64_t n, uint64_t rk_in,
                                                const uint64_t *rk_dev, int32_t S, bool fill,
                                                int64_t *cnt, int32_t *bucket, uint8_t *sub_byte,
                                                const uint32_t *o32, const uint64_t *o64,
                                                uint64_t *rec, const int32_t *gid,
                                                const int64_t *vb) {
  __shared__ int32_t chunk_cnt[kBucketChunks][32];  // [chunk][sub-round], S <= 32
  const int lane = lane_id(), w = threadIdx.x >> 5;
  const int64_t nblocks = gridDim.x;
  const int64_t lo = (int64_t)blockIdx.x * kBucketSpan;
  for (int i = threadIdx.x; i < kBucketChunks * 32; i += blockDim.x) (&chunk_cnt[0][0])[i] = 0;
  __syncthreads();
  const uint64_t rk = fill ? 0 : (rk_dev ? *rk_dev : rk_in);
  int32_t sub_of[kBucketChunks / 8];
  for (int q = 0; q < kBucketChunks / 8; ++q) {
    const int chunk = w + 8 * q;
    const int64_t u = lo + 32 * chunk + lane;
    int32_t sub = -1;
    if (u < n) {
      if (fill) {
        sub = tier[u] == TIER_LANE ? (int32_t)sub_byte[u] - 1 : -1;
      } else {
        // every vertex's sub-round is kept (the other tiers test it); only
        // the lane tier is listed
        const int64_t lu = gid ? u - vb[gid[u]] : u;
        const int32_t sr = sub_round_of(hstep(rk, (uint64_t)lu), S);
        sub_byte[u] = (uint8_t)(sr + 1);
        sub = tier[u] == TIER_LANE ? sr : -1;
      }
    }
    sub_of[q] = sub;
    const unsigned peers = __match_any_sync(kFull, sub);
    if (sub >= 0 && (peers & lanemask_lt()) == 0) chunk_cnt[chunk][sub] = __popc(peers);
  }
  __syncthreads();
  if (!fill) {
    for (int32_t k = threadIdx.x; k < S; k += blockDim.x) {
      int64_t t = 0;
      for (int ch = 0; ch < kBucketChunks; ++ch) t += chunk_cnt[ch][k];
      cnt[(int64_t)k * nblocks + blockIdx.x] = t;
    }
    return;
  }
  // exclusive prefix over the chunks of this block, per sub-round
  if (threadIdx.x < S) {
    const int k = threadIdx.x;
    int32_t run = 0;
    for (int ch = 0; ch < kBucketChunks; ++ch) {
      const int32_t c = chunk_cnt[ch][k];
      chunk_cnt[ch][k] = run;
      run += c;
    }
  }
  __syncthreads();
  for (int q = 0; q < kBucketChunks / 8; ++q) {
    const int chunk = w + 8 * q;
    const int32_t sub = sub_of[q];
    const unsigned peers = __match_any_sync(kFull, sub);
    if (sub >= 0) {
      const int64_t pos = cnt[(int64_t)sub * nblocks + blockIdx.x] + chunk_cnt[chunk][sub] +
                          __popc(peers & lanemask_lt());
      const int64_t u = lo + 32 * chunk + lane;
      bucket[pos] = (int32_t)u;
      if (rec) {
        const uint64_t b = o32 ? o32[u] : o64[u], e = o32 ? o32[u + 1] : o64[u + 1];
        rec[pos] = b << 8 | (e - b);
      }
    }
  }
}

// Tier buckets: count a list's vertices per sub-round (from sub_byte).
__global__ void k_tier_count(const int32_t *list, int64_t n, const uint8_t *sub_byte, int32_t S,
                             int64_t *cnt) {
  __shared__ int32_t sc[32];
  if (threadIdx.x < 32) sc[threadIdx.x] = 0;
  __syncthreads();
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&sc[sub_byte[list[k]] - 1], 1);
  __syncthreads();
  if (threadIdx.x < S && sc[threadIdx.x])
    atomicAdd((unsigned long long *)&cnt[threadIdx.x], (unsigned long long)sc[threadIdx.x]);
}

// Offsets of every tier's sub-rounds (one block): off[t * (S + 1) + s].
__global__ void k_tier_offsets(const int64_t *cnt, int32_t S, int tiers, int64_t *off, int64_t *cur) {
  if (threadIdx.x >= tiers) return;
  const int t = threadIdx.x;
  int64_t run = 0;
  for (int s = 0; s < S; ++s) {
    const int64_t c = cnt[t * S + s];  // cnt and cur may be the same array
    off[t * (S + 1) + s] = run;
    cur[t * S + s] = run;
    run += c;
  }
  off[t * (S + 1) + S] = run;
}

// Scatters a list's positions into its sub-round buckets: each block counts
// its slice per sub-round, reserves the ranges with one atomic each, then
// places its entries (the order inside a bucket does not matter).
constexpr int kTierSlice = 4096;
__global__ void k_tier_scatter(const int32_t *list, int64_t n, const uint8_t *sub_byte, int32_t S,
                               int64_t *cur, int32_t *pos) {
  __shared__ int32_t sc[32];
  __shared__ int64_t base[32];
  for (int64_t lo = (int64_t)blockIdx.x * kTierSlice; lo < n; lo += (int64_t)gridDim.x * kTierSlice) {
    const int64_t hi = min(lo + kTierSlice, n);
    if (threadIdx.x < 32) sc[threadIdx.x] = 0;
    __syncthreads();
    for (int64_t k = lo + threadIdx.x; k < hi; k += blockDim.x) atomicAdd(&sc[sub_byte[list[k]] - 1], 1);
    __syncthreads();
    if (threadIdx.x < S) {
      base[threadIdx.x] = sc[threadIdx.x]
                              ? (int64_t)atomicAdd((unsigned long long *)&cur[threadIdx.x],
                                                   (unsigned long long)sc[threadIdx.x])
                              : 0;
      sc[threadIdx.x] = 0;
    }
    __syncthreads();
    for (int64_t k = lo + threadIdx.x; k < hi; k += blockDim.x) {
      const int s = sub_byte[list[k]] - 1;
      pos[base[s] + atomicAdd(&sc[s], 1)] = (int32_t)k;
    }
    __syncthreads();
  }
}

// Huge tier: chunk and segment counts of the hubs in bucket order.
__global__ void k_huge_counts(const int32_t *bpos, int64_t nh, const int64_t *chunk_start,
                              const int64_t *seg_start, int64_t *hc, int64_t *hs) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nh;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = bpos[k];
    hc[k] = chunk_start[p + 1] - chunk_start[p];
    hs[k] = seg_start[p + 1] - seg_start[p];
  }
}

// Huge tier: the items of every hub (warp per hub), hub position << 32 | index.
__global__ void k_huge_items(const int32_t *bpos, int64_t nh, const int64_t *pre,
                             int64_t *item) {
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t k = gw; k < nh; k += nw) {
    const int64_t p = bpos[k];
    for (int64_t j = pre[k] + lane_id(); j < pre[k + 1]; j += 32) item[j] = p << 32 | (j - pre[k]);
  }
}

}  // namespace

// Buckets the warp and block tiers' lists of this round by sub-round.
static void tier_buckets(tp_graph *g, LpWork &w, int32_t S, cudaStream_t stream) {
  TierCache &T = g->tiers;
  const int32_t *lists[LpWork::kTiers] = {T.small.get(), T.mid.get(),  T.mid2.get(),
                                          T.big0.get(),  T.big1.get(), T.big.get(),
                                          T.big2.get(),  T.huge.get()};
  const int64_t lens[LpWork::kTiers] = {T.n_small, T.n_mid, T.n_mid2, T.n_big0,
                                        T.n_big1,  T.n_big, T.n_big2, T.n_huge};
  int64_t total = 0;
  for (int t = 0; t < LpWork::kTiers; ++t) w.tb_base[t] = total, total += lens[t];
  w.tb_valid = false;
  if (total == 0) return;
  if ((int64_t)w.tb_pos.n < total) w.tb_pos.alloc(total, stream);
  if ((int64_t)w.tb_off.n < LpWork::kTiers * 33) {
    w.tb_off.alloc(LpWork::kTiers * 33, stream);
    w.tb_cur.alloc(LpWork::kTiers * 32, stream);
  }
  TP_CUDA(cudaMemsetAsync(w.tb_cur.get(), 0, sizeof(int64_t) * LpWork::kTiers * S, stream));
  const int sms = num_sms();
  for (int t = 0; t < LpWork::kTiers; ++t)
    if (lens[t])
      launch(k_tier_count, grid_for(lens[t], 256, (int64_t)sms * 4), 256, 0, stream, lists[t],
             lens[t], w.bucket_sub.get(), S, w.tb_cur.get() + (int64_t)t * S);
  launch(k_tier_offsets, 1, 32, 0, stream, w.tb_cur.get(), S, LpWork::kTiers, w.tb_off.get(),
         w.tb_cur.get());
  for (int t = 0; t < LpWork::kTiers; ++t)
    if (lens[t])
      launch(k_tier_scatter, grid_for(lens[t], kTierSlice, (int64_t)sms * 4), 256, 0, stream,
             lists[t], lens[t], w.bucket_sub.get(), S, w.tb_cur.get() + (int64_t)t * S,
             w.tb_pos.get() + w.tb_base[t]);
  TP_LAUNCH_CHECK();
  if (T.n_huge) {
    const int64_t nh = T.n_huge;
    if ((int64_t)w.hc_pre.n < nh + 1) {
      w.hc_pre.alloc(nh + 1, stream);
      w.hs_pre.alloc(nh + 1, stream);
    }
    if ((int64_t)w.hc_item.n < std::max<int64_t>(T.n_huge_chunks, 1))
      w.hc_item.alloc(std::max<int64_t>(T.n_huge_chunks, 1), stream);
    if ((int64_t)w.hs_item.n < std::max<int64_t>(T.n_huge_segs, 1))
      w.hs_item.alloc(std::max<int64_t>(T.n_huge_segs, 1), stream);
    const int32_t *hp = w.tb_pos.get() + w.tb_base[7];
    launch(k_huge_counts, grid_for(nh, 256), 256, 0, stream, hp, nh, T.huge_chunk_start.get(),
           T.huge_seg_start.get(), w.hc_pre.get(), w.hs_pre.get());
    exclusive_scan_i64(w.hc_pre.get(), w.hc_pre.get(), nh, stream);
    exclusive_scan_i64(w.hs_pre.get(), w.hs_pre.get(), nh, stream);
    launch(k_huge_items, grid_for(nh * 32, 256), 256, 0, stream, hp, nh, w.hc_pre.get(),
           w.hc_item.get());
    launch(k_huge_items, grid_for(nh * 32, 256), 256, 0, stream, hp, nh, w.hs_pre.get(),
           w.hs_item.get());
    TP_LAUNCH_CHECK();
  }
  w.tb_valid = true;
}

void lp_bucket(tp_graph *g, LpWork &w, uint64_t rk, int32_t S, const tp_params &p,
               cudaStream_t stream, const uint64_t *rk_dev, bool tiers, const SegLp *seg) {
  const int32_t *gid = seg ? seg->gid : nullptr;
  const int64_t *vb = seg ? seg->vb : nullptr;
  build_tiers(g, p, stream);
  w.bucket_S = 0;
  if (S > 32) return;
  const int64_t nblocks = (g->n + kBucketSpan - 1) / kBucketSpan;
  if (!w.bucket.get()) w.bucket.alloc(std::max<int64_t>(w.n, 1), stream);
  if (!w.bucket_sub.get()) w.bucket_sub.alloc(std::max<int64_t>(w.n, 1), stream);
  if ((int64_t)w.bucket_off.n < S * nblocks + 1) w.bucket_off.alloc(S * nblocks + 1, stream);
  const bool zrec = g->compressed != 0;
  if (zrec && !w.bucket_rec.get()) w.bucket_rec.alloc(std::max<int64_t>(w.n, 1), stream);
  const uint32_t *o32 = zrec && !g->off_is64 ? g->off32.get() : nullptr;
  const uint64_t *o64 = zrec && g->off_is64 ? g->off64.get() : nullptr;
  uint64_t *rec = zrec ? w.bucket_rec.get() : nullptr;
  launch(k_bucket, (unsigned)nblocks, 256, 0, stream, g->tiers.tier.get(), g->n, rk, rk_dev, S,
         false, w.bucket_off.get(), w.bucket.get(), w.bucket_sub.get(), o32, o64, rec, gid, vb);
  exclusive_scan_i64(w.bucket_off.get(), w.bucket_off.get(), S * nblocks, stream);
  launch(k_bucket, (unsigned)nblocks, 256, 0, stream, g->tiers.tier.get(), g->n, rk, rk_dev, S,
         true, w.bucket_off.get(), w.bucket.get(), w.bucket_sub.get(), o32, o64, rec, gid, vb);
  TP_LAUNCH_CHECK();
  w.bucket_S = S;
  w.bucket_nblocks = nblocks;
  w.tb_valid = false;
  if (tiers) tier_buckets(g, w, S, stream);
}

void LpWork::init(int64_t n_vertices, int64_t n_labels, cudaStream_t s) {
  if (n_vertices <= n && n_labels <= nlabels) return;
  n = std::max(n, n_vertices);
  nlabels = std::max(nlabels, n_labels);
  size_t L = (size_t)std::max<int64_t>(nlabels, 1), N = (size_t)std::max<int64_t>(n, 1);
  in_w.alloc(L, s);
  ccnt.alloc(L, s);
  cfill.alloc(L, s);
  cbase.alloc(L, s);
  ctarget.alloc(L, s);
  mv_u.alloc(N, s);
  mv_t.alloc(N, s);
  mv_o.alloc(N, s);
  mv_g.alloc(N, s);
  mv_ok.alloc(N, s);
  cseg.alloc(N, s);
  counters.alloc(4, s);
  TP_CUDA(cudaMemsetAsync(in_w.get(), 0, L * 8, s));
  TP_CUDA(cudaMemsetAsync(ccnt.get(), 0, L * 4, s));
  TP_CUDA(cudaMemsetAsync(cfill.get(), 0, L * 4, s));
  TP_CUDA(cudaMemsetAsync(counters.get(), 0, 4 * 8, s));
}

// The approval of one sub-round: the same five kernels and counter reset on
// every sub-round of a level (only the data differs).
constexpr int kApproveKernels = 5;
void launch_approval(const ApproveCtx &a, int64_t wn, int64_t *counters, cudaStream_t stream) {
  const unsigned blocks = (unsigned)num_sms() * 4;
  const unsigned wide = grid_for(std::max<int64_t>(wn, 1), 256, (int64_t)num_sms() * 64);
  launch(k_approve_fit, wide, 256, 0, stream, a);
  launch(k_approve_alloc, (unsigned)num_sms(), 256, 0, stream, a);
  launch(k_approve_scatter, blocks, 256, 0, stream, a);
  launch(k_approve_contested, (unsigned)num_sms() * 2, 256, 0, stream, a);
  launch(k_apply, wide, 256, 0, stream, a);
  TP_LAUNCH_CHECK();
  TP_CUDA(cudaMemsetAsync(counters, 0, 4 * sizeof(int64_t), stream));
}

// Records the approval of a level's sub-rounds into a CUDA graph on a
// private stream, so each sub-round replays it with one launch. Returns null
// (callers then launch directly) if capturing is not possible.
struct ApprovalGraph {
  cudaStream_t cs = nullptr;
  cudaGraphExec_t exec = nullptr;
  ApprovalGraph(const ApproveCtx &a, int64_t wn, int64_t *counters) {
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
      (void)cudaGetLastError();
      cs = nullptr;
      return;
    }
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      (void)cudaGetLastError();
      return;
    }
    capture_counting(true);
    bool ok = true;
    try {
      launch_approval(a, wn, counters, cs);
    } catch (...) {
      ok = false;
    }
    capture_counting(false);
    cudaGraph_t graph = nullptr;
    if (cudaStreamEndCapture(cs, &graph) != cudaSuccess || !ok || !graph) {
      (void)cudaGetLastError();
      if (graph) cudaGraphDestroy(graph);
      return;
    }
    if (cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
      (void)cudaGetLastError();
      exec = nullptr;
    }
    cudaGraphDestroy(graph);
  }
  ~ApprovalGraph() {
    if (exec) cudaGraphExecDestroy(exec);
    if (cs) cudaStreamDestroy(cs);
  }
};

void lp_subround(tp_graph *g, const LpState &st, LpWork &w, uint64_t rk, int32_t S, int32_t s,
                 const tp_params &p, cudaStream_t stream, cudaGraphExec_t approval,
                 const uint64_t *rk_dev) {
  configure_kernels();
  RateCtx c{};
  c.label = st.label;
  c.lw = st.lw;
  c.cap = st.cap;
  c.seg = st.seg;
  c.rk = rk;
  c.rk_dev = rk_dev;
  c.S = S;
  c.s = s;
  c.mv_u = w.mv_u.get();
  c.mv_o = w.mv_o.get();
  c.mv_t = w.mv_t.get();
  c.mv_g = w.mv_g.get();
  c.in_w = w.in_w.get();
  c.counters = (unsigned long long *)w.counters.get();
  if (w.bucket_S == S) {
    c.bucket = w.bucket.get();
    c.bucket_off = w.bucket_off.get();
    c.bucket_nb = w.bucket_nblocks;
    c.bucket_rec = g->compressed ? w.bucket_rec.get() : nullptr;
    c.sub_byte = w.bucket_sub.get();
    if (w.tb_valid) {
      c.tb_pos = w.tb_pos.get();
      c.tb_off = w.tb_off.get();
      for (int t = 0; t < LpWork::kTiers; ++t) c.tb_base[t] = w.tb_base[t];
      c.hc_pre = w.hc_pre.get();
      c.hs_pre = w.hs_pre.get();
      c.hc_item = w.hc_item.get();
      c.hs_item = w.hs_item.get();
    }
  }
  rate_tiers<M_LP>(g, c, p, stream);
  prof_begin(PF_APPROVE, stream);
  if (approval) {
    TP_CUDA(cudaGraphLaunch(approval, stream));
    count_launches(kApproveKernels);
  } else {
    launch_approval(approve_ctx(g, st, w), w.n, w.counters.get(), stream);
  }
  prof_end(PF_APPROVE, stream, 0.0);
}

// Round key of round *r (then r advances): the first node of a replayed
// round graph.
__global__ void k_round_key(uint64_t seed, uint64_t tag, uint64_t a, uint64_t b0, int32_t *r,
                            uint64_t *rk) {
  *rk = round_key(seed, tag, a, b0 + (uint64_t)*r);
  *r += 1;
}

// Small levels: a whole LP round (round key, bucketing, every sub-round's
// rating and approval) is recorded once as a CUDA graph on a private stream
// and replayed once per round on the caller's stream, the round key coming
// from device memory. Levels above this size launch directly (their kernels
// are long enough to hide launch costs, and their bucket scan would allocate
// inside the graph).
constexpr int64_t kRoundGraphMaxN = (int64_t)1 << 19;

bool lp_rounds_graph(tp_graph *g, const LpState &st, LpWork &w, uint64_t seed, uint64_t tag,
                     uint64_t a, uint64_t b0, int32_t rounds, int32_t S, const tp_params &p,
                     cudaStream_t stream) {
  configure_kernels();
  build_tiers(g, p, stream);  // synchronises; must not run while capturing
  ensure_hub_tables(g, stream);  // nor may the tables be allocated inside the capture
  const int64_t nblocks = (g->n + kBucketSpan - 1) / kBucketSpan;
  if (S > 32 || S * nblocks > 2048) return false;
  if (!w.bucket.get()) w.bucket.alloc(std::max<int64_t>(w.n, 1), stream);
  if (!w.bucket_sub.get()) w.bucket_sub.alloc(std::max<int64_t>(w.n, 1), stream);
  if ((int64_t)w.bucket_off.n < S * nblocks + 1) w.bucket_off.alloc(S * nblocks + 1, stream);
  if (g->compressed && !w.bucket_rec.get()) w.bucket_rec.alloc(std::max<int64_t>(w.n, 1), stream);
  Buf<int32_t> d_r(1, stream);
  Buf<uint64_t> d_rk(1, stream);
  TP_CUDA(cudaMemsetAsync(d_r.get(), 0, sizeof(int32_t), stream));
  cudaStream_t cs = nullptr;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  struct StreamGuard {
    cudaStream_t s;
    ~StreamGuard() { cudaStreamDestroy(s); }
  } sg{cs};
  if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  capture_counting(true);
  bool ok = true;
  try {
    launch(k_round_key, 1u, 1u, 0, cs, seed, tag, a, b0, d_r.get(), d_rk.get());
    lp_bucket(g, w, 0, S, p, cs, d_rk.get(), false, &st.seg);
    for (int32_t s = 0; s < S; ++s) lp_subround(g, st, w, 0, S, s, p, cs, nullptr, d_rk.get());
    w.bucket_S = 0;
  } catch (...) {
    ok = false;
  }
  const uint64_t kernels = capture_counting(false);
  cudaGraph_t graph = nullptr;
  if (cudaStreamEndCapture(cs, &graph) != cudaSuccess || !ok || !graph) {
    (void)cudaGetLastError();
    if (graph) cudaGraphDestroy(graph);
    return false;
  }
  cudaGraphExec_t exec = nullptr;
  const bool inst = cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
  cudaGraphDestroy(graph);
  if (!inst) {
    (void)cudaGetLastError();
    return false;
  }
  struct ExecGuard {
    cudaGraphExec_t e;
    ~ExecGuard() { cudaGraphExecDestroy(e); }
  } eg{exec};
  for (int32_t r = 0; r < rounds; ++r) {
    TP_CUDA(cudaGraphLaunch(exec, stream));
    count_launches(kernels);
  }
  return true;
}

void lp_rounds(tp_graph *g, const LpState &st, LpWork &w, uint64_t seed, uint64_t tag, uint64_t a,
               uint64_t b0, int32_t rounds, int32_t S, const tp_params &p, cudaStream_t stream) {
  if (rounds <= 0) return;
  if (p.use_graphs && g->n <= std::min<int64_t>(p.graph_n, kRoundGraphMaxN) && !prof_active() &&
      lp_rounds_graph(g, st, w, seed, tag, a, b0, rounds, S, p, stream))
    return;
  ApprovalGraph ag(approve_ctx(g, st, w), w.n, w.counters.get());
  for (int32_t r = 0; r < rounds; ++r) {
    uint64_t rk = round_key(seed, tag, a, b0 + (uint64_t)r);
    lp_bucket(g, w, rk, S, p, stream, nullptr, true, &st.seg);
    for (int32_t s = 0; s < S; ++s) lp_subround(g, st, w, rk, S, s, p, stream, ag.exec);
    w.bucket_S = 0;
    w.tb_valid = false;
  }
}

// ---------------------------------------------------------------- two-hop packing
namespace {

__global__ void k_fav_init(int32_t *fav, int64_t n) {
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n;
       u += (int64_t)gridDim.x * blockDim.x)
    fav[u] = -2;
}

__global__ void k_th_flags(const int32_t *fav, int64_t n, int32_t *flag) {
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n;
       u += (int64_t)gridDim.x * blockDim.x)
    flag[u] = fav[u] >= 0;
}

__global__ void k_th_gather(const int32_t *fav, const int32_t *flag, const int64_t *pos, int64_t n,
                            uint64_t *keys, uint64_t *vals) {
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n;
       u += (int64_t)gridDim.x * blockDim.x)
    if (flag[u]) {
      keys[pos[u]] = (uint64_t)fav[u];
      vals[pos[u]] = (uint64_t)u;
    }
}

// weights in sorted order and run-start markers
__global__ void k_th_prep(const uint64_t *keys, const uint64_t *vals, const int64_t *vw, int64_t m,
                          int64_t *wt, int64_t *rs) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x) {
    wt[i] = vw ? vw[vals[i]] : 1;
    rs[i] = (i == 0 || keys[i] != keys[i - 1]) ? i : -1;
  }
}

// bins, straddlers and group heads (batched graphs: a group lies in one
// graph, whose U is gU[gid[vertex]])
__global__ void k_th_heads(const int64_t *excl, const int64_t *rs, const int64_t *wt, int64_t m,
                           int64_t U_one, const uint64_t *vals, const int32_t *gid,
                           const int64_t *gU, int64_t *head) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t U = gid ? gU[gid[vals[i]]] : U_one;
    int64_t P = excl[i] - excl[rs[i]];
    int64_t bin = P / U;
    bool str = P + wt[i] > (bin + 1) * U;
    bool h = false;
    if (!str) {
      if (i == rs[i]) h = true;
      else {
        int64_t Pp = excl[i - 1] - excl[rs[i - 1]];
        int64_t binp = Pp / U;
        bool strp = Pp + wt[i - 1] > (binp + 1) * U;
        h = strp || binp != bin;
      }
    }
    head[i] = str ? -2 : (h ? i : -1);
  }
}

__global__ void k_th_assign(const int64_t *head_raw, const int64_t *head_scan,
                            const uint64_t *vals, int64_t m, int32_t *C) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (head_raw[i] == -2) continue;  // straddler stays alone
    C[vals[i]] = (int32_t)vals[head_scan[i]];
  }
}

}  // namespace

void favourites(tp_graph *g, const int32_t *C, const int64_t *Wc, uint64_t rk, int32_t *fav,
                const tp_params &p, cudaStream_t s, const SegLp *seg) {
  configure_kernels();
  launch(k_fav_init, grid_for(g->n, 256), 256, 0, s, fav, g->n);
  TP_LAUNCH_CHECK();
  RateCtx c{};
  c.label = C;
  c.lw = Wc;
  c.rk = rk;
  c.fav = fav;
  if (seg) c.seg = *seg;
  rate_tiers<M_FAV>(g, c, p, s);
}

void two_hop(tp_graph *g, int32_t *C, const int64_t *Wc, int64_t U, uint64_t seed, int32_t level,
             const tp_params &p, cudaStream_t s, const SegLp *seg) {
  int64_t n = g->n;
  if (n == 0) return;
  const bool sg = seg && seg->gid;
  Buf<int32_t> fav(n, s), flag(n, s);
  favourites(g, C, Wc, round_key(seed, kTagTwoHop, (uint64_t)level, 0), fav.get(), p, s, seg);
  launch(k_th_flags, grid_for(n, 256), 256, 0, s, fav.get(), n, flag.get());
  TP_LAUNCH_CHECK();
  Buf<int64_t> pos(n + 1, s);
  exclusive_scan_i32_to_i64(flag.get(), pos.get(), n, s);
  int64_t m = read_scalar(pos.get() + n, s);
  if (m == 0) return;
  Buf<uint64_t> keys(m, s), vals(m, s);
  launch(k_th_gather, grid_for(n, 256), 256, 0, s, fav.get(), flag.get(), pos.get(), n, keys.get(),
                                                 vals.get());
  TP_LAUNCH_CHECK();
  // keys: favourites (vertex ids) and the no-favourite key n (per graph:
  // n + graph), so no group spans two graphs
  radix_sort_pairs(keys.get(), vals.get(), m,
                   bits_for((uint64_t)n + (sg ? (uint64_t)seg->ngraphs : 0)), s);
  Buf<int64_t> wt(m, s), rs(m, s), excl(m + 1, s), head(m, s), hs(m, s);
  launch(k_th_prep, grid_for(m, 256), 256, 0, s, keys.get(), vals.get(),
                                               g->unit_vw ? nullptr : g->vw.get(), m, wt.get(),
                                               rs.get());
  TP_LAUNCH_CHECK();
  inclusive_max_scan_i64(rs.get(), rs.get(), m, s);
  exclusive_scan_i64(wt.get(), excl.get(), m, s);
  launch(k_th_heads, grid_for(m, 256), 256, 0, s, excl.get(), rs.get(), wt.get(), m, U, vals.get(),
         sg ? seg->gid : nullptr, sg ? seg->cap : nullptr, head.get());
  TP_LAUNCH_CHECK();
  inclusive_max_scan_i64(head.get(), hs.get(), m, s);
  launch(k_th_assign, grid_for(m, 256), 256, 0, s, head.get(), hs.get(), vals.get(), m, C);
  TP_LAUNCH_CHECK();
}

void lp_cluster(tp_graph *g, int64_t U, const tp_params &p, int32_t level, int32_t *d_cluster,
                cudaStream_t s, cudaEvent_t ev_begin, cudaEvent_t ev_end, const SegLp *seg) {
  int64_t n = g->n;
  if (n == 0) return;
  Buf<int64_t> Wc(n, s);
  launch(k_init_singletons, grid_for(n, 256), 256, 0, s, g->unit_vw ? nullptr : g->vw.get(), n,
                                                       d_cluster, Wc.get());
  TP_LAUNCH_CHECK();
  LpWork w;
  w.init(n, n, s);
  LpState st{d_cluster, Wc.get(), n, U};
  if (seg) {  // labels are vertices: a label's graph and base are its vertex's
    st.seg = *seg;
    st.seg.lgid = seg->gid;
    st.seg.lb = seg->vb;
  }
  prof_scope(level == 0 && !seg);
  if (ev_begin) TP_CUDA(cudaEventRecord(ev_begin, s));
  lp_rounds(g, st, w, p.seed, kTagCluster, (uint64_t)level, 0, p.cluster_rounds, p.sub_rounds, p, s);
  if (ev_end) TP_CUDA(cudaEventRecord(ev_end, s));
  prof_scope(false);
  if (p.two_hop) two_hop(g, d_cluster, Wc.get(), U, p.seed, level, p, s, seg ? &st.seg : nullptr);
  release_hub_tables(g, s);
}

void lp_refine(tp_graph *g, int32_t k, int64_t l_max, const tp_params &p, int32_t level,
               int32_t *d_part, int64_t *d_B, cudaStream_t s, const SegLp *seg) {
  if (g->n == 0) return;
  LpWork w;
  w.init(g->n, k, s);
  LpState st{d_part, d_B, k, l_max};
  if (seg) st.seg = *seg;
  lp_rounds(g, st, w, p.seed, kTagRefine, (uint64_t)level, 0, p.refine_rounds, p.sub_rounds, p, s);
  release_hub_tables(g, s);
}

// ---------------------------------------------------------------- rebalancing
namespace {

__global__ void k_find_over(const int64_t *B, int32_t k, int64_t l_max, int32_t *out) {
  __shared__ int32_t best;
  if (threadIdx.x == 0) best = INT32_MAX;
  __syncthreads();
  for (int32_t b = threadIdx.x; b < k; b += blockDim.x)
    if (B[b] > l_max) atomicMin(&best, b);
  __syncthreads();
  if (threadIdx.x == 0) out[0] = best == INT32_MAX ? -1 : best;
}

__global__ void k_rb_pick(const int32_t *part, int32_t blk, const int32_t *rb_t,
                          const int64_t *rb_loss, const long long *best, int64_t n, int32_t *best_u) {
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n;
       u += (int64_t)gridDim.x * blockDim.x)
    if (part[u] == blk && rb_t[u] >= 0 && rb_loss[u] == *best) atomicMin(best_u, (int32_t)u);
}

__global__ void k_rb_apply(int32_t *part, int64_t *B, const int64_t *vw, const int32_t *rb_t,
                           const int32_t *best_u) {
  int32_t u = *best_u;
  if (u == INT32_MAX) return;
  int32_t t = rb_t[u], b = part[u];
  int64_t w = vw ? vw[u] : 1;
  B[b] -= w;
  B[t] += w;
  part[u] = t;
}

}  // namespace

void rebalance_moves(tp_graph *g, int32_t k, int64_t l_max, int32_t *d_part, int64_t *d_B,
                     int *balanced, const tp_params &p, cudaStream_t s) {
  configure_kernels();
  int64_t n = g->n;
  Buf<int32_t> small(4, s);  // [0] overloaded block [1] best vertex
  Buf<long long> best(1, s);
  Buf<int32_t> rb_t(std::max<int64_t>(n, 1), s);
  Buf<int64_t> rb_loss(std::max<int64_t>(n, 1), s);
  *balanced = 1;
  for (;;) {
    launch(k_find_over, 1, 256, 0, s, d_B, k, l_max, small.get());
    TP_LAUNCH_CHECK();
    int32_t blk = read_scalar(small.get(), s);
    if (blk < 0) return;
    long long init_best = INT64_MAX;
    int32_t init_u = INT32_MAX;
    TP_CUDA(cudaMemcpyAsync(best.get(), &init_best, sizeof(init_best), cudaMemcpyHostToDevice, s));
    TP_CUDA(cudaMemcpyAsync(small.get() + 1, &init_u, sizeof(init_u), cudaMemcpyHostToDevice, s));
    RateCtx c{};
    c.label = d_part;
    c.lw = d_B;
    c.cap = l_max;
    c.blk = blk;
    c.k = k;
    c.rb_loss = rb_loss.get();
    c.rb_t = rb_t.get();
    c.rb_best = best.get();
    rate_tiers<M_REBAL>(g, c, p, s);
    launch(k_rb_pick, grid_for(n, 256), 256, 0, s, d_part, blk, rb_t.get(), rb_loss.get(), best.get(),
                                                 n, small.get() + 1);
    launch(k_rb_apply, 1, 1, 0, s, d_part, d_B, g->unit_vw ? nullptr : g->vw.get(), rb_t.get(),
                               small.get() + 1);
    TP_LAUNCH_CHECK();
    int32_t bu = read_scalar(small.get() + 1, s);
    if (bu == INT32_MAX) {
      *balanced = 0;
      return;
    }
  }
}

namespace {

// Batched rebalancing, step 1 (one block per graph of the union): the
// smallest overloaded block of every graph still rebalancing, or -1; resets
// the graph's best loss and vertex and counts the graphs with one.
__global__ void k_find_over_seg(const int64_t *B, SegLp seg, const int32_t *graphs, int64_t ng,
                                const int32_t *stuck, int32_t *blk_of, long long *best,
                                int32_t *best_u, int32_t *n_over) {
  __shared__ int32_t bmin;
  for (int64_t j = blockIdx.x; j < ng; j += gridDim.x) {
    const int32_t i = graphs[j];
    if (threadIdx.x == 0) bmin = INT32_MAX;
    __syncthreads();
    const int64_t lb = seg.lb[i], cap = seg.cap[i];
    if (!stuck[i])
      for (int32_t b = threadIdx.x; b < seg.k[i]; b += blockDim.x)
        if (B[lb + b] > cap) atomicMin(&bmin, b);
    __syncthreads();
    if (threadIdx.x == 0) {
      const bool over = bmin != INT32_MAX;
      blk_of[i] = over ? (int32_t)(lb + bmin) : -1;
      best[i] = INT64_MAX;
      best_u[i] = INT32_MAX;
      if (over) atomicAdd(n_over, 1);
    }
    __syncthreads();
  }
}

// Step 2: per graph, the smallest vertex among those of least loss.
__global__ void k_rb_pick_seg(const int32_t *part, const int32_t *gid, const int32_t *blk_of,
                              const int32_t *rb_t, const int64_t *rb_loss, const long long *best,
                              int64_t n, int32_t *best_u) {
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n;
       u += (int64_t)gridDim.x * blockDim.x) {
    const int32_t g = gid[u], blk = blk_of[g];
    if (blk >= 0 && part[u] == blk && rb_t[u] >= 0 && rb_loss[u] == best[g])
      atomicMin(&best_u[g], (int32_t)u);
  }
}

// Step 3 (one thread per graph): make the move, or retire a graph without one.
__global__ void k_rb_apply_seg(const int32_t *graphs, int64_t ng, const int32_t *blk_of,
                               const int32_t *best_u, const int32_t *rb_t, const int64_t *vw,
                               int32_t *part, int64_t *B, int32_t *stuck) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < ng;
       j += (int64_t)gridDim.x * blockDim.x) {
    const int32_t i = graphs[j];
    if (blk_of[i] < 0) continue;
    const int32_t u = best_u[i];
    if (u == INT32_MAX) {
      stuck[i] = 1;
      continue;
    }
    const int32_t t = rb_t[u], b = part[u];
    const int64_t w = vw ? vw[u] : 1;
    B[b] -= w;
    B[t] += w;
    part[u] = t;
  }
}

}  // namespace

void rebalance_moves_seg(tp_graph *g, const SegLp &seg, const int32_t *d_graphs, int64_t ng,
                         int32_t *d_part, int64_t *d_B, const tp_params &p, cudaStream_t s) {
  configure_kernels();
  const int64_t n = g->n, G = seg.ngraphs;
  if (n == 0 || ng == 0) return;
  Buf<int32_t> blk_of(G, s), best_u(G, s), stuck(G, s), n_over(1, s);
  Buf<long long> best(G, s);
  Buf<int32_t> rb_t(n, s);
  Buf<int64_t> rb_loss(n, s);
  TP_CUDA(cudaMemsetAsync(stuck.get(), 0, G * sizeof(int32_t), s));
  const unsigned gb = (unsigned)std::min<int64_t>(ng, (int64_t)num_sms() * 8);
  for (;;) {
    TP_CUDA(cudaMemsetAsync(n_over.get(), 0, sizeof(int32_t), s));
    launch(k_find_over_seg, gb, 128, 0, s, d_B, seg, d_graphs, ng, stuck.get(), blk_of.get(),
           best.get(), best_u.get(), n_over.get());
    TP_LAUNCH_CHECK();
    if (read_scalar(n_over.get(), s) == 0) return;
    RateCtx c{};
    c.label = d_part;
    c.lw = d_B;
    c.seg = seg;
    c.blk_of = blk_of.get();
    c.rb_loss = rb_loss.get();
    c.rb_t = rb_t.get();
    c.rb_best = best.get();
    rate_tiers<M_REBAL>(g, c, p, s);
    launch(k_rb_pick_seg, grid_for(n, 256), 256, 0, s, d_part, seg.gid, blk_of.get(), rb_t.get(),
           rb_loss.get(), best.get(), n, best_u.get());
    launch(k_rb_apply_seg, grid_for(ng, 256), 256, 0, s, d_graphs, ng, blk_of.get(), best_u.get(),
           rb_t.get(), g->unit_vw ? nullptr : g->vw.get(), d_part, d_B, stuck.get());
    TP_LAUNCH_CHECK();
  }
}

}  // namespace tp
