// Initial partitioning of the coarsest graph by recursive bisection (the
// paper's KaMinPar uses a portfolio of greedy graph growing and 2-way FM,
// Section "KaMinPar"). Deterministic GPU form: every node of the bisection
// tree owns the blocks [offset, offset + kk); its vertices are bisected with
// kk0 = ceil(kk/2) and kk1 = floor(kk/2) blocks per side by T seeded attempts,
// one CTA each:
//   1. BFS from a hashed seed vertex (FIFO order, neighbours in ascending id,
//      unreached vertices appended in ascending id), computed level by level:
//      a vertex joins the next frontier behind the earliest frontier vertex
//      adjacent to it;
//   2. side 0 = the longest prefix of that order weighing at most
//      floor(W_sub * kk0 / kk);
//   3. refine_rounds rounds of 2-way label propagation with side caps
//      kk0 * L_max and kk1 * L_max and the same prefix approval as k-way LP;
//   4. the cut of the induced subgraph.
// The attempt with the smallest cut (lowest attempt on ties) wins; the tree
// is processed depth by depth, all nodes of a depth in one launch. Batched
// graphs form a forest: every graph's root carries the hash key offset and
// L_max its graph would use alone, so each tree's result is that graph's.
#include <algorithm>
#include <vector>

#include "tp_internal.cuh"

namespace tp {

namespace {

// Threads per attempt: 1024 for large nodes or few attempts in flight,
// 512, 256 or 128 when many smaller nodes share the GPU (several CTAs per SM).
constexpr int kIPThreads = 1024;

struct IPCtx {
  int64_t n;
  const int64_t *xadj;
  const int32_t *adj;
  const int64_t *vw, *ew;  // null: unit
  const int32_t *node_of;  // node index per vertex (-1: done)
  const int32_t *vlist;    // vertices sorted by (node, id)
  const int64_t *nstart;   // node start in vlist
  const int32_t *loc;      // position of a vertex inside its node
  // the subgraph induced by every node, in local positions: vertex vlist[p]
  // has neighbours ladj[lxadj[p] .. lxadj[p + 1]) (ascending, as in the graph)
  const int64_t *lxadj;
  const int32_t *ladj;
  const int64_t *lew;  // null: unit
  const int32_t *noff, *nkk;
  const int32_t *nkey;    // per node: the block offset its graph alone would give it (hash key)
  const int64_t *nlmax;  // per node: its graph's L_max
  int32_t T;
  uint64_t seed;
  int32_t rounds, S;
  // scratch, T * n entries each
  int32_t *ord, *disc, *claimer, *cnt, *side, *mvx0, *mvx1, *ok0, *ok1;
  int64_t *mvg0, *mvg1;
  uint8_t *sub;  // sub-round of every vertex in the current 2-way LP round
  int64_t *cut;  // nodes * T
};

template <int NT>
__device__ __forceinline__ int64_t bscan_excl(int64_t v, int64_t &total) {
  constexpr int NW = NT / 32;
  __shared__ int64_t ws[NW];
  int l = lane_id(), w = threadIdx.x >> 5;
  int64_t incl = warp_incl_scan(v);
  if (l == 31) ws[w] = incl;
  __syncthreads();
  if (w == 0) {
    int64_t x = l < NW ? ws[l] : 0;
    x = warp_incl_scan(x);
    if (l < NW) ws[l] = x;
  }
  __syncthreads();
  int64_t off = w > 0 ? ws[w - 1] : 0;
  total = ws[NW - 1];
  __syncthreads();
  return off + incl - v;
}

template <int NT>
__device__ __forceinline__ int64_t bsum(int64_t v) {
  int64_t t;
  bscan_excl<NT>(v, t);
  return t;
}

// Weighted radix select (same contract as in lp.cu): first key in ascending
// (hi, lo) order whose inclusive weight prefix exceeds rem.
// Called only when the keys' total weight exceeds rem, so every pass selects
// a byte some remaining key carries: bytes on which all keys agree are taken
// without a histogram pass.
template <class Item>
__device__ void ip_select(int64_t cnt, int64_t rem, Item item, uint64_t &khi, uint32_t &klo) {
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
  {
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
    if (same == 0) {
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
      if (in_hi) fhi |= (uint64_t)b << shift, mhi |= 255ull << shift;
      else flo |= (uint32_t)b << shift, mlo |= 255u << shift;
    }
    __syncthreads();
  }
  khi = fhi;
  klo = flo;
  __syncthreads();
}

// Adjacency of a node's vertex (vlist position p) in the node's induced
// subgraph is scanned by a whole warp, lanes striding over the neighbours
// (coalesced, and a hub does not serialise one thread); f(in, y, w) is called
// by every lane for every 32 neighbours, y a position inside the node.
template <class F>
__device__ __forceinline__ void node_nbrs(const IPCtx &c, int64_t p, F &&f) {
  const int64_t b = c.lxadj[p], e = c.lxadj[p + 1];
  for (int64_t i0 = b; i0 < e; i0 += 32) {
    const int64_t i = i0 + lane_id();
    const bool in = i < e;
    f(in, in ? c.ladj[i] : 0, in ? (c.lew ? c.lew[i] : (int64_t)1) : (int64_t)0);
  }
}

// Induced subgraphs of all nodes of a depth: neighbour counts, then (after a
// scan into lxadj) the neighbours' positions, one warp per listed vertex.
__global__ void k_local_deg(const int64_t *xadj, const int32_t *adj, const int32_t *node_of,
                            const int32_t *vlist, int64_t m, int64_t *ldeg) {
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t p = gw; p < m; p += nw) {
    const int32_t u = vlist[p], j = node_of[u];
    int64_t k = 0;
    for (int64_t i = xadj[u] + lane_id(); i < xadj[u + 1]; i += 32) k += node_of[adj[i]] == j;
    k = warp_sum(k);
    if (lane_id() == 0) ldeg[p] = k;
  }
}

__global__ void k_local_fill(const int64_t *xadj, const int32_t *adj, const int64_t *ew,
                             const int32_t *node_of, const int32_t *loc, const int32_t *vlist,
                             int64_t m, const int64_t *lxadj, int32_t *ladj, int64_t *lew) {
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t p = gw; p < m; p += nw) {
    const int32_t u = vlist[p], j = node_of[u];
    int64_t pos = lxadj[p];
    const int64_t b = xadj[u], e = xadj[u + 1];
    for (int64_t i0 = b; i0 < e; i0 += 32) {
      const int64_t i = i0 + lane_id();
      int32_t v = 0;
      const bool in = i < e && node_of[v = adj[i]] == j;
      const unsigned msk = __ballot_sync(kFull, in);
      if (in) {
        const int64_t at = pos + __popc(msk & lanemask_lt());
        ladj[at] = loc[v];
        if (lew) lew[at] = ew[i];
      }
      pos += __popc(msk);
    }
  }
}

// Exclusive scan of x[0..len) in place, block-wide; returns the total.
template <int NT>
__device__ int64_t block_scan_array(int32_t *x, int64_t len) {
  int64_t carry = 0;
  for (int64_t q0 = 0; q0 < len; q0 += blockDim.x) {
    const int64_t q = q0 + threadIdx.x;
    const int64_t v = q < len ? x[q] : 0;
    int64_t tot;
    const int64_t ex = bscan_excl<NT>(v, tot);
    if (q < len) x[q] = (int32_t)(carry + ex);
    carry += tot;
  }
  __syncthreads();
  return carry;
}

template <int NT>
__global__ void __launch_bounds__(NT, kIPThreads / NT) k_bisect(IPCtx c) {
  const int32_t j = blockIdx.x / c.T, a = blockIdx.x % c.T;
  const int64_t nb = c.nstart[j], ns = c.nstart[j + 1] - nb;
  const int64_t R = (int64_t)a * c.n + nb;  // scratch region of this attempt
  int32_t *ord = c.ord + R, *disc = c.disc + R, *claimer = c.claimer + R, *cnt = c.cnt + R;
  int32_t *side = c.side + R, *mvx0 = c.mvx0 + R, *mvx1 = c.mvx1 + R, *ok0 = c.ok0 + R,
          *ok1 = c.ok1 + R;
  int64_t *mvg0 = c.mvg0 + R, *mvg1 = c.mvg1 + R;
  uint8_t *sub = c.sub + R;
  const int32_t *vs = c.vlist + nb;
  const int32_t kk = c.nkk[j], k0 = (kk + 1) / 2, k1 = kk / 2;
  const uint64_t key = ((uint64_t)(uint32_t)c.nkey[j] << 32) | (uint32_t)kk;
  const int lane = lane_id(), warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  auto cw = [&](int64_t x) -> int64_t { return c.vw ? c.vw[vs[x]] : 1; };
  if (ns == 0) {
    if (threadIdx.x == 0) c.cut[blockIdx.x] = 0;
    return;
  }
  // ---------------- BFS order
  for (int64_t x = threadIdx.x; x < ns; x += blockDim.x) disc[x] = 0, claimer[x] = INT32_MAX;
  __syncthreads();
  __shared__ int64_t sh_fb, sh_fe, sh_tail;
  if (threadIdx.x == 0) {
    int64_t s0 = (int64_t)(round_key(c.seed, kTagIPSeed, key, (uint64_t)a) % (uint64_t)ns);
    ord[0] = (int32_t)s0;
    disc[s0] = 1;
    sh_fb = 0, sh_fe = 1, sh_tail = 1;
  }
  __syncthreads();
  for (;;) {
    const int64_t fb = sh_fb, fe = sh_fe, tail = sh_tail;
    if (fb >= fe) break;
    // every undiscovered neighbour is claimed by its earliest frontier vertex
    for (int64_t i = fb + warp; i < fe; i += nwarps)
      node_nbrs(c, nb + ord[i], [&](bool in, int32_t y, int64_t) {
        if (in && !disc[y]) atomicMin(&claimer[y], (int32_t)i);
      });
    __syncthreads();
    for (int64_t i = fb + warp; i < fe; i += nwarps) {
      int32_t k = 0;
      node_nbrs(c, nb + ord[i], [&](bool in, int32_t y, int64_t) {
        k += __popc(__ballot_sync(kFull, in && !disc[y] && claimer[y] == i));
      });
      if (lane == 0) cnt[i - fb] = k;
    }
    __syncthreads();
    const int64_t carry = block_scan_array<NT>(cnt, fe - fb);
    // claimed neighbours in frontier order, then adjacency order
    for (int64_t i = fb + warp; i < fe; i += nwarps) {
      int64_t pos = tail + cnt[i - fb];
      node_nbrs(c, nb + ord[i], [&](bool in, int32_t y, int64_t) {
        const bool mine = in && !disc[y] && claimer[y] == i;
        const unsigned m = __ballot_sync(kFull, mine);
        if (mine) ord[pos + __popc(m & lanemask_lt())] = y;
        pos += __popc(m);
      });
    }
    __syncthreads();
    for (int64_t q = tail + threadIdx.x; q < tail + carry; q += blockDim.x) disc[ord[q]] = 1;
    __syncthreads();
    if (threadIdx.x == 0) sh_fb = tail, sh_fe = tail + carry, sh_tail = tail + carry;
    __syncthreads();
  }
  {  // append unreached vertices in ascending id
    int64_t carry = 0, tail = sh_tail;
    for (int64_t x0 = 0; x0 < ns; x0 += blockDim.x) {
      int64_t x = x0 + threadIdx.x;
      int64_t f = x < ns && !disc[x];
      int64_t tot;
      int64_t ex = bscan_excl<NT>(f, tot);
      if (f) ord[tail + carry + ex] = (int32_t)x;
      carry += tot;
    }
    __syncthreads();
  }
  // ---------------- greedy growing: longest prefix within target0
  __shared__ int64_t lw[2], inw[2], ncnt[2];
  __shared__ int64_t sh_nact;
  int64_t W = 0;
  for (int64_t x = threadIdx.x; x < ns; x += blockDim.x) W += cw(x);
  W = bsum<NT>(W);
  const int64_t target0 = (int64_t)(((__int128)W * k0) / kk);
  const int64_t caps[2] = {(int64_t)k0 * c.nlmax[j], (int64_t)k1 * c.nlmax[j]};
  {
    int64_t carry = 0, w0 = 0;
    for (int64_t q0 = 0; q0 < ns; q0 += blockDim.x) {
      int64_t q = q0 + threadIdx.x;
      int64_t w = q < ns ? cw(ord[q]) : 0;
      int64_t tot;
      int64_t incl = carry + bscan_excl<NT>(w, tot) + w;
      if (q < ns) {
        bool in0 = incl <= target0;
        side[ord[q]] = in0 ? 0 : 1;
        if (in0) w0 += w;
      }
      carry += tot;
    }
    w0 = bsum<NT>(w0);
    if (threadIdx.x == 0) lw[0] = w0, lw[1] = W - w0;
    __syncthreads();
  }
  // ---------------- 2-way label propagation
  for (int32_t r = 0; r < c.rounds; ++r) {
    const uint64_t rk = round_key(c.seed, kTagIPLP, key, ((uint64_t)a << 8) + (uint64_t)r);
    for (int64_t x = threadIdx.x; x < ns; x += blockDim.x)
      sub[x] = (uint8_t)sub_round_of(hstep(rk, (uint64_t)x), c.S);
    __syncthreads();
    for (int32_t s = 0; s < c.S; ++s) {
      // this sub-round's vertices, listed in cnt (ascending)
      {
        int64_t carry = 0;
        for (int64_t x0 = 0; x0 < ns; x0 += blockDim.x) {
          const int64_t x = x0 + threadIdx.x;
          const int64_t f = x < ns && sub[x] == s;
          int64_t tot;
          const int64_t ex = bscan_excl<NT>(f, tot);
          if (f) cnt[carry + ex] = (int32_t)x;
          carry += tot;
        }
        if (threadIdx.x == 0) sh_nact = carry, inw[0] = inw[1] = 0, ncnt[0] = ncnt[1] = 0;
        __syncthreads();
      }
      const int64_t nact = sh_nact;
      for (int64_t q = warp; q < nact; q += nwarps) {
        const int32_t x = cnt[q];
        int64_t r0 = 0, r1 = 0;
        node_nbrs(c, nb + x, [&](bool in, int32_t y, int64_t w) {
          if (in) (side[y] ? r1 : r0) += w;
        });
        r0 = warp_sum(r0);
        r1 = warp_sum(r1);
        if (lane != 0) continue;
        const int32_t own = side[x], oth = 1 - own;
        const int64_t Rown = own ? r1 : r0, Roth = own ? r0 : r1;
        const int64_t w = cw(x);
        if (Roth > Rown && lw[oth] + w <= caps[oth]) {
          const int64_t g = Roth - Rown;
          unsigned long long p = atomicAdd((unsigned long long *)&ncnt[oth], 1ull);
          atomicAdd((unsigned long long *)&inw[oth], (unsigned long long)w);
          if (oth == 0) mvx0[p] = x, mvg0[p] = g, ok0[p] = 0;
          else mvx1[p] = x, mvg1[p] = g, ok1[p] = 0;
        }
      }
      __syncthreads();
      for (int t = 0; t < 2; ++t) {
        int32_t *mx = t == 0 ? mvx0 : mvx1, *ok = t == 0 ? ok0 : ok1;
        int64_t *mg = t == 0 ? mvg0 : mvg1;
        int64_t m = ncnt[t];
        if (lw[t] + inw[t] <= caps[t]) {
          for (int64_t q = threadIdx.x; q < m; q += blockDim.x) ok[q] = 1;
        } else if (caps[t] - lw[t] >= 0) {
          auto item = [&](int64_t q, uint64_t &hi, uint32_t &lo, int64_t &w) {
            hi = ~(uint64_t)mg[q];
            lo = (uint32_t)mx[q];
            w = cw(mx[q]);
          };
          uint64_t khi;
          uint32_t klo;
          ip_select(m, caps[t] - lw[t], item, khi, klo);
          for (int64_t q = threadIdx.x; q < m; q += blockDim.x) {
            uint64_t hi = ~(uint64_t)mg[q];
            uint32_t lo = (uint32_t)mx[q];
            ok[q] = hi < khi || (hi == khi && lo < klo);
          }
        }
        __syncthreads();
      }
      for (int t = 0; t < 2; ++t) {
        int32_t *mx = t == 0 ? mvx0 : mvx1, *ok = t == 0 ? ok0 : ok1;
        for (int64_t q = threadIdx.x; q < ncnt[t]; q += blockDim.x) {
          if (!ok[q]) continue;
          int64_t w = cw(mx[q]);
          side[mx[q]] = t;
          atomicAdd((unsigned long long *)&lw[t], (unsigned long long)w);
          atomicAdd((unsigned long long *)&lw[1 - t], (unsigned long long)(-w));
        }
      }
      __syncthreads();
    }
  }
  // ---------------- cut of the induced subgraph
  int64_t cutv = 0;
  for (int64_t x = warp; x < ns; x += nwarps) {
    const int32_t sx = side[x];
    node_nbrs(c, nb + x, [&](bool in, int32_t y, int64_t w) {
      if (in && side[y] != sx) cutv += w;
    });
  }
  cutv = bsum<NT>(cutv);
  if (threadIdx.x == 0) c.cut[blockIdx.x] = cutv / 2;
}

// Pick the winning attempt of every node and move its vertices on.
__global__ void k_pick(IPCtx c, const int32_t *child0, const int32_t *child1, int32_t *next_node,
                       int32_t *part) {
  const int32_t j = blockIdx.x;
  __shared__ int32_t best;
  if (threadIdx.x == 0) {
    int32_t b = 0;
    for (int32_t a = 1; a < c.T; ++a)
      if (c.cut[j * c.T + a] < c.cut[j * c.T + b]) b = a;
    best = b;
  }
  __syncthreads();
  const int64_t nb = c.nstart[j], ns = c.nstart[j + 1] - nb;
  const int32_t kk = c.nkk[j], k0 = (kk + 1) / 2;
  for (int64_t x = threadIdx.x; x < ns; x += blockDim.x) {
    int32_t u = c.vlist[nb + x];
    int32_t sd = c.side[(int64_t)best * c.n + nb + x];
    int32_t ch = sd == 0 ? child0[j] : child1[j];
    next_node[u] = ch;
    if (ch < 0) part[u] = sd == 0 ? c.noff[j] : c.noff[j] + k0;
  }
}

__global__ void k_node_keys(const int32_t *node_of, int64_t n, uint64_t *keys, int64_t *count) {
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n;
       u += (int64_t)gridDim.x * blockDim.x) {
    int32_t nd = node_of[u];
    keys[u] = nd < 0 ? ~0ull : ((uint64_t)nd << 32) | (uint64_t)u;
    if (nd >= 0) atomicAdd((unsigned long long *)&count[nd], 1ull);
  }
}

__global__ void k_node_lists(const uint64_t *keys, const int64_t *nstart, int64_t m, int32_t *vlist,
                             int32_t *loc) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t k = keys[i];
    int32_t u = (int32_t)(k & 0xffffffffu), nd = (int32_t)(k >> 32);
    vlist[i] = u;
    loc[u] = (int32_t)(i - nstart[nd]);
  }
}

__global__ void k_fill_i32(int32_t *p, int64_t n, int32_t v) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = v;
}

}  // namespace

void initial_partition(const tp_graph *g, int32_t k, int64_t l_max, const tp_params &p,
                       int32_t *d_part, cudaStream_t s) {
  TP_REQUIRE(!g->compressed, TP_ERR_INVALID);
  const int64_t n = g->n;
  if (n == 0) return;
  if (k <= 1) {
    launch(k_fill_i32, grid_for(n, 256), 256, 0, s, d_part, n, 0);
    TP_LAUNCH_CHECK();
    return;
  }
  initial_partition_roots(g, {IPRoot{0, 0, k, l_max}}, nullptr, p, d_part, s);
}

void initial_partition_roots(const tp_graph *g, const std::vector<IPRoot> &roots,
                             const int32_t *d_node_of, const tp_params &p, int32_t *d_part,
                             cudaStream_t s) {
  TP_REQUIRE(!g->compressed, TP_ERR_INVALID);
  const int64_t n = g->n;
  if (n == 0 || roots.empty()) return;
  launch(k_fill_i32, grid_for(n, 256), 256, 0, s, d_part, n, 0);
  TP_LAUNCH_CHECK();
  const int32_t T = std::max(1, p.ip_attempts);
  Buf<int32_t> node_of(n, s), next_node(n, s), vlist(n, s), loc(n, s);
  if (d_node_of)
    TP_CUDA(cudaMemcpyAsync(node_of.get(), d_node_of, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
  else
    launch(k_fill_i32, grid_for(n, 256), 256, 0, s, node_of.get(), n, 0);
  Buf<int32_t> ord(T * n, s), disc(T * n, s), claimer(T * n, s), cnt(T * n, s), side(T * n, s),
      mvx0(T * n, s), mvx1(T * n, s), ok0(T * n, s), ok1(T * n, s);
  Buf<int64_t> mvg0(T * n, s), mvg1(T * n, s);
  Buf<uint8_t> sub(T * n, s);
  Buf<uint64_t> keys(n, s);
  std::vector<int32_t> off, kks, hkey;
  std::vector<int64_t> lmx;
  for (const IPRoot &r : roots) {
    TP_REQUIRE(r.k >= 2, TP_ERR_INVALID);
    off.push_back(r.off), kks.push_back(r.k), hkey.push_back(r.key), lmx.push_back(r.l_max);
  }
  while (!off.empty()) {
    const int32_t nodes = (int32_t)off.size();
    // vertex lists per node
    Buf<int64_t> nstart(nodes + 1, s);
    TP_CUDA(cudaMemsetAsync(nstart.get(), 0, (nodes + 1) * sizeof(int64_t), s));
    launch(k_node_keys, grid_for(n, 256), 256, 0, s, node_of.get(), n, keys.get(), nstart.get());
    TP_LAUNCH_CHECK();
    radix_sort_pairs(keys.get(), nullptr, n, 64, s);
    exclusive_scan_i64(nstart.get(), nstart.get(), nodes, s);
    std::vector<int64_t> hstart((size_t)nodes + 1);
    TP_CUDA(cudaMemcpyAsync(hstart.data(), nstart.get(), (nodes + 1) * sizeof(int64_t),
                            cudaMemcpyDeviceToHost, s));
    TP_CUDA(cudaStreamSynchronize(s));
    const int64_t m = hstart[(size_t)nodes];
    int64_t max_ns = 0;
    for (int32_t jn = 0; jn < nodes; ++jn) max_ns = std::max(max_ns, hstart[jn + 1] - hstart[jn]);
    if (m) {
      launch(k_node_lists, grid_for(m, 256), 256, 0, s, keys.get(), nstart.get(), m, vlist.get(), loc.get());
      TP_LAUNCH_CHECK();
    }
    // induced subgraph of every node in local positions
    const bool weighted = !g->unit_ew;
    Buf<int64_t> lxadj(m + 1, s);
    Buf<int32_t> ladj;
    Buf<int64_t> lew;
    if (m) {
      const unsigned wg = grid_for(m * 32, 256);
      launch(k_local_deg, wg, 256, 0, s, g->xadj.get(), g->adj.get(), node_of.get(), vlist.get(), m,
             lxadj.get());
      TP_LAUNCH_CHECK();
      exclusive_scan_i64(lxadj.get(), lxadj.get(), m, s);
      const int64_t lm = read_scalar(lxadj.get() + m, s);
      ladj.alloc(std::max<int64_t>(lm, 1), s);
      if (weighted) lew.alloc(std::max<int64_t>(lm, 1), s);
      launch(k_local_fill, wg, 256, 0, s, g->xadj.get(), g->adj.get(),
             weighted ? g->ew.get() : nullptr, node_of.get(), loc.get(), vlist.get(), m, lxadj.get(),
             ladj.get(), weighted ? lew.get() : nullptr);
      TP_LAUNCH_CHECK();
    }
    // children of every node at the next depth (-1: leaf, assign the block)
    std::vector<int32_t> c0(nodes), c1(nodes), noff, nkk, nkey;
    std::vector<int64_t> nlmx;
    for (int32_t jn = 0; jn < nodes; ++jn) {
      int32_t k0 = (kks[jn] + 1) / 2, k1 = kks[jn] / 2;
      c0[jn] = -1, c1[jn] = -1;
      if (k0 >= 2) {
        c0[jn] = (int32_t)noff.size();
        noff.push_back(off[jn]), nkk.push_back(k0), nkey.push_back(hkey[jn]), nlmx.push_back(lmx[jn]);
      }
      if (k1 >= 2) {
        c1[jn] = (int32_t)noff.size();
        noff.push_back(off[jn] + k0), nkk.push_back(k1), nkey.push_back(hkey[jn] + k0);
        nlmx.push_back(lmx[jn]);
      }
    }
    // one upload of the node table: off, kk, key, child0, child1 (int32), l_max
    std::vector<int32_t> tbl32((size_t)5 * nodes);
    for (int32_t jn = 0; jn < nodes; ++jn) {
      tbl32[jn] = off[jn], tbl32[nodes + jn] = kks[jn], tbl32[2 * nodes + jn] = hkey[jn];
      tbl32[3 * nodes + jn] = c0[jn], tbl32[4 * nodes + jn] = c1[jn];
    }
    Buf<int32_t> d_tbl(5 * nodes, s);
    Buf<int64_t> d_lmax(nodes, s);
    TP_CUDA(cudaMemcpyAsync(d_tbl.get(), tbl32.data(), tbl32.size() * 4, cudaMemcpyHostToDevice, s));
    TP_CUDA(cudaMemcpyAsync(d_lmax.get(), lmx.data(), nodes * 8, cudaMemcpyHostToDevice, s));
    const int32_t *d_off = d_tbl.get(), *d_kk = d_tbl.get() + nodes, *d_key = d_tbl.get() + 2 * nodes;
    const int32_t *d_c0 = d_tbl.get() + 3 * nodes, *d_c1 = d_tbl.get() + 4 * nodes;
    Buf<int64_t> cut((int64_t)nodes * T, s);
    IPCtx c;
    c.n = n;
    c.xadj = g->xadj.get();
    c.adj = g->adj.get();
    c.vw = g->unit_vw ? nullptr : g->vw.get();
    c.ew = g->unit_ew ? nullptr : g->ew.get();
    c.node_of = node_of.get();
    c.vlist = vlist.get();
    c.nstart = nstart.get();
    c.loc = loc.get();
    c.lxadj = lxadj.get();
    c.ladj = ladj.get();
    c.lew = weighted ? lew.get() : nullptr;
    c.noff = d_off;
    c.nkk = d_kk;
    c.nkey = d_key;
    c.nlmax = d_lmax.get();
    c.T = T;
    c.seed = p.seed;
    c.rounds = p.refine_rounds;
    c.S = p.sub_rounds;
    c.ord = ord.get(), c.disc = disc.get(), c.claimer = claimer.get(), c.cnt = cnt.get();
    c.side = side.get(), c.mvx0 = mvx0.get(), c.mvx1 = mvx1.get(), c.ok0 = ok0.get(),
    c.ok1 = ok1.get();
    c.mvg0 = mvg0.get(), c.mvg1 = mvg1.get();
    c.sub = sub.get();
    c.cut = cut.get();
    // small nodes with enough attempts in flight: smaller CTAs, several per SM
    const int64_t ctas = (int64_t)nodes * T;
    const bool many = ctas >= 4LL * num_sms();
    if (many && max_ns <= 512) launch(k_bisect<128>, (unsigned)ctas, 128, 0, s, c);
    else if (many && max_ns <= 4096) launch(k_bisect<256>, (unsigned)ctas, 256, 0, s, c);
    else if (many && max_ns <= 16384) launch(k_bisect<512>, (unsigned)ctas, 512, 0, s, c);
    else launch(k_bisect<kIPThreads>, (unsigned)ctas, kIPThreads, 0, s, c);
    TP_LAUNCH_CHECK();
    launch(k_fill_i32, grid_for(n, 256), 256, 0, s, next_node.get(), n, -1);
    launch(k_pick, (unsigned)nodes, 256, 0, s, c, d_c0, d_c1, next_node.get(), d_part);
    TP_LAUNCH_CHECK();
    std::swap(node_of, next_node);
    TP_CUDA(cudaStreamSynchronize(s));  // host vectors above outlive their copies
    off.swap(noff);
    kks.swap(nkk);
    hkey.swap(nkey);
    lmx.swap(nlmx);
  }
}

}  // namespace tp
