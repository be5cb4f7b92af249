/*
 * Size-constrained label propagation, made synchronous and deterministic.
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Paper, Algorithm 1 and Section "Label Propagation Clustering": every vertex
 * u sums the edge weights towards each neighbouring cluster in a rating map,
 * R[C[v]] += w(u,v) for v in N(u), and joins the cluster with the largest
 * rating; five rounds are run per level; the clustering is size-constrained
 * (Section "KaMinPar": size-constrained label propagation for refinement, and
 * a cluster weight cap for coarsening).
 *
 * Readings where the paper is silent (they are the algorithm the GPU path must
 * reproduce bit for bit):
 *  - Synchrony: a round is S sub-rounds; vertex u is active in sub-round
 *    hash(u) mod S and rates against the state at the start of the sub-round.
 *  - A vertex only considers clusters x != own with R[x] > 0 whose weight
 *    still admits it, lw[x] + c(u) <= cap(x).
 *  - Strict improvement: u moves only if the best admissible rating exceeds
 *    R[own] (R[own] may be 0).
 *  - Ties: larger rating first, then the smaller 32-bit tie hash of (u, x),
 *    then the smaller label x.
 *  - Approval: per target t, if lw[t] + (sum of mover weights) <= cap(t) all
 *    movers are approved; otherwise the movers are ordered by gain descending,
 *    vertex id ascending, and exactly those whose inclusive weight prefix p
 *    satisfies lw[t] + p <= cap(t) are approved. Departures from t in the same
 *    sub-round are not credited.
 *  - Two-hop packing (Section "KaMinPar": two-hop matching ensures coarsening
 *    progress on irregular graphs): see orc_two_hop.
 */
#include "oracle.h"
#include <stdlib.h>
#include <string.h>

static uint32_t tie_hash(uint64_t hv, int64_t x) {
  return (uint32_t)(orc_step(hv, (uint64_t)x) >> 32);
}

/* 1 iff candidate (ra, ta, xa) precedes (rb, tb, xb) in the rating order. */
static int better(int64_t ra, uint32_t ta, int64_t xa, int64_t rb, uint32_t tb, int64_t xb) {
  if (ra != rb) return ra > rb;
  if (ta != tb) return ta < tb;
  return xa < xb;
}

static int64_t cap_of(int64_t cap_uniform, const int64_t *cap, int64_t x) {
  return cap ? cap[x] : cap_uniform;
}

/* Rating map as a plain dense array R over all labels plus the list of
 * touched labels (the "sparse array" of the paper). */
typedef struct {
  int64_t *R;
  int32_t *touched;
} rating_map;

static int rate_with(const orc_graph *g, int64_t u, const int32_t *label, const int64_t *lw,
                     int64_t cap_uniform, const int64_t *cap, int ignore_cap, uint64_t hv,
                     rating_map *rm, int32_t *target, int64_t *gain) {
  int64_t nt = 0;
  int32_t own = label[u];
  for (int64_t e = g->xadj[u]; e < g->xadj[u + 1]; ++e) {
    int32_t x = label[g->adj[e]];
    if (rm->R[x] == 0) rm->touched[nt++] = x;
    rm->R[x] += orc_ew(g, e);
  }
  int64_t r_own = rm->R[own];
  int64_t best = -1, best_r = 0;
  uint32_t best_t = 0;
  for (int64_t i = 0; i < nt; ++i) {
    int32_t x = rm->touched[i];
    if (x == own) continue;
    if (!ignore_cap && lw[x] + orc_vw(g, u) > cap_of(cap_uniform, cap, x)) continue;
    uint32_t t = tie_hash(hv, x);
    if (best < 0 || better(rm->R[x], t, x, best_r, best_t, best)) {
      best = x;
      best_r = rm->R[x];
      best_t = t;
    }
  }
  for (int64_t i = 0; i < nt; ++i) rm->R[rm->touched[i]] = 0;
  if (best < 0 || best_r <= r_own) return 0;
  *target = (int32_t)best;
  *gain = best_r - r_own;
  return 1;
}

static int max_label_bound(const orc_graph *g, const int32_t *label, int64_t *nl) {
  int64_t m = 0;
  for (int64_t u = 0; u < g->n; ++u)
    if (label[u] + 1 > m) m = label[u] + 1;
  *nl = m;
  return 0;
}

int orc_rate_vertex(const orc_graph *g, int64_t u, const int32_t *label, const int64_t *lw,
                    int64_t cap_uniform, const int64_t *cap, int ignore_cap, uint64_t hv,
                    int32_t *target, int64_t *gain) {
  int64_t nl;
  max_label_bound(g, label, &nl);
  rating_map rm;
  rm.R = (int64_t *)calloc((size_t)(nl + 1), sizeof(int64_t));
  rm.touched = (int32_t *)malloc(sizeof(int32_t) * (size_t)(g->xadj[u + 1] - g->xadj[u] + 1));
  int r = rate_with(g, u, label, lw, cap_uniform, cap, ignore_cap, hv, &rm, target, gain);
  free(rm.R);
  free(rm.touched);
  return r;
}

typedef struct {
  int32_t x;
  int64_t w;
} label_weight;

static int cmp_label_weight(const void *pa, const void *pb) {
  const label_weight *a = (const label_weight *)pa, *b = (const label_weight *)pb;
  return a->x < b->x ? -1 : (a->x > b->x);
}

/* The same decision as orc_rate_vertex, with the ratings formed by sorting
 * the (label, weight) pairs of N(u) and summing runs of equal labels, so a
 * single vertex costs O(deg log deg) on graphs of any size. Null vw / ew
 * arrays mean unit weights (large graphs need not carry arrays of ones). */
int orc_rate_vertex_sorted(const orc_graph *g, int64_t u, const int32_t *label, const int64_t *lw,
                           int64_t cap_uniform, const int64_t *cap, int ignore_cap, uint64_t hv,
                           int32_t *target, int64_t *gain) {
  int64_t d = g->xadj[u + 1] - g->xadj[u];
  label_weight *p = (label_weight *)malloc(sizeof(label_weight) * (size_t)(d + 1));
  for (int64_t i = 0; i < d; ++i) {
    p[i].x = label[g->adj[g->xadj[u] + i]];
    p[i].w = orc_ew(g, g->xadj[u] + i);
  }
  qsort(p, (size_t)d, sizeof(label_weight), cmp_label_weight);
  int32_t own = label[u];
  int64_t r_own = 0, best = -1, best_r = 0;
  uint32_t best_t = 0;
  for (int64_t i = 0; i < d;) {
    int64_t j = i, r = 0;
    while (j < d && p[j].x == p[i].x) r += p[j++].w;
    int32_t x = p[i].x;
    i = j;
    if (x == own) {
      r_own = r;
      continue;
    }
    if (!ignore_cap && lw[x] + orc_vw(g, u) > cap_of(cap_uniform, cap, x)) continue;
    uint32_t t = tie_hash(hv, x);
    if (best < 0 || better(r, t, x, best_r, best_t, best)) {
      best = x;
      best_r = r;
      best_t = t;
    }
  }
  free(p);
  if (best < 0 || best_r <= r_own) return 0;
  *target = (int32_t)best;
  *gain = best_r - r_own;
  return 1;
}

typedef struct {
  int64_t u;
  int64_t gain;
  int64_t w;
  int32_t t;
  int32_t approved;
} mover;

static int cmp_mover(const void *pa, const void *pb) {
  const mover *a = (const mover *)pa, *b = (const mover *)pb;
  if (a->t != b->t) return a->t < b->t ? -1 : 1;
  if (a->gain != b->gain) return a->gain > b->gain ? -1 : 1;
  if (a->u != b->u) return a->u < b->u ? -1 : 1;
  return 0;
}

static int64_t subround_with(const orc_graph *g, int32_t *label, int64_t *lw, int64_t cap_uniform,
                             const int64_t *cap, uint64_t rk, int32_t S, int32_t s,
                             rating_map *rm, mover *mv) {
  uint64_t tie_tag = orc_tag(5);
  int64_t nm = 0;
  /* Rating: every active vertex decides against the snapshot. */
  for (int64_t u = 0; u < g->n; ++u) {
    uint64_t hu = orc_step(rk, (uint64_t)u);
    if ((int32_t)(hu % (uint64_t)S) != s) continue;
    int32_t t;
    int64_t gain;
    if (rate_with(g, u, label, lw, cap_uniform, cap, 0, orc_step(hu, tie_tag), rm, &t, &gain)) {
      mv[nm].u = u;
      mv[nm].t = t;
      mv[nm].gain = gain;
      mv[nm].w = orc_vw(g, u);
      mv[nm].approved = 0;
      ++nm;
    }
  }
  /* Approval per target, still against the snapshot weights. */
  qsort(mv, (size_t)nm, sizeof(mover), cmp_mover);
  for (int64_t i = 0; i < nm;) {
    int64_t j = i, in = 0;
    while (j < nm && mv[j].t == mv[i].t) in += mv[j++].w;
    int32_t t = mv[i].t;
    int64_t c = cap_of(cap_uniform, cap, t);
    if (lw[t] + in <= c) {
      for (int64_t q = i; q < j; ++q) mv[q].approved = 1;
    } else {
      int64_t p = 0;
      for (int64_t q = i; q < j; ++q) {
        p += mv[q].w;
        mv[q].approved = lw[t] + p <= c;
      }
    }
    i = j;
  }
  /* Apply. */
  int64_t applied = 0;
  for (int64_t i = 0; i < nm; ++i) {
    if (!mv[i].approved) continue;
    int64_t u = mv[i].u;
    lw[label[u]] -= mv[i].w;
    lw[mv[i].t] += mv[i].w;
    label[u] = mv[i].t;
    ++applied;
  }
  return applied;
}

int64_t orc_lp_subround(const orc_graph *g, int32_t *label, int64_t *lw, int64_t nlabels,
                        int64_t cap_uniform, const int64_t *cap, uint64_t rk, int32_t S,
                        int32_t s) {
  rating_map rm;
  rm.R = (int64_t *)calloc((size_t)nlabels + 1, sizeof(int64_t));
  rm.touched = (int32_t *)malloc(sizeof(int32_t) * (size_t)(g->m2 + 1));
  mover *mv = (mover *)malloc(sizeof(mover) * (size_t)(g->n + 1));
  int64_t r = subround_with(g, label, lw, cap_uniform, cap, rk, S, s, &rm, mv);
  free(mv);
  free(rm.touched);
  free(rm.R);
  return r;
}

int64_t orc_lp_rounds(const orc_graph *g, int32_t *label, int64_t *lw, int64_t nlabels,
                      int64_t cap_uniform, const int64_t *cap, uint64_t seed, uint64_t tag,
                      uint64_t a, uint64_t b0, int32_t rounds, int32_t S) {
  rating_map rm;
  rm.R = (int64_t *)calloc((size_t)nlabels + 1, sizeof(int64_t));
  rm.touched = (int32_t *)malloc(sizeof(int32_t) * (size_t)(g->m2 + 1));
  mover *mv = (mover *)malloc(sizeof(mover) * (size_t)(g->n + 1));
  int64_t total = 0;
  for (int32_t r = 0; r < rounds; ++r) {
    uint64_t rk = orc_round_key(seed, tag, a, b0 + (uint64_t)r);
    for (int32_t s = 0; s < S; ++s)
      total += subround_with(g, label, lw, cap_uniform, cap, rk, S, s, &rm, mv);
  }
  free(mv);
  free(rm.touched);
  free(rm.R);
  return total;
}

typedef struct {
  int64_t key;
  int64_t u;
} fav_entry;

static int cmp_fav(const void *pa, const void *pb) {
  const fav_entry *a = (const fav_entry *)pa, *b = (const fav_entry *)pb;
  if (a->key != b->key) return a->key < b->key ? -1 : 1;
  return a->u < b->u ? -1 : (a->u > b->u);
}

/*
 * Two-hop packing of leftover singletons (reading of the paper's two-hop
 * matching, Section "KaMinPar"):
 *  - a singleton is a vertex u with C[u] = u and Wc[u] = c(u) (alone in its
 *    own cluster);
 *  - its favourite is the best neighbouring cluster by the rating order,
 *    ignoring the cap (two-hop tag, round 0); isolated vertices get the
 *    sentinel favourite n;
 *  - singletons are sorted by (favourite, u); inside a run of equal favourite
 *    with exclusive weight prefix P, vertex u goes to bin floor(P / U) unless
 *    it straddles the bin end (P + c(u) > (bin+1) U), in which case it stays
 *    alone; every bin becomes one cluster labelled by its first (smallest) u.
 * Every bin weighs at most U.
 */
void orc_two_hop(const orc_graph *g, int32_t *C, const int64_t *Wc, int64_t U, uint64_t seed,
                 int64_t level) {
  int64_t n = g->n;
  uint64_t rk = orc_round_key(seed, orc_tag(2), (uint64_t)level, 0);
  uint64_t tie_tag = orc_tag(5);
  fav_entry *f = (fav_entry *)malloc(sizeof(fav_entry) * (size_t)(n + 1));
  int64_t nf = 0;
  rating_map rm;
  rm.R = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
  rm.touched = (int32_t *)malloc(sizeof(int32_t) * (size_t)(g->m2 + 1));
  for (int64_t u = 0; u < n; ++u) {
    if (C[u] != u || Wc[u] != orc_vw(g, u)) continue;
    uint64_t hu = orc_step(rk, (uint64_t)u);
    int32_t t;
    int64_t gain;
    int64_t key = n;
    if (rate_with(g, u, C, Wc, 0, NULL, 1, orc_step(hu, tie_tag), &rm, &t, &gain)) key = t;
    f[nf].key = key;
    f[nf].u = u;
    ++nf;
  }
  qsort(f, (size_t)nf, sizeof(fav_entry), cmp_fav);
  int64_t i = 0;
  while (i < nf) {
    int64_t j = i;
    while (j < nf && f[j].key == f[i].key) ++j;
    int64_t P = 0, cur_bin = -1, head = -1;
    for (int64_t q = i; q < j; ++q) {
      int64_t u = f[q].u, c = orc_vw(g, u);
      int64_t bin = P / U;
      int straddle = P + c > (bin + 1) * U;
      P += c;
      if (straddle) continue;
      if (bin != cur_bin) {
        cur_bin = bin;
        head = u;
      }
      C[u] = (int32_t)head;
    }
    i = j;
  }
  free(rm.touched);
  free(rm.R);
  free(f);
}

void orc_cluster(const orc_graph *g, int64_t U, const orc_params *p, int64_t level, int32_t *C) {
  int64_t n = g->n;
  int64_t *Wc = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
  for (int64_t u = 0; u < n; ++u) {
    C[u] = (int32_t)u;
    Wc[u] = orc_vw(g, u);
  }
  orc_lp_rounds(g, C, Wc, n, U, NULL, p->seed, orc_tag(0), (uint64_t)level, 0, p->cluster_rounds,
                p->sub_rounds);
  if (p->two_hop) orc_two_hop(g, C, Wc, U, p->seed, level);
  free(Wc);
}
