/*
 * Balance constraint, metrics, initial partitioning, refinement, rebalancing
 * and the multilevel driver. TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Paper: the balanced k-way partitioning problem (Section "Introduction": every
 * block weighs at most (1+eps)|V|/k, minimise the edge cut), the multilevel
 * scheme (Section "The Multilevel Scheme": coarsen, partition the coarsest
 * graph, project and refine level by level) and KaMinPar's components (Section
 * "KaMinPar": label propagation clustering with two-hop matching, initial
 * bipartitioning by greedy graph growing plus 2-way refinement, size-
 * constrained label propagation refinement).
 *
 * Readings where the paper is silent or real-valued:
 *  - eps is carried as integer parts per million, eps_ppm.
 *  - Block cap L_max = floor((1e6 + eps_ppm) * ceil(W/k) / 1e6) (the paper's
 *    (1+eps)|V|/k with the perfectly balanced weight rounded up, so that unit
 *    weights always admit a feasible partition).
 *  - Cluster cap U = max(1, floor(eps_ppm * W / (1e6 * k))).
 *  - Coarsening stops once n <= c_lim * k, when a level shrinks by less than
 *    5% (20 n' > 19 n: the level is discarded), or at max_levels graphs.
 *  - Initial partitioning is recursive bisection; each bisection tries T
 *    seeded attempts of BFS growing plus 2-way label propagation and keeps the
 *    smallest cut (see bisect_node).
 *  - Every level: project, rebalance if a block exceeds L_max, then refine
 *    with label propagation (cap L_max), then (fm_passes > 0, off by default)
 *    with k-way FM over the gain table.
 */
#include "oracle.h"
#include <stdlib.h>
#include <string.h>

int64_t orc_cluster_cap(int64_t W, int32_t k, int64_t eps_ppm) {
  __int128 num = (__int128)eps_ppm * W;
  int64_t u = (int64_t)(num / ((__int128)1000000 * k));
  return u < 1 ? 1 : u;
}

int64_t orc_block_cap(int64_t W, int32_t k, int64_t eps_ppm) {
  int64_t perfect = (W + k - 1) / k;
  __int128 num = (__int128)(1000000 + eps_ppm) * perfect;
  return (int64_t)(num / 1000000);
}

static int64_t find_in(const orc_graph *g, int64_t v, int64_t u) {
  int64_t lo = g->xadj[v], hi = g->xadj[v + 1];
  while (lo < hi) {
    int64_t mid = lo + (hi - lo) / 2;
    if (g->adj[mid] < u)
      lo = mid + 1;
    else
      hi = mid;
  }
  return (lo < g->xadj[v + 1] && g->adj[lo] == u) ? lo : -1;
}

/* 0 = valid; otherwise a positive code naming the first violated rule. */
int orc_validate(const orc_graph *g) {
  if (g->n < 0 || g->xadj[0] != 0 || g->xadj[g->n] != g->m2) return 1;
  for (int64_t u = 0; u < g->n; ++u) {
    if (g->xadj[u + 1] < g->xadj[u]) return 2;
    if (orc_vw(g, u) <= 0) return 3;
    for (int64_t e = g->xadj[u]; e < g->xadj[u + 1]; ++e) {
      int64_t v = g->adj[e];
      if (v < 0 || v >= g->n) return 4;
      if (v == u) return 5;
      if (e > g->xadj[u] && g->adj[e - 1] >= v) return 6;
      if (orc_ew(g, e) <= 0) return 7;
      int64_t r = find_in(g, v, u);
      if (r < 0 || orc_ew(g, r) != orc_ew(g, e)) return 8;
    }
  }
  return 0;
}

void orc_block_weights(const orc_graph *g, const int32_t *part, int32_t k, int64_t *B) {
  for (int32_t b = 0; b < k; ++b) B[b] = 0;
  for (int64_t u = 0; u < g->n; ++u) B[part[u]] += orc_vw(g, u);
}

/* Edge cut: half the weight of adjacency entries whose ends lie in different
 * blocks (both directions are stored). */
int64_t orc_cut(const orc_graph *g, const int32_t *part) {
  int64_t c = 0;
  for (int64_t u = 0; u < g->n; ++u)
    for (int64_t e = g->xadj[u]; e < g->xadj[u + 1]; ++e)
      if (part[u] != part[g->adj[e]]) c += orc_ew(g, e);
  return c / 2;
}

/* Induced subgraph on the sorted vertex list vs (local id = list position). */
static void induced(const orc_graph *g, const int64_t *vs, int64_t ns, int64_t *loc,
                    orc_graph *sub) {
  for (int64_t i = 0; i < ns; ++i) loc[vs[i]] = i;
  int64_t m2 = 0;
  for (int64_t i = 0; i < ns; ++i)
    for (int64_t e = g->xadj[vs[i]]; e < g->xadj[vs[i] + 1]; ++e)
      if (loc[g->adj[e]] >= 0) ++m2;
  sub->n = ns;
  sub->m2 = m2;
  sub->xadj = (int64_t *)malloc(sizeof(int64_t) * (size_t)(ns + 1));
  sub->adj = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m2 + 1));
  sub->ew = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m2 + 1));
  sub->vw = (int64_t *)malloc(sizeof(int64_t) * (size_t)(ns + 1));
  int64_t p = 0;
  for (int64_t i = 0; i < ns; ++i) {
    sub->xadj[i] = p;
    sub->vw[i] = orc_vw(g, vs[i]);
    for (int64_t e = g->xadj[vs[i]]; e < g->xadj[vs[i] + 1]; ++e) {
      int64_t l = loc[g->adj[e]];
      if (l < 0) continue;
      sub->adj[p] = (int32_t)l;
      sub->ew[p] = orc_ew(g, e);
      ++p;
    }
  }
  sub->xadj[ns] = p;
  for (int64_t i = 0; i < ns; ++i) loc[vs[i]] = -1;
}

/* BFS order from s: FIFO queue, neighbours pushed in ascending id; vertices
 * the search does not reach are appended in ascending id. */
static void bfs_order(const orc_graph *g, int64_t s, int64_t *order) {
  char *seen = (char *)calloc((size_t)g->n + 1, 1);
  int64_t head = 0, tail = 0;
  order[tail++] = s;
  seen[s] = 1;
  while (head < tail) {
    int64_t x = order[head++];
    for (int64_t e = g->xadj[x]; e < g->xadj[x + 1]; ++e) {
      int64_t v = g->adj[e];
      if (!seen[v]) {
        seen[v] = 1;
        order[tail++] = v;
      }
    }
  }
  for (int64_t v = 0; v < g->n; ++v)
    if (!seen[v]) order[tail++] = v;
  free(seen);
}

/*
 * One node of the recursive bisection (reading of "a portfolio of randomized
 * sequential greedy graph growing heuristics and 2-way FM", Section
 * "KaMinPar"). The node owns the sorted vertex list vs and the blocks
 * [offset, offset + kk). With k0 = ceil(kk/2), k1 = floor(kk/2):
 *  - target0 = floor(W_sub * k0 / kk); side caps k0 * L_max and k1 * L_max;
 *  - attempt a: seed vertex hash(seed, ip-seed tag, node key, a) mod n_sub;
 *    side 0 is the longest prefix of the BFS order whose weight stays within
 *    target0; then refine_rounds rounds of 2-way label propagation (ip-lp tag,
 *    a = node key, rounds numbered from a << 8) with the side caps;
 *  - the attempt with the smallest cut wins, the lowest attempt on ties.
 * Node key = (offset << 32) | kk. Local ids (positions in vs) are the vertex
 * ids for hashing and ordering.
 */
static void bisect_node(const orc_graph *g, const int64_t *vs, int64_t ns, int32_t kk,
                        int32_t offset, int64_t l_max, const orc_params *p, int64_t *loc,
                        int32_t *part) {
  if (kk == 1) {
    for (int64_t i = 0; i < ns; ++i) part[vs[i]] = offset;
    return;
  }
  if (ns == 0) return;
  int32_t k0 = (kk + 1) / 2, k1 = kk / 2;
  orc_graph sub;
  induced(g, vs, ns, loc, &sub);
  int64_t W = 0;
  for (int64_t i = 0; i < ns; ++i) W += sub.vw[i];
  int64_t target0 = (int64_t)((__int128)W * k0 / kk);
  int64_t caps[2] = {(int64_t)k0 * l_max, (int64_t)k1 * l_max};
  uint64_t key = ((uint64_t)(uint32_t)offset << 32) | (uint32_t)kk;
  int32_t *side = (int32_t *)malloc(sizeof(int32_t) * (size_t)ns);
  int32_t *best = (int32_t *)malloc(sizeof(int32_t) * (size_t)ns);
  int64_t *order = (int64_t *)malloc(sizeof(int64_t) * (size_t)ns);
  int64_t best_cut = -1;
  for (int32_t a = 0; a < p->ip_attempts; ++a) {
    uint64_t h = orc_round_key(p->seed, orc_tag(3), key, (uint64_t)a);
    int64_t s = (int64_t)(h % (uint64_t)ns);
    bfs_order(&sub, s, order);
    for (int64_t i = 0; i < ns; ++i) side[i] = 1;
    int64_t pre = 0;
    for (int64_t i = 0; i < ns; ++i) {
      int64_t x = order[i];
      if (pre + sub.vw[x] > target0) break;
      pre += sub.vw[x];
      side[x] = 0;
    }
    int64_t lw[2] = {pre, W - pre};
    orc_lp_rounds(&sub, side, lw, 2, 0, caps, p->seed, orc_tag(4), key, (uint64_t)a << 8,
                  p->refine_rounds, p->sub_rounds);
    int64_t cut = orc_cut(&sub, side);
    if (best_cut < 0 || cut < best_cut) {
      best_cut = cut;
      memcpy(best, side, sizeof(int32_t) * (size_t)ns);
    }
  }
  int64_t *v0 = (int64_t *)malloc(sizeof(int64_t) * (size_t)ns);
  int64_t *v1 = (int64_t *)malloc(sizeof(int64_t) * (size_t)ns);
  int64_t n0 = 0, n1 = 0;
  for (int64_t i = 0; i < ns; ++i) {
    if (best[i] == 0)
      v0[n0++] = vs[i];
    else
      v1[n1++] = vs[i];
  }
  free(order);
  free(best);
  free(side);
  orc_graph_free(&sub);
  bisect_node(g, v0, n0, k0, offset, l_max, p, loc, part);
  bisect_node(g, v1, n1, k1, offset + k0, l_max, p, loc, part);
  free(v0);
  free(v1);
}

void orc_initial_partition(const orc_graph *g, int32_t k, int64_t l_max, const orc_params *p,
                           int32_t *part) {
  int64_t n = g->n;
  int64_t *vs = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
  int64_t *loc = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
  for (int64_t u = 0; u < n; ++u) {
    vs[u] = u;
    loc[u] = -1;
  }
  bisect_node(g, vs, n, k, 0, l_max, p, loc, part);
  free(loc);
  free(vs);
}

/*
 * Rebalancing (the paper repairs balance violations after label propagation in
 * its distributed variant, Section "KaMinPar"). Reading: while some block
 * exceeds L_max, take the overloaded block b with the smallest index; every
 * u in b picks the block t != b with the largest affinity R[t] among those
 * with B[t] + c(u) <= L_max (ties: smaller t; zero affinity allowed); the u
 * with the smallest loss R[b] - R[t] (ties: smaller u) moves. Returns 0 when
 * balanced, 1 if no vertex fits anywhere.
 */
int orc_rebalance(const orc_graph *g, int32_t *part, int64_t *B, int32_t k, int64_t l_max) {
  int64_t *R = (int64_t *)calloc((size_t)k + 1, sizeof(int64_t));
  int ret = 0;
  for (;;) {
    int32_t b = -1;
    for (int32_t i = 0; i < k; ++i)
      if (B[i] > l_max) {
        b = i;
        break;
      }
    if (b < 0) break;
    int64_t best_u = -1, best_loss = 0;
    int32_t best_t = -1;
    for (int64_t u = 0; u < g->n; ++u) {
      if (part[u] != b) continue;
      int64_t c = orc_vw(g, u);
      for (int64_t e = g->xadj[u]; e < g->xadj[u + 1]; ++e) R[part[g->adj[e]]] += orc_ew(g, e);
      int32_t t = -1;
      for (int32_t x = 0; x < k; ++x) {
        if (x == b || B[x] + c > l_max) continue;
        if (t < 0 || R[x] > R[t]) t = x;
      }
      if (t >= 0) {
        int64_t loss = R[b] - R[t];
        if (best_u < 0 || loss < best_loss) {
          best_u = u;
          best_loss = loss;
          best_t = t;
        }
      }
      for (int64_t e = g->xadj[u]; e < g->xadj[u + 1]; ++e) R[part[g->adj[e]]] = 0;
    }
    if (best_u < 0) {
      ret = 1;
      break;
    }
    B[b] -= orc_vw(g, best_u);
    B[best_t] += orc_vw(g, best_u);
    part[best_u] = best_t;
  }
  free(R);
  return ret;
}

int64_t orc_refine(const orc_graph *g, int32_t *part, int64_t *B, int32_t k, int64_t l_max,
                   const orc_params *p, int64_t level) {
  return orc_lp_rounds(g, part, B, k, l_max, NULL, p->seed, orc_tag(1), (uint64_t)level, 0,
                       p->refine_rounds, p->sub_rounds);
}

int orc_partition(const orc_graph *g0, int32_t k, int64_t eps_ppm, const orc_params *p,
                  int32_t *part, orc_stats *st) {
  memset(st, 0, sizeof(*st));
  if (k < 1 || eps_ppm < 0) return 1;
  int64_t W = 0;
  for (int64_t u = 0; u < g0->n; ++u) W += orc_vw(g0, u);
  int64_t U = orc_cluster_cap(W, k, eps_ppm);
  int64_t l_max = orc_block_cap(W, k, eps_ppm);
  st->l_max = l_max;
  st->u_max = U;
  int32_t maxl = p->max_levels < 64 ? p->max_levels : 64;
  orc_graph levels[64];
  int32_t *maps[64];
  levels[0] = *g0;
  int32_t L = 0;
  st->level_n[0] = g0->n;
  st->level_m2[0] = g0->m2;
  if (k > 1) {
    while (levels[L].n > (int64_t)p->c_lim * k && L + 1 < maxl) {
      orc_graph *g = &levels[L];
      int32_t *C = (int32_t *)malloc(sizeof(int32_t) * (size_t)(g->n + 1));
      int32_t *map = (int32_t *)malloc(sizeof(int32_t) * (size_t)(g->n + 1));
      orc_cluster(g, U, p, L, C);
      orc_graph cg;
      int64_t nc = orc_contract(g, C, &cg, map);
      free(C);
      if (20 * nc > 19 * g->n) {
        orc_graph_free(&cg);
        free(map);
        break;
      }
      maps[L] = map;
      levels[L + 1] = cg;
      ++L;
      st->level_n[L] = cg.n;
      st->level_m2[L] = cg.m2;
    }
  }
  st->levels = L + 1;
  int32_t *cur = (int32_t *)calloc((size_t)levels[L].n + 1, sizeof(int32_t));
  int64_t *B = (int64_t *)calloc((size_t)k, sizeof(int64_t));
  if (k > 1) orc_initial_partition(&levels[L], k, l_max, p, cur);
  for (int32_t l = L; l >= 0; --l) {
    if (l < L) {
      int32_t *fine = (int32_t *)malloc(sizeof(int32_t) * (size_t)(levels[l].n + 1));
      for (int64_t u = 0; u < levels[l].n; ++u) fine[u] = cur[maps[l][u]];
      free(cur);
      cur = fine;
    }
    if (k > 1) {
      orc_block_weights(&levels[l], cur, k, B);
      int over = 0;
      for (int32_t b = 0; b < k; ++b) over |= B[b] > l_max;
      if (over) orc_rebalance(&levels[l], cur, B, k, l_max);
      orc_refine(&levels[l], cur, B, k, l_max, p, l);
      if (p->fm_passes > 0) orc_fm_refine(&levels[l], cur, B, k, l_max, p->fm_passes);
    }
  }
  memcpy(part, cur, sizeof(int32_t) * (size_t)g0->n);
  orc_block_weights(g0, part, k, B);
  st->cut = orc_cut(g0, part);
  int64_t mx = 0;
  for (int32_t b = 0; b < k; ++b)
    if (B[b] > mx) mx = B[b];
  st->max_block_weight = mx;
  st->balanced = mx <= l_max;
  int64_t perfect = (W + k - 1) / k;
  st->imbalance = perfect > 0 ? (double)mx / (double)perfect - 1.0 : 0.0;
  free(B);
  free(cur);
  for (int32_t l = 1; l <= L; ++l) orc_graph_free(&levels[l]);
  for (int32_t l = 0; l < L; ++l) free(maps[l]);
  return 0;
}
