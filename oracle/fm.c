/*
 * k-way FM refinement over the space-efficient gain table (Section
 * "Space-Efficient Gain Tables": FM inspects vertex gains far more often than
 * it moves vertices, so the gains come from cached affinities).
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * The paper names FM (Fiduccia and Mattheyses) and its gain table but not the
 * search itself. Reading taken here, a plain sequential k-way FM:
 *  - A pass starts with every vertex unlocked. While some unlocked vertex v
 *    has an admissible move (a block t != part(v) that holds a neighbour of v
 *    and has B[t] + c(v) <= L_max), it makes the best such move: largest gain
 *    w(v, V_t) - w(v, V_part(v)), then smaller v, then smaller t. Negative
 *    gains are allowed. The vertex is locked, block weights and the gain
 *    table are updated and the running gain is recorded.
 *  - At the end of the pass the moves after the best prefix (largest running
 *    gain, the shortest such prefix) are undone in reverse order; a pass whose
 *    best prefix gains nothing undoes all its moves.
 *  - Passes repeat while the last one gained something, at most `passes`.
 * Consequences the tests check: the cut never increases, it drops by the sum
 * of the kept prefix gains, the block caps hold if they held before, and when
 * FM stops because a pass gained nothing, no admissible move has a positive
 * gain.
 */
#include <stdlib.h>

#include "oracle.h"

typedef struct {
  int64_t v;
  int32_t from, to;
} fm_move;

static void apply(orc_gain_table *t, const orc_graph *g, int32_t *part, int64_t *B, int64_t v,
                  int32_t from, int32_t to) {
  orc_gt_move(t, g, v, from, to);
  B[from] -= orc_vw(g, v);
  B[to] += orc_vw(g, v);
  part[v] = to;
}

int64_t orc_fm_refine(const orc_graph *g, int32_t *part, int64_t *B, int32_t k, int64_t l_max,
                      int32_t passes) {
  int64_t n = g->n, total = 0;
  orc_gain_table *t = orc_gt_build(g, part, k);
  char *locked = (char *)malloc((size_t)n + 1);
  fm_move *log = (fm_move *)malloc(sizeof(fm_move) * (size_t)(n + 1));
  for (int32_t pass = 0; pass < passes; ++pass) {
    for (int64_t v = 0; v < n; ++v) locked[v] = 0;
    int64_t nmoves = 0, run = 0, best_run = 0, best_len = 0;
    for (;;) {
      int64_t bv = -1, bgain = 0;
      int32_t bt = -1;
      for (int64_t v = 0; v < n; ++v) {
        if (locked[v]) continue;
        int32_t own = part[v];
        int64_t a_own = orc_gt_get(t, v, own);
        for (int64_t e = g->xadj[v]; e < g->xadj[v + 1]; ++e) {
          int32_t x = part[g->adj[e]];
          if (x == own || B[x] + orc_vw(g, v) > l_max) continue;
          int64_t gain = orc_gt_get(t, v, x) - a_own;
          /* v ascends in the scan: a later v wins only with a larger gain */
          if (bv < 0 || gain > bgain || (v == bv && gain == bgain && x < bt)) {
            bv = v;
            bgain = gain;
            bt = x;
          }
        }
      }
      if (bv < 0) break;
      log[nmoves].v = bv;
      log[nmoves].from = part[bv];
      log[nmoves].to = bt;
      ++nmoves;
      apply(t, g, part, B, bv, part[bv], bt);
      locked[bv] = 1;
      run += bgain;
      if (run > best_run) {
        best_run = run;
        best_len = nmoves;
      }
    }
    for (int64_t i = nmoves - 1; i >= best_len; --i)
      apply(t, g, part, B, log[i].v, log[i].to, log[i].from);
    total += best_run;
    if (best_run <= 0) break;
  }
  free(log);
  free(locked);
  orc_gt_free(t);
  return total;
}
