/*
 * Cluster contraction. TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Paper, Section "Contraction": clusters of G become the vertices of G'; an
 * edge (u,v) of G with C[u] != C[v] becomes the edge (C[u], C[v]) of G' and
 * duplicate edges are merged by summing weights,
 *     w'(a,b) = sum of w(u,v) over u in C^-1[a], v in C^-1[b], (u,v) in E;
 * the coarse edges of cluster a are obtained by scanning the neighbourhoods of
 * its members and adding w(u,v) to w'(a, C[v]) (the same aggregation as the
 * rating map of label propagation). Coarse node weights are the cluster
 * weights.
 *
 * Readings where the paper is silent: coarse ids are the ranks of the
 * non-empty cluster labels in ascending order (the paper's atomic-counter ids
 * depend on thread timing); each coarse neighbourhood is sorted ascending.
 */
#include "oracle.h"
#include <stdlib.h>
#include <string.h>

static int cmp_i32(const void *a, const void *b) {
  int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
  return x < y ? -1 : (x > y);
}

void orc_graph_free(orc_graph *g) {
  free(g->xadj);
  free(g->adj);
  free(g->vw);
  free(g->ew);
  memset(g, 0, sizeof(*g));
}

int64_t orc_contract(const orc_graph *g, const int32_t *C, orc_graph *out, int32_t *map) {
  int64_t n = g->n;
  int64_t *cid = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
  for (int64_t x = 0; x < n; ++x) cid[x] = 0;
  for (int64_t u = 0; u < n; ++u) cid[C[u]] = 1;
  int64_t nc = 0;
  for (int64_t x = 0; x < n; ++x) {
    int64_t f = cid[x];
    cid[x] = f ? nc : -1;
    nc += f;
  }
  for (int64_t u = 0; u < n; ++u) map[u] = (int32_t)cid[C[u]];

  /* members of every coarse vertex, by counting sort on the coarse id */
  int64_t *mstart = (int64_t *)calloc((size_t)nc + 1, sizeof(int64_t));
  int64_t *members = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
  for (int64_t u = 0; u < n; ++u) mstart[map[u] + 1]++;
  for (int64_t a = 0; a < nc; ++a) mstart[a + 1] += mstart[a];
  int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nc + 1));
  memcpy(fill, mstart, sizeof(int64_t) * (size_t)nc);
  for (int64_t u = 0; u < n; ++u) members[fill[map[u]]++] = u;

  out->n = nc;
  out->xadj = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nc + 1));
  out->vw = (int64_t *)calloc((size_t)nc + 1, sizeof(int64_t));
  int64_t cap = g->m2 > 0 ? g->m2 : 1;
  out->adj = (int32_t *)malloc(sizeof(int32_t) * (size_t)cap);
  out->ew = (int64_t *)malloc(sizeof(int64_t) * (size_t)cap);

  int64_t *R = (int64_t *)calloc((size_t)nc + 1, sizeof(int64_t));
  int32_t *touched = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nc + 1));
  int64_t pos = 0;
  for (int64_t a = 0; a < nc; ++a) {
    out->xadj[a] = pos;
    int64_t nt = 0;
    for (int64_t q = mstart[a]; q < mstart[a + 1]; ++q) {
      int64_t u = members[q];
      out->vw[a] += orc_vw(g, u);
      for (int64_t e = g->xadj[u]; e < g->xadj[u + 1]; ++e) {
        int32_t b = map[g->adj[e]];
        if (b == a) continue;
        if (R[b] == 0) touched[nt++] = b;
        R[b] += orc_ew(g, e);
      }
    }
    qsort(touched, (size_t)nt, sizeof(int32_t), cmp_i32);
    for (int64_t i = 0; i < nt; ++i) {
      out->adj[pos] = touched[i];
      out->ew[pos] = R[touched[i]];
      R[touched[i]] = 0;
      ++pos;
    }
  }
  out->xadj[nc] = pos;
  out->m2 = pos;
  free(touched);
  free(R);
  free(fill);
  free(members);
  free(mstart);
  free(cid);
  return nc;
}
