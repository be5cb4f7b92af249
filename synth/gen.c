/*
 * Seeded synthetic graph generators. They hold none of the partitioner's
 * arithmetic and feed both the GPU path and the CPU oracle with identical
 * inputs. Every random number is output i of the splitmix64 stream (Steele,
 * Lea and Flood, OOPSLA 2014) seeded with the graph seed, so the graphs are
 * identical on every machine (floating point is used only in the geometric
 * generator, compiled without contraction of multiply-adds).
 *
 * All generators return a simple undirected graph in CSR form: neighbours
 * sorted ascending, no self-loops, no duplicates, both directions stored.
 *
 *  - G(n,m): m distinct unordered pairs {u,v}, u != v, drawn uniformly by
 *    rejection; vertex ids carry no locality.
 *  - RGG-2D: n points uniform in [0,1)^2 (no torus); an edge joins two points
 *    at distance <= r, r = sqrt(d / (pi n)) for expected degree d. Vertex ids
 *    follow grid cells of side >= r in row-major order, then x, then y, so
 *    neighbour ids are close (the locality KaGen's generator gives).
 *  - R-MAT: 2^scale vertices, ef * 2^scale sampled directed edges; each of the
 *    scale recursion levels picks a quadrant with probabilities (a, b, c, d)
 *    using 21 random bits (three levels per 64-bit draw); no noise, no id
 *    permutation; symmetrised, deduplicated, self-loops dropped, isolated
 *    vertices kept.
 *  - RHG (threshold random hyperbolic graph): see syn_rhg.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define SYN_GAMMA 0x9e3779b97f4a7c15ULL

typedef struct {
  int64_t n, m2;
  int64_t *xadj;
  int32_t *adj;
} syn_graph;

static uint64_t sm64(uint64_t seed, uint64_t i) {
  uint64_t z = seed + (i + 1) * SYN_GAMMA;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

static double unit01(uint64_t r) { return (double)(r >> 11) * (1.0 / 9007199254740992.0); }

static int cmp_i32(const void *a, const void *b) {
  int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
  return x < y ? -1 : (x > y);
}

/* Build a symmetric CSR from undirected pairs (u != v, possibly duplicated):
 * both directions inserted, each neighbourhood sorted and deduplicated. */
static syn_graph *from_pairs(int64_t n, const int32_t *pu, const int32_t *pv, int64_t np) {
  int64_t *deg = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
  for (int64_t i = 0; i < np; ++i) {
    deg[pu[i]]++;
    deg[pv[i]]++;
  }
  int64_t *start = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
  start[0] = 0;
  for (int64_t u = 0; u < n; ++u) start[u + 1] = start[u] + deg[u];
  int32_t *tmp = (int32_t *)malloc(sizeof(int32_t) * (size_t)(start[n] + 1));
  int64_t *fill = deg; /* reuse as fill pointer */
  for (int64_t u = 0; u < n; ++u) fill[u] = start[u];
  for (int64_t i = 0; i < np; ++i) {
    tmp[fill[pu[i]]++] = pv[i];
    tmp[fill[pv[i]]++] = pu[i];
  }
  int64_t *newdeg = fill;
#pragma omp parallel for schedule(dynamic, 1024)
  for (int64_t u = 0; u < n; ++u) {
    int32_t *a = tmp + start[u];
    int64_t d = start[u + 1] - start[u];
    qsort(a, (size_t)d, sizeof(int32_t), cmp_i32);
    int64_t w = 0;
    for (int64_t i = 0; i < d; ++i)
      if (a[i] != u && (w == 0 || a[w - 1] != a[i])) a[w++] = a[i];
    newdeg[u] = w;
  }
  syn_graph *g = (syn_graph *)malloc(sizeof(syn_graph));
  g->n = n;
  g->xadj = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
  g->xadj[0] = 0;
  for (int64_t u = 0; u < n; ++u) g->xadj[u + 1] = g->xadj[u] + newdeg[u];
  g->m2 = g->xadj[n];
  g->adj = (int32_t *)malloc(sizeof(int32_t) * (size_t)(g->m2 + 1));
#pragma omp parallel for schedule(dynamic, 1024)
  for (int64_t u = 0; u < n; ++u)
    memcpy(g->adj + g->xadj[u], tmp + start[u], sizeof(int32_t) * (size_t)newdeg[u]);
  free(tmp);
  free(start);
  free(deg);
  return g;
}

/* ---------------------------------------------------------------- G(n,m) */
syn_graph *syn_gnm(int64_t n, int64_t m, uint64_t seed) {
  if (n < 2) m = 0;
  int64_t maxm = n * (n - 1) / 2;
  if (m > maxm) m = maxm;
  int64_t cap = 1;
  while (cap < 2 * m + 16) cap <<= 1;
  uint64_t *set = (uint64_t *)calloc((size_t)cap, sizeof(uint64_t));
  int32_t *pu = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m + 1));
  int32_t *pv = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m + 1));
  int64_t got = 0;
  uint64_t i = 0;
  while (got < m) {
    uint64_t r = sm64(seed, i++);
    uint64_t u = ((r >> 32) * (uint64_t)n) >> 32;
    uint64_t v = ((r & 0xffffffffULL) * (uint64_t)n) >> 32;
    if (u == v) continue;
    if (u > v) {
      uint64_t t = u;
      u = v;
      v = t;
    }
    uint64_t key = (u << 32 | v) + 1;
    uint64_t h = sm64(key, 0) & (uint64_t)(cap - 1);
    int dup = 0;
    while (set[h]) {
      if (set[h] == key) {
        dup = 1;
        break;
      }
      h = (h + 1) & (uint64_t)(cap - 1);
    }
    if (dup) continue;
    set[h] = key;
    pu[got] = (int32_t)u;
    pv[got] = (int32_t)v;
    ++got;
  }
  syn_graph *g = from_pairs(n, pu, pv, m);
  free(set);
  free(pu);
  free(pv);
  return g;
}

/* ---------------------------------------------------------------- RGG-2D */
typedef struct {
  double x, y;
  int64_t cell;
  int64_t orig;
} pt;

static int cmp_pt(const void *pa, const void *pb) {
  const pt *a = (const pt *)pa, *b = (const pt *)pb;
  if (a->cell != b->cell) return a->cell < b->cell ? -1 : 1;
  if (a->x != b->x) return a->x < b->x ? -1 : 1;
  if (a->y != b->y) return a->y < b->y ? -1 : 1;
  return a->orig < b->orig ? -1 : (a->orig > b->orig);
}

syn_graph *syn_rgg2d(int64_t n, double avg_deg, uint64_t seed) {
  const double PI = 3.14159265358979323846;
  double r = sqrt(avg_deg / (PI * (double)(n > 0 ? n : 1)));
  int64_t gdim = (int64_t)floor(1.0 / r);
  if (gdim < 1) gdim = 1;
  double r2 = r * r;
  pt *p = (pt *)malloc(sizeof(pt) * (size_t)(n + 1));
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    p[i].x = unit01(sm64(seed, 2 * (uint64_t)i));
    p[i].y = unit01(sm64(seed, 2 * (uint64_t)i + 1));
    int64_t cx = (int64_t)(p[i].x * (double)gdim), cy = (int64_t)(p[i].y * (double)gdim);
    if (cx >= gdim) cx = gdim - 1;
    if (cy >= gdim) cy = gdim - 1;
    p[i].cell = cy * gdim + cx;
    p[i].orig = i;
  }
  /* counting sort by cell, then order inside each cell */
  int64_t ncell = gdim * gdim;
  int64_t *cstart = (int64_t *)calloc((size_t)ncell + 1, sizeof(int64_t));
  for (int64_t i = 0; i < n; ++i) cstart[p[i].cell + 1]++;
  for (int64_t c = 0; c < ncell; ++c) cstart[c + 1] += cstart[c];
  int64_t *cfill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(ncell + 1));
  memcpy(cfill, cstart, sizeof(int64_t) * (size_t)ncell);
  pt *q = (pt *)malloc(sizeof(pt) * (size_t)(n + 1));
  for (int64_t i = 0; i < n; ++i) q[cfill[p[i].cell]++] = p[i];
  free(p);
  free(cfill);
#pragma omp parallel for schedule(dynamic, 256)
  for (int64_t c = 0; c < ncell; ++c)
    qsort(q + cstart[c], (size_t)(cstart[c + 1] - cstart[c]), sizeof(pt), cmp_pt);
  /* count, then fill, neighbours (ids = positions in q) */
  int64_t *xadj = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
  int32_t *adj = NULL;
  for (int pass = 0; pass < 2; ++pass) {
    if (pass == 1) {
      for (int64_t i = 0; i < n; ++i) xadj[i + 1] += xadj[i];
      adj = (int32_t *)malloc(sizeof(int32_t) * (size_t)(xadj[n] + 1));
    }
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t i = 0; i < n; ++i) {
      int64_t cx = q[i].cell % gdim, cy = q[i].cell / gdim;
      int64_t cnt = 0, base = pass ? xadj[i] : 0;
      for (int64_t yy = cy - 1; yy <= cy + 1; ++yy) {
        if (yy < 0 || yy >= gdim) continue;
        for (int64_t xx = cx - 1; xx <= cx + 1; ++xx) {
          if (xx < 0 || xx >= gdim) continue;
          int64_t c = yy * gdim + xx;
          for (int64_t j = cstart[c]; j < cstart[c + 1]; ++j) {
            if (j == i) continue;
            double ddx = q[i].x - q[j].x, ddy = q[i].y - q[j].y;
            if (ddx * ddx + ddy * ddy <= r2) {
              if (pass) adj[base + cnt] = (int32_t)j;
              ++cnt;
            }
          }
        }
      }
      if (pass)
        qsort(adj + base, (size_t)cnt, sizeof(int32_t), cmp_i32);
      else
        xadj[i + 1] = cnt;
    }
  }
  free(q);
  free(cstart);
  syn_graph *g = (syn_graph *)malloc(sizeof(syn_graph));
  g->n = n;
  g->xadj = xadj;
  g->adj = adj;
  g->m2 = xadj[n];
  return g;
}

/* ----------------------------------------------------------------- R-MAT */
syn_graph *syn_rmat(int32_t scale, int64_t edge_factor, double a, double b, double c,
                    uint64_t seed) {
  int64_t n = (int64_t)1 << scale;
  int64_t E = edge_factor * n;
  const double S21 = 2097152.0;
  uint64_t A = (uint64_t)(a * S21), AB = (uint64_t)((a + b) * S21),
           ABC = (uint64_t)((a + b + c) * S21);
  int32_t draws = (scale + 2) / 3;
  int32_t *pu = (int32_t *)malloc(sizeof(int32_t) * (size_t)(E + 1));
  int32_t *pv = (int32_t *)malloc(sizeof(int32_t) * (size_t)(E + 1));
#pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < E; ++j) {
    uint64_t u = 0, v = 0, r = 0;
    for (int32_t l = 0; l < scale; ++l) {
      if (l % 3 == 0) r = sm64(seed, (uint64_t)j * (uint64_t)draws + (uint64_t)(l / 3));
      uint64_t q = (r >> (21 * (l % 3))) & 0x1fffffULL;
      uint64_t row = q >= AB, col = (q >= A && q < AB) || q >= ABC;
      u |= row << (scale - 1 - l);
      v |= col << (scale - 1 - l);
    }
    pu[j] = (int32_t)u;
    pv[j] = (int32_t)v;
  }
  /* drop self-loops before symmetrising */
  int64_t w = 0;
  for (int64_t j = 0; j < E; ++j)
    if (pu[j] != pv[j]) {
      pu[w] = pu[j];
      pv[w] = pv[j];
      ++w;
    }
  syn_graph *g = from_pairs(n, pu, pv, w);
  free(pu);
  free(pv);
  return g;
}

/* ------------------------------------------------------------------- RHG */
/* Threshold random hyperbolic graph (Krioukov, Papadopoulos, Kitsak, Vahdat,
 * Boguna, Phys. Rev. E 82, 2010): n points in a hyperbolic disk of radius R.
 * Point i takes draws 2i (angle, uniform in [0, 2 pi)) and 2i + 1 (radius,
 * density alpha sinh(alpha r) / (cosh(alpha R) - 1) on [0, R], sampled by
 * its inverse CDF r = acosh(1 + (cosh(alpha R) - 1) U) / alpha), with
 * alpha = (gamma - 1) / 2 for the power-law exponent gamma. Two points are
 * adjacent iff their hyperbolic distance is <= R:
 *   cosh r1 cosh r2 - sinh r1 sinh r2 cos(t1 - t2) <= cosh R.
 * R = 2 ln n + C. C starts from the asymptotic average degree
 * 2 alpha^2 e^{-C/2} / (pi (alpha - 1/2)^2) (Gugelmann, Panagiotou, Peter,
 * ICALP 2012) and is then bisected on the measured average degree of these
 * points (the radii are redrawn from the same uniforms for every trial C).
 * Vertex ids follow the angle order, so neighbour ids are close.
 * Candidates come from radial bands (the band idea of von Looz, Meyerhenke,
 * Prutkin, ISAAC 2015): points of each band are kept in angle order, and for
 * u and a band whose lower radius is b > 0 only angles within
 * acos((cosh r_u cosh b - cosh R) / (sinh r_u sinh b)) of u's can be close
 * enough (that bound only tightens as r grows). Windows are widened by 1e-9
 * and every pair is tested with one expression in canonical order, so the
 * adjacency is symmetric. */
typedef struct {
  int64_t n, nb;
  double R, coshR;
  double *th, *ch, *sh; /* angle, cosh r, sinh r per vertex (angle order) */
  double *r;
  int64_t *bstart;      /* band b holds vertices bidx[bstart[b] .. bstart[b+1]) */
  int32_t *bidx;        /* vertex ids, angle order within a band */
  double *bth;          /* their angles */
  double *blo;          /* lower radius of each band */
} rhg_pts;

static int cmp_dbl_idx(const void *a, const void *b) {
  const double *x = (const double *)a, *y = (const double *)b;
  return x[0] < y[0] ? -1 : x[0] > y[0] ? 1 : (x[1] < y[1] ? -1 : x[1] > y[1]);
}

static int rhg_adjacent(const rhg_pts *P, int32_t u, int32_t v) {
  int32_t a = u < v ? u : v, b = u < v ? v : u;
  double lhs = P->ch[a] * P->ch[b] - P->sh[a] * P->sh[b] * cos(P->th[a] - P->th[b]);
  return lhs <= P->coshR;
}

/* radii and bands for disk radius R (angles and uniforms fixed) */
static void rhg_place(rhg_pts *P, const double *ur, double alpha, double R) {
  int64_t n = P->n;
  P->R = R;
  P->coshR = cosh(R);
  double ca = cosh(alpha * R) - 1.0;
  for (int64_t i = 0; i < n; ++i) {
    double r = acosh(1.0 + ca * ur[i]) / alpha;
    if (r > R) r = R;
    P->r[i] = r;
    P->ch[i] = cosh(r);
    P->sh[i] = sinh(r);
  }
  int64_t nb = P->nb;
  for (int64_t b = 0; b <= nb; ++b) P->bstart[b] = 0;
  for (int64_t b = 0; b < nb; ++b) P->blo[b] = R * (double)b / (double)nb;
  for (int64_t i = 0; i < n; ++i) {
    int64_t b = (int64_t)(P->r[i] / R * (double)nb);
    if (b >= nb) b = nb - 1;
    P->bstart[b + 1]++;
  }
  for (int64_t b = 0; b < nb; ++b) P->bstart[b + 1] += P->bstart[b];
  int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)nb);
  for (int64_t b = 0; b < nb; ++b) fill[b] = P->bstart[b];
  for (int64_t i = 0; i < n; ++i) { /* ids ascend with angle, so bands stay angle-sorted */
    int64_t b = (int64_t)(P->r[i] / R * (double)nb);
    if (b >= nb) b = nb - 1;
    P->bidx[fill[b]] = (int32_t)i;
    P->bth[fill[b]] = P->th[i];
    fill[b]++;
  }
  free(fill);
}

/* first position in band [lo, hi) of bth with angle >= t */
static int64_t lower_angle(const double *bth, int64_t lo, int64_t hi, double t) {
  while (lo < hi) {
    int64_t mid = lo + (hi - lo) / 2;
    if (bth[mid] < t) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

/* Visits every v != u adjacent to u (emit != NULL) or counts them; brute:
 * test every other point instead of the band windows (for tests). */
static int64_t rhg_scan(const rhg_pts *P, int32_t u, int32_t *emit, int brute) {
  const double TWO_PI = 6.283185307179586;
  int64_t cnt = 0;
  if (brute) {
    for (int32_t v = 0; v < (int32_t)P->n; ++v) {
      if (v == u || !rhg_adjacent(P, u, v)) continue;
      if (emit) emit[cnt] = v;
      ++cnt;
    }
    return cnt;
  }
  for (int64_t b = 0; b < P->nb; ++b) {
    int64_t lo = P->bstart[b], hi = P->bstart[b + 1];
    if (lo == hi) continue;
    double lb = P->blo[b], w = 4.0; /* > pi: the whole band */
    if (lb > 0.0 && P->sh[u] > 0.0) {
      double q = (P->ch[u] * cosh(lb) - P->coshR) / (P->sh[u] * sinh(lb));
      if (q > 1.0) continue;
      if (q > -1.0) w = acos(q) + 1e-9;
    }
    /* angle ranges [t0, t1] intersected with [0, 2 pi), up to two pieces */
    double t0 = P->th[u] - w, t1 = P->th[u] + w;
    double seg[4];
    int ns = 0;
    if (w >= 3.14159265358979) {
      seg[0] = 0.0, seg[1] = TWO_PI, ns = 1;
    } else {
      if (t0 < 0.0) {
        seg[0] = t0 + TWO_PI, seg[1] = TWO_PI, seg[2] = 0.0, seg[3] = t1, ns = 2;
      } else if (t1 >= TWO_PI) {
        seg[0] = t0, seg[1] = TWO_PI, seg[2] = 0.0, seg[3] = t1 - TWO_PI, ns = 2;
      } else {
        seg[0] = t0, seg[1] = t1, ns = 1;
      }
    }
    for (int sgi = 0; sgi < ns; ++sgi) {
      int64_t i = lower_angle(P->bth, lo, hi, seg[2 * sgi]);
      for (; i < hi && P->bth[i] <= seg[2 * sgi + 1]; ++i) {
        int32_t v = P->bidx[i];
        if (v == u || !rhg_adjacent(P, u, v)) continue;
        if (emit) emit[cnt] = v;
        ++cnt;
      }
    }
  }
  return cnt;
}

static int64_t rhg_count(const rhg_pts *P) {
  int64_t total = 0;
#pragma omp parallel for schedule(dynamic, 256) reduction(+ : total)
  for (int64_t u = 0; u < P->n; ++u) total += rhg_scan(P, (int32_t)u, NULL, 0);
  return total;
}

static syn_graph *rhg_build(int64_t n, double avg_deg, double gamma, uint64_t seed, int brute) {
  const double TWO_PI = 6.283185307179586;
  double alpha = (gamma - 1.0) / 2.0;
  rhg_pts P;
  memset(&P, 0, sizeof(P));
  P.n = n;
  P.nb = n > 1 ? (int64_t)ceil(log((double)n)) : 1;
  P.th = (double *)malloc(sizeof(double) * (size_t)(n + 1));
  P.ch = (double *)malloc(sizeof(double) * (size_t)(n + 1));
  P.sh = (double *)malloc(sizeof(double) * (size_t)(n + 1));
  P.r = (double *)malloc(sizeof(double) * (size_t)(n + 1));
  P.bidx = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n + 1));
  P.bth = (double *)malloc(sizeof(double) * (size_t)(n + 1));
  P.bstart = (int64_t *)malloc(sizeof(int64_t) * (size_t)(P.nb + 1));
  P.blo = (double *)malloc(sizeof(double) * (size_t)P.nb);
  /* angles sorted (ids follow angle order); each point keeps its radius draw */
  double *pair = (double *)malloc(sizeof(double) * 2 * (size_t)(n + 1));
  for (int64_t i = 0; i < n; ++i) {
    pair[2 * i] = unit01(sm64(seed, 2 * (uint64_t)i)) * TWO_PI;
    pair[2 * i + 1] = unit01(sm64(seed, 2 * (uint64_t)i + 1));
  }
  qsort(pair, (size_t)n, 2 * sizeof(double), cmp_dbl_idx);
  double *ur = (double *)malloc(sizeof(double) * (size_t)(n + 1));
  for (int64_t i = 0; i < n; ++i) {
    P.th[i] = pair[2 * i];
    ur[i] = pair[2 * i + 1];
  }
  free(pair);
  double am = alpha - 0.5;
  double C = -2.0 * log(avg_deg * 3.141592653589793 * am * am / (2.0 * alpha * alpha));
  double lnn = log((double)(n > 1 ? n : 2));
  if (n > 1) { /* bisection on the measured degree: larger C, sparser graph */
    double lo = C - 1.5, hi = C + 1.5;
    for (int it = 0; it < 8; ++it) {
      double mid = 0.5 * (lo + hi);
      rhg_place(&P, ur, alpha, 2.0 * lnn + mid);
      double d = (double)rhg_count(&P) / (double)n;
      if (d > avg_deg) lo = mid;
      else hi = mid;
    }
    C = 0.5 * (lo + hi);
  }
  rhg_place(&P, ur, alpha, 2.0 * lnn + C);
  syn_graph *g = (syn_graph *)malloc(sizeof(syn_graph));
  g->n = n;
  g->xadj = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
  int64_t *deg = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
#pragma omp parallel for schedule(dynamic, 256)
  for (int64_t u = 0; u < n; ++u) deg[u] = rhg_scan(&P, (int32_t)u, NULL, brute);
  g->xadj[0] = 0;
  for (int64_t u = 0; u < n; ++u) g->xadj[u + 1] = g->xadj[u] + deg[u];
  g->m2 = g->xadj[n];
  g->adj = (int32_t *)malloc(sizeof(int32_t) * (size_t)(g->m2 + 1));
#pragma omp parallel for schedule(dynamic, 256)
  for (int64_t u = 0; u < n; ++u) {
    int32_t *a = g->adj + g->xadj[u];
    rhg_scan(&P, (int32_t)u, a, brute);
    qsort(a, (size_t)deg[u], sizeof(int32_t), cmp_i32);
  }
  free(deg);
  free(ur);
  free(P.th), free(P.ch), free(P.sh), free(P.r), free(P.bidx), free(P.bth), free(P.bstart),
      free(P.blo);
  return g;
}

syn_graph *syn_rhg(int64_t n, double avg_deg, double gamma, uint64_t seed) {
  return rhg_build(n, avg_deg, gamma, seed, 0);
}

/* The same graph with every pair tested directly (small n, for tests). */
syn_graph *syn_rhg_brute(int64_t n, double avg_deg, double gamma, uint64_t seed) {
  return rhg_build(n, avg_deg, gamma, seed, 1);
}

/* ---------------------------------------------------------------- access */
int64_t syn_n(const syn_graph *g) { return g->n; }
int64_t syn_m2(const syn_graph *g) { return g->m2; }
void syn_copy(const syn_graph *g, int64_t *xadj, int32_t *adj) {
  memcpy(xadj, g->xadj, sizeof(int64_t) * (size_t)(g->n + 1));
  memcpy(adj, g->adj, sizeof(int32_t) * (size_t)g->m2);
}
void syn_free(syn_graph *g) {
  if (!g) return;
  free(g->xadj);
  free(g->adj);
  free(g);
}
