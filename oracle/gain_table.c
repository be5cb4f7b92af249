/*
 * Space-efficient gain table (Section "Space-Efficient Gain Tables").
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * The table caches the affinity w(v, V_b) = sum of w(v, x) over neighbours x
 * of v in block b, for every vertex v and block b, so that the gain of moving
 * v to b is w(v, V_b) - w(v, V_part(v)). After a move of u from block s to
 * block t, every neighbour v of u loses w(u, v) of affinity to s and gains it
 * to t.
 *
 * Memory is O(sum over v of min(deg(v), k)) instead of O(n k):
 *  - a vertex with deg(v) > k keeps k values (dense slice);
 *  - a vertex with deg(v) <= k keeps a small linear-probing hash table with a
 *    capacity proportional to its degree, holding only the blocks it has
 *    non-zero affinity to; an affinity that drops to zero is deleted, and
 *    deletion closes the gap in the probe sequence by moving later entries
 *    up (backward-shift deletion), so no tombstones are kept;
 *  - every value of v is stored in the smallest width of 8, 16, 32 or 64 bits
 *    that holds v's total incident edge weight, the upper bound of every
 *    affinity of v;
 *  - all slices live in one contiguous byte array, with a start offset per
 *    vertex.
 *
 * Readings where the paper is silent:
 *  - sparse capacity: the smallest power of two >= 2 deg(v) (load <= 1/2);
 *  - a sparse slot is a 32-bit block id (-1 = empty) followed by the value;
 *  - home slot of block b: Fibonacci hashing, the top log2(capacity) bits of
 *    b * 0x9e3779b97f4a7c15 (64-bit product), probing forward cyclically;
 *  - values are little-endian; degree-0 vertices keep no slice.
 * The paper protects each sparse table with a spinlock for concurrent moves;
 * the oracle applies moves one at a time.
 */
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

struct orc_gain_table {
  int64_t n;
  int32_t k;
  int64_t *start;  /* byte offset of v's slice in mem */
  int64_t *cap;    /* sparse: slots; dense: k; degree 0: 0 */
  uint8_t *width;  /* bytes per value: 1, 2, 4 or 8 */
  uint8_t *dense;  /* 1 iff deg(v) > k */
  uint8_t *mem;
  int64_t bytes;
};

static uint64_t load_value(const uint8_t *p, int w) {
  uint64_t x = 0;
  for (int i = 0; i < w; ++i) x |= (uint64_t)p[i] << (8 * i);
  return x;
}

static void store_value(uint8_t *p, int w, uint64_t x) {
  for (int i = 0; i < w; ++i) p[i] = (uint8_t)(x >> (8 * i));
}

static int32_t load_key(const uint8_t *p) {
  uint32_t x = 0;
  for (int i = 0; i < 4; ++i) x |= (uint32_t)p[i] << (8 * i);
  return (int32_t)x;
}

static void store_key(uint8_t *p, int32_t key) {
  for (int i = 0; i < 4; ++i) p[i] = (uint8_t)((uint32_t)key >> (8 * i));
}

static int64_t home_slot(int32_t b, int64_t cap) {
  int lg = 0;
  while (((int64_t)1 << lg) < cap) ++lg;
  uint64_t h = (uint64_t)(uint32_t)b * 0x9e3779b97f4a7c15ull;
  return lg == 0 ? 0 : (int64_t)(h >> (64 - lg));
}

static uint8_t *slot_at(const orc_gain_table *t, int64_t v, int64_t i) {
  return t->mem + t->start[v] + i * (4 + t->width[v]);
}

/* Slot of block b in v's sparse table, or -1 (then *free_slot, if given,
 * receives the empty slot where b would go). */
static int64_t find(const orc_gain_table *t, int64_t v, int32_t b, int64_t *free_slot) {
  int64_t cap = t->cap[v], i = home_slot(b, cap);
  for (int64_t probes = 0; probes < cap; ++probes, i = (i + 1) & (cap - 1)) {
    int32_t key = load_key(slot_at(t, v, i));
    if (key == b) return i;
    if (key < 0) {
      if (free_slot) *free_slot = i;
      return -1;
    }
  }
  if (free_slot) *free_slot = -1; /* full: cannot happen at load <= 1/2 */
  return -1;
}

/* Backward-shift deletion of slot i (linear probing without tombstones). */
static void erase_slot(orc_gain_table *t, int64_t v, int64_t i) {
  int64_t cap = t->cap[v], mask = cap - 1, j = i;
  int w = t->width[v];
  for (;;) {
    store_key(slot_at(t, v, i), -1);
    store_value(slot_at(t, v, i) + 4, w, 0);
    for (;;) {
      j = (j + 1) & mask;
      int32_t key = load_key(slot_at(t, v, j));
      if (key < 0) return;
      int64_t h = home_slot(key, cap);
      /* the entry at j stays iff its home lies cyclically in (i, j] */
      int stays = i <= j ? (h > i && h <= j) : (h > i || h <= j);
      if (!stays) {
        memcpy(slot_at(t, v, i), slot_at(t, v, j), (size_t)(4 + w));
        i = j;
        break;
      }
    }
  }
}

static int64_t degree(const orc_graph *g, int64_t v) { return g->xadj[v + 1] - g->xadj[v]; }

/* Adds delta (may be negative) to the affinity of v to block b. */
static void add_affinity(orc_gain_table *t, int64_t v, int32_t b, int64_t delta) {
  int w = t->width[v];
  if (t->dense[v]) {
    uint8_t *p = t->mem + t->start[v] + (int64_t)b * w;
    store_value(p, w, (uint64_t)((int64_t)load_value(p, w) + delta));
    return;
  }
  int64_t free_slot = -1;
  int64_t i = find(t, v, b, &free_slot);
  if (i < 0) { /* a new block: delta > 0 */
    store_key(slot_at(t, v, free_slot), b);
    store_value(slot_at(t, v, free_slot) + 4, w, (uint64_t)delta);
    return;
  }
  int64_t x = (int64_t)load_value(slot_at(t, v, i) + 4, w) + delta;
  if (x == 0)
    erase_slot(t, v, i);
  else
    store_value(slot_at(t, v, i) + 4, w, (uint64_t)x);
}

orc_gain_table *orc_gt_build(const orc_graph *g, const int32_t *part, int32_t k) {
  orc_gain_table *t = (orc_gain_table *)calloc(1, sizeof(*t));
  int64_t n = g->n;
  t->n = n;
  t->k = k;
  t->start = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
  t->cap = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
  t->width = (uint8_t *)malloc((size_t)n + 1);
  t->dense = (uint8_t *)malloc((size_t)n + 1);
  int64_t pos = 0;
  for (int64_t v = 0; v < n; ++v) {
    int64_t d = degree(g, v), total = 0;
    for (int64_t e = g->xadj[v]; e < g->xadj[v + 1]; ++e) total += orc_ew(g, e);
    int w = 1;
    while (w < 8 && (uint64_t)total >> (8 * w) != 0) w *= 2;
    t->width[v] = (uint8_t)w;
    t->dense[v] = d > k;
    int64_t cap = 0;
    if (d > k) {
      cap = k;
    } else if (d > 0) {
      cap = 1;
      while (cap < 2 * d) cap *= 2;
    }
    t->cap[v] = cap;
    t->start[v] = pos;
    pos += t->dense[v] ? cap * w : cap * (4 + w);
  }
  t->start[n] = pos;
  t->bytes = pos;
  t->mem = (uint8_t *)calloc((size_t)pos + 1, 1);
  for (int64_t v = 0; v < n; ++v) {
    if (t->dense[v]) continue;
    for (int64_t i = 0; i < t->cap[v]; ++i) store_key(slot_at(t, v, i), -1);
  }
  for (int64_t v = 0; v < n; ++v)
    for (int64_t e = g->xadj[v]; e < g->xadj[v + 1]; ++e) add_affinity(t, v, part[g->adj[e]], orc_ew(g, e));
  return t;
}

int64_t orc_gt_get(const orc_gain_table *t, int64_t v, int32_t b) {
  if (t->cap[v] == 0) return 0;
  int w = t->width[v];
  if (t->dense[v]) return (int64_t)load_value(t->mem + t->start[v] + (int64_t)b * w, w);
  int64_t i = find(t, v, b, NULL);
  return i < 0 ? 0 : (int64_t)load_value(slot_at(t, v, i) + 4, w);
}

void orc_gt_move(orc_gain_table *t, const orc_graph *g, int64_t u, int32_t from, int32_t to) {
  if (from == to) return;
  for (int64_t e = g->xadj[u]; e < g->xadj[u + 1]; ++e) {
    int64_t v = g->adj[e];
    add_affinity(t, v, to, orc_ew(g, e)); /* add first: a sparse table never overflows */
    add_affinity(t, v, from, -orc_ew(g, e));
  }
}

int64_t orc_gt_bytes(const orc_gain_table *t) { return t->bytes; }

void orc_gt_layout(const orc_gain_table *t, int64_t v, int64_t *cap, int32_t *width,
                   int32_t *dense, int64_t *stored) {
  *cap = t->cap[v];
  *width = t->width[v];
  *dense = t->dense[v];
  int64_t c = 0;
  if (!t->dense[v])
    for (int64_t i = 0; i < t->cap[v]; ++i) c += load_key(slot_at(t, v, i)) >= 0;
  *stored = t->dense[v] ? t->k : c;
}

int orc_gt_check(const orc_gain_table *t) {
  for (int64_t v = 0; v < t->n; ++v) {
    if (t->dense[v] || t->cap[v] == 0) continue;
    int64_t cap = t->cap[v];
    for (int64_t i = 0; i < cap; ++i) {
      int32_t key = load_key(slot_at(t, v, i));
      if (key < 0) continue;
      if (key >= t->k) return 1;
      if (load_value(slot_at(t, v, i) + 4, t->width[v]) == 0) return 2; /* stored zero */
      /* reachable: no empty slot between its home and i */
      for (int64_t j = home_slot(key, cap); j != i; j = (j + 1) & (cap - 1))
        if (load_key(slot_at(t, v, j)) < 0) return 3;
      for (int64_t j = i + 1; j < cap; ++j)
        if (load_key(slot_at(t, v, j)) == key) return 4; /* duplicate key */
    }
  }
  return 0;
}

void orc_gt_free(orc_gain_table *t) {
  if (!t) return;
  free(t->start);
  free(t->cap);
  free(t->width);
  free(t->dense);
  free(t->mem);
  free(t);
}
