/*
 * Compressed adjacency with interval encoding and compressed edge weights.
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Section "Compression Scheme" of the paper, the two parts that the plain
 * gap + VarInt format (codec.c) leaves out:
 *  - interval encoding (after the WebGraph framework): a run of l >= 3
 *    consecutive neighbour ids {x, x+1, ..., x+l-1} is stored as the pair
 *    (x, l) instead of l gaps of one;
 *  - edge weights are gap encoded with VarInt as well, with a sign bit since
 *    they are not sorted, and are stored interleaved with the gaps and the
 *    intervals of their neighbourhood.
 * Header (first edge id), chunking of neighbourhoods above 10 000 neighbours
 * into chunks of 1 000 with a table of u32 chunk offsets, the terminal header
 * and the VarInt byte order are those of codec.c.
 *
 * Readings where the paper is silent:
 *  - A chunk with intervals starts with VarInt(number of intervals). The
 *    intervals are the maximal runs of at least three consecutive ids inside
 *    the chunk, taken from the smallest id up. Interval j is
 *    VarInt(start code) VarInt(l - 3); the start code of the first interval
 *    is 2|x - u| + [x < u], of a later one x - (end of the previous
 *    interval) - 2, which is >= 0 because maximal runs are separated by at
 *    least one missing id.
 *  - The remaining ids of the chunk (residuals) follow in ascending order as
 *    in codec.c: the first as 2|v - u| + [v < u], later ones as the gap to the
 *    previous residual (>= 1). Their count is the chunk's size minus the
 *    interval lengths, so it is not stored.
 *  - Weights follow the code they belong to: an interval's l weights follow
 *    its length, a residual's weight follows its gap. Each weight is stored
 *    as 2|w - w'| + [w < w'], w' the previous weight of the chunk in storage
 *    order (0 before the first), so that chunks decode independently.
 *  - Without intervals a chunk is the plain format of codec.c with the
 *    weights interleaved; without weights as well it is byte for byte the
 *    plain format.
 */
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

#define CHUNK_THRESHOLD 10000
#define CHUNK_SIZE 1000

static uint64_t signed_code(int64_t x, int64_t ref) {
  return x >= ref ? 2ull * (uint64_t)(x - ref) : 2ull * (uint64_t)(ref - x) + 1ull;
}

static int64_t unsigned_code(uint64_t c, int64_t ref) {
  return (c & 1u) ? ref - (int64_t)(c >> 1) : ref + (int64_t)(c >> 1);
}

static int64_t nchunks_of(int64_t d) {
  if (d <= CHUNK_THRESHOLD) return 1;
  return (d + CHUNK_SIZE - 1) / CHUNK_SIZE;
}

/* Appends x as a VarInt at out[*pos] (out may be NULL: only counts). */
static void put(uint8_t *out, int64_t *pos, uint64_t x) {
  if (out)
    *pos += orc_varint_put(out + *pos, x);
  else
    *pos += orc_varint_len(x);
}

static void put_weight(uint8_t *out, int64_t *pos, const int64_t *w, int64_t i, int64_t *wprev) {
  if (!w) return;
  put(out, pos, signed_code(w[i], *wprev));
  *wprev = w[i];
}

/* One chunk: ids a[0..cnt) ascending, weights w (or NULL), owner u. */
static void put_chunk(uint8_t *out, int64_t *pos, int64_t u, const int32_t *a, const int64_t *w,
                      int64_t cnt, int intervals) {
  int64_t wprev = 0;
  if (!intervals) {
    for (int64_t i = 0; i < cnt; ++i) {
      put(out, pos, i == 0 ? signed_code(a[0], u) : (uint64_t)(a[i] - a[i - 1]));
      put_weight(out, pos, w, i, &wprev);
    }
    return;
  }
  /* mark the members of maximal runs of length >= 3 */
  char *in_run = (char *)calloc((size_t)cnt + 1, 1);
  int64_t nint = 0;
  for (int64_t i = 0; i < cnt;) {
    int64_t j = i;
    while (j + 1 < cnt && a[j + 1] == a[j] + 1) ++j;
    if (j - i + 1 >= 3) {
      ++nint;
      for (int64_t q = i; q <= j; ++q) in_run[q] = 1;
    }
    i = j + 1;
  }
  put(out, pos, (uint64_t)nint);
  int64_t prev_end = -1;
  int first = 1;
  for (int64_t i = 0; i < cnt;) {
    if (!in_run[i]) {
      ++i;
      continue;
    }
    int64_t j = i;
    while (j + 1 < cnt && in_run[j + 1] && a[j + 1] == a[j] + 1) ++j;
    put(out, pos, first ? signed_code(a[i], u) : (uint64_t)(a[i] - prev_end - 2));
    put(out, pos, (uint64_t)(j - i + 1 - 3));
    for (int64_t q = i; q <= j; ++q) put_weight(out, pos, w, q, &wprev);
    prev_end = a[j];
    first = 0;
    i = j + 1;
  }
  int64_t prev = -1;
  first = 1;
  for (int64_t i = 0; i < cnt; ++i) {
    if (in_run[i]) continue;
    put(out, pos, first ? signed_code(a[i], u) : (uint64_t)(a[i] - prev));
    put_weight(out, pos, w, i, &wprev);
    prev = a[i];
    first = 0;
  }
  free(in_run);
}

int64_t orc_encode_ex(int64_t n, const int64_t *xadj, const int32_t *adj, const int64_t *ew,
                      int intervals, uint8_t *bytes, uint64_t *off) {
  int64_t pos = 0;
  for (int64_t u = 0; u < n; ++u) {
    if (off) off[u] = (uint64_t)pos;
    const int64_t start = pos;
    int64_t b = xadj[u], d = xadj[u + 1] - b;
    put(bytes, &pos, (uint64_t)b);
    if (d == 0) continue;
    int64_t nch = nchunks_of(d);
    int64_t csz = nch > 1 ? CHUNK_SIZE : d;
    int64_t table = pos;
    pos += 4 * (nch - 1);
    for (int64_t j = 0; j < nch; ++j) {
      if (j > 0 && bytes) {
        uint32_t rel = (uint32_t)(pos - start);
        for (int q = 0; q < 4; ++q) bytes[table + 4 * (j - 1) + q] = (uint8_t)(rel >> (8 * q));
      }
      int64_t lo = b + j * csz, hi = lo + csz < b + d ? lo + csz : b + d;
      put_chunk(bytes, &pos, u, adj + lo, ew ? ew + lo : NULL, hi - lo, intervals);
    }
  }
  if (off) off[n] = (uint64_t)pos;
  put(bytes, &pos, (uint64_t)xadj[n]);
  return pos;
}

/* Reads one VarInt from [*p, end); 0 on error. */
static int get(const uint8_t *bytes, int64_t *p, int64_t end, uint64_t *x) {
  int l = orc_varint_get(bytes + *p, end - *p, x);
  *p += l;
  return l;
}

static int get_weight(const uint8_t *bytes, int64_t *p, int64_t end, int weighted,
                      int64_t *wprev, int64_t *w) {
  if (!weighted) {
    *w = 1;
    return 1;
  }
  uint64_t x;
  if (!get(bytes, p, end, &x)) return 0;
  *w = unsigned_code(x, *wprev);
  if (*w < 1) return 0; /* weights are positive */
  *wprev = *w;
  return 1;
}

/* Decodes one chunk of cnt neighbours of u into ids/ws (ascending ids).
 * Returns 0 on success, -1 on a malformed chunk. */
static int get_chunk(const uint8_t *bytes, int64_t *p, int64_t end, int64_t n, int64_t u,
                     int64_t cnt, int intervals, int weighted, int32_t *ids, int64_t *ws) {
  int64_t wprev = 0;
  if (!intervals) {
    int64_t prev = -1;
    for (int64_t i = 0; i < cnt; ++i) {
      uint64_t x;
      if (!get(bytes, p, end, &x)) return -1;
      int64_t v = i == 0 ? unsigned_code(x, u) : prev + (int64_t)x;
      if (v < 0 || v >= n || (i > 0 && x == 0)) return -1;
      if (!get_weight(bytes, p, end, weighted, &wprev, &ws[i])) return -1;
      ids[i] = (int32_t)v;
      prev = v;
    }
    return 0;
  }
  uint64_t nint;
  if (!get(bytes, p, end, &nint) || (int64_t)nint > cnt / 3) return -1;
  /* intervals first (storage order), then residuals; merged afterwards */
  int32_t *sid = (int32_t *)malloc(sizeof(int32_t) * (size_t)(cnt + 1));
  int64_t *sw = (int64_t *)malloc(sizeof(int64_t) * (size_t)(cnt + 1));
  int64_t k = 0, prev_end = -1, ni = 0;
  int ok = 0;
  for (uint64_t j = 0; j < nint; ++j) {
    uint64_t c, lm3;
    if (!get(bytes, p, end, &c) || !get(bytes, p, end, &lm3)) goto done;
    int64_t x = j == 0 ? unsigned_code(c, u) : prev_end + 2 + (int64_t)c;
    if (lm3 > (uint64_t)cnt) goto done;
    int64_t l = (int64_t)lm3 + 3;
    if (x < 0 || k + l > cnt || x + l > n) goto done;
    for (int64_t q = 0; q < l; ++q) {
      sid[k] = (int32_t)(x + q);
      if (!get_weight(bytes, p, end, weighted, &wprev, &sw[k])) goto done;
      ++k;
    }
    prev_end = x + l - 1;
  }
  ni = k;
  {
    int64_t prev = -1;
    for (int64_t i = 0; k < cnt; ++i, ++k) {
      uint64_t x;
      if (!get(bytes, p, end, &x)) goto done;
      int64_t v = i == 0 ? unsigned_code(x, u) : prev + (int64_t)x;
      if (v < 0 || v >= n || (i > 0 && x == 0)) goto done;
      sid[k] = (int32_t)v;
      if (!get_weight(bytes, p, end, weighted, &wprev, &sw[k])) goto done;
      prev = v;
    }
  }
  {
    /* merge the ascending interval ids [0, ni) and residuals [ni, cnt) */
    int64_t a = 0, r = ni;
    for (int64_t o = 0; o < cnt; ++o) {
      int take_a = r >= cnt || (a < ni && sid[a] < sid[r]);
      int64_t s = take_a ? a++ : r++;
      ids[o] = sid[s];
      ws[o] = sw[s];
      if (o > 0 && ids[o] <= ids[o - 1]) goto done; /* a residual inside an interval */
    }
  }
  ok = 1;
done:
  free(sid);
  free(sw);
  return ok ? 0 : -1;
}

int orc_decode_ex(int64_t n, const uint8_t *bytes, int64_t nbytes, const uint64_t *off,
                  int intervals, int weighted, int64_t *xadj_out, int32_t *adj_out,
                  int64_t *ew_out, int64_t adj_cap) {
  uint64_t first = 0, next = 0;
  for (int64_t u = 0; u <= n; ++u) {
    if ((int64_t)off[u] >= nbytes) return -1;
    if (u > 0 && off[u] < off[u - 1]) return -1;
  }
  if (!orc_varint_get(bytes + off[0], nbytes - (int64_t)off[0], &first) || first != 0) return -1;
  int64_t *wtmp = (int64_t *)malloc(sizeof(int64_t) * (size_t)(CHUNK_THRESHOLD + 1));
  int rc = -1;
  for (int64_t u = 0; u < n; ++u) {
    int64_t p = (int64_t)off[u];
    if (!get(bytes, &p, nbytes, &first)) goto out;
    if (!orc_varint_get(bytes + off[u + 1], nbytes - (int64_t)off[u + 1], &next)) goto out;
    if (next < first || (int64_t)next > adj_cap) goto out;
    xadj_out[u] = (int64_t)first;
    int64_t d = (int64_t)(next - first), end = (int64_t)off[u + 1];
    if (d == 0) {
      if (p != end) goto out;
      continue;
    }
    int64_t nch = nchunks_of(d);
    int64_t csz = nch > 1 ? CHUNK_SIZE : d;
    int64_t table = p;
    p += 4 * (nch - 1);
    if (p > end) goto out;
    for (int64_t j = 0; j < nch; ++j) {
      if (j > 0) {
        uint32_t rel = 0;
        for (int q = 0; q < 4; ++q) rel |= (uint32_t)bytes[table + 4 * (j - 1) + q] << (8 * q);
        if ((int64_t)off[u] + (int64_t)rel != p) goto out;
      }
      int64_t cnt = d - j * csz < csz ? d - j * csz : csz;
      int64_t e0 = (int64_t)first + j * csz;
      if (get_chunk(bytes, &p, end, n, u, cnt, intervals, weighted, adj_out + e0, wtmp)) goto out;
      if (j > 0 && adj_out[e0] <= adj_out[e0 - 1]) goto out; /* chunks continue ascending */
      if (ew_out) memcpy(ew_out + e0, wtmp, sizeof(int64_t) * (size_t)cnt);
    }
    if (p != end) goto out;
  }
  if (!orc_varint_get(bytes + off[n], nbytes - (int64_t)off[n], &next)) goto out;
  xadj_out[n] = (int64_t)next;
  rc = 0;
out:
  free(wtmp);
  return rc;
}
