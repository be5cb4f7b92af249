/*
 * Compressed adjacency format: gap encoding + VarInt + high-degree chunks.
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Section "Compression Scheme" of the paper: each neighbourhood is sorted
 * ascending and stored as differences (gap encoding); every number is a VarInt
 * with 7 payload bits per byte and one continuation bit; neighbourhoods with
 * more than 10 000 neighbours are split into chunks of 1 000 that decode
 * independently; the neighbourhoods are concatenated and every vertex keeps a
 * pointer to its start; the first edge id of a neighbourhood is stored as a
 * VarInt in front of it so that degrees follow from consecutive headers.
 *
 * Readings where the paper is silent:
 *  - VarInt byte order is LEB128: low 7 bits first, bit 7 set on every byte
 *    except the last one of a number.
 *  - The first neighbour v0 of every chunk is stored relative to the owner u as
 *    2*|v0-u| + [v0 < u] (a sign bit in the lowest position, as for the signed
 *    edge-weight gaps the paper mentions); later neighbours of the chunk store
 *    the plain gap v_i - v_{i-1} >= 1.
 *  - A chunked neighbourhood stores, right after its header, nchunks-1 unsigned
 *    32-bit little-endian byte offsets of chunks 1..nchunks-1, measured from the
 *    neighbourhood start off[u].
 *  - off[n] points at a terminal header holding 2m, so the degree of every
 *    vertex, the last one included, is the difference of two headers.
 */
#include "oracle.h"
#include <stdlib.h>
#include <string.h>

#define CHUNK_THRESHOLD 10000
#define CHUNK_SIZE 1000

int orc_varint_len(uint64_t x) {
  int len = 1;
  while (x >= 128) {
    x >>= 7;
    ++len;
  }
  return len;
}

int orc_varint_put(uint8_t *out, uint64_t x) {
  int len = 0;
  while (x >= 128) {
    out[len++] = (uint8_t)(0x80u | (x & 0x7fu));
    x >>= 7;
  }
  out[len++] = (uint8_t)x;
  return len;
}

int orc_varint_get(const uint8_t *in, int64_t avail, uint64_t *x) {
  uint64_t v = 0;
  for (int i = 0; i < 10; ++i) {
    if (i >= avail) return 0;
    uint64_t b = in[i];
    if (i == 9 && (b & 0x7eu)) return 0; /* more than 64 bits */
    v |= (b & 0x7fu) << (7 * i);
    if (!(b & 0x80u)) {
      *x = v;
      return i + 1;
    }
  }
  return 0;
}

static uint64_t signed_first(int64_t v0, int64_t u) {
  return v0 >= u ? 2ull * (uint64_t)(v0 - u) : 2ull * (uint64_t)(u - v0) + 1ull;
}

static int64_t nchunks_of(int64_t d) {
  if (d <= CHUNK_THRESHOLD) return 1;
  return (d + CHUNK_SIZE - 1) / CHUNK_SIZE;
}

/* Byte size of one neighbourhood including its header. */
static int64_t vertex_size(int64_t u, const int64_t *xadj, const int32_t *adj) {
  int64_t b = xadj[u], d = xadj[u + 1] - b;
  int64_t size = orc_varint_len((uint64_t)b);
  if (d == 0) return size;
  int64_t nch = nchunks_of(d);
  int64_t csz = nch > 1 ? CHUNK_SIZE : d;
  size += 4 * (nch - 1);
  for (int64_t i = 0; i < d; ++i) {
    if (i % csz == 0)
      size += orc_varint_len(signed_first(adj[b + i], u));
    else
      size += orc_varint_len((uint64_t)(adj[b + i] - adj[b + i - 1]));
  }
  return size;
}

int64_t orc_encoded_size(int64_t n, const int64_t *xadj, const int32_t *adj) {
  int64_t total = 0;
  for (int64_t u = 0; u < n; ++u) total += vertex_size(u, xadj, adj);
  return total + orc_varint_len((uint64_t)xadj[n]);
}

int64_t orc_encode(int64_t n, const int64_t *xadj, const int32_t *adj, uint8_t *bytes,
                   uint64_t *off) {
  int64_t pos = 0;
  for (int64_t u = 0; u < n; ++u) {
    off[u] = (uint64_t)pos;
    int64_t b = xadj[u], d = xadj[u + 1] - b;
    pos += orc_varint_put(bytes + pos, (uint64_t)b);
    if (d == 0) continue;
    int64_t nch = nchunks_of(d);
    int64_t csz = nch > 1 ? CHUNK_SIZE : d;
    int64_t table = pos;
    pos += 4 * (nch - 1);
    for (int64_t j = 0; j < nch; ++j) {
      if (j > 0) {
        uint32_t rel = (uint32_t)(pos - (int64_t)off[u]);
        for (int q = 0; q < 4; ++q) bytes[table + 4 * (j - 1) + q] = (uint8_t)(rel >> (8 * q));
      }
      int64_t lo = b + j * csz, hi = lo + csz;
      if (hi > b + d) hi = b + d;
      pos += orc_varint_put(bytes + pos, signed_first(adj[lo], u));
      for (int64_t e = lo + 1; e < hi; ++e)
        pos += orc_varint_put(bytes + pos, (uint64_t)(adj[e] - adj[e - 1]));
    }
  }
  off[n] = (uint64_t)pos;
  pos += orc_varint_put(bytes + pos, (uint64_t)xadj[n]);
  return pos;
}

int orc_decode(int64_t n, const uint8_t *bytes, int64_t nbytes, const uint64_t *off,
               int64_t *xadj_out, int32_t *adj_out, int64_t adj_cap) {
  uint64_t first = 0, next = 0;
  for (int64_t u = 0; u <= n; ++u) {
    if ((int64_t)off[u] >= nbytes) return -1;
    if (u > 0 && off[u] < off[u - 1]) return -1;
  }
  if (!orc_varint_get(bytes + off[0], nbytes - (int64_t)off[0], &first) || first != 0) return -1;
  for (int64_t u = 0; u < n; ++u) {
    int64_t p = (int64_t)off[u];
    int hl = orc_varint_get(bytes + p, nbytes - p, &first);
    if (!hl) return -1;
    if (!orc_varint_get(bytes + off[u + 1], nbytes - (int64_t)off[u + 1], &next)) return -1;
    if (next < first || (int64_t)next > adj_cap) return -1;
    xadj_out[u] = (int64_t)first;
    int64_t d = (int64_t)(next - first);
    int64_t end = (int64_t)off[u + 1];
    p += hl;
    if (d == 0) {
      if (p != end) return -1;
      continue;
    }
    int64_t nch = nchunks_of(d);
    int64_t csz = nch > 1 ? CHUNK_SIZE : d;
    int64_t table = p;
    p += 4 * (nch - 1);
    if (p > end) return -1;
    int64_t e = (int64_t)first, prev = -1;
    for (int64_t j = 0; j < nch; ++j) {
      if (j > 0) {
        uint32_t rel = 0;
        for (int q = 0; q < 4; ++q) rel |= (uint32_t)bytes[table + 4 * (j - 1) + q] << (8 * q);
        if ((int64_t)off[u] + (int64_t)rel != p) return -1;
      }
      int64_t cnt = d - j * csz < csz ? d - j * csz : csz;
      for (int64_t i = 0; i < cnt; ++i) {
        uint64_t x;
        int l = orc_varint_get(bytes + p, end - p, &x);
        if (!l) return -1;
        p += l;
        int64_t v;
        if (i == 0)
          v = (x & 1u) ? u - (int64_t)(x >> 1) : u + (int64_t)(x >> 1);
        else
          v = prev + (int64_t)x;
        if (v < 0 || v >= n || v <= prev || (x == 0 && i > 0)) return -1;
        adj_out[e++] = (int32_t)v;
        prev = v;
      }
    }
    if (p != end) return -1;
  }
  if (!orc_varint_get(bytes + off[n], nbytes - (int64_t)off[n], &next)) return -1;
  xadj_out[n] = (int64_t)next;
  return 0;
}
