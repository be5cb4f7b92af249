// Neighbourhood access for CSR and for the compressed format (Section
// "Compression Scheme" of the paper: gap + VarInt, first edge id header,
// chunks of 1000 neighbours above degree 10000).
//
// The compressed decoder is warp-cooperative: a warp reads a 32-byte window
// of the stream (one byte per lane, coalesced), finds value ends with a
// ballot of the continuation bits, lets the lane holding the last byte of a
// value assemble it from up to four preceding lanes by shuffles, and turns
// gaps into neighbour ids with a warp prefix sum. Each window yields up to 32
// neighbour ids, one per lane, delivered to the caller as a batch.
#pragma once
#include "tp_internal.cuh"

namespace tp {

// Single-thread VarInt read (up to 10 bytes). Returns bytes consumed.
__device__ __forceinline__ int read_varint(const uint8_t *p, uint64_t &x) {
  uint64_t v = 0;
  int i = 0;
  for (; i < 10; ++i) {
    uint64_t b = p[i];
    v |= (b & 0x7fu) << (7 * i);
    if (!(b & 0x80u)) break;
  }
  x = v;
  return i + 1;
}

__device__ __forceinline__ uint64_t off_at(const GView &g, int64_t u) {
  return g.off32 ? (uint64_t)g.off32[u] : g.off64[u];
}

// Layout of one compressed neighbourhood.
struct ZipNbr {
  uint64_t begin;  // byte offset of u's record
  uint64_t data;   // first byte after header and chunk table
  uint64_t end;    // one past the last byte
  int64_t first;   // first edge id
  int64_t deg;
  int64_t nchunks;
};

__device__ __forceinline__ ZipNbr zip_nbr(const GView &g, int64_t u) {
  ZipNbr z;
  z.begin = off_at(g, u);
  z.end = off_at(g, u + 1);
  uint64_t a, b;
  int hl = read_varint(g.bytes + z.begin, a);
  read_varint(g.bytes + z.end, b);
  z.first = (int64_t)a;
  z.deg = (int64_t)(b - a);
  z.nchunks = z.deg > kChunkThreshold ? (z.deg + kChunkSize - 1) / kChunkSize : 1;
  z.data = z.begin + hl + 4 * (z.nchunks - 1);
  return z;
}

__device__ __forceinline__ uint32_t read_u32le(const uint8_t *p) {
  return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}

// Byte range and neighbour count of chunk j of a compressed neighbourhood.
__device__ __forceinline__ void zip_chunk(const GView &g, const ZipNbr &z, int64_t j, uint64_t &cb,
                                          uint64_t &ce, int64_t &cnt) {
  if (z.nchunks == 1) {
    cb = z.data, ce = z.end, cnt = z.deg;
    return;
  }
  const uint8_t *tab = g.bytes + z.begin + (z.data - z.begin - 4 * (z.nchunks - 1));
  cb = j == 0 ? z.data : z.begin + read_u32le(tab + 4 * (j - 1));
  ce = j + 1 < z.nchunks ? z.begin + read_u32le(tab + 4 * j) : z.end;
  int64_t rest = z.deg - j * kChunkSize;
  cnt = rest < kChunkSize ? rest : kChunkSize;
}

// Decodes `count` neighbour ids of u from the chunk occupying bytes
// [p, end). f(bool has, int32_t v) is called by every lane once per window.
// Returns false (and latches TP_ERR_CORRUPT) on a malformed chunk.
template <class F>
__device__ __forceinline__ bool warp_decode_chunk(const GView &g, int64_t u, uint64_t p,
                                                  uint64_t end, int64_t count, F &&f) {
  const int lane = lane_id();
  int64_t done = 0, prev = 0;
  bool first = true;
  while (done < count) {
    uint64_t q = p + lane;
    uint32_t b = q < end ? (uint32_t)g.bytes[q] : 0x80u;  // past the end: never a value end
    unsigned endmask = __ballot_sync(kFull, !(b & 0x80u));
    int64_t rem = count - done;
    if (__popc(endmask) > rem) {  // only on a malformed chunk: keep the first rem ends
      unsigned m = endmask, keep = 0;
      for (int64_t i = 0; i < rem; ++i) {
        unsigned low = m & (0u - m);
        keep |= low;
        m ^= low;
      }
      endmask = keep;
    }
    if (endmask == 0) {
      if (lane == 0) latch_error(g.err, TP_ERR_CORRUPT);
      return false;
    }
    unsigned below = endmask & lanemask_lt();
    int s = below ? 32 - __clz(below) : 0;  // first lane of my value
    uint32_t pay = b & 0x7fu;
    uint64_t val = 0;
#pragma unroll
    for (int d = 0; d < 5; ++d) {
      uint32_t pb = __shfl_up_sync(kFull, pay, d);
      int src = lane - d;
      if (src >= s && src >= 0) val |= (uint64_t)pb << (7 * (src - s));
    }
    bool mine = (endmask >> lane) & 1u;
    bool bad = mine && (lane - s >= 5);
    int64_t c = 0;
    if (mine) {
      if (first && below == 0) {
        c = (val & 1u) ? u - (int64_t)(val >> 1) : u + (int64_t)(val >> 1);
      } else {
        c = (int64_t)val;
        bad |= val == 0;  // gaps of a sorted duplicate-free list are >= 1
      }
    }
    int64_t v = (first ? 0 : prev) + warp_incl_scan(c);
    bad |= mine && (v < 0 || v >= g.n);
    if (__any_sync(kFull, bad)) {
      if (lane == 0) latch_error(g.err, TP_ERR_CORRUPT);
      return false;
    }
    f(mine, (int32_t)v);
    int last = 31 - __clz(endmask);
    prev = __shfl_sync(kFull, v, last);
    first = false;
    done += __popc(endmask);
    p += (uint64_t)last + 1;
  }
  if (p != end) {
    if (lane == 0) latch_error(g.err, TP_ERR_CORRUPT);
    return false;
  }
  return true;
}

// Visits the neighbours of u in warp-wide batches: f(bool has, int32_t v,
// int64_t w). For CSR the batch is 32 consecutive entries; for the
// compressed format it is one decoded window of one chunk. chunk < 0 visits
// the whole neighbourhood; otherwise only chunk `chunk` (chunks of
// kChunkSize entries, for CSR as well).
template <bool COMP, class F>
__device__ __forceinline__ void warp_neighbours(const GView &g, int64_t u, int64_t chunk, F &&f) {
  const int lane = lane_id();
  if (!COMP) {
    int64_t b = g.xadj[u], e = g.xadj[u + 1];
    if (chunk >= 0) {
      b += chunk * kChunkSize;
      e = b + kChunkSize < e ? b + kChunkSize : e;
    }
    for (int64_t i = b; i < e; i += 32) {
      int64_t k = i + lane;
      bool has = k < e;
      int32_t v = has ? g.adj[k] : 0;
      int64_t w = (has && g.ew) ? g.ew[k] : 1;
      f(has, v, w);
    }
  } else {
    ZipNbr z = zip_nbr(g, u);
    if (z.deg == 0) return;
    int64_t j0 = chunk >= 0 ? chunk : 0, j1 = chunk >= 0 ? chunk + 1 : z.nchunks;
    for (int64_t j = j0; j < j1; ++j) {
      uint64_t cb, ce;
      int64_t cnt;
      zip_chunk(g, z, j, cb, ce, cnt);
      if (!warp_decode_chunk(g, u, cb, ce, cnt, [&](bool has, int32_t v) { f(has, v, (int64_t)1); }))
        return;
    }
  }
}

// Visits the neighbours of u with a single thread: f(int32_t v, int64_t w).
// Only for vertices that are not chunked (degree <= 10000 in the compressed
// format). The adjacency is read with evict-first loads (it is streamed once
// per pass); compressed streams were validated when the graph was created,
// so ids are only clamped into [0, n) to keep later accesses in bounds.
// Returns the degree.
template <bool COMP, class F>
__device__ __forceinline__ int64_t thread_neighbours(const GView &g, int64_t u, F &&f) {
  if (!COMP) {
    const int64_t b = __ldcs(g.xadj + u), e = __ldcs(g.xadj + u + 1);
    for (int64_t k = b; k < e; ++k) f(__ldcs(g.adj + k), g.ew ? __ldcs(g.ew + k) : (int64_t)1);
    return e - b;
  }
  const uint64_t b = g.off32 ? (uint64_t)__ldcs(g.off32 + u) : __ldcs(g.off64 + u);
  const uint64_t e = g.off32 ? (uint64_t)__ldcs(g.off32 + u + 1) : __ldcs(g.off64 + u + 1);
  const int32_t nmax = (int32_t)(g.n - 1);
  const uint32_t *wp = reinterpret_cast<const uint32_t *>(g.bytes + (b & ~(uint64_t)3));
  uint32_t word = __ldcs(wp) >> (8 * (b & 3));
  uint32_t nextw = __ldcs(wp + 1);
  int left = 4 - (int)(b & 3);     // bytes still unread in `word`
  int remaining = (int)(e - b);    // one record (degree <= 10000) is far below 2^31 bytes
  while (remaining > 0) {  // header (first edge id): skip to its last byte
    const uint32_t byte = word & 255u;
    word >>= 8;
    --remaining;
    if (--left == 0) word = nextw, nextw = __ldcs(++wp + 1), left = 4;
    if (!(byte & 0x80u)) break;
  }
  uint32_t val = 0;
  int shift = 0, cnt = 0;
  int32_t prev = (int32_t)u;
  bool first = true;
  while (remaining > 0) {
    const uint32_t byte = word & 255u;
    word >>= 8;
    --remaining;
    if (--left == 0) word = nextw, nextw = __ldcs(++wp + 1), left = 4;  // padded stream
    val |= (byte & 0x7fu) << shift;
    shift += 7;
    if (byte & 0x80u) continue;
    int32_t v = first ? ((val & 1u) ? prev - (int32_t)(val >> 1) : prev + (int32_t)(val >> 1))
                      : prev + (int32_t)val;
    v = min(max(v, 0), nmax);
    first = false;
    prev = v;
    f(v, (int64_t)1);
    ++cnt;
    val = 0;
    shift = 0;
  }
  return cnt;
}

}  // namespace tp
