// Neighbourhood access for CSR and for the compressed format (Section
// "Compression Scheme" of the paper: gap + VarInt, first edge id header,
// chunks of 1000 neighbours above degree 10000).
//
// The compressed decoder is warp-cooperative: a warp reads a 128-byte window
// of the stream (one aligned word per lane, coalesced), assembles every
// value in the lane holding its last byte, and turns gaps into neighbour ids
// with warp prefix sums. A window yields up to 128 ids, up to four per lane,
// delivered to the caller in four batches.
#pragma once
#include "tp_internal.cuh"

namespace tp {

// Single-thread VarInt read (up to 10 bytes). Returns bytes consumed. The
// stream is padded with zero bytes, so all ten bytes a VarInt may span are
// loaded at once (one memory round trip instead of one per byte).
__device__ __forceinline__ int read_varint(const uint8_t *p, uint64_t &x) {
  uint32_t b[10];
#pragma unroll
  for (int i = 0; i < 10; ++i) b[i] = p[i];
  uint64_t v = 0;
  int len = 10;
  bool open = true;
#pragma unroll
  for (int i = 0; i < 10; ++i) {
    if (open) v |= (uint64_t)(b[i] & 0x7fu) << (7 * i);
    if (open && !(b[i] & 0x80u)) len = i + 1, open = false;
  }
  x = v;
  return len;
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
  int hl = read_varint(g.bytes + z.begin, a);  // both headers' loads are independent
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
// [p, end), 128 bytes per warp step: every lane loads one aligned 32-bit
// word (bytes before p are turned into value ends that are discarded, bytes
// from end on into continuation bytes), and for each byte that ends a value
// assembles the value from it and the (at most four) continuation bytes
// before it, which lie in its own word or the previous lane's. A warp scan
// of the values per lane gives their indices, a second one the prefix sums
// of the gaps. f(bool has, int32_t v, int64_t idx) is called by every lane
// four times per step (the lane's first..fourth value of the step, or
// has = false); idx is the value's position in the chunk. Returns false
// (and latches TP_ERR_CORRUPT) on a malformed chunk.
template <class F>
__device__ __forceinline__ bool warp_decode_chunk(const GView &g, int64_t u, uint64_t p,
                                                  uint64_t end, int64_t count, F &&f) {
  const int lane = lane_id();
  int64_t done = 0;
  int64_t prev = 0;  // id of the last value of the previous step
  while (done < count) {
    const uint64_t base = p & ~(uint64_t)3;
    const uint64_t q = base + 4 * (uint64_t)lane;
    uint32_t w = q < end ? *reinterpret_cast<const uint32_t *>(g.bytes + q) : 0x80808080u;
    // bytes before p: value ends (0x00), discarded below; from end on: continuation
    uint32_t lead = 0;  // bytes of w before p
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const uint64_t qj = q + j;
      if (qj < p) w &= ~(0xffu << (8 * j)), lead |= 1u << j;
      else if (qj >= end) w |= 0x80u << (8 * j);
    }
    const uint32_t prevw = __shfl_up_sync(kFull, w, 1);
    const uint32_t prev2 = __shfl_up_sync(kFull, w, 2);
    const uint32_t pw = lane >= 1 ? prevw : 0u;  // bytes before the window: value ends
    const uint32_t pw2 = lane >= 2 ? prev2 : 0u;
    const uint64_t cat = (uint64_t)w << 32 | pw;  // bytes of pw then w, in stream order
    uint32_t val[4];
    uint32_t ends = 0;  // real value ends of this lane (bit j: byte j)
    bool bad = false;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const uint32_t bj = (w >> (8 * j)) & 0xffu;
      // the four bytes before byte j, the nearest in bits 0..7
      const uint32_t win = __byte_perm((uint32_t)(cat >> (8 * j)), 0, 0x0123);
      const uint32_t stop = ~win & 0x80808080u;
      const int k = stop ? (__ffs(stop) - 8) >> 3 : 4;
      uint32_t pk = (win & 0x7fu) | ((win >> 1) & 0x3f80u) | ((win >> 2) & 0x1fc000u) |
                    ((win >> 3) & 0xfe00000u);
      uint32_t v = bj & 0x7fu;
#pragma unroll
      for (int d = 0; d < 4; ++d) {
        v = d < k ? (v << 7) | (pk & 0x7fu) : v;
        pk >>= 7;
      }
      val[j] = v;
      const bool is_end = !(bj & 0x80u) && !((lead >> j) & 1u);
      ends |= (uint32_t)is_end << j;
      // a fifth continuation byte: the value is longer than a VarInt of 32 bits
      const uint32_t fifth = j >= 1 ? (pw >> (8 * (j - 1))) & 0xffu : (pw2 >> 24) & 0xffu;
      bad |= is_end && k == 4 && (fifth & 0x80u);
    }
    const uint32_t nl = __popc(ends);
    const uint32_t incl = warp_incl_scan(nl);
    const uint32_t total = __shfl_sync(kFull, incl, 31);
    if (total == 0 || done + total > count) bad = true;
    // gap sums: the chunk's first value is the signed offset from u
    int64_t gs = 0;
    int64_t ids[4];
    {
      uint32_t idx = incl - nl;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        if (!((ends >> j) & 1u)) continue;
        const bool first = done == 0 && idx == 0;
        if (!first) {
          gs += val[j];
          bad |= val[j] == 0;  // gaps of a sorted duplicate-free list are >= 1
        }
        ++idx;
      }
    }
    const int64_t gincl = warp_incl_scan(gs);
    int64_t run = (done == 0 ? 0 : prev) + gincl - gs;
    {
      uint32_t idx = incl - nl;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        ids[j] = 0;
        if (!((ends >> j) & 1u)) continue;
        if (done == 0 && idx == 0) {
          run = (val[j] & 1u) ? u - (int64_t)(val[j] >> 1) : u + (int64_t)(val[j] >> 1);
          // the first value's offset feeds every later id of this step
        } else {
          run += val[j];
        }
        ids[j] = run;
        bad |= run < 0 || run >= g.n;
        ++idx;
      }
    }
    if (done == 0) {
      // ids after the first value were summed without its offset: add it
      const uint32_t owner = __ffs(__ballot_sync(kFull, nl > 0)) - 1;
      const int64_t id0 = __shfl_sync(kFull, ((ends & 1u) ? ids[0] : (ends & 2u) ? ids[1]
                                                     : (ends & 4u) ? ids[2] : ids[3]),
                                      owner);
      if (lane != (int)owner) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          ids[j] += id0;
          bad |= ((ends >> j) & 1u) && (ids[j] < 0 || ids[j] >= g.n);
        }
      }
    }
    if (__any_sync(kFull, bad)) {
      if (lane == 0) latch_error(g.err, TP_ERR_CORRUPT);
      return false;
    }
    {
      uint32_t idx = incl - nl;
      uint32_t e = ends;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const bool has = e != 0;
        const int b = has ? __ffs(e) - 1 : 0;
        e &= e - 1;
        const int64_t v = b == 0 ? ids[0] : b == 1 ? ids[1] : b == 2 ? ids[2] : ids[3];
        f(has, (int32_t)v, done + (int64_t)idx);
        idx += has;
      }
    }
    // the last value of the step continues into the next one
    const uint32_t lastlane = 31 - __clz(__ballot_sync(kFull, nl > 0));
    const int hb = 31 - __clz(__shfl_sync(kFull, ends, lastlane));
    const int64_t lastid = __shfl_sync(kFull, hb == 0 ? ids[0] : hb == 1 ? ids[1] : hb == 2 ? ids[2] : ids[3], lastlane);
    prev = lastid;
    done += total;
    p = base + 4 * (uint64_t)lastlane + (uint64_t)hb + 1;
  }
  if (p != end) {
    if (lane == 0) latch_error(g.err, TP_ERR_CORRUPT);
    return false;
  }
  return true;
}

// Visits the neighbours of u in warp-wide batches: f(bool has, int32_t v,
// int64_t w, int64_t idx), idx = position of v in u's neighbourhood (the
// batches are not in neighbourhood order for the compressed format). For
// CSR a batch is 32 consecutive entries; for the compressed format a
// decoder step calls f four times. chunk < 0 visits the whole
// neighbourhood; otherwise only chunk `chunk` (chunks of kChunkSize
// entries, for CSR as well).
template <bool COMP, class F>
__device__ __forceinline__ void warp_neighbours(const GView &g, int64_t u, int64_t chunk, F &&f) {
  const int lane = lane_id();
  if (!COMP) {
    const int64_t b0 = g.xadj[u];
    int64_t b = b0, e = g.xadj[u + 1];
    if (chunk >= 0) {
      b += chunk * kChunkSize;
      e = b + kChunkSize < e ? b + kChunkSize : e;
    }
    for (int64_t i = b; i < e; i += 32) {
      int64_t k = i + lane;
      bool has = k < e;
      int32_t v = has ? g.adj[k] : 0;
      int64_t w = (has && g.ew) ? g.ew[k] : 1;
      f(has, v, w, k - b0);
    }
  } else {
    ZipNbr z = zip_nbr(g, u);
    if (z.deg == 0) return;
    int64_t j0 = chunk >= 0 ? chunk : 0, j1 = chunk >= 0 ? chunk + 1 : z.nchunks;
    for (int64_t j = j0; j < j1; ++j) {
      uint64_t cb, ce;
      int64_t cnt;
      zip_chunk(g, z, j, cb, ce, cnt);
      const int64_t at = j * kChunkSize;
      if (!warp_decode_chunk(g, u, cb, ce, cnt,
                             [&](bool has, int32_t v, int64_t i) { f(has, v, (int64_t)1, at + i); }))
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
