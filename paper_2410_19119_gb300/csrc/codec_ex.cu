// The interval + edge-weight stream on the GPU (Section "Compression Scheme"
// of the paper: runs of consecutive neighbour ids stored as intervals, after
// the WebGraph framework, and edge weights VarInt-coded and interleaved with
// the codes they belong to). The layout, which the oracle's encoder also
// writes (the tests compare the two byte for byte):
//   per vertex u: VarInt(first edge id); above 10 000 neighbours a table of
//   nchunks - 1 little-endian u32 chunk offsets relative to the vertex's
//   first byte and chunks of 1 000 neighbours (one chunk otherwise); a
//   terminal VarInt(2m) at off[n].
//   A chunk without intervals: every neighbour v in ascending order as its
//   code (the first 2|v - u| + [v < u], later the gap to the previous one),
//   followed, with weights, by VarInt(2|w - w'| + [w < w']) where w' is the
//   chunk's previous weight in storage order (0 first).
//   A chunk with intervals: VarInt(number of maximal runs of >= 3
//   consecutive ids); per run, smallest first, VarInt(start code: the first
//   run 2|x - u| + [x < u], a later one x - (previous run's end) - 2),
//   VarInt(length - 3) and, with weights, its members' weights; then the
//   remaining ids (residuals) as in a chunk without intervals.
// Without intervals and weights the stream is the plain format that the
// rating kernels read; with either, graphs are decoded to CSR here.
#include <algorithm>
#include <vector>

#include "tp_internal.cuh"

namespace tp {
tp_graph *from_csr(int64_t n, const int64_t *xadj, const int32_t *adj, const int64_t *vwgt,
                   const int64_t *ewgt, int host, cudaStream_t s);

namespace {

__device__ __forceinline__ int vbytes(uint64_t x) {
  int l = 1;
  while (x >= 128) x >>= 7, ++l;
  return l;
}

// Appends VarInt(x) at out + pos (out null: counts only).
__device__ __forceinline__ void vput(uint8_t *out, int64_t &pos, uint64_t x) {
  if (out) {
    while (x >= 128) {
      out[pos++] = (uint8_t)(x | 128u);
      x >>= 7;
    }
    out[pos++] = (uint8_t)x;
  } else {
    pos += vbytes(x);
  }
}

// Reads a VarInt from [p, lim); false if it is truncated or longer than 64 bits.
__device__ __forceinline__ bool vget(const uint8_t *bytes, int64_t &p, int64_t lim, uint64_t &x) {
  x = 0;
  for (int shift = 0; shift < 64; shift += 7) {
    if (p >= lim) return false;
    const uint8_t b = bytes[p++];
    x |= (uint64_t)(b & 127u) << shift;
    if (!(b & 128u)) return true;
  }
  return false;
}

__device__ __forceinline__ uint64_t code_from(int64_t x, int64_t ref) {
  return x >= ref ? 2ull * (uint64_t)(x - ref) : 2ull * (uint64_t)(ref - x) + 1ull;
}
__device__ __forceinline__ int64_t value_of(uint64_t c, int64_t ref) {
  return (c & 1u) ? ref - (int64_t)(c >> 1) : ref + (int64_t)(c >> 1);
}

// End of the run of consecutive ids that starts at a[i].
__device__ __forceinline__ int64_t run_end(const int32_t *a, int64_t i, int64_t cnt) {
  int64_t j = i;
  while (j + 1 < cnt && a[j + 1] == a[j] + 1) ++j;
  return j;
}

// One chunk (ids a[0..cnt) ascending, weights w or null) of vertex u at
// out + pos (out null: counts); advances pos.
__device__ void put_chunk(uint8_t *out, int64_t &pos, int64_t u, const int32_t *a,
                          const int64_t *w, int64_t cnt, bool intervals) {
  int64_t wprev = 0;
  auto put_w = [&](int64_t i) {
    if (!w) return;
    vput(out, pos, code_from(w[i], wprev));
    wprev = w[i];
  };
  if (!intervals) {
    for (int64_t i = 0; i < cnt; ++i) {
      vput(out, pos, i == 0 ? code_from(a[0], u) : (uint64_t)(a[i] - a[i - 1]));
      put_w(i);
    }
    return;
  }
  int64_t runs = 0;
  for (int64_t i = 0; i < cnt;) {
    const int64_t j = run_end(a, i, cnt);
    runs += j - i + 1 >= 3;
    i = j + 1;
  }
  vput(out, pos, (uint64_t)runs);
  int64_t prev_end = -1;
  bool first = true;
  for (int64_t i = 0; i < cnt;) {
    const int64_t j = run_end(a, i, cnt);
    if (j - i + 1 >= 3) {
      vput(out, pos, first ? code_from(a[i], u) : (uint64_t)(a[i] - prev_end - 2));
      vput(out, pos, (uint64_t)(j - i + 1 - 3));
      for (int64_t q = i; q <= j; ++q) put_w(q);
      prev_end = a[j];
      first = false;
    }
    i = j + 1;
  }
  int64_t prev = -1;
  first = true;
  for (int64_t i = 0; i < cnt;) {
    const int64_t j = run_end(a, i, cnt);
    if (j - i + 1 < 3)
      for (int64_t q = i; q <= j; ++q) {
        vput(out, pos, first ? code_from(a[q], u) : (uint64_t)(a[q] - prev));
        put_w(q);
        prev = a[q];
        first = false;
      }
    i = j + 1;
  }
}

// Vertex u's bytes at out + pos (out null: counts); returns the length.
__device__ int64_t put_vertex(uint8_t *out, int64_t pos, int64_t u, const int64_t *xadj,
                              const int32_t *adj, const int64_t *ew, bool intervals) {
  const int64_t start = pos, b = xadj[u], d = xadj[u + 1] - b;
  vput(out, pos, (uint64_t)b);
  if (d == 0) return pos - start;
  const int64_t nch = d > kChunkThreshold ? (d + kChunkSize - 1) / kChunkSize : 1;
  const int64_t csz = nch > 1 ? kChunkSize : d;
  const int64_t table = pos;
  pos += 4 * (nch - 1);
  for (int64_t j = 0; j < nch; ++j) {
    if (j > 0 && out) {
      const uint32_t rel = (uint32_t)(pos - start);
      for (int q = 0; q < 4; ++q) out[table + 4 * (j - 1) + q] = (uint8_t)(rel >> (8 * q));
    }
    const int64_t lo = b + j * csz, hi = min(lo + csz, b + d);
    put_chunk(out, pos, u, adj + lo, ew ? ew + lo : nullptr, hi - lo, intervals);
  }
  return pos - start;
}

__global__ void k_fill_one(int64_t *p, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = 1;
}

__global__ void k_ex_size(const int64_t *xadj, const int32_t *adj, const int64_t *ew, int64_t n,
                          bool intervals, uint64_t *size) {
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n;
       u += (int64_t)gridDim.x * blockDim.x)
    size[u] = (uint64_t)put_vertex(nullptr, 0, u, xadj, adj, ew, intervals);
}

__global__ void k_ex_write(const int64_t *xadj, const int32_t *adj, const int64_t *ew, int64_t n,
                           bool intervals, const uint64_t *off, uint8_t *bytes) {
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n;
       u += (int64_t)gridDim.x * blockDim.x)
    put_vertex(bytes, (int64_t)off[u], u, xadj, adj, ew, intervals);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    int64_t pos = (int64_t)off[n];
    vput(bytes, pos, (uint64_t)xadj[n]);
  }
}

// Exclusive prefix over n u64 sizes, off[n] = total (one block; encoding is
// a one-time step, and the library's scans are for signed types).
__global__ void k_ex_offsets(const uint64_t *size, int64_t n, uint64_t *off) {
  __shared__ uint64_t part[1024];
  const int64_t per = (n + blockDim.x - 1) / blockDim.x;
  const int64_t lo = min((int64_t)threadIdx.x * per, n), hi = min(lo + per, n);
  uint64_t s = 0;
  for (int64_t i = lo; i < hi; ++i) s += size[i];
  part[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint64_t run = 0;
    for (unsigned t = 0; t < blockDim.x; ++t) {
      const uint64_t v = part[t];
      part[t] = run;
      run += v;
    }
  }
  __syncthreads();
  uint64_t run = part[threadIdx.x];
  for (int64_t i = lo; i < hi; ++i) {
    off[i] = run;
    run += size[i];
  }
  if (hi == n && lo < hi) off[n] = run;
  if (n == 0 && threadIdx.x == 0) off[0] = 0;
}

// Decoder, one thread per vertex: first edge ids into xadj, neighbours and
// weights into adj / ew (scratch: the storage order of chunks with
// intervals); any inconsistency latches *bad.
__global__ void k_ex_decode(const uint8_t *bytes, int64_t nbytes, const uint64_t *off, int64_t n,
                            int64_t m2, bool intervals, bool weighted, int64_t *xadj,
                            int32_t *adj, int64_t *ew, int32_t *sid, int64_t *sw, int32_t *bad) {
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n;
       u += (int64_t)gridDim.x * blockDim.x) {
    bool ok = false;
    do {
      const int64_t p0 = (int64_t)off[u], end = (int64_t)off[u + 1];
      if (p0 > end || end >= nbytes) break;
      int64_t p = p0, q = end;
      uint64_t b, e;
      if (!vget(bytes, p, end, b) || !vget(bytes, q, nbytes, e)) break;
      if (e < b || (int64_t)e > m2) break;
      xadj[u] = (int64_t)b;
      const int64_t d = (int64_t)(e - b);
      if (d == 0) {
        ok = p == end;
        break;
      }
      const int64_t nch = d > kChunkThreshold ? (d + kChunkSize - 1) / kChunkSize : 1;
      const int64_t csz = nch > 1 ? kChunkSize : d;
      const int64_t table = p;
      p += 4 * (nch - 1);
      if (p > end) break;
      bool chunks_ok = true;
      for (int64_t j = 0; j < nch && chunks_ok; ++j) {
        if (j > 0) {
          uint32_t rel = 0;
          for (int t = 0; t < 4; ++t) rel |= (uint32_t)bytes[table + 4 * (j - 1) + t] << (8 * t);
          if (p0 + (int64_t)rel != p) {
            chunks_ok = false;
            break;
          }
        }
        const int64_t cnt = min(csz, d - j * csz), e0 = (int64_t)b + j * csz;
        int64_t wprev = 0;
        auto get_w = [&](int64_t &w) -> bool {
          if (!weighted) {
            w = 1;
            return true;
          }
          uint64_t c;
          if (!vget(bytes, p, end, c)) return false;
          w = value_of(c, wprev);
          wprev = w;
          return w >= 1;
        };
        if (!intervals) {
          int64_t prev = -1;
          for (int64_t i = 0; i < cnt && chunks_ok; ++i) {
            uint64_t c;
            int64_t w;
            if (!vget(bytes, p, end, c)) chunks_ok = false;
            const int64_t v = i == 0 ? value_of(c, u) : prev + (int64_t)c;
            if (!chunks_ok || v < 0 || v >= n || (i > 0 && c == 0) || !get_w(w)) {
              chunks_ok = false;
              break;
            }
            adj[e0 + i] = (int32_t)v;
            ew[e0 + i] = w;
            prev = v;
          }
        } else {
          uint64_t runs;
          if (!vget(bytes, p, end, runs) || (int64_t)runs > cnt / 3) {
            chunks_ok = false;
            break;
          }
          int64_t k = 0, prev_end = -1;
          for (uint64_t r = 0; r < runs && chunks_ok; ++r) {
            uint64_t c, lm3;
            if (!vget(bytes, p, end, c) || !vget(bytes, p, end, lm3) || lm3 > (uint64_t)cnt) {
              chunks_ok = false;
              break;
            }
            const int64_t x = r == 0 ? value_of(c, u) : prev_end + 2 + (int64_t)c;
            const int64_t l = (int64_t)lm3 + 3;
            if (x < 0 || k + l > cnt || x + l > n) {
              chunks_ok = false;
              break;
            }
            for (int64_t t = 0; t < l; ++t) {
              int64_t w;
              if (!get_w(w)) {
                chunks_ok = false;
                break;
              }
              sid[e0 + k] = (int32_t)(x + t);
              sw[e0 + k] = w;
              ++k;
            }
            prev_end = x + l - 1;
          }
          const int64_t ni = k;
          int64_t prev = -1;
          for (int64_t i = 0; k < cnt && chunks_ok; ++i, ++k) {
            uint64_t c;
            int64_t w;
            if (!vget(bytes, p, end, c)) {
              chunks_ok = false;
              break;
            }
            const int64_t v = i == 0 ? value_of(c, u) : prev + (int64_t)c;
            if (v < 0 || v >= n || (i > 0 && c == 0) || !get_w(w)) {
              chunks_ok = false;
              break;
            }
            sid[e0 + k] = (int32_t)v;
            sw[e0 + k] = w;
            prev = v;
          }
          if (!chunks_ok) break;
          // the ascending runs [0, ni) and residuals [ni, cnt) merged in id order
          int64_t a = 0, rr = ni;
          for (int64_t o = 0; o < cnt; ++o) {
            const bool take_a = rr >= cnt || (a < ni && sid[e0 + a] < sid[e0 + rr]);
            const int64_t s = take_a ? a++ : rr++;
            adj[e0 + o] = sid[e0 + s];
            ew[e0 + o] = sw[e0 + s];
            if (o > 0 && adj[e0 + o] <= adj[e0 + o - 1]) {  // a residual inside a run
              chunks_ok = false;
              break;
            }
          }
        }
        if (chunks_ok && j > 0 && adj[e0] <= adj[e0 - 1]) chunks_ok = false;
      }
      ok = chunks_ok && p == end;
    } while (false);
    if (!ok) atomicCAS(bad, 0, 1);
  }
}

}  // namespace

// Offsets (and, with d_bytes, the stream) of g in the interval + weight format.
uint64_t encode_ex(const tp_graph *g, bool intervals, bool weights, uint64_t *d_off,
                   uint8_t *d_bytes, cudaStream_t s) {
  TP_REQUIRE(!g->compressed, TP_ERR_INVALID);
  const int64_t n = g->n;
  Buf<int64_t> ones;
  const int64_t *ew = nullptr;
  if (weights) {
    if (g->unit_ew) {  // unit weights, stored explicitly
      ones.alloc(std::max<int64_t>(g->m2, 1), s);
      if (g->m2) {
        launch(k_fill_one, grid_for(g->m2, 256), 256, 0, s, ones.get(), g->m2);
        TP_LAUNCH_CHECK();
      }
      ew = ones.get();
    } else {
      ew = g->ew.get();
    }
  }
  Buf<uint64_t> size(std::max<int64_t>(n, 1), s);
  if (n) {
    launch(k_ex_size, grid_for(n, 128), 128, 0, s, g->xadj.get(), g->adj.get(), ew, n, intervals,
           size.get());
    TP_LAUNCH_CHECK();
  }
  launch(k_ex_offsets, 1, 1024, 0, s, size.get(), n, d_off);
  TP_LAUNCH_CHECK();
  uint64_t body = 0;
  TP_CUDA(cudaMemcpyAsync(&body, d_off + n, 8, cudaMemcpyDeviceToHost, s));
  TP_CUDA(cudaStreamSynchronize(s));
  int tail = 1;
  for (uint64_t x = (uint64_t)g->m2; x >= 128; x >>= 7) ++tail;
  if (d_bytes) {
    launch(k_ex_write, grid_for(std::max<int64_t>(n, 1), 128), 128, 0, s, g->xadj.get(),
           g->adj.get(), ew, n, intervals, d_off, d_bytes);
    TP_LAUNCH_CHECK();
    TP_CUDA(cudaStreamSynchronize(s));
  }
  return body + (uint64_t)tail;
}

// A CSR graph decoded from a stream in the interval + weight format.
tp_graph *decode_ex(int64_t n, uint64_t nbytes, const uint8_t *d_bytes, const uint64_t *d_off,
                    bool intervals, bool weighted, cudaStream_t s) {
  TP_REQUIRE(n >= 0 && n < (int64_t)INT32_MAX && d_off && (nbytes == 0 || d_bytes), TP_ERR_INVALID);
  TP_REQUIRE(nbytes >= 1, TP_ERR_CORRUPT);
  // 2m from the terminal header
  std::vector<uint64_t> hoff(2);
  TP_CUDA(cudaMemcpyAsync(hoff.data(), d_off + n, 8, cudaMemcpyDeviceToHost, s));
  TP_CUDA(cudaMemcpyAsync(hoff.data() + 1, d_off, 8, cudaMemcpyDeviceToHost, s));
  TP_CUDA(cudaStreamSynchronize(s));
  TP_REQUIRE(hoff[0] < nbytes && hoff[1] == 0, TP_ERR_CORRUPT);
  uint8_t tail[10] = {0};
  const uint64_t tl = std::min<uint64_t>(10, nbytes - hoff[0]);
  TP_CUDA(cudaMemcpyAsync(tail, d_bytes + hoff[0], tl, cudaMemcpyDeviceToHost, s));
  TP_CUDA(cudaStreamSynchronize(s));
  uint64_t m2 = 0;
  {
    uint64_t i = 0;
    int shift = 0;
    for (; i < tl; ++i, shift += 7) {
      m2 |= (uint64_t)(tail[i] & 127u) << shift;
      if (!(tail[i] & 128u)) break;
    }
    TP_REQUIRE(i < tl && hoff[0] + i + 1 == nbytes && m2 < ((uint64_t)1 << 40), TP_ERR_CORRUPT);
  }
  const int64_t M = (int64_t)m2;
  Buf<int64_t> xadj(n + 1, s), ew(std::max<int64_t>(M, 1), s), sw(std::max<int64_t>(M, 1), s);
  Buf<int32_t> adj(std::max<int64_t>(M, 1), s), sid(std::max<int64_t>(M, 1), s), bad(1, s);
  TP_CUDA(cudaMemsetAsync(bad.get(), 0, sizeof(int32_t), s));
  const int64_t m2h = M;
  TP_CUDA(cudaMemcpyAsync(xadj.get() + n, &m2h, 8, cudaMemcpyHostToDevice, s));
  if (n) {
    launch(k_ex_decode, grid_for(n, 128), 128, 0, s, d_bytes, (int64_t)nbytes, d_off, n, M,
           intervals, weighted, xadj.get(), adj.get(), ew.get(), sid.get(), sw.get(), bad.get());
    TP_LAUNCH_CHECK();
  }
  TP_REQUIRE(read_scalar(bad.get(), s) == 0, TP_ERR_CORRUPT);
  return from_csr(n, xadj.get(), adj.get(), nullptr, weighted ? ew.get() : nullptr, 0, s);
}

}  // namespace tp
