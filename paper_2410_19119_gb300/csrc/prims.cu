// Device-wide primitives: prefix scans and a stable LSD radix sort.
// Hand-written for sm_103a; used by contraction, two-hop packing, tier lists
// and initial partitioning.
#include <climits>

#include "tp_internal.cuh"

namespace tp {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

struct SumOp {
  template <class T>
  __device__ __forceinline__ T operator()(T a, T b) const { return a + b; }
  template <class T>
  __device__ __forceinline__ static T identity() { return T(0); }
};
struct MaxOp {
  template <class T>
  __device__ __forceinline__ T operator()(T a, T b) const { return a > b ? a : b; }
  template <class T>
  __device__ __forceinline__ static T identity() { return T(INT64_MIN); }
};

__device__ __forceinline__ int spad(int i) { return i + (i >> 5); }

// Block-wide scan of a tile held in shared memory (kScanTile entries, padded).
// Returns the tile aggregate; sm becomes the inclusive (or exclusive) scan.
template <class T, class Op>
__device__ T block_scan_tile(T *sm, bool exclusive, Op op) {
  __shared__ T warp_tot[kScanThreads / 32];
  int t = threadIdx.x;
  T v[kScanItems];
  T acc = Op::template identity<T>();
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    v[j] = sm[spad(t * kScanItems + j)];
    acc = op(acc, v[j]);
  }
  // warp inclusive scan of thread totals
  T x = acc;
  int l = t & 31, w = t >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(kFull, x, o);
    if (l >= o) x = op(x, y);
  }
  if (l == 31) warp_tot[w] = x;
  __syncthreads();
  if (w == 0) {
    T y = l < kScanThreads / 32 ? warp_tot[l] : Op::template identity<T>();
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      T z = __shfl_up_sync(kFull, y, o);
      if (l >= o) y = op(y, z);
    }
    if (l < kScanThreads / 32) warp_tot[l] = y;
  }
  __syncthreads();
  T total = warp_tot[kScanThreads / 32 - 1];
  T prefix = x;  // inclusive over threads <= t within warp
  // exclusive prefix of this thread = (warp prefix of previous warps) op (exclusive in warp)
  T excl_thread = __shfl_up_sync(kFull, prefix, 1);
  if (l == 0) excl_thread = Op::template identity<T>();
  if (w > 0) excl_thread = op(warp_tot[w - 1], excl_thread);
  T run = excl_thread;
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    T nv = op(run, v[j]);
    sm[spad(t * kScanItems + j)] = exclusive ? run : nv;
    run = nv;
  }
  __syncthreads();
  return total;
}

template <class Tin, class T, class Op>
__global__ void k_scan_reduce(const Tin *in, T *block_tot, int64_t n) {
  __shared__ T sm[kScanTile + kScanTile / 32];
  int64_t base = (int64_t)blockIdx.x * kScanTile;
  Op op;
  for (int j = 0; j < kScanItems; ++j) {
    int i = j * kScanThreads + threadIdx.x;
    sm[spad(i)] = base + i < n ? (T)in[base + i] : Op::template identity<T>();
  }
  __syncthreads();
  T tot = block_scan_tile<T>(sm, false, op);
  if (threadIdx.x == 0) block_tot[blockIdx.x] = tot;
}

template <class Tin, class T, class Op>
__global__ void k_scan_down(const Tin *in, T *out, const T *block_off, int64_t n, bool exclusive,
                            T *total_out) {
  __shared__ T sm[kScanTile + kScanTile / 32];
  int64_t base = (int64_t)blockIdx.x * kScanTile;
  Op op;
  for (int j = 0; j < kScanItems; ++j) {
    int i = j * kScanThreads + threadIdx.x;
    sm[spad(i)] = base + i < n ? (T)in[base + i] : Op::template identity<T>();
  }
  __syncthreads();
  T tot = block_scan_tile<T>(sm, exclusive, op);
  T off = block_off ? block_off[blockIdx.x] : Op::template identity<T>();
  for (int j = 0; j < kScanItems; ++j) {
    int i = j * kScanThreads + threadIdx.x;
    if (base + i < n) out[base + i] = op(off, sm[spad(i)]);
  }
  if (total_out && blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) *total_out = op(off, tot);
}

// Generic scan; out may alias in. total_out (device, nullable) receives the aggregate.
template <class Tin, class T, class Op>
void scan(const Tin *in, T *out, int64_t n, bool exclusive, T *total_out, cudaStream_t s) {
  if (n <= 0) {
    if (total_out) {
      T z = T(0);
      TP_CUDA(cudaMemcpyAsync(total_out, &z, sizeof(T), cudaMemcpyHostToDevice, s));
      TP_CUDA(cudaStreamSynchronize(s));
    }
    return;
  }
  int64_t tiles = (n + kScanTile - 1) / kScanTile;
  if (tiles == 1) {
    launch(k_scan_down<Tin, T, Op>, 1, kScanThreads, 0, s, in, out, nullptr, n, exclusive, total_out);
    TP_LAUNCH_CHECK();
    return;
  }
  Buf<T> tot(tiles, s);
  launch(k_scan_reduce<Tin, T, Op>, (unsigned)tiles, kScanThreads, 0, s, in, tot.get(), n);
  TP_LAUNCH_CHECK();
  scan<T, T, Op>(tot.get(), tot.get(), tiles, true, (T *)nullptr, s);
  launch(k_scan_down<Tin, T, Op>, (unsigned)tiles, kScanThreads, 0, s, in, out, tot.get(), n, exclusive,
                                                                   total_out);
  TP_LAUNCH_CHECK();
}

// ---------------------------------------------------------------- radix sort
constexpr int kSortWarps = 8;
constexpr int kSortBatches = 32;                      // 32-key batches per warp
constexpr int kSortWarpTile = 32 * kSortBatches;      // keys per warp

__global__ void k_sort_hist(const uint64_t *keys, int64_t n, int shift, int64_t nwarps,
                            uint32_t *counts) {
  __shared__ uint32_t hist[kSortWarps][256];
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  for (int i = l; i < 256; i += 32) hist[w][i] = 0;
  __syncwarp();
  int64_t gw = (int64_t)blockIdx.x * kSortWarps + w;
  int64_t base = gw * kSortWarpTile;
  for (int b = 0; b < kSortBatches; ++b) {
    int64_t i = base + (int64_t)b * 32 + l;
    unsigned active = __ballot_sync(kFull, i < n);
    if (i < n) {
      uint32_t d = (uint32_t)(keys[i] >> shift) & 255u;
      unsigned peers = __match_any_sync(active, d);
      if ((peers & lanemask_lt()) == 0) hist[w][d] += __popc(peers);
    }
    __syncwarp();
  }
  if (gw < nwarps)
    for (int d = l; d < 256; d += 32) counts[(int64_t)d * nwarps + gw] = hist[w][d];
}

__global__ void k_sort_scatter(const uint64_t *keys, const uint64_t *vals, uint64_t *okeys,
                               uint64_t *ovals, int64_t n, int shift, int64_t nwarps,
                               const int64_t *offsets) {
  __shared__ int64_t ctr[kSortWarps][256];
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  int64_t gw = (int64_t)blockIdx.x * kSortWarps + w;
  if (gw < nwarps)
    for (int d = l; d < 256; d += 32) ctr[w][d] = offsets[(int64_t)d * nwarps + gw];
  __syncwarp();
  int64_t base = gw * kSortWarpTile;
  for (int b = 0; b < kSortBatches; ++b) {
    int64_t i = base + (int64_t)b * 32 + l;
    unsigned active = __ballot_sync(kFull, i < n);
    if (i < n) {
      uint64_t k = keys[i];
      uint32_t d = (uint32_t)(k >> shift) & 255u;
      unsigned peers = __match_any_sync(active, d);
      int64_t pos = ctr[w][d] + __popc(peers & lanemask_lt());
      okeys[pos] = k;
      if (vals) ovals[pos] = vals[i];
      __syncwarp(active);
      if ((peers & lanemask_lt()) == 0) ctr[w][d] += __popc(peers);
    }
    __syncwarp();
  }
}

__global__ void k_max_i64(const int64_t *d, int64_t n, unsigned long long *out) {
  long long m = LLONG_MIN;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    m = d[i] > m ? d[i] : m;
  m = warp_max(m);
  if (lane_id() == 0) atomicMax((long long *)out, m);
}

}  // namespace

int64_t max_i64(const int64_t *d, int64_t n, cudaStream_t s) {
  if (n <= 0) return 0;
  Buf<unsigned long long> out(1, s);
  long long init = LLONG_MIN;
  TP_CUDA(cudaMemcpyAsync(out.get(), &init, sizeof(init), cudaMemcpyHostToDevice, s));
  launch(k_max_i64, grid_for(n, 256, (int64_t)num_sms() * 8), 256, 0, s, d, n, out.get());
  TP_LAUNCH_CHECK();
  return (int64_t)read_scalar(out.get(), s);
}

void exclusive_scan_i64(const int64_t *in, int64_t *out, int64_t n, cudaStream_t s) {
  scan<int64_t, int64_t, SumOp>(in, out, n, true, out + n, s);
}
void exclusive_scan_i32_to_i64(const int32_t *in, int64_t *out, int64_t n, cudaStream_t s) {
  scan<int32_t, int64_t, SumOp>(in, out, n, true, out + n, s);
}
void inclusive_max_scan_i64(const int64_t *in, int64_t *out, int64_t n, cudaStream_t s) {
  scan<int64_t, int64_t, MaxOp>(in, out, n, false, (int64_t *)nullptr, s);
}

int bits_for(uint64_t v) {
  int b = 0;
  while (b < 64 && (v >> b) != 0) ++b;
  return b;
}

void radix_sort_pairs(uint64_t *keys, uint64_t *vals, int64_t n, int bits, cudaStream_t s,
                      int lo) {
  if (n <= 1 || bits <= 0) return;
  int passes = (bits + 7) / 8;
  int64_t nwarps = (n + kSortWarpTile - 1) / kSortWarpTile;
  unsigned blocks = (unsigned)((nwarps + kSortWarps - 1) / kSortWarps);
  Buf<uint64_t> tk(n, s), tv;
  if (vals) tv.alloc(n, s);
  Buf<uint32_t> counts(256 * nwarps, s);
  Buf<int64_t> offs(256 * nwarps + 1, s);
  uint64_t *ka = keys, *kb = tk.get(), *va = vals, *vb = vals ? tv.get() : nullptr;
  for (int p = 0; p < passes; ++p) {
    int shift = lo + 8 * p;
    launch(k_sort_hist, blocks, kSortWarps * 32, 0, s, ka, n, shift, nwarps, counts.get());
    TP_LAUNCH_CHECK();
    scan<uint32_t, int64_t, SumOp>(counts.get(), offs.get(), 256 * nwarps, true,
                                   (int64_t *)nullptr, s);
    launch(k_sort_scatter, blocks, kSortWarps * 32, 0, s, ka, va, kb, vb, n, shift, nwarps,
                                                      offs.get());
    TP_LAUNCH_CHECK();
    std::swap(ka, kb);
    std::swap(va, vb);
  }
  if (ka != keys) {
    TP_CUDA(cudaMemcpyAsync(keys, ka, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
    if (vals) TP_CUDA(cudaMemcpyAsync(vals, va, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
  }
}

}  // namespace tp
