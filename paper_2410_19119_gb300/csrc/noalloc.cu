// Partition metrics without any device allocation.
//
// tp_metrics needs a little device scratch (the cut accumulator and the
// per-block weight sums) and takes it from the allocator. Some callers
// cannot allocate device memory at the point where they want the metrics:
// code with a device-memory footprint fixed up front (a service that admits
// work by memory budget, or a pool that must not grow), and callers that own
// no allocator of their own. tp_metrics_static serves them: its scratch is
// the file-scope array below, so it calls no cudaMalloc, cudaFree or
// allocating library routine. It synchronises the stream to return host
// values, so it cannot be recorded into a CUDA graph; on a stream that is
// being captured it returns TP_ERR_INVALID before enqueuing anything, which
// leaves the caller's capture intact.
#include <mutex>

#include "decode.cuh"

namespace tp {
namespace {

// Largest k accepted. Scratch = 8 bytes x (2 + kStaticMaxBlocks), about
// 128 KiB, held by every GPU that loads this library until the process exits.
constexpr int32_t kStaticMaxBlocks = 16383;
constexpr int kScratchCut = 0;     // edge-cut accumulator (both directions)
constexpr int kScratchBad = 1;     // set when a block id lies outside [0, k)
constexpr int kScratchBlocks = 2;  // [2, 2 + k): block weights

__device__ __align__(256) unsigned long long g_static_scratch[kScratchBlocks + kStaticMaxBlocks];

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
unsigned long long *g_static_ptr[kMaxDevices] = {};

// Device address of the scratch array for the current device. In host code
// the array's name is only a host-side stand-in, so the address is looked up
// once per device (with that device current) and cached.
unsigned long long *scratch_address() {
  int dev = 0;
  TP_CUDA(cudaGetDevice(&dev));
  TP_REQUIRE(dev >= 0 && dev < kMaxDevices, TP_ERR_INVALID);
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_ptr[dev]) {
    void *p = nullptr;
    TP_CUDA(cudaGetSymbolAddress(&p, g_static_scratch));
    g_static_ptr[dev] = static_cast<unsigned long long *>(p);
  }
  return g_static_ptr[dev];
}

// Block ids outside [0, k) are skipped (they would index past the array)
// and flagged in bad.
__global__ void k_static_weights(const int32_t *part, const int64_t *vw, int64_t n, int32_t k,
                                 unsigned long long *B, unsigned long long *bad) {
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n;
       u += (int64_t)gridDim.x * blockDim.x) {
    const int32_t b = part[u];
    if (b < 0 || b >= k) {
      *bad = 1;
      continue;
    }
    atomicAdd(&B[b], (unsigned long long)(vw ? vw[u] : 1));
  }
}

template <bool COMP>
__global__ void k_static_cut(GView g, const int32_t *part, unsigned long long *acc) {
  int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  int64_t sum = 0;
  for (int64_t u = warp; u < g.n; u += nw) {
    int32_t pu = part[u];
    warp_neighbours<COMP>(g, u, -1, [&](bool has, int32_t v, int64_t w, int64_t) {
      if (has && part[v] != pu) sum += w;
    });
  }
  sum = warp_sum(sum);
  if (lane_id() == 0 && sum) atomicAdd(acc, (unsigned long long)sum);
}

}  // namespace
}  // namespace tp

using namespace tp;

extern "C" tp_status tp_metrics_static(const tp_graph *g, const int32_t *d_part, int32_t k,
                                       int64_t *cut, int64_t *h_block_weights, void *stream) {
  if (!g || k < 1 || (g->n && !d_part)) return TP_ERR_INVALID;
  if (k > kStaticMaxBlocks) return TP_ERR_BUDGET;
  cudaStream_t s = (cudaStream_t)stream;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) {
    (void)cudaGetLastError();
    return TP_ERR_CUDA;
  }
  if (cap != cudaStreamCaptureStatusNone) return TP_ERR_INVALID;  // nothing enqueued
  return guard([&] {
    unsigned long long *scratch = scratch_address();
    // the array keeps the previous call's sums: clear what this call uses
    TP_CUDA(cudaMemsetAsync(scratch, 0, (size_t)(kScratchBlocks + k) * sizeof(unsigned long long),
                            s));
    if (g->n) {
      launch(k_static_weights, grid_for(g->n, 256), 256, 0, s, d_part,
             g->unit_vw ? nullptr : g->vw.get(), g->n, k, scratch + kScratchBlocks,
             scratch + kScratchBad);
      unsigned blocks = grid_for(g->n * 32, 256);
      if (g->compressed)
        launch(k_static_cut<true>, blocks, 256, 0, s, view(g), d_part, scratch + kScratchCut);
      else launch(k_static_cut<false>, blocks, 256, 0, s, view(g), d_part, scratch + kScratchCut);
      TP_LAUNCH_CHECK();
    }
    unsigned long long head[2] = {0, 0};  // cut, bad-id flag
    TP_CUDA(cudaMemcpyAsync(head, scratch, sizeof(head), cudaMemcpyDeviceToHost, s));
    if (h_block_weights)
      TP_CUDA(cudaMemcpyAsync(h_block_weights, scratch + kScratchBlocks,
                              (size_t)k * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    TP_CUDA(cudaStreamSynchronize(s));
    TP_REQUIRE(head[kScratchBad] == 0, TP_ERR_INVALID);
    if (cut) *cut = (int64_t)(head[kScratchCut] / 2);
  });
}
