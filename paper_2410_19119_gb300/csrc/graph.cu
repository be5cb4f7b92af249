// Graph handles: creation and validation, degrees and degree tiers, the
// compressed format (Section "Compression Scheme") and the small ABI calls.
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <unordered_map>
#include <mutex>
#include <new>

#include "decode.cuh"

namespace tp {

// ---------------------------------------------------------------- allocator
namespace {
// The current hook; hooks are immutable and never freed (buffers keep
// pointing at the one that made them). Null functions: cudaMallocAsync.
const AllocHook g_default_hook{nullptr, nullptr, nullptr};
std::atomic<const AllocHook *> g_hook{&g_default_hook};
std::atomic<int> g_sms{0};
}  // namespace

// Device bytes this host thread holds and its high-water mark (a call runs
// on one thread, so the peak of its working set is the mark's rise), and the
// most it may hold (mem_cap; an allocation beyond it fails with TP_ERR_BUDGET
// before anything is allocated).
thread_local int64_t t_live = 0, t_peak = 0, t_cap = INT64_MAX;

void mem_cap(int64_t bytes_above_now) {
  t_cap = bytes_above_now < 0 ? INT64_MAX : t_live + bytes_above_now;
}

int64_t mem_mark() {
  t_peak = t_live;
  return t_live;
}
int64_t mem_peak_since(int64_t mark) { return t_peak - mark; }

// Opt-in (environment TP_MEM_TRACE=1): the sizes of the buffers live at this
// thread's high-water mark, printed by mem_trace_dump (a diagnostic of what a
// call's peak consists of).
static bool mem_trace_on() {
  static const bool on = getenv("TP_MEM_TRACE") != nullptr;
  return on;
}
thread_local std::unordered_map<void *, int64_t> *t_live_bufs = nullptr;
thread_local std::vector<int64_t> *t_peak_bufs = nullptr;

static void mem_add(int64_t b) {
  t_live += b;
  if (t_live > t_peak) {
    t_peak = t_live;
    if (mem_trace_on() && t_live_bufs) {
      if (!t_peak_bufs) t_peak_bufs = new std::vector<int64_t>();
      t_peak_bufs->clear();
      for (const auto &kv : *t_live_bufs) t_peak_bufs->push_back(kv.second);
    }
  }
}

static void mem_track(void *p, int64_t b) {
  if (!mem_trace_on()) return;
  if (!t_live_bufs) t_live_bufs = new std::unordered_map<void *, int64_t>();
  if (b > 0) (*t_live_bufs)[p] = b;
  else t_live_bufs->erase(p);
}

void mem_trace_dump(const char *what) {
  if (!mem_trace_on() || !t_peak_bufs) return;
  std::vector<int64_t> v = *t_peak_bufs;
  std::sort(v.begin(), v.end(), std::greater<int64_t>());
  fprintf(stderr, "terapart mem: %s peak %.3f GB in %zu buffers; largest (GB):", what,
          (double)t_peak / 1e9, v.size());
  for (size_t i = 0; i < v.size() && i < 16; ++i) fprintf(stderr, " %.3f", (double)v[i] / 1e9);
  fprintf(stderr, "\n");
}

void *dev_alloc(size_t bytes, cudaStream_t s, const AllocHook **from) {
  if (bytes == 0) return nullptr;
  if (t_live + (int64_t)bytes > t_cap) throw Error{TP_ERR_BUDGET};
  void *p = nullptr;
  const AllocHook *h = g_hook.load();
  if (h->alloc) {
    p = h->alloc(bytes, (void *)s, h->ctx);
    if (!p) throw Error{TP_ERR_OOM};
  } else {
    cudaError_t e = cudaMallocAsync(&p, bytes, s);
    if (e != cudaSuccess) {
      (void)cudaGetLastError();
      throw Error{e == cudaErrorMemoryAllocation ? TP_ERR_OOM : TP_ERR_CUDA};
    }
  }
  mem_track(p, (int64_t)bytes);
  mem_add((int64_t)bytes);
  *from = h;
  return p;
}

void dev_free(void *p, size_t bytes, cudaStream_t s, const AllocHook *from) {
  if (!p) return;
  t_live -= (int64_t)bytes;
  mem_track(p, 0);
  if (from && from->free) {
    from->free(p, bytes, (void *)s, from->ctx);
    return;
  }
  cudaFreeAsync(p, s);
}

namespace {
std::atomic<uint64_t> g_launches{0};

struct ProfRecord {
  int family;
  cudaEvent_t a, b;
  double bytes;
};
// The profiler serves one host thread at a time (benchmarks); the scope flag
// is per thread so concurrent partitions (tp_partition_batch) never record.
thread_local bool t_prof_scope = false;
struct Profiler {
  bool enabled = false;
  std::vector<ProfRecord> recs;
  std::vector<cudaEvent_t> pool;
  cudaEvent_t open[PF_COUNT] = {};
  cudaEvent_t get() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e;
    TP_CUDA(cudaEventCreate(&e));
    return e;
  }
} g_prof;
}  // namespace

// Launches recorded into a CUDA graph are counted when the graph runs.
thread_local bool t_capturing = false;
thread_local uint64_t t_captured = 0;
void count_launch() {
  if (t_capturing) ++t_captured;
  else g_launches.fetch_add(1, std::memory_order_relaxed);
}
void count_launches(uint64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
uint64_t capture_counting(bool on) {
  t_capturing = on;
  if (on) t_captured = 0;
  return t_captured;
}
bool prof_active() { return t_prof_scope && g_prof.enabled; }
void prof_scope(bool on) { t_prof_scope = on; }
void prof_begin(int family, cudaStream_t s) {
  if (!prof_active()) return;
  cudaEvent_t e = g_prof.get();
  TP_CUDA(cudaEventRecord(e, s));
  g_prof.open[family] = e;
}
void prof_end(int family, cudaStream_t s, double alg_bytes) {
  if (!prof_active() || !g_prof.open[family]) return;
  cudaEvent_t e = g_prof.get();
  TP_CUDA(cudaEventRecord(e, s));
  g_prof.recs.push_back({family, g_prof.open[family], e, alg_bytes});
  g_prof.open[family] = nullptr;
}

int num_sms() {
  int v = g_sms.load(std::memory_order_relaxed);
  if (!v) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    if (v <= 0) v = 1;
    g_sms.store(v, std::memory_order_relaxed);  // every thread computes the same value
  }
  return v;
}

GView view(const tp_graph *g) {
  GView v;
  v.n = g->n;
  v.m2 = g->m2;
  v.xadj = g->xadj.get();
  v.adj = g->adj.get();
  v.vw = g->unit_vw ? nullptr : g->vw.get();
  v.ew = g->unit_ew ? nullptr : g->ew.get();
  v.bytes = g->bytes.get();
  v.off32 = g->off_is64 ? nullptr : g->off32.get();
  v.off64 = g->off_is64 ? g->off64.get() : nullptr;
  v.compressed = g->compressed;
  v.err = g->err.get();
  return v;
}

tp_graph *new_graph() { return new tp_graph(); }

// ---------------------------------------------------------------- reductions
namespace {

__global__ void k_sum_max(const int64_t *vw, const int64_t *xadj, int64_t n, int64_t *out) {
  // out[0] += sum vw (or n if vw null); out[1] = max degree
  int64_t s = 0, m = 0;
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n;
       u += (int64_t)gridDim.x * blockDim.x) {
    s += vw ? vw[u] : 1;
    if (xadj) {
      int64_t d = xadj[u + 1] - xadj[u];
      m = d > m ? d : m;
    }
  }
  s = warp_sum(s);
  m = warp_max(m);
  if (lane_id() == 0) {
    atomicAdd((unsigned long long *)&out[0], (unsigned long long)s);
    atomicMax((long long *)&out[1], (long long)m);
  }
}

// Structural validation of a CSR graph, one warp per vertex.
__global__ void k_validate(GView g, int32_t *bad) {
  int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  int lane = lane_id();
  if (warp == 0 && lane == 0 && (g.xadj[0] != 0 || g.xadj[g.n] != g.m2)) atomicCAS(bad, 0, 1);
  for (int64_t u = warp; u < g.n; u += nw) {
    int64_t b = g.xadj[u], e = g.xadj[u + 1];
    int code = 0;
    if (e < b || b < 0 || e > g.m2) code = 2;
    if (!code && g.vw && lane == 0 && g.vw[u] <= 0) code = 3;
    for (int64_t i = b + lane; !code && i < e; i += 32) {
      int64_t v = g.adj[i];
      if (v < 0 || v >= g.n) {
        code = 4;
        break;
      }
      if (v == u) code = 5;
      else if (i > b && g.adj[i - 1] >= v) code = 6;
      else if (g.ew && g.ew[i] <= 0) code = 7;
      else {
        // u must appear in N(v) with the same weight
        int64_t lo = g.xadj[v], hi = g.xadj[v + 1];
        while (lo < hi) {
          int64_t mid = lo + (hi - lo) / 2;
          if (g.adj[mid] < u) lo = mid + 1;
          else hi = mid;
        }
        if (lo >= g.xadj[v + 1] || g.adj[lo] != u) code = 8;
        else if (g.ew && g.ew[lo] != g.ew[i]) code = 8;
      }
    }
    if (code) atomicCAS(bad, 0, code);
  }
}

__global__ void k_zip_degrees(GView g, int64_t *deg) {
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < g.n;
       u += (int64_t)gridDim.x * blockDim.x) {
    uint64_t a, b;
    read_varint(g.bytes + off_at(g, u), a);
    read_varint(g.bytes + off_at(g, u + 1), b);
    deg[u] = (int64_t)(b - a);
  }
}

__global__ void k_csr_degrees(const int64_t *xadj, int64_t n, int64_t *deg) {
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n;
       u += (int64_t)gridDim.x * blockDim.x)
    deg[u] = xadj[u + 1] - xadj[u];
}

}  // namespace

void compute_degrees(const tp_graph *g, int64_t *d_deg, cudaStream_t s) {
  if (g->n == 0) return;
  GView v = view(g);
  if (g->compressed)
    launch(k_zip_degrees, grid_for(g->n, 256), 256, 0, s, v, d_deg);
  else
    launch(k_csr_degrees, grid_for(g->n, 256), 256, 0, s, g->xadj.get(), g->n, d_deg);
  TP_LAUNCH_CHECK();
}

// ---------------------------------------------------------------- tiers
namespace {

// Compressed lane-tier records longer than this take the decoder that loads
// beyond its 80-byte window; they join the lane tier only where they are
// common (skewed graphs: long gaps), else the warp tier rates them.
constexpr uint64_t kLaneShortRecord = 65;

// Lane-tier candidates (degree <= lane_max) and how many have long records.
__global__ void k_lane_records(const int64_t *deg, int64_t n, int32_t lane_max,
                               const uint32_t *off32, const uint64_t *off64,
                               unsigned long long *cnt) {
  unsigned long long a = 0, l = 0;
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n;
       u += (int64_t)gridDim.x * blockDim.x) {
    if (deg[u] > lane_max) continue;
    const uint64_t len = off32 ? (uint64_t)(off32[u + 1] - off32[u]) : off64[u + 1] - off64[u];
    ++a;
    l += len > kLaneShortRecord;
  }
  a = warp_sum(a);
  l = warp_sum(l);
  if (lane_id() == 0 && a) atomicAdd(&cnt[0], a);
  if (lane_id() == 0 && l) atomicAdd(&cnt[1], l);
}

__global__ void k_classify(const int64_t *deg, int64_t n, int32_t lane_max, int32_t small_max,
                           int32_t mid_max, const uint32_t *off32, const uint64_t *off64,
                           bool long_records, uint8_t *tier, int32_t *flag_small,
                           int32_t *flag_mid, int32_t *flag_mid2, int32_t *flag_big0,
                           int32_t *flag_big1, int32_t *flag_big,
                           int32_t *flag_big2, int32_t *flag_huge, unsigned long long *stats) {
  int64_t e[5] = {0, 0, 0, 0, 0}, c[5] = {0, 0, 0, 0, 0};
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n;
       u += (int64_t)gridDim.x * blockDim.x) {
    int64_t d = deg[u];
    bool lane = lane_max > 0 && d <= lane_max;
    if (lane && !long_records && (off32 || off64)) {
      const uint64_t len = off32 ? (uint64_t)(off32[u + 1] - off32[u]) : off64[u + 1] - off64[u];
      lane = len <= kLaneShortRecord;
    }
    uint8_t t = lane ? TIER_LANE
                : d <= small_max ? TIER_SMALL
                : d <= mid_max ? TIER_MID
                : d <= kChunkThreshold ? TIER_BIG
                               : TIER_HUGE;
    tier[u] = t;
    flag_small[u] = t == TIER_SMALL;
    flag_mid[u] = t == TIER_MID && d <= kMidSplit;
    flag_mid2[u] = t == TIER_MID && d > kMidSplit;
    flag_big0[u] = t == TIER_BIG && d <= kBigTinySplit;
    flag_big1[u] = t == TIER_BIG && d > kBigTinySplit && d <= kBigMidSplit;
    flag_big[u] = t == TIER_BIG && d > kBigMidSplit && d <= kBigSplit;
    flag_big2[u] = t == TIER_BIG && d > kBigSplit;
    flag_huge[u] = t == TIER_HUGE;
    e[t] += d;
    c[t] += 1;
  }
  for (int t = 0; t < 5; ++t) {
    int64_t v = warp_sum(e[t]), w = warp_sum(c[t]);
    if (lane_id() == 0 && v) atomicAdd(&stats[t], (unsigned long long)v);
    if (lane_id() == 0 && w) atomicAdd(&stats[5 + t], (unsigned long long)w);
  }
}

__global__ void k_compact(const int32_t *flag, const int64_t *pos, int64_t n, int32_t *out) {
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n;
       u += (int64_t)gridDim.x * blockDim.x)
    if (flag[u]) out[pos[u]] = (int32_t)u;
}

// Table capacity per listed vertex: the smallest power of two >= 2*deg.
__global__ void k_table_caps(const int32_t *list, int64_t cnt, const int64_t *deg, int64_t *slots,
                             int32_t *logcap, int64_t *chunks) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt;
       i += (int64_t)gridDim.x * blockDim.x) {
    int64_t d = deg[list[i]];
    int lc = 1;
    while (((int64_t)1 << lc) < 2 * d) ++lc;
    logcap[i] = lc;
    slots[i] = (int64_t)1 << lc;
    if (chunks) chunks[i] = (d + kChunkSize - 1) / kChunkSize;
  }
}

// Segments per huge table (tables above kSegLog slots are cut into segments).
__global__ void k_table_segs(const int32_t *logcap, int64_t cnt, int64_t *segs) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt;
       i += (int64_t)gridDim.x * blockDim.x)
    segs[i] = logcap[i] - 1 > kSegLog ? (int64_t)1 << (logcap[i] - 1 - kSegLog) : 1;  // list = half
}

__global__ void k_fill_table(int32_t *keys, int64_t *vals, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    keys[i] = -1;
    vals[i] = 0;
  }
}

}  // namespace

void build_tiers(tp_graph *g, const tp_params &p, cudaStream_t s) {
  TierCache &T = g->tiers;
  // the lane tier rates with one lane per vertex and needs unit edge weights
  const bool lane_ok = g->unit_ew || g->max_ew < kLaneMaxEdgeWeight;
  int32_t lane_max = lane_ok ? std::max(0, std::min(p.tier_lane, kLaneMaxDeg)) : 0;
  int32_t small_max = std::max(lane_max, std::min(p.tier_small, 64));
  int32_t mid_max = std::max(small_max, std::min(p.tier_mid, 512));  // tables of 1024 slots
  if (T.built && T.small_max == small_max && T.mid_max == mid_max && T.lane_max == lane_max) return;
  // the old cache is freed on this call's stream: the stream it was built on
  // may be gone (calls on one graph are ordered by the caller)
  T.rehome(s);
  T = TierCache();
  T.lane_max = lane_max;
  T.small_max = small_max;
  T.mid_max = mid_max;
  int64_t n = g->n;
  T.tier.alloc(n, s);
  if (n == 0) {
    T.built = true;
    return;
  }
  Buf<int64_t> deg(n, s);
  compute_degrees(g, deg.get(), s);
  Buf<int32_t> fs(n, s), fm(n, s), fm2(n, s), fb0(n, s), fb1(n, s), fb(n, s), fb2(n, s), fh(n, s);
  Buf<unsigned long long> te(10, s);
  TP_CUDA(cudaMemsetAsync(te.get(), 0, 10 * sizeof(unsigned long long), s));
  const uint32_t *o32 = g->compressed && !g->off_is64 ? g->off32.get() : nullptr;
  const uint64_t *o64 = g->compressed && g->off_is64 ? g->off64.get() : nullptr;
  bool long_records = false;
  if ((o32 || o64) && lane_max > 0) {  // long lane records where more than 5% are long
    launch(k_lane_records, grid_for(n, 256), 256, 0, s, deg.get(), n, lane_max, o32, o64, te.get());
    unsigned long long lc[2];
    TP_CUDA(cudaMemcpyAsync(lc, te.get(), sizeof(lc), cudaMemcpyDeviceToHost, s));
    TP_CUDA(cudaStreamSynchronize(s));
    long_records = lc[1] * 20 > lc[0];
    T.lane_long = long_records;
    TP_CUDA(cudaMemsetAsync(te.get(), 0, 2 * sizeof(unsigned long long), s));
  }
  launch(k_classify, grid_for(n, 256), 256, 0, s, deg.get(), n, lane_max, small_max, mid_max,
         o32, o64, long_records, T.tier.get(), fs.get(), fm.get(), fm2.get(), fb0.get(), fb1.get(),
         fb.get(), fb2.get(), fh.get(), te.get());
  TP_LAUNCH_CHECK();
  unsigned long long hte[10];
  TP_CUDA(cudaMemcpyAsync(hte, te.get(), sizeof(hte), cudaMemcpyDeviceToHost, s));
  TP_CUDA(cudaStreamSynchronize(s));
  for (int t = 0; t < 5; ++t) T.edges[t] = (int64_t)hte[t], T.count[t] = (int64_t)hte[5 + t];
  Buf<int64_t> pos(n + 1, s);
  auto make_list = [&](Buf<int32_t> &flag, Buf<int32_t> &list, int64_t &cnt) {
    exclusive_scan_i32_to_i64(flag.get(), pos.get(), n, s);
    cnt = read_scalar(pos.get() + n, s);
    list.alloc(cnt, s);
    if (cnt) {
      launch(k_compact, grid_for(n, 256), 256, 0, s, flag.get(), pos.get(), n, list.get());
      TP_LAUNCH_CHECK();
    }
  };
  make_list(fs, T.small, T.n_small);
  make_list(fm, T.mid, T.n_mid);
  make_list(fm2, T.mid2, T.n_mid2);
  make_list(fb0, T.big0, T.n_big0);
  make_list(fb1, T.big1, T.n_big1);
  make_list(fb, T.big, T.n_big);
  make_list(fb2, T.big2, T.n_big2);
  make_list(fh, T.huge, T.n_huge);
  // global rating tables for the huge tier (the big tier rates in shared memory)
  auto tables = [&](Buf<int32_t> &list, int64_t cnt, Buf<int64_t> &toff, Buf<int32_t> &tcap,
                    int64_t &slots, Buf<int64_t> *chunk_start, int64_t *nchunks) {
    toff.alloc(cnt + 1, s);
    tcap.alloc(std::max<int64_t>(cnt, 1), s);
    slots = 0;
    if (!cnt) return;
    Buf<int64_t> ch;
    if (chunk_start) {
      chunk_start->alloc(cnt + 1, s);
      ch.alloc(cnt, s);
    }
    launch(k_table_caps, grid_for(cnt, 256), 256, 0, s, list.get(), cnt, deg.get(), toff.get(),
                                                      tcap.get(), chunk_start ? ch.get() : nullptr);
    TP_LAUNCH_CHECK();
    exclusive_scan_i64(toff.get(), toff.get(), cnt, s);
    slots = read_scalar(toff.get() + cnt, s);
    if (chunk_start) {
      exclusive_scan_i64(ch.get(), chunk_start->get(), cnt, s);
      *nchunks = read_scalar(chunk_start->get() + cnt, s);
    }
  };
  tables(T.huge, T.n_huge, T.huge_toff, T.huge_tcap, T.huge_slots, &T.huge_chunk_start,
         &T.n_huge_chunks);
  if (T.n_huge) {
    T.huge_seg_start.alloc(T.n_huge + 1, s);
    launch(k_table_segs, grid_for(T.n_huge, 256), 256, 0, s, T.huge_tcap.get(), T.n_huge,
           T.huge_seg_start.get());
    TP_LAUNCH_CHECK();
    exclusive_scan_i64(T.huge_seg_start.get(), T.huge_seg_start.get(), T.n_huge, s);
    T.n_huge_segs = read_scalar(T.huge_seg_start.get() + T.n_huge, s);
    T.huge_seg_best.alloc((size_t)T.n_huge_segs * kSegBestBytes, s);
  }
  if (T.huge_slots) {
    T.tcount.alloc(std::max<int64_t>(T.n_huge, 1), s);
    TP_CUDA(cudaMemsetAsync(T.tcount.get(), 0, sizeof(int32_t) * std::max<int64_t>(T.n_huge, 1), s));
  }
  T.built = true;
}

// The hubs' global rating tables (2 to 4 slots of 14 bytes per hub
// neighbour) exist only while a rating call needs them: allocated empty on
// first use, left empty by every rating launch, freed when the call ends.
void ensure_hub_tables(tp_graph *g, cudaStream_t s) {
  TierCache &T = g->tiers;
  const int64_t total = T.huge_slots;
  if (!total || T.tkeys.get()) return;
  T.tkeys.alloc(total, s);
  T.tvals.alloc(total, s);
  T.tlist.alloc(total / 2 + 1, s);
  launch(k_fill_table, grid_for(total, 256), 256, 0, s, T.tkeys.get(), T.tvals.get(), total);
  TP_LAUNCH_CHECK();
}

void release_hub_tables(tp_graph *g, cudaStream_t s) {
  TierCache &T = g->tiers;
  T.tkeys.s = T.tvals.s = T.tlist.s = s;
  T.tkeys.release();
  T.tvals.release();
  T.tlist.release();
}

// ---------------------------------------------------------------- compression
namespace {

__device__ __forceinline__ int vlen(uint64_t x) {
  int l = 1;
  while (x >= 128) x >>= 7, ++l;
  return l;
}

__device__ __forceinline__ uint64_t first_code(int64_t v0, int64_t u) {
  return v0 >= u ? 2ull * (uint64_t)(v0 - u) : 2ull * (uint64_t)(u - v0) + 1ull;
}

constexpr int64_t kZipLaneMax = 256;  // thread per vertex up to this degree

// Encoded size of every neighbourhood of degree <= kZipLaneMax, one thread
// per vertex (the warp kernel below takes the rest).
__global__ void k_zip_size_lane(GView g, int64_t *size) {
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < g.n;
       u += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = g.xadj[u], d = g.xadj[u + 1] - b;
    if (d > kZipLaneMax) continue;
    int64_t acc = vlen((uint64_t)b);
    int32_t prev = 0;
    for (int64_t i = 0; i < d; ++i) {
      const int32_t v = g.adj[b + i];
      acc += i == 0 ? vlen(first_code(v, u)) : vlen((uint64_t)(v - prev));
      prev = v;
    }
    size[u] = acc;
  }
}

// Writes every neighbourhood of degree <= kZipLaneMax, one thread per vertex.
__global__ void k_zip_write_lane(GView g, const int64_t *off, uint8_t *out) {
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < g.n;
       u += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = g.xadj[u], d = g.xadj[u + 1] - b;
    if (d > kZipLaneMax) continue;
    uint64_t p = (uint64_t)off[u];
    auto put = [&](uint64_t x) {
      while (x >= 128) {
        out[p++] = (uint8_t)(0x80u | (x & 0x7fu));
        x >>= 7;
      }
      out[p++] = (uint8_t)x;
    };
    put((uint64_t)b);
    int32_t prev = 0;
    for (int64_t i = 0; i < d; ++i) {
      const int32_t v = g.adj[b + i];
      put(i == 0 ? first_code(v, u) : (uint64_t)(v - prev));
      prev = v;
    }
  }
}

// Encoded size of every neighbourhood above kZipLaneMax (warp per vertex).
__global__ void k_zip_size(GView g, int64_t *size) {
  int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  int lane = lane_id();
  for (int64_t u = warp; u < g.n; u += nw) {
    int64_t b = g.xadj[u], d = g.xadj[u + 1] - b;
    if (d <= kZipLaneMax) continue;
    int64_t nch = d > kChunkThreshold ? (d + kChunkSize - 1) / kChunkSize : 1;
    int64_t csz = nch > 1 ? kChunkSize : d;
    int64_t acc = 0;
    for (int64_t i = lane; i < d; i += 32) {
      int64_t v = g.adj[b + i];
      acc += (i % csz == 0) ? vlen(first_code(v, u)) : vlen((uint64_t)(v - g.adj[b + i - 1]));
    }
    acc = warp_sum(acc);
    if (lane == 0) size[u] = acc + vlen((uint64_t)b) + (d ? 4 * (nch - 1) : 0);
  }
}

// Writes every neighbourhood above kZipLaneMax at its offset (warp per vertex).
__global__ void k_zip_write(GView g, const int64_t *off, uint8_t *out) {
  int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  int lane = lane_id();
  for (int64_t u = warp; u < g.n; u += nw) {
    int64_t b = g.xadj[u], d = g.xadj[u + 1] - b;
    if (d <= kZipLaneMax) continue;
    uint64_t pos = (uint64_t)off[u];
    int hl = vlen((uint64_t)b);
    if (lane == 0) {
      uint64_t x = (uint64_t)b;
      for (int i = 0; i < hl; ++i, x >>= 7) out[pos + i] = (uint8_t)((x & 0x7f) | (i + 1 < hl ? 0x80 : 0));
    }
    if (d == 0) continue;
    int64_t nch = d > kChunkThreshold ? (d + kChunkSize - 1) / kChunkSize : 1;
    int64_t csz = nch > 1 ? kChunkSize : d;
    uint64_t p = pos + hl + 4 * (nch - 1);
    for (int64_t i0 = 0; i0 < d; i0 += 32) {
      int64_t i = i0 + lane;
      uint64_t x = 0;
      int len = 0;
      if (i < d) {
        int64_t v = g.adj[b + i];
        x = (i % csz == 0) ? first_code(v, u) : (uint64_t)(v - g.adj[b + i - 1]);
        len = vlen(x);
      }
      int incl = warp_incl_scan(len);
      uint64_t at = p + (uint64_t)(incl - len);
      if (i < d) {
        for (int q = 0; q < len; ++q, x >>= 7)
          out[at + q] = (uint8_t)((x & 0x7f) | (q + 1 < len ? 0x80 : 0));
        if (i % csz == 0 && i > 0) {
          uint32_t rel = (uint32_t)(at - pos);
          uint64_t t = pos + hl + 4 * (i / csz - 1);
          for (int q = 0; q < 4; ++q) out[t + q] = (uint8_t)(rel >> (8 * q));
        }
      }
      p += (uint64_t)__shfl_sync(kFull, incl, 31);
    }
  }
}

__global__ void k_zip_terminal(uint64_t pos, int64_t m2, uint8_t *out) {
  uint64_t x = (uint64_t)m2;
  int l = vlen(x);
  for (int i = 0; i < l; ++i, x >>= 7) out[pos + i] = (uint8_t)((x & 0x7f) | (i + 1 < l ? 0x80 : 0));
}

__global__ void k_off_narrow(const int64_t *off, int64_t cnt, uint32_t *o32) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt;
       i += (int64_t)gridDim.x * blockDim.x)
    o32[i] = (uint32_t)off[i];
}

__global__ void k_off_narrow_u64(const uint64_t *off, int64_t cnt, uint32_t *o32) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt;
       i += (int64_t)gridDim.x * blockDim.x)
    o32[i] = (uint32_t)off[i];
}

__global__ void k_off_copy(const int64_t *off, int64_t cnt, uint64_t *o64) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt;
       i += (int64_t)gridDim.x * blockDim.x)
    o64[i] = (uint64_t)off[i];
}

// Decode every neighbourhood into CSR (round trip), warp per vertex.
__global__ void k_unzip(GView g, const int64_t *xadj, int32_t *adj) {
  int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t u = warp; u < g.n; u += nw) {
    const int64_t pos = xadj[u];
    const int64_t deg = xadj[u + 1] - pos;
    int64_t seen = 0;
    warp_neighbours<true>(g, u, -1, [&](bool has, int32_t v, int64_t, int64_t idx) {
      if (has && idx < deg) adj[pos + idx] = v;
      seen += __popc(__ballot_sync(kFull, has));
    });
    if (lane_id() == 0 && seen != deg) latch_error(g.err, TP_ERR_CORRUPT);
  }
}

__global__ void k_zip_header_check(GView g, int32_t *bad) {
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < g.n;
       u += (int64_t)gridDim.x * blockDim.x) {
    uint64_t a, b;
    if (off_at(g, u + 1) < off_at(g, u)) {
      atomicCAS(bad, 0, 1);
      continue;
    }
    read_varint(g.bytes + off_at(g, u), a);
    read_varint(g.bytes + off_at(g, u + 1), b);
    if (b < a || (u == 0 && a != 0)) atomicCAS(bad, 0, 1);
  }
}

__global__ void k_widen(const uint32_t *a, uint64_t *b, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    b[i] = a[i];
}

__global__ void k_ones(int64_t *p, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = 1;
}

}  // namespace

static void finish_graph_stats(tp_graph *g, cudaStream_t s) {
  Buf<int64_t> acc(2, s);
  TP_CUDA(cudaMemsetAsync(acc.get(), 0, 2 * sizeof(int64_t), s));
  if (g->n) {
    launch(k_sum_max, grid_for(g->n, 256), 256, 0, s, g->unit_vw ? nullptr : g->vw.get(),
                                                    g->compressed ? nullptr : g->xadj.get(), g->n,
                                                    acc.get());
    TP_LAUNCH_CHECK();
  }
  int64_t h[2];
  TP_CUDA(cudaMemcpyAsync(h, acc.get(), sizeof(h), cudaMemcpyDeviceToHost, s));
  TP_CUDA(cudaStreamSynchronize(s));
  g->total_vw = h[0];
  if (!g->compressed) g->max_deg = h[1];
  g->max_ew = g->unit_ew ? 1 : max_i64(g->ew.get(), g->m2, s);
}

// Offsets are u32 while the byte stream is below 4 GiB, else u64. Setting
// TP_OFFSETS_U64=1 in the environment selects u64 offsets for any stream, so
// that the wide-offset path can be checked on small graphs.
static bool wide_offsets(uint64_t nbytes) {
  if (nbytes >= (1ull << 32)) return true;
  const char *e = getenv("TP_OFFSETS_U64");
  return e && e[0] == '1' && e[1] == 0;
}

tp_graph *compress(const tp_graph *c, cudaStream_t s) {
  TP_REQUIRE(!c->compressed && c->unit_ew && c->unit_vw, TP_ERR_INVALID);
  tp_graph *z = new_graph();
  try {
    z->n = c->n;
    z->m2 = c->m2;
    z->compressed = 1;
    z->max_deg = c->max_deg;
    z->err.alloc(1, s);
    TP_CUDA(cudaMemsetAsync(z->err.get(), 0, sizeof(int32_t), s));
    GView v = view(c);
    int64_t n = c->n;
    Buf<int64_t> off(n + 1, s);
    if (n) {
      launch(k_zip_size_lane, grid_for(n, 256), 256, 0, s, v, off.get());
      if (c->max_deg > kZipLaneMax || c->max_deg == 0) launch(k_zip_size, grid_for(n * 32, 256), 256, 0, s, v, off.get());
      TP_LAUNCH_CHECK();
    }
    exclusive_scan_i64(off.get(), off.get(), n, s);
    int64_t body = read_scalar(off.get() + n, s);
    int tl = 1;
    for (uint64_t x = (uint64_t)c->m2; x >= 128; x >>= 7) ++tl;
    z->nbytes = (uint64_t)body + tl;
    z->bytes.alloc(z->nbytes + kBytePad, s);
    TP_CUDA(cudaMemsetAsync(z->bytes.get(), 0, z->nbytes + kBytePad, s));
    if (n) {
      launch(k_zip_write_lane, grid_for(n, 256), 256, 0, s, v, off.get(), z->bytes.get());
      if (c->max_deg > kZipLaneMax || c->max_deg == 0)
        launch(k_zip_write, grid_for(n * 32, 256), 256, 0, s, v, off.get(), z->bytes.get());
      TP_LAUNCH_CHECK();
    }
    launch(k_zip_terminal, 1, 1, 0, s, (uint64_t)body, c->m2, z->bytes.get());
    TP_LAUNCH_CHECK();
    z->off_is64 = wide_offsets(z->nbytes);
    if (z->off_is64) {
      z->off64.alloc(n + 1, s);
      launch(k_off_copy, grid_for(n + 1, 256), 256, 0, s, off.get(), n + 1, z->off64.get());
    } else {
      z->off32.alloc(n + 1, s);
      launch(k_off_narrow, grid_for(n + 1, 256), 256, 0, s, off.get(), n + 1, z->off32.get());
    }
    TP_LAUNCH_CHECK();
    z->total_vw = c->total_vw;
    TP_CUDA(cudaStreamSynchronize(s));
  } catch (...) {
    delete z;
    throw;
  }
  return z;
}

tp_graph *decompress(const tp_graph *z, cudaStream_t s) {
  TP_REQUIRE(z->compressed, TP_ERR_INVALID);
  tp_graph *c = new_graph();
  try {
    c->n = z->n;
    c->m2 = z->m2;
    c->err.alloc(1, s);
    TP_CUDA(cudaMemsetAsync(c->err.get(), 0, sizeof(int32_t), s));
    GView v = view(z);
    int64_t n = z->n;
    Buf<int32_t> bad(1, s);
    TP_CUDA(cudaMemsetAsync(bad.get(), 0, sizeof(int32_t), s));
    if (n) {
      launch(k_zip_header_check, grid_for(n, 256), 256, 0, s, v, bad.get());
      TP_LAUNCH_CHECK();
    }
    TP_REQUIRE(read_scalar(bad.get(), s) == 0, TP_ERR_CORRUPT);
    c->xadj.alloc(n + 1, s);
    compute_degrees(z, c->xadj.get(), s);
    exclusive_scan_i64(c->xadj.get(), c->xadj.get(), n, s);
    int64_t m2 = read_scalar(c->xadj.get() + n, s);
    TP_REQUIRE(m2 == z->m2, TP_ERR_CORRUPT);
    c->adj.alloc(m2 + kAdjPad, s);
    TP_CUDA(cudaMemsetAsync(c->adj.get() + m2, 0, kAdjPad * sizeof(int32_t), s));
    if (n) {
      launch(k_unzip, grid_for(n * 32, 256), 256, 0, s, v, c->xadj.get(), c->adj.get());
      TP_LAUNCH_CHECK();
    }
    int32_t e = read_scalar(z->err.get(), s);
    if (e) {
      TP_CUDA(cudaMemsetAsync(z->err.get(), 0, sizeof(int32_t), s));
      throw Error{(tp_status)e};
    }
    finish_graph_stats(c, s);
  } catch (...) {
    delete c;
    throw;
  }
  return c;
}

__global__ void k_terminal_m2(const uint8_t *bytes, const uint64_t *off, int64_t n, int64_t *m2) {
  uint64_t x;
  read_varint(bytes + off[n], x);
  *m2 = (int64_t)x;
}

tp_graph *from_compressed(int64_t n, uint64_t nbytes, const uint8_t *bytes, const uint64_t *off,
                          int host, cudaStream_t s) {
  TP_REQUIRE(n >= 0 && n < (int64_t)INT32_MAX && bytes && off && nbytes > 0, TP_ERR_INVALID);
  cudaMemcpyKind kind = host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  tp_graph *z = new_graph();
  try {
    z->n = n;
    z->compressed = 1;
    z->nbytes = nbytes;
    z->err.alloc(1, s);
    TP_CUDA(cudaMemsetAsync(z->err.get(), 0, sizeof(int32_t), s));
    z->bytes.alloc(nbytes + kBytePad, s);
    TP_CUDA(cudaMemsetAsync(z->bytes.get(), 0, nbytes + kBytePad, s));
    TP_CUDA(cudaMemcpyAsync(z->bytes.get(), bytes, nbytes, kind, s));
    Buf<uint64_t> o(n + 1, s);
    TP_CUDA(cudaMemcpyAsync(o.get(), off, (n + 1) * sizeof(uint64_t), kind, s));
    // offsets must lie inside the stream before anything dereferences them
    std::vector<uint64_t> ho(n + 1);
    TP_CUDA(cudaMemcpyAsync(ho.data(), o.get(), (n + 1) * sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
    TP_CUDA(cudaStreamSynchronize(s));
    for (int64_t u = 0; u <= n; ++u)
      TP_REQUIRE(ho[u] < nbytes && (u == 0 || ho[u] >= ho[u - 1]), TP_ERR_CORRUPT);
    z->off_is64 = wide_offsets(nbytes);
    if (z->off_is64) {
      z->off64 = std::move(o);
    } else {
      z->off32.alloc(n + 1, s);
      launch(k_off_narrow_u64, grid_for(n + 1, 256), 256, 0, s, o.get(), n + 1, z->off32.get());
      TP_LAUNCH_CHECK();
    }
    Buf<int64_t> m2(1, s);
    launch(k_terminal_m2, 1, 1, 0, s, z->bytes.get(), z->off_is64 ? z->off64.get() : o.get(), n, m2.get());
    TP_LAUNCH_CHECK();
    z->m2 = read_scalar(m2.get(), s);
    TP_REQUIRE(z->m2 >= 0, TP_ERR_CORRUPT);
    tp_graph *c = decompress(z, s);  // throws TP_ERR_CORRUPT on a malformed stream
    Buf<int32_t> bad(1, s);
    TP_CUDA(cudaMemsetAsync(bad.get(), 0, sizeof(int32_t), s));
    launch(k_validate, grid_for(std::max<int64_t>(n, 1) * 32, 256), 256, 0, s, view(c), bad.get());
    TP_LAUNCH_CHECK();
    int32_t b = read_scalar(bad.get(), s);
    z->total_vw = n;
    z->max_deg = c->max_deg;
    delete c;
    TP_REQUIRE(b == 0, TP_ERR_CORRUPT);
  } catch (...) {
    delete z;
    throw;
  }
  return z;
}

tp_graph *from_csr(int64_t n, const int64_t *xadj, const int32_t *adj, const int64_t *vwgt,
                   const int64_t *ewgt, int host, cudaStream_t s) {
  TP_REQUIRE(n >= 0 && n < (int64_t)INT32_MAX && xadj != nullptr, TP_ERR_INVALID);
  tp_graph *g = new_graph();
  try {
    cudaMemcpyKind kind = host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    g->n = n;
    g->err.alloc(1, s);
    TP_CUDA(cudaMemsetAsync(g->err.get(), 0, sizeof(int32_t), s));
    g->xadj.alloc(n + 1, s);
    TP_CUDA(cudaMemcpyAsync(g->xadj.get(), xadj, (n + 1) * sizeof(int64_t), kind, s));
    int64_t m2 = host ? xadj[n] : read_scalar(g->xadj.get() + n, s);
    TP_REQUIRE(m2 >= 0, TP_ERR_INVALID);
    g->m2 = m2;
    TP_REQUIRE(m2 == 0 || adj != nullptr, TP_ERR_INVALID);
    g->adj.alloc(m2 + kAdjPad, s);  // padded: 16-byte loads may run past the last entry
    TP_CUDA(cudaMemsetAsync(g->adj.get() + m2, 0, kAdjPad * sizeof(int32_t), s));
    if (m2) TP_CUDA(cudaMemcpyAsync(g->adj.get(), adj, m2 * sizeof(int32_t), kind, s));
    g->unit_vw = vwgt == nullptr;
    g->unit_ew = ewgt == nullptr;
    if (vwgt) {
      g->vw.alloc(n, s);
      if (n) TP_CUDA(cudaMemcpyAsync(g->vw.get(), vwgt, n * sizeof(int64_t), kind, s));
    }
    if (ewgt) {
      g->ew.alloc(m2, s);
      if (m2) TP_CUDA(cudaMemcpyAsync(g->ew.get(), ewgt, m2 * sizeof(int64_t), kind, s));
    }
    Buf<int32_t> bad(1, s);
    TP_CUDA(cudaMemsetAsync(bad.get(), 0, sizeof(int32_t), s));
    launch(k_validate, grid_for(std::max<int64_t>(n, 1) * 32, 256), 256, 0, s, view(g), bad.get());
    TP_LAUNCH_CHECK();
    TP_REQUIRE(read_scalar(bad.get(), s) == 0, TP_ERR_INVALID);
    finish_graph_stats(g, s);
  } catch (...) {
    delete g;
    throw;
  }
  return g;
}

void export_csr(const tp_graph *g, int64_t *xadj, int32_t *adj, int64_t *vw, int64_t *ew,
                cudaStream_t s) {
  TP_REQUIRE(!g->compressed, TP_ERR_INVALID);
  if (xadj) TP_CUDA(cudaMemcpyAsync(xadj, g->xadj.get(), (g->n + 1) * 8, cudaMemcpyDeviceToDevice, s));
  if (adj && g->m2) TP_CUDA(cudaMemcpyAsync(adj, g->adj.get(), g->m2 * 4, cudaMemcpyDeviceToDevice, s));
  if (vw && g->n) {
    if (g->unit_vw) launch(k_ones, grid_for(g->n, 256), 256, 0, s, vw, g->n);
    else TP_CUDA(cudaMemcpyAsync(vw, g->vw.get(), g->n * 8, cudaMemcpyDeviceToDevice, s));
  }
  if (ew && g->m2) {
    if (g->unit_ew) launch(k_ones, grid_for(g->m2, 256), 256, 0, s, ew, g->m2);
    else TP_CUDA(cudaMemcpyAsync(ew, g->ew.get(), g->m2 * 8, cudaMemcpyDeviceToDevice, s));
  }
  TP_LAUNCH_CHECK();
}

void export_compressed(const tp_graph *g, uint8_t *bytes, uint64_t *off, cudaStream_t s) {
  TP_REQUIRE(g->compressed, TP_ERR_INVALID);
  if (bytes) TP_CUDA(cudaMemcpyAsync(bytes, g->bytes.get(), g->nbytes, cudaMemcpyDeviceToDevice, s));
  if (off) {
    if (g->off_is64) {
      TP_CUDA(cudaMemcpyAsync(off, g->off64.get(), (g->n + 1) * 8, cudaMemcpyDeviceToDevice, s));
    } else {
      launch(k_widen, grid_for(g->n + 1, 256), 256, 0, s, g->off32.get(), off, g->n + 1);
      TP_LAUNCH_CHECK();
    }
  }
}

}  // namespace tp

extern "C" uint64_t tp_launch_count(void) { return tp::g_launches.load(); }

extern "C" void tp_profile_enable(int on) {
  tp::g_prof.enabled = on != 0;
}

extern "C" int tp_profile_read(tp_profile_entry *out, int max, void *stream) {
  using namespace tp;
  for (int f = 0; f < max && f < PF_COUNT; ++f) out[f] = tp_profile_entry{f, 0, 0.0, 0.0};
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return -1;
  for (const ProfRecord &r : g_prof.recs) {
    float ms = 0;
    cudaEventElapsedTime(&ms, r.a, r.b);
    if (r.family < max) {
      out[r.family].launches += 1;
      out[r.family].ms += ms;
      out[r.family].bytes += r.bytes;
    }
    g_prof.pool.push_back(r.a);
    g_prof.pool.push_back(r.b);
  }
  g_prof.recs.clear();
  return PF_COUNT < max ? PF_COUNT : max;
}

extern "C" tp_status tp_set_allocator(void *(*alloc)(size_t, void *, void *),
                                      void (*free_fn)(void *, size_t, void *, void *), void *ctx) {
  if ((alloc == nullptr) != (free_fn == nullptr)) return TP_ERR_INVALID;
  if (!alloc) {
    tp::g_hook.store(&tp::g_default_hook);
    return TP_OK;
  }
  // kept for the process lifetime: buffers made through it free through it
  const tp::AllocHook *h = new (std::nothrow) tp::AllocHook{alloc, free_fn, ctx};
  if (!h) return TP_ERR_OOM;
  tp::g_hook.store(h);
  return TP_OK;
}
