// Internal definitions shared by the library's CUDA translation units.
// Target: sm_103a (GB300). Nothing here is visible through the C-ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <atomic>
#include <utility>
#include <vector>

#include "../../include/terapart.h"

namespace tp {

// ---------------------------------------------------------------- status / errors
struct Error {
  tp_status code;
};

#define TP_CUDA(call)                                                                    \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess) {                                                             \
      fprintf(stderr, "terapart: %s failed: %s (%s:%d)\n", #call, cudaGetErrorString(e_), \
              __FILE__, __LINE__);                                                       \
      throw ::tp::Error{e_ == cudaErrorMemoryAllocation ? TP_ERR_OOM : TP_ERR_CUDA};     \
    }                                                                                    \
  } while (0)

#define TP_REQUIRE(cond, code)          \
  do {                                  \
    if (!(cond)) throw ::tp::Error{code}; \
  } while (0)

#define TP_LAUNCH_CHECK() TP_CUDA(cudaGetLastError())

// Runs f, converting library exceptions into status codes at the ABI edge.
template <class F>
tp_status guard(F &&f) {
  try {
    f();
    return TP_OK;
  } catch (const Error &e) {
    return e.code;
  } catch (...) {
    return TP_ERR_CUDA;
  }
}

// ---------------------------------------------------------------- device memory
// The allocator a buffer came from (tp_set_allocator's functions, or null
// functions for the library's own cudaMallocAsync). Every buffer is released
// through the allocator that made it, even if the hook changed meanwhile.
struct AllocHook {
  void *(*alloc)(size_t, void *, void *);
  void (*free)(void *, size_t, void *, void *);
  void *ctx;
};
void *dev_alloc(size_t bytes, cudaStream_t s, const AllocHook **from);
void dev_free(void *p, size_t bytes, cudaStream_t s, const AllocHook *from);
// Per-thread device-memory high-water mark: mem_mark() starts a window and
// returns the current holding; mem_peak_since(mark) is the rise since then.
int64_t mem_mark();
int64_t mem_peak_since(int64_t mark);
// Caps what this thread may hold at its current holding plus bytes (< 0: no
// cap); allocations beyond it throw TP_ERR_BUDGET.
void mem_cap(int64_t bytes_above_now);
// With TP_MEM_TRACE set: prints the buffers live at this thread's peak.
void mem_trace_dump(const char *what);

// Owning, stream-ordered device buffer.
template <class T>
struct Buf {
  T *p = nullptr;
  size_t n = 0;
  cudaStream_t s = nullptr;
  const AllocHook *from = nullptr;
  Buf() = default;
  Buf(size_t count, cudaStream_t st) { alloc(count, st); }
  void alloc(size_t count, cudaStream_t st) {
    release();
    s = st;
    p = count ? static_cast<T *>(dev_alloc(count * sizeof(T), st, &from)) : nullptr;
    n = count;
  }
  void release() {
    if (p) dev_free(p, n * sizeof(T), s, from);
    p = nullptr;
    n = 0;
  }
  T *get() const { return p; }
  ~Buf() { release(); }
  Buf(const Buf &) = delete;
  Buf &operator=(const Buf &) = delete;
  Buf(Buf &&o) noexcept : p(o.p), n(o.n), s(o.s), from(o.from) { o.p = nullptr, o.n = 0; }
  Buf &operator=(Buf &&o) noexcept {
    release();
    p = o.p, n = o.n, s = o.s, from = o.from;
    o.p = nullptr, o.n = 0;
    return *this;
  }
};

// ---------------------------------------------------------------- graph
// Degree tiers used by the rating kernels (performance only; the result of
// a rating never depends on its tier).
enum : uint8_t { TIER_SMALL = 0, TIER_MID = 1, TIER_BIG = 2, TIER_HUGE = 3, TIER_LANE = 4 };
constexpr int kLaneMaxDeg = 32;  // lane tier: one lane per vertex
constexpr int64_t kLaneMaxEdgeWeight = (int64_t)1 << 26;  // weighted lane tier: ratings fit 32 bits
constexpr int64_t kChunkThreshold = 10000;  // compressed format: chunked above this degree
constexpr int64_t kChunkSize = 1000;        // neighbours per chunk
constexpr int kSegLog = 12;                 // huge tables are scanned 4096 slots per block
constexpr int kSegBestBytes = 48;           // one segment's best label and best admissible label
constexpr int64_t kMidSplit = 256;          // mid tier: degrees up to here use 512-slot tables
constexpr int64_t kBigTinySplit = 1024;     // big tier: degrees up to here use 2048-slot tables
constexpr int64_t kBigMidSplit = 2048;      // big tier: degrees up to here use 4096-slot tables
constexpr int64_t kBigSplit = 4096;         // big tier: degrees up to here use 8192-slot tables

struct TierCache {
  bool built = false;
  int32_t small_max = 0, mid_max = 0, lane_max = 0;
  bool lane_long = false;  // compressed lane records may exceed 80 bytes (skewed graphs)
  int64_t count[5] = {0, 0, 0, 0, 0};  // vertices per tier
  Buf<uint8_t> tier;         // n
  // vertex lists per tier (ascending); the mid tier is listed in two parts,
  // degree <= kMidSplit (warp tables of 512 slots) and above (1024), the big
  // tier in four, degree <= kBigTinySplit (block tables of 2048 slots, many
  // blocks per SM), <= kBigMidSplit (4096), <= kBigSplit (8192) and above
  // (16384)
  Buf<int32_t> small, mid, mid2, big0, big1, big, big2, huge;
  int64_t n_small = 0, n_mid = 0, n_mid2 = 0, n_big0 = 0, n_big1 = 0, n_big = 0, n_big2 = 0,
          n_huge = 0;
  Buf<int64_t> huge_toff;  // global table offsets (slots), size n_huge + 1
  Buf<int32_t> huge_tcap;  // log2 of the table capacity per vertex
  int64_t huge_slots = 0;
  int64_t edges[5] = {0, 0, 0, 0, 0};  // adjacency entries per tier
  Buf<int64_t> huge_chunk_start;  // prefix of chunk counts over the huge list (n_huge + 1)
  int64_t n_huge_chunks = 0;
  // the huge tables are scanned in segments of kSegSlots slots by many blocks
  Buf<int64_t> huge_seg_start;    // prefix of segment counts over the huge list (n_huge + 1)
  int64_t n_huge_segs = 0;
  Buf<unsigned char> huge_seg_best;  // per segment: its best label (see lp.cu)
  Buf<int32_t> tkeys;  // global rating tables (huge tier), EMPTY = -1
  Buf<int64_t> tvals;
  // per hub: the slots its table has filled (region toff/2 of half the
  // table's size) and how many, so scans read filled slots only
  Buf<int32_t> tlist;
  Buf<int32_t> tcount;
  // Later frees go to stream s (the cache may have been built on a stream
  // that no longer exists; see tp_graph::rehome).
  void rehome(cudaStream_t s) {
    tier.s = small.s = mid.s = mid2.s = big0.s = big1.s = big.s = big2.s = huge.s = s;
    huge_toff.s = huge_tcap.s = s;
    huge_chunk_start.s = tkeys.s = tvals.s = tlist.s = tcount.s = s;
    huge_seg_start.s = huge_seg_best.s = s;
  }
};

}  // namespace tp

struct tp_graph {
  int64_t n = 0, m2 = 0;
  int compressed = 0;
  int unit_vw = 1, unit_ew = 1;
  int64_t total_vw = 0;
  int64_t max_deg = 0;
  int64_t max_ew = 1;  // largest edge weight (1 for unit weights)
  // CSR
  tp::Buf<int64_t> xadj;
  tp::Buf<int32_t> adj;
  tp::Buf<int64_t> vw, ew;
  // compressed
  tp::Buf<uint8_t> bytes;  // padded by kBytePad zero bytes
  uint64_t nbytes = 0;
  tp::Buf<uint32_t> off32;
  tp::Buf<uint64_t> off64;
  int off_is64 = 0;
  // per-graph error word (device)
  tp::Buf<int32_t> err;
  tp::TierCache tiers;
  // Buffers remember the stream they were allocated on and are freed on it.
  // A graph outlives those streams (its tier cache may have been built by a
  // partition on a batch worker's stream), so once the device is idle its
  // buffers are freed on the legacy stream instead.
  void rehome() {
    xadj.s = adj.s = vw.s = ew.s = err.s = nullptr;
    bytes.s = off32.s = off64.s = nullptr;
    tiers.rehome(nullptr);
  }
};

namespace tp {
constexpr int kBytePad = 64;  // zero bytes after a compressed stream
constexpr int kAdjPad = 4;    // int32 entries after a CSR adjacency array

// Read-only device view of a graph for kernels.
struct GView {
  int64_t n, m2;
  const int64_t *xadj;
  const int32_t *adj;
  const int64_t *vw;  // null: unit
  const int64_t *ew;  // null: unit
  const uint8_t *bytes;
  const uint32_t *off32;
  const uint64_t *off64;
  int compressed;
  int32_t *err;
};
GView view(const tp_graph *g);

// ---------------------------------------------------------------- hashing
// Counter-based hashing of the deterministic LP (library's own statement of
// the splitmix64 output function, Steele, Lea and Flood, OOPSLA 2014; the
// golden-gamma offset keeps a zero input off the fixed point mix(0) = 0).
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}
constexpr uint64_t kGamma = 0x9e3779b97f4a7c15ULL;  // golden-gamma offset of hstep
__host__ __device__ __forceinline__ uint64_t hstep(uint64_t h, uint64_t x) {
  return mix64(h ^ (x + kGamma));
}
__host__ __device__ __forceinline__ uint64_t round_key(uint64_t seed, uint64_t tag, uint64_t a,
                                                       uint64_t b) {
  return hstep(hstep(hstep(seed, tag), a), b);
}
// Phase tags: ASCII mnemonics packed into 64 bits.
constexpr uint64_t kTagCluster = 0x4c50436c75737472ULL;  // "LPClustr"
constexpr uint64_t kTagRefine = 0x4c50526566696e65ULL;   // "LPRefine"
constexpr uint64_t kTagTwoHop = 0x54776f486f704d74ULL;   // "TwoHopMt"
constexpr uint64_t kTagIPSeed = 0x495053656564566bULL;   // "IPSeedVk"
constexpr uint64_t kTagIPLP = 0x49504c5032576179ULL;     // "IPLP2Way"
constexpr uint64_t kTagTie = 0x5469654272656b72ULL;      // "TieBrekr"

// hash mod S; a mask when S is a power of two (the same value, no division).
__host__ __device__ __forceinline__ int32_t sub_round_of(uint64_t h, int32_t S) {
  return (S & (S - 1)) == 0 ? (int32_t)(h & (uint64_t)(S - 1)) : (int32_t)(h % (uint64_t)S);
}

__device__ __forceinline__ uint32_t tie_hash(uint64_t hv, int32_t x) {
  return (uint32_t)(hstep(hv, (uint64_t)(int64_t)x) >> 32);
}

// Rating order: larger rating, then smaller tie hash, then smaller label.
__device__ __forceinline__ bool better(int64_t ra, uint32_t ta, int32_t xa, int64_t rb, uint32_t tb,
                                       int32_t xb) {
  if (ra != rb) return ra > rb;
  if (ta != tb) return ta < tb;
  return xa < xb;
}

// ---------------------------------------------------------------- warp helpers
constexpr unsigned kFull = 0xffffffffu;
__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }
__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Warp argmax under the rating order; returns the winner in all lanes.
__device__ __forceinline__ void warp_best(int64_t &r, uint32_t &t, int32_t &x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    int64_t r2 = __shfl_xor_sync(kFull, r, o);
    uint32_t t2 = __shfl_xor_sync(kFull, t, o);
    int32_t x2 = __shfl_xor_sync(kFull, x, o);
    if (better(r2, t2, x2, r, t, x)) r = r2, t = t2, x = x2;
  }
}

template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}
template <class T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    T w = __shfl_xor_sync(kFull, v, o);
    v = w > v ? w : v;
  }
  return v;
}

// Inclusive warp scan (sum).
template <class T>
__device__ __forceinline__ T warp_incl_scan(T v) {
  int l = lane_id();
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T w = __shfl_up_sync(kFull, v, o);
    if (l >= o) v += w;
  }
  return v;
}

__device__ __forceinline__ void latch_error(int32_t *err, int32_t code) {
  if (err) atomicCAS(err, 0, code);
}

// ---------------------------------------------------------------- launch helpers
int num_sms();
void count_launch();
void count_launches(uint64_t k);  // kernels a replayed CUDA graph ran
// Launches on this thread are being recorded into a CUDA graph (on) or no
// longer (off, returning how many were recorded since on).
uint64_t capture_counting(bool on);

// Every kernel of the library is launched through here (counts launches).
template <class... KArgs, class... Args>
inline void launch(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                   Args &&...args) {
  k<<<grid, block, smem, s>>>(static_cast<KArgs>(args)...);
  count_launch();
}

// Opt-in kernel timing (CUDA events around selected launches).
enum ProfFamily {
  PF_RATE_SMALL = 0,
  PF_RATE_MID,
  PF_RATE_BIG,
  PF_RATE_HUGE,
  PF_APPROVE,
  PF_RATE_LANE,
  PF_COUNT
};
bool prof_active();                 // profiling enabled and inside a profiled scope
void prof_scope(bool on);           // level-0 clustering rounds open/close the scope
void prof_begin(int family, cudaStream_t s);
void prof_end(int family, cudaStream_t s, double alg_bytes);
inline unsigned grid_for(int64_t work, int block, int64_t max_blocks = 0) {
  int64_t b = (work + block - 1) / block;
  if (b < 1) b = 1;
  int64_t cap = max_blocks ? max_blocks : (int64_t)num_sms() * 32;
  if (b > cap) b = cap;
  return (unsigned)b;
}

// ---------------------------------------------------------------- primitives (prims.cu)
// Exclusive prefix sum of in[0..n) into out[0..n]; out[n] = total. In-place allowed.
void exclusive_scan_i64(const int64_t *in, int64_t *out, int64_t n, cudaStream_t s);
void exclusive_scan_i32_to_i64(const int32_t *in, int64_t *out, int64_t n, cudaStream_t s);
// Inclusive max-scan of int64.
void inclusive_max_scan_i64(const int64_t *in, int64_t *out, int64_t n, cudaStream_t s);
// Stable LSD radix sort of (key, value) pairs by the low `bits` key bits.
// vals may be null. Buffers are sorted in place (temporary storage internal).
// lo: the sort key is bits lo .. lo + bits - 1 (lower bits ride along).
void radix_sort_pairs(uint64_t *keys, uint64_t *vals, int64_t n, int bits, cudaStream_t s,
                      int lo = 0);
// Reads one device value synchronously.
template <class T>
T read_scalar(const T *d, cudaStream_t s) {
  T h;
  TP_CUDA(cudaMemcpyAsync(&h, d, sizeof(T), cudaMemcpyDeviceToHost, s));
  TP_CUDA(cudaStreamSynchronize(s));
  return h;
}
int bits_for(uint64_t max_value);  // bits needed to represent values <= max_value
int64_t max_i64(const int64_t *d, int64_t n, cudaStream_t s);  // 0 for n == 0; synchronises

// ---------------------------------------------------------------- graph helpers (graph.cu)
tp_graph *new_graph();
void compute_degrees(const tp_graph *g, int64_t *d_deg, cudaStream_t s);  // n entries
void build_tiers(tp_graph *g, const tp_params &p, cudaStream_t s);
// Hub rating tables: allocated (empty) for a rating call, released after it.
void ensure_hub_tables(tp_graph *g, cudaStream_t s);
void release_hub_tables(tp_graph *g, cudaStream_t s);

// ---------------------------------------------------------------- LP (lp.cu)
// Batched graphs: one union graph holds many graphs side by side (each a
// contiguous vertex range, labels of a graph only ever its own), and every
// per-vertex decision is taken exactly as for that graph alone: hashes see
// the graph's own vertex and label numbers, caps are the graph's. Tables are
// indexed by the graph's position in the batch. gid == null: one graph.
struct SegLp {
  const int32_t *gid = nullptr;   // graph of every vertex
  const int32_t *lgid = nullptr;  // graph of every label
  const int64_t *vb = nullptr;    // per graph: its first vertex in this union
  const int64_t *lb = nullptr;    // per graph: its first label
  const int64_t *cap = nullptr;   // per graph: the label-weight cap
  const int32_t *k = nullptr;     // per graph: its blocks (refinement, rebalancing)
  int64_t ngraphs = 0;            // table entries
};
struct LpState {
  int32_t *label;
  int64_t *lw;
  int64_t nlabels;
  int64_t cap;  // uniform cap for every label (one graph)
  SegLp seg{};
};
// Workspace for sub-rounds on one graph (per-label counters + mover lists).
struct LpWork {
  int64_t nlabels = 0, n = 0;
  Buf<int64_t> in_w;   // nlabels: weight of this sub-round's movers per target
  Buf<int32_t> ccnt;   // nlabels: contested movers per target (zero between sub-rounds)
  Buf<int32_t> cfill;  // nlabels: fill pointer inside a contested segment
  Buf<int64_t> cbase;   // nlabels
  Buf<int32_t> mv_u, mv_t;  // n
  Buf<int32_t> mv_o;        // n: the mover's label when it was rated (its source)
  Buf<int64_t> mv_g;        // n
  Buf<int8_t> mv_ok;        // n
  Buf<int32_t> cseg;        // n (contested mover indices grouped by target)
  Buf<int32_t> ctarget;     // nlabels (contested targets)
  Buf<int64_t> counters;    // [0] movers, [1] contested targets, [2] contested pool
  // lane-tier vertices of the current round grouped by sub-round (A3)
  Buf<int32_t> bucket;       // n
  Buf<uint8_t> bucket_sub;   // n: sub-round + 1 of every vertex this round (0: not listed)
  Buf<uint64_t> bucket_rec;  // n: record start << 8 | length per listed vertex (compressed)
  Buf<int64_t> bucket_off;   // S * nblocks + 1 offsets (sub-round major)
  int64_t bucket_nblocks = 0;
  int32_t bucket_S = 0;      // S of the current buckets (0: none)
  // the other tiers' lists (small, mid, mid2, big0, big1, big, big2, huge) grouped by sub-round:
  // tb_pos holds list positions, tb_off[t * (S + 1) + s] where sub-round s of
  // tier t starts in tb_pos (tier t's entries begin at tb_base[t])
  static constexpr int kTiers = 8;
  Buf<int32_t> tb_pos;       // sum of the tier list lengths
  Buf<int64_t> tb_off;       // kTiers * (S + 1)
  Buf<int64_t> tb_cur;       // kTiers * S cursors
  int64_t tb_base[kTiers] = {0, 0, 0, 0, 0, 0, 0, 0};
  bool tb_valid = false;
  // huge tier, in bucket order of its hubs: prefix of chunk and segment
  // counts (n_huge + 1) and the items themselves (hub position << 32 | index)
  Buf<int64_t> hc_pre, hs_pre, hc_item, hs_item;
  void init(int64_t n_vertices, int64_t n_labels, cudaStream_t s);
};
// approval (nullable): a CUDA graph of this level's approval kernels to
// replay instead of launching them.
void lp_subround(tp_graph *g, const LpState &st, LpWork &w, uint64_t rk, int32_t S, int32_t s,
                 const tp_params &p, cudaStream_t stream, cudaGraphExec_t approval = nullptr,
                 const uint64_t *rk_dev = nullptr);
// Buckets the lane-tier vertices of round key rk by sub-round (A3), and with
// tiers = true also the other tiers' lists (not inside a stream capture).
void lp_bucket(tp_graph *g, LpWork &w, uint64_t rk, int32_t S, const tp_params &p,
               cudaStream_t stream, const uint64_t *rk_dev = nullptr, bool tiers = false,
               const SegLp *seg = nullptr);
void lp_rounds(tp_graph *g, const LpState &st, LpWork &w, uint64_t seed, uint64_t tag, uint64_t a,
               uint64_t b0, int32_t rounds, int32_t S, const tp_params &p, cudaStream_t stream);
// ev_begin / ev_end (nullable) are recorded around the LP rounds alone.
// seg (batched graphs): vb, cap (U of every graph) and gid; lgid and lb are
// taken equal to gid and vb (labels are vertices).
void lp_cluster(tp_graph *g, int64_t U, const tp_params &p, int32_t level, int32_t *d_cluster,
                cudaStream_t s, cudaEvent_t ev_begin = nullptr, cudaEvent_t ev_end = nullptr,
                const SegLp *seg = nullptr);
// seg (batched graphs): labels are global block ids, lgid maps them to graphs,
// lb is every graph's first block, cap its L_max, k its block count; k is then
// the total number of blocks.
void lp_refine(tp_graph *g, int32_t k, int64_t l_max, const tp_params &p, int32_t level,
               int32_t *d_part, int64_t *d_B, cudaStream_t s, const SegLp *seg = nullptr);
// Per-vertex favourite cluster of singletons (two-hop): fav[u] = best label or
// n (batched graphs: n + the vertex's graph).
void favourites(tp_graph *g, const int32_t *C, const int64_t *Wc, uint64_t rk, int32_t *fav,
                const tp_params &p, cudaStream_t s, const SegLp *seg = nullptr);
void two_hop(tp_graph *g, int32_t *C, const int64_t *Wc, int64_t U, uint64_t seed, int32_t level,
             const tp_params &p, cudaStream_t s, const SegLp *seg = nullptr);
void rebalance_moves(tp_graph *g, int32_t k, int64_t l_max, int32_t *d_part, int64_t *d_B,
                     int *balanced, const tp_params &p, cudaStream_t s);
// Rebalancing of batched graphs (seg as for lp_refine): every graph with an
// overloaded block makes, per iteration, the move rebalance_moves would make
// next for it alone; a graph leaves when balanced or when no move is left.
// d_graphs: the ng batch positions of the union's graphs.
void rebalance_moves_seg(tp_graph *g, const SegLp &seg, const int32_t *d_graphs, int64_t ng,
                         int32_t *d_part, int64_t *d_B, const tp_params &p, cudaStream_t s);

// ---------------------------------------------------------------- contraction / IP / metrics
// seg_voff (nullable, nseg + 1 vertex offsets of batched graphs): seg_coff
// receives the coarse offsets (coarse ids of a graph stay contiguous).
tp_graph *contract(const tp_graph *g, const int32_t *C, int32_t *d_map, cudaStream_t s,
                   const int64_t *seg_voff = nullptr, int64_t nseg = 0,
                   int64_t *seg_coff = nullptr);
tp_graph *decompress(const tp_graph *z, cudaStream_t s);
void initial_partition(const tp_graph *g, int32_t k, int64_t l_max, const tp_params &p,
                       int32_t *d_part, cudaStream_t s);
// Roots of a bisection forest (batched graphs): root j owns the vertices with
// node_of[u] == j and assigns blocks off .. off + k - 1; key is the block
// offset its graph alone would use (it seeds the hashes), l_max its graph's.
struct IPRoot {
  int32_t off, key, k;
  int64_t l_max;
};
void initial_partition_roots(const tp_graph *g, const std::vector<IPRoot> &roots,
                             const int32_t *d_node_of, const tp_params &p, int32_t *d_part,
                             cudaStream_t s);
void block_weights(const tp_graph *g, const int32_t *part, int32_t k, int64_t *d_B,
                   cudaStream_t s);
int64_t edge_cut(const tp_graph *g, const int32_t *part, cudaStream_t s);
void project(const int32_t *coarse_part, const int32_t *map, int64_t n, int32_t *fine_part,
             cudaStream_t s);

int64_t cluster_cap(int64_t W, int32_t k, int64_t eps_ppm);
int64_t block_cap(int64_t W, int32_t k, int64_t eps_ppm);

}  // namespace tp
