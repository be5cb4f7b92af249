// Batched partitioning (the serving side of the method: the paper partitions
// one graph per run, many small graphs keep the GPU busy only together).
//
// The graphs of a batch are laid side by side in one union graph per level:
// graph i owns a contiguous range of vertex ids, its edges stay inside it,
// and every kernel of the multilevel scheme (Section "The Multilevel
// Scheme") runs once over the whole union instead of once per graph. What
// makes each graph's result equal to partitioning it alone:
//   - every per-vertex decision reads the graph's own numbers: sub-round and
//     tie hashes see the vertex's and the label's ids inside their graph,
//     caps (U, L_max) and block ranges are the graph's (SegLp in lp.cu);
//   - contraction ranks non-empty clusters with one scan, so a graph's coarse
//     ids stay contiguous and in the same order as alone;
//   - the per-graph stopping rules (n <= c_lim k, shrink by less than 5%,
//     max_levels) take graphs out of the union of the next level;
//   - initial partitioning is one bisection forest, a tree per graph with
//     the hash key offsets and L_max of that graph;
//   - blocks are numbered globally (graph i owns boff_i .. boff_i + k_i - 1),
//     each graph's block weights and caps are its own, and rebalancing moves
//     one vertex per graph and iteration, as it would for the graph alone.
// Kernel launches then grow with the number of levels, not of graphs.
#include <algorithm>
#include <memory>
#include <thread>
#include <vector>

#include "decode.cuh"

namespace tp {

namespace {

// One input graph (CSR, device).
struct SrcGraph {
  const int64_t *xadj;
  const int32_t *adj;
  const int64_t *vw, *ew;  // null: unit
};

// Level-0 union, vertices: graph j = blockIdx.y fills its range of xadj,
// vertex weights and graph ids.
__global__ void k_union_vertices(const SrcGraph *src, const int64_t *voff, const int64_t *eoff,
                                 const int32_t *gl, int64_t *xadj, int64_t *vw, int32_t *gid) {
  const int j = blockIdx.y;
  const int64_t v0 = voff[j], n = voff[j + 1] - v0, e0 = eoff[j];
  const SrcGraph g = src[j];
  const int32_t bi = gl[j];
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n;
       u += (int64_t)gridDim.x * blockDim.x) {
    xadj[v0 + u] = e0 + g.xadj[u];
    if (vw) vw[v0 + u] = g.vw ? g.vw[u] : 1;
    gid[v0 + u] = bi;
  }
}

// Level-0 union, edges: neighbour ids shifted by the graph's first vertex.
__global__ void k_union_edges(const SrcGraph *src, const int64_t *voff, const int64_t *eoff,
                              int32_t *adj, int64_t *ew) {
  const int j = blockIdx.y;
  const int64_t e0 = eoff[j], m = eoff[j + 1] - e0;
  const int32_t v0 = (int32_t)voff[j];
  const SrcGraph g = src[j];
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x) {
    adj[e0 + e] = v0 + g.adj[e];
    if (ew) ew[e0 + e] = g.ew ? g.ew[e] : 1;
  }
}

// Extraction of some graphs of a union (sel[j'] = source position of new
// graph j'), vertices: xadj, weights, graph ids, new -> old and old -> new.
__global__ void k_extract_vertices(const int32_t *sel, const int64_t *ovoff, const int64_t *oeoff,
                                   const int64_t *nvoff, const int64_t *neoff, const int64_t *oxadj,
                                   const int64_t *ovw, const int32_t *ogid, int64_t *xadj,
                                   int64_t *vw, int32_t *gid, int32_t *n2o, int32_t *o2n) {
  const int jn = blockIdx.y, jo = sel[jn];
  const int64_t ov = ovoff[jo], nv = nvoff[jn], n = nvoff[jn + 1] - nv;
  const int64_t shift = neoff[jn] - oeoff[jo];
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n;
       u += (int64_t)gridDim.x * blockDim.x) {
    xadj[nv + u] = oxadj[ov + u] + shift;
    if (vw) vw[nv + u] = ovw[ov + u];
    gid[nv + u] = ogid[ov + u];
    if (n2o) n2o[nv + u] = (int32_t)(ov + u);
    if (o2n) o2n[ov + u] = (int32_t)(nv + u);
  }
}

__global__ void k_extract_edges(const int32_t *sel, const int64_t *ovoff, const int64_t *oeoff,
                                const int64_t *nvoff, const int64_t *neoff, const int32_t *oadj,
                                const int64_t *oew, int32_t *adj, int64_t *ew) {
  const int jn = blockIdx.y, jo = sel[jn];
  const int64_t oe = oeoff[jo], ne = neoff[jn], m = neoff[jn + 1] - ne;
  const int32_t shift = (int32_t)(nvoff[jn] - ovoff[jo]);
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x) {
    adj[ne + e] = oadj[oe + e] + shift;
    if (ew) ew[ne + e] = oew[oe + e];
  }
}

// Graph ids of a union whose graphs follow voff (graph j has batch index gl[j]).
__global__ void k_fill_gid(const int64_t *voff, const int32_t *gl, int32_t *gid) {
  const int j = blockIdx.y;
  const int64_t v0 = voff[j], n = voff[j + 1] - v0;
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n;
       u += (int64_t)gridDim.x * blockDim.x)
    gid[v0 + u] = gl[j];
}

// Position of every vertex's graph inside the union (the bisection roots).
__global__ void k_fill_pos(const int64_t *voff, int32_t *pos) {
  const int j = blockIdx.y;
  const int64_t v0 = voff[j], n = voff[j + 1] - v0;
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n;
       u += (int64_t)gridDim.x * blockDim.x)
    pos[v0 + u] = j;
}

// First vertex of every graph of the union, indexed by batch position.
__global__ void k_vbase(const int64_t *voff, const int32_t *gl, int64_t G, int64_t *vb) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < G;
       j += (int64_t)gridDim.x * blockDim.x)
    vb[gl[j]] = voff[j];
}

// Coarse edge offsets of the graphs: xadj at their coarse vertex offsets.
__global__ void k_gather_i64(const int64_t *src, const int64_t *idx, int64_t n, int64_t *dst) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[idx[i]];
}

__global__ void k_fill(int32_t *p, int64_t n, int32_t v) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = v;
}

// up[sel(w)] = the next level's vertex of fine vertex w of the clustered
// union (through the old -> new map of the next level's extraction, if any).
__global__ void k_up(const int32_t *map, const int32_t *wsel, const int32_t *keep, int64_t nw,
                     int32_t *up) {
  for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < nw;
       w += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c = map[w];
    up[wsel ? wsel[w] : w] = keep ? keep[c] : c;
  }
}

// Projection: vertices whose graph continues take the block of their coarse
// vertex (the others keep the initial partition written before).
__global__ void k_project_up(const int32_t *up, const int32_t *coarse, int64_t n, int32_t *part) {
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n;
       u += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c = up[u];
    if (c >= 0) part[u] = coarse[c];
  }
}

__global__ void k_scatter_i32(const int32_t *src, const int32_t *to, int64_t n, int32_t *dst) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[to[i]] = src[i];
}

// Final blocks of every graph into its own output buffer, numbered from 0.
__global__ void k_write_out(const int32_t *part, const int64_t *voff, const int32_t *gl,
                            const int64_t *boff, int32_t *const *out) {
  const int j = blockIdx.y;
  const int64_t v0 = voff[j], n = voff[j + 1] - v0;
  const int32_t b0 = (int32_t)boff[gl[j]];
  int32_t *o = out[gl[j]];
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n;
       u += (int64_t)gridDim.x * blockDim.x)
    o[u] = part[v0 + u] - b0;
}

// Cut weight leaving every vertex, one warp per vertex.
__global__ void k_ext_weight(GView g, const int32_t *part, int64_t *ext) {
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t u = gw; u < g.n; u += nw) {
    const int32_t pu = part[u];
    int64_t acc = 0;
    warp_neighbours<false>(g, u, -1, [&](bool has, int32_t v, int64_t w, int64_t) {
      if (has && part[v] != pu) acc += w;
    });
    acc = warp_sum(acc);
    if (lane_id() == 0) ext[u] = acc;
  }
}

// 2-D grid over the graphs of a union: x strides inside a graph.
dim3 per_graph_grid(int64_t G, int64_t max_len) {
  const int64_t bx = std::max<int64_t>(1, std::min<int64_t>((max_len + 255) / 256, 64));
  return dim3((unsigned)bx, (unsigned)G, 1);
}

// One level of the hierarchy: the union of the graphs that have this level.
struct ULevel {
  std::unique_ptr<tp_graph> g;
  std::vector<int32_t> gl;          // batch position of every graph, in union order
  std::vector<int64_t> voff, eoff;  // G + 1 vertex / adjacency offsets
  Buf<int32_t> gid;                 // n: batch position of every vertex's graph
  Buf<int32_t> d_gl;                // G
  Buf<int64_t> d_voff, d_eoff;      // G + 1
  Buf<int64_t> d_vb;                // batch-sized: first vertex of every member graph
  Buf<int32_t> up;                  // n: vertex in the next level, -1 if the graph ends here
  int64_t G() const { return (int64_t)gl.size(); }
  int64_t n() const { return g->n; }
};

// Device copies of a level's tables (and the batch-indexed first vertices).
void upload_tables(ULevel &L, int64_t nb, cudaStream_t s) {
  const int64_t G = L.G();
  L.d_gl.alloc(G, s);
  L.d_voff.alloc(G + 1, s);
  L.d_eoff.alloc(G + 1, s);
  L.d_vb.alloc(nb, s);
  TP_CUDA(cudaMemcpyAsync(L.d_gl.get(), L.gl.data(), G * 4, cudaMemcpyHostToDevice, s));
  TP_CUDA(cudaMemcpyAsync(L.d_voff.get(), L.voff.data(), (G + 1) * 8, cudaMemcpyHostToDevice, s));
  TP_CUDA(cudaMemcpyAsync(L.d_eoff.get(), L.eoff.data(), (G + 1) * 8, cudaMemcpyHostToDevice, s));
  launch(k_vbase, grid_for(G, 256), 256, 0, s, L.d_voff.get(), L.d_gl.get(), G, L.d_vb.get());
  TP_LAUNCH_CHECK();
}

// Allocates the arrays of a union CSR graph with n vertices and m2 entries.
tp_graph *alloc_union(int64_t n, int64_t m2, bool unit_vw, bool unit_ew, int64_t W,
                      int64_t max_ew, cudaStream_t s) {
  tp_graph *g = new_graph();
  try {
    g->n = n;
    g->m2 = m2;
    g->unit_vw = unit_vw;
    g->unit_ew = unit_ew;
    g->total_vw = W;
    g->max_ew = max_ew;
    g->xadj.alloc(n + 1, s);
    g->adj.alloc(m2 + kAdjPad, s);
    TP_CUDA(cudaMemsetAsync(g->adj.get() + m2, 0, kAdjPad * sizeof(int32_t), s));
    TP_CUDA(cudaMemcpyAsync(g->xadj.get() + n, &g->m2, 8, cudaMemcpyHostToDevice, s));
    if (!unit_vw) g->vw.alloc(std::max<int64_t>(n, 1), s);
    if (!unit_ew) g->ew.alloc(std::max<int64_t>(m2, 1), s);
    g->err.alloc(1, s);
    TP_CUDA(cudaMemsetAsync(g->err.get(), 0, sizeof(int32_t), s));
  } catch (...) {
    delete g;
    throw;
  }
  return g;
}

// The graphs at positions sel of union L as a new union (same order);
// n2o / o2n (nullable) receive the vertex maps new -> old and old -> new
// (o2n entries of vertices not taken are -1).
void extract(const ULevel &L, const std::vector<int32_t> &sel, int64_t nb, const int64_t *gW,
             ULevel &X, int32_t *n2o, int32_t *o2n, cudaStream_t s) {
  const int64_t G = (int64_t)sel.size();
  X.gl.resize(G);
  X.voff.assign(G + 1, 0);
  X.eoff.assign(G + 1, 0);
  int64_t W = 0, maxlen = 0;
  for (int64_t j = 0; j < G; ++j) {
    const int32_t o = sel[j];
    X.gl[j] = L.gl[o];
    const int64_t n = L.voff[o + 1] - L.voff[o], m = L.eoff[o + 1] - L.eoff[o];
    X.voff[j + 1] = X.voff[j] + n;
    X.eoff[j + 1] = X.eoff[j] + m;
    W += gW[L.gl[o]];
    maxlen = std::max(maxlen, std::max(n, m));
  }
  const tp_graph *og = L.g.get();
  X.g.reset(alloc_union(X.voff[G], X.eoff[G], og->unit_vw, og->unit_ew, W, og->max_ew, s));
  upload_tables(X, nb, s);
  X.gid.alloc(std::max<int64_t>(X.voff[G], 1), s);
  Buf<int32_t> d_sel(G, s);
  TP_CUDA(cudaMemcpyAsync(d_sel.get(), sel.data(), G * 4, cudaMemcpyHostToDevice, s));
  if (o2n) launch(k_fill, grid_for(L.n(), 256), 256, 0, s, o2n, L.n(), -1);
  const dim3 grid = per_graph_grid(G, maxlen);
  launch(k_extract_vertices, grid, 256, 0, s, d_sel.get(), L.d_voff.get(), L.d_eoff.get(),
         X.d_voff.get(), X.d_eoff.get(), og->xadj.get(), og->unit_vw ? nullptr : og->vw.get(),
         L.gid.get(), X.g->xadj.get(), X.g->unit_vw ? nullptr : X.g->vw.get(), X.gid.get(), n2o,
         o2n);
  launch(k_extract_edges, grid, 256, 0, s, d_sel.get(), L.d_voff.get(), L.d_eoff.get(),
         X.d_voff.get(), X.d_eoff.get(), og->adj.get(), og->unit_ew ? nullptr : og->ew.get(),
         X.g->adj.get(), X.g->unit_ew ? nullptr : X.g->ew.get());
  TP_LAUNCH_CHECK();
  TP_CUDA(cudaStreamSynchronize(s));  // d_sel and the host tables outlive their copies
}

struct Timer {
  cudaEvent_t a{}, b{};
  cudaStream_t s;
  explicit Timer(cudaStream_t st) : s(st) {
    TP_CUDA(cudaEventCreate(&a));
    TP_CUDA(cudaEventCreate(&b));
  }
  void start() { TP_CUDA(cudaEventRecord(a, s)); }
  double stop() {
    TP_CUDA(cudaEventRecord(b, s));
    TP_CUDA(cudaEventSynchronize(b));
    float m = 0;
    TP_CUDA(cudaEventElapsedTime(&m, a, b));
    return m;
  }
  ~Timer() {
    cudaEventDestroy(a);
    cudaEventDestroy(b);
  }
};

}  // namespace

// Partitions the graphs idx[0..) of a batch (CSR, k >= 2, n >= 1) as one
// union per level; every graph's stats get its own figures and the group's
// timings and peak memory.
void partition_union(const std::vector<const tp_graph *> &gs, const std::vector<int32_t> &idx,
                     const int32_t *k, int64_t eps_ppm, const tp_params &p,
                     int32_t *const *d_part, tp_stats *stats, cudaStream_t s) {
  const int64_t nb = (int64_t)gs.size();  // batch-indexed tables span the whole batch
  const int64_t G0 = (int64_t)idx.size();
  if (G0 == 0) return;
  const int64_t mark = mem_mark();
  // batch-constant per-graph tables
  std::vector<int64_t> W(nb, 0), U(nb, 1), lmax(nb, 0), boff(nb, 0);
  std::vector<int32_t> kk(nb, 1);
  int64_t K = 0;
  for (int32_t i : idx) {
    W[i] = gs[i]->total_vw;
    kk[i] = k[i];
    U[i] = cluster_cap(W[i], k[i], eps_ppm);
    lmax[i] = block_cap(W[i], k[i], eps_ppm);
    boff[i] = K;
    K += k[i];
  }
  TP_REQUIRE(K < INT32_MAX, TP_ERR_INVALID);
  std::vector<int32_t> bgid((size_t)K);
  for (int32_t i : idx)
    for (int32_t b = 0; b < k[i]; ++b) bgid[(size_t)(boff[i] + b)] = i;
  Buf<int64_t> d_U(nb, s), d_lmax(nb, s), d_boff(nb, s);
  Buf<int32_t> d_k(nb, s), d_bgid(K, s);
  Buf<int32_t *> d_out(nb, s);
  TP_CUDA(cudaMemcpyAsync(d_U.get(), U.data(), nb * 8, cudaMemcpyHostToDevice, s));
  TP_CUDA(cudaMemcpyAsync(d_lmax.get(), lmax.data(), nb * 8, cudaMemcpyHostToDevice, s));
  TP_CUDA(cudaMemcpyAsync(d_boff.get(), boff.data(), nb * 8, cudaMemcpyHostToDevice, s));
  TP_CUDA(cudaMemcpyAsync(d_k.get(), kk.data(), nb * 4, cudaMemcpyHostToDevice, s));
  TP_CUDA(cudaMemcpyAsync(d_bgid.get(), bgid.data(), K * 4, cudaMemcpyHostToDevice, s));
  TP_CUDA(cudaMemcpyAsync(d_out.get(), d_part, nb * sizeof(int32_t *), cudaMemcpyHostToDevice, s));

  Timer t_phase(s);
  double ms_coarsen = 0, ms_initial = 0, ms_uncoarsen = 0;
  t_phase.start();
  // ---------------- level 0: the union of the input graphs
  std::vector<std::unique_ptr<ULevel>> levels;
  {
    auto L = std::make_unique<ULevel>();
    L->gl = idx;
    L->voff.assign(G0 + 1, 0);
    L->eoff.assign(G0 + 1, 0);
    bool unit_vw = true, unit_ew = true;
    int64_t Wt = 0, max_ew = 1, maxlen = 0;
    std::vector<SrcGraph> src(G0);
    for (int64_t j = 0; j < G0; ++j) {
      const tp_graph *g = gs[idx[j]];
      L->voff[j + 1] = L->voff[j] + g->n;
      L->eoff[j + 1] = L->eoff[j] + g->m2;
      unit_vw &= g->unit_vw != 0;
      unit_ew &= g->unit_ew != 0;
      Wt += g->total_vw;
      max_ew = std::max(max_ew, g->max_ew);
      maxlen = std::max(maxlen, std::max(g->n, g->m2));
      src[j] = SrcGraph{g->xadj.get(), g->adj.get(), g->unit_vw ? nullptr : g->vw.get(),
                        g->unit_ew ? nullptr : g->ew.get()};
    }
    TP_REQUIRE(L->voff[G0] + nb < INT32_MAX, TP_ERR_INVALID);
    L->g.reset(alloc_union(L->voff[G0], L->eoff[G0], unit_vw, unit_ew, Wt, max_ew, s));
    upload_tables(*L, nb, s);
    L->gid.alloc(std::max<int64_t>(L->n(), 1), s);
    Buf<SrcGraph> d_src(G0, s);
    TP_CUDA(cudaMemcpyAsync(d_src.get(), src.data(), G0 * sizeof(SrcGraph), cudaMemcpyHostToDevice, s));
    const dim3 grid = per_graph_grid(G0, maxlen);
    launch(k_union_vertices, grid, 256, 0, s, d_src.get(), L->d_voff.get(), L->d_eoff.get(),
           L->d_gl.get(), L->g->xadj.get(), unit_vw ? nullptr : L->g->vw.get(), L->gid.get());
    launch(k_union_edges, grid, 256, 0, s, d_src.get(), L->d_voff.get(), L->d_eoff.get(),
           L->g->adj.get(), unit_ew ? nullptr : L->g->ew.get());
    TP_LAUNCH_CHECK();
    TP_CUDA(cudaStreamSynchronize(s));  // src outlives its copy
    levels.push_back(std::move(L));
  }
  // ---------------- coarsening
  const int32_t max_levels = std::max(1, std::min(p.max_levels, 64));
  for (int32_t lev = 0;; ++lev) {
    ULevel &L = *levels.back();
    std::vector<int32_t> A;  // positions of the graphs clustered at this level
    for (int64_t j = 0; j < L.G(); ++j) {
      const int32_t i = L.gl[j];
      if (L.voff[j + 1] - L.voff[j] > (int64_t)p.c_lim * k[i] && lev + 1 < max_levels)
        A.push_back((int32_t)j);
    }
    if (A.empty()) break;
    // the working union: this level, or the clustered graphs extracted
    ULevel Wx;
    Buf<int32_t> wsel;
    const bool all = (int64_t)A.size() == L.G();
    if (!all) {
      int64_t nw = 0;
      for (int32_t j : A) nw += L.voff[j + 1] - L.voff[j];
      wsel.alloc(std::max<int64_t>(nw, 1), s);
      extract(L, A, nb, W.data(), Wx, wsel.get(), nullptr, s);
    }
    ULevel &Wl = all ? L : Wx;
    const int64_t GA = Wl.G(), nw = Wl.n();
    Buf<int32_t> C(nw, s), map(nw, s);
    SegLp seg;
    seg.gid = Wl.gid.get();
    seg.vb = Wl.d_vb.get();
    seg.cap = d_U.get();
    seg.ngraphs = nb;
    lp_cluster(Wl.g.get(), 0, p, lev, C.get(), s, nullptr, nullptr, &seg);
    Buf<int64_t> coff(GA + 1, s), ceoff(GA + 1, s);
    std::unique_ptr<tp_graph> cg(contract(Wl.g.get(), C.get(), map.get(), s, Wl.d_voff.get(), GA,
                                          coff.get()));
    C.release();
    launch(k_gather_i64, grid_for(GA + 1, 256), 256, 0, s, cg->xadj.get(), coff.get(), GA + 1,
           ceoff.get());
    TP_LAUNCH_CHECK();
    std::vector<int64_t> hc(GA + 1), he(GA + 1);
    TP_CUDA(cudaMemcpyAsync(hc.data(), coff.get(), (GA + 1) * 8, cudaMemcpyDeviceToHost, s));
    TP_CUDA(cudaMemcpyAsync(he.data(), ceoff.get(), (GA + 1) * 8, cudaMemcpyDeviceToHost, s));
    TP_CUDA(cudaStreamSynchronize(s));
    // graphs that shrank by at least 5% go on
    std::vector<int32_t> keep;
    for (int64_t j = 0; j < GA; ++j) {
      const int64_t n0 = Wl.voff[j + 1] - Wl.voff[j], n1 = hc[j + 1] - hc[j];
      if (20 * n1 <= 19 * n0) keep.push_back((int32_t)j);
    }
    if (keep.empty()) break;
    auto next = std::make_unique<ULevel>();
    ULevel C1;  // the contracted union of the working graphs
    C1.g = std::move(cg);
    C1.gl = Wl.gl;
    C1.voff = hc;
    C1.eoff = he;
    {
      int64_t Wt = 0;
      for (int32_t i : C1.gl) Wt += W[i];
      C1.g->total_vw = Wt;
    }
    Buf<int32_t> kmap;
    if ((int64_t)keep.size() == GA) {
      upload_tables(C1, nb, s);
      C1.gid.alloc(std::max<int64_t>(C1.n(), 1), s);
      int64_t maxlen = 0;
      for (int64_t j = 0; j < GA; ++j) maxlen = std::max(maxlen, hc[j + 1] - hc[j]);
      launch(k_fill_gid, per_graph_grid(GA, maxlen), 256, 0, s, C1.d_voff.get(), C1.d_gl.get(),
             C1.gid.get());
      TP_LAUNCH_CHECK();
      *next = std::move(C1);
    } else {
      upload_tables(C1, nb, s);
      C1.gid.alloc(std::max<int64_t>(C1.n(), 1), s);
      int64_t maxlen = 0;
      for (int64_t j = 0; j < GA; ++j) maxlen = std::max(maxlen, hc[j + 1] - hc[j]);
      launch(k_fill_gid, per_graph_grid(GA, maxlen), 256, 0, s, C1.d_voff.get(), C1.d_gl.get(),
             C1.gid.get());
      TP_LAUNCH_CHECK();
      kmap.alloc(std::max<int64_t>(C1.n(), 1), s);
      extract(C1, keep, nb, W.data(), *next, nullptr, kmap.get(), s);
    }
    L.up.alloc(std::max<int64_t>(L.n(), 1), s);
    launch(k_fill, grid_for(L.n(), 256), 256, 0, s, L.up.get(), L.n(), -1);
    launch(k_up, grid_for(nw, 256), 256, 0, s, map.get(), all ? nullptr : wsel.get(),
           kmap.get(), nw, L.up.get());
    TP_LAUNCH_CHECK();
    TP_CUDA(cudaStreamSynchronize(s));  // the working union and maps are freed below
    levels.push_back(std::move(next));
  }
  ms_coarsen = t_phase.stop();
  // ---------------- initial partitioning and uncoarsening
  const int32_t top = (int32_t)levels.size() - 1;
  std::vector<int32_t> coarsest(nb, -1);
  for (int32_t l = 0; l <= top; ++l)
    for (int32_t i : levels[l]->gl) coarsest[i] = l;
  Buf<int32_t> cur;
  Buf<int64_t> B(K, s);
  for (int32_t l = top; l >= 0; --l) {
    ULevel &L = *levels[l];
    Buf<int32_t> part(std::max<int64_t>(L.n(), 1), s);
    std::vector<int32_t> F;  // graphs whose coarsest level this is
    for (int64_t j = 0; j < L.G(); ++j)
      if (coarsest[L.gl[j]] == l) F.push_back((int32_t)j);
    if (!F.empty()) {
      t_phase.start();
      const bool all = (int64_t)F.size() == L.G();
      ULevel Xl;
      Buf<int32_t> xsel;
      if (!all) {
        int64_t nx = 0;
        for (int32_t j : F) nx += L.voff[j + 1] - L.voff[j];
        xsel.alloc(std::max<int64_t>(nx, 1), s);
        extract(L, F, nb, W.data(), Xl, xsel.get(), nullptr, s);
      }
      ULevel &X = all ? L : Xl;
      std::vector<IPRoot> roots;
      int64_t maxlen = 0;
      for (int64_t j = 0; j < X.G(); ++j) {
        const int32_t i = X.gl[j];
        roots.push_back(IPRoot{(int32_t)boff[i], 0, k[i], lmax[i]});
        maxlen = std::max(maxlen, X.voff[j + 1] - X.voff[j]);
      }
      Buf<int32_t> pos(std::max<int64_t>(X.n(), 1), s);
      launch(k_fill_pos, per_graph_grid(X.G(), maxlen), 256, 0, s, X.d_voff.get(), pos.get());
      TP_LAUNCH_CHECK();
      if (all) {
        initial_partition_roots(X.g.get(), roots, pos.get(), p, part.get(), s);
      } else {
        Buf<int32_t> xp(std::max<int64_t>(X.n(), 1), s);
        initial_partition_roots(X.g.get(), roots, pos.get(), p, xp.get(), s);
        launch(k_scatter_i32, grid_for(X.n(), 256), 256, 0, s, xp.get(), xsel.get(), X.n(),
               part.get());
        TP_LAUNCH_CHECK();
        TP_CUDA(cudaStreamSynchronize(s));
      }
      ms_initial += t_phase.stop();
    }
    t_phase.start();
    if (l < top) {
      launch(k_project_up, grid_for(L.n(), 256), 256, 0, s, L.up.get(), cur.get(), L.n(),
             part.get());
      TP_LAUNCH_CHECK();
    }
    cur = std::move(part);
    block_weights(L.g.get(), cur.get(), (int32_t)K, B.get(), s);
    SegLp seg;
    seg.gid = L.gid.get();
    seg.lgid = d_bgid.get();
    seg.vb = L.d_vb.get();
    seg.lb = d_boff.get();
    seg.cap = d_lmax.get();
    seg.k = d_k.get();
    seg.ngraphs = nb;
    rebalance_moves_seg(L.g.get(), seg, L.d_gl.get(), L.G(), cur.get(), B.get(), p, s);
    lp_refine(L.g.get(), (int32_t)K, 0, p, l, cur.get(), B.get(), s, &seg);
    ms_uncoarsen += t_phase.stop();
  }
  // ---------------- results and statistics
  ULevel &L0 = *levels[0];
  int64_t maxlen = 0;
  for (int64_t j = 0; j < L0.G(); ++j) maxlen = std::max(maxlen, L0.voff[j + 1] - L0.voff[j]);
  launch(k_write_out, per_graph_grid(L0.G(), maxlen), 256, 0, s, cur.get(), L0.d_voff.get(),
         L0.d_gl.get(), d_boff.get(), d_out.get());
  block_weights(L0.g.get(), cur.get(), (int32_t)K, B.get(), s);
  Buf<int64_t> ext(L0.n() + 1, s);
  launch(k_ext_weight, grid_for(L0.n() * 32, 256), 256, 0, s, view(L0.g.get()), cur.get(), ext.get());
  TP_LAUNCH_CHECK();
  exclusive_scan_i64(ext.get(), ext.get(), L0.n(), s);
  Buf<int64_t> cutpre(L0.G() + 1, s);
  launch(k_gather_i64, grid_for(L0.G() + 1, 256), 256, 0, s, ext.get(), L0.d_voff.get(),
         L0.G() + 1, cutpre.get());
  std::vector<int64_t> hB(K), hcut(L0.G() + 1);
  TP_CUDA(cudaMemcpyAsync(hB.data(), B.get(), K * 8, cudaMemcpyDeviceToHost, s));
  TP_CUDA(cudaMemcpyAsync(hcut.data(), cutpre.get(), (L0.G() + 1) * 8, cudaMemcpyDeviceToHost, s));
  TP_CUDA(cudaStreamSynchronize(s));
  const int32_t e = read_scalar(L0.g->err.get(), s);
  TP_REQUIRE(e == 0, (tp_status)e);
  for (int32_t l = 1; l <= top; ++l) {
    const int32_t el = read_scalar(levels[l]->g->err.get(), s);
    TP_REQUIRE(el == 0, (tp_status)el);
  }
  if (!stats) return;
  const int64_t peak = mem_peak_since(mark);
  std::vector<int64_t> posn(nb, -1);
  for (int32_t l = 0; l <= top; ++l) {
    const ULevel &Lv = *levels[l];
    for (int64_t j = 0; j < Lv.G(); ++j) {
      tp_stats &S = stats[Lv.gl[j]];
      if (l == 0) {
        S = tp_stats{};
        const int32_t i = Lv.gl[j];
        S.l_max = lmax[i];
        S.u_max = U[i];
        S.levels = coarsest[i] + 1;
        S.cut = (hcut[j + 1] - hcut[j]) / 2;
        int64_t mx = 0;
        for (int32_t b = 0; b < k[i]; ++b) mx = std::max(mx, hB[(size_t)(boff[i] + b)]);
        S.max_block_weight = mx;
        S.balanced = mx <= lmax[i];
        const int64_t perfect = (W[i] + k[i] - 1) / k[i];
        S.imbalance = perfect > 0 ? (double)mx / (double)perfect - 1.0 : 0.0;
        S.ms_coarsen = ms_coarsen;
        S.ms_initial = ms_initial;
        S.ms_uncoarsen = ms_uncoarsen;
        S.peak_bytes = peak;
      }
      S.level_n[l] = Lv.voff[j + 1] - Lv.voff[j];
      S.level_m2[l] = Lv.eoff[j + 1] - Lv.eoff[j];
    }
  }
}

}  // namespace tp
