/*
 * terapart.h — C-ABI of the GB300 (sm_103a) multilevel graph partitioner.
 *
 * The library computes the deterministic variant of the multilevel k-way
 * partitioner of "Tera-Scale Multilevel Graph Partitioning" (TeraPart):
 * size-constrained label propagation (LP) clustering (Algorithm 1, with the
 * two-phase idea of Algorithm 2 recast as GPU degree tiers), over either a
 * plain CSR graph or the paper's gap + VarInt compressed adjacency (Section
 * "Compression Scheme"), cluster contraction (Section "Contraction"), initial
 * bisection on the coarsest graph and LP refinement during uncoarsening
 * (Section "KaMinPar"). Every step runs in the library's CUDA kernels; there is
 * no CPU fallback.
 *
 * Conventions shared by every entry point
 *  - Pointers named d_* are device pointers; pointers named h_* are host
 *    pointers. Graph handles (tp_graph) are opaque, device-resident and own
 *    their memory until tp_graph_destroy.
 *  - stream is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Work is stream-ordered: an entry point may return before its kernels
 *    finish, except where it says it synchronises.
 *  - Errors are status codes; nothing throws or aborts across the ABI.
 *    Errors that kernels detect (a corrupt compressed stream, a full rating
 *    hash table) are latched in the graph's error word and returned by
 *    tp_graph_check or by the next entry point that synchronises.
 *  - Vertex ids are int32 (n < 2^31); edge offsets, node and edge weights are
 *    int64. Graphs are undirected: each edge stored in both directions,
 *    neighbour lists sorted ascending, no self-loops or duplicates, weights
 *    positive; tp_graph_from_csr rejects anything else with TP_ERR_INVALID.
 *  - A handle is not thread-safe; distinct handles may be used concurrently
 *    on distinct streams.
 *
 * Determinism: results depend only on the graph, k, eps and the semantic
 * fields of tp_params. The performance fields never change a single output
 * bit; tests run with randomised performance fields to check that.
 */
#ifndef TERAPART_H
#define TERAPART_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TP_OK = 0,
  TP_ERR_INVALID = 1, /* bad argument or malformed graph */
  TP_ERR_OOM = 2,     /* device allocation failed (nothing leaked) */
  TP_ERR_CUDA = 3,    /* a CUDA runtime call failed */
  TP_ERR_CORRUPT = 4, /* compressed stream failed validation in a kernel */
  TP_ERR_TIMEOUT = 5, /* reserved: the kernels never wait on one another */
  TP_ERR_BUDGET = 6   /* request exceeds a memory budget */
} tp_status;

typedef struct tp_graph tp_graph;

/* Parameters. The first block is semantic (changes results; the defaults are
 * the paper's five LP rounds per level and this library's readings of what
 * the paper leaves open). The second block only steers performance. */
typedef struct {
  uint64_t seed;          /* hashing seed (sub-rounds, ties, bisection seeds) */
  int32_t cluster_rounds; /* LP rounds per coarsening level (5) */
  int32_t refine_rounds;  /* LP rounds per uncoarsening level and bisection (5) */
  int32_t sub_rounds;     /* synchronous sub-rounds per round, S (8) */
  int32_t c_lim;          /* stop coarsening once n <= c_lim * k (160) */
  int32_t ip_attempts;    /* bisection attempts per tree node, T (8) */
  int32_t two_hop;        /* pack leftover singletons after clustering (1) */
  int32_t max_levels;     /* hierarchy depth limit, <= 64 (64) */
  /* performance only */
  int32_t tier_lane;     /* max degree rated one lane per vertex (32; 0 = off) */
  int32_t tier_small;    /* max degree rated with the small shared table (64) */
  int32_t tier_mid;      /* max degree rated with the large shared table (512; at most 512) */
  int32_t warps_per_block; /* warps per block in the small tier (8) */
  int32_t use_graphs;    /* 1: levels of at most graph_n vertices replay whole LP
                            rounds from a CUDA graph; 0: every round launches its
                            kernels directly (results are the same) */
  int32_t graph_n;       /* largest level (vertices, at most 2^19) whose rounds
                            are replayed from a CUDA graph (default 2^19) */
  int32_t table_slack;   /* hash-table slots per neighbour in the warp tiers,
                            rounded up to a power of two (2; 1..8) */
} tp_params;

typedef struct {
  int64_t cut;              /* edge cut of the final partition */
  int64_t max_block_weight; /* heaviest block */
  int64_t l_max;            /* block cap floor((1e6+eps_ppm) ceil(W/k) / 1e6) */
  int64_t u_max;            /* cluster cap max(1, floor(eps_ppm W / (1e6 k))) */
  double imbalance;         /* max_block_weight / ceil(W/k) - 1 */
  int32_t levels;           /* graphs in the hierarchy, input included */
  int32_t balanced;         /* 1 iff max_block_weight <= l_max */
  int64_t level_n[64];      /* vertices per level */
  int64_t level_m2[64];     /* adjacency entries (2m) per level */
  double ms_coarsen, ms_initial, ms_uncoarsen; /* device time per phase */
  double ms_lp_level0;      /* device time of the level-0 clustering rounds */
  int64_t peak_bytes;       /* most device memory the call held at once (working
                               set, including the caches it attaches to the graph) */
} tp_stats;

/* Fills p with the defaults listed above. */
void tp_params_default(tp_params *p);

/* Human-readable name of a status code (static string). */
const char *tp_status_string(tp_status s);

/* Device memory hook. alloc(bytes, stream, ctx) must return stream-ordered
 * device memory or NULL (the call then fails with TP_ERR_OOM); free(ptr,
 * bytes, stream, ctx) releases it. Passing NULL functions restores the
 * default (cudaMallocAsync / cudaFreeAsync). The hook is process-wide and
 * applies to allocations made after the call; memory is always released
 * through the hook that allocated it (graphs made earlier keep theirs), so
 * the functions must stay callable while such memory lives. The Python
 * binding installs PyTorch's caching allocator with use_torch_allocator().
 * Set it while no other library call is running. */
tp_status tp_set_allocator(void *(*alloc)(size_t, void *, void *),
                           void (*free_fn)(void *, size_t, void *, void *), void *ctx);

/* Makes a graph from CSR arrays (Section "Graph Representation": the
 * neighbours of u are adj[xadj[u] .. xadj[u+1])). host_ptrs = 1: the arrays
 * are host memory and are copied in; 0: device memory, also copied (the
 * caller keeps ownership of its arrays either way). vwgt / ewgt may be NULL
 * for unit weights (kept implicit, no array is stored). The graph is
 * validated on the device; violations return TP_ERR_INVALID. Synchronises. */
tp_status tp_graph_from_csr(int64_t n, const int64_t *xadj, const int32_t *adj,
                            const int64_t *vwgt, const int64_t *ewgt, int host_ptrs,
                            void *stream, tp_graph **out);

/* Compresses a unit-weight CSR graph into the gap + VarInt format of Section
 * "Compression Scheme": per vertex a VarInt header holding its first edge id,
 * then (degree > 10 000) a table of nchunks-1 little-endian u32 chunk offsets
 * relative to the neighbourhood start and chunks of 1 000 neighbours, each
 * chunk starting with VarInt(2|v0-u| + [v0<u]) followed by VarInt gaps; a
 * terminal header holding 2m sits at off[n]. Offsets are u32 when the stream
 * is below 4 GiB, else u64 (u64 for any stream when the environment variable
 * TP_OFFSETS_U64 is "1", to check the wide-offset path on small graphs; the
 * results do not depend on the width). TP_ERR_INVALID for weighted graphs or an already
 * compressed input. Synchronises (to size the output). */
tp_status tp_graph_compress(const tp_graph *csr, void *stream, tp_graph **out);

/* Makes a compressed graph from a stream in the format above: nbytes bytes
 * and n+1 u64 offsets (host_ptrs as for tp_graph_from_csr; copied in; kept
 * on the device as u32 or u64 by the rule of tp_graph_compress). Every
 * neighbourhood is decoded once on the device to validate it; a malformed
 * stream (bad header, truncated VarInt, id out of range, wrong chunk table,
 * unsorted ids) gives TP_ERR_CORRUPT. Synchronises. */
tp_status tp_graph_from_compressed(int64_t n, uint64_t nbytes, const uint8_t *bytes,
                                   const uint64_t *off, int host_ptrs, void *stream,
                                   tp_graph **out);

/* The interval + edge-weight format (Section "Compression Scheme": runs of
 * >= 3 consecutive neighbour ids stored as intervals, edge weights VarInt-
 * coded and interleaved with the codes they belong to). Headers, chunking
 * and the terminal header are those of tp_graph_compress. A chunk with
 * intervals (intervals != 0) starts with VarInt(number of maximal runs of >= 3
 * consecutive ids); each run, smallest first, is VarInt(start code: the
 * first run 2|x-u| + [x<u], a later one x - previous end - 2), VarInt(length
 * - 3) and, with weights, its members' weights; the remaining ids follow as
 * in the plain format. With weights (weights != 0; a unit-weight graph writes
 * ones) every id or gap code is followed by VarInt(2|w - w'| + [w < w']), w'
 * the chunk's previous weight in storage order (0 first). Without either it
 * is the plain stream of tp_graph_compress.
 * tp_encode_ex encodes the CSR graph g: d_off (n + 1 u64, device, caller-
 * owned) receives every vertex's byte offset (off[n]: the terminal header),
 * *nbytes the stream's length, and, when d_bytes (device, at least *nbytes
 * bytes) is not NULL, the stream itself. TP_ERR_INVALID for a compressed g.
 * Synchronises. */
tp_status tp_encode_ex(const tp_graph *g, int32_t intervals, int32_t weights, uint64_t *d_off,
                       uint8_t *d_bytes, uint64_t *nbytes, void *stream);

/* Decodes such a stream (device pointers, caller-owned) into a new CSR graph
 * (with its edge weights when weighted != 0, unit weights otherwise). A
 * malformed stream (bad header or chunk table, truncated VarInt, id out of
 * range, unsorted ids, a residual inside a run, a weight below 1) gives
 * TP_ERR_CORRUPT; a decoded graph that is not a valid symmetric graph gives
 * TP_ERR_INVALID. The rating kernels read the plain format only, so such a
 * graph is partitioned as CSR. Synchronises. */
tp_status tp_graph_from_stream_ex(int64_t n, uint64_t nbytes, const uint8_t *d_bytes,
                                  const uint64_t *d_off, int32_t intervals, int32_t weighted,
                                  void *stream, tp_graph **out);

/* Decodes a compressed graph back to CSR (round-trip check); corrupt streams
 * give TP_ERR_CORRUPT. Synchronises. */
tp_status tp_graph_decompress(const tp_graph *g, void *stream, tp_graph **out_csr);

/* Sizes of a graph: n, adjacency entries 2m, whether it is compressed, the
 * bytes its arrays occupy on the device, and (compressed graphs) the length
 * of the byte stream alone. Any output pointer may be NULL. */
tp_status tp_graph_info(const tp_graph *g, int64_t *n, int64_t *m2, int *compressed,
                        size_t *bytes, size_t *stream_bytes);

/* Copies a CSR graph out to caller device buffers (xadj n+1, adj 2m, vw n,
 * ew 2m; any may be NULL; unit weights are written as ones). */
tp_status tp_graph_export_csr(const tp_graph *g, int64_t *d_xadj, int32_t *d_adj, int64_t *d_vw,
                              int64_t *d_ew, void *stream);

/* Copies a compressed graph out: d_bytes gets the stream (size from
 * tp_graph_info), d_off gets n+1 offsets widened to u64. */
tp_status tp_graph_export_compressed(const tp_graph *g, uint8_t *d_bytes, uint64_t *d_off,
                                     void *stream);

/* Returns (and clears) the error latched by kernels working on g. Synchronises. */
tp_status tp_graph_check(const tp_graph *g, void *stream);

void tp_graph_destroy(tp_graph *g);

/* One synchronous LP sub-round (Algorithm 1 restricted to the vertices u with
 * hash(round_key, u) mod S == s) on caller state: d_label[n] in [0, nlabels),
 * d_lw[nlabels] the label weights (sum of node weights per label). A vertex
 * moves to the admissible label with the largest rating (ties: 32-bit tie
 * hash, then label) if that rating exceeds the rating of its own label;
 * admissible means lw + c(u) <= cap. Movers into a label whose weight would
 * overflow are approved in (gain desc, vertex asc) order while the inclusive
 * prefix fits. round_key = hash(seed, phase tag, a, b) as documented in the
 * library's determinism notes. In place on d_label and d_lw. */
tp_status tp_lp_subround(const tp_graph *g, int32_t *d_label, int64_t *d_lw, int64_t nlabels,
                         int64_t cap, uint64_t round_key, int32_t S, int32_t s, void *stream);

/* Size-constrained LP clustering of one coarsening level (Algorithm 1;
 * Algorithm 2's split into low-degree and high-degree work becomes the
 * library's degree tiers and never changes the result): singleton start,
 * p->cluster_rounds rounds of p->sub_rounds sub-rounds with cluster cap
 * max_cluster_weight, then (p->two_hop) packing of leftover singletons that
 * share a favourite cluster. d_cluster[n] receives the cluster label of
 * every vertex (a label is a vertex id). */
tp_status tp_lp_cluster(const tp_graph *g, int64_t max_cluster_weight, const tp_params *p,
                        int32_t level, int32_t *d_cluster, void *stream);

/* Contraction (Section "Contraction"): coarse vertex = cluster, coarse ids =
 * ranks of the labels in ascending order, coarse node weight = cluster
 * weight, coarse edge weight w'(a,b) = sum of w(u,v) over fine edges between
 * the clusters (intra-cluster edges dropped), neighbours sorted ascending.
 * *coarse receives a new CSR graph; d_map[n] (nullable) the coarse id of
 * every fine vertex. Synchronises (to size the coarse graph). */
tp_status tp_contract(const tp_graph *g, const int32_t *d_cluster, void *stream,
                      tp_graph **coarse, int32_t *d_map);

/* Initial partition of (usually) the coarsest graph by recursive bisection
 * (Section "KaMinPar": greedy graph growing plus 2-way refinement; here BFS
 * growing plus 2-way LP, p->ip_attempts seeded attempts per bisection, the
 * smallest cut wins). d_part[n] receives blocks in [0, k). Synchronises. */
tp_status tp_initial_partition(const tp_graph *g, int32_t k, int64_t l_max, const tp_params *p,
                               int32_t *d_part, void *stream);

/* Size-constrained LP refinement (Section "KaMinPar"): p->refine_rounds rounds
 * of LP over blocks with cap l_max, in place on d_part[n]. */
tp_status tp_lp_refine(const tp_graph *g, int32_t k, int64_t l_max, const tp_params *p,
                       int32_t level, int32_t *d_part, void *stream);

/* Greedy rebalancing: while a block exceeds l_max, move the vertex of the
 * lowest-index overloaded block with the smallest connectivity loss to the
 * best admissible block. *balanced = 1 when done, 0 if no vertex fits.
 * Synchronises. */
tp_status tp_rebalance(const tp_graph *g, int32_t k, int64_t l_max, int32_t *d_part,
                       int *balanced, void *stream);

/* Edge cut and block weights of a partition (problem statement of the
 * paper's introduction). h_block_weights (nullable) has k entries.
 * Synchronises. */
tp_status tp_metrics(const tp_graph *g, const int32_t *d_part, int32_t k, int64_t *cut,
                     int64_t *h_block_weights, void *stream);

/* tp_metrics without device allocation: the same cut and block weights,
 * with the scratch (cut accumulator, a bad-id flag and k block sums) in a
 * fixed array inside the library instead of memory from the allocator. For
 * callers that cannot allocate device memory when they need the metrics:
 * services whose device-memory footprint is fixed up front (admission by
 * memory budget, pools that must not grow) and callers without an allocator
 * of their own. The paper has no counterpart; this is an interface
 * convenience.
 *  - k must be <= 16383 (scratch of 16 385 eight-byte words, about 128 KiB,
 *    kept by every GPU that loads the library until the process exits);
 *    larger k returns TP_ERR_BUDGET.
 *  - Every d_part[u] must lie in [0, k); otherwise TP_ERR_INVALID (such
 *    entries are skipped on the device, never written out of bounds).
 *  - The first call on a device looks up the array's device address.
 *  - The call synchronises the stream and writes host outputs, so it cannot
 *    be captured into a CUDA graph: on a capturing stream it returns
 *    TP_ERR_INVALID before enqueuing anything (the capture is not broken).
 *  - Every call uses the same array: calls whose work overlaps on the GPU
 *    (concurrent streams, other host threads) race and give wrong sums.
 *  - cut and h_block_weights (nullable, k entries) are host outputs. */
tp_status tp_metrics_static(const tp_graph *g, const int32_t *d_part, int32_t k, int64_t *cut,
                            int64_t *h_block_weights, void *stream);

/* The full multilevel partitioner (Section "The Multilevel Scheme"):
 * coarsen with LP clustering + contraction until n <= c_lim * k (or a level
 * shrinks by less than 5%, or max_levels), partition the coarsest graph,
 * then per level project, rebalance if needed and refine. Block cap
 * L_max = floor((1e6 + eps_ppm) * ceil(W/k) / 1e6), eps_ppm = llround(eps * 1e6).
 * p may be NULL (defaults). d_part[n] receives blocks in [0, k). stats
 * (nullable) is filled on return; the call synchronises the stream. */
tp_status tp_partition(const tp_graph *g, int32_t k, double eps, const tp_params *p,
                       int32_t *d_part, tp_stats *stats, void *stream);

/* Batched mode: partitions count independent graphs, graph i into k[i]
 * blocks written to the device buffer d_part[i] (graphs[i]->n entries),
 * with the shared eps and params p (NULL: defaults). The graphs are laid
 * side by side in one union graph per level and every step of the
 * multilevel scheme runs once over the union, each vertex hashing its own
 * graph's ids and checked against its own graph's caps, so every result
 * equals tp_partition of that graph alone (stats: the graph's own cut,
 * levels and sizes; the timings and peak_bytes are the group's). Graphs with
 * k = 1 or no vertices are trivial; compressed inputs are decompressed
 * first. Batches beyond 2^28 vertices, 2^30 adjacency entries or 2^15
 * graphs are cut into groups in input order; up to `concurrency` groups run
 * at once, each on a CUDA stream that a host thread creates, uses and
 * destroys on the calling thread's device. The paper partitions one graph
 * at a time; this is the serving side of the method (many small graphs keep
 * the GPU busy only together).
 *  - stats (nullable, count entries) and status (nullable, count entries)
 *    receive each graph's stats and status.
 *  - A handle may appear only once; every graph must live on the calling
 *    thread's device.
 *  - Blocks until all graphs are done; returns TP_OK or the first failing
 *    graph's status (in graph order); TP_ERR_INVALID for bad arguments
 *    before any work starts. */
tp_status tp_partition_batch(int32_t count, tp_graph *const *graphs, const int32_t *k, double eps,
                             const tp_params *p, int32_t *const *d_part, tp_stats *stats,
                             tp_status *status, int32_t concurrency);

/* ---- serving: continuous batching under a device-memory budget ---- */

/* A request server. Worker threads, each with its own CUDA stream, take
 * submitted requests in FIFO order: the oldest waiting request starts as
 * soon as a worker is free, its footprint fits in what is left of the
 * budget, and (on a resident graph) no other request is using that graph.
 * Started requests run concurrently on the device; a finished request
 * returns its footprint to the budget, which admits the next. Every request
 * runs the tp_partition path unchanged (after uploading and, if asked,
 * compressing a host graph), so its result equals tp_partition of that
 * graph alone. The paper partitions one graph per run; this is a serving
 * layer around the method. */
typedef struct tp_server tp_server;

typedef struct {
  const tp_graph *graph; /* resident device graph (not owned; the server runs one
                            request on it at a time, and the caller must not use
                            or destroy it while a request on it is queued or
                            running), or NULL: */
  int64_t n;             /*   host CSR with n vertices, uploaded per request */
  const int64_t *xadj;   /*   host, n + 1 entries; must stay valid until waited */
  const int32_t *adj;    /*   host, xadj[n] entries, same lifetime */
  int32_t compress;      /*   compress the uploaded graph before partitioning */
  int32_t k;             /* blocks (>= 1) */
  double eps;            /* imbalance, 0 <= eps < 1 */
  int32_t *part;         /* host output, n entries, valid once waited */
} tp_request;

typedef struct {
  double queued_ms;        /* submit -> start */
  double run_ms;           /* start -> done */
  double total_ms;         /* submit -> done (the request's latency) */
  int64_t footprint_bytes; /* budget the request held (tp_footprint_bytes, or the
                              whole budget when it ran again alone) */
  int64_t peak_bytes;      /* device memory it actually held at its peak */
  int32_t retries;         /* 1 if it outgrew its footprint and ran again alone */
} tp_request_info;

/* Device memory one request may hold: the partitioner's working set (and,
 * with upload != 0, the uploaded CSR and, with compress, the compressed
 * copy) for a graph of n vertices, m2 adjacency entries and k blocks, summed
 * phase by phase from the library's allocations with the default params.
 * It bounds every graph whose coarse levels together hold at most n
 * vertices and 2 m2 entries and whose coarsest graph has at most
 * min(n, 4 c_lim k) vertices (any level may consist of hubs entirely); the
 * server enforces it per request (see tp_server_create). Returns -1 for
 * invalid sizes. */
int64_t tp_footprint_bytes(int64_t n, int64_t m2, int32_t k, int32_t upload, int32_t compress);

/* Starts a server with budget_bytes of device memory for requests and
 * `workers` worker threads (1..256) on the calling thread's device. p may be
 * NULL (defaults); it applies to every request. A request is admitted by its
 * footprint and its thread may allocate at most that much: one that would
 * need more fails before allocating and runs again alone, holding the whole
 * budget, so requests never hold more than budget_bytes of device memory in
 * total. (Diagnostics: the environment variable TP_FOOTPRINT_SCALE, read
 * here, scales every footprint, which lets a test provoke such reruns.) */
tp_status tp_server_create(int64_t budget_bytes, int32_t workers, const tp_params *p,
                           tp_server **out);

/* Queues a request and returns its ticket; TP_ERR_INVALID for bad
 * arguments. A request whose footprint exceeds the whole budget is queued to
 * run alone with the budget as its cap (tp_server_wait then returns
 * TP_ERR_BUDGET if it would really need more). Never blocks on the device. */
tp_status tp_server_submit(tp_server *sv, const tp_request *req, uint64_t *ticket);

/* Blocks until the request is done, fills stats and info (both nullable)
 * and returns its status; a ticket can be waited once (TP_ERR_INVALID for
 * an unknown ticket, one already waited, or one another thread waits on). */
tp_status tp_server_wait(tp_server *sv, uint64_t ticket, tp_stats *stats, tp_request_info *info);

/* Largest sum of footprints the server has had running at once. */
int64_t tp_server_peak_in_use(tp_server *sv);

/* Runs every queued request to completion, then stops the workers and frees
 * the server. Results not yet waited for are dropped. No other thread may be
 * inside tp_server_submit or tp_server_wait on this server when it is
 * called. */
void tp_server_destroy(tp_server *sv);

/* ---- tracing ---- */

/* Number of kernels the library has launched in this process so far. */
uint64_t tp_launch_count(void);

/* Opt-in kernel timing. When enabled, the library records a CUDA event pair
 * around selected launches of the level-0 clustering rounds (the hot path
 * of Algorithm 1 / Algorithm 2) on the stream they run on, together with
 * the algorithmic bytes the launch must move. Families: 0 small-degree
 * rating (one warp per vertex), 1 mid-degree rating, 2 big-degree rating,
 * 3 chunked hub rating (both of its kernels), 4 approval and apply,
 * 5 low-degree rating with one lane per vertex. */
typedef struct {
  int32_t family;
  int64_t launches;
  double ms;    /* summed event time */
  double bytes; /* summed algorithmic bytes */
} tp_profile_entry;
void tp_profile_enable(int on);

/* Synchronises stream, folds the recorded events into out[0..max) (one
 * entry per family, index = family) and clears them. Returns the number of
 * entries written, -1 on a CUDA error. */
int tp_profile_read(tp_profile_entry *out, int max, void *stream);

#ifdef __cplusplus
}
#endif
#endif
