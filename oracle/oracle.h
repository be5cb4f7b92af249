/*
 * Sequential CPU oracle for the deterministic multilevel partitioner of
 * "Tera-Scale Multilevel Graph Partitioning" (TeraPart).
 *
 * TEST INFRASTRUCTURE ONLY. This code is the plain, slow, obviously correct
 * statement of what the GPU path computes. Only the test-suite, the smoke check
 * and the CPU-baseline leg of the benchmark may load it. The GPU library shares
 * no code, header, table or constant with it.
 *
 * Every function cites the passage of the paper it restates (section, equation
 * or algorithm). Where the paper is silent the reading taken is stated at the
 * function.
 *
 * Parity status per function:
 *   orc_varint_*, orc_encode, orc_decode  pinned (hand-computed bytes, round trip)
 *   orc_encode_ex, orc_decode_ex          pinned (hand-computed bytes, equal to
 *                                          orc_encode without intervals and
 *                                          weights, size formula, round trip)
 *   orc_lp_*                              pinned (brute-force argmax, cap invariant,
 *                                                  approval vs subset enumeration)
 *   orc_two_hop                           pinned (hand cases, restated packing)
 *   orc_cluster                           pinned (rounds by enumeration + restated
 *                                                  packing)
 *   orc_contract                          pinned (weight sums, identity, all-in-one)
 *   orc_initial_partition                 pinned: recursive bisection
 *                                          restated (growing, 2-way LP by
 *                                          enumeration, recursion)
 *   orc_refine                            pinned: rounds restated by
 *                                          enumeration (blocks as labels)
 *   orc_rebalance                         pinned: brute-force restatement
 *   orc_gt_*                              pinned (affinities recounted by brute
 *                                          force after random moves, probe-path
 *                                          invariant, footprint and widths by
 *                                          formula)
 *   orc_fm_refine                         pinned (restated by brute force on
 *                                          tiny graphs, cut and balance
 *                                          invariants, 1-opt at the end)
 *   orc_partition                         pinned: driver restated (caps,
 *                                          stop rules, projection, rebalance
 *                                          then refine) over the pinned stages,
 *                                          plus invariants (balance, cut
 *                                          bounds, projection preserves cut)
 */
#ifndef TERAPART_ORACLE_H
#define TERAPART_ORACLE_H
#include <stdint.h>
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Undirected graph in CSR form (Section "Graph Representation"): the
 * neighbours of u are adj[xadj[u] .. xadj[u+1]), sorted ascending, no
 * self-loops, no duplicates, every edge stored in both directions.
 * vw = node weights c(u) (> 0), ew = edge weights w(u,v) (> 0). A NULL vw or
 * ew means unit weights (an input graph need not carry arrays of ones);
 * every function reads weights through orc_vw / orc_ew, and coarse graphs
 * built by contraction always carry both arrays. */
typedef struct {
  int64_t n;
  int64_t m2; /* adjacency entries = 2m */
  int64_t *xadj;
  int32_t *adj;
  int64_t *vw;
  int64_t *ew;
} orc_graph;

static inline int64_t orc_vw(const orc_graph *g, int64_t u) { return g->vw ? g->vw[u] : 1; }
static inline int64_t orc_ew(const orc_graph *g, int64_t e) { return g->ew ? g->ew[e] : 1; }

/* Semantic parameters: they change results. */
typedef struct {
  uint64_t seed;
  int32_t cluster_rounds; /* LP rounds per coarsening level (5, Section "Label Propagation Clustering") */
  int32_t refine_rounds;  /* LP rounds per refinement level (5) */
  int32_t sub_rounds;     /* synchronous sub-rounds per round, S (8) */
  int32_t c_lim;          /* coarsening stops once n <= c_lim * k (160) */
  int32_t ip_attempts;    /* bisection attempts per tree node, T (8) */
  int32_t two_hop;        /* 1: pack leftover singletons after clustering */
  int32_t max_levels;     /* at most this many graphs in the hierarchy (64) */
  int32_t fm_passes;      /* k-way FM passes after LP refinement per level (0: none;
                             the GPU path has no FM, so parity runs use 0) */
} orc_params;

typedef struct {
  int64_t cut;
  int64_t max_block_weight;
  int64_t l_max;
  int64_t u_max; /* cluster weight cap U */
  double imbalance;
  int32_t levels;
  int32_t balanced; /* 1 iff every block <= l_max */
  int64_t level_n[64];
  int64_t level_m2[64];
} orc_stats;

/* ---- hashing (counter-based, used for sub-round assignment and ties) ---- */
uint64_t orc_mix64(uint64_t z);
uint64_t orc_step(uint64_t h, uint64_t x);
uint64_t orc_round_key(uint64_t seed, uint64_t tag, uint64_t a, uint64_t b);
uint64_t orc_tag(int which); /* 0 cluster, 1 refine, 2 two-hop, 3 ip-seed, 4 ip-lp, 5 tie */

/* ---- compressed adjacency (Section "Compression Scheme") ---- */
int orc_varint_len(uint64_t x);
int orc_varint_put(uint8_t *out, uint64_t x);                 /* returns bytes written */
int orc_varint_get(const uint8_t *in, int64_t avail, uint64_t *x); /* returns bytes read, 0 on error */
int64_t orc_encoded_size(int64_t n, const int64_t *xadj, const int32_t *adj);
int64_t orc_encode(int64_t n, const int64_t *xadj, const int32_t *adj, uint8_t *bytes, uint64_t *off);
/* Returns 0 on success, -1 on a corrupt stream. xadj_out has n+1 entries,
 * adj_out has m2 entries (m2 taken from the terminal header). */
int orc_decode(int64_t n, const uint8_t *bytes, int64_t nbytes, const uint64_t *off,
               int64_t *xadj_out, int32_t *adj_out, int64_t adj_cap);

/* Interval encoding and compressed edge weights (codec_iv.c). ew may be NULL
 * (unit weights, none stored); intervals = 0 gives the plain format with the
 * weights interleaved (byte for byte orc_encode without weights). bytes and
 * off may be NULL to size the stream. Returns the stream length. */
int64_t orc_encode_ex(int64_t n, const int64_t *xadj, const int32_t *adj, const int64_t *ew,
                      int intervals, uint8_t *bytes, uint64_t *off);
/* Returns 0 on success, -1 on a corrupt stream; ew_out may be NULL. */
int orc_decode_ex(int64_t n, const uint8_t *bytes, int64_t nbytes, const uint64_t *off,
                  int intervals, int weighted, int64_t *xadj_out, int32_t *adj_out,
                  int64_t *ew_out, int64_t adj_cap);

/* ---- space-efficient gain table (Section "Space-Efficient Gain Tables"; gain_table.c) ---- */
typedef struct orc_gain_table orc_gain_table;
orc_gain_table *orc_gt_build(const orc_graph *g, const int32_t *part, int32_t k);
int64_t orc_gt_get(const orc_gain_table *t, int64_t v, int32_t b); /* affinity w(v, V_b) */
/* Updates the neighbours of u for a move of u from block `from` to `to`. */
void orc_gt_move(orc_gain_table *t, const orc_graph *g, int64_t u, int32_t from, int32_t to);
int64_t orc_gt_bytes(const orc_gain_table *t); /* size of the value array */
/* v's slots (k when dense), bytes per value, dense flag and stored entries. */
void orc_gt_layout(const orc_gain_table *t, int64_t v, int64_t *cap, int32_t *width,
                   int32_t *dense, int64_t *stored);
/* 0 if every sparse table holds only non-zero values, no duplicate and every
 * key on its probe path; else a code naming the broken rule. */
int orc_gt_check(const orc_gain_table *t);
void orc_gt_free(orc_gain_table *t);

/* k-way FM over the gain table (fm.c): at most `passes` passes, in place on
 * part and B; returns the total cut reduction. */
int64_t orc_fm_refine(const orc_graph *g, int32_t *part, int64_t *B, int32_t k, int64_t l_max,
                      int32_t passes);

/* ---- label propagation (Algorithm 1, made synchronous and deterministic) ---- */
/* Decision for one vertex against a state snapshot. Returns 1 if u moves. */
int orc_rate_vertex(const orc_graph *g, int64_t u, const int32_t *label, const int64_t *lw,
                    int64_t cap_uniform, const int64_t *cap, int ignore_cap, uint64_t hv,
                    int32_t *target, int64_t *gain);
/* Same decision, ratings formed by sorting N(u) (no n-sized scratch). */
int orc_rate_vertex_sorted(const orc_graph *g, int64_t u, const int32_t *label, const int64_t *lw,
                           int64_t cap_uniform, const int64_t *cap, int ignore_cap, uint64_t hv,
                           int32_t *target, int64_t *gain);
/* One sub-round s of round key rk. Returns the number of applied moves.
 */
int64_t orc_lp_subround(const orc_graph *g, int32_t *label, int64_t *lw, int64_t nlabels,
                        int64_t cap_uniform, const int64_t *cap, uint64_t rk, int32_t S, int32_t s);
int64_t orc_lp_rounds(const orc_graph *g, int32_t *label, int64_t *lw, int64_t nlabels,
                      int64_t cap_uniform, const int64_t *cap, uint64_t seed, uint64_t tag,
                      uint64_t a, uint64_t b0, int32_t rounds, int32_t S);
void orc_two_hop(const orc_graph *g, int32_t *C, const int64_t *Wc, int64_t U, uint64_t seed,
                 int64_t level);
/* Full clustering of one coarsening level: singletons, LP rounds, two-hop. */
void orc_cluster(const orc_graph *g, int64_t U, const orc_params *p, int64_t level, int32_t *C);

/* ---- contraction (Section "Contraction") ---- */
/* Fills *out (arrays malloc'ed, release with orc_graph_free) and map[n].
 * Returns n'. */
int64_t orc_contract(const orc_graph *g, const int32_t *C, orc_graph *out, int32_t *map);
void orc_graph_free(orc_graph *g);

/* ---- initial partitioning, refinement, balance, metrics ---- */
void orc_initial_partition(const orc_graph *g, int32_t k, int64_t l_max, const orc_params *p,
                           int32_t *part);
void orc_block_weights(const orc_graph *g, const int32_t *part, int32_t k, int64_t *B);
int64_t orc_cut(const orc_graph *g, const int32_t *part);
int orc_rebalance(const orc_graph *g, int32_t *part, int64_t *B, int32_t k, int64_t l_max);
int64_t orc_refine(const orc_graph *g, int32_t *part, int64_t *B, int32_t k, int64_t l_max,
                   const orc_params *p, int64_t level);
int64_t orc_cluster_cap(int64_t W, int32_t k, int64_t eps_ppm);
int64_t orc_block_cap(int64_t W, int32_t k, int64_t eps_ppm);
int orc_validate(const orc_graph *g);
int orc_partition(const orc_graph *g, int32_t k, int64_t eps_ppm, const orc_params *p,
                  int32_t *part, orc_stats *st);

#ifdef __cplusplus
}
#endif
#endif
