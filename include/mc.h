/*
 * mc.h -- C ABI of the GB300 exact maximum-clique library.
 *
 * The library implements the method of Rossi, Gleich, Gebremedhin and Patwary,
 * "Parallel Maximum Clique Algorithms with Applications to Network Analysis and
 * Storage": core numbers (Section 3), the heuristic clique of Algorithm 1
 * (Section 4.1), pruning by core number (Section 4.2) and the neighbourhood
 * branch and bound of Algorithm 2 (Section 4.3) with the incumbent shared by
 * all workers (Section 4.5).  Every step runs in hand-written CUDA kernels for
 * sm_103a; nothing falls back to the CPU.
 *
 * Conventions (all functions):
 *  - Return an int status: MC_OK (0) or a negative MC_ERR_* code.  Nothing
 *    throws across the ABI.  mc_strerror() gives a message for a code.
 *  - Graphs are simple and undirected, in CSR form: row_ptr has n+1 int64
 *    entries with row_ptr[0] = 0, col_idx has row_ptr[n] int32 entries, each
 *    row sorted ascending, no self-loops, no duplicates, and the pattern is
 *    symmetric (u in N(v) iff v in N(u)).  MC_VALIDATE checks this on load.
 *  - Any array argument may be a host pointer or a device pointer of the
 *    current device; the library tells them apart by pointer attributes.  The
 *    caller owns every array it passes; without MC_BORROW the library copies
 *    its inputs, so the caller may free them as soon as the call returns.
 *  - All work of a graph runs on the CUDA stream given to its load call.  Calls
 *    are synchronous with respect to their outputs: when a call returns, its
 *    outputs (host or device) are written.
 *  - Vertex ids are 0..n-1 in the caller's numbering; witnesses are sorted
 *    ascending.  An empty graph (n = 0) has omega = 0; a graph with vertices but
 *    no edges has omega = 1 (witness {0}).
 *  - If an output capacity is smaller than the result, the call returns
 *    MC_ERR_BUFFER and still writes the required size to the size output.
 *  - A handle may be used from one host thread at a time.
 */
#ifndef MC_H
#define MC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define MC_OK 0
#define MC_ERR_ARG (-1)           /* bad argument (NULL handle, negative size, ...) */
#define MC_ERR_INVALID_GRAPH (-2) /* CSR not simple / not symmetric / out of range */
#define MC_ERR_OOM (-3)           /* device allocation failed */
#define MC_ERR_BUFFER (-4)        /* output capacity too small */
#define MC_ERR_TIMEOUT (-5)       /* a device spin-wait exceeded its iteration limit */
#define MC_ERR_CUDA (-6)          /* a CUDA runtime call failed */
#define MC_ERR_DEVICE_CHECK (-7)  /* a device-side consistency check failed */
#define MC_ERR_UNSUPPORTED (-8)   /* a batch graph with K(G) above 4,096, the largest neighbourhood a worker holds */
#define MC_ERR_TOO_LARGE (-9)     /* input larger than mc_core_numbers_noalloc's fixed scratch */

/* load flags */
#define MC_VALIDATE 1u /* check the CSR invariants on the device (MC_ERR_INVALID_GRAPH) */
#define MC_BORROW 2u   /* keep the caller's device arrays instead of copying them;
                          they must stay valid and unchanged until mc_free */

typedef struct mc_graph mc_graph;
typedef struct mc_mlp mc_mlp; /* the learned ordering's scoring network (below) */

/* Search options.  Zero-initialise for the defaults. */
typedef struct {
  /* order in which root vertices are searched: 0 = degeneracy order, smallest
   * core first (Algorithm 2's smallest reduced degree, Section 4.3);
   * 1 = decreasing learned score (scores below); 2 = native vertex-id order
   * (the paper's "pmc-native" variant, Section 5) */
  int32_t ordering;
  /* 1 = skip the neighbourhood-core test of InitialBranch (the paper's
   * "pmc no neigh cores" variant, Section 5); 0 = use it (default) */
  int32_t no_neigh_cores;
  /* heuristic: 0 = Algorithm 1 with the running maximum shared by all
   * workers (default); 1 = deterministic form; 2 = skip (start from 0);
   * 3 = its warm-up part only: the printed algorithm from the seeds and the
   * 256 start vertices of highest core number, each grown by a whole block
   * (on graphs whose densest core holds a maximum clique this reaches the
   * full heuristic's bound at a fraction of its cost) */
  int32_t heuristic;
  /* worker split: neighbourhoods with more than this many candidates go to
   * block workers; 0 = tuned default */
  int32_t warp_max;
  /* device spin-wait iteration limit; 0 = default (about ten seconds) */
  int64_t spin_limit;
  /* ordering == 1: one float score per vertex (host or device), higher first;
   * for a batch, one score per vertex of the union */
  const float *scores;
  /* heuristic seeds from the scores: the `seeds` vertices of highest score
   * (over all graphs of a batch) are grown first, each by Algorithm 1's
   * greedy step with one change: the next member is the remaining candidate
   * of highest score (ties: larger core number, smaller id); 0 = none */
  int32_t seeds;
  /* 1 = run the whole solve as one CUDA graph: the first call with these
   * options solves directly (sizing every buffer), then captures the solve;
   * later calls replay it with one graph launch.  Host-resident scores are
   * copied to the device before every replay, so a replay sees their
   * current values.  0 = direct launches. */
  int32_t graph;
  /* 1 = every worker searches its root's whole tree itself (the warps of a
   * block worker still share it through the block's pool); 0 = (default) a
   * worker that expands more than its budget of Branch nodes on one root
   * copies the root's adjacency matrix to a device arena and turns the
   * untried branches of its stack into tasks of one GPU-wide queue, which
   * every block serves, so one hard neighbourhood spreads over the GPU */
  int32_t no_split;
  /* Branch nodes a warp worker expands on one root before it spills the
   * rest of its tree to the task queue (a block worker: four times as
   * many); 0 = default (4096) */
  int32_t split_nodes;
  /* The learned form (an extension; the paper has no learned part): a
   * scoring network from mc_mlp_create, or NULL.  With a network, the solve
   * first runs the warm-up part of Algorithm 1, then scores only the
   * vertices that can still be in a clique larger than its bound (K(v) >=
   * bound; features and network fused in one kernel, nothing written for
   * the others), grows the `seeds` best-scored of them first (for a batch:
   * of every graph; 0 = 64 for one graph, 2 per graph for a batch; at most
   * 1,024 for one graph), each by Algorithm 1's greedy step with the next
   * member chosen by score, and then the rest of Algorithm 1 (heuristic 0)
   * or nothing more (heuristic 3; other heuristic values are refused).
   * Roots stay in degeneracy order unless ordering = 1, which orders them by
   * these scores (scores must be NULL).  omega is exact whatever the
   * network predicts.  The network must not be freed or changed while a
   * captured solve (graph = 1) that uses it can be replayed. */
  const mc_mlp *mlp;
  /* Root partition over several ranks (Section 4.5 spreads the roots of the
   * search over processors).  With part_count > 1 the search takes only the
   * roots whose position in the degeneracy order is congruent to part_rank
   * modulo part_count; everything else (core numbers, heuristic, pruning)
   * runs whole.  Every clique has exactly one lowest-ranked member, so the
   * largest clique over all parts is omega -- provided every part uses the
   * same order: pass one rank's mc_peel_order() as `order` on every rank.
   * order: n int32, host or device, a degeneracy order of this graph (each
   * vertex has at most K(v) neighbours after it), or NULL for the library's
   * own; an order that is not one is refused with MC_ERR_ARG.  Not with
   * graph = 1 or a batch (MC_ERR_ARG).  part_count 0 or 1: every root. */
  const int32_t *order;
  int32_t part_rank, part_count;
  /* Block-worker layout (an autotuner coordinate): 0 = (default) roots of at
   * most 512 candidates searched in a 512-bit-row layout at two blocks per
   * SM, larger ones in the 1,024-bit-row layout at one block per SM; 1 =
   * every block-class root in the 1,024-bit-row layout. */
  int32_t layout;
  /* 1 = neighbourhood builds look up P's members in a hash table only; 0 =
   * (default) in a shared-memory bitmap of the root's later ranks when those
   * fit (196,608 ranks), in the hash table otherwise (an autotuner
   * coordinate). */
  int32_t no_bitmap;
  /* Work-triggered re-pruning (the paper's periodic explicit rebuild,
   * Algorithm 2 line 9, triggered by progress instead of a clock): with
   * repeel = R >= 2 the roots are searched in R ranges of peel positions,
   * the densest first; before each later range, if omega has risen above the
   * bound the pruned graph was built with, the pruned graph is rebuilt with
   * the new bound (vertices with K(v) < omega dropped, rows shortened).
   * One graph, degeneracy-order roots, direct launches only (MC_ERR_ARG
   * with graph = 1, ordering != 0 or a batch).  0 or 1 = one pass. */
  int32_t repeel;
} mc_options;

/* Per-call statistics (all times in milliseconds, CUDA events). */
typedef struct {
  double ms_total, ms_cores, ms_heuristic, ms_prune, ms_search, ms_verify;
  /* the search stage by kernel: block workers, big-neighbourhood workers,
   * warp workers, the task queue (0 where a kernel did not run) */
  double ms_search_block, ms_search_big, ms_search_warp, ms_search_tasks;
  int64_t n, edges;            /* vertices and undirected edges */
  int64_t pruned_n;            /* vertices left after the core pruning (Section 4.2) */
  int64_t pruned_arcs;         /* arcs of the oriented pruned graph */
  int64_t roots;               /* root vertices queued for InitialBranch */
  int64_t roots_colored;       /* roots that reached the colouring test */
  int64_t roots_branched;      /* roots that reached Branch */
  int64_t nodes;               /* Branch nodes expanded */
  int64_t donations;           /* subproblems handed to other warps */
  int64_t neighbourhood_entries; /* later-neighbour row entries read to build the
                                    roots' adjacency matrices (Fact 3's work) */
  int64_t neighbourhood_entries_block; /* ... of which read by block workers */
  int64_t tasks;               /* subproblems spilled to the task queue */
  int64_t heuristic_grows;     /* start vertices grown by Algorithm 1 */
  int64_t heuristic_tests;     /* adjacency tests of its greedy steps */
  int64_t heuristic_row_entries; /* CSR row entries it read (gathers, merges) */
  int32_t max_core, heuristic_size, omega, verified;
  int64_t prune_row_entries;   /* CSR row entries the pruning read (the kept vertices' rows) */
  double ms_learned;           /* of ms_heuristic: scoring the candidates and picking the seeds
                                  (the learned form only) */
  int64_t learned_scored;      /* vertices the learned form scored */
  int64_t rebuilds;            /* pruned-graph rebuilds of a re-pruning solve (repeel) */
  int64_t huge_roots;          /* roots of more than 4,096 candidates, solved as induced subgraphs */
} mc_stats;

/* ------------------------------------------------------------ graphs --- */

/* Load a graph (CSR as described above).  flags: MC_VALIDATE, MC_BORROW.
 * cuda_stream: a cudaStream_t (NULL = legacy default stream).
 * On success *out owns a device copy (or borrows, with MC_BORROW). */
int mc_load_csr(int64_t n, const int64_t *row_ptr, const int32_t *col_idx, uint32_t flags,
                void *cuda_stream, mc_graph **out);

/* Load a batch of independent graphs as one block-diagonal CSR: graph g owns
 * vertices voff[g] .. voff[g+1]-1 (voff has count+1 int64 entries, voff[0] = 0,
 * voff[count] = n) and its columns are ids of the union.  No edge may join two
 * graphs (checked with MC_VALIDATE).  Every per-graph call below then works on
 * all graphs at once. */
int mc_load_batch(int32_t count, const int64_t *voff, const int64_t *row_ptr, const int32_t *col_idx,
                  uint32_t flags, void *cuda_stream, mc_graph **out);

/* Release a graph and all device memory it holds.  NULL is accepted. */
void mc_free(mc_graph *g);

/* Vertices, undirected edges and graph count of a loaded graph. */
int mc_graph_info(const mc_graph *g, int64_t *n, int64_t *edges, int32_t *count);

/* ------------------------------------------------------- the method --- */

/* Core numbers (Section 3: K(v) = largest k with v in the k-core), computed by
 * a bucketed parallel peel.  core_out: n int32 (nullable); max_core_out: the
 * largest core number K(G) (nullable; for a batch, the largest over graphs). */
int mc_core_numbers(mc_graph *g, int32_t *core_out, int32_t *max_core_out);

/* Heuristic clique (Algorithm 1, Section 4.1).  mode 0: the algorithm with the
 * running maximum shared by all workers (the result may differ from run to
 * run; it is always a clique); mode 1: deterministic -- the largest greedy
 * clique over all start vertices, ties to the smallest start vertex.
 * core: accepted for the interface and not read -- core numbers are unique,
 * and the library uses its own (computed on first use).  clique_out: capacity
 * int32 (sorted ascending); size_out: its size.  For a batch, graph 0 only;
 * use mc_max_clique_batch for all graphs. */
int mc_heuristic_clique(mc_graph *g, const int32_t *core, int32_t mode, int32_t *clique_out,
                        int32_t capacity, int32_t *size_out);

/* Exact maximum clique (Algorithm 2: CoreNumbers, HeuristicClique, pruning,
 * InitialBranch and Branch for every root, incumbent shared by all workers).
 * opt: NULL for defaults.  omega_out: omega(G); witness_out: capacity int32, a
 * maximum clique sorted ascending and verified on the device; stats nullable.
 * A root with more than 4,096 candidates (possible only when K(G) > 4,096)
 * does not fit a worker's adjacency matrix: it is solved as the graph its
 * candidates induce, by the same pipeline, from the incumbent as a lower
 * bound (stats->huge_roots counts them; such graphs are never captured with
 * opt->graph).  For a batch handle, K(G) > 4,096 gives MC_ERR_UNSUPPORTED
 * before anything of the search is launched. */
int mc_max_clique(mc_graph *g, const mc_options *opt, int32_t *omega_out, int32_t *witness_out,
                  int32_t capacity, mc_stats *stats);

/* Exact maximum clique of every graph of a batch in one pass of the pipeline
 * (one persistent search launch over all graphs' roots).  omegas_out: count
 * int32; witness_out: capacity int32 entries, graph g's witness at
 * witness_offsets[g] .. witness_offsets[g+1]-1 (witness_offsets: count+1 int64,
 * written by the call, in caller's vertex numbering of graph g, i.e. minus
 * voff[g]); stats nullable (summed over graphs). */
int mc_max_clique_batch(mc_graph *g, const mc_options *opt, int32_t *omegas_out, int32_t *witness_out,
                        int64_t capacity, int64_t *witness_offsets, mc_stats *stats);

/* Autotuner (an extension; the paper tunes nothing on a GPU): solves the
 * graph `repeats` times per candidate setting, one coordinate at a time,
 * starting from `base` (NULL = defaults): the work split between warp and
 * block workers (warp_max 32, 64, 128), then the task queue (no_split, or
 * split_nodes 1024, 4096, 16384), then the block-worker layout (layout 0,
 * 1) and the build's member lookup (no_bitmap 0, 1), then, from the default
 * heuristic, its warm-up part alone (heuristic 3), then CUDA-graph replay
 * (graph 0, 1).  It
 * writes the fastest setting to *best_out and its mean time (ms) to
 * *best_ms_out (nullable).  Every trial is a full exact solve. */
int mc_autotune(mc_graph *g, const mc_options *base, int32_t repeats, mc_options *best_out, double *best_ms_out);

/* The degeneracy order of the core numbers' peel (Section 3: each vertex has
 * at most K(v) neighbours after it), as computed by the last core-number
 * computation of this graph (computed now if there is none).  order_out: n
 * int32, host or device.  The order depends on the timing of the peel; pass
 * it as mc_options.order to make other solves (on this or another GPU) use
 * the same one. */
int mc_peel_order(mc_graph *g, int32_t *order_out);

/* Check a vertex set on the device: *is_clique_out = 1 iff the k vertices are
 * distinct, in range and pairwise adjacent (the definition of a clique). */
int mc_verify_clique(mc_graph *g, const int32_t *vertices, int32_t k, int32_t *is_clique_out);

/* Core numbers, like mc_core_numbers, for callers that cannot allocate
 * device memory.  The paper has no counterpart: this exists for code that
 * must not call cudaMalloc -- for example inside an allocator hook, or under
 * a host that owns every byte of device memory it gives the library.
 * Nothing is allocated: the peel's working memory is one fixed device array
 * of about 33 MB inside the library, which every GPU that loads the library
 * holds until the process exits.
 *   n: vertices, at most 1,048,576; row_ptr (n+1 int64) and col_idx
 *   (row_ptr[n] int32, at most 67,108,864 entries): a simple symmetric CSR
 *   in DEVICE memory of the current device (the caller owns it; it is only
 *   read); core_out: n int32 in device memory, written; max_core_out: host
 *   int32 or NULL, receives K(G).  cuda_stream: the stream to run on.
 * Larger inputs are rejected with MC_ERR_TOO_LARGE before anything runs.
 * What is checked: before the peel, a pass over the input checks the bounds
 * that the peel's memory accesses rely on -- row_ptr[0] = 0, row_ptr
 * nondecreasing, and every col_idx entry in [0, n) -- and returns
 * MC_ERR_INVALID_GRAPH, with nothing else run, if one fails.  What is not
 * checked: that rows are sorted, free of duplicates and self-loops, and
 * that the pattern is symmetric; on such input the call stays within its
 * buffers but the numbers it writes are not core numbers.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current.  The call synchronises
 * its stream before it returns (it reads K(G) and the device error word), so
 * it cannot be recorded into a CUDA graph.  All calls share the one array,
 * so calls that overlap on the GPU (other host threads, other streams) race
 * and must be serialised by the caller. */
int mc_core_numbers_noalloc(int64_t n, const int64_t *row_ptr, const int32_t *col_idx, int32_t *core_out,
                            int32_t *max_core_out, void *cuda_stream);

/* ------------------------------------- clique-peeling vertex order --- */
/* Section 6.2 orders the vertices for compression: take a large clique
 * (with the heuristic), remove it, repeat; the vertices follow the cliques
 * in the order they were taken, each clique's members by degree.  Here the
 * cliques are taken in rounds.  In a round every remaining vertex v grows
 * Algorithm 1's greedy clique C(v) over the remaining vertices (candidates
 * by decreasing core number, then degree, then smaller id; core numbers and
 * degrees of the whole graph); C(v) is taken iff no clique of a larger key
 * (|C|, then the smaller tie rank of its start vertex) holds one of its
 * vertices.  The cliques taken in a round are disjoint and include the one
 * of largest key; they are appended by increasing start vertex, members by
 * decreasing degree (ties: smaller id).  The first clique is the
 * deterministic heuristic's (mc_heuristic_clique mode 1) when rank is NULL.
 *   rank: NULL (tie rank = vertex id) or n int32, a permutation of [0, n)
 *     (MC_ERR_ARG otherwise).  A rank that follows the graph's structure
 *     (a path numbered end to end) takes a round per clique; a random
 *     permutation avoids that.
 *   order_out: n int32, order_out[i] = the vertex placed at position i.
 *   group_starts_out: n+1 int64 capacity; clique j occupies positions
 *     group_starts_out[j] .. group_starts_out[j+1]-1 (groups+1 entries
 *     written, the last = n).
 *   group_round_out: NULL or n int32 capacity: the round of clique j.
 *   groups_out: number of cliques.  stats: NULL or filled.
 * Outputs may be host or device memory.  Only single graphs (a batch handle
 * gives MC_ERR_ARG).  Device memory: about 4 bytes per CSR entry plus 30
 * bytes per vertex of workspace, kept by the handle. */
typedef struct {
  int32_t rounds;  /* rounds taken */
  int32_t pad_;
  int64_t grows;   /* greedy cliques grown (a clique is regrown only when a member was taken) */
  int64_t tests;   /* candidate tests of the greedy filters */
  double ms;       /* device time of the call */
} mc_order_stats;
int mc_clique_order(mc_graph *g, const int32_t *rank, int32_t *order_out, int64_t *group_starts_out,
                    int32_t *group_round_out, int64_t *groups_out, mc_order_stats *stats);

/* The graph relabelled by an order: new vertex i is order[i] (n int32, a
 * permutation, MC_ERR_ARG otherwise); row_ptr_out (n+1 int64) and col_idx_out
 * (row_ptr[n] int32) receive the new CSR with every row sorted ascending.
 * Host or device memory.  Single graphs only. */
int mc_relabel(mc_graph *g, const int32_t *order, int64_t *row_ptr_out, int32_t *col_idx_out);

/* Gap-coding cost of an order, the locality that gap-based adjacency
 * compression (bvgraph and its kind) exploits: relabel by the order (NULL =
 * the graph as it is), then in every row p, sorted, code the gap from p to
 * the first entry and between consecutive entries; *bits_out = the mean of
 * log2(1 + gap) over all entries (0 without edges).  Lower is better.
 * Each term is taken in single precision (relative error below 2^-22), the
 * sum in double. */
int mc_gap_bits(mc_graph *g, const int32_t *order, double *bits_out);

/* ------------------------------------------ learned vertex ordering --- */
/* An extension of the method, not in the paper: a small network scores the
 * vertices, and the scores only order the search's roots (mc_options.ordering
 * = 1, .scores) and seed the heuristic (.seeds).  omega stays exact whatever
 * the network predicts.  Network: 6 features -> 64 -> 64 -> 1, ReLU, BF16
 * weights with FP32 accumulation; FP32 master weights trained with Adam on
 * the mean binary cross-entropy of the logit, positives weighted by
 * pos_weight.  Parameters are a flat float array of mc_mlp_num_params()
 * entries: W1[64][6], b1[64], W2[64][64], b2[64], w3[64], b3. */
/* Per-vertex features (n x 6 float, row-major, host or device), each in
 * [0, 1]: degree, core number, a triangle count and a neighbourhood
 * colouring bound over the first 8 neighbours of core number >= K(v), and
 * the count of those neighbours (as a fraction of the degree and log-scaled);
 * the exact definitions are in learned.cu.  Computes the core numbers if
 * needed. */
int mc_features(mc_graph *g, float *feat_out);
/* Create a network with He-uniform weights from `seed` on `cuda_stream`. */
int mc_mlp_create(uint64_t seed, void *cuda_stream, mc_mlp **out);
void mc_mlp_free(mc_mlp *m);
int mc_mlp_num_params(void);
/* Copy the FP32 master parameters out / in (setting resets Adam's moments). */
int mc_mlp_get_params(mc_mlp *m, float *out);
int mc_mlp_set_params(mc_mlp *m, const float *in);
/* Logits of n feature rows (feat: n x 6; score_out: n). */
int mc_mlp_forward(mc_mlp *m, const float *feat, int64_t n, float *score_out);
/* Gradient of the loss over n rows (labels 0/1) into grad_out (num_params
 * floats) and the loss into *loss_out (nullable); parameters unchanged. */
int mc_mlp_gradient(mc_mlp *m, const float *feat, const float *label, int64_t n, float pos_weight, float *grad_out,
                    float *loss_out);
/* One Adam step (beta 0.9 / 0.999) with learning rate lr on n rows. */
int mc_mlp_train_step(mc_mlp *m, const float *feat, const float *label, int64_t n, float pos_weight, float lr,
                      float *loss_out);

/* ----------------------------------------------------- miscellaneous --- */

const char *mc_strerror(int code);
/* Library version as major*10000 + minor*100 + patch. */
int mc_version(void);
/* Number of kernel launches the library has issued in this process. */
int64_t mc_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* MC_H */
