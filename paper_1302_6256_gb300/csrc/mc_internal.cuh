// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <map>
#include <string>
#include <vector>

#include "../../include/mc.h"

namespace mc {

// ------------------------------------------------------------------ host ---

extern std::atomic<int64_t> g_launches;

#define MC_CUDA_TRY(expr)                                 \
  do {                                                    \
    cudaError_t _e = (expr);                              \
    if (_e != cudaSuccess) {                              \
      mc::set_last_cuda_error(_e, #expr, __FILE__, __LINE__); \
      return (_e == cudaErrorMemoryAllocation) ? MC_ERR_OOM : MC_ERR_CUDA; \
    }                                                     \
  } while (0)

#define MC_TRY(expr)              \
  do {                            \
    int _rc = (expr);             \
    if (_rc != MC_OK) return _rc; \
  } while (0)

void set_last_cuda_error(cudaError_t e, const char *what, const char *file, int line);

// Largest candidate set a search worker holds (the big class's adjacency
// matrix); roots with more candidates are solved as induced subgraphs.
constexpr int32_t kBigCap = 4096;

// Batches whose graphs all have at most this many vertices are peeled one
// graph per block (kcore.cu); their peel order is one segment per graph.
constexpr int64_t kBatchPeelCap = 4096;

// Default device spin-wait limit (iterations of a ~100 ns back-off loop).
constexpr long long kDefaultSpinLimit = 100000000LL;

struct DevBuf {
  void *p = nullptr;
  size_t bytes = 0;
};

// Device-side error word values (0 = fine).
enum DevErr : int {
  kDevOk = 0,
  kDevTimeout = 1,      // a bounded spin-wait gave up
  kDevOverflow = 2,     // an internal capacity was exceeded
  kDevUnsupported = 3,  // neighbourhood larger than the supported maximum
  kDevCheck = 4,        // consistency check failed
};

}  // namespace mc

namespace mc {

// Workspace buffer of at least `bytes` bytes under `name` (kept across calls).
int ws_get(mc_graph *g, const char *name, size_t bytes, void **out);
// Read the device error word, reset it, and map it to an MC_ERR_* code.
int check_device_error(mc_graph *g);
// True if p is a device (or managed) pointer.
bool is_device_ptr(const void *p);

// ---- kernels (launch wrappers; each returns MC_OK or an error) ----

// Core numbers, peel (degeneracy) order and peel positions.
int launch_core_numbers(mc_graph *g, long long spin_limit);

// Heuristic (Algorithm 1).  mode 0 racy, 1 deterministic.  Raises the
// incumbent of every graph.  seeds (nullable, device; -1 = empty slot):
// vertices grown first.  warm_only (mode 0): only the warm-up part -- the
// seeds and the first warm_top positions of the visiting order (-1: 256, or
// one per graph of an interleaved batch if more).  skip: positions of the
// visiting order an earlier launch of this solve has grown already.
// grown_top (nullable): how many visiting-order positions the warm-up part
// covered.
int launch_heuristic(mc_graph *g, int mode, long long spin_limit, const int32_t *seeds, int64_t nseeds,
                     const float *scores, bool warm_only = false, int64_t skip = 0, int64_t warm_top = -1,
                     int64_t *grown_top = nullptr);
// The learned form (learned.cu): scores of the vertices with K(v) >= their
// graph's current bound (features and network fused), and the seeds -- the
// k best-scored of them (of every graph of a batch: k per graph).
int learned_scores(mc_graph *g, const mc_mlp *m, float *score);
int learned_seeds(mc_graph *g, const float *score, int32_t k, int32_t *seeds);

// Pruned, oriented graph and the root lists (see prune.cu).
struct Pruned {
  int64_t n = 0, arcs = 0;         // vertices and arcs of the oriented graph
  int32_t max_out = 0;             // largest out-degree
  int64_t nroots_small = 0, nroots_block = 0, nroots_big = 0;
  int64_t row_entries = 0;         // CSR row entries read for the kept vertices
  int64_t *orow = nullptr;         // n+1, each row start a multiple of 4 (int4 loads)
  int32_t *ocol = nullptr;         // arcs (padded rows, pad = -1)
  int32_t *ocore = nullptr;        // core number per pruned vertex
  int32_t *oold = nullptr;         // original vertex id
  int32_t *ogid = nullptr;         // graph id (nullptr for one graph)
  int32_t *roots = nullptr;        // root list storage
  int32_t *roots_small = nullptr;  // roots by class, each in processing order
  int32_t *roots_block = nullptr;
  int32_t *roots_big = nullptr;
  int32_t *roots_huge = nullptr;   // more than kBigCap candidates (single graphs only)
  int64_t nroots_huge = 0;
  int32_t *odeg = nullptr;         // out-degree per pruned vertex
  int64_t *d_counts = nullptr;     // device: [0] n', [1] arcs, [2] max out-degree, [3..5] roots per class,
                                   // [6] row entries, [7] roots of more than kBigCap candidates
};
// No host synchronisation: sizes stay in pg.d_counts (see read_pruned_counts).
// part_rank / part_count: keep only the roots whose position in the peel
// order is part_rank modulo part_count (1: every root).
// pos_lo / pos_hi: keep only the roots at peel positions [pos_lo, pos_hi).
int launch_prune(mc_graph *g, int ordering, const float *scores, int32_t warp_max, Pruned *out,
                 long long spin_limit, int32_t part_rank = 0, int32_t part_count = 1, int64_t pos_lo = 0,
                 int64_t pos_hi = INT64_MAX);
// New root lists over an existing pruned graph (ordering 0), for the roots at
// peel positions [pos_lo, pos_hi).
int relaunch_roots(mc_graph *g, int32_t warp_max, Pruned *pg, int32_t part_rank, int32_t part_count, int64_t pos_lo,
                   int64_t pos_hi);
int read_pruned_counts(mc_graph *g, Pruned *out);

// Search (InitialBranch + Branch) over all roots.
struct SearchCounters {
  unsigned long long roots_colored, roots_branched, nodes, donations, entries, entries_block, tasks;
  unsigned long long *d_counters;  // device copy, read by read_search_counters
};
int read_search_counters(mc_graph *g, SearchCounters *cnt);
// Record event i of the graph on its stream (external when capturing).
int record_event(mc_graph *g, int i);
// layout 1: every block-class root in the 1,024-candidate layout; no_bitmap:
// member lookups by hash table only.
int launch_search(mc_graph *g, const Pruned &pg, int no_neigh_cores, int no_split, int split_nodes,
                  long long spin_limit, SearchCounters *counters, int layout = 0, int no_bitmap = 0);

}  // namespace mc

struct mc_graph {
  int64_t n = 0, nnz = 0;
  int32_t count = 1;
  int device = 0, sm_count = 0;
  cudaStream_t stream = nullptr;
  bool borrowed = false;
  // CSR (device)
  int64_t *row_ptr = nullptr;
  int32_t *col_idx = nullptr;
  int64_t *voff = nullptr;    // count+1 (device)
  int64_t *h_voff = nullptr;  // count+1 (host)
  int32_t *gid = nullptr;     // n graph ids (device), nullptr for a single graph
  int32_t max_degree = 0;
  int64_t max_graph_n = 0;  // largest graph of a batch
  // core numbers cache
  bool cores_valid = false;
  int32_t max_core = 0;
  int32_t heur0 = 0;  // heuristic clique size of graph 0 in the last solve
  unsigned long long *d_heur_ctr = nullptr;  // heuristic work counters of the last solve (device)
  bool heur_ran = false;                     // the last solve ran the heuristic
  bool learned_ran = false;                  // the last solve was the learned form
  bool repeel_ran = false;                   // the last solve searched its roots in ranges
  mc::SearchCounters repeel_acc{};           // ... and these are its counters summed over the ranges
  int32_t repeel_rebuilds = 0;               // ... and the pruned graph was rebuilt this often
  int64_t repeel_roots = 0;                  // ... over this many roots in all
  int32_t lb = 0;                            // incumbent a solve starts from (induced subgraphs of large roots)
  bool huge_mark_ready = false;              // the induced-subgraph member map is all -1
  int64_t huge_roots = 0;                    // roots of the last solve solved as induced subgraphs
  int32_t warp_max_used = 128;  // warp/block split of the current solve
  bool capturing = false;       // inside CUDA graph capture: no host synchronisation
  int32_t *core = nullptr, *order = nullptr, *pos = nullptr;  // n each (device)
  // incumbent, one per graph: size, lock, witness area (vertex-offset indexed)
  int32_t *best = nullptr, *lock = nullptr, *wit = nullptr;
  // device error word and small control block
  int32_t *err = nullptr;
  // named workspace buffers (grown on demand, reused across calls)
  std::map<std::string, mc::DevBuf> ws;
  // pinned host staging for small results
  void *h_small = nullptr;
  cudaEvent_t ev[15] = {};  // 0-5 stages, 6-7 graph replay order, 8-12 search kernels, 13-14 learned scoring
  // captured solve (CUDA graph replay) and what it was captured with
  cudaGraphExec_t graph_exec = nullptr;
  cudaStream_t cap_stream = nullptr;
  uint64_t graph_key = 0;
  mc::Pruned graph_pg;
  mc::SearchCounters graph_sc{};
  int32_t *graph_ok = nullptr;
};

namespace mc {

// Witness verification of every graph's incumbent: writes per-graph flags.
int launch_verify(mc_graph *g, int32_t *d_ok);
int launch_verify_set(mc_graph *g, const int32_t *d_vs, int32_t k, int32_t *d_ok);
// Replace the peel order by the caller's (host or device) after checking that
// it is a degeneracy order of the graph (MC_ERR_ARG otherwise).
int use_order(mc_graph *g, const int32_t *order);
int launch_validate(mc_graph *g, int32_t *d_bad);
// Candidates of pruned root j (original ids, padding dropped), read to the host.
int gather_root_row(mc_graph *g, const Pruned &pg, int32_t j, std::vector<int32_t> *out);
// CSR of the subgraph induced by `verts` (sorted original ids; local id =
// index in verts), in workspace buffers of g; *nnz its entries.
int induced_csr(mc_graph *g, const std::vector<int32_t> &verts, int64_t **d_rp, int32_t **d_ci, int64_t *nnz);
// Clique-peeling order (order.cu) into device arrays (order n, gstart n+1,
// ground n); work_out (nullable): [0] grows, [1] candidate tests.
int clique_order(mc_graph *g, const int32_t *rank, int32_t *d_order, int64_t *d_gstart, int32_t *d_ground,
                 int64_t *groups_out, int32_t *rounds_out, int64_t *work_out);
// Relabelled CSR (rows sorted) by an order (host or device), into device
// arrays; MC_ERR_ARG if the order is not a permutation.
int relabel(mc_graph *g, const int32_t *order, int64_t *d_nrp, int32_t *d_nci);
// *d_total = sum over the entries of a sorted CSR of log2(1 + gap).
int gap_bits(mc_graph *g, const int64_t *d_nrp, const int32_t *d_nci, double *d_total);
int launch_gid(mc_graph *g);
// Stable radix sort of (key, value) pairs by decreasing key (sort.cu); the
// result is back in keys / vals, ktmp / vtmp are n-entry scratch.
int radix_sort_desc(mc_graph *g, uint32_t *keys, int32_t *vals, uint32_t *ktmp, int32_t *vtmp, int64_t n);
// Indices of the k largest scores (descending), over all vertices.
int top_scores(mc_graph *g, const float *scores, int64_t k, int32_t *out);

}  // namespace mc

// ---------------------------------------------------------------- device ---

#ifdef __CUDACC__
namespace mc {
namespace dev {

__device__ __forceinline__ int ld_cg(const int *p) { return __ldcg(p); }
__device__ __forceinline__ int ld_volatile(const int *p) { return *(const volatile int *)p; }

__device__ __forceinline__ int warp_sum(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ int warp_max(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Raise the incumbent of graph gidx to `size` with the members written by
// `write(lane, base)` -- called by all 32 lanes of a warp; base is the start
// of the graph's witness area.  A per-graph lock (bounded spin) keeps the
// witness consistent with the size.  Returns true if this call raised it.
template <class WriteFn>
__device__ bool raise_incumbent(int32_t *best, int32_t *lock, int32_t *wit, const int64_t *voff, int gidx,
                                int size, int32_t *err, long long spin_limit, WriteFn write) {
  const int lane = threadIdx.x & 31;
  int ok = 0;
  if (lane == 0) {
    if (size > ld_volatile(best + gidx)) {
      long long it = 0;
      while (atomicCAS(lock + gidx, 0, 1) != 0) {
        if (++it > spin_limit) { atomicExch(err, kDevTimeout); break; }
        __nanosleep(64);
      }
      if (it <= spin_limit) ok = (size > ld_volatile(best + gidx)) ? 1 : 2;
    }
  }
  ok = __shfl_sync(0xffffffffu, ok, 0);
  if (ok == 0) return false;
  if (ok == 1) {
    int32_t *base = wit + (voff ? voff[gidx] : 0);
    write(lane, base);
    __syncwarp();
    __threadfence();
  }
  if (lane == 0) {
    if (ok == 1) {
      *(volatile int32_t *)(best + gidx) = size;
      __threadfence();
    }
    atomicExch(lock + gidx, 0);
  }
  __syncwarp();
  return ok == 1;
}

// Grid-wide barrier for a cooperative launch (all blocks co-resident).
// Bounded spin: on timeout the error word is set and the caller must return.
__device__ __forceinline__ void grid_barrier(unsigned *count, unsigned *gen, unsigned nblocks, int32_t *err,
                                             long long spin_limit) {
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned g0 = *(volatile unsigned *)gen;
    __threadfence();
    if (atomicAdd(count, 1u) == nblocks - 1) {
      *(volatile unsigned *)count = 0;
      __threadfence();
      atomicAdd(gen, 1u);
    } else {
      long long it = 0;
      while (*(volatile unsigned *)gen == g0) {
        if (++it > spin_limit) { atomicExch(err, kDevTimeout); break; }
        __nanosleep(20);
      }
    }
    __threadfence();
  }
  __syncthreads();
}

}  // namespace dev
}  // namespace mc
#endif
