// C ABI (include/mc.h): argument checks, device memory, and the pipeline of
// Algorithm 2 -- core numbers, heuristic, pruning, search, verification --
// on the graph's stream.  Every step runs in this library's CUDA kernels.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "mc_internal.cuh"

namespace mc {

std::atomic<int64_t> g_launches{0};
static thread_local char g_errbuf[320];

void set_last_cuda_error(cudaError_t e, const char *what, const char *file, int line) {
  snprintf(g_errbuf, sizeof(g_errbuf), "%s (%s) at %s:%d", cudaGetErrorString(e), what, file, line);
}

// Device-memory pool for workspace buffers: buffers of freed graphs are kept
// per device and handed to the next graph that needs one of a similar size,
// so short-lived handles (one per small graph) do not pay cudaMalloc and
// cudaFree every time.  The pool is emptied when an allocation fails.
namespace {
std::mutex g_pool_mu;
std::multimap<size_t, void *> g_pool[64];
size_t g_pool_bytes[64];
constexpr size_t kPoolLimit = (size_t)8 << 30;  // keep at most 8 GiB cached per device

void *pool_take(int dev, size_t bytes, size_t *got) {
  std::lock_guard<std::mutex> lk(g_pool_mu);
  auto &p = g_pool[dev];
  auto it = p.lower_bound(bytes);
  if (it == p.end() || it->first > 2 * bytes + (1 << 20)) return nullptr;
  void *ptr = it->second;
  *got = it->first;
  g_pool_bytes[dev] -= it->first;
  p.erase(it);
  return ptr;
}

void pool_give(int dev, void *ptr, size_t bytes) {
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (g_pool_bytes[dev] + bytes > kPoolLimit) {
    cudaFree(ptr);
    return;
  }
  g_pool[dev].emplace(bytes, ptr);
  g_pool_bytes[dev] += bytes;
}

void pool_flush(int dev) {
  std::lock_guard<std::mutex> lk(g_pool_mu);
  for (auto &kv : g_pool[dev]) cudaFree(kv.second);
  g_pool[dev].clear();
  g_pool_bytes[dev] = 0;
}
}  // namespace

int ws_get(mc_graph *g, const char *name, size_t bytes, void **out) {
  DevBuf &b = g->ws[name];
  if (bytes == 0) bytes = 16;
  if (b.bytes >= bytes) {
    *out = b.p;
    return MC_OK;
  }
  if (b.p) {
    cudaError_t e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) return MC_ERR_CUDA;
    pool_give(g->device, b.p, b.bytes);
    b.p = nullptr;
    b.bytes = 0;
  }
  size_t got = 0;
  if (void *p = pool_take(g->device, bytes, &got)) {
    b.p = p;
    b.bytes = got;
    *out = p;
    return MC_OK;
  }
  size_t want = bytes + bytes / 8;
  cudaError_t e = cudaMalloc(&b.p, want);
  if (e != cudaSuccess) {
    cudaGetLastError();
    pool_flush(g->device);
    e = cudaMalloc(&b.p, bytes);
    want = bytes;
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    b.p = nullptr;
    return MC_ERR_OOM;
  }
  b.bytes = want;
  *out = b.p;
  return MC_OK;
}

int check_device_error(mc_graph *g) {
  int32_t *h = (int32_t *)((char *)g->h_small + 2048);
  MC_CUDA_TRY(cudaMemcpyAsync(h, g->err, sizeof(int32_t), cudaMemcpyDeviceToHost, g->stream));
  MC_CUDA_TRY(cudaStreamSynchronize(g->stream));
  int e = *h;
  if (e == kDevOk) return MC_OK;
  MC_CUDA_TRY(cudaMemsetAsync(g->err, 0, sizeof(int32_t), g->stream));
  switch (e) {
    case kDevTimeout: return MC_ERR_TIMEOUT;
    case kDevUnsupported: return MC_ERR_UNSUPPORTED;
    default: return MC_ERR_DEVICE_CHECK;
  }
}

bool is_device_ptr(const void *p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// graphs whose incumbent is still 0 but have a vertex: omega = 1, witness =
// their first vertex (a graph without edges)
__global__ void trivial_kernel(int32_t count, const int64_t *voff, int64_t n, int32_t *best, int32_t *wit) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < count; g += (int64_t)gridDim.x * blockDim.x) {
    int64_t v0 = voff ? voff[g] : 0, v1 = voff ? voff[g + 1] : n;
    if (best[g] == 0 && v1 > v0) {
      wit[v0] = (int32_t)v0;
      best[g] = 1;
    }
  }
}

static void free_graph(mc_graph *g) {
  if (!g) return;
  if (g->stream) cudaStreamSynchronize(g->stream);
  // the graph's own arrays are named workspace buffers too (the CSR copy,
  // per-vertex arrays, incumbents): all go back to the pool below
  if (g->graph_exec) cudaGraphExecDestroy(g->graph_exec);
  if (g->cap_stream) cudaStreamDestroy(g->cap_stream);
  for (auto &kv : g->ws)
    if (kv.second.p) pool_give(g->device, kv.second.p, kv.second.bytes);
  if (g->h_small) cudaFreeHost(g->h_small);
  delete[] g->h_voff;
  for (auto &e : g->ev)
    if (e) cudaEventDestroy(e);
  delete g;
}

static int copy_in(void *dst, const void *src, size_t bytes, cudaStream_t s) {
  if (bytes == 0) return MC_OK;
  MC_CUDA_TRY(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, s));
  return MC_OK;
}

static int load_common(int32_t count, const int64_t *voff_in, int64_t n, const int64_t *row_ptr,
                       const int32_t *col_idx, uint32_t flags, void *stream, mc_graph **out) {
  if (!out) return MC_ERR_ARG;
  *out = nullptr;
  if (n < 0 || n > 2147483000LL || count < 1 || (n > 0 && !row_ptr)) return MC_ERR_ARG;
  if ((flags & ~(MC_VALIDATE | MC_BORROW)) != 0) return MC_ERR_ARG;
  mc_graph *g = new mc_graph();
  g->stream = (cudaStream_t)stream;
  g->count = count;
  g->n = n;
  int rc = MC_OK;
  auto fail = [&](int code) {
    free_graph(g);
    return code;
  };
  if (cudaGetDevice(&g->device) != cudaSuccess) return fail(MC_ERR_CUDA);
  if (cudaDeviceGetAttribute(&g->sm_count, cudaDevAttrMultiProcessorCount, g->device) != cudaSuccess)
    return fail(MC_ERR_CUDA);
  if (cudaMallocHost(&g->h_small, 4096) != cudaSuccess) return fail(MC_ERR_OOM);
  for (auto &e : g->ev)
    if (cudaEventCreate(&e) != cudaSuccess) return fail(MC_ERR_CUDA);
  // nnz = row_ptr[n]
  int64_t nnz = 0;
  if (n > 0) {
    if (cudaMemcpyAsync(g->h_small, row_ptr + n, sizeof(int64_t), cudaMemcpyDefault, g->stream) != cudaSuccess ||
        cudaStreamSynchronize(g->stream) != cudaSuccess)
      return fail(MC_ERR_ARG);
    nnz = *(int64_t *)g->h_small;
  }
  if (nnz < 0 || (nnz > 0 && !col_idx)) return fail(MC_ERR_ARG);
  g->nnz = nnz;
  // device arrays come from the per-device pool (as named workspace
  // buffers), so a handle loaded after another one was freed reuses its
  // memory instead of allocating
  void *wp = nullptr;
  auto take = [&](const char *name, size_t bytes) -> void * {
    return ws_get(g, name, bytes, &wp) == MC_OK ? wp : nullptr;
  };
  if (flags & MC_BORROW) {
    if ((n > 0 && !is_device_ptr(row_ptr)) || (nnz > 0 && !is_device_ptr(col_idx))) return fail(MC_ERR_ARG);
    g->row_ptr = const_cast<int64_t *>(row_ptr);
    g->col_idx = const_cast<int32_t *>(col_idx);
    g->borrowed = true;
  } else {
    if (!(g->row_ptr = (int64_t *)take("g.row_ptr", (n + 1) * sizeof(int64_t)))) return fail(MC_ERR_OOM);
    if (!(g->col_idx = (int32_t *)take("g.col_idx", std::max<int64_t>(nnz, 4) * sizeof(int32_t))))
      return fail(MC_ERR_OOM);
    if (n > 0) {
      if ((rc = copy_in(g->row_ptr, row_ptr, (n + 1) * sizeof(int64_t), g->stream)) != MC_OK) return fail(rc);
      if ((rc = copy_in(g->col_idx, col_idx, nnz * sizeof(int32_t), g->stream)) != MC_OK) return fail(rc);
    } else {
      cudaMemsetAsync(g->row_ptr, 0, sizeof(int64_t), g->stream);
    }
  }
  const size_t nv = (size_t)std::max<int64_t>(n, 1);
  if (!(g->core = (int32_t *)take("g.core", nv * 4)) || !(g->order = (int32_t *)take("g.order", nv * 4)) ||
      !(g->pos = (int32_t *)take("g.pos", nv * 4)) || !(g->wit = (int32_t *)take("g.wit", (nv + 1) * 4)) ||
      !(g->best = (int32_t *)take("g.best", count * 4)) || !(g->lock = (int32_t *)take("g.lock", count * 4)) ||
      !(g->err = (int32_t *)take("g.err", 64)) || !(g->voff = (int64_t *)take("g.voff", (count + 1) * 8)))
    return fail(MC_ERR_OOM);
  cudaMemsetAsync(g->err, 0, 64, g->stream);
  cudaMemsetAsync(g->lock, 0, count * 4, g->stream);
  cudaMemsetAsync(g->best, 0, count * 4, g->stream);
  g->h_voff = new int64_t[count + 1];
  if (voff_in) {
    if (cudaMemcpyAsync(g->h_voff, voff_in, (count + 1) * 8, cudaMemcpyDefault, g->stream) != cudaSuccess ||
        cudaStreamSynchronize(g->stream) != cudaSuccess)
      return fail(MC_ERR_ARG);
    if (g->h_voff[0] != 0 || g->h_voff[count] != n) return fail(MC_ERR_ARG);
    for (int32_t i = 0; i < count; i++) {
      if (g->h_voff[i + 1] < g->h_voff[i]) return fail(MC_ERR_ARG);
      g->max_graph_n = std::max<int64_t>(g->max_graph_n, g->h_voff[i + 1] - g->h_voff[i]);
    }
  } else {
    g->h_voff[0] = 0;
    g->h_voff[1] = n;
    g->max_graph_n = n;
  }
  if (cudaMemcpyAsync(g->voff, g->h_voff, (count + 1) * 8, cudaMemcpyHostToDevice, g->stream) != cudaSuccess)
    return fail(MC_ERR_CUDA);
  if (count > 1) {
    if (!(g->gid = (int32_t *)take("g.gid", nv * 4))) return fail(MC_ERR_OOM);
    if ((rc = launch_gid(g)) != MC_OK) return fail(rc);
  }
  if (flags & MC_VALIDATE) {
    int32_t *bad = g->err + 8;
    cudaMemsetAsync(bad, 0, 4, g->stream);
    if ((rc = launch_validate(g, bad)) != MC_OK) return fail(rc);
    if (cudaMemcpyAsync(g->h_small, bad, 4, cudaMemcpyDeviceToHost, g->stream) != cudaSuccess ||
        cudaStreamSynchronize(g->stream) != cudaSuccess)
      return fail(MC_ERR_CUDA);
    if (*(int32_t *)g->h_small) return fail(MC_ERR_INVALID_GRAPH);
  }
  if (cudaStreamSynchronize(g->stream) != cudaSuccess) return fail(MC_ERR_CUDA);
  *out = g;
  return MC_OK;
}

static long long spin_of(const mc_options *o) { return (o && o->spin_limit > 0) ? o->spin_limit : kDefaultSpinLimit; }

static int ensure_cores(mc_graph *g, long long spin) {
  if (g->cores_valid) return MC_OK;
  return launch_core_numbers(g, spin);
}

// Milliseconds between two recorded events; 0 when either was never
// recorded (the failed query's error is consumed, so a later launch check
// does not report it).
static float elapsed(cudaEvent_t a, cudaEvent_t b) {
  float ms = 0.f;
  if (cudaEventElapsedTime(&ms, a, b) != cudaSuccess) {
    (void)cudaGetLastError();
    ms = 0.f;
  }
  return ms;
}

// Record a stage event; inside capture it becomes an external event-record
// node, so the replayed graph records it and the host can wait on it.
int record_event(mc_graph *g, int i) {
  if (g->capturing) {
    MC_CUDA_TRY(cudaEventRecordWithFlags(g->ev[i], g->stream, cudaEventRecordExternal));
  } else {
    MC_CUDA_TRY(cudaEventRecord(g->ev[i], g->stream));
  }
  return MC_OK;
}

// Validated copy of the options.
static int check_options(const mc_options *opt, mc_options *o) {
  *o = mc_options{};
  if (opt) *o = *opt;
  if (o->ordering < 0 || o->ordering > 2 || o->heuristic < 0 || o->heuristic > 3 || o->warp_max < 0 ||
      o->seeds < 0 || o->graph < 0 || o->graph > 1 || o->no_split < 0 || o->no_split > 1 ||
      o->split_nodes < 0)
    return MC_ERR_ARG;
  if (o->ordering == 1 && !o->scores && !o->mlp) return MC_ERR_ARG;
  if (o->mlp && (o->scores || (o->heuristic != 0 && o->heuristic != 3) || o->seeds > 1024)) return MC_ERR_ARG;
  if (o->part_count < 0 || o->part_rank < 0 || (o->part_count > 1 && o->part_rank >= o->part_count) ||
      (o->part_count <= 1 && o->part_rank != 0))
    return MC_ERR_ARG;
  if (o->order && o->graph) return MC_ERR_ARG;
  if (o->layout < 0 || o->layout > 1 || o->no_bitmap < 0 || o->no_bitmap > 1) return MC_ERR_ARG;
  if (o->repeel < 0 || (o->repeel > 1 && (o->graph || o->ordering != 0))) return MC_ERR_ARG;
  return MC_OK;
}

static int run_max_clique(mc_graph *g, const mc_options *opt, mc_stats *st);

// Roots with more than kBigCap candidates (single graphs): each is solved as
// the graph its candidates P induce, by the whole pipeline, starting from
// the incumbent minus one as its lower bound -- a clique of G[P] of size at
// least omega extends by the root to a larger clique (every clique is found
// from its earliest member, whatever the root's class).  A root with fewer
// than omega candidates is skipped (it cannot hold omega + 1).  Synchronises
// the stream (reads the root list and the incumbent).
static int search_huge_roots(mc_graph *g, const mc_options &o, Pruned *pg) {
  if (g->count != 1 || g->max_core <= kBigCap || g->n == 0) return MC_OK;
  MC_TRY(read_pruned_counts(g, pg));
  const int64_t nh = pg->nroots_huge;
  if (nh == 0) return MC_OK;
  std::vector<int32_t> roots((size_t)nh);
  MC_CUDA_TRY(cudaMemcpyAsync(roots.data(), pg->roots_huge, (size_t)nh * 4, cudaMemcpyDeviceToHost, g->stream));
  MC_CUDA_TRY(cudaStreamSynchronize(g->stream));
  int32_t *hb = (int32_t *)((char *)g->h_small + 3584);
  for (int32_t j : roots) {
    MC_CUDA_TRY(cudaMemcpyAsync(hb, g->best, 4, cudaMemcpyDeviceToHost, g->stream));
    MC_CUDA_TRY(cudaMemcpyAsync(hb + 1, pg->odeg + j, 4, cudaMemcpyDeviceToHost, g->stream));
    MC_CUDA_TRY(cudaMemcpyAsync(hb + 2, pg->oold + j, 4, cudaMemcpyDeviceToHost, g->stream));
    MC_CUDA_TRY(cudaStreamSynchronize(g->stream));
    const int32_t om = hb[0], d = hb[1], u = hb[2];
    if (d < om) continue;
    std::vector<int32_t> P;
    MC_TRY(gather_root_row(g, *pg, j, &P));
    std::sort(P.begin(), P.end());
    int64_t *srp = nullptr;
    int32_t *sci = nullptr;
    int64_t snnz = 0;
    MC_TRY(induced_csr(g, P, &srp, &sci, &snnz));
    mc_graph *sub = nullptr;
    MC_TRY(load_common(1, nullptr, (int64_t)P.size(), srp, sci, 0, g->stream, &sub));
    sub->lb = std::max(om - 1, 0);
    mc_options so = o;
    so.graph = 0;
    so.order = nullptr;
    so.part_rank = 0;
    so.part_count = 0;
    so.repeel = 0;
    so.scores = nullptr;
    so.seeds = 0;
    so.mlp = nullptr;
    if (so.ordering == 1) so.ordering = 0;
    mc_stats sst;
    int rc = run_max_clique(sub, &so, &sst);
    int32_t sb = 0;
    std::vector<int32_t> w;
    if (rc == MC_OK) {
      if (cudaMemcpy(&sb, sub->best, 4, cudaMemcpyDeviceToHost) != cudaSuccess) rc = MC_ERR_CUDA;
      if (rc == MC_OK && sb > sub->lb && sb + 1 > om) {
        w.resize((size_t)sb + 1);
        if (cudaMemcpy(w.data() + 1, sub->wit, (size_t)sb * 4, cudaMemcpyDeviceToHost) != cudaSuccess) rc = MC_ERR_CUDA;
        w[0] = u;
        for (int32_t i = 1; i <= sb; i++) w[i] = P[w[i]];
      }
    }
    g->huge_roots += 1 + sub->huge_roots;
    free_graph(sub);
    if (rc != MC_OK) return rc;
    if (!w.empty()) {
      const int32_t size = sb + 1;
      MC_CUDA_TRY(cudaMemcpyAsync(g->wit, w.data(), (size_t)size * 4, cudaMemcpyHostToDevice, g->stream));
      MC_CUDA_TRY(cudaMemcpyAsync(g->best, &size, 4, cudaMemcpyHostToDevice, g->stream));
      MC_CUDA_TRY(cudaStreamSynchronize(g->stream));
    }
  }
  return MC_OK;
}

// The search with work-triggered re-pruning: the kept vertices form a suffix
// of the peel order (K(v) >= bound); its roots are searched in o.repeel
// ranges of peel positions, densest first, and before each later range the
// pruned graph is rebuilt if the incumbent has risen above the bound it was
// built with (else only the root lists are made).  Reads the incumbent and
// the pruned size on the host between ranges.
static int search_in_ranges(mc_graph *g, const mc_options &o, Pruned *pg, SearchCounters *sc, long long spin) {
  const int32_t pr = o.part_count > 1 ? o.part_rank : 0, pc = std::max(o.part_count, 1);
  int32_t *h = (int32_t *)((char *)g->h_small + 3072);
  MC_CUDA_TRY(cudaMemcpyAsync(h, g->best, sizeof(int32_t), cudaMemcpyDeviceToHost, g->stream));
  MC_TRY(launch_prune(g, 0, nullptr, g->warp_max_used, pg, spin, pr, pc));
  MC_TRY(read_pruned_counts(g, pg));  // synchronises: *h is the bound the pruned graph was built with
  int32_t bound = *h;
  const int64_t n0 = pg->n;
  MC_TRY(record_event(g, 3));
  SearchCounters acc{};
  g->repeel_rebuilds = 0;
  g->repeel_roots = 0;
  const int R = o.repeel;
  bool searched = false;
  for (int c = 0; c < R; c++) {
    const int64_t hi = g->n - n0 * c / R, lo = g->n - n0 * (c + 1) / R;
    if (hi <= lo) continue;
    if (c > 0) {
      MC_CUDA_TRY(cudaMemcpyAsync(h, g->best, sizeof(int32_t), cudaMemcpyDeviceToHost, g->stream));
      MC_CUDA_TRY(cudaStreamSynchronize(g->stream));
    }
    if (c > 0 && *h > bound) {
      bound = *h;
      MC_TRY(launch_prune(g, 0, nullptr, g->warp_max_used, pg, spin, pr, pc, lo, hi));
      g->repeel_rebuilds++;
    } else {
      MC_TRY(relaunch_roots(g, g->warp_max_used, pg, pr, pc, lo, hi));
    }
    MC_TRY(launch_search(g, *pg, o.no_neigh_cores, o.no_split, o.split_nodes, spin, sc, o.layout, o.no_bitmap));
    MC_TRY(search_huge_roots(g, o, pg));
    searched = true;
    MC_TRY(read_search_counters(g, sc));
    MC_TRY(read_pruned_counts(g, pg));
    g->repeel_roots += pg->nroots_small + pg->nroots_block + pg->nroots_big;
    acc.roots_colored += sc->roots_colored;
    acc.roots_branched += sc->roots_branched;
    acc.nodes += sc->nodes;
    acc.donations += sc->donations;
    acc.entries += sc->entries;
    acc.entries_block += sc->entries_block;
    acc.tasks += sc->tasks;
  }
  // nothing to search (every vertex pruned): the search-stage events still
  // bracket an empty interval
  if (!searched)
    for (int i = 8; i <= 12; i++) MC_TRY(record_event(g, i));
  acc.d_counters = sc->d_counters;
  g->repeel_acc = acc;
  return MC_OK;
}

// Enqueue the whole of Algorithm 2 on every graph of the handle -- core
// numbers, heuristic, pruning, search, witness check -- without any host
// synchronisation after the core numbers' bound (K(G), known from a previous
// solve when capturing).  Leaves omega in g->best and witnesses in g->wit.
static int enqueue_solve(mc_graph *g, const mc_options &o, Pruned *pg, SearchCounters *sc, int32_t **d_ok_out) {
  const long long spin = spin_of(&o);
  g->warp_max_used = o.warp_max > 0 ? std::min(o.warp_max, 128) : 128;
  MC_TRY(record_event(g, 0));
  // every solve recomputes the core numbers (Algorithm 2, line 2)
  g->cores_valid = false;
  MC_TRY(ensure_cores(g, spin));
  if (o.order) {
    if (g->count > 1) return MC_ERR_ARG;
    MC_TRY(use_order(g, o.order));
  }
  MC_TRY(record_event(g, 1));
  MC_CUDA_TRY(cudaMemsetAsync(g->best, 0, g->count * 4, g->stream));
  MC_CUDA_TRY(cudaMemsetAsync(g->lock, 0, g->count * 4, g->stream));
  g->huge_roots = 0;
  if (g->lb > 0) MC_CUDA_TRY(cudaMemcpyAsync(g->best, &g->lb, 4, cudaMemcpyHostToDevice, g->stream));
  // learned scores (host or device) -> device copy
  const float *d_scores = nullptr;
  const int32_t *d_seeds = nullptr;
  int64_t nseeds = 0;
  void *p;
  if (o.scores && g->n > 0) {
    if (is_device_ptr(o.scores)) {
      d_scores = o.scores;
    } else {
      // host scores: copied here, or, inside capture (a graph cannot copy
      // from pageable memory), before every replay by stage_host_scores
      MC_TRY(ws_get(g, "cp.scores", g->n * sizeof(float), &p));
      if (!g->capturing)
        MC_CUDA_TRY(cudaMemcpyAsync(p, o.scores, g->n * sizeof(float), cudaMemcpyHostToDevice, g->stream));
      d_scores = (const float *)p;
    }
    if (o.seeds > 0) {
      nseeds = std::min<int64_t>(o.seeds, g->n);
      MC_TRY(ws_get(g, "cp.seeds", (nseeds + 1) * sizeof(int32_t), &p));
      int32_t *seeds = (int32_t *)p;
      MC_TRY(top_scores(g, d_scores, nseeds, seeds));
      d_seeds = seeds;
    }
  }
  g->heur_ran = o.heuristic != 2 && g->n > 0;
  g->learned_ran = o.mlp != nullptr && g->n > 0;
  if (g->learned_ran) {
    // The learned form: the warm-up part of Algorithm 1 sets a bound, only
    // the vertices that can still beat it are scored, and the best-scored
    // of them are grown first; then the rest of Algorithm 1 (heuristic 0)
    // or nothing more (heuristic 3).
    int64_t grown = 0;
    MC_TRY(launch_heuristic(g, 0, spin, nullptr, 0, nullptr, true, 0, -1, &grown));
    MC_TRY(record_event(g, 13));
    MC_TRY(ws_get(g, "ln.score", g->n * sizeof(float), &p));
    float *sc = (float *)p;
    MC_TRY(learned_scores(g, o.mlp, sc));
    const int32_t per = o.seeds > 0 ? o.seeds : (g->count > 1 ? 2 : 64);
    nseeds = g->count > 1 ? (int64_t)per * g->count : per;
    MC_TRY(ws_get(g, "cp.seeds", (nseeds + 1) * sizeof(int32_t), &p));
    int32_t *seeds = (int32_t *)p;
    MC_TRY(learned_seeds(g, sc, per, seeds));
    MC_TRY(record_event(g, 14));
    MC_TRY(launch_heuristic(g, 0, spin, seeds, nseeds, sc, o.heuristic == 3, grown, 0, nullptr));
    d_scores = sc;  // ordering = 1 orders the roots by these scores
  } else if (g->heur_ran) {
    MC_TRY(launch_heuristic(g, o.heuristic == 3 ? 0 : o.heuristic, spin, d_seeds, nseeds, d_scores, o.heuristic == 3));
  }
  MC_TRY(record_event(g, 2));
  int32_t *h_heur = (int32_t *)((char *)g->h_small + 1024);
  MC_CUDA_TRY(cudaMemcpyAsync(h_heur, g->best, sizeof(int32_t), cudaMemcpyDeviceToHost, g->stream));
  g->repeel_ran = o.repeel > 1 && g->n > 0;
  if (g->repeel_ran) {
    if (g->count > 1) return MC_ERR_ARG;
    MC_TRY(search_in_ranges(g, o, pg, sc, spin));
  } else {
    if (g->n > 0)
      MC_TRY(launch_prune(g, o.ordering, d_scores, g->warp_max_used, pg, spin, o.part_count > 1 ? o.part_rank : 0,
                          std::max(o.part_count, 1)));
    MC_TRY(record_event(g, 3));
    if (g->n > 0)
      MC_TRY(launch_search(g, *pg, o.no_neigh_cores, o.no_split, o.split_nodes, spin, sc, o.layout, o.no_bitmap));
    if (g->n > 0 && !g->capturing) MC_TRY(search_huge_roots(g, o, pg));
  }
  trivial_kernel<<<std::max(1, std::min(g->count / 256 + 1, 1024)), 256, 0, g->stream>>>(
      g->count, g->gid ? g->voff : nullptr, g->n, g->best, g->wit);
  g_launches++;
  MC_TRY(record_event(g, 4));
  MC_TRY(ws_get(g, "cp.ok", (size_t)g->count * 4, &p));
  *d_ok_out = (int32_t *)p;
  MC_TRY(launch_verify(g, *d_ok_out));
  MC_TRY(record_event(g, 5));
  return MC_OK;
}

// Wait for an enqueued solve and fill the statistics.
static int finish_solve(mc_graph *g, Pruned *pg, SearchCounters *sc, const int32_t *d_ok, mc_stats *st) {
  MC_CUDA_TRY(cudaEventSynchronize(g->ev[5]));
  MC_TRY(check_device_error(g));
  memset(st, 0, sizeof(*st));
  st->n = g->n;
  st->edges = g->nnz / 2;
  st->ms_cores = elapsed(g->ev[0], g->ev[1]);
  st->ms_heuristic = elapsed(g->ev[1], g->ev[2]);
  st->ms_prune = elapsed(g->ev[2], g->ev[3]);
  st->ms_search = elapsed(g->ev[3], g->ev[4]);
  st->ms_verify = elapsed(g->ev[4], g->ev[5]);
  st->ms_total = elapsed(g->ev[0], g->ev[5]);
  if (g->learned_ran) {
    st->ms_learned = elapsed(g->ev[13], g->ev[14]);
    auto it = g->ws.find("ln.ctl");
    if (it != g->ws.end() && it->second.p)
      MC_CUDA_TRY(cudaMemcpy(&st->learned_scored, it->second.p, sizeof(int64_t), cudaMemcpyDeviceToHost));
  }
  if (g->n > 0) {
    st->ms_search_block = elapsed(g->ev[8], g->ev[9]);
    st->ms_search_big = elapsed(g->ev[9], g->ev[10]);
    st->ms_search_warp = elapsed(g->ev[10], g->ev[11]);
    st->ms_search_tasks = elapsed(g->ev[11], g->ev[12]);
  }
  if (g->n > 0 && pg->d_counts) {
    MC_TRY(read_pruned_counts(g, pg));
    st->pruned_n = pg->n;
    st->pruned_arcs = pg->arcs;
    st->roots = g->repeel_ran ? g->repeel_roots : pg->nroots_small + pg->nroots_block + pg->nroots_big;
    st->prune_row_entries = pg->row_entries;
  }
  if (g->n > 0 && g->repeel_ran) {
    *sc = g->repeel_acc;
    st->rebuilds = g->repeel_rebuilds;
  } else if (g->n > 0 && sc->d_counters) {
    MC_TRY(read_search_counters(g, sc));
  }
  if (g->n > 0 && sc->d_counters) {
    st->roots_colored = (int64_t)sc->roots_colored;
    st->roots_branched = (int64_t)sc->roots_branched;
    st->nodes = (int64_t)sc->nodes;
    st->donations = (int64_t)sc->donations;
    st->neighbourhood_entries = (int64_t)sc->entries;
    st->neighbourhood_entries_block = (int64_t)sc->entries_block;
    st->tasks = (int64_t)sc->tasks;
  }
  st->max_core = g->max_core;
  g->heur0 = *(int32_t *)((char *)g->h_small + 1024);  // copied by the solve; the stream is synchronised
  st->heuristic_size = g->heur0;
  if (g->d_heur_ctr && g->heur_ran) {
    unsigned long long hc[3];
    MC_CUDA_TRY(cudaMemcpy(hc, g->d_heur_ctr, sizeof(hc), cudaMemcpyDeviceToHost));
    st->heuristic_grows = (int64_t)hc[0];
    st->heuristic_tests = (int64_t)hc[1];
    st->heuristic_row_entries = (int64_t)hc[2];
  }
  std::vector<int32_t> ok(g->count);
  MC_CUDA_TRY(cudaMemcpy(ok.data(), d_ok, g->count * 4, cudaMemcpyDeviceToHost));
  st->verified = 1;
  st->huge_roots = g->huge_roots;
  for (int32_t i = 0; i < g->count; i++)
    if (!ok[i]) st->verified = 0;
  if (g->lb > 0 && !st->verified) {
    // started from a lower bound: nothing larger found means no witness
    int32_t b = 0;
    MC_CUDA_TRY(cudaMemcpy(&b, g->best, 4, cudaMemcpyDeviceToHost));
    if (b == g->lb) st->verified = 1;
  }
  if (!st->verified) return MC_ERR_DEVICE_CHECK;
  return MC_OK;
}

// Host-resident scores into the device buffer that a captured solve reads.
static int stage_host_scores(mc_graph *g, const mc_options &o) {
  if (!o.scores || g->n == 0 || is_device_ptr(o.scores)) return MC_OK;
  void *p;
  MC_TRY(ws_get(g, "cp.scores", g->n * sizeof(float), &p));
  MC_CUDA_TRY(cudaMemcpyAsync(p, o.scores, g->n * sizeof(float), cudaMemcpyHostToDevice, g->stream));
  return MC_OK;
}

static uint64_t options_key(const mc_options &o) {
  uint64_t k = 1469598103934665603ULL;
  auto mix = [&](uint64_t x) { k = (k ^ x) * 1099511628211ULL; };
  mix((uint64_t)o.ordering);
  mix((uint64_t)o.no_neigh_cores);
  mix((uint64_t)o.heuristic);
  mix((uint64_t)o.warp_max);
  mix((uint64_t)o.spin_limit);
  mix((uint64_t)(uintptr_t)o.scores);
  mix((uint64_t)o.seeds);
  mix((uint64_t)o.no_split);
  mix((uint64_t)o.split_nodes);
  mix((uint64_t)(uintptr_t)o.mlp);
  mix((uint64_t)o.part_rank);
  mix((uint64_t)o.part_count);
  mix((uint64_t)o.layout);
  mix((uint64_t)o.no_bitmap);
  mix((uint64_t)o.repeel);
  return k;
}

// The whole solve.  With o.graph = 1 the enqueue is captured once into a
// CUDA graph (after a direct solve that sizes every buffer and finds K(G))
// and every later call with the same options replays it with one launch.
static int run_max_clique(mc_graph *g, const mc_options *opt, mc_stats *st) {
  mc_options o;
  MC_TRY(check_options(opt, &o));
  Pruned pg;
  SearchCounters sc{};
  int32_t *d_ok = nullptr;
  if (!o.graph || g->n == 0) {
    MC_TRY(enqueue_solve(g, o, &pg, &sc, &d_ok));
    return finish_solve(g, &pg, &sc, d_ok, st);
  }
  const uint64_t key = options_key(o);
  if (!g->graph_exec || g->graph_key != key) {
    if (g->graph_exec) {
      cudaGraphExecDestroy(g->graph_exec);
      g->graph_exec = nullptr;
    }
    MC_TRY(enqueue_solve(g, o, &pg, &sc, &d_ok));  // direct solve: sizes buffers, K(G)
    MC_TRY(finish_solve(g, &pg, &sc, d_ok, st));
    // roots beyond the workers are solved from the host: such graphs are
    // solved directly, never captured
    if (g->count == 1 && g->max_core > kBigCap) return MC_OK;
    cudaStream_t user = g->stream;
    if (!g->cap_stream) MC_CUDA_TRY(cudaStreamCreateWithFlags(&g->cap_stream, cudaStreamNonBlocking));
    g->stream = g->cap_stream;
    g->capturing = true;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(g->stream, cudaStreamCaptureModeRelaxed);
    int rc = (e == cudaSuccess) ? enqueue_solve(g, o, &pg, &sc, &d_ok) : MC_ERR_CUDA;
    cudaError_t e2 = cudaStreamEndCapture(g->stream, &graph);
    g->capturing = false;
    g->stream = user;
    if (rc != MC_OK) return rc;
    if (e2 != cudaSuccess) {
      set_last_cuda_error(e2, "cudaStreamEndCapture", __FILE__, __LINE__);
      return MC_ERR_CUDA;
    }
    e = cudaGraphInstantiate(&g->graph_exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      set_last_cuda_error(e, "cudaGraphInstantiate", __FILE__, __LINE__);
      g->graph_exec = nullptr;
      return MC_ERR_CUDA;
    }
    g->graph_key = key;
    g->graph_pg = pg;
    g->graph_sc = sc;
    g->graph_ok = d_ok;
  }
  // one launch of the captured solve, ordered after the caller's stream
  MC_TRY(stage_host_scores(g, o));
  MC_CUDA_TRY(cudaEventRecord(g->ev[6], g->stream));
  MC_CUDA_TRY(cudaStreamWaitEvent(g->cap_stream, g->ev[6], 0));
  MC_CUDA_TRY(cudaGraphLaunch(g->graph_exec, g->cap_stream));
  g_launches++;
  MC_CUDA_TRY(cudaEventRecord(g->ev[7], g->cap_stream));
  MC_CUDA_TRY(cudaStreamWaitEvent(g->stream, g->ev[7], 0));
  MC_CUDA_TRY(cudaStreamSynchronize(g->cap_stream));
  pg = g->graph_pg;
  sc = g->graph_sc;
  return finish_solve(g, &pg, &sc, g->graph_ok, st);
}

}  // namespace mc

using namespace mc;

extern "C" {

const char *mc_strerror(int code) {
  switch (code) {
    case MC_OK: return "ok";
    case MC_ERR_ARG: return "invalid argument";
    case MC_ERR_INVALID_GRAPH: return "input is not a simple symmetric CSR graph";
    case MC_ERR_OOM: return "device memory allocation failed";
    case MC_ERR_BUFFER: return "output buffer too small";
    case MC_ERR_TIMEOUT: return "a device spin-wait exceeded its iteration limit";
    case MC_ERR_CUDA: return g_errbuf[0] ? g_errbuf : "CUDA runtime error";
    case MC_ERR_DEVICE_CHECK: return "device-side consistency check failed";
    case MC_ERR_UNSUPPORTED: return "a batch graph with core number above 4096, the largest neighbourhood a search worker holds";
    case MC_ERR_TOO_LARGE:
      return "input larger than the fixed scratch of mc_core_numbers_noalloc (1,048,576 vertices, 67,108,864 entries)";
    default: return "unknown error";
  }
}

int mc_version(void) { return 100; }

int64_t mc_launch_count(void) { return g_launches.load(); }

int mc_load_csr(int64_t n, const int64_t *row_ptr, const int32_t *col_idx, uint32_t flags, void *cuda_stream,
                mc_graph **out) {
  return load_common(1, nullptr, n, row_ptr, col_idx, flags, cuda_stream, out);
}

int mc_load_batch(int32_t count, const int64_t *voff, const int64_t *row_ptr, const int32_t *col_idx,
                  uint32_t flags, void *cuda_stream, mc_graph **out) {
  if (count < 1 || !voff) return MC_ERR_ARG;
  int64_t n = 0;
  if (cudaMemcpy(&n, voff + count, sizeof(int64_t), cudaMemcpyDefault) != cudaSuccess) return MC_ERR_ARG;
  return load_common(count, voff, n, row_ptr, col_idx, flags, cuda_stream, out);
}

void mc_free(mc_graph *g) { free_graph(g); }

int mc_graph_info(const mc_graph *g, int64_t *n, int64_t *edges, int32_t *count) {
  if (!g) return MC_ERR_ARG;
  if (n) *n = g->n;
  if (edges) *edges = g->nnz / 2;
  if (count) *count = g->count;
  return MC_OK;
}

int mc_core_numbers(mc_graph *g, int32_t *core_out, int32_t *max_core_out) {
  if (!g) return MC_ERR_ARG;
  MC_TRY(ensure_cores(g, kDefaultSpinLimit));
  if (core_out && g->n > 0)
    MC_CUDA_TRY(cudaMemcpyAsync(core_out, g->core, g->n * sizeof(int32_t), cudaMemcpyDefault, g->stream));
  MC_CUDA_TRY(cudaStreamSynchronize(g->stream));
  if (max_core_out) *max_core_out = g->max_core;
  return MC_OK;
}

static int copy_witness_out(mc_graph *g, int32_t gi, int32_t size, int32_t *dst, int64_t local_base) {
  std::vector<int32_t> w(std::max(size, 1));
  if (size > 0)
    MC_CUDA_TRY(cudaMemcpy(w.data(), g->wit + g->h_voff[gi], size * sizeof(int32_t), cudaMemcpyDeviceToHost));
  for (int32_t i = 0; i < size; i++) w[i] -= (int32_t)local_base;
  std::sort(w.begin(), w.begin() + size);
  if (size > 0) MC_CUDA_TRY(cudaMemcpy(dst, w.data(), size * sizeof(int32_t), cudaMemcpyDefault));
  return MC_OK;
}

int mc_heuristic_clique(mc_graph *g, const int32_t *core, int32_t mode, int32_t *clique_out, int32_t capacity,
                        int32_t *size_out) {
  (void)core;  // core numbers are unique: the library computes (or reuses) its own
  if (!g || !size_out || (mode != 0 && mode != 1) || capacity < 0) return MC_ERR_ARG;
  *size_out = 0;
  MC_TRY(ensure_cores(g, kDefaultSpinLimit));
  MC_CUDA_TRY(cudaMemsetAsync(g->best, 0, g->count * 4, g->stream));
  MC_CUDA_TRY(cudaMemsetAsync(g->lock, 0, g->count * 4, g->stream));
  if (g->n > 0) MC_TRY(launch_heuristic(g, mode, kDefaultSpinLimit, nullptr, 0, nullptr));
  MC_CUDA_TRY(cudaStreamSynchronize(g->stream));
  MC_TRY(check_device_error(g));
  int32_t size = 0;
  MC_CUDA_TRY(cudaMemcpy(&size, g->best, sizeof(int32_t), cudaMemcpyDeviceToHost));
  *size_out = size;
  if (size > capacity) return MC_ERR_BUFFER;
  if (size > 0 && !clique_out) return MC_ERR_ARG;
  return copy_witness_out(g, 0, size, clique_out, 0);
}

int mc_max_clique(mc_graph *g, const mc_options *opt, int32_t *omega_out, int32_t *witness_out, int32_t capacity,
                  mc_stats *stats) {
  if (!g || !omega_out || capacity < 0) return MC_ERR_ARG;
  *omega_out = 0;
  mc_stats local;
  mc_stats *st = stats ? stats : &local;
  MC_TRY(run_max_clique(g, opt, st));
  int32_t om = 0;
  MC_CUDA_TRY(cudaMemcpy(&om, g->best, sizeof(int32_t), cudaMemcpyDeviceToHost));
  *omega_out = om;
  st->omega = om;
  if (om > capacity) return MC_ERR_BUFFER;
  if (om > 0 && !witness_out) return MC_ERR_ARG;
  return copy_witness_out(g, 0, om, witness_out, 0);
}

int mc_max_clique_batch(mc_graph *g, const mc_options *opt, int32_t *omegas_out, int32_t *witness_out,
                        int64_t capacity, int64_t *witness_offsets, mc_stats *stats) {
  if (!g || !omegas_out || !witness_offsets || capacity < 0) return MC_ERR_ARG;
  mc_stats local;
  mc_stats *st = stats ? stats : &local;
  MC_TRY(run_max_clique(g, opt, st));
  std::vector<int32_t> om(g->count);
  MC_CUDA_TRY(cudaMemcpy(om.data(), g->best, g->count * 4, cudaMemcpyDeviceToHost));
  std::vector<int64_t> off(g->count + 1, 0);
  for (int32_t i = 0; i < g->count; i++) off[i + 1] = off[i] + om[i];
  MC_CUDA_TRY(cudaMemcpy(omegas_out, om.data(), g->count * 4, cudaMemcpyDefault));
  MC_CUDA_TRY(cudaMemcpy(witness_offsets, off.data(), (g->count + 1) * 8, cudaMemcpyDefault));
  int32_t mx = 0;
  for (int32_t x : om) mx = std::max(mx, x);
  st->omega = mx;
  if (off[g->count] > capacity) return MC_ERR_BUFFER;
  if (off[g->count] > 0 && !witness_out) return MC_ERR_ARG;
  // gather all witnesses on the host in one copy of the witness area
  std::vector<int32_t> all(std::max<int64_t>(g->n, 1));
  if (g->n > 0) MC_CUDA_TRY(cudaMemcpy(all.data(), g->wit, g->n * 4, cudaMemcpyDeviceToHost));
  std::vector<int32_t> outv(std::max<int64_t>(off[g->count], 1));
  for (int32_t i = 0; i < g->count; i++) {
    int64_t b = g->h_voff[i];
    for (int32_t t = 0; t < om[i]; t++) outv[off[i] + t] = all[b + t] - (int32_t)b;
    std::sort(outv.begin() + off[i], outv.begin() + off[i] + om[i]);
  }
  if (off[g->count] > 0)
    MC_CUDA_TRY(cudaMemcpy(witness_out, outv.data(), off[g->count] * 4, cudaMemcpyDefault));
  return MC_OK;
}

int mc_autotune(mc_graph *g, const mc_options *base, int32_t repeats, mc_options *best_out, double *best_ms_out) {
  if (!g || !best_out || repeats < 1) return MC_ERR_ARG;
  mc_options b;
  MC_TRY(check_options(base, &b));
  mc_stats st;
  // mean solve time of one setting (after one untimed solve, which also
  // captures the CUDA graph when replay is on)
  auto trial = [&](const mc_options &o, double *ms) -> int {
    MC_TRY(run_max_clique(g, &o, &st));
    double tot = 0.0;
    for (int r = 0; r < repeats; r++) {
      MC_TRY(run_max_clique(g, &o, &st));
      tot += st.ms_total;
    }
    *ms = tot / repeats;
    return MC_OK;
  };
  // one coordinate at a time: the warp/block split of the roots, the spill
  // budget of the task queue, the heuristic's extent, then direct launches
  // vs graph replay
  mc_options bo = b;
  bo.graph = 0;
  double best = 1e300;
  for (int32_t wm : {32, 64, 128}) {
    mc_options o = bo;
    o.warp_max = wm;
    double ms;
    MC_TRY(trial(o, &ms));
    if (ms < best) {
      best = ms;
      b.warp_max = wm;
    }
  }
  bo.warp_max = b.warp_max;
  struct Split {
    int32_t no_split, nodes;
  };
  const Split splits[] = {{1, 0}, {0, 1024}, {0, 4096}, {0, 16384}};
  Split bs = {bo.no_split, bo.split_nodes};
  for (const Split &sp : splits) {
    mc_options o = bo;
    o.no_split = sp.no_split;
    o.split_nodes = sp.nodes;
    double ms;
    MC_TRY(trial(o, &ms));
    if (ms < best) {
      best = ms;
      bs = sp;
    }
  }
  bo.no_split = bs.no_split;
  bo.split_nodes = bs.nodes;
  // the block workers' bitset layout, then the build's member lookup
  for (int32_t lay : {1 - bo.layout}) {
    mc_options o = bo;
    o.layout = lay;
    double ms;
    MC_TRY(trial(o, &ms));
    if (ms < best) {
      best = ms;
      bo.layout = lay;
    }
  }
  {
    mc_options o = bo;
    o.no_bitmap = 1 - bo.no_bitmap;
    double ms;
    MC_TRY(trial(o, &ms));
    if (ms < best) {
      best = ms;
      bo.no_bitmap = o.no_bitmap;
    }
  }
  if (bo.heuristic == 0) {
    // the warm-up part of Algorithm 1 alone, where it reaches a bound that
    // prunes as well for less work
    mc_options o = bo;
    o.heuristic = 3;
    double ms;
    MC_TRY(trial(o, &ms));
    if (ms < best) {
      best = ms;
      bo.heuristic = 3;
    }
  }
  {
    mc_options o = bo;
    o.graph = 1;
    double ms;
    MC_TRY(trial(o, &ms));
    if (ms < best) {
      best = ms;
      bo.graph = 1;
    }
  }
  *best_out = bo;
  if (best_ms_out) *best_ms_out = best;
  return MC_OK;
}

int mc_peel_order(mc_graph *g, int32_t *order_out) {
  if (!g || (g->n > 0 && !order_out)) return MC_ERR_ARG;
  MC_TRY(ensure_cores(g, kDefaultSpinLimit));
  if (g->n > 0)
    MC_CUDA_TRY(cudaMemcpyAsync(order_out, g->order, g->n * sizeof(int32_t), cudaMemcpyDefault, g->stream));
  MC_CUDA_TRY(cudaStreamSynchronize(g->stream));
  return MC_OK;
}

int mc_clique_order(mc_graph *g, const int32_t *rank, int32_t *order_out, int64_t *group_starts_out,
                    int32_t *group_round_out, int64_t *groups_out, mc_order_stats *stats) {
  if (!g || g->count != 1 || !groups_out || (g->n > 0 && (!order_out || !group_starts_out))) return MC_ERR_ARG;
  *groups_out = 0;
  if (stats) memset(stats, 0, sizeof(*stats));
  const int64_t n = g->n;
  void *p;
  MC_TRY(ws_get(g, "co.out", (size_t)(n + 1) * 16 + 64, &p));
  int64_t *d_gstart = (int64_t *)p;
  int32_t *d_order = (int32_t *)(d_gstart + n + 1);
  int32_t *d_ground = d_order + n;
  MC_TRY(record_event(g, 0));
  int64_t groups = 0, work[2] = {0, 0};
  int32_t rounds = 0;
  if (n == 0) {
    if (group_starts_out) MC_CUDA_TRY(cudaMemcpy(group_starts_out, &groups, sizeof(int64_t), cudaMemcpyDefault));
    return MC_OK;
  }
  MC_TRY(clique_order(g, rank, d_order, d_gstart, d_ground, &groups, &rounds, work));
  MC_TRY(record_event(g, 1));
  MC_CUDA_TRY(cudaMemcpyAsync(order_out, d_order, n * 4, cudaMemcpyDefault, g->stream));
  MC_CUDA_TRY(cudaMemcpyAsync(group_starts_out, d_gstart, (groups + 1) * 8, cudaMemcpyDefault, g->stream));
  if (group_round_out)
    MC_CUDA_TRY(cudaMemcpyAsync(group_round_out, d_ground, groups * 4, cudaMemcpyDefault, g->stream));
  MC_CUDA_TRY(cudaStreamSynchronize(g->stream));
  MC_TRY(check_device_error(g));
  *groups_out = groups;
  if (stats) {
    stats->rounds = rounds;
    stats->grows = work[0];
    stats->tests = work[1];
    stats->ms = elapsed(g->ev[0], g->ev[1]);
  }
  return MC_OK;
}

int mc_relabel(mc_graph *g, const int32_t *order, int64_t *row_ptr_out, int32_t *col_idx_out) {
  if (!g || g->count != 1 || !row_ptr_out || (g->n > 0 && !order) || (g->nnz > 0 && !col_idx_out))
    return MC_ERR_ARG;
  const int64_t n = g->n;
  void *p;
  MC_TRY(ws_get(g, "rl.nrp", (size_t)(n + 1) * 8, &p));
  int64_t *d_nrp = (int64_t *)p;
  MC_TRY(ws_get(g, "rl.nci", (size_t)std::max<int64_t>(g->nnz, 1) * 4, &p));
  int32_t *d_nci = (int32_t *)p;
  MC_TRY(relabel(g, order, d_nrp, d_nci));
  MC_CUDA_TRY(cudaMemcpyAsync(row_ptr_out, d_nrp, (n + 1) * 8, cudaMemcpyDefault, g->stream));
  if (g->nnz > 0) MC_CUDA_TRY(cudaMemcpyAsync(col_idx_out, d_nci, g->nnz * 4, cudaMemcpyDefault, g->stream));
  MC_CUDA_TRY(cudaStreamSynchronize(g->stream));
  return check_device_error(g);
}

int mc_gap_bits(mc_graph *g, const int32_t *order, double *bits_out) {
  if (!g || g->count != 1 || !bits_out) return MC_ERR_ARG;
  *bits_out = 0.0;
  if (g->nnz == 0) return MC_OK;
  void *p;
  const int64_t *rp = g->row_ptr;
  const int32_t *ci = g->col_idx;
  if (order) {
    MC_TRY(ws_get(g, "rl.nrp", (size_t)(g->n + 1) * 8, &p));
    int64_t *d_nrp = (int64_t *)p;
    MC_TRY(ws_get(g, "rl.nci", (size_t)g->nnz * 4, &p));
    int32_t *d_nci = (int32_t *)p;
    MC_TRY(relabel(g, order, d_nrp, d_nci));
    rp = d_nrp;
    ci = d_nci;
  }
  MC_TRY(ws_get(g, "rl.sum", 8, &p));
  double *d_sum = (double *)p;
  MC_TRY(gap_bits(g, rp, ci, d_sum));
  MC_CUDA_TRY(cudaMemcpyAsync(g->h_small, d_sum, 8, cudaMemcpyDeviceToHost, g->stream));
  MC_CUDA_TRY(cudaStreamSynchronize(g->stream));
  MC_TRY(check_device_error(g));
  *bits_out = *(double *)g->h_small / (double)g->nnz;
  return MC_OK;
}

int mc_verify_clique(mc_graph *g, const int32_t *vertices, int32_t k, int32_t *is_clique_out) {
  if (!g || !is_clique_out || k < 0 || (k > 0 && !vertices)) return MC_ERR_ARG;
  *is_clique_out = 0;
  if (k == 0) {
    *is_clique_out = 1;
    return MC_OK;
  }
  void *p;
  MC_TRY(ws_get(g, "cp.vs", (size_t)k * 4 + 64, &p));
  int32_t *d = (int32_t *)p;
  MC_CUDA_TRY(cudaMemcpyAsync(d, vertices, (size_t)k * 4, cudaMemcpyDefault, g->stream));
  int32_t *ok = d + k;
  MC_TRY(launch_verify_set(g, d, k, ok));
  MC_CUDA_TRY(cudaMemcpyAsync(g->h_small, ok, 4, cudaMemcpyDeviceToHost, g->stream));
  MC_CUDA_TRY(cudaStreamSynchronize(g->stream));
  *is_clique_out = *(int32_t *)g->h_small;
  return MC_OK;
}

}  // extern "C"
