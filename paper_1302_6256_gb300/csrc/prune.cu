// Initial pruning and the oriented search graph (Section 4.2; Algorithm 2,
// line 4: vertices with K(v) < |H| are removed explicitly).
//
// The kept vertices are renumbered in peel (degeneracy) order, and each keeps
// only the neighbours that come later in that order.  A root u of the search
// then sees exactly the candidates a sequential run of Algorithm 2 would see
// when it reaches u: the neighbours not yet searched (the set X of Section 4.3
// is "every vertex earlier in the order").  Every clique is searched once,
// from its earliest member, and a vertex has at most K(v) later neighbours.
// Rows start at multiples of 4 entries so the search reads them with int4
// loads (pad entries are -1).

#include "mc_internal.cuh"
#include "scan.cuh"

namespace mc {

__global__ void scan_blocks_kernel(int64_t nb, int64_t *bsum) {
  __shared__ int64_t wsum[32];
  __shared__ int64_t carry;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < nb; base += blockDim.x) {
    int64_t i = base + threadIdx.x;
    int64_t x = (i < nb) ? bsum[i] : 0;
    int64_t incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int64_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[wid] = incl;
    __syncthreads();
    if (threadIdx.x == 0) {
      int64_t t = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
        int64_t s = wsum[w];
        wsum[w] = t;
        t += s;
      }
    }
    __syncthreads();
    int64_t excl = carry + wsum[wid] + incl - x;
    if (i < nb) bsum[i] = excl;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = excl + x;
    __syncthreads();
  }
  if (threadIdx.x == 0) bsum[nb] = carry;
}

namespace {

struct KeepF {
  const int32_t *order, *core, *gid, *best;
  __device__ int64_t operator()(int64_t i) const {
    int v = order[i];
    int g = gid ? gid[v] : 0;
    return core[v] >= best[g] ? 1 : 0;
  }
};
struct KeepG {
  const int32_t *order, *core, *gid;
  int32_t *nid, *oold, *ocore, *ogid;
  __device__ void operator()(int64_t i, int64_t excl, int64_t val) const {
    int v = order[i];
    if (val) {
      nid[v] = (int32_t)excl;
      oold[excl] = v;
      ocore[excl] = core[v];
      if (ogid) ogid[excl] = gid[v];
    } else {
      nid[v] = -1;
    }
  }
};

// Rows of the kept vertices in chunks of kRowChunk entries, so that a hub's
// row (163,305 entries at R-MAT scale 22) is split over many warps instead
// of holding one warp while the rest of the grid idles.
constexpr int kRowChunk = 1024;

struct ChunkF {  // chunks of kept row j
  const int64_t *rp, *np;
  const int32_t *oold;
  __device__ int64_t operator()(int64_t j) const {
    if (j >= *np) return 0;
    const int v = oold[j];
    return (rp[v + 1] - rp[v] + kRowChunk - 1) / kRowChunk;
  }
};
struct ChunkG {  // row offsets in chunk space, and each chunk's row
  int64_t *coff;
  int32_t *crow;
  __device__ void operator()(int64_t j, int64_t excl, int64_t val) const {
    coff[j] = excl;
    for (int64_t c = excl; c < excl + val; c++) crow[c] = (int32_t)j;
  }
};
struct CntF {  // kept entries of chunk c
  const int32_t *ccnt;
  __device__ int64_t operator()(int64_t c) const { return ccnt[c]; }
};
struct PosG {
  int64_t *cpos;
  __device__ void operator()(int64_t c, int64_t excl, int64_t) const { cpos[c] = excl; }
};

// kept entries (later neighbours) per chunk, summed into the row's
// out-degree; one warp per chunk
__global__ void outdeg_chunk_kernel(const int64_t *__restrict__ d_np, const int64_t *__restrict__ coff,
                                    const int32_t *__restrict__ crow, const int64_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                    const int32_t *__restrict__ oold, const int32_t *__restrict__ nid,
                                    int32_t *__restrict__ ccnt, int32_t *__restrict__ odeg,
                                    unsigned long long *__restrict__ scanned) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t np = *d_np, nch = coff[np];
  unsigned long long rows = 0;
  for (int64_t c = w0; c < nch; c += nw) {
    const int64_t j = crow[c];
    const int v = oold[j];
    const int64_t e0 = rp[v] + (c - coff[j]) * kRowChunk, e1 = min(rp[v + 1], e0 + kRowChunk);
    int k = 0;
    for (int64_t e = e0 + lane; e < e1; e += 32) k += (nid[ci[e]] > (int32_t)j) ? 1 : 0;
    k = dev::warp_sum(k);
    if (lane == 0) {
      ccnt[c] = k;
      if (k) atomicAdd(odeg + j, k);
    }
    rows += (unsigned long long)(e1 - e0);
  }
  if (lane == 0 && rows) atomicAdd(scanned, rows);
}

__global__ void maxout_kernel(const int64_t *__restrict__ d_np, const int32_t *__restrict__ odeg,
                              int32_t *__restrict__ maxout) {
  int m = 0;
  const int64_t np = *d_np;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < np; j += (int64_t)gridDim.x * blockDim.x)
    m = max(m, odeg[j]);
  m = dev::warp_max(m);
  if ((threadIdx.x & 31) == 0 && m) atomicMax(maxout, m);
}

struct PadF {
  const int32_t *odeg;
  const int64_t *np;
  __device__ int64_t operator()(int64_t j) const { return j < *np ? (int64_t)((odeg[j] + 3) & ~3) : 0; }
};
struct RowG {
  int64_t *orow;
  __device__ void operator()(int64_t j, int64_t excl, int64_t) const { orow[j] = excl; }
};

// the oriented rows, one warp per chunk: a chunk's kept entries go after
// those of the row's earlier chunks (row order kept), and the row's last
// chunk writes its padding
__global__ void fill_chunk_kernel(const int64_t *__restrict__ d_np, const int64_t *__restrict__ coff,
                                  const int32_t *__restrict__ crow, const int64_t *__restrict__ cpos,
                                  const int64_t *__restrict__ rp,
                                  const int32_t *__restrict__ ci, const int32_t *__restrict__ oold,
                                  const int32_t *__restrict__ nid, const int64_t *__restrict__ orow,
                                  const int32_t *__restrict__ odeg, int32_t *__restrict__ ocol) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t np = *d_np, nch = coff[np];
  for (int64_t c = w0; c < nch; c += nw) {
    const int64_t j = crow[c];
    const int v = oold[j];
    const int64_t e0 = rp[v] + (c - coff[j]) * kRowChunk, e1 = min(rp[v + 1], e0 + kRowChunk);
    int64_t out = orow[j] + (cpos[c] - cpos[coff[j]]);
    for (int64_t eb = e0; eb < e1; eb += 32) {
      const int64_t e = eb + lane;
      const int y = (e < e1) ? nid[ci[e]] : -1;
      const bool k = y > (int32_t)j;
      const unsigned m = __ballot_sync(0xffffffffu, k);
      if (k) ocol[out + __popc(m & lt)] = y;
      out += __popc(m);
    }
    if (c == coff[j + 1] - 1) {
      const int padded = (odeg[j] + 3) & ~3;
      for (int t = odeg[j] + lane; t < padded; t += 32) ocol[orow[j] + t] = -1;
    }
  }
}

// root flags and classes
struct RootInfo {
  const int32_t *odeg, *ogid, *best;
  int32_t warp_max;
  const int32_t *oold, *pos;  // position of a pruned vertex in the peel order
  int32_t part_rank, part_count;  // root partition over ranks
  int64_t pos_lo, pos_hi;         // roots at peel positions [pos_lo, pos_hi) only
  __device__ int cls(int64_t j) const {
    if (j < 0) return -1;
    const int64_t pp = pos[oold[j]];
    if (pp < pos_lo || pp >= pos_hi) return -1;                    // outside this range of roots
    if (part_count > 1 && pp % part_count != part_rank) return -1;  // another part's root
    int g = ogid ? ogid[j] : 0;
    int d = odeg[j];
    if (d < best[g] || d == 0) return -1;  // |P| >= omega~ is needed for a larger clique
    return d <= warp_max ? 0 : (d <= 1024 ? 1 : (d <= kBigCap ? 2 : 3));
  }
};

// index space t -> pruned vertex j for the root order
struct PermDesc {  // ordering 0: decreasing rank (dense core first)
  const int64_t *np;
  __device__ int64_t operator()(int64_t t) const { return t < *np ? *np - 1 - t : -1; }
};
struct PermTable {  // ordering 1/2: explicit table of np entries
  const int32_t *tab;
  const int64_t *np;
  __device__ int64_t operator()(int64_t t) const { return t < *np ? tab[t] : -1; }
};

template <class Perm>
struct ClassF {
  RootInfo ri;
  Perm perm;
  int c;
  __device__ int64_t operator()(int64_t t) const { return ri.cls(perm(t)) == c ? 1 : 0; }
};
template <class Perm>
struct ClassG {
  Perm perm;
  int32_t *out;
  __device__ void operator()(int64_t t, int64_t excl, int64_t val) const {
    if (val) out[excl] = (int32_t)perm(t);
  }
};

// native order: kept vertices by increasing original id
struct NativeF {
  const int32_t *nid;
  __device__ int64_t operator()(int64_t v) const { return nid[v] >= 0 ? 1 : 0; }
};
struct NativeG {
  const int32_t *nid;
  int32_t *tab;
  __device__ void operator()(int64_t v, int64_t excl, int64_t val) const {
    if (val) tab[excl] = nid[v];
  }
};

// Sort keys of the pruned vertices: each score's bits mapped to an unsigned
// integer of the same order (positives: sign bit set; negatives: all bits
// flipped), then raised to at least 1, so that every score -- -inf and NaN
// included -- sorts before the slots past the pruned count, which get 0.
__global__ void gather_scores_kernel(int64_t n, const int64_t *__restrict__ d_np, const int32_t *__restrict__ oold,
                                     const float *__restrict__ score, uint32_t *__restrict__ key,
                                     int32_t *__restrict__ idx) {
  const int64_t np = *d_np;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    uint32_t k = 0u;
    if (j < np) {
      const uint32_t b = __float_as_uint(score[oold[j]]);
      k = max((b & 0x80000000u) ? ~b : (b | 0x80000000u), 1u);
    }
    key[j] = k;
    idx[j] = (int32_t)j;
  }
}

}  // namespace

int launch_prune(mc_graph *g, int ordering, const float *scores, int32_t warp_max, Pruned *out,
                 long long spin_limit, int32_t part_rank, int32_t part_count, int64_t pos_lo, int64_t pos_hi) {
  (void)spin_limit;
  // Everything stays on the device: the pruned size, arc count and root
  // counts are written to out->d_counts and read by the later kernels, and
  // every buffer is sized for the worst case, so this step needs no host
  // synchronisation (and can be captured into a CUDA graph).
  const int64_t n = g->n;
  void *p;
  MC_TRY(ws_get(g, "pr.nid", (n + 1) * sizeof(int32_t), &p));
  int32_t *nid = (int32_t *)p;
  MC_TRY(ws_get(g, "pr.oold", (n + 1) * sizeof(int32_t), &p));
  int32_t *oold = (int32_t *)p;
  MC_TRY(ws_get(g, "pr.ocore", (n + 1) * sizeof(int32_t), &p));
  int32_t *ocore = (int32_t *)p;
  int32_t *ogid = nullptr;
  if (g->gid) {
    MC_TRY(ws_get(g, "pr.ogid", (n + 1) * sizeof(int32_t), &p));
    ogid = (int32_t *)p;
  }
  MC_TRY(ws_get(g, "pr.small", 16 * sizeof(int64_t), &p));
  int64_t *dsm = (int64_t *)p;  // [0] n', [1] arcs, [2] maxout (int32 in low), [3..5] class counts,
                                // [6] row entries of the kept vertices
  MC_CUDA_TRY(cudaMemsetAsync(dsm, 0, 16 * sizeof(int64_t), g->stream));
  out->d_counts = dsm;
  out->n = n;  // upper bound until read back
  out->oold = oold;
  out->ocore = ocore;
  out->ogid = ogid;
  if (n == 0) return MC_OK;

  KeepF kf{g->order, g->core, g->gid, g->best};
  KeepG kg{g->order, g->core, g->gid, nid, oold, ocore, ogid};
  MC_TRY(device_scan(g, n, kf, kg, dsm + 0, "pr.scan"));

  MC_TRY(ws_get(g, "pr.odeg", (n + 1) * sizeof(int32_t), &p));
  int32_t *odeg = (int32_t *)p;
  int32_t *maxout = (int32_t *)(dsm + 2);
  const int blocks = (int)std::min<int64_t>((n * 32 + 255) / 256, (int64_t)g->sm_count * 16);
  // chunks of the kept rows: offsets per row (coff[n'] = their count), kept
  // entries per chunk, out-degrees as sums of those
  const int64_t ncap = n + g->nnz / kRowChunk + 2;  // at least the chunk count
  MC_TRY(ws_get(g, "pr.coff", (n + 1) * sizeof(int64_t), &p));
  int64_t *coff = (int64_t *)p;
  MC_TRY(ws_get(g, "pr.ccnt", ncap * sizeof(int32_t), &p));
  int32_t *ccnt = (int32_t *)p;
  MC_TRY(ws_get(g, "pr.crow", ncap * sizeof(int32_t), &p));
  int32_t *crow = (int32_t *)p;
  MC_TRY(ws_get(g, "pr.cpos", ncap * sizeof(int64_t), &p));
  int64_t *cpos = (int64_t *)p;
  MC_CUDA_TRY(cudaMemsetAsync(odeg, 0, (n + 1) * sizeof(int32_t), g->stream));
  MC_CUDA_TRY(cudaMemsetAsync(ccnt, 0, ncap * sizeof(int32_t), g->stream));
  MC_TRY(device_scan(g, n + 1, ChunkF{g->row_ptr, dsm + 0, oold}, ChunkG{coff, crow}, nullptr, "pr.scan"));
  const int cblocks = (int)std::min<int64_t>((ncap * 32 + 255) / 256, (int64_t)g->sm_count * 16);
  outdeg_chunk_kernel<<<cblocks, 256, 0, g->stream>>>(dsm + 0, coff, crow, g->row_ptr, g->col_idx, oold, nid, ccnt, odeg,
                                                      (unsigned long long *)(dsm + 6));
  maxout_kernel<<<(int)std::min<int64_t>((n + 255) / 256, (int64_t)g->sm_count * 4), 256, 0, g->stream>>>(dsm + 0,
                                                                                                     odeg, maxout);
  g_launches += 2;
  MC_CUDA_TRY(cudaGetLastError());
  MC_TRY(device_scan(g, ncap, CntF{ccnt}, PosG{cpos}, nullptr, "pr.scan"));
  MC_TRY(ws_get(g, "pr.orow", (n + 1) * sizeof(int64_t), &p));
  int64_t *orow = (int64_t *)p;
  // n + 1 entries: rows past n' (and the end offset orow[n]) get the total,
  // so orow[n'] is the arc count even when nothing was pruned (n' = n)
  MC_TRY(device_scan(g, n + 1, PadF{odeg, dsm + 0}, RowG{orow}, dsm + 1, "pr.scan"));
  // worst case: every edge kept once plus row padding
  const size_t arcs_cap = (size_t)(g->nnz / 2 + 4 * n + 4);
  MC_TRY(ws_get(g, "pr.ocol", arcs_cap * sizeof(int32_t), &p));
  int32_t *ocol = (int32_t *)p;
  fill_chunk_kernel<<<cblocks, 256, 0, g->stream>>>(dsm + 0, coff, crow, cpos, g->row_ptr, g->col_idx, oold, nid,
                                                    orow, odeg, ocol);
  g_launches++;
  MC_CUDA_TRY(cudaGetLastError());

  // roots in processing order, split by class
  MC_TRY(ws_get(g, "pr.roots", (4 * n + 4) * sizeof(int32_t), &p));
  int32_t *roots = (int32_t *)p;
  RootInfo ri{odeg, ogid, g->best, warp_max, oold, g->pos, part_rank, part_count, pos_lo, pos_hi};
  int32_t *tab = nullptr;
  if (ordering == 1 || ordering == 2) {
    MC_TRY(ws_get(g, "pr.tab", (n + 1) * sizeof(int32_t), &p));
    tab = (int32_t *)p;
  }
  if (ordering == 2) {
    MC_TRY(device_scan(g, n, NativeF{nid}, NativeG{nid, tab}, nullptr, "pr.scan"));
  } else if (ordering == 1) {
    if (!scores) return MC_ERR_ARG;
    MC_TRY(ws_get(g, "pr.skey", (2 * n + 2) * sizeof(uint32_t), &p));
    uint32_t *skey = (uint32_t *)p;
    MC_TRY(ws_get(g, "pr.sidx", (n + 1) * sizeof(int32_t), &p));
    int32_t *sidx = (int32_t *)p;
    gather_scores_kernel<<<blocks, 256, 0, g->stream>>>(n, dsm + 0, oold, scores, skey, sidx);
    g_launches++;
    MC_CUDA_TRY(cudaGetLastError());
    // stable: equal scores keep increasing pruned id; tab = the sorted ids
    MC_TRY(radix_sort_desc(g, skey, sidx, skey + n + 1, tab, n));
    MC_CUDA_TRY(cudaMemcpyAsync(tab, sidx, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, g->stream));
  }
  const int ncls = (g->count == 1 && g->max_core > kBigCap) ? 4 : 3;
  for (int c = 0; c < ncls; c++) {
    int32_t *dst = roots + (int64_t)c * n;
    int64_t *cnt = dsm + (c < 3 ? 3 + c : 7);
    if (ordering == 0) {
      MC_TRY(device_scan(g, n, ClassF<PermDesc>{ri, PermDesc{dsm + 0}, c},
                         ClassG<PermDesc>{PermDesc{dsm + 0}, dst}, cnt, "pr.scan"));
    } else {
      MC_TRY(device_scan(g, n, ClassF<PermTable>{ri, PermTable{tab, dsm + 0}, c},
                         ClassG<PermTable>{PermTable{tab, dsm + 0}, dst}, cnt, "pr.scan"));
    }
  }
  out->orow = orow;
  out->ocol = ocol;
  out->roots = roots;
  out->roots_small = roots;
  out->roots_block = roots + n;
  out->roots_big = roots + 2 * n;
  out->roots_huge = roots + 3 * n;
  out->odeg = odeg;
  return MC_OK;
}

// New root lists (degeneracy order, by class) over the pruned graph that
// `pg` already holds, for the roots at peel positions [pos_lo, pos_hi).
int relaunch_roots(mc_graph *g, int32_t warp_max, Pruned *pg, int32_t part_rank, int32_t part_count, int64_t pos_lo,
                   int64_t pos_hi) {
  const int64_t n = g->n;
  if (n == 0) return MC_OK;
  int64_t *dsm = pg->d_counts;
  RootInfo ri{pg->odeg, pg->ogid, g->best, warp_max, pg->oold, g->pos, part_rank, part_count, pos_lo, pos_hi};
  const int ncls = (g->count == 1 && g->max_core > kBigCap) ? 4 : 3;
  for (int c = 0; c < ncls; c++) {
    int32_t *dst = pg->roots + (int64_t)c * n;
    MC_TRY(device_scan(g, n, ClassF<PermDesc>{ri, PermDesc{dsm + 0}, c}, ClassG<PermDesc>{PermDesc{dsm + 0}, dst},
                       dsm + (c < 3 ? 3 + c : 7), "pr.scan"));
  }
  return MC_OK;
}

// Host copy of the pruned graph's sizes (one small device-to-host read).
int read_pruned_counts(mc_graph *g, Pruned *out) {
  int64_t *h = (int64_t *)g->h_small;
  MC_CUDA_TRY(cudaMemcpyAsync(h, out->d_counts, 8 * sizeof(int64_t), cudaMemcpyDeviceToHost, g->stream));
  MC_CUDA_TRY(cudaStreamSynchronize(g->stream));
  out->n = h[0];
  out->arcs = h[1];
  out->max_out = (int32_t)(h[2] & 0xffffffff);
  out->nroots_small = h[3];
  out->nroots_block = h[4];
  out->nroots_big = h[5];
  out->row_entries = h[6];
  out->nroots_huge = h[7];
  return MC_OK;
}

namespace {
// sort keys of the scores (the order of the float values, as in
// gather_scores_kernel) and their indices
__global__ void iota_kernel(int64_t n, const float *__restrict__ s, uint32_t *__restrict__ key,
                            int32_t *__restrict__ idx) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t b = __float_as_uint(s[i]);
    key[i] = (b & 0x80000000u) ? ~b : (b | 0x80000000u);
    idx[i] = (int32_t)i;
  }
}
}  // namespace

int top_scores(mc_graph *g, const float *scores, int64_t k, int32_t *out) {
  const int64_t n = g->n;
  void *p;
  MC_TRY(ws_get(g, "ts.key", (2 * n + 2) * sizeof(uint32_t), &p));
  uint32_t *key = (uint32_t *)p;
  MC_TRY(ws_get(g, "ts.idx", (2 * n + 2) * sizeof(int32_t), &p));
  int32_t *idx = (int32_t *)p;
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, (int64_t)g->sm_count * 8);
  iota_kernel<<<blocks, 256, 0, g->stream>>>(n, scores, key, idx);
  g_launches++;
  MC_CUDA_TRY(cudaGetLastError());
  MC_TRY(radix_sort_desc(g, key, idx, key + n + 1, idx + n + 1, n));
  MC_CUDA_TRY(cudaMemcpyAsync(out, idx, k * sizeof(int32_t), cudaMemcpyDeviceToDevice, g->stream));
  return MC_OK;
}

}  // namespace mc
