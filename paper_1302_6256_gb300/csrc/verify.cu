// Device checks: the witness of every graph is a clique (pairwise adjacent,
// distinct, inside its graph) and the input CSR is a simple symmetric graph.
#include <algorithm>

#include "mc_internal.cuh"

namespace mc {

namespace {

__device__ __forceinline__ bool adjacent(const int64_t *rp, const int32_t *ci, int x, int y) {
  int64_t lo = rp[x], hi = rp[x + 1];
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (ci[mid] < y) lo = mid + 1; else hi = mid;
  }
  return lo < rp[x + 1] && ci[lo] == y;
}

// one warp per graph: ok[g] = 1 iff wit[voff[g] .. + best[g]) is a clique
__global__ void verify_kernel(int32_t count, const int64_t *voff, int64_t n, const int64_t *rp, const int32_t *ci,
                              const int32_t *best, const int32_t *wit, int32_t *ok) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t g = gw; g < count; g += nw) {
    const int64_t v0 = voff ? voff[g] : 0, v1 = voff ? voff[g + 1] : n;
    const int k = best[g];
    const int32_t *w = wit + v0;
    bool good = k >= 0 && k <= v1 - v0;
    if (good) {
      const int64_t pairs = (int64_t)k * k;
      for (int64_t t = lane; t < pairs && good; t += 32) {
        int i = (int)(t / k), j = (int)(t % k);
        int x = w[i];
        if (x < v0 || x >= v1) good = false;
        else if (i < j && (x == w[j] || !adjacent(rp, ci, x, w[j]))) good = false;
      }
    }
    good = __all_sync(0xffffffffu, good);
    if (lane == 0) ok[g] = good ? 1 : 0;
  }
}

__global__ void verify_set_kernel(int64_t n, const int64_t *rp, const int32_t *ci, const int32_t *vs, int32_t k,
                                  int32_t *ok) {
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  const int64_t pairs = (int64_t)k * k;
  for (int64_t t = threadIdx.x; t < pairs; t += blockDim.x) {
    int i = (int)(t / k), j = (int)(t % k);
    int x = vs[i];
    if (x < 0 || x >= n) bad = 1;
    else if (i < j) {
      int y = vs[j];
      if (y < 0 || y >= n || x == y || !adjacent(rp, ci, x, y)) bad = 1;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) *ok = bad ? 0 : 1;
}

// warp per vertex: sorted strictly increasing rows, no self-loop, columns in
// range (and inside the vertex's graph for a batch), reverse edge present
__global__ void validate_kernel(int64_t n, int64_t nnz, const int64_t *rp, const int32_t *ci, const int32_t *gid,
                                const int64_t *voff, int32_t *bad) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  if (gw == 0 && lane == 0 && (rp[0] != 0 || rp[n] != nnz)) atomicExch(bad, 1);
  for (int64_t v = gw; v < n; v += nw) {
    const int64_t e0 = rp[v], e1 = rp[v + 1];
    if (e1 < e0 || e0 < 0 || e1 > nnz) {
      if (lane == 0) atomicExch(bad, 1);
      continue;
    }
    const int64_t lo = gid ? voff[gid[v]] : 0, hi = gid ? voff[gid[v] + 1] : n;
    bool ok = true;
    for (int64_t e = e0 + lane; e < e1; e += 32) {
      int u = ci[e];
      if (u < lo || u >= hi || u == v) ok = false;
      else if (e > e0 && ci[e - 1] >= u) ok = false;
      else {
        // row u is searched only inside [0, nnz): a broken row_ptr is
        // reported (by u's own warp) instead of read out of bounds
        const int64_t u0 = rp[u], u1 = rp[u + 1];
        if (u0 < 0 || u1 < u0 || u1 > nnz || !adjacent(rp, ci, u, (int)v)) ok = false;
      }
    }
    if (!__all_sync(0xffffffffu, ok) && lane == 0) atomicExch(bad, 1);
  }
}

__global__ void gid_kernel(int32_t count, const int64_t *voff, int32_t *gid) {
  for (int64_t g = blockIdx.x; g < count; g += gridDim.x)
    for (int64_t v = voff[g] + threadIdx.x; v < voff[g + 1]; v += blockDim.x) gid[v] = (int32_t)g;
}

// one graph: pairs spread over the grid; ok = 0 on any failure
__global__ void verify_one_kernel(int64_t n, const int64_t *rp, const int32_t *ci, const int32_t *best,
                                  const int32_t *wit, int32_t *ok) {
  const int k = best[0];
  if (k < 0 || k > n) {
    *ok = 0;
    return;
  }
  const int64_t pairs = (int64_t)k * k;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < pairs; t += (int64_t)gridDim.x * blockDim.x) {
    int i = (int)(t / k), j = (int)(t % k);
    int x = wit[i];
    bool good = x >= 0 && x < n;
    if (good && i < j) good = x != wit[j] && adjacent(rp, ci, x, wit[j]);
    if (!good) *ok = 0;
  }
}

__global__ void set_one_kernel(int32_t *p) { *p = 1; }

// A caller's vertex order: positions (a duplicate or out-of-range entry sets
// *bad), then every vertex's later neighbours counted against its core
// number (a degeneracy order has at most K(v) of them).
__global__ void order_pos_kernel(int64_t n, const int32_t *__restrict__ order, int32_t *__restrict__ ord,
                                 int32_t *__restrict__ pos, int32_t *bad) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = order[i];
    if (v < 0 || (int64_t)v >= n || atomicCAS(pos + v, -1, (int32_t)i) != -1) {
      atomicExch(bad, 1);
      continue;
    }
    ord[i] = v;
  }
}

__global__ void order_check_kernel(int64_t n, const int64_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                   const int32_t *__restrict__ pos, const int32_t *__restrict__ core, int32_t *bad) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t v = w0; v < n; v += nw) {
    const int pv = pos[v];
    int later = 0;
    for (int64_t e = rp[v] + lane; e < rp[v + 1]; e += 32) later += pos[ci[e]] > pv ? 1 : 0;
    later = dev::warp_sum(later);
    if (lane == 0 && later > core[v]) atomicExch(bad, 1);
  }
}

}  // namespace

int launch_verify(mc_graph *g, int32_t *d_ok) {
  if (g->count == 1) {
    set_one_kernel<<<1, 1, 0, g->stream>>>(d_ok);
    verify_one_kernel<<<g->sm_count * 4, 256, 0, g->stream>>>(g->n, g->row_ptr, g->col_idx, g->best, g->wit, d_ok);
    g_launches += 2;
    MC_CUDA_TRY(cudaGetLastError());
    return MC_OK;
  }
  const int blocks = (int)std::min<int64_t>((g->count + 7) / 8, (int64_t)g->sm_count * 8);
  verify_kernel<<<std::max(blocks, 1), 256, 0, g->stream>>>(g->count, g->gid ? g->voff : nullptr, g->n, g->row_ptr,
                                                            g->col_idx, g->best, g->wit, d_ok);
  g_launches++;
  MC_CUDA_TRY(cudaGetLastError());
  return MC_OK;
}

int launch_verify_set(mc_graph *g, const int32_t *d_vs, int32_t k, int32_t *d_ok) {
  verify_set_kernel<<<1, 512, 0, g->stream>>>(g->n, g->row_ptr, g->col_idx, d_vs, k, d_ok);
  g_launches++;
  MC_CUDA_TRY(cudaGetLastError());
  return MC_OK;
}

int launch_validate(mc_graph *g, int32_t *d_bad) {
  if (g->n == 0) return MC_OK;
  const int blocks = (int)std::min<int64_t>((g->n * 32 + 255) / 256, (int64_t)g->sm_count * 16);
  validate_kernel<<<blocks, 256, 0, g->stream>>>(g->n, g->nnz, g->row_ptr, g->col_idx, g->gid, g->voff, d_bad);
  g_launches++;
  MC_CUDA_TRY(cudaGetLastError());
  return MC_OK;
}

int use_order(mc_graph *g, const int32_t *order) {
  if (g->n == 0) return MC_OK;
  void *p;
  MC_TRY(ws_get(g, "ord.in", (size_t)g->n * 4 + 64, &p));
  int32_t *staged = (int32_t *)p, *bad = (int32_t *)((char *)p + (size_t)g->n * 4);
  MC_CUDA_TRY(cudaMemcpyAsync(staged, order, g->n * 4, cudaMemcpyDefault, g->stream));
  MC_CUDA_TRY(cudaMemsetAsync(bad, 0, 4, g->stream));
  MC_CUDA_TRY(cudaMemsetAsync(g->pos, 0xff, g->n * 4, g->stream));
  const int blocks = (int)std::min<int64_t>((g->n + 255) / 256, (int64_t)g->sm_count * 8);
  order_pos_kernel<<<blocks, 256, 0, g->stream>>>(g->n, staged, g->order, g->pos, bad);
  g_launches++;
  int32_t *h = (int32_t *)g->h_small;
  MC_CUDA_TRY(cudaMemcpyAsync(h, bad, 4, cudaMemcpyDeviceToHost, g->stream));
  MC_CUDA_TRY(cudaStreamSynchronize(g->stream));
  if (*h == 0) {
    const int wblocks = (int)std::min<int64_t>((g->n * 32 + 255) / 256, (int64_t)g->sm_count * 16);
    order_check_kernel<<<wblocks, 256, 0, g->stream>>>(g->n, g->row_ptr, g->col_idx, g->pos, g->core, bad);
    g_launches++;
    MC_CUDA_TRY(cudaMemcpyAsync(h, bad, 4, cudaMemcpyDeviceToHost, g->stream));
    MC_CUDA_TRY(cudaStreamSynchronize(g->stream));
  }
  if (*h) {
    g->cores_valid = false;  // the peel order was overwritten: recompute it next time
    return MC_ERR_ARG;
  }
  return MC_OK;
}

int launch_gid(mc_graph *g) {
  gid_kernel<<<std::min<int>(g->count, 65535), 256, 0, g->stream>>>(g->count, g->voff, g->gid);
  g_launches++;
  MC_CUDA_TRY(cudaGetLastError());
  return MC_OK;
}

}  // namespace mc
