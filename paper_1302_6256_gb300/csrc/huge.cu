// Induced subgraphs for neighbourhoods beyond the workers' 4,096 candidates.
//
// A root u whose candidate set P (later neighbours kept by the pruning) holds
// more than 4,096 vertices is searched as a graph of its own: G[P] is built
// here as a CSR with sorted rows (local id = rank of the vertex id within
// P), solved by the whole pipeline with the incumbent as a lower bound, and
// a clique C of G[P] of size >= omega gives the clique {u} + C (Section 4.4:
// large neighbourhoods are searched without the adjacency matrix; here they
// are split once more by the same root rule instead).
#include <algorithm>

#include "mc_internal.cuh"
#include "scan.cuh"

namespace mc {

namespace {

// mark[verts[i]] = i (mark starts at -1 everywhere)
__global__ void mark_kernel(int32_t s, const int32_t *__restrict__ verts, int32_t *__restrict__ mark) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < s; i += (int64_t)gridDim.x * blockDim.x)
    mark[verts[i]] = (int32_t)i;
}
__global__ void unmark_kernel(int32_t s, const int32_t *__restrict__ verts, int32_t *__restrict__ mark) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < s; i += (int64_t)gridDim.x * blockDim.x)
    mark[verts[i]] = -1;
}

// a warp per member: how many of its neighbours are members
__global__ void sub_count_kernel(int32_t s, const int32_t *__restrict__ verts, const int64_t *__restrict__ rp,
                                 const int32_t *__restrict__ ci, const int32_t *__restrict__ mark,
                                 int64_t *__restrict__ cnt) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = gw; i < s; i += nw) {
    const int v = verts[i];
    int c = 0;
    for (int64_t e = rp[v] + lane; e < rp[v + 1]; e += 32) c += mark[ci[e]] >= 0 ? 1 : 0;
    c = dev::warp_sum(c);
    if (lane == 0) cnt[i] = c;
  }
}

// a warp per member: its member neighbours' local ids, in row order (members
// are ranked by vertex id, so the local ids come out sorted)
__global__ void sub_fill_kernel(int32_t s, const int32_t *__restrict__ verts, const int64_t *__restrict__ rp,
                                const int32_t *__restrict__ ci, const int32_t *__restrict__ mark,
                                const int64_t *__restrict__ srp, int32_t *__restrict__ sci) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = gw; i < s; i += nw) {
    const int v = verts[i];
    int64_t out = srp[i];
    for (int64_t eb = rp[v]; eb < rp[v + 1]; eb += 32) {
      const int64_t e = eb + lane;
      const int loc = e < rp[v + 1] ? mark[ci[e]] : -1;
      const unsigned m = __ballot_sync(0xffffffffu, loc >= 0);
      if (loc >= 0) sci[out + __popc(m & lt)] = loc;
      out += __popc(m);
    }
  }
}

// gather: out[i] = oold[ocol[row0 + i]] for the entries that are not padding
__global__ void gather_row_kernel(int64_t len, const int32_t *__restrict__ ocol, const int32_t *__restrict__ oold,
                                  int32_t *__restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x) {
    const int x = ocol[i];
    out[i] = x >= 0 ? oold[x] : -1;
  }
}

struct CntF {
  const int64_t *cnt;
  __device__ int64_t operator()(int64_t i) const { return cnt[i]; }
};
struct RowG {
  int64_t *srp;
  __device__ void operator()(int64_t i, int64_t excl, int64_t) const { srp[i] = excl; }
};

}  // namespace

int gather_root_row(mc_graph *g, const Pruned &pg, int32_t j, std::vector<int32_t> *out) {
  int64_t span[2];
  MC_CUDA_TRY(cudaMemcpyAsync(span, pg.orow + j, 2 * sizeof(int64_t), cudaMemcpyDeviceToHost, g->stream));
  MC_CUDA_TRY(cudaStreamSynchronize(g->stream));
  const int64_t len = span[1] - span[0];
  out->assign((size_t)std::max<int64_t>(len, 0), -1);
  if (len <= 0) return MC_OK;
  void *p;
  MC_TRY(ws_get(g, "hg.row", (size_t)len * 4, &p));
  int32_t *d = (int32_t *)p;
  gather_row_kernel<<<(int)std::min<int64_t>((len + 255) / 256, 1024), 256, 0, g->stream>>>(len, pg.ocol + span[0],
                                                                                          pg.oold, d);
  g_launches++;
  MC_CUDA_TRY(cudaGetLastError());
  MC_CUDA_TRY(cudaMemcpyAsync(out->data(), d, (size_t)len * 4, cudaMemcpyDeviceToHost, g->stream));
  MC_CUDA_TRY(cudaStreamSynchronize(g->stream));
  out->erase(std::remove(out->begin(), out->end(), -1), out->end());
  return MC_OK;
}

int induced_csr(mc_graph *g, const std::vector<int32_t> &verts, int64_t **d_rp, int32_t **d_ci, int64_t *nnz) {
  const int32_t s = (int32_t)verts.size();
  void *p;
  MC_TRY(ws_get(g, "hg.mark", (size_t)std::max<int64_t>(g->n, 1) * 4, &p));
  int32_t *mark = (int32_t *)p;
  if (!g->huge_mark_ready) {
    MC_CUDA_TRY(cudaMemsetAsync(mark, 0xff, (size_t)g->n * 4, g->stream));
    g->huge_mark_ready = true;
  }
  MC_TRY(ws_get(g, "hg.verts", (size_t)s * 4 + 16, &p));
  int32_t *dv = (int32_t *)p;
  MC_CUDA_TRY(cudaMemcpyAsync(dv, verts.data(), (size_t)s * 4, cudaMemcpyHostToDevice, g->stream));
  MC_TRY(ws_get(g, "hg.cnt", (size_t)s * 8 + 16, &p));
  int64_t *cnt = (int64_t *)p;
  MC_TRY(ws_get(g, "hg.rp", (size_t)(s + 1) * 8, &p));
  int64_t *srp = (int64_t *)p;
  const int tb = (int)std::min<int64_t>((s + 255) / 256, 1024);
  const int wb = (int)std::min<int64_t>(((int64_t)s * 32 + 255) / 256, (int64_t)g->sm_count * 8);
  mark_kernel<<<tb, 256, 0, g->stream>>>(s, dv, mark);
  sub_count_kernel<<<wb, 256, 0, g->stream>>>(s, dv, g->row_ptr, g->col_idx, mark, cnt);
  g_launches += 2;
  MC_CUDA_TRY(cudaGetLastError());
  MC_TRY(device_scan(g, s, CntF{cnt}, RowG{srp}, srp + s, "hg.scan"));
  MC_CUDA_TRY(cudaMemcpyAsync(nnz, srp + s, sizeof(int64_t), cudaMemcpyDeviceToHost, g->stream));
  MC_CUDA_TRY(cudaStreamSynchronize(g->stream));
  MC_TRY(ws_get(g, "hg.ci", (size_t)std::max<int64_t>(*nnz, 1) * 4, &p));
  int32_t *sci = (int32_t *)p;
  sub_fill_kernel<<<wb, 256, 0, g->stream>>>(s, dv, g->row_ptr, g->col_idx, mark, srp, sci);
  unmark_kernel<<<tb, 256, 0, g->stream>>>(s, dv, mark);
  g_launches += 2;
  MC_CUDA_TRY(cudaGetLastError());
  *d_rp = srp;
  *d_ci = sci;
  return MC_OK;
}

}  // namespace mc
