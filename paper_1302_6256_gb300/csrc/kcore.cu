// Core numbers by a bucketed parallel peel (Section 3: K(v) is the largest k
// such that v lies in the k-core; the peel removes, level by level, every
// vertex whose remaining degree is at most k).
//
// One cooperative persistent launch processes all levels:
//   scan    every vertex with remaining degree == k joins the level-k frontier
//           (warp-aggregated appends); if none does, k jumps to the smallest
//           remaining degree;
//   process a warp takes a frontier vertex, reads its row with coalesced
//           loads and decrements each neighbour whose degree is still above
//           k; a neighbour whose degree falls to k joins the frontier and is
//           processed by the same warp (warp-local chain in shared memory,
//           overflow to a global work list handled in a further sub-round).
// The append order is a degeneracy order: every vertex has at most K(v)
// neighbours appended after it.  It becomes the search's vertex ranking.
#include "mc_internal.cuh"

#include <algorithm>
#include <climits>

namespace mc {

namespace {

constexpr int kThreads = 512;
constexpr int kWarps = kThreads / 32;
constexpr int kLocalCap = 128;

struct KcoreCtl {
  unsigned bar_count, bar_gen;
  int otail;     // vertices appended to the peel order
  int ptail;     // vertices appended to the global work list
  int ctr[3];    // work-list grab counters, rotated per sub-round
  int minrem[3]; // smallest remaining degree, rotated per level scan
  int snap[2][2]; // (otail, ptail) captured by the last block into each barrier
};

// Grid barrier that also snapshots (otail, ptail) at the moment every block
// has arrived, so all blocks act on the same values even though fast blocks
// append again right after the barrier.  Bounded spin (error word on timeout).
__device__ __forceinline__ void barrier_snap(KcoreCtl *ctl, unsigned nblocks, int32_t *err, long long spin_limit,
                                             int *otail_out, int *ptail_out) {
  __shared__ int s_o, s_p;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned g0 = *(volatile unsigned *)&ctl->bar_gen;
    __threadfence();
    if (atomicAdd(&ctl->bar_count, 1u) == nblocks - 1) {
      __threadfence();
      ctl->snap[(g0 + 1) & 1][0] = *(volatile int *)&ctl->otail;
      ctl->snap[(g0 + 1) & 1][1] = *(volatile int *)&ctl->ptail;
      *(volatile unsigned *)&ctl->bar_count = 0;
      __threadfence();
      atomicAdd(&ctl->bar_gen, 1u);
    } else {
      long long it = 0;
      while (*(volatile unsigned *)&ctl->bar_gen == g0) {
        if (++it > spin_limit) { atomicExch(err, kDevTimeout); break; }
        __nanosleep(20);
      }
    }
    __threadfence();
    s_o = *(volatile int *)&ctl->snap[(g0 + 1) & 1][0];
    s_p = *(volatile int *)&ctl->snap[(g0 + 1) & 1][1];
  }
  __syncthreads();
  *otail_out = s_o;
  *ptail_out = s_p;
}

__global__ void degree_init_kernel(int64_t n, const int64_t *__restrict__ rp, int32_t *__restrict__ deg,
                                   int32_t *__restrict__ maxdeg) {
  int local = 0;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    int d = (int)(rp[v + 1] - rp[v]);
    deg[v] = d;
    local = max(local, d);
  }
  local = dev::warp_max(local);
  if ((threadIdx.x & 31) == 0) atomicMax(maxdeg, local);
}

__global__ void __launch_bounds__(kThreads) kcore_peel_kernel(int64_t n, const int64_t *__restrict__ rp,
                                                              const int32_t *__restrict__ ci, int32_t *deg,
                                                              int32_t *core, int32_t *order, int32_t *pend,
                                                              KcoreCtl *ctl, int32_t *err, long long spin_limit) {
  __shared__ int lstack[kWarps][kLocalCap];
  __shared__ int lcount[kWarps];
  __shared__ int bmin;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t gwarp = (int64_t)blockIdx.x * kWarps + wib;
  const int64_t nwarps = (int64_t)gridDim.x * kWarps;
  const unsigned nblocks = gridDim.x;
  const bool leader = blockIdx.x == 0 && threadIdx.x == 0;
  const unsigned lt_mask = (1u << lane) - 1u;

  int k = 0, phead = 0;
  unsigned level = 0, round = 0;
  if (lane == 0) lcount[wib] = 0;
  __syncwarp();
  int otail_now = 0, ptail_now = 0;

  for (;;) {
    // ---------------- scan: frontier of level k ----------------
    if (threadIdx.x == 0) bmin = INT_MAX;
    if (leader) ctl->minrem[(level + 1) % 3] = INT_MAX;
    __syncthreads();
    int lmin = INT_MAX;
    for (int64_t base = gwarp * 32; base < n; base += nwarps * 32) {
      int64_t v = base + lane;
      int d = (v < n) ? __ldcg(deg + v) : INT_MIN;
      bool hit = d == k;
      if (d > k) lmin = min(lmin, d);
      unsigned m = __ballot_sync(0xffffffffu, hit);
      if (m) {
        int cnt = __popc(m), ob = 0, pb = 0;
        if (lane == 0) { ob = atomicAdd(&ctl->otail, cnt); pb = atomicAdd(&ctl->ptail, cnt); }
        ob = __shfl_sync(0xffffffffu, ob, 0);
        pb = __shfl_sync(0xffffffffu, pb, 0);
        if (hit) {
          int r = __popc(m & lt_mask);
          core[v] = k;
          order[ob + r] = (int)v;
          pend[pb + r] = (int)v;
        }
      }
    }
    lmin = -dev::warp_max(-lmin);
    if (lane == 0 && lmin != INT_MAX) atomicMin(&bmin, lmin);
    __syncthreads();
    if (threadIdx.x == 0 && bmin != INT_MAX) atomicMin(&ctl->minrem[level % 3], bmin);
    barrier_snap(ctl, nblocks, err, spin_limit, &otail_now, &ptail_now);
    if (*(volatile int32_t *)err) return;

    if (ptail_now == phead) {
      // empty level: every remaining vertex has degree > k
      if (otail_now >= n) break;
      int mk = *(volatile int *)&ctl->minrem[level % 3];
      level++;
      if (mk == INT_MAX) break;  // unreachable: some vertex remains
      k = mk;
      continue;
    }
    level++;

    // ---------------- process sub-rounds ----------------
    while (phead < ptail_now) {
      if (leader) ctl->ctr[(round + 1) % 3] = 0;
      for (;;) {
        int cur;
        int lc = lcount[wib];
        if (lc > 0) {
          cur = lstack[wib][lc - 1];
          __syncwarp();
          if (lane == 0) lcount[wib] = lc - 1;
          __syncwarp();
        } else {
          int idx = 0;
          if (lane == 0) idx = phead + atomicAdd(&ctl->ctr[round % 3], 1);
          idx = __shfl_sync(0xffffffffu, idx, 0);
          if (idx >= ptail_now) break;
          cur = pend[idx];
        }
        const int64_t e0 = rp[cur], e1 = rp[cur + 1];
        for (int64_t eb = e0; eb < e1; eb += 32) {
          int64_t e = eb + lane;
          bool nf = false;
          int u = -1;
          if (e < e1) {
            u = ci[e];
            if (__ldcg(deg + u) > k) {
              int old = atomicSub(deg + u, 1);
              nf = (old == k + 1);
            }
          }
          unsigned m = __ballot_sync(0xffffffffu, nf);
          if (m) {
            int cnt = __popc(m), ob = 0;
            if (lane == 0) ob = atomicAdd(&ctl->otail, cnt);
            ob = __shfl_sync(0xffffffffu, ob, 0);
            int lc2 = lcount[wib];
            int room = kLocalCap - lc2;
            int take = min(room, cnt);
            int pb = 0;
            if (lane == 0 && cnt > take) pb = atomicAdd(&ctl->ptail, cnt - take);
            pb = __shfl_sync(0xffffffffu, pb, 0);
            if (nf) {
              int r = __popc(m & lt_mask);
              core[u] = k;
              order[ob + r] = u;
              if (r < take) lstack[wib][lc2 + r] = u;
              else pend[pb + (r - take)] = u;
            }
            __syncwarp();
            if (lane == 0) lcount[wib] = lc2 + take;
            __syncwarp();
          }
        }
      }
      int next_ptail;
      barrier_snap(ctl, nblocks, err, spin_limit, &otail_now, &next_ptail);
      if (*(volatile int32_t *)err) return;
      round++;
      phead = ptail_now;
      ptail_now = next_ptail;
    }
    if (otail_now >= n) break;
    k++;
  }
}

__global__ void peel_pos_kernel(int64_t n, const int32_t *__restrict__ order, int32_t *__restrict__ pos,
                                const int32_t *__restrict__ core, int32_t *__restrict__ maxcore) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int v = order[i];
    pos[v] = (int32_t)i;
    if (i == n - 1) *maxcore = core[v];  // the peel order is nondecreasing in K
  }
}

}  // namespace

int launch_core_numbers(mc_graph *g, long long spin_limit) {
  const int64_t n = g->n;
  if (n == 0) {
    g->max_core = 0;
    g->cores_valid = true;
    return MC_OK;
  }
  void *p;
  MC_TRY(ws_get(g, "kc.deg", n * sizeof(int32_t), &p));
  int32_t *deg = (int32_t *)p;
  MC_TRY(ws_get(g, "kc.pend", n * sizeof(int32_t), &p));
  int32_t *pend = (int32_t *)p;
  MC_TRY(ws_get(g, "kc.ctl", sizeof(KcoreCtl) + 64, &p));
  KcoreCtl *ctl = (KcoreCtl *)p;
  int32_t *maxdeg = (int32_t *)((char *)p + sizeof(KcoreCtl) + 16);
  MC_CUDA_TRY(cudaMemsetAsync(ctl, 0, sizeof(KcoreCtl) + 64, g->stream));

  int ib = (int)std::min<int64_t>((n + 255) / 256, (int64_t)g->sm_count * 8);
  degree_init_kernel<<<ib, 256, 0, g->stream>>>(n, g->row_ptr, deg, maxdeg);
  g_launches++;
  MC_CUDA_TRY(cudaGetLastError());

  int per_sm = 0;
  MC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kcore_peel_kernel, kThreads, 0));
  if (per_sm < 1) return MC_ERR_CUDA;
  int blocks = g->sm_count * std::min(per_sm, 2);
  int64_t need = (n + kThreads - 1) / kThreads;
  if (need < blocks) blocks = (int)std::max<int64_t>(1, need);
  int64_t n_arg = n;
  const int64_t *rp = g->row_ptr;
  const int32_t *ci = g->col_idx;
  int32_t *core = g->core, *order = g->order, *err = g->err;
  long long sl = spin_limit;
  void *args[] = {&n_arg, (void *)&rp, (void *)&ci, &deg, &core, &order, &pend, &ctl, &err, &sl};
  MC_CUDA_TRY(cudaLaunchCooperativeKernel((const void *)kcore_peel_kernel, dim3(blocks), dim3(kThreads), args, 0,
                                          g->stream));
  g_launches++;
  peel_pos_kernel<<<ib, 256, 0, g->stream>>>(n, g->order, g->pos, g->core, maxdeg + 1);
  g_launches++;
  MC_CUDA_TRY(cudaGetLastError());
  int32_t *host = (int32_t *)g->h_small;
  MC_CUDA_TRY(cudaMemcpyAsync(host, maxdeg, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, g->stream));
  MC_CUDA_TRY(cudaStreamSynchronize(g->stream));
  MC_TRY(check_device_error(g));
  g->max_degree = host[0];
  g->max_core = host[1];
  g->cores_valid = true;
  return MC_OK;
}

}  // namespace mc
