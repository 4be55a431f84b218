// Core numbers by a bucketed parallel peel (Section 3: K(v) is the largest k
// such that v lies in the k-core; the peel removes, level by level, every
// vertex whose remaining degree is at most k).
//
// One cooperative persistent launch processes all levels:
//   scan    every live vertex with remaining degree == k joins the level-k
//           frontier; vertices of larger degree are compacted into the next
//           live list, so later scans only touch what is left; if nothing
//           joins, k jumps to the smallest remaining degree.  A warp reads
//           kScanSlices slices of 32 live entries at once (one atomic for
//           their place in the next list).  Up to kScanLocalLive live
//           vertices, each block peels the frontier its warps found right
//           after its scan, from lists in shared memory that all its warps
//           share: rows of at most 32 edges one lane each, the 128-edge
//           chunks of rows of up to kLocalRow edges one warp each, the
//           cascade they start as further generations of the same lists, up
//           to kBlockDrainEdges edges; everything else becomes work items,
//           one per 128-edge chunk;
//   process after a grid barrier, the work items appended so far are split
//           statically over all warps (rows under 32 edges one lane per
//           item, longer chunks one warp per item, coalesced); every
//           neighbour whose degree is still above k is decremented, and one
//           whose degree falls to k joins the frontier: onto its block's
//           lists (walked by that block in the same phase) or as items of the
//           next sub-round, until a sub-round appends nothing.
// In the scan phase a vertex joins by claiming its core number
// (compare-and-swap from -1), so one that a scan reads at degree k just after
// a decrement made it k joins once; where decrements skip the read of the
// degree (degree arrays that fit in L2), a decrement from k also claims, for a
// vertex still at k that the scan has not reached.  In the sub-rounds only the
// decrement that takes a degree from k + 1 to k finds a vertex, and a plain
// store does.  The
// append order is a degeneracy order: when a vertex joins, every neighbour
// that joins later is still counted in its remaining degree, which is at most
// k.  It becomes the search's vertex ranking.
#include "mc_internal.cuh"

#include <algorithm>
#include <climits>
#include <mutex>

namespace mc {

namespace {

constexpr int kThreads = 1024;
constexpr int kWarps = kThreads / 32;
constexpr int kChunk = 128;  // edges per work item
constexpr int kPer = 4;      // edges per lane in flight
constexpr int kLocalRow = 4096;  // rows of at most this many edges may go onto the block lists
constexpr int kPoolShort = 4096;  // block list of rows of 1..32 edges (one lane per row)
constexpr int kPoolLong = 2048;   // block list of 128-edge chunks of rows of 33..kLocalRow edges (a warp each)
constexpr long long kBlockDrainEdges = 65536;  // edges a block walks from its lists per phase (then it spills)
constexpr int64_t kScanLocalLive = (int64_t)1 << 21;  // live vertices up to which the scan peels locally
constexpr int kScanSlices = 8;  // slices of 32 live entries a warp's scan reads at once
constexpr int64_t kNoCheckMaxN = (int64_t)1 << 24;  // degree arrays up to 64 MB stay in L2: decrements unread

struct KcoreCtl {
  unsigned bar_count, bar_gen;
  int otail;          // vertices appended to the peel order
  int live_n[2];      // live-list sizes (ping-pong)
  int pad;
  long long wtail;    // work items appended
  int minrem[3];      // smallest remaining degree, rotated per level scan
  long long snap[2][3];  // (otail, wtail, live) captured by the last block into each barrier
};

__device__ __forceinline__ long long ld_vol64(const long long *p) { return *(const volatile long long *)p; }

// Grid barrier that also snapshots (otail, wtail) when every block has
// arrived.  Bounded spin: on timeout the error word is set.
__device__ __forceinline__ void barrier_snap(KcoreCtl *ctl, unsigned nblocks, int32_t *err, long long spin_limit,
                                             long long *otail_out, long long *wtail_out, const int *live_src,
                                             long long *live_out) {
  __shared__ long long s_o, s_w, s_l;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned g0 = *(volatile unsigned *)&ctl->bar_gen;
    __threadfence();
    if (atomicAdd(&ctl->bar_count, 1u) == nblocks - 1) {
      __threadfence();
      ctl->snap[(g0 + 1) & 1][0] = *(volatile int *)&ctl->otail;
      ctl->snap[(g0 + 1) & 1][1] = ld_vol64(&ctl->wtail);
      ctl->snap[(g0 + 1) & 1][2] = live_src ? *(volatile const int *)live_src : 0;
      *(volatile unsigned *)&ctl->bar_count = 0;
      __threadfence();
      atomicAdd(&ctl->bar_gen, 1u);
    } else {
      long long it = 0;
      while (*(volatile unsigned *)&ctl->bar_gen == g0) {
        if (++it > spin_limit) { atomicExch(err, kDevTimeout); break; }
        __nanosleep(16);
      }
    }
    __threadfence();
    s_o = ld_vol64(&ctl->snap[(g0 + 1) & 1][0]);
    s_w = ld_vol64(&ctl->snap[(g0 + 1) & 1][1]);
    s_l = ld_vol64(&ctl->snap[(g0 + 1) & 1][2]);
  }
  __syncthreads();
  *otail_out = s_o;
  *wtail_out = s_w;
  if (live_out) *live_out = s_l;
}

__global__ void degree_init_kernel(int64_t n, const int64_t *__restrict__ rp, int32_t *__restrict__ deg,
                                   int32_t *__restrict__ core, int32_t *__restrict__ maxdeg) {
  int local = 0;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    int d = (int)(rp[v + 1] - rp[v]);
    deg[v] = d;
    core[v] = -1;  // not yet in the peel order
    local = max(local, d);
  }
  local = dev::warp_max(local);
  if ((threadIdx.x & 31) == 0) atomicMax(maxdeg, local);
}

// The rows a block peels within one phase: two generations of two lists
// (rows of 1..32 edges, walked one lane per row; the 128-edge chunks of rows
// of 33..kLocalRow edges, encoded like work items and walked by one warp
// each).  The new frontier found while one generation is walked goes to the
// other, so the block's 32 warps share its cascade.  A counter may run past
// its list's capacity: the entries beyond it were not stored (those rows or
// chunks became work items instead).
struct BlockPool {
  int s[2][kPoolShort];
  long long l[2][kPoolLong];
  int ns[2], nl[2];
  long long edges;  // edges walked from the lists in this phase
  int fscan[kWarps][32 * kScanSlices];  // a warp's scanned frontier, compacted
};

// Append the lanes' new frontier vertices (flag nf, vertex u): core and
// peel order; then their rows' work.  With a block pool (bp, generation
// gen), rows of 1..kLocalRow edges go onto its lists while there is room,
// to be walked by this block in the same phase; the others become one work
// item per chunk of their row, walked in the next sub-round.  All lanes
// call.
template <bool CLAIM>
__device__ __forceinline__ void append_frontier(bool nf, int u, int k, const int64_t *__restrict__ rp, int32_t *core,
                                                int32_t *order, long long *wq, KcoreCtl *ctl,
                                                BlockPool *bp = nullptr, int gen = 0) {
  const int lane = threadIdx.x & 31;
  if (!__any_sync(0xffffffffu, nf)) return;
  // claim: a vertex found by a scan and by a decrement in the same phase
  // joins once; after the scan only decrements find vertices, each exactly
  // once (the one that takes its degree from k + 1 to k), so a store does
  if (CLAIM) {
    if (nf) nf = atomicCAS(core + u, -1, k) == -1;
  } else if (nf) {
    core[u] = k;
  }
  const unsigned m = __ballot_sync(0xffffffffu, nf);
  if (!m) return;
  const unsigned lt = (1u << lane) - 1u;
  int64_t d = 0;
  if (nf) d = rp[u + 1] - rp[u];
  // chunks [c0, c0 + nch) of the lane's row become work items
  int c0 = 0, nch = (nf && d > 0) ? (int)((d + kChunk - 1) / kChunk) : 0;
  if (bp) {
    const bool sh = nf && d > 0 && d <= 32;
    const bool lg = nf && d > 32 && d <= kLocalRow;
    const unsigned ms = __ballot_sync(0xffffffffu, sh);
    int lincl = lg ? nch : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, lincl, o);
      if (lane >= o) lincl += y;
    }
    const int ltot = __shfl_sync(0xffffffffu, lincl, 31);
    int bs = 0, bl = 0;
    if (lane == 0) {
      if (ms) bs = atomicAdd(&bp->ns[gen], __popc(ms));
      if (ltot) bl = atomicAdd(&bp->nl[gen], ltot);
    }
    bs = __shfl_sync(0xffffffffu, bs, 0);
    bl = __shfl_sync(0xffffffffu, bl, 0);
    if (sh) {
      const int at = bs + __popc(ms & lt);
      if (at < kPoolShort) {
        bp->s[gen][at] = u;
        nch = 0;
      }
    }
    if (lg) {
      // the chunks that fit go onto the list, the rest become work items
      const int at = bl + lincl - nch;
      const int fit = max(0, min(nch, kPoolLong - at));
      for (int c = 0; c < fit; c++) bp->l[gen][at + c] = ((long long)u << 32) | (unsigned)c;
      c0 = fit;
      nch -= fit;
    }
  }
  int incl = nch;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  const int tot = __shfl_sync(0xffffffffu, incl, 31);
  int ob = 0;
  long long wb = 0;
  if (lane == 0) {
    ob = atomicAdd(&ctl->otail, __popc(m));
    if (tot) wb = (long long)atomicAdd((unsigned long long *)&ctl->wtail, (unsigned long long)tot);
  }
  ob = __shfl_sync(0xffffffffu, ob, 0);
  wb = __shfl_sync(0xffffffffu, wb, 0);
  if (nf) {
    order[ob + __popc(m & lt)] = u;
    long long at = wb + incl - nch;
    for (int c = 0; c < nch; c++) wq[at + c] = ((long long)u << 32) | (unsigned)(c0 + c);
  }
  __syncwarp();
}

// One work item per lane that has one (a chunk entry of a block list).
__device__ __forceinline__ void push_entry(bool has, long long e, long long *wq, KcoreCtl *ctl) {
  const int lane = threadIdx.x & 31;
  const unsigned m = __ballot_sync(0xffffffffu, has);
  if (!m) return;
  long long wb = 0;
  if (lane == 0) wb = (long long)atomicAdd((unsigned long long *)&ctl->wtail, (unsigned long long)__popc(m));
  wb = __shfl_sync(0xffffffffu, wb, 0);
  if (has) wq[wb + __popc(m & ((1u << lane) - 1u))] = e;
}

// Work items (one per chunk) for lanes' vertices already in the peel order:
// what is left on a block's lists at the end of its budget.
__device__ __forceinline__ void push_items(bool has, int u, const int64_t *__restrict__ rp, long long *wq,
                                           KcoreCtl *ctl) {
  const int lane = threadIdx.x & 31;
  const int nch = has ? (int)((rp[u + 1] - rp[u] + kChunk - 1) / kChunk) : 0;
  int incl = nch;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  const int tot = __shfl_sync(0xffffffffu, incl, 31);
  if (!tot) return;
  long long wb = 0;
  if (lane == 0) wb = (long long)atomicAdd((unsigned long long *)&ctl->wtail, (unsigned long long)tot);
  wb = __shfl_sync(0xffffffffu, wb, 0);
  long long at = wb + incl - nch;
  for (int c = 0; c < nch; c++) wq[at + c] = ((long long)u << 32) | (unsigned)c;
}

// One decrement of neighbour u at level k; true when u joins the level-k
// frontier through it.  With chk the degree is read first and only a degree
// above k is decremented, so the decrement that takes it from k + 1 to k is
// the one that finds u.  Without chk the read is skipped: a peeled
// neighbour's degree (at most k, no longer read) just goes lower.  In the
// sub-rounds every vertex at degree k or below is already peeled, so again
// only k + 1 -> k finds one; while a scan may still read the degrees
// (CLAIM), a vertex still at exactly k may not have been reached by it yet,
// so the decrement from k claims it too (the claim's compare-and-swap keeps
// each vertex to one join).
template <bool CLAIM>
__device__ __forceinline__ bool decrement(int32_t *deg, int u, int k, bool chk) {
  if (u < 0) return false;
  if (chk && __ldcg(deg + u) <= k) return false;
  const int old = atomicSub(deg + u, 1);
  return old == k + 1 || (CLAIM && !chk && old == k);
}

// Walk one row (b0, len) with the whole warp (coalesced), kPer edges per
// lane in flight before the frontier appends.
template <bool CLAIM>
__device__ __forceinline__ void walk_row(int64_t b0, int len, int k, bool chk, const int64_t *__restrict__ rp,
                                         const int32_t *__restrict__ ci, int32_t *deg, int32_t *core, int32_t *order,
                                         long long *wq, KcoreCtl *ctl, BlockPool *bp, int gen) {
  const int lane = threadIdx.x & 31;
  for (int eb = 0; eb < len; eb += 32 * kPer) {
    int u[kPer];
    bool nf[kPer];
#pragma unroll
    for (int q = 0; q < kPer; q++) {
      const int e = eb + q * 32 + lane;
      u[q] = e < len ? ci[b0 + e] : -1;
    }
#pragma unroll
    for (int q = 0; q < kPer; q++) nf[q] = decrement<CLAIM>(deg, u[q], k, chk);
#pragma unroll
    for (int q = 0; q < kPer; q++) append_frontier<CLAIM>(nf[q], u[q], k, rp, core, order, wq, ctl, bp, gen);
  }
}

// Walk rows of at most 32 edges, one lane per row (b0, len; len 0 for idle
// lanes), decrementing every neighbour whose degree is still above k; new
// frontier vertices are appended (to the block's lists when given).
template <bool CLAIM>
__device__ __forceinline__ void walk_short_rows(int64_t b0, int len, int k, bool chk, const int64_t *__restrict__ rp,
                                                const int32_t *__restrict__ ci, int32_t *deg, int32_t *core,
                                                int32_t *order, long long *wq, KcoreCtl *ctl, BlockPool *bp,
                                                int gen) {
  const int maxlen = dev::warp_max(len);
  for (int j0 = 0; j0 < maxlen; j0 += kPer) {
    int u[kPer];
    bool nf[kPer];
#pragma unroll
    for (int q = 0; q < kPer; q++) u[q] = (j0 + q < len) ? ci[b0 + j0 + q] : -1;
#pragma unroll
    for (int q = 0; q < kPer; q++) nf[q] = decrement<CLAIM>(deg, u[q], k, chk);
#pragma unroll
    for (int q = 0; q < kPer; q++) append_frontier<CLAIM>(nf[q], u[q], k, rp, core, order, wq, ctl, bp, gen);
  }
}

// The block's own cascade: the rows on its lists of generation gen, walked
// by all its warps (short rows 32 to a warp, one lane each; chunks of long
// rows one warp each), the new frontier going to the other generation, until the
// lists are empty or kBlockDrainEdges edges were walked; what is left
// becomes work items of the next sub-round.  Every thread of the block
// calls; the lists are empty on return.
template <bool CLAIM>
__device__ void block_drain(int k, bool chk, const int64_t *__restrict__ rp, const int32_t *__restrict__ ci,
                            int32_t *deg, int32_t *core, int32_t *order, long long *wq, KcoreCtl *ctl, BlockPool *bp,
                            int gen) {
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  for (;;) {
    __syncthreads();  // the generation's rows are in place, its edges counted
    const int ns = min(bp->ns[gen], kPoolShort), nl = min(bp->nl[gen], kPoolLong);
    const long long walked = bp->edges;
    __syncthreads();  // every thread has read the counters before they change
    if (ns + nl == 0) break;
    if (walked >= kBlockDrainEdges) {
      for (int j0 = wib * 32; j0 < ns; j0 += kThreads) {
        const int j = j0 + lane;
        push_items(j < ns, j < ns ? bp->s[gen][j] : 0, rp, wq, ctl);
      }
      for (int j0 = wib * 32; j0 < nl; j0 += kThreads) {
        const int j = j0 + lane;
        push_entry(j < nl, j < nl ? bp->l[gen][j] : 0, wq, ctl);
      }
      break;
    }
    if (threadIdx.x == 0) {
      bp->ns[gen ^ 1] = 0;
      bp->nl[gen ^ 1] = 0;
    }
    __syncthreads();
    int mine = 0;
    for (int j0 = wib * 32; j0 < ns; j0 += kThreads) {
      const int j = j0 + lane;
      const int u = j < ns ? bp->s[gen][j] : -1;
      const int64_t b0 = u >= 0 ? rp[u] : 0;
      const int len = u >= 0 ? (int)(rp[u + 1] - b0) : 0;
      mine += len;
      walk_short_rows<CLAIM>(b0, len, k, chk, rp, ci, deg, core, order, wq, ctl, bp, gen ^ 1);
    }
    for (int j = wib; j < nl; j += kWarps) {
      const long long e = bp->l[gen][j];
      const int u = (int)(e >> 32), c = (int)(e & 0xffffffff);
      const int64_t b0 = rp[u] + (int64_t)c * kChunk;
      const int len = (int)(min(rp[u + 1], b0 + kChunk) - b0);
      if (lane == 0) mine += len;
      walk_row<CLAIM>(b0, len, k, chk, rp, ci, deg, core, order, wq, ctl, bp, gen ^ 1);
    }
    mine = dev::warp_sum(mine);
    if (lane == 0 && mine) atomicAdd((unsigned long long *)&bp->edges, (unsigned long long)mine);
    gen ^= 1;
  }
  if (threadIdx.x == 0) {
    bp->ns[0] = bp->ns[1] = 0;
    bp->nl[0] = bp->nl[1] = 0;
    bp->edges = 0;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kThreads, 1) kcore_peel_kernel(int64_t n, const int64_t *__restrict__ rp,
                                                                 const int32_t *__restrict__ ci, int32_t *deg,
                                                                 int32_t *core, int32_t *order, int32_t *live0,
                                                                 int32_t *live1, long long *wq, KcoreCtl *ctl,
                                                                 int32_t *err, long long spin_limit, int nocheck) {
  __shared__ int bmin;
  extern __shared__ __align__(16) unsigned char s_pool[];
  BlockPool *bp = (BlockPool *)s_pool;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t gwarp = (int64_t)blockIdx.x * kWarps + wib;
  const int64_t nwarps = (int64_t)gridDim.x * kWarps;
  const unsigned nblocks = gridDim.x;
  const bool leader = blockIdx.x == 0 && threadIdx.x == 0;
  const unsigned lt = (1u << lane) - 1u;
  const bool chk = nocheck == 0;
  if (threadIdx.x == 0) {
    bp->ns[0] = bp->ns[1] = 0;
    bp->nl[0] = bp->nl[1] = 0;
    bp->edges = 0;
  }

  int k = 0;
  unsigned level = 0;
  long long otail_now = 0, otail_prev = 0, wtail_now = 0, wstart = 0;
  int64_t live_count = n;  // level 0 scans every vertex (identity list)
  int32_t *lin = live0, *lout = live1;

  for (;;) {
    // ---------------- scan: frontier of level k, compaction of the rest ----
    if (threadIdx.x == 0) bmin = INT_MAX;
    if (leader) {
      ctl->minrem[(level + 1) % 3] = INT_MAX;
      ctl->live_n[(level + 1) & 1] = 0;
    }
    __syncthreads();
    int lmin = INT_MAX;
    int *lout_n = &ctl->live_n[level & 1];
    const bool scan_local = live_count <= kScanLocalLive;  // the same in every block
    // groups of kScanSlices slices of 32 live entries go round-robin over the
    // blocks first, so a run of frontier vertices in the list is spread over
    // many blocks; a warp reads a group's entries and degrees at once, takes
    // its place in the next live list with one atomic, and appends the
    // group's frontier 32 vertices at a time
    int *fw = bp->fscan[wib];
    constexpr int kGroup = 32 * kScanSlices;
    for (int64_t sg = blockIdx.x + (int64_t)nblocks * wib; sg * kGroup < live_count; sg += nwarps) {
      int v[kScanSlices], d[kScanSlices];
#pragma unroll
      for (int q = 0; q < kScanSlices; q++) {
        const int64_t i = sg * kGroup + q * 32 + lane;
        v[q] = -1;
        if (i < live_count) v[q] = (level == 0) ? (int)i : lin[i];
      }
#pragma unroll
      for (int q = 0; q < kScanSlices; q++) d[q] = v[q] >= 0 ? __ldcg(deg + v[q]) : INT_MIN;
      int ktot = 0;
#pragma unroll
      for (int q = 0; q < kScanSlices; q++) {
        if (d[q] > k) lmin = min(lmin, d[q]);
        ktot += __popc(__ballot_sync(0xffffffffu, d[q] > k));
      }
      int ob = 0;
      if (lane == 0 && ktot) ob = atomicAdd(lout_n, ktot);
      ob = __shfl_sync(0xffffffffu, ob, 0);
      int ftot = 0;
#pragma unroll
      for (int q = 0; q < kScanSlices; q++) {
        const unsigned km = __ballot_sync(0xffffffffu, d[q] > k);
        if (d[q] > k) lout[ob + __popc(km & lt)] = v[q];
        ob += __popc(km);
        const unsigned fm = __ballot_sync(0xffffffffu, d[q] == k);
        if (d[q] == k) fw[ftot + __popc(fm & lt)] = v[q];
        ftot += __popc(fm);
      }
      __syncwarp();
      for (int f0 = 0; f0 < ftot; f0 += 32) {
        const bool has = f0 + lane < ftot;
        const int u = has ? fw[f0 + lane] : -1;
        if (scan_local)
          append_frontier<true>(has, u, k, rp, core, order, wq, ctl, bp, 0);
        else
          append_frontier<false>(has, u, k, rp, core, order, wq, ctl);
      }
      __syncwarp();
    }
    // the frontier a block found (up to its lists) is peeled at once by that
    // block, while others may still be scanning: a vertex they read at
    // degree k after a decrement here is claimed once; one kept at k + 1 and
    // then peeled here is dropped by the next scan, its degree being <= k.
    // Above kScanLocalLive live vertices the frontier is large enough to
    // keep every warp busy in the sub-rounds: the scan only lists it (no
    // decrement runs during the scan, so each vertex joins once without a
    // claim)
    if (scan_local) block_drain<true>(k, chk, rp, ci, deg, core, order, wq, ctl, bp, 0);
    lmin = -dev::warp_max(-lmin);
    if (lane == 0 && lmin != INT_MAX) atomicMin(&bmin, lmin);
    __syncthreads();
    if (threadIdx.x == 0 && bmin != INT_MAX) atomicMin(&ctl->minrem[level % 3], bmin);
    long long live_next = 0;
    barrier_snap(ctl, nblocks, err, spin_limit, &otail_now, &wtail_now, lout_n, &live_next);
    if (*(volatile int32_t *)err) return;
    live_count = live_next;
    { int32_t *t = lin; lin = lout; lout = t; }

    if (otail_now >= n) break;
    if (otail_now == otail_prev) {
      // nothing at level k: no decrement happened, so the smallest kept
      // degree is exact
      int mk = *(volatile int *)&ctl->minrem[level % 3];
      level++;
      if (mk == INT_MAX) break;  // unreachable while vertices remain
      k = mk;
      continue;
    }

    // ---------------- process: sub-rounds over fixed item ranges ----------
    // Items [s0, e0) were appended before the last barrier; those appended
    // while processing them form the next sub-round.  Warps take groups of
    // 32 items statically: rows shorter than 32 edges are walked one lane per
    // item (lanes in step, so appends stay warp-aggregated), longer chunks by
    // the whole warp.  The frontier they find goes to the block's lists.
    long long s0 = wstart, e0 = wtail_now;
    while (s0 < e0) {
      // pass A: items of fewer than 32 edges, 32 per warp, one lane each
      for (long long gb = s0 + gwarp * 32; gb < e0; gb += nwarps * 32) {
        const long long t = gb + lane;
        const bool valid = t < e0;
        const long long item = valid ? __ldcg(wq + t) : -1LL;
        int64_t b0 = 0;
        int len = 0;
        if (valid) {
          const int v = (int)(item >> 32), c = (int)(item & 0xffffffff);
          b0 = rp[v] + (int64_t)c * kChunk;
          len = (int)(min(rp[v + 1], b0 + kChunk) - b0);
        }
        walk_short_rows<false>(b0, (valid && len < 32) ? len : 0, k, chk, rp, ci, deg, core, order, wq, ctl, bp,
                               0);
      }
      // pass B: longer chunks, one warp each (coalesced row reads)
      for (long long t = s0 + gwarp; t < e0; t += nwarps) {
        const long long item = __ldcg(wq + t);
        const int v = (int)(item >> 32), c = (int)(item & 0xffffffff);
        const int64_t b0 = rp[v] + (int64_t)c * kChunk;
        const int len = (int)(min(rp[v + 1], b0 + kChunk) - b0);
        if (len < 32) continue;
        walk_row<false>(b0, len, k, chk, rp, ci, deg, core, order, wq, ctl, bp, 0);
      }
      block_drain<false>(k, chk, rp, ci, deg, core, order, wq, ctl, bp, 0);
      long long e1 = 0;
      barrier_snap(ctl, nblocks, err, spin_limit, &otail_now, &e1, nullptr, nullptr);
      if (*(volatile int32_t *)err) return;
      s0 = e0;
      e0 = e1;
      wtail_now = e1;
    }
    wstart = wtail_now;
    otail_prev = otail_now;
    level++;
    if (otail_now >= n) break;
    k++;
  }
}

// A peel that stopped early (its spin limit ran out) leaves the tail of the
// order unwritten: such entries are skipped and reported, never used as an
// index.
__global__ void peel_pos_kernel(int64_t n, const int32_t *__restrict__ order, int32_t *__restrict__ pos,
                                const int32_t *__restrict__ core, int32_t *__restrict__ maxcore, int32_t *err) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int v = order[i];
    if (v < 0 || (int64_t)v >= n) {
      atomicCAS(err, kDevOk, kDevCheck);
      continue;
    }
    pos[v] = (int32_t)i;
    if (i == n - 1) *maxcore = core[v];  // the peel order is nondecreasing in K
  }
}

// Batches of small graphs: one block peels one whole graph at a time
// (degrees in shared memory, shared-memory atomics, block barriers between
// sub-rounds), blocks taking graphs from a counter.  The peel order of graph
// g is written to order[voff[g] ..), so each graph's segment is its own
// degeneracy order.
constexpr int kBatchCap = (int)kBatchPeelCap;  // largest graph this kernel takes
constexpr int kBatchThreads = 512;

__global__ void __launch_bounds__(kBatchThreads) kcore_batch_kernel(int32_t count, const int64_t *__restrict__ voff,
                                                                    const int64_t *__restrict__ rp,
                                                                    const int32_t *__restrict__ ci,
                                                                    int32_t *__restrict__ core,
                                                                    int32_t *__restrict__ order, int32_t *next,
                                                                    int32_t *maxdeg, int32_t *maxcore, int32_t *err) {
  __shared__ int deg[kBatchCap];
  __shared__ int q[kBatchCap];
  __shared__ int s_g, s_tail, s_min;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = kBatchThreads / 32;
  const unsigned lt = (1u << lane) - 1u;
  for (;;) {
    __syncthreads();
    if (tid == 0) s_g = atomicAdd(next, 1);
    __syncthreads();
    const int g = s_g;
    if (g >= count) break;
    const int64_t v0 = voff[g];
    const int ng = (int)(voff[g + 1] - v0);
    int lmax = 0;
    for (int i = tid; i < ng; i += kBatchThreads) {
      deg[i] = (int)(rp[v0 + i + 1] - rp[v0 + i]);
      lmax = max(lmax, deg[i]);
    }
    lmax = dev::warp_max(lmax);
    if (lane == 0) atomicMax(maxdeg, lmax);
    if (tid == 0) s_tail = 0;
    __syncthreads();
    int k = 0, head = 0, kmax_g = 0;
    while (true) {
      // scan: every unpeeled vertex with degree == k joins the level
      __syncthreads();  // everyone has read s_min / s_tail of the last level
      if (tid == 0) s_min = INT_MAX;
      __syncthreads();
      int lmin = INT_MAX;
      for (int b = wid * 32; b < ng; b += kBatchThreads) {
        const int i = b + lane;
        const int d = (i < ng) ? deg[i] : INT_MIN;
        const bool hit = d == k;
        if (d > k) lmin = min(lmin, d);
        const unsigned m = __ballot_sync(0xffffffffu, hit);
        if (m) {
          int base = 0;
          if (lane == 0) base = atomicAdd(&s_tail, __popc(m));
          base = __shfl_sync(0xffffffffu, base, 0);
          if (hit) {
            q[base + __popc(m & lt)] = i;
            core[v0 + i] = k;
          }
        }
      }
      lmin = -dev::warp_max(-lmin);
      if (lane == 0 && lmin != INT_MAX) atomicMin(&s_min, lmin);
      __syncthreads();
      int tail = s_tail;
      if (tail == head) {  // nothing at level k
        if (s_min == INT_MAX) break;  // every vertex peeled
        k = s_min;
        continue;
      }
      kmax_g = k;
      // sub-rounds: warps walk the rows of q[head, tail); neighbours that fall
      // to k join q for the next sub-round
      while (head < tail) {
        for (int j = head + wid; j < tail; j += nw) {
          const int i = q[j];
          const int64_t e0 = rp[v0 + i], e1 = rp[v0 + i + 1];
          for (int64_t eb = e0; eb < e1; eb += 32) {
            const int64_t e = eb + lane;
            bool nf = false;
            int u = -1;
            if (e < e1) {
              u = (int)(ci[e] - v0);
              if ((unsigned)u >= (unsigned)ng) {  // an edge leaving the graph: not a valid batch
                atomicExch(err, kDevCheck);
                u = -1;
              } else if (deg[u] > k) {
                nf = (atomicSub(&deg[u], 1) == k + 1);
              }
            }
            const unsigned m = __ballot_sync(0xffffffffu, nf);
            if (m) {
              int base = 0;
              if (lane == 0) base = atomicAdd(&s_tail, __popc(m));
              base = __shfl_sync(0xffffffffu, base, 0);
              if (nf) {
                q[base + __popc(m & lt)] = u;
                core[v0 + u] = k;
              }
            }
          }
        }
        __syncthreads();
        head = tail;
        tail = s_tail;
        __syncthreads();
      }
      k++;
    }
    // the queue is the graph's peel order (core numbers were written on append)
    __syncthreads();
    for (int j = tid; j < ng; j += kBatchThreads) order[v0 + j] = (int32_t)(v0 + q[j]);
    if (tid == 0) atomicMax(maxcore, kmax_g);
    __syncthreads();
  }
}

__global__ void batch_pos_kernel(int64_t n, const int32_t *__restrict__ order, int32_t *__restrict__ pos) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    pos[order[i]] = (int32_t)i;
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
  if (g->count > 1 && g->max_graph_n <= kBatchCap) {
    MC_TRY(ws_get(g, "kc.bctl", 64, &p));
    int32_t *bctl = (int32_t *)p;  // [0] graph counter, [1] max degree, [2] max core
    MC_CUDA_TRY(cudaMemsetAsync(bctl, 0, 64, g->stream));
    int per_sm = 0;
    MC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kcore_batch_kernel, kBatchThreads, 0));
    const int blocks = (int)std::min<int64_t>(g->count, (int64_t)g->sm_count * std::max(per_sm, 1));
    kcore_batch_kernel<<<blocks, kBatchThreads, 0, g->stream>>>(g->count, g->voff, g->row_ptr, g->col_idx, g->core,
                                                                g->order, bctl, bctl + 1, bctl + 2, g->err);
    batch_pos_kernel<<<(int)std::min<int64_t>((n + 255) / 256, (int64_t)g->sm_count * 8), 256, 0, g->stream>>>(
        n, g->order, g->pos);
    g_launches += 2;
    MC_CUDA_TRY(cudaGetLastError());
    if (g->capturing) {
      g->cores_valid = true;
      return MC_OK;
    }
    int32_t *host = (int32_t *)g->h_small;
    MC_CUDA_TRY(cudaMemcpyAsync(host, bctl + 1, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, g->stream));
    MC_CUDA_TRY(cudaStreamSynchronize(g->stream));
    MC_TRY(check_device_error(g));
    g->max_degree = host[0];
    g->max_core = host[1];
    g->cores_valid = true;
    return MC_OK;
  }
  MC_TRY(ws_get(g, "kc.deg", n * sizeof(int32_t), &p));
  int32_t *deg = (int32_t *)p;
  MC_TRY(ws_get(g, "kc.live", 2 * n * sizeof(int32_t) + 64, &p));
  int32_t *live0 = (int32_t *)p, *live1 = live0 + n;
  const int64_t wcap = n + g->nnz / kChunk + 64;
  MC_TRY(ws_get(g, "kc.wq", wcap * sizeof(long long), &p));
  long long *wq = (long long *)p;
  MC_TRY(ws_get(g, "kc.ctl", sizeof(KcoreCtl) + 64, &p));
  KcoreCtl *ctl = (KcoreCtl *)p;
  int32_t *maxdeg = (int32_t *)((char *)p + sizeof(KcoreCtl) + 16);
  MC_CUDA_TRY(cudaMemsetAsync(ctl, 0, sizeof(KcoreCtl) + 64, g->stream));
  MC_CUDA_TRY(cudaMemsetAsync(wq, 0xff, wcap * sizeof(long long), g->stream));

  int ib = (int)std::min<int64_t>((n + 255) / 256, (int64_t)g->sm_count * 8);
  degree_init_kernel<<<ib, 256, 0, g->stream>>>(n, g->row_ptr, deg, g->core, maxdeg);
  g_launches++;
  MC_CUDA_TRY(cudaGetLastError());

  int per_sm = 0;
  const size_t pool = sizeof(BlockPool);
  MC_CUDA_TRY(cudaFuncSetAttribute((const void *)kcore_peel_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)pool));
  MC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kcore_peel_kernel, kThreads, pool));
  if (per_sm < 1) return MC_ERR_CUDA;
  int blocks = g->sm_count;
  int64_t need = (n + kThreads - 1) / kThreads;
  if (need < blocks) blocks = (int)std::max<int64_t>(1, need);
  int64_t n_arg = n;
  const int64_t *rp = g->row_ptr;
  const int32_t *ci = g->col_idx;
  int32_t *core = g->core, *order = g->order, *err = g->err;
  long long sl = spin_limit;
  int nocheck = n <= kNoCheckMaxN ? 1 : 0;
  void *args[] = {&n_arg, (void *)&rp, (void *)&ci, &deg, &core, &order, &live0, &live1, &wq, &ctl, &err, &sl,
                  &nocheck};
  MC_CUDA_TRY(cudaLaunchCooperativeKernel((const void *)kcore_peel_kernel, dim3(blocks), dim3(kThreads), args, pool,
                                          g->stream));
  g_launches++;
  peel_pos_kernel<<<ib, 256, 0, g->stream>>>(n, g->order, g->pos, g->core, maxdeg + 1, g->err);
  g_launches++;
  MC_CUDA_TRY(cudaGetLastError());
  if (g->capturing) {  // K(G) and the degree bound are kept from the direct solve before capture
    g->cores_valid = true;
    return MC_OK;
  }
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

// ------------------------------------------------------------------------
// Core numbers without any device allocation.
//
// Some callers cannot call cudaMalloc: allocator hooks that must not
// re-enter the allocator, or hosts that hand the library a fixed memory
// budget and own every byte of it.  For them this entry point
// runs the same peel with its working memory in a file-scope device array of
// fixed size, reserved when the library is loaded and held by every GPU that
// loads it until the process exits.
// ------------------------------------------------------------------------

namespace mc {
namespace {

constexpr int64_t kNoAllocMaxN = 1 << 20;     // vertices
constexpr int64_t kNoAllocMaxNnz = 1 << 26;   // CSR entries (2 x edges)
constexpr int64_t kNoAllocWq = kNoAllocMaxN + kNoAllocMaxNnz / kChunk + 64;
constexpr size_t kNoAllocCtlBytes = 4096;
// layout: control block | degrees | two live lists | peel order | positions | work items
constexpr size_t kNaOffDeg = kNoAllocCtlBytes;
constexpr size_t kNaOffLive = kNaOffDeg + 4 * kNoAllocMaxN;
constexpr size_t kNaOffOrder = kNaOffLive + 8 * kNoAllocMaxN;
constexpr size_t kNaOffPos = kNaOffOrder + 4 * kNoAllocMaxN;
constexpr size_t kNaOffWq = kNaOffPos + 4 * kNoAllocMaxN;
constexpr size_t kNoAllocBytes = kNaOffWq + 8 * kNoAllocWq;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// The bounds the peel's memory accesses rely on, checked before it runs:
// row_ptr[0] = 0, row_ptr nondecreasing (so every row lies inside
// [0, row_ptr[n]) = [0, nnz)), and every column index in [0, n).  Reads
// only row_ptr[0..n] and col_idx[0..nnz); a failure sets *bad.
__global__ void csr_bounds_kernel(int64_t n, int64_t nnz, const int64_t *__restrict__ rp,
                                  const int32_t *__restrict__ ci, int32_t *bad) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  bool ok = true;
  for (int64_t v = t0; v < n; v += stride) {
    const int64_t a = rp[v], b = rp[v + 1];
    if (b < a || (v == 0 && a != 0)) ok = false;
  }
  for (int64_t e = t0; e < nnz; e += stride) {
    const int32_t u = ci[e];
    if (u < 0 || (int64_t)u >= n) ok = false;
  }
  if (!ok) atomicExch(bad, 1);
}

// device address of g_noalloc_scratch, per device (set up on first use)
static void *g_noalloc_ptr[64];
static std::mutex g_noalloc_mu;

int noalloc_setup(int dev, unsigned char **out) {
  if (dev < 0 || dev >= 64) return MC_ERR_ARG;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      set_last_cuda_error(e, "cudaGetSymbolAddress(g_noalloc_scratch)", __FILE__, __LINE__);
      return MC_ERR_CUDA;
    }
    g_noalloc_ptr[dev] = p;
  }
  *out = (unsigned char *)g_noalloc_ptr[dev];
  return MC_OK;
}

}  // namespace
}  // namespace mc

extern "C" int mc_core_numbers_noalloc(int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
                                       int32_t *core_out, int32_t *max_core_out, void *cuda_stream) {
  using namespace mc;
  if (n < 0 || (n > 0 && (!row_ptr || !col_idx || !core_out))) return MC_ERR_ARG;
  if (n > kNoAllocMaxN) return MC_ERR_TOO_LARGE;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  if (max_core_out) *max_core_out = 0;
  if (n == 0) return MC_OK;
  int dev = 0, sms = 0;
  MC_CUDA_TRY(cudaGetDevice(&dev));
  MC_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  unsigned char *base = nullptr;
  MC_TRY(noalloc_setup(dev, &base));
  int64_t nnz = 0;
  MC_CUDA_TRY(cudaMemcpyAsync(&nnz, row_ptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  MC_CUDA_TRY(cudaStreamSynchronize(s));
  if (nnz < 0) return MC_ERR_ARG;
  if (nnz > kNoAllocMaxNnz) return MC_ERR_TOO_LARGE;

  KcoreCtl *ctl = (KcoreCtl *)base;
  int32_t *maxdeg = (int32_t *)(base + 1024);  // [0] max degree, [1] max core
  int32_t *err = (int32_t *)(base + 2048);
  int32_t *bad = (int32_t *)(base + 3072);
  int32_t *deg = (int32_t *)(base + kNaOffDeg);
  int32_t *live0 = (int32_t *)(base + kNaOffLive), *live1 = live0 + n;
  int32_t *order = (int32_t *)(base + kNaOffOrder);
  int32_t *pos = (int32_t *)(base + kNaOffPos);
  long long *wq = (long long *)(base + kNaOffWq);
  // the array keeps the previous call's contents: clear the control block
  MC_CUDA_TRY(cudaMemsetAsync(base, 0, kNoAllocCtlBytes, s));

  // the peel indexes its arrays by row offsets and column entries, so those
  // are checked first; the caller's graph is not otherwise validated
  const int cb = (int)std::min<int64_t>((std::max(n, nnz) + 255) / 256, (int64_t)sms * 8);
  csr_bounds_kernel<<<cb, 256, 0, s>>>(n, nnz, row_ptr, col_idx, bad);
  g_launches++;
  MC_CUDA_TRY(cudaGetLastError());
  int32_t h_bad = 0;
  MC_CUDA_TRY(cudaMemcpyAsync(&h_bad, bad, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  MC_CUDA_TRY(cudaStreamSynchronize(s));
  if (h_bad) return MC_ERR_INVALID_GRAPH;

  const int ib = (int)std::min<int64_t>((n + 255) / 256, (int64_t)sms * 8);
  degree_init_kernel<<<ib, 256, 0, s>>>(n, row_ptr, deg, core_out, maxdeg);
  g_launches++;
  MC_CUDA_TRY(cudaGetLastError());
  int per_sm = 0;
  const size_t pool = sizeof(BlockPool);
  MC_CUDA_TRY(cudaFuncSetAttribute((const void *)kcore_peel_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)pool));
  MC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kcore_peel_kernel, kThreads, pool));
  if (per_sm < 1) return MC_ERR_CUDA;
  int blocks = sms;
  const int64_t need = (n + kThreads - 1) / kThreads;
  if (need < blocks) blocks = (int)std::max<int64_t>(1, need);
  int64_t n_arg = n;
  long long sl = kDefaultSpinLimit;
  int nocheck = n <= kNoCheckMaxN ? 1 : 0;
  void *args[] = {&n_arg, (void *)&row_ptr, (void *)&col_idx, &deg, &core_out, &order, &live0, &live1, &wq, &ctl,
                  &err, &sl, &nocheck};
  MC_CUDA_TRY(cudaLaunchCooperativeKernel((const void *)kcore_peel_kernel, dim3(blocks), dim3(kThreads), args, pool,
                                          s));
  g_launches++;
  peel_pos_kernel<<<ib, 256, 0, s>>>(n, order, pos, core_out, maxdeg + 1, err);
  g_launches++;
  MC_CUDA_TRY(cudaGetLastError());
  int32_t host[3] = {0, 0, 0};
  MC_CUDA_TRY(cudaMemcpyAsync(host, maxdeg, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  MC_CUDA_TRY(cudaMemcpyAsync(host + 2, err, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  MC_CUDA_TRY(cudaStreamSynchronize(s));
  if (host[2] == kDevTimeout) return MC_ERR_TIMEOUT;
  if (host[2] != kDevOk) return MC_ERR_DEVICE_CHECK;
  if (max_core_out) *max_core_out = host[1];
  return MC_OK;
}
