// Clique-peeling vertex order (Section 6.2) and the gap cost of an order.
//
// Section 6.2 orders the vertices for compression by taking a large clique
// with the heuristic, removing it and repeating, the vertices following the
// cliques in the order found and each clique's members by degree.  Here the
// cliques are taken in rounds, all vertices at once:
//
//   grow    every alive vertex v with no valid stored clique grows Algorithm
//           1's greedy clique C(v) over the alive vertices: candidates are
//           its alive neighbours, the next member is the remaining candidate
//           of largest core number (ties: larger degree, then smaller id),
//           and the candidates are filtered to that member's neighbours.  A
//           stored clique stays valid while all its members are alive (the
//           vertices that died were rejected candidates, whose removal
//           changes no decision of the greedy scan).  Warps check 32
//           vertices at a time and grow the stale ones one after the other;
//           vertices of more than 4,096 neighbours are grown by a whole
//           block, one candidate slice per warp.
//   scatter key(v) = |C(v)| << 32 | (2^31 - 1 - rank(v)); every member u of
//           C(v) takes the largest key of the cliques holding it (atomicMax).
//   accept  C(v) is accepted iff it holds the largest key at every member;
//           accepted cliques are disjoint, and the globally largest key is
//           always accepted.
//   place   an exclusive scan over v of (1 << 32 | |C(v)|) for the accepted
//           ones gives each its group index and position; a warp per
//           accepted clique writes its members ranked by decreasing degree
//           (ties: smaller id) and marks them dead.
//
// Rounds repeat until every vertex is placed (the host reads the placed
// count after each round).  Cliques live in one arena laid out like the
// CSR: vertex v's candidates occupy the front of [rp[v], rp[v+1]) while it
// grows, and its members other than v end at the top of that range, so the
// arena is nnz int32 and needs no per-warp buffers or size limits.
//
// The gap cost relabels the graph by an order (new id = position), sorts
// every new row (bitonic networks: a warp in registers up to 32 entries, a
// warp in shared memory up to 1,024, a block in shared memory up to 16,384,
// a block over a global scratch row beyond), and sums log2(1 + gap) over the
// entries, the first gap of row p taken from p itself: 1 + gap rounded once
// to single precision, log2f (within 1 ulp), summed in double.
#include <algorithm>
#include <climits>

#include "mc_internal.cuh"
#include "scan.cuh"

namespace mc {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int kOT = 256;         // threads per block of the warp-per-vertex kernels
constexpr int kWarpSortMax = 1024;
constexpr int kBlockSortMax = 16384;
constexpr int kBigT = 1024;      // threads of the block sorter
constexpr int kBG = 512;         // threads of the block grower
constexpr int kBGW = kBG / 32;
constexpr int64_t kBlockGrowMin = 4096;  // neighbours above which a block grows the clique
constexpr int kTake = 4;                 // listed vertices a warp takes at a time

struct OA {
  int64_t n;
  const int64_t *rp;
  const int32_t *ci, *core;
  const int32_t *rank;  // tie rank per vertex, nullptr: the vertex id
  uint8_t *alive;
  int32_t *csize;  // stored clique size; 0: grow; negative: accepted this round
  int32_t *arena;
  unsigned long long *bestkey;
  int64_t *ctl;  // [0] placed, [1] groups, [2] grows, [3] candidate tests, [4] rounds, [5] scan total,
                 // [6] the block grower's list length and next entry, [7] the warps' (two unsigned each)
  int64_t *goff;
  int32_t *order;
  int64_t *gstart;
  int32_t *ground;
  int32_t round;
  int32_t *err;
  int32_t *big;     // vertices for the block grower this round
  unsigned *nbig;
  int32_t *stale;   // vertices for the warps this round
  unsigned *nstale, *take, *take_big;
};

struct CKey {
  int k, d, id;
};
__device__ __forceinline__ bool ahead(const CKey &a, const CKey &b) {
  if (a.k != b.k) return a.k > b.k;
  if (a.d != b.d) return a.d > b.d;
  return a.id < b.id;
}
__device__ __forceinline__ CKey warp_first(CKey x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    CKey y{__shfl_xor_sync(FULL, x.k, o), __shfl_xor_sync(FULL, x.d, o), __shfl_xor_sync(FULL, x.id, o)};
    if (ahead(y, x)) x = y;
  }
  return x;
}
__device__ __forceinline__ CKey ckey(const OA &a, int u) {
  return CKey{a.core[u], (int)(a.rp[u + 1] - a.rp[u]), u};
}
__device__ __forceinline__ bool in_row(const int64_t *rp, const int32_t *ci, int x, int y) {
  int64_t lo = rp[x], hi = rp[x + 1];
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (ci[mid] < y) lo = mid + 1; else hi = mid;
  }
  return lo < rp[x + 1] && ci[lo] == y;
}
__device__ __forceinline__ unsigned long long key_of(const OA &a, int v, int size) {
  const int r = a.rank ? a.rank[v] : v;
  return ((unsigned long long)(unsigned)size << 32) | (unsigned)(0x7fffffff - r);
}

// Windowed merge step of a greedy filter (all 32 lanes): lane candidate x
// (INT_MAX past the end; `last` = the last valid lane) against w's row from
// pos, which only moves forward; true iff x is in the row.
__device__ __forceinline__ bool merge_hit(const OA &a, int x, int last, int64_t &pos, int64_t r1) {
  const int xmin = __shfl_sync(FULL, x, 0), xmax = __shfl_sync(FULL, x, last);
  int64_t p = pos;
  while (p < r1) {
    const int64_t e = min(p + 31, r1 - 1);
    if (a.ci[e] >= xmin) break;
    p = e + 1;
  }
  bool hit = false;
  while (p < r1) {
    const int y = (p + (threadIdx.x & 31) < r1) ? a.ci[p + (threadIdx.x & 31)] : INT_MAX;
    int l = -1;  // largest window index with y <= x
#pragma unroll
    for (int st = 32; st >= 1; st >>= 1) {
      const int t = l + st;
      const int yt = __shfl_sync(FULL, y, t & 31);
      if (t < 32 && yt <= x) l = t;
    }
    const int yl = __shfl_sync(FULL, y, l & 31);
    if (l >= 0 && yl == x) hit = true;
    const int ymax = __shfl_sync(FULL, y, 31);
    if (ymax >= xmax) break;
    p += 32;
  }
  pos = p;
  return hit;
}

// Greedy growth of C(v) by one warp (all lanes): v's alive neighbours to the
// front of its arena range (row order: ascending id), then pick the first
// candidate by (core, degree, id) and keep the candidates adjacent to it
// (binary search per candidate when the candidates are few against w's row,
// else a merge), until none is left.  Member j (from 1) goes to rp[v+1] - j
// after its filter: with cnt candidates left, cnt + j <= deg(v), so it lies
// past them.  Returns |C(v)|.
__device__ __forceinline__ int warp_grow(const OA &a, int v, unsigned long long &tests) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const CKey none{INT_MIN, INT_MIN, INT_MAX};
  const int64_t e0 = a.rp[v], e1 = a.rp[v + 1];
  int32_t *cand = a.arena + e0;
  int cnt = 0;
  CKey bk = none;
  for (int64_t eb = e0; eb < e1; eb += 32) {
    const int64_t e = eb + lane;
    int u = -1;
    bool ok = false;
    if (e < e1) {
      u = a.ci[e];
      ok = a.alive[u] != 0;
    }
    const unsigned m = __ballot_sync(FULL, ok);
    if (ok) {
      cand[cnt + __popc(m & lt)] = u;
      const CKey k = ckey(a, u);
      if (ahead(k, bk)) bk = k;
    }
    cnt += __popc(m);
  }
  __syncwarp();
  bk = warp_first(bk);
  int j = 0;
  while (cnt > 0) {
    const int w = bk.id;
    const int64_t r0 = a.rp[w], r1 = a.rp[w + 1];
    const bool merge = (int64_t)cnt * 16 >= (r1 - r0);
    tests += (unsigned long long)cnt;
    int out = 0;
    CKey nb = none;
    int64_t pos = r0;
    for (int base = 0; base < cnt; base += 32) {
      const int i = base + lane;
      const int x = (i < cnt) ? cand[i] : INT_MAX;
      bool keep;
      if (!merge) keep = i < cnt && x != w && in_row(a.rp, a.ci, w, x);
      else keep = merge_hit(a, x, min(31, cnt - 1 - base), pos, r1) && i < cnt && x != w;
      const unsigned m = __ballot_sync(FULL, keep);
      __syncwarp();
      if (keep) {
        cand[out + __popc(m & lt)] = x;
        const CKey k = ckey(a, x);
        if (ahead(k, nb)) nb = k;
      }
      out += __popc(m);
      __syncwarp();
    }
    cnt = out;
    j++;
    if (lane == 0) a.arena[e1 - j] = w;
    __syncwarp();
    bk = warp_first(nb);
  }
  return 1 + j;
}

// Lane test: v's stored clique is missing or holds a placed member.
__device__ __forceinline__ bool needs_grow(const OA &a, int v) {
  const int s = a.csize[v];
  if (s <= 0) return true;
  const int64_t e1 = a.rp[v + 1];
  for (int i = 0; i < s - 1; i++)
    if (!a.alive[a.arena[e1 - 1 - i]]) return true;
  return false;
}

// check: a thread per vertex resets the alive vertices' keys and lists the
// ones that need a clique (warp-aggregated appends): vertices of more than
// kBlockGrowMin neighbours for the block grower, the rest for the warps
__global__ void check_kernel(OA a) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31); base < a.n; base += stride) {
    const int64_t vv = base + lane;
    bool need = false, big = false;
    if (vv < a.n && a.alive[vv]) {
      a.bestkey[vv] = 0ull;
      need = needs_grow(a, (int)vv);
      big = need && a.rp[vv + 1] - a.rp[vv] > kBlockGrowMin;
    }
    const unsigned ms = __ballot_sync(FULL, need && !big), mb = __ballot_sync(FULL, big);
    unsigned at_s = 0, at_b = 0;
    if (lane == 0) {
      if (ms) at_s = atomicAdd(a.nstale, (unsigned)__popc(ms));
      if (mb) at_b = atomicAdd(a.nbig, (unsigned)__popc(mb));
    }
    at_s = __shfl_sync(FULL, at_s, 0);
    at_b = __shfl_sync(FULL, at_b, 0);
    if (need && !big) a.stale[at_s + __popc(ms & lt)] = (int32_t)vv;
    if (big) a.big[at_b + __popc(mb & lt)] = (int32_t)vv;
  }
}

// grow: each warp takes the next kTake listed vertices as it frees up, so a
// few long growths (the dense core's, every round) do not hold back the rest
__global__ void __launch_bounds__(kOT) grow_kernel(OA a) {
  const int lane = threadIdx.x & 31;
  const unsigned total = *a.nstale;
  unsigned long long grows = 0, tests = 0;
  for (;;) {
    unsigned idx = 0;
    if (lane == 0) idx = atomicAdd(a.take, (unsigned)kTake);
    idx = __shfl_sync(FULL, idx, 0);
    if (idx >= total) break;
    const unsigned end = min(total, idx + (unsigned)kTake);
    for (unsigned t = idx; t < end; t++) {
      const int v = a.stale[t];
      const int size = warp_grow(a, v, tests);
      if (lane == 0) {
        a.csize[v] = size;
        grows++;
      }
    }
  }
  if (lane == 0 && grows) atomicAdd((unsigned long long *)(a.ctl + 2), grows);
  if (lane == 0 && tests) atomicAdd((unsigned long long *)(a.ctl + 3), tests);
}

// First candidate over the block (contains two __syncthreads).
__device__ __forceinline__ CKey block_first(CKey x, CKey *sk) {
  x = warp_first(x);
  if ((threadIdx.x & 31) == 0) sk[threadIdx.x >> 5] = x;
  __syncthreads();
  CKey r = sk[0];
#pragma unroll
  for (int i = 1; i < kBGW; i++)
    if (ahead(sk[i], r)) r = sk[i];
  __syncthreads();
  return r;
}

// The same greedy growth by a whole block, for vertices of many neighbours:
// the candidates are split into one slice per warp, each warp merges its
// slice against w's row from the slice's first candidate on and writes what
// it keeps to a scratch row, and the kept runs are packed back in order.
__global__ void __launch_bounds__(kBG) grow_big_kernel(OA a, int32_t *scratch, int64_t scratch_stride) {
  __shared__ CKey sk[kBGW];
  __shared__ int scnt[kBGW];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  const CKey none{INT_MIN, INT_MIN, INT_MAX};
  __shared__ unsigned s_b;
  const unsigned nbig = *a.nbig;
  int32_t *B = scratch + blockIdx.x * scratch_stride;
  unsigned long long grows = 0, tests = 0;
  for (;;) {
    // the next listed vertex, taken as the block frees up
    if (threadIdx.x == 0) s_b = atomicAdd(a.take_big, 1u);
    __syncthreads();
    const unsigned b = s_b;
    __syncthreads();
    if (b >= nbig) break;
    const int v = a.big[b];
    const int64_t e0 = a.rp[v], e1 = a.rp[v + 1];
    int32_t *A = a.arena + e0;
    int cnt = 0;
    CKey bk = none;
    for (int64_t tb = e0; tb < e1; tb += kBG) {
      const int64_t e = tb + threadIdx.x;
      int u = -1;
      bool ok = false;
      if (e < e1) {
        u = a.ci[e];
        ok = a.alive[u] != 0;
      }
      const unsigned m = __ballot_sync(FULL, ok);
      if (lane == 0) scnt[wid] = __popc(m);
      __syncthreads();
      int before = 0, tot = 0;
#pragma unroll
      for (int i = 0; i < kBGW; i++) {
        const int c = scnt[i];
        before += i < wid ? c : 0;
        tot += c;
      }
      if (ok) {
        A[cnt + before + __popc(m & lt)] = u;
        const CKey k = ckey(a, u);
        if (ahead(k, bk)) bk = k;
      }
      cnt += tot;
      __syncthreads();
    }
    bk = block_first(bk, sk);
    int j = 0;
    while (cnt > 0) {
      const int w = bk.id;
      const int64_t r0 = a.rp[w], r1 = a.rp[w + 1];
      if (threadIdx.x == 0) tests += (unsigned long long)cnt;
      const int s0 = (int)((int64_t)cnt * wid / kBGW), s1 = (int)((int64_t)cnt * (wid + 1) / kBGW);
      int out = 0;
      CKey nb = none;
      if (s0 < s1) {
        // the row from its first entry >= A[s0]
        const int x0 = A[s0];
        int64_t lo = r0, hi = r1;
        while (lo < hi) {
          const int64_t mid = (lo + hi) >> 1;
          if (a.ci[mid] < x0) lo = mid + 1; else hi = mid;
        }
        int64_t pos = lo;
        for (int base = s0; base < s1; base += 32) {
          const int i = base + lane;
          const int x = i < s1 ? A[i] : INT_MAX;
          const bool keep = merge_hit(a, x, min(31, s1 - 1 - base), pos, r1) && i < s1 && x != w;
          const unsigned m = __ballot_sync(FULL, keep);
          if (keep) {
            B[s0 + out + __popc(m & lt)] = x;
            const CKey k = ckey(a, x);
            if (ahead(k, nb)) nb = k;
          }
          out += __popc(m);
        }
      }
      if (lane == 0) scnt[wid] = out;
      __syncthreads();
      int before = 0, tot = 0;
#pragma unroll
      for (int i = 0; i < kBGW; i++) {
        const int c = scnt[i];
        before += i < wid ? c : 0;
        tot += c;
      }
      for (int i = lane; i < out; i += 32) A[before + i] = B[s0 + i];
      cnt = tot;
      j++;
      bk = block_first(nb, sk);
      // cnt + j <= deg(v): the member slot lies past the packed candidates
      if (threadIdx.x == 0) a.arena[e1 - j] = w;
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      a.csize[v] = 1 + j;
      grows++;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0 && grows) atomicAdd((unsigned long long *)(a.ctl + 2), grows);
  if (threadIdx.x == 0 && tests) atomicAdd((unsigned long long *)(a.ctl + 3), tests);
}

// scatter: every member takes the largest key of the cliques holding it
__global__ void scatter_kernel(OA a) {
  for (int64_t vv = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; vv < a.n; vv += (int64_t)gridDim.x * blockDim.x) {
    const int v = (int)vv;
    if (!a.alive[v]) continue;
    const int s = a.csize[v];
    const unsigned long long k = key_of(a, v, s);
    const int64_t e1 = a.rp[v + 1];
    atomicMax(a.bestkey + v, k);
    for (int i = 0; i < s - 1; i++) atomicMax(a.bestkey + a.arena[e1 - 1 - i], k);
  }
}

// accept: the clique holds its key at every member
__global__ void accept_kernel(OA a) {
  for (int64_t vv = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; vv < a.n; vv += (int64_t)gridDim.x * blockDim.x) {
    const int v = (int)vv;
    if (!a.alive[v]) continue;
    const int s = a.csize[v];
    const unsigned long long k = key_of(a, v, s);
    const int64_t e1 = a.rp[v + 1];
    bool ok = a.bestkey[v] == k;
    for (int i = 0; i < s - 1 && ok; i++) ok = a.bestkey[a.arena[e1 - 1 - i]] == k;
    if (ok) a.csize[v] = -s;
  }
}

struct AccF {
  const int32_t *csize;
  __device__ int64_t operator()(int64_t v) const {
    const int s = csize[v];
    return s < 0 ? ((int64_t)1 << 32) | (int64_t)(-s) : 0;
  }
};
struct AccG {
  int64_t *goff;
  __device__ void operator()(int64_t v, int64_t excl, int64_t val) const {
    if (val) goff[v] = excl;
  }
};

// place: warps take 32 vertices at a time and write each accepted clique's
// members ranked by degree (whole warp per clique)
__global__ void __launch_bounds__(kOT) place_kernel(OA a) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t placed = a.ctl[0], groups = a.ctl[1];
  for (int64_t base = gw * 32; base < a.n; base += nw * 32) {
    const int64_t vv = base + lane;
    const int sl = vv < a.n ? -a.csize[vv] : 0;
    unsigned m = __ballot_sync(FULL, sl > 0);
    while (m) {
      const int src = __ffs(m) - 1;
      m &= m - 1;
      const int v = (int)base + src;
      const int s = __shfl_sync(FULL, sl, src);
      const int64_t packed = a.goff[v];
      const int64_t gi = groups + (packed >> 32), pos = placed + (packed & 0xffffffffLL);
      const int64_t e1 = a.rp[v + 1];
      // accepted cliques are disjoint sets of unplaced vertices, so they fit;
      // anything else is a broken invariant: report it, write nothing
      if (pos + s > a.n || gi >= a.n) {
        if (lane == 0) atomicExch(a.err, kDevCheck);
        continue;
      }
      for (int i = lane; i < s; i += 32) {
        const int x = i == 0 ? v : a.arena[e1 - i];
        const int64_t dx = a.rp[x + 1] - a.rp[x];
        int r = 0;
        for (int t = 0; t < s; t++) {
          const int y = t == 0 ? v : a.arena[e1 - t];
          const int64_t dy = a.rp[y + 1] - a.rp[y];
          r += (dy > dx || (dy == dx && y < x)) ? 1 : 0;
        }
        a.order[pos + r] = x;
      }
      __syncwarp();
      for (int i = lane; i < s; i += 32) a.alive[i == 0 ? v : a.arena[e1 - i]] = 0;
      if (lane == 0) {
        a.gstart[gi] = pos;
        a.ground[gi] = a.round;
        a.csize[v] = 0;
      }
    }
  }
}

__global__ void advance_kernel(int64_t *ctl) {
  const int64_t t = ctl[5];
  ctl[0] += t & 0xffffffffLL;
  ctl[1] += t >> 32;
  ctl[4] += 1;
  ((unsigned *)(ctl + 6))[0] = 0u;  // the growers' lists, empty for the next round
  ((unsigned *)(ctl + 6))[1] = 0u;
  ((unsigned *)(ctl + 7))[0] = 0u;
  ((unsigned *)(ctl + 7))[1] = 0u;
}

// a caller's tie rank must be a permutation of [0, n): seen[] starts at 0
__global__ void rank_check_kernel(int64_t n, const int32_t *rank, unsigned long long *seen, int32_t *bad) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int r = rank[v];
    if (r < 0 || r >= n || atomicExch(seen + r, 1ull) != 0ull) atomicExch(bad, 1);
  }
}

// ---- relabelling by an order and the gap cost ----

// pos[order[p]] = p; pos starts at -1 everywhere, a repeat or an id out of
// range sets *bad
__global__ void inverse_kernel(int64_t n, const int32_t *order, int32_t *pos, int32_t *bad) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    const int v = order[p];
    if (v < 0 || v >= n || atomicCAS(pos + v, -1, (int)p) != -1) atomicExch(bad, 1);
  }
}

struct DegF {
  const int64_t *rp;
  const int32_t *order;
  __device__ int64_t operator()(int64_t p) const {
    const int v = order[p];
    return rp[v + 1] - rp[v];
  }
};
struct RowG {
  int64_t *nrp;
  __device__ void operator()(int64_t p, int64_t excl, int64_t) const { nrp[p] = excl; }
};

// a warp per new row: copy the old row through pos, sort rows of at most
// kWarpSortMax entries at once (bitonic; registers up to 32, shared memory
// above), and list the longer rows for the block sorter
__global__ void __launch_bounds__(kOT) fill_sort_kernel(int64_t n, const int64_t *rp, const int32_t *ci,
                                                        const int32_t *order, const int32_t *pos,
                                                        const int64_t *nrp, int32_t *nci, int32_t *big,
                                                        unsigned long long *nbig) {
  __shared__ int32_t sm[kOT / 32][kWarpSortMax];
  const int lane = threadIdx.x & 31;
  int32_t *buf = sm[threadIdx.x >> 5];
  const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t p = gw; p < n; p += nw) {
    const int v = order[p];
    const int64_t e0 = rp[v], L = rp[v + 1] - e0, o0 = nrp[p];
    if (L > kWarpSortMax) {
      for (int64_t i = lane; i < L; i += 32) nci[o0 + i] = pos[ci[e0 + i]];
      if (lane == 0) big[atomicAdd(nbig, 1ull)] = (int32_t)p;
      continue;
    }
    if (L <= 32) {
      int x = lane < L ? pos[ci[e0 + lane]] : INT_MAX;
      // bitonic network over the 32 lanes
      for (int k = 2; k <= 32; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
          const int y = __shfl_xor_sync(FULL, x, j);
          const bool up = (lane & k) == 0, lower = (lane & j) == 0;
          x = (lower == up) ? min(x, y) : max(x, y);
        }
      if (lane < L) nci[o0 + lane] = x;
      continue;
    }
    int P = 64;
    while (P < L) P <<= 1;
    for (int i = lane; i < P; i += 32) buf[i] = i < L ? pos[ci[e0 + i]] : INT_MAX;
    __syncwarp();
    for (int k = 2; k <= P; k <<= 1)
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int i = lane; i < P; i += 32) {
          const int l = i ^ j;
          if (l > i) {
            const int x = buf[i], y = buf[l];
            const bool up = (i & k) == 0;
            if ((x > y) == up) {
              buf[i] = y;
              buf[l] = x;
            }
          }
        }
        __syncwarp();
      }
    for (int i = lane; i < L; i += 32) nci[o0 + i] = buf[i];
    __syncwarp();
  }
}

// compare-exchange stages (k, j >= jlo) of a bitonic sort over buf[0..P) by
// the whole block; global index base + i decides the direction
__device__ __forceinline__ void bitonic_stages(int32_t *buf, int P, int64_t base, int k, int jhi, int jlo) {
  for (int j = jhi; j >= jlo; j >>= 1) {
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
      const int l = i ^ j;
      if (l > i) {
        const int x = buf[i], y = buf[l];
        const bool up = ((base + i) & k) == 0;
        if ((x > y) == up) {
          buf[i] = y;
          buf[l] = x;
        }
      }
    }
    __syncthreads();
  }
}

// a block per long row: shared memory up to kBlockSortMax entries, else a
// scratch row of the next power of two in global memory whose stages with
// j below kBlockSortMax run chunk by chunk in shared memory
__global__ void __launch_bounds__(kBigT) block_sort_kernel(const int64_t *nrp, int32_t *nci, const int32_t *big,
                                                           const unsigned long long *nbig, int32_t *scratch,
                                                           int64_t scratch_stride) {
  extern __shared__ int32_t sbuf[];
  const int64_t cnt = (int64_t)*nbig;
  for (int64_t b = blockIdx.x; b < cnt; b += gridDim.x) {
    const int64_t p = big[b];
    const int64_t o0 = nrp[p], L = nrp[p + 1] - o0;
    int64_t P = 1;
    while (P < L) P <<= 1;
    if (P <= kBlockSortMax) {
      for (int64_t i = threadIdx.x; i < P; i += blockDim.x) sbuf[i] = i < L ? nci[o0 + i] : INT_MAX;
      __syncthreads();
      for (int k = 2; k <= P; k <<= 1) bitonic_stages(sbuf, (int)P, 0, k, k >> 1, 1);
      for (int64_t i = threadIdx.x; i < L; i += blockDim.x) nci[o0 + i] = sbuf[i];
      __syncthreads();
      continue;
    }
    int32_t *row = scratch + blockIdx.x * scratch_stride;
    for (int64_t i = threadIdx.x; i < P; i += blockDim.x) row[i] = i < L ? nci[o0 + i] : INT_MAX;
    __syncthreads();
    const int C = kBlockSortMax;
    // every stage with k <= C stays inside a chunk
    for (int64_t c = 0; c < P; c += C) {
      for (int i = threadIdx.x; i < C; i += blockDim.x) sbuf[i] = row[c + i];
      __syncthreads();
      for (int k = 2; k <= C; k <<= 1) bitonic_stages(sbuf, C, c, k, k >> 1, 1);
      for (int i = threadIdx.x; i < C; i += blockDim.x) row[c + i] = sbuf[i];
      __syncthreads();
    }
    for (int64_t k = 2 * (int64_t)C; k <= P; k <<= 1) {
      for (int64_t j = k >> 1; j >= C; j >>= 1) {
        for (int64_t i = threadIdx.x; i < P; i += blockDim.x) {
          const int64_t l = i ^ j;
          if (l > i) {
            const int x = row[i], y = row[l];
            const bool up = (i & k) == 0;
            if ((x > y) == up) {
              row[i] = y;
              row[l] = x;
            }
          }
        }
        __syncthreads();
      }
      for (int64_t c = 0; c < P; c += C) {
        for (int i = threadIdx.x; i < C; i += blockDim.x) sbuf[i] = row[c + i];
        __syncthreads();
        bitonic_stages(sbuf, C, c, (int)k, C >> 1, 1);
        for (int i = threadIdx.x; i < C; i += blockDim.x) row[c + i] = sbuf[i];
        __syncthreads();
      }
    }
    for (int64_t i = threadIdx.x; i < L; i += blockDim.x) nci[o0 + i] = row[i];
    __syncthreads();
  }
}

// sum over the entries of the relabelled graph of log2(1 + gap): each term
// in single precision (one rounding of 1 + gap, log2f within 1 ulp, so a
// relative error below 2^-22), the sum in double
__global__ void __launch_bounds__(kOT) gap_kernel(int64_t n, const int64_t *nrp, const int32_t *nci, double *total) {
  __shared__ double red[kOT / 32];
  const int lane = threadIdx.x & 31;
  const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  double s = 0.0;
  for (int64_t p = gw; p < n; p += nw) {
    const int64_t e0 = nrp[p], e1 = nrp[p + 1];
    for (int64_t e = e0 + lane; e < e1; e += 32) {
      const int64_t x = nci[e];
      const int64_t prev = e == e0 ? p : (int64_t)nci[e - 1];
      const int64_t gap = e == e0 ? (x > p ? x - p : p - x) : x - prev;
      s += (double)log2f((float)(gap + 1));
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
  if (lane == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kOT / 32; w++) t += red[w];
    atomicAdd(total, t);
  }
}

int grid_of(mc_graph *g, int64_t items, int per_block, int per_sm) {
  const int64_t want = (items + per_block - 1) / per_block;
  return (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)g->sm_count * per_sm));
}

}  // namespace

int clique_order(mc_graph *g, const int32_t *rank, int32_t *d_order, int64_t *d_gstart, int32_t *d_ground,
                 int64_t *groups_out, int32_t *rounds_out, int64_t *work_out) {
  const int64_t n = g->n;
  *groups_out = 0;
  *rounds_out = 0;
  if (n == 0) return MC_OK;
  if (!g->cores_valid) MC_TRY(launch_core_numbers(g, kDefaultSpinLimit));
  void *p;
  OA a{};
  a.n = n;
  a.rp = g->row_ptr;
  a.ci = g->col_idx;
  a.core = g->core;
  MC_TRY(ws_get(g, "co.alive", (size_t)n, &p));
  a.alive = (uint8_t *)p;
  MC_TRY(ws_get(g, "co.csize", (size_t)n * 4, &p));
  a.csize = (int32_t *)p;
  MC_TRY(ws_get(g, "co.arena", (size_t)std::max<int64_t>(g->nnz, 1) * 4, &p));
  a.arena = (int32_t *)p;
  MC_TRY(ws_get(g, "co.key", (size_t)n * 8, &p));
  a.bestkey = (unsigned long long *)p;
  MC_TRY(ws_get(g, "co.goff", (size_t)n * 8, &p));
  a.goff = (int64_t *)p;
  MC_TRY(ws_get(g, "co.ctl", 64, &p));
  a.ctl = (int64_t *)p;
  a.err = g->err;
  a.order = d_order;
  a.gstart = d_gstart;
  a.ground = d_ground;
  MC_CUDA_TRY(cudaMemsetAsync(a.ctl, 0, 64, g->stream));
  if (rank) {
    MC_TRY(ws_get(g, "co.rank", (size_t)n * 4, &p));
    MC_CUDA_TRY(cudaMemcpyAsync(p, rank, (size_t)n * 4, cudaMemcpyDefault, g->stream));
    a.rank = (const int32_t *)p;
    int32_t *bad = g->err + 9;
    MC_CUDA_TRY(cudaMemsetAsync(bad, 0, 4, g->stream));
    MC_CUDA_TRY(cudaMemsetAsync(a.bestkey, 0, (size_t)n * 8, g->stream));
    rank_check_kernel<<<grid_of(g, n, 256, 8), 256, 0, g->stream>>>(n, a.rank, a.bestkey, bad);
    g_launches++;
    MC_CUDA_TRY(cudaGetLastError());
    MC_CUDA_TRY(cudaMemcpyAsync(g->h_small, bad, 4, cudaMemcpyDeviceToHost, g->stream));
    MC_CUDA_TRY(cudaStreamSynchronize(g->stream));
    if (*(int32_t *)g->h_small) return MC_ERR_ARG;
  }
  MC_CUDA_TRY(cudaMemsetAsync(a.alive, 1, (size_t)n, g->stream));
  MC_CUDA_TRY(cudaMemsetAsync(a.csize, 0, (size_t)n * 4, g->stream));
  a.nbig = (unsigned *)(a.ctl + 6);
  a.take_big = a.nbig + 1;
  a.nstale = (unsigned *)(a.ctl + 7);
  a.take = a.nstale + 1;
  MC_TRY(ws_get(g, "co.stale", (size_t)n * 4, &p));
  a.stale = (int32_t *)p;
  int32_t *scratch = nullptr;
  const int big_blocks = 2 * g->sm_count;
  const int64_t stride = std::max<int64_t>(g->max_degree, 1);
  const bool any_big = g->max_degree > kBlockGrowMin;
  if (any_big) {
    MC_TRY(ws_get(g, "co.big", (size_t)n * 4, &p));
    a.big = (int32_t *)p;
    MC_TRY(ws_get(g, "co.bscratch", (size_t)big_blocks * stride * 4, &p));
    scratch = (int32_t *)p;
  }
  const int gw = grid_of(g, (n + 31) / 32, kOT / 32, 8), gt = grid_of(g, n, 256, 8);
  int64_t *h = (int64_t *)((char *)g->h_small + 2560);
  int64_t placed = 0;
  for (int32_t r = 0;; r++) {
    a.round = r;
    check_kernel<<<gt, 256, 0, g->stream>>>(a);
    grow_kernel<<<gw, kOT, 0, g->stream>>>(a);
    g_launches++;
    if (any_big) {
      grow_big_kernel<<<big_blocks, kBG, 0, g->stream>>>(a, scratch, stride);
      g_launches++;
    }
    scatter_kernel<<<gt, 256, 0, g->stream>>>(a);
    accept_kernel<<<gt, 256, 0, g->stream>>>(a);
    g_launches += 3;
    MC_CUDA_TRY(cudaGetLastError());
    MC_TRY(device_scan(g, n, AccF{a.csize}, AccG{a.goff}, a.ctl + 5, "co.scan"));
    place_kernel<<<gw, kOT, 0, g->stream>>>(a);
    advance_kernel<<<1, 1, 0, g->stream>>>(a.ctl);
    g_launches += 2;
    MC_CUDA_TRY(cudaGetLastError());
    MC_CUDA_TRY(cudaMemcpyAsync(h, a.ctl, 6 * sizeof(int64_t), cudaMemcpyDeviceToHost, g->stream));
    MC_CUDA_TRY(cudaStreamSynchronize(g->stream));
    // every round places at least the clique of the largest key
    if (h[0] <= placed || h[0] > n) {
      MC_TRY(check_device_error(g));
      return MC_ERR_DEVICE_CHECK;
    }
    placed = h[0];
    if (placed == n) break;
  }
  *groups_out = h[1];
  *rounds_out = (int32_t)h[4];
  if (work_out) {
    work_out[0] = h[2];
    work_out[1] = h[3];
  }
  MC_CUDA_TRY(cudaMemcpyAsync(d_gstart + h[1], &g->n, sizeof(int64_t), cudaMemcpyHostToDevice, g->stream));
  MC_CUDA_TRY(cudaStreamSynchronize(g->stream));
  return MC_OK;
}

int relabel(mc_graph *g, const int32_t *order, int64_t *d_nrp, int32_t *d_nci) {
  const int64_t n = g->n;
  if (n == 0) {
    MC_CUDA_TRY(cudaMemsetAsync(d_nrp, 0, sizeof(int64_t), g->stream));
    return MC_OK;
  }
  if (!g->cores_valid) MC_TRY(launch_core_numbers(g, kDefaultSpinLimit));  // sets max_degree
  void *p;
  MC_TRY(ws_get(g, "rl.order", (size_t)n * 4, &p));
  int32_t *d_order = (int32_t *)p;
  MC_CUDA_TRY(cudaMemcpyAsync(d_order, order, (size_t)n * 4, cudaMemcpyDefault, g->stream));
  MC_TRY(ws_get(g, "rl.pos", (size_t)n * 4, &p));
  int32_t *pos = (int32_t *)p;
  int32_t *bad = g->err + 10;
  MC_CUDA_TRY(cudaMemsetAsync(bad, 0, 4, g->stream));
  MC_CUDA_TRY(cudaMemsetAsync(pos, 0xff, (size_t)n * 4, g->stream));
  inverse_kernel<<<grid_of(g, n, 256, 8), 256, 0, g->stream>>>(n, d_order, pos, bad);
  g_launches++;
  MC_CUDA_TRY(cudaGetLastError());
  MC_CUDA_TRY(cudaMemcpyAsync(g->h_small, bad, 4, cudaMemcpyDeviceToHost, g->stream));
  MC_CUDA_TRY(cudaStreamSynchronize(g->stream));
  if (*(int32_t *)g->h_small) return MC_ERR_ARG;
  MC_TRY(device_scan(g, n, DegF{g->row_ptr, d_order}, RowG{d_nrp}, d_nrp + n, "rl.scan"));
  MC_TRY(ws_get(g, "rl.big", (size_t)n * 4, &p));
  int32_t *big = (int32_t *)p;
  MC_TRY(ws_get(g, "rl.nbig", 8, &p));
  unsigned long long *nbig = (unsigned long long *)p;
  MC_CUDA_TRY(cudaMemsetAsync(nbig, 0, 8, g->stream));
  fill_sort_kernel<<<grid_of(g, n * 32, kOT, 8), kOT, 0, g->stream>>>(n, g->row_ptr, g->col_idx, d_order, pos,
                                                                        d_nrp, d_nci, big, nbig);
  g_launches++;
  MC_CUDA_TRY(cudaGetLastError());
  if (g->max_degree > kWarpSortMax) {
    int64_t P = 1;
    while (P < g->max_degree) P <<= 1;
    const int blocks = g->sm_count;
    int32_t *scratch = nullptr;
    int64_t stride = 0;
    if (P > kBlockSortMax) {
      stride = P;
      MC_TRY(ws_get(g, "rl.scratch", (size_t)blocks * P * 4, &p));
      scratch = (int32_t *)p;
    }
    const int smem = kBlockSortMax * 4;
    MC_CUDA_TRY(cudaFuncSetAttribute(block_sort_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    block_sort_kernel<<<blocks, kBigT, smem, g->stream>>>(d_nrp, d_nci, big, nbig, scratch, stride);
    g_launches++;
    MC_CUDA_TRY(cudaGetLastError());
  }
  return MC_OK;
}

int gap_bits(mc_graph *g, const int64_t *d_nrp, const int32_t *d_nci, double *d_total) {
  MC_CUDA_TRY(cudaMemsetAsync(d_total, 0, sizeof(double), g->stream));
  if (g->n == 0) return MC_OK;
  gap_kernel<<<grid_of(g, g->n * 32, kOT, 8), kOT, 0, g->stream>>>(g->n, d_nrp, d_nci, d_total);
  g_launches++;
  MC_CUDA_TRY(cudaGetLastError());
  return MC_OK;
}

}  // namespace mc
