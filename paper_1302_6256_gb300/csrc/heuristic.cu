// Heuristic clique (Algorithm 1, Section 4.1), one warp (or block) per start vertex.
//
// Vertices are visited in decreasing core number (the peel order reversed).
// For a start vertex v the warp gathers S = neighbours with K >= threshold
// into a per-warp candidate buffer (coalesced row reads, ballot compaction),
// then grows C = {v} greedily: the next member is the remaining candidate of
// largest core number (ties: larger degree, then smaller id), and the
// candidates are filtered to that member's neighbours (binary search in its
// sorted CSR row, or a warp-cooperative merge when the candidate list is long
// compared with the row).  Taking the first remaining candidate each time is the
// same as Algorithm 1's scan "add u if C + u is still a clique" in that order.
//
// mode 0 (Algorithm 1 as printed, run by all warps at once): the running
//   maximum is the incumbent shared through global memory; a warp skips v if
//   K(v) < max, filters S by K >= max, and raises the incumbent when it finds
//   a larger clique.  The result depends on timing; it is always a clique.
// mode 1 (deterministic): every start vertex is grown with threshold 0 and
//   the largest clique wins, ties to the smallest start vertex (a 64-bit
//   atomicMax key); a second kernel regrows the winner and writes it.
// Seeds (learned scores): the top-scored vertices are also grown first, by
//   the same greedy step with the next member chosen by highest score; in
//   mode 1 they only add candidates, so the bound can only rise.
// Start vertices that cannot reach the current best (K(v) + 1 below it) are
// skipped, and a greedy run stops once C plus all remaining candidates cannot
// beat the best (re-read at every step); neither changes the result of either
// mode.
//
// Launches: a warm-up launch grows the first 256 start vertices (the seeds
// and the largest core numbers, whose candidate sets are whole neighbourhoods
// before any clique is known) with one 512-thread block each, two blocks per
// SM so that all 256 run in one wave; the main launch runs 32
// warps per SM with candidate buffers sharing 2 GiB; start vertices with more
// candidates than a buffer holds go to a last launch with full-degree
// buffers.  Every growth, by a block or a warp, yields the same clique.
// The warm-up launch can also run alone (mc_options.heuristic = 3).
#include <algorithm>
#include <climits>

#include "mc_internal.cuh"

namespace mc {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int kHT = 256;  // threads per block
constexpr int64_t kSmallCap = 4096;  // least candidate entries per warp in the first launch
constexpr int64_t kWarm = 256;       // start vertices of the warm-up launch

struct HA {
  int64_t n;
  const int64_t *rp;
  const int32_t *ci, *core, *order, *gid;
  unsigned long long *ctr;  // [0] start vertices grown, [1] adjacency tests, [2] row entries read
  const int64_t *voff;
  int32_t *best, *lock, *wit, *err;
  long long spin;
  int mode;
  int32_t *cand;            // per-warp candidate buffers
  int64_t cand_stride;
  int32_t *cl;              // per-warp clique buffers
  int64_t cl_stride;
  int32_t *next;
  unsigned long long *detkey;  // per graph (mode 1)
  const int32_t *seeds;
  int64_t nseeds;
  const float *score;    // learned vertex scores (seeded start vertices grow by them)
  int64_t begin, limit;  // start vertices [begin, limit) of the visiting order in this launch
  int64_t cap;           // candidate buffer entries per warp
  // start vertices whose candidate set exceeds cap are appended to defer and
  // grown by a second launch with larger buffers, which visits list[0..*nlist)
  int32_t *defer;
  unsigned long long *ndefer;
  const int32_t *list;
  const unsigned long long *nlist;
  // batches peeled graph by graph: visit the j-th highest vertex of every
  // graph before the (j+1)-th of any, so each graph's maximum is set early
  int32_t count;
  int64_t max_graph_n;
  int interleave;
  // positions of the visiting order (after the seeds) grown by an earlier
  // launch of the same solve: position i >= nseeds maps to i - nseeds + skip
  int64_t skip;
};

struct Key {
  int k, d, id;
};
__device__ __forceinline__ bool better(const Key &a, const Key &b) {
  if (a.k != b.k) return a.k > b.k;
  if (a.d != b.d) return a.d > b.d;
  return a.id < b.id;
}
__device__ __forceinline__ Key warp_best(Key x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    Key y{__shfl_xor_sync(FULL, x.k, o), __shfl_xor_sync(FULL, x.d, o), __shfl_xor_sync(FULL, x.id, o)};
    if (better(y, x)) x = y;
  }
  return x;
}
__device__ __forceinline__ Key key_of(const HA &a, int u) {
  return Key{a.core[u], (int)(a.rp[u + 1] - a.rp[u]), u};
}
// Order of a float score as an int (larger score, larger int).
__device__ __forceinline__ int score_order(float f) {
  const int i = __float_as_int(f);
  return i >= 0 ? i : i ^ 0x7fffffff;
}
// Candidate key of a seeded growth: higher score first, then Algorithm 1's
// order (larger core number, then smaller id).
__device__ __forceinline__ Key key_of_scored(const HA &a, int u) {
  return Key{score_order(a.score[u]), a.core[u], u};
}
__device__ __forceinline__ bool in_row(const HA &a, int x, int y) {
  int64_t lo = a.rp[x], hi = a.rp[x + 1];
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    int c = a.ci[mid];
    if (c < y) lo = mid + 1; else hi = mid;
  }
  return lo < a.rp[x + 1] && a.ci[lo] == y;
}

// Greedy clique from v (all lanes).  thr: candidate core threshold; stop_at:
// stop once |C| + |cand| < stop_at (cannot reach it).  by_score: the next
// member is the candidate of highest learned score instead of Algorithm 1's
// largest core number.  Writes the clique to cl[0..size) and returns its
// size, or -1 if the candidates do not fit in cap entries (nothing is grown
// then).
__device__ int grow(const HA &a, int v, int thr, int stop_at, int32_t *cand, int32_t *cl, int64_t cap,
                    bool by_score = false, int g = 0) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const Key none{INT_MIN, INT_MIN, INT_MAX};
  int cnt = 0;
  Key bk = none;
  const int64_t e0 = a.rp[v], e1 = a.rp[v + 1];
  for (int64_t eb = e0; eb < e1; eb += 32) {
    int64_t e = eb + lane;
    int u = -1;
    bool ok = false;
    if (e < e1) {
      u = a.ci[e];
      ok = a.core[u] >= thr;
    }
    unsigned m = __ballot_sync(FULL, ok);
    if (ok) {
      const int at = cnt + __popc(m & lt);
      if (at < cap) cand[at] = u;
      Key k = by_score ? key_of_scored(a, u) : key_of(a, u);
      if (better(k, bk)) bk = k;
    }
    cnt += __popc(m);
  }
  if (cnt > cap) return -1;
  if (lane == 0) {
    atomicAdd(a.ctr + 0, 1ull);
    atomicAdd(a.ctr + 2, (unsigned long long)(e1 - e0));
  }
  bk = warp_best(bk);
  int size = 1;
  if (lane == 0) cl[0] = v;
  for (;;) {
    // the shared best rises while this clique grows: re-read it every step
    // (mode 0: prune candidates below it and stop when C plus candidates
    // cannot beat it; mode 1: stop when they cannot reach its size)
    int cur = 0;
    if (lane == 0)
      cur = a.mode == 0 ? *(volatile int32_t *)(a.best + g)
                        : (int)(*(volatile unsigned long long *)(a.detkey + g) >> 32);
    cur = __shfl_sync(FULL, cur, 0);
    if (a.mode == 0) {
      thr = max(thr, cur);
      stop_at = max(stop_at, cur + 1);
    } else {
      stop_at = max(stop_at, cur);
    }
    if (cnt == 0 || size + cnt < stop_at) break;
    const int w = bk.id;
    if (lane == 0) cl[size] = w;
    size++;
    __syncwarp();
    // keep the candidates adjacent to w (in-place compaction, reads ahead of
    // writes).  Few candidates against a long row: binary search per
    // candidate; otherwise a warp-cooperative merge of the two sorted lists.
    int out = 0;
    Key nb = none;
    const int64_t r0 = a.rp[w], r1 = a.rp[w + 1];
    const bool merge = (int64_t)cnt * 16 >= (r1 - r0);
    if (lane == 0) {
      atomicAdd(a.ctr + 1, (unsigned long long)cnt);
      if (merge) atomicAdd(a.ctr + 2, (unsigned long long)(r1 - r0));
    }
    int64_t pos = r0;
    for (int base = 0; base < cnt; base += 32) {
      const int i = base + lane;
      const int x = (i < cnt) ? cand[i] : INT_MAX;
      bool keep = false;
      if (!merge) {
        keep = i < cnt && x != w && in_row(a, w, x);
      } else {
        const int last = min(31, cnt - 1 - base);
        const int xmin = __shfl_sync(FULL, x, 0), xmax = __shfl_sync(FULL, x, last);
        // skip whole windows of the row below this tile
        while (pos < r1) {
          const int64_t e = min(pos + 31, r1 - 1);
          if (a.ci[e] >= xmin) break;
          pos = e + 1;
        }
        int64_t wp = pos;
        while (wp < r1) {
          const int y = (wp + lane < r1) ? a.ci[wp + lane] : INT_MAX;
          int l = -1;  // largest window index with y <= x
#pragma unroll
          for (int st = 32; st >= 1; st >>= 1) {
            const int t = l + st;
            const int yt = __shfl_sync(FULL, y, t & 31);
            if (t < 32 && yt <= x) l = t;
          }
          const int yl = __shfl_sync(FULL, y, l & 31);
          if (l >= 0 && yl == x) keep = true;
          const int ymax = __shfl_sync(FULL, y, 31);
          if (ymax >= xmax) break;
          wp += 32;
        }
        pos = wp;
        keep = keep && i < cnt && x != w;
      }
      if (keep && thr > 0) keep = a.core[x] >= thr;
      unsigned m = __ballot_sync(FULL, keep);
      __syncwarp();
      if (keep) {
        cand[out + __popc(m & lt)] = x;
        Key k = by_score ? key_of_scored(a, x) : key_of(a, x);
        if (better(k, nb)) nb = k;
      }
      out += __popc(m);
      __syncwarp();
    }
    cnt = out;
    bk = warp_best(nb);
  }
  __syncwarp();
  return size;
}


// Start vertex of visiting position i (false: position past its graph).
__device__ __forceinline__ bool pick_vertex(const HA &a, int64_t i, int *v) {
  if (a.list) {
    *v = a.list[i];
  } else if (i < a.nseeds) {
    *v = a.seeds[i];
    return *v >= 0;  // an empty seed slot (a graph with fewer candidates)
  } else if (a.interleave) {
    const int64_t r = i - a.nseeds + a.skip, gi = r % a.count, j = r / a.count;
    const int64_t v0 = a.voff[gi], v1 = a.voff[gi + 1];
    if (j >= v1 - v0) return false;
    *v = a.order[v1 - 1 - j];
  } else {
    const int64_t r = i - a.nseeds + a.skip;
    if (r >= a.n) return false;
    *v = a.order[a.n - 1 - r];
  }
  return true;
}

constexpr int kWT = 512;       // threads of a warm-up block (two per SM: all 256 starts in one wave)
constexpr int kWW = kWT / 32;  // its warps

// The greedy clique of grow() (same arguments, same result), grown by a whole
// block: the candidate list is split into one contiguous slice per warp, each
// warp filters its slice (binary search, or a merge that starts at the
// slice's first candidate) into its part of the second buffer, and the kept
// candidates are packed back in order.  For the warm-up, where the first
// start vertices have every neighbour as a candidate.
__device__ int grow_block(const HA &a, int v, int thr, int stop_at, int32_t *cur, int32_t *nxt, int32_t *cl,
                          bool by_score, int g) {
  __shared__ int s_cnt[kWW];
  __shared__ Key s_key[kWW];
  __shared__ int s_best;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const unsigned lt = (1u << lane) - 1u;
  const Key none{INT_MIN, INT_MIN, INT_MAX};
  // candidates: neighbours of v with core >= thr, in row order
  const int64_t e0 = a.rp[v], e1 = a.rp[v + 1];
  const int64_t per = (((e1 - e0) + kWW - 1) / kWW + 31) & ~(int64_t)31;
  const int64_t sb = min(e1, e0 + wid * per), se = min(e1, sb + per);
  int c = 0;
  Key bk = none;
  for (int64_t eb = sb; eb < se; eb += 32) {
    const int64_t e = eb + lane;
    int u = -1;
    bool ok = false;
    if (e < se) {
      u = a.ci[e];
      ok = a.core[u] >= thr;
    }
    const unsigned m = __ballot_sync(FULL, ok);
    if (ok) {
      nxt[(sb - e0) + c + __popc(m & lt)] = u;
      const Key k = by_score ? key_of_scored(a, u) : key_of(a, u);
      if (better(k, bk)) bk = k;
    }
    c += __popc(m);
  }
  bk = warp_best(bk);
  if (lane == 0) {
    s_cnt[wid] = c;
    s_key[wid] = bk;
    atomicAdd(a.ctr + 2, (unsigned long long)(se - sb));
  }
  __syncthreads();
  int off = 0, cnt = 0;
  Key best = none;
  for (int w = 0; w < kWW; w++) {
    if (w < wid) off += s_cnt[w];
    cnt += s_cnt[w];
    if (better(s_key[w], best)) best = s_key[w];
  }
  for (int j = lane; j < c; j += 32) cur[off + j] = nxt[(sb - e0) + j];
  if (tid == 0) {
    atomicAdd(a.ctr + 0, 1ull);
    cl[0] = v;
  }
  __syncthreads();
  int size = 1;
  for (;;) {
    if (tid == 0)
      s_best = a.mode == 0 ? *(volatile int32_t *)(a.best + g)
                           : (int)(*(volatile unsigned long long *)(a.detkey + g) >> 32);
    __syncthreads();
    const int cb = s_best;
    if (a.mode == 0) {
      thr = max(thr, cb);
      stop_at = max(stop_at, cb + 1);
    } else {
      stop_at = max(stop_at, cb);
    }
    if (cnt == 0 || size + cnt < stop_at) break;
    const int w = best.id;
    if (tid == 0) {
      cl[size] = w;
      atomicAdd(a.ctr + 1, (unsigned long long)cnt);
    }
    size++;
    const int64_t r0 = a.rp[w], r1 = a.rp[w + 1];
    const int per2 = ((cnt + kWW - 1) / kWW + 31) & ~31;
    const int b0 = min(cnt, wid * per2), b1 = min(cnt, b0 + per2);
    const bool merge = (int64_t)(b1 - b0) * 16 >= (r1 - r0);
    int64_t pos = r0;
    if (merge && b0 < b1) {
      // first row entry not below the slice's first candidate
      const int x0 = cur[b0];
      int64_t lo = r0, hi = r1;
      while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (a.ci[mid] < x0) lo = mid + 1; else hi = mid;
      }
      pos = lo;
      if (lane == 0) atomicAdd(a.ctr + 2, (unsigned long long)(r1 - pos));
    }
    int kept = 0;
    Key nb = none;
    for (int base = b0; base < b1; base += 32) {
      const int i = base + lane;
      const int x = (i < b1) ? cur[i] : INT_MAX;
      bool keep = false;
      if (!merge) {
        keep = i < b1 && x != w && in_row(a, w, x);
      } else {
        const int last = min(31, b1 - 1 - base);
        const int xmin = __shfl_sync(FULL, x, 0), xmax = __shfl_sync(FULL, x, last);
        while (pos < r1) {
          const int64_t e = min(pos + 31, r1 - 1);
          if (a.ci[e] >= xmin) break;
          pos = e + 1;
        }
        int64_t wp = pos;
        while (wp < r1) {
          const int y = (wp + lane < r1) ? a.ci[wp + lane] : INT_MAX;
          int l = -1;
#pragma unroll
          for (int st = 32; st >= 1; st >>= 1) {
            const int t = l + st;
            const int yt = __shfl_sync(FULL, y, t & 31);
            if (t < 32 && yt <= x) l = t;
          }
          const int yl = __shfl_sync(FULL, y, l & 31);
          if (l >= 0 && yl == x) keep = true;
          const int ymax = __shfl_sync(FULL, y, 31);
          if (ymax >= xmax) break;
          wp += 32;
        }
        pos = wp;
        keep = keep && i < b1 && x != w;
      }
      if (keep && thr > 0) keep = a.core[x] >= thr;
      const unsigned m = __ballot_sync(FULL, keep);
      if (keep) {
        nxt[b0 + kept + __popc(m & lt)] = x;
        const Key k = by_score ? key_of_scored(a, x) : key_of(a, x);
        if (better(k, nb)) nb = k;
      }
      kept += __popc(m);
    }
    nb = warp_best(nb);
    __syncthreads();  // every warp has read its slice of cur
    if (lane == 0) {
      s_cnt[wid] = kept;
      s_key[wid] = nb;
    }
    __syncthreads();
    int off2 = 0, tot = 0;
    Key nbest = none;
    for (int ww = 0; ww < kWW; ww++) {
      if (ww < wid) off2 += s_cnt[ww];
      tot += s_cnt[ww];
      if (better(s_key[ww], nbest)) nbest = s_key[ww];
    }
    for (int j = lane; j < kept; j += 32) cur[off2 + j] = nxt[b0 + j];
    __syncthreads();
    cnt = tot;
    best = nbest;
  }
  __syncthreads();
  return size;
}

// Warm-up launch: one block per start vertex (the first positions of the
// visiting order), so the maximum is high before the warp-per-vertex launch.
__global__ void __launch_bounds__(kWT, 2) heuristic_warm_kernel(HA a) {
  __shared__ int64_t s_i;
  __shared__ int s_x;
  int32_t *cur = a.cand + (int64_t)blockIdx.x * 2 * a.cand_stride;
  int32_t *nxt = cur + a.cand_stride;
  int32_t *cl = a.cl + (int64_t)blockIdx.x * a.cl_stride;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_i = *(volatile int32_t *)a.err ? a.limit : a.begin + atomicAdd(a.next, 1);
    __syncthreads();
    const int64_t i = s_i;
    if (i >= a.limit) break;
    int v = 0;
    if (!pick_vertex(a, i, &v)) continue;
    const int g = a.gid ? a.gid[v] : 0;
    const int kv = a.core[v];
    const bool seeded = i < a.nseeds && a.score;
    __syncthreads();
    if (a.mode == 0) {
      if (threadIdx.x == 0) s_x = *(volatile int32_t *)(a.best + g);
      __syncthreads();
      const int mx = s_x;
      if (kv < mx) continue;
      const int size = grow_block(a, v, mx, mx + 1, cur, nxt, cl, seeded, g);
      if (size > mx && threadIdx.x < 32) {
        dev::raise_incumbent(a.best, a.lock, a.wit, a.voff, g, size, a.err, a.spin, [&](int ln, int32_t *base) {
          for (int t = ln; t < size; t += 32) base[t] = cl[t];
        });
      }
    } else {
      if (threadIdx.x == 0) s_x = (int)(*(volatile unsigned long long *)(a.detkey + g) >> 32);
      __syncthreads();
      const int bsz = s_x;
      if (kv + 1 < bsz) continue;
      const int size = grow_block(a, v, 0, bsz, cur, nxt, cl, seeded, g);
      const unsigned long long key = ((unsigned long long)size << 32) | ((seeded ? 1ull : 0ull) << 31) |
                                     (unsigned)(0x7fffffff - v);
      if (threadIdx.x == 0) atomicMax(a.detkey + g, key);
    }
  }
}

__global__ void __launch_bounds__(kHT) heuristic_kernel(HA a) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int32_t *cand = a.cand + gw * a.cand_stride;
  int32_t *cl = a.cl + gw * a.cl_stride;
  const int64_t total = a.list ? (int64_t)*a.nlist : a.limit;
  for (;;) {
    int64_t i = 0;
    if (lane == 0) i = *(volatile int32_t *)a.err ? total : a.begin + atomicAdd(a.next, 1);
    i = __shfl_sync(FULL, (long long)i, 0);
    if (i >= total) break;
    int v = 0;
    if (!pick_vertex(a, i, &v)) continue;
    const int g = a.gid ? a.gid[v] : 0;
    const int kv = a.core[v];
    if (a.mode == 0) {
      int mx = 0;
      if (lane == 0) mx = *(volatile int32_t *)(a.best + g);
      mx = __shfl_sync(FULL, mx, 0);
      if (kv < mx) continue;
      const bool seeded = !a.list && i < a.nseeds && a.score;
      int size = grow(a, v, mx, mx + 1, cand, cl, a.cap, seeded, g);
      if (size < 0) {
        if (lane == 0) a.defer[atomicAdd(a.ndefer, 1ull)] = v;
        continue;
      }
      if (size > mx) {
        dev::raise_incumbent(a.best, a.lock, a.wit, a.voff, g, size, a.err, a.spin, [&](int ln, int32_t *base) {
          for (int t = ln; t < size; t += 32) base[t] = cl[t];
        });
      }
    } else {
      unsigned long long cur = 0;
      if (lane == 0) cur = *(volatile unsigned long long *)(a.detkey + g);
      cur = __shfl_sync(FULL, cur, 0);
      int bsz = (int)(cur >> 32);
      if (kv + 1 < bsz) continue;
      const bool seeded = !a.list && i < a.nseeds && a.score;
      int size = grow(a, v, 0, bsz, cand, cl, a.cap, seeded, g);
      if (size < 0) {
        if (lane == 0) a.defer[atomicAdd(a.ndefer, 1ull)] = v;
        continue;
      }
      // key: size, then seeded growth, then the smaller start vertex
      unsigned long long key = ((unsigned long long)size << 32) | ((seeded ? 1ull : 0ull) << 31) |
                               (unsigned)(0x7fffffff - v);
      if (lane == 0 && key > cur) atomicMax(a.detkey + g, key);
    }
  }
}

// mode 1: regrow each graph's winning start vertex and publish it
__global__ void heuristic_finalize_kernel(HA a, int32_t ngraphs) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  int32_t *cand = a.cand + gw * a.cand_stride;
  int32_t *cl = a.cl + gw * a.cl_stride;
  for (int64_t g = gw; g < ngraphs; g += nw) {
    unsigned long long key = a.detkey[g];
    int size = (int)(key >> 32);
    if (size == 0) continue;
    const bool seeded = ((key >> 31) & 1ull) != 0;
    int v = 0x7fffffff - (int)(key & 0x7fffffffu);
    int s2 = grow(a, v, 0, 0, cand, cl, a.cap, seeded && a.score, (int)g);
    if (s2 != size) {
      if (lane == 0) atomicExch(a.err, kDevCheck);
      continue;
    }
    int32_t *base = a.wit + (a.voff ? a.voff[g] : 0);
    for (int t = lane; t < size; t += 32) base[t] = cl[t];
    __syncwarp();
    __threadfence();
    if (lane == 0) a.best[g] = size;
  }
  (void)lane;
}

}  // namespace

int launch_heuristic(mc_graph *g, int mode, long long spin_limit, const int32_t *seeds, int64_t nseeds,
                     const float *scores, bool warm_only, int64_t skip, int64_t warm_top, int64_t *grown_top) {
  if (grown_top) *grown_top = 0;
  if (g->n == 0) return MC_OK;
  if (warm_only && mode != 0) return MC_ERR_ARG;  // the deterministic form needs every start vertex
  void *p;
  // First launch: 32 warps per SM with candidate buffers that share 2 GiB;
  // start vertices with more candidates are deferred to a second launch with
  // buffers for the largest degree (as many warps as 2 GiB allows).
  const int64_t full = (int64_t)g->max_degree + 1;
  const int64_t budget = (int64_t)1 << 29;  // int32 entries (2 GiB)
  const int64_t cap_s = std::min<int64_t>(full, std::max<int64_t>(kSmallCap, budget / ((int64_t)g->sm_count * 32)));
  const bool two = full > cap_s;
  const int64_t lstride = (int64_t)g->max_core + 2;
  int64_t warps_s = std::min<int64_t>((int64_t)g->sm_count * 32, budget / cap_s);
  warps_s = std::max<int64_t>(32, std::min<int64_t>(warps_s, g->n + nseeds + 32));
  warps_s = (warps_s + 7) / 8 * 8;
  int64_t warps_b = std::max<int64_t>(32, std::min<int64_t>((int64_t)g->sm_count * 16, budget / full));
  warps_b = (warps_b + 7) / 8 * 8;
  // warm-up blocks hold two full-degree candidate buffers each
  const int64_t warm_blocks =
      std::max<int64_t>(1, std::min<int64_t>({(int64_t)g->sm_count * 2, kWarm, budget / (2 * full)}));
  const int64_t cand_entries =
      std::max({warps_s * cap_s, warm_blocks * 2 * full, two || mode == 1 ? warps_b * full : (int64_t)0});
  MC_TRY(ws_get(g, "he.cand", (size_t)cand_entries * 4, &p));
  int32_t *cand = (int32_t *)p;
  MC_TRY(ws_get(g, "he.cl", (size_t)std::max({warps_s, warps_b, warm_blocks}) * lstride * 4, &p));
  int32_t *cl = (int32_t *)p;
  MC_TRY(ws_get(g, "he.ctl", 64 + (size_t)g->count * 8, &p));
  int32_t *next = (int32_t *)p;  // [0] warm-up, [2] main launch, [1] deferred launch; [4..5] deferred count
  unsigned long long *ndefer = (unsigned long long *)((char *)p + 16);
  unsigned long long *hctr = (unsigned long long *)((char *)p + 24);  // three counters, bytes 24..47
  unsigned long long *detkey = (unsigned long long *)((char *)p + 64);
  MC_CUDA_TRY(cudaMemsetAsync(p, 0, 64 + (size_t)g->count * 8, g->stream));
  int32_t *defer = nullptr;
  if (two) {
    MC_TRY(ws_get(g, "he.defer", (size_t)(g->n + nseeds) * 4, &p));
    defer = (int32_t *)p;
  }
  HA a{};
  a.n = g->n;
  a.ctr = hctr;
  g->d_heur_ctr = hctr;
  a.rp = g->row_ptr;
  a.ci = g->col_idx;
  a.core = g->core;
  a.order = g->order;
  a.gid = g->gid;
  a.voff = g->gid ? g->voff : nullptr;
  a.best = g->best;
  a.lock = g->lock;
  a.wit = g->wit;
  a.err = g->err;
  a.spin = spin_limit;
  a.mode = mode;
  a.cand = cand;
  a.cand_stride = cap_s;
  a.cap = two ? cap_s : full;
  a.defer = defer;
  a.ndefer = ndefer;
  a.cl = cl;
  a.cl_stride = lstride;
  a.next = next;
  a.detkey = detkey;
  a.seeds = seeds;
  a.nseeds = seeds ? nseeds : 0;
  a.score = seeds ? scores : nullptr;
  a.count = g->count;
  a.max_graph_n = g->max_graph_n;
  a.interleave = (g->count > 1 && g->max_graph_n <= kBatchPeelCap) ? 1 : 0;
  a.skip = skip;
  const int64_t order_len = a.interleave ? (int64_t)g->count * g->max_graph_n : g->n;
  const int64_t total = std::max<int64_t>(order_len - skip, 0) + a.nseeds;
  // The warm-up part: the seeds, then the first positions of the visiting
  // order (the largest core numbers; for an interleaved batch, each graph's
  // highest vertex), kWarm of them by default.  Its first kWarm positions
  // are grown with a whole block each, so the shared maximum is already high
  // when the warps start and prunes their candidate sets.
  const int64_t top = warm_top >= 0 ? warm_top : (a.interleave ? std::max<int64_t>(kWarm, g->count) : kWarm);
  const int64_t warm_end = std::min<int64_t>(total, a.nseeds + top);
  const int64_t warm = std::min<int64_t>(warm_end, kWarm);
  if (grown_top) *grown_top = std::max<int64_t>(warm_end - a.nseeds, 0);
  a.begin = 0;
  a.limit = warm;
  a.cand_stride = full;
  if (warm > 0) {
    heuristic_warm_kernel<<<(int)warm_blocks, kWT, 0, g->stream>>>(a);
    g_launches++;
    MC_CUDA_TRY(cudaGetLastError());
  }
  a.cand_stride = cap_s;
  const int64_t main_end = warm_only ? warm_end : total;
  if (warm < main_end) {
    a.begin = warm;
    a.limit = main_end;
    a.next = next + 2;
    heuristic_kernel<<<(int)((warps_s * 32 + kHT - 1) / kHT), kHT, 0, g->stream>>>(a);
    g_launches++;
    MC_CUDA_TRY(cudaGetLastError());
  }
  // second launch (deferred start vertices) and the mode-1 regrow use the
  // large buffers
  a.cand_stride = full;
  a.cap = full;
  const int blocks_b = (int)((warps_b * 32 + kHT - 1) / kHT);
  if (two && warm < main_end) {
    a.list = defer;
    a.nlist = ndefer;
    a.next = next + 1;
    heuristic_kernel<<<blocks_b, kHT, 0, g->stream>>>(a);
    g_launches++;
    MC_CUDA_TRY(cudaGetLastError());
  }
  if (mode == 1) {
    heuristic_finalize_kernel<<<blocks_b, kHT, 0, g->stream>>>(a, g->count);
    g_launches++;
    MC_CUDA_TRY(cudaGetLastError());
  }
  return MC_OK;
}

}  // namespace mc
