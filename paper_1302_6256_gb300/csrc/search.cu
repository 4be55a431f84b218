// Neighbourhood branch and bound: InitialBranch and Branch of Algorithm 2
// (Section 4.3), with the incumbent shared by every worker as soon as it
// changes (Section 4.5).
//
// For a root u of the oriented pruned graph the candidate set is
//   P = { w in N+(u) : K(w) >= omega }           (N_R(u) of Section 4.3)
// and the search looks for a clique larger than omega containing u:
//   1. |P| < omega                    -> return (degree bound, Fact 2 (3))
//   2. bitset adjacency of G[P]       (the small-graph adjacency matrix of
//      Section 4.4): each member's later-neighbour row is probed against a
//      hash table of P, which sets the lower triangle (a later neighbour has
//      a smaller index in P); warp-ballot transposes of 32 x 32 tiles fill
//      the upper triangle
//   3. (omega-1)-core of G[P]: exactly the vertices with neighbourhood core
//      number K_N >= |H| when u is counted (lines 15-18 of InitialBranch;
//      the tight form of the test); fewer than omega left -> return
//   4. greedy colouring, L colours; 1 + L <= omega -> return (Fact 2 (1))
//   5. Branch({u}, P): depth-first, each node colours its candidates
//      greedily in index order (independent-set extraction with ballot and
//      popc over bit rows) and branches on the vertices whose colour can still
//      beat omega; a maximal clique larger than omega raises the incumbent.
// Bit positions are P sorted by decreasing rank, so "index order" colours the
// latest vertices of the degeneracy order first (the degeneracy-order
// colouring of InitialBranch) and every node uses the same natural order.
//
// Workers, split by the out-degree of the root (an upper bound on |P|):
//   warp class   |N+(u)| <= 128: one warp per root, matrix in shared memory;
//   block class  |N+(u)| <= 1024: one block per root, matrix in shared
//                memory; a 512-candidate layout at two blocks per SM first,
//                then a 1,024-candidate launch for the roots it deferred; the
//                block's 16 warps share the root's search tree through a
//                shared-memory pool (a busy warp hands the shallowest untried
//                branch to an idle one);
//   big class    larger: as the block class with the matrix in global memory.
// Task queue: a warp (block) that expands more than its budget of Branch
// nodes on one root copies the root's matrix to an arena and turns every
// untried branch of its stack into a task in a GPU-wide ring; the task
// kernel searches tasks with whole blocks and spills again while the queue
// is short, so one hard neighbourhood spreads over the whole GPU.
// Every spin-wait is bounded; on timeout the device error word is set.
#include <algorithm>
#include <climits>

#include "mc_internal.cuh"

namespace mc {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int kBW = 16;  // warps per block-class block
constexpr int kBT = kBW * 32;
constexpr int kSW = 8;   // warps per warp-class block
constexpr int kWarpCap = 128;
constexpr int kPoolCap = 16;

struct SA {
  const int64_t *orow;
  const int32_t *ocol, *ocore, *oold, *ogid;
  const int32_t *roots;
  const int64_t *nroots;    // device: number of roots in this class
  const int64_t *np_count;  // device: vertices of the pruned graph
  int32_t use_bitmap;       // look members up in a bitmap of the later ranks when they fit
  int32_t *best, *lock, *wit;
  const int64_t *voff;
  int32_t *err;
  long long spin;
  int32_t *next;            // root grab counter
  uint32_t *stack;          // per-warp DFS stacks
  int64_t stack_stride;     // words per warp stack
  uint32_t *gmat;           // per-block global matrix (big class)
  int64_t gmat_stride;      // words per block matrix
  int32_t neigh_cores;
  unsigned long long *counters;  // colored, branched, nodes, donations, entries
  // published roots: matrix + P list in a global arena, first-level tasks
  uint32_t *arena;
  long long arena_cap;           // words
  unsigned long long *arena_used;
  struct RootRec *recs;
  int32_t rec_cap;
  int32_t *nrec;
  uint32_t *tasks;               // kTaskWords words per task
  int32_t *ready;                // per ring slot: 2*lap free for lap's writer, 2*lap+1 written
  int32_t task_cap;              // ring slots (a power of two)
  int32_t *ntasks;               // positions taken (the queue's tail, monotonic)
  int32_t *task_next;            // positions handed out (the queue's head)
  int32_t *active;               // blocks of the task kernel holding a task
  int32_t *progress;             // heartbeat: bumped every 256 Branch nodes
  int32_t queue_gate;            // spill only while fewer tasks wait (0 = always)
  int32_t *overflow;             // roots too large for this launch's layout (or null)
  int64_t *noverflow;
  long long budget_warp;         // Branch nodes before a warp worker spills
  long long budget_block;        // ... and a block, on one root or task
};

struct RootRec {
  int u, g, p, W, Ws, pad;
  long long off;  // arena word offset: matrix (p x Ws words), then the P list (p ints)
};
constexpr int kTaskWords = 2 + 64;  // root record, clique size, C bits, P bits (32 words each)
constexpr long long kArenaWords = 64ll << 20;  // 256 MB of published matrices
constexpr int kRecCap = 1 << 16;
constexpr int kTaskCap = 1 << 20;          // ring slots, 277 MB
constexpr long long kSpillNodes = 4096;    // default Branch-node budget of a warp worker
constexpr int kMidCap = 512;               // candidates of the two-blocks-per-SM block layout

template <int WPL>
struct Bits {
  uint32_t w[WPL];
};

template <int WPL>
__device__ __forceinline__ void bzero(Bits<WPL> &b) {
#pragma unroll
  for (int k = 0; k < WPL; k++) b.w[k] = 0;
}
template <int WPL>
__device__ __forceinline__ bool bany(const Bits<WPL> &b) {
  uint32_t x = 0;
#pragma unroll
  for (int k = 0; k < WPL; k++) x |= b.w[k];
  return __any_sync(FULL, x != 0);
}
template <int WPL>
__device__ __forceinline__ int bcount(const Bits<WPL> &b) {
  int c = 0;
#pragma unroll
  for (int k = 0; k < WPL; k++) c += __popc(b.w[k]);
  return dev::warp_sum(c);
}
template <int WPL>
__device__ __forceinline__ int blowest(const Bits<WPL> &b) {
#pragma unroll
  for (int k = 0; k < WPL; k++) {
    unsigned m = __ballot_sync(FULL, b.w[k] != 0);
    if (m) {
      int l = __ffs(m) - 1;
      uint32_t x = __shfl_sync(FULL, b.w[k], l);
      return ((k * 32 + l) << 5) + __ffs(x) - 1;
    }
  }
  return -1;
}
template <int WPL>
__device__ __forceinline__ int bhighest(const Bits<WPL> &b) {
#pragma unroll
  for (int k = WPL - 1; k >= 0; k--) {
    unsigned m = __ballot_sync(FULL, b.w[k] != 0);
    if (m) {
      int l = 31 - __clz(m);
      uint32_t x = __shfl_sync(FULL, b.w[k], l);
      return ((k * 32 + l) << 5) + 31 - __clz(x);
    }
  }
  return -1;
}
template <int WPL>
__device__ __forceinline__ void bclear(Bits<WPL> &b, int v) {
  const int lane = threadIdx.x & 31, wi = v >> 5;
  const uint32_t m = ~(1u << (v & 31));
#pragma unroll
  for (int k = 0; k < WPL; k++)
    if ((wi >> 5) == k && (wi & 31) == lane) b.w[k] &= m;
}
template <int WPL>
__device__ __forceinline__ void bset(Bits<WPL> &b, int v) {
  const int lane = threadIdx.x & 31, wi = v >> 5;
  const uint32_t m = 1u << (v & 31);
#pragma unroll
  for (int k = 0; k < WPL; k++)
    if ((wi >> 5) == k && (wi & 31) == lane) b.w[k] |= m;
}
template <bool SM>
__device__ __forceinline__ uint32_t rw(const uint32_t *A, int64_t i) {
  if (SM) return A[i];
  return __ldcg(A + i);
}
// b &= row v  (words >= W are zero)
template <int WPL, bool SM>
__device__ __forceinline__ void band_row(Bits<WPL> &b, const uint32_t *A, int Ws, int W, int v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < WPL; k++) {
    int w = k * 32 + lane;
    b.w[k] = (w < W) ? (b.w[k] & rw<SM>(A, (int64_t)v * Ws + w)) : 0u;
  }
}
template <int WPL, bool SM>
__device__ __forceinline__ void bandnot_row(Bits<WPL> &b, const uint32_t *A, int Ws, int W, int v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < WPL; k++) {
    int w = k * 32 + lane;
    if (w < W) b.w[k] &= ~rw<SM>(A, (int64_t)v * Ws + w);
  }
}

// Greedy colouring of P in index order by independent-set extraction: colour
// class c takes, in index order, every remaining vertex with no neighbour
// already in class c.  (This is exactly the sequential greedy colouring.)
// B receives the vertices with colour > kmin.  Returns the colour count.
template <int WPL, bool SM>
__device__ int color_ise(const uint32_t *A, int Ws, int W, const Bits<WPL> &P, int kmin, Bits<WPL> &B) {
  Bits<WPL> U = P;
  bzero(B);
  int col = 0;
  while (bany(U)) {
    col++;
    Bits<WPL> Q = U;
    for (;;) {
      int v = blowest(Q);
      if (v < 0) break;
      bclear(Q, v);
      bclear(U, v);
      if (col > kmin) bset(B, v);
      bandnot_row<WPL, SM>(Q, A, Ws, W, v);
    }
  }
  return col;
}

__device__ __forceinline__ int read_best(const int32_t *best, int g) {
  int x = 0;
  if ((threadIdx.x & 31) == 0) x = *(const volatile int32_t *)(best + g);
  return __shfl_sync(FULL, x, 0);
}

__device__ __forceinline__ int hash_slot(int key, int mask) { return (int)(((unsigned)key * 2654435761u) >> 7) & mask; }

__device__ __forceinline__ int hash_find(const int *hk, const short *hv, int mask, int key) {
  int s = hash_slot(key, mask);
  for (;;) {
    int k = hk[s];
    if (k == key) return hv[s];
    if (k < 0) return -1;
    s = (s + 1) & mask;
  }
}

__device__ __forceinline__ void hash_insert(int *hk, short *hv, int mask, int key, int val) {
  int s = hash_slot(key, mask);
  for (;;) {
    int prev = atomicCAS(hk + s, -1, key);
    if (prev == -1 || prev == key) {
      hv[s] = (short)val;
      return;
    }
    s = (s + 1) & mask;
  }
}

// Index in P of a later-neighbour entry y, or -1 if y is not in P.
// Hash form: P's members in an open-addressing table.
struct HashLookup {
  const int *hk;
  const short *hv;
  int mask;
  __device__ __forceinline__ int operator()(int y) const { return hash_find(hk, hv, mask, y); }
};
// Bitmap form, for a root u whose later ranks (u, n') fit the block's
// bitmap: bit y - base marks a member of P, pre[w] counts the members in
// words before w, and P is sorted by decreasing id, so the member y has
// index p - 1 - (members below y).  Every entry a build reads is a later
// neighbour of a member, so y - base is never negative.
struct BitmapLookup {
  const uint32_t *bm;
  const uint16_t *pre;
  int base, p;
  __device__ __forceinline__ int operator()(int y) const {
    const int r = y - base;
    const uint32_t w = bm[r >> 5], bit = 1u << (r & 31);
    if (!(w & bit)) return -1;
    return p - 1 - ((int)pre[r >> 5] + __popc(w & (bit - 1u)));
  }
};
constexpr int kBitmapWords = 6144;  // later-rank window of the bitmap lookup: 196,608 ranks

// bitonic sort (descending) of a[0..npow2) in shared memory by `nthr`
// cooperating threads (thread index t); BLOCK selects the barrier.
template <bool BLOCK>
__device__ void bitonic_desc(int *a, int npow2, int t, int nthr) {
  for (int k = 2; k <= npow2; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = t; i < npow2; i += nthr) {
        int ixj = i ^ j;
        if (ixj > i) {
          int x = a[i], y = a[ixj];
          bool desc = (i & k) == 0;
          if (desc ? (x < y) : (x > y)) {
            a[i] = y;
            a[ixj] = x;
          }
        }
      }
      if (BLOCK) __syncthreads(); else __syncwarp();
    }
  }
}

// Write the clique {u} + C (+ v) in original ids.  All lanes.
template <int WPL>
__device__ void write_clique(int32_t *base, const Bits<WPL> &C, int v, const int32_t *Pidx, const int32_t *oold,
                             int u) {
  const int lane = threadIdx.x & 31;
  Bits<WPL> X = C;
  if (v >= 0) bset(X, v);
  int cnt = 0;
#pragma unroll
  for (int k = 0; k < WPL; k++) cnt += __popc(X.w[k]);
  int incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(FULL, incl, o);
    if (lane >= o) incl += y;
  }
  int pos = 1 + incl - cnt;
#pragma unroll
  for (int k = 0; k < WPL; k++) {
    uint32_t x = X.w[k];
    while (x) {
      int b = __ffs(x) - 1;
      x &= x - 1;
      int idx = ((k * 32 + lane) << 5) + b;
      base[pos++] = oold[Pidx[idx]];
    }
  }
  if (lane == 0) base[0] = oold[u];
}

// A word of a stack level that lane 0 wrote (omega at colouring, the chosen
// vertex), read back by lane 0 and broadcast: the other lanes did not write
// it and must not act on a copy of their own.
__device__ __forceinline__ int level_word(const uint32_t *p) {
  int x = 0;
  if ((threadIdx.x & 31) == 0) x = (int)*p;
  return __shfl_sync(FULL, x, 0);
}

// Shared-memory task pool of a block worker.
template <int WPL>
struct Pool {
  int lock, count, idle, beat;
  int spent;  // Branch nodes the block has expanded on this root or task
  int spill;  // 0 searching here, 2 record being written, 1 spilling, 3 no room
  int rec;    // record of the root's matrix in the arena, -1 none yet
  int csize[kPoolCap];
  uint32_t C[kPoolCap][32 * WPL];
  uint32_t P[kPoolCap][32 * WPL];
};

template <int WPL>
__device__ bool pool_lock(Pool<WPL> *pl, int32_t *err, long long spin) {
  long long it = 0;
  while (atomicCAS(&pl->lock, 0, 1) != 0) {
    if (++it > spin) {
      atomicExch(err, kDevTimeout);
      return false;
    }
    __nanosleep(32);
  }
  __threadfence_block();
  return true;
}
template <int WPL>
__device__ void pool_unlock(Pool<WPL> *pl) {
  __threadfence_block();
  atomicExch(&pl->lock, 0);
}

struct Root {
  int u, g;
  const int32_t *Pidx;
  int p;  // |P|: rows of the root's matrix
};

// Take k consecutive queue positions, all or none; returns the first or -1.
// The queue is a ring of task_cap slots: positions are taken only while
// fewer than task_cap are taken and not yet handed out.
__device__ int reserve_tasks(const SA &a, int k) {
  int cur = *(volatile int32_t *)a.ntasks;
  for (long long it = 0; it < a.spin; it++) {
    const int head = *(volatile int32_t *)a.task_next;
    if (cur - head + k > a.task_cap || cur > INT_MAX - k) return -1;
    const int prev = atomicCAS(a.ntasks, cur, cur + k);
    if (prev == cur) return cur;
    cur = prev;
  }
  return -1;
}

// True while the queue is short enough that splitting work pays.
__device__ __forceinline__ bool queue_short(const SA &a) {
  if (a.queue_gate <= 0) return true;
  const int tail = *(volatile int32_t *)a.ntasks, head = *(volatile int32_t *)a.task_next;
  return tail - head < a.queue_gate;
}

// Reserve arena room and a record for a root's matrix and P list.  Returns
// the record index (and the arena offset) or -1 without room.
__device__ int reserve_record(const SA &a, const Root &r, int Ws, long long *off_out) {
  const long long need = (long long)r.p * Ws + r.p;
  const long long off = (long long)atomicAdd(a.arena_used, (unsigned long long)need);
  if (off + need > a.arena_cap) return -1;
  const int rec = atomicAdd(a.nrec, 1);
  if (rec >= a.rec_cap) return -1;
  *off_out = off;
  return rec;
}

// Copy a root's matrix and P list to its arena room and write its record,
// over the 32 lanes of a warp.
__device__ void write_record(const SA &a, const Root &r, const uint32_t *A, int Ws, int W, int rec, long long off) {
  const int lane = threadIdx.x & 31;
  uint32_t *dm = a.arena + off;
  for (int i = lane; i < r.p * Ws; i += 32) dm[i] = A[i];
  int *dp = (int *)(dm + (int64_t)r.p * Ws);
  for (int i = lane; i < r.p; i += 32) dp[i] = r.Pidx[i];
  if (lane == 0) {
    RootRec rr;
    rr.u = r.u;
    rr.g = r.g;
    rr.p = r.p;
    rr.W = W;
    rr.Ws = Ws;
    rr.pad = 0;
    rr.off = off;
    a.recs[rec] = rr;
  }
  __syncwarp();
  __threadfence();
}

// Write the task at queue position t (clique size cs counting u, 0 =
// empty; clique bits C; candidates P) and mark its slot written.  Position
// t uses slot t mod task_cap in lap t / task_cap: the slot's word counts
// 2*lap when the previous lap's task has been read (its reader already
// holds it, since t was reserved after that position was handed out) and
// 2*lap+1 once this task is written.  Warp-collective.
__device__ void write_task(const SA &a, int t, int rec, int cs, const Bits<1> &C, const Bits<1> &P) {
  const int lane = threadIdx.x & 31;
  const int slot = t & (a.task_cap - 1);
  const int lap2 = 2 * (t / a.task_cap);
  if (lane == 0) {
    long long w = 0;
    while (*(volatile int32_t *)(a.ready + slot) != lap2) {
      if (++w > a.spin) {
        atomicExch(a.err, kDevTimeout);
        break;
      }
      __nanosleep(32);
    }
  }
  __syncwarp();
  __threadfence();
  uint32_t *tk = a.tasks + (int64_t)slot * kTaskWords;
  if (lane == 0) {
    tk[0] = (uint32_t)rec;
    tk[1] = (uint32_t)cs;
  }
  tk[2 + lane] = C.w[0];
  tk[34 + lane] = P.w[0];
  __syncwarp();
  __threadfence();
  if (lane == 0) atomicExch(a.ready + slot, lap2 + 1);
}

// The branch x of a node with clique Cl (csl vertices with u) and candidates
// Pl (x and its earlier siblings already removed) as task slot t; the task
// is empty when x's subproblem is decided at once (raising the incumbent if
// {u} + Cl + x is a larger maximal clique).
__device__ void emit_task(const SA &a, const Root &r, const uint32_t *A, int Ws, int W, int rec, int t,
                          const Bits<1> &Cl, int csl, const Bits<1> &Pl, int x) {
  Bits<1> TP = Pl;
  band_row<1, true>(TP, A, Ws, W, x);
  const int om = read_best(a.best, r.g);
  int cs = csl + 1;
  if (!bany(TP)) {
    if (csl + 1 > om) {
      const Bits<1> Cc = Cl;
      dev::raise_incumbent(a.best, a.lock, a.wit, a.voff, r.g, csl + 1, a.err, a.spin,
                           [&](int, int32_t *base) { write_clique<1>(base, Cc, x, r.Pidx, a.oold, r.u); });
    }
    cs = 0;
  } else if (csl + 1 + bcount(TP) <= om) {
    cs = 0;
  }
  Bits<1> Cx = Cl;
  bset(Cx, x);
  write_task(a, t, rec, cs, Cx, TP);
}

// Hand the untried rest of one warp's depth-first search to the task queue:
// every untried branch at each stored level and at the current level becomes
// a task of record rec.  All or nothing: returns false, publishing nothing,
// without room in the queue.
__device__ bool spill_levels(const SA &a, const Root &r, const uint32_t *A, int Ws, int W, const uint32_t *stk, int d,
                             int csize0, const Bits<1> &P, const Bits<1> &B, const Bits<1> &C, int rec) {
  const int lane = threadIdx.x & 31;
  const int stride = 64 + 2;
  int ntask = bcount(B);
  for (int l = 0; l < d; l++) {
    Bits<1> Bl;
    Bl.w[0] = stk[(int64_t)l * stride + 32 + lane];
    ntask += bcount(Bl);
  }
  if (ntask == 0) return true;
  int t = -1;
  if (lane == 0) t = reserve_tasks(a, ntask);
  t = __shfl_sync(FULL, t, 0);
  if (t < 0) return false;
  for (int l = 0; l <= d; l++) {
    Bits<1> Pl, Bl, Cl = C;
    if (l < d) {
      const uint32_t *q = stk + (int64_t)l * stride;
      Pl.w[0] = q[lane];
      Bl.w[0] = q[32 + lane];
      for (int m = l; m < d; m++) bclear(Cl, level_word(stk + (int64_t)m * stride + 65));
    } else {
      Pl = P;
      Bl = B;
    }
    for (;;) {
      const int x = bhighest(Bl);
      if (x < 0) break;
      bclear(Bl, x);
      bclear(Pl, x);
      emit_task(a, r, A, Ws, W, rec, t++, Cl, csize0 + l, Pl, x);
    }
  }
  return true;
}

// Spill state of a block worker past its node budget (warp-collective):
// the first warp to see the budget spent writes the root's record (unless
// the task already has one) and opens the spill; returns 1 when this warp
// should spill now, 3 when there is no room, 0 or 2 to keep searching.
__device__ int block_spill_state(const SA &a, const Root &r, const uint32_t *A, int Ws, int W, Pool<1> *pool,
                                 long long budget) {
  const int lane = threadIdx.x & 31;
  int s = 0;
  if (lane == 0) {
    s = *(volatile int *)&pool->spill;
    if (s == 0 && *(volatile int *)&pool->spent > budget && queue_short(a)) {
      if (atomicCAS(&pool->spill, 0, 2) == 0) s = 4;
      else s = *(volatile int *)&pool->spill;
    }
  }
  s = __shfl_sync(FULL, s, 0);
  if (s != 4) return s;
  int rec = __shfl_sync(FULL, lane == 0 ? *(volatile int *)&pool->rec : 0, 0);
  if (rec < 0) {
    long long off = 0;
    if (lane == 0) rec = reserve_record(a, r, Ws, &off);
    rec = __shfl_sync(FULL, rec, 0);
    off = __shfl_sync(FULL, off, 0);
    if (rec >= 0) write_record(a, r, A, Ws, W, rec, off);
  }
  s = rec >= 0 ? 1 : 3;
  if (lane == 0) {
    *(volatile int *)&pool->rec = rec;
    __threadfence_block();
    atomicExch(&pool->spill, s);
  }
  __syncwarp();
  return s;
}

// Depth-first Branch from one level (csize0 = |C| including the root u).
// Stack levels above the start hold (P, B, omega-at-colouring, chosen).
// If `pool` is not null, untried branches are handed to idle warps.
template <int WPL, bool SM>
__device__ void dfs(const SA &a, const Root &r, const uint32_t *A, int Ws, int W, uint32_t *stk, int csize0,
                    Bits<WPL> P, Bits<WPL> B, Bits<WPL> C, int wat, Pool<WPL> *pool, unsigned long long &nodes,
                    unsigned long long &donations, long long budget = 0) {
  const int lane = threadIdx.x & 31;
  const int stride = 64 * WPL + 2;
  int d = 0, csize = csize0;
  long long spent = 0;
  for (;;) {
    if (__shfl_sync(FULL, lane == 0 ? *(volatile int32_t *)a.err : 0, 0)) return;
    int om = read_best(a.best, r.g);
    if (om > wat) {
      color_ise<WPL, SM>(A, Ws, W, P, om - csize, B);
      wat = om;
    }
    if constexpr (WPL == 1 && SM) {
      // Past its node budget a worker hands the untried rest of its tree to
      // the task queue, where whole blocks search it.
      if (budget > 0 && !pool && spent > budget) {
        int rec = -1;
        long long off = 0;
        if (lane == 0) rec = reserve_record(a, r, Ws, &off);
        rec = __shfl_sync(FULL, rec, 0);
        off = __shfl_sync(FULL, off, 0);
        if (rec >= 0) {
          write_record(a, r, A, Ws, W, rec, off);
          if (spill_levels(a, r, A, Ws, W, stk, d, csize0, P, B, C, rec)) return;
        }
        budget = 0;
      } else if (budget > 0 && pool) {
        const int st = block_spill_state(a, r, A, Ws, W, pool, budget);
        if (st == 1) {
          int rec = lane == 0 ? *(volatile int *)&pool->rec : 0;
          rec = __shfl_sync(FULL, rec, 0);
          if (spill_levels(a, r, A, Ws, W, stk, d, csize0, P, B, C, rec)) return;
          budget = 0;
        } else if (st == 3) {
          budget = 0;
        }
      }
    }
    int v = bhighest(B);
    if (v < 0) {
      if (d == 0) return;
      d--;
      uint32_t *lv = stk + (int64_t)d * stride;
#pragma unroll
      for (int k = 0; k < WPL; k++) {
        P.w[k] = lv[k * 32 + lane];
        B.w[k] = lv[32 * WPL + k * 32 + lane];
      }
      wat = level_word(lv + 64 * WPL);
      const int ch = level_word(lv + 64 * WPL + 1);
      bclear(C, ch);
      csize--;
      continue;
    }
    bclear(B, v);
    bclear(P, v);
    Bits<WPL> NP = P;
    band_row<WPL, SM>(NP, A, Ws, W, v);
    nodes++;
    spent++;
    if (lane == 0) {
      if (pool && budget > 0) atomicAdd(&pool->spent, 1);
      if (a.progress && (spent & 255) == 0) atomicAdd(a.progress, 1);
    }
    if (!bany(NP)) {
      if (csize + 1 > om) {
        const Bits<WPL> Cc = C;
        dev::raise_incumbent(a.best, a.lock, a.wit, a.voff, r.g, csize + 1, a.err, a.spin,
                             [&](int, int32_t *base) { write_clique<WPL>(base, Cc, v, r.Pidx, a.oold, r.u); });
      }
      continue;
    }
    if (csize + 1 + bcount(NP) <= om) continue;
    Bits<WPL> NB;
    color_ise<WPL, SM>(A, Ws, W, NP, om - csize - 1, NB);
    if (!bany(NB)) continue;  // csize + 1 + L <= omega
    // descend: save this level
    uint32_t *lv = stk + (int64_t)d * stride;
#pragma unroll
    for (int k = 0; k < WPL; k++) {
      lv[k * 32 + lane] = P.w[k];
      lv[32 * WPL + k * 32 + lane] = B.w[k];
    }
    if (lane == 0) {
      lv[64 * WPL] = (uint32_t)wat;
      lv[64 * WPL + 1] = (uint32_t)v;
    }
    d++;
    bset(C, v);
    csize++;
    P = NP;
    B = NB;
    wat = om;

    // hand the shallowest untried branch to an idle warp of the block
    if (pool) {
      if (lane == 0) atomicAdd(&pool->beat, 1);  // progress signal for waiting warps
      int hungry = 0;
      if (lane == 0) {
        int idle = *(volatile int *)&pool->idle, cnt = *(volatile int *)&pool->count;
        hungry = idle > 0 && cnt < idle && cnt < kPoolCap;
      }
      hungry = __shfl_sync(FULL, hungry, 0);
      if (hungry) {
        __syncwarp();
        // shallowest stored level with an untried branch (levels 0..d-1 are in memory)
        int lev = -1;
        Bits<WPL> Bl, Pl;
        for (int l = 0; l < d; l++) {
          uint32_t *q = stk + (int64_t)l * stride;
#pragma unroll
          for (int k = 0; k < WPL; k++) Bl.w[k] = q[32 * WPL + k * 32 + lane];
          if (bany(Bl)) {
            lev = l;
            break;
          }
        }
        if (lev >= 0) {
          uint32_t *q = stk + (int64_t)lev * stride;
#pragma unroll
          for (int k = 0; k < WPL; k++) Pl.w[k] = q[k * 32 + lane];
          int x = bhighest(Bl);
          bclear(Bl, x);
          bclear(Pl, x);
#pragma unroll
          for (int k = 0; k < WPL; k++) {
            q[k * 32 + lane] = Pl.w[k];
            q[32 * WPL + k * 32 + lane] = Bl.w[k];
          }
          // clique at level lev: C minus the vertices chosen at levels >= lev
          Bits<WPL> Cl = C;
          for (int l = lev; l < d; l++) bclear(Cl, level_word(stk + (int64_t)l * stride + 64 * WPL + 1));
          bset(Cl, x);
          Bits<WPL> TP = Pl;
          band_row<WPL, SM>(TP, A, Ws, W, x);
          int tcs = csize0 + lev + 1;
          int om2 = read_best(a.best, r.g);
          if (bany(TP) && tcs + bcount(TP) > om2) {
            int ok = 0;
            if (lane == 0) {
              if (pool_lock(pool, a.err, a.spin)) {
                if (pool->count < kPoolCap) ok = 1 + pool->count++;
                else pool_unlock(pool);
              }
            }
            ok = __shfl_sync(FULL, ok, 0);
            if (ok) {
              int slot = ok - 1;
#pragma unroll
              for (int k = 0; k < WPL; k++) {
                pool->C[slot][k * 32 + lane] = Cl.w[k];
                pool->P[slot][k * 32 + lane] = TP.w[k];
              }
              // a *_sync exchange does not reconverge the warp: every lane's
              // words must be written before lane 0 releases the pool
              __syncwarp();
              if (lane == 0) {
                pool->csize[slot] = tcs;
                pool_unlock(pool);
              }
              donations++;
            } else {
              // pool full: search the branch here, later, by restoring it
              bset(Bl, x);
              bset(Pl, x);
#pragma unroll
              for (int k = 0; k < WPL; k++) {
                q[k * 32 + lane] = Pl.w[k];
                q[32 * WPL + k * 32 + lane] = Bl.w[k];
              }
            }
          } else if (!bany(TP) && tcs > om2) {
            // nothing left to add: {u} + Cl is maximal and beats the incumbent
            const Bits<WPL> Cc = Cl;
            dev::raise_incumbent(a.best, a.lock, a.wit, a.voff, r.g, tcs, a.err, a.spin,
                                 [&](int, int32_t *base) { write_clique<WPL>(base, Cc, -1, r.Pidx, a.oold, r.u); });
          }
        }
        __syncwarp();
      }
    }
  }
}

// Load P = {w in N+(u) : K(w) >= om} into Pidx (unsorted).  Cooperative over
// nthr threads; *cnt is a shared counter (pre-zeroed).  Reads rows as int4.
__device__ __forceinline__ void load_P(const SA &a, int u, int om, int *Pidx, int cap, int *cnt, int t, int nthr) {
  const int64_t e0 = a.orow[u], e1 = a.orow[u + 1];
  const int4 *row = reinterpret_cast<const int4 *>(a.ocol + e0);
  const int64_t nq = (e1 - e0) >> 2;
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  // whole warps step together (t - lane is the warp's first index), so the
  // members a warp finds take one shared atomic per ballot
  for (int64_t q0 = t - lane; q0 < nq; q0 += nthr) {
    const int64_t q = q0 + lane;
    int ys[4] = {-1, -1, -1, -1};
    if (q < nq) {
      const int4 y = __ldg(row + q);
      ys[0] = y.x;
      ys[1] = y.y;
      ys[2] = y.z;
      ys[3] = y.w;
    }
#pragma unroll
    for (int j = 0; j < 4; j++) {
      const bool keep = ys[j] >= 0 && __ldg(a.ocore + ys[j]) >= om;
      const unsigned m = __ballot_sync(FULL, keep);
      int base = 0;
      if (lane == 0 && m) base = atomicAdd(cnt, __popc(m));
      base = __shfl_sync(FULL, base, 0);
      if (keep) {
        const int p = base + __popc(m & lt);
        if (p < cap) Pidx[p] = ys[j];
      }
    }
  }
}

// Matrix rows of P: for each member x (index i), every later neighbour y of x
// that is in P (index j) sets bits (i, j) and (j, i).  The lanes of a warp
// form four groups of eight, each walking a different member's row, with two
// int4 loads per lane in flight, so a warp keeps eight rows' loads in the
// memory system instead of one.
template <class Lookup>
__device__ __forceinline__ void build_rows(const SA &a, const int *Pidx, int p, const Lookup &find, uint32_t *A, int Ws,
                                           int wid, int nw, unsigned long long *count, int *dyn = nullptr) {
  const int lane = threadIdx.x & 31;
  const int grp = lane >> 3, gl = lane & 7;
  unsigned long long scanned = 0;
  // groups of 4 rows: statically wid, wid + nw, ...; or, with a shared
  // counter (dyn, zero before the call), taken by each warp as it frees up,
  // so rows of uneven length do not leave warps waiting at the next barrier
  int i0 = wid * 4;
  if (dyn) {
    if (lane == 0) i0 = atomicAdd(dyn, 4);
    i0 = __shfl_sync(FULL, i0, 0);
  }
  for (; i0 < p;) {
    const int i = i0 + grp;
    int64_t e0 = 0, e1 = 0;
    if (i < p) {
      const int x = Pidx[i];
      e0 = a.orow[x];
      e1 = a.orow[x + 1];
    }
    const int4 *row = reinterpret_cast<const int4 *>(a.ocol + e0);
    const int nq = (int)((e1 - e0) >> 2);
    const int nqmax = max(max(__shfl_sync(FULL, nq, 0), __shfl_sync(FULL, nq, 8)),
                          max(__shfl_sync(FULL, nq, 16), __shfl_sync(FULL, nq, 24)));
    if (gl == 0) scanned += 4ull * (unsigned long long)nq;
    for (int q0 = gl; q0 < nqmax; q0 += 16) {
      int4 ys[2];
#pragma unroll
      for (int u = 0; u < 2; u++) {
        const int q = q0 + 8 * u;
        ys[u] = (q < nq) ? __ldg(row + q) : make_int4(-1, -1, -1, -1);
      }
#pragma unroll
      for (int u = 0; u < 2; u++) {
        const int yy[4] = {ys[u].x, ys[u].y, ys[u].z, ys[u].w};
#pragma unroll
        for (int j = 0; j < 4; j++) {
          if (yy[j] < 0) continue;
          int b = find(yy[j]);
          if (b >= 0) atomicOr(A + (int64_t)i * Ws + (b >> 5), 1u << (b & 31));
        }
      }
    }
    if (dyn) {
      if (lane == 0) i0 = atomicAdd(dyn, 4);
      i0 = __shfl_sync(FULL, i0, 0);
    } else {
      i0 += nw * 4;
    }
  }
  // row entries scanned (Fact 3's work), one atomic per warp
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) scanned += __shfl_xor_sync(FULL, scanned, o);
  if (lane == 0 && scanned) atomicAdd(count, scanned);
}

// 32 x 32 bit transpose across a warp: lane r holds row r (bit c = column
// c); returns row c of the transpose for lane c (bit r = row r's bit c).
// Five exchange stages swap ever smaller off-diagonal blocks: in the stage
// of width j, the lane with bit j clear trades its upper j-bit halves for its
// partner's lower ones.
__device__ __forceinline__ uint32_t transpose32(uint32_t x) {
  const int lane = threadIdx.x & 31;
  uint32_t m = 0x0000ffffu;
#pragma unroll
  for (int j = 16; j != 0; j >>= 1, m ^= (m << j)) {
    const uint32_t y = __shfl_xor_sync(FULL, x, j);
    x = (lane & j) ? (((y >> j) & m) | (x & ~m)) : ((x & m) | ((y & m) << j));
  }
  return x;
}

// Complete the adjacency matrix from its lower triangle.  build_rows sets
// bit (i, b) for every edge of G[P] with b < i (a later neighbour has a
// higher rank, hence a smaller index in P); the 32 x 32 tiles on and below
// the diagonal are transposed with warp ballots and OR-ed into their mirror
// tiles.  A tile's reads (lower words) and writes (upper words, or the same
// diagonal tile after all its rows were read) never overlap another tile's.
template <bool SM>
__device__ void symmetrize(uint32_t *A, int Ws, int W, int p, int wid, int nw) {
  const int lane = threadIdx.x & 31;
  const int tiles = W * (W + 1) / 2;
  for (int t = wid; t < tiles; t += nw) {
    // tile t = (I, J) with J <= I, row-major over the lower triangle
    int I = (int)((sqrtf(8.0f * t + 1.0f) - 1.0f) * 0.5f);
    while (I * (I + 1) / 2 > t) I--;
    while ((I + 1) * (I + 2) / 2 <= t) I++;
    const int J = t - I * (I + 1) / 2;
    const int r = 32 * I + lane;
    const uint32_t x = (r < p) ? rw<SM>(A, (int64_t)r * Ws + J) : 0u;
    const uint32_t col = transpose32(x);
    const int rt = 32 * J + lane;
    if (rt < p) {
      const int64_t at = (int64_t)rt * Ws + I;
      A[at] = (I == J) ? (x | col) : (rw<SM>(A, at) | col);
    }
  }
}

// ------------------------------------------------------------ warp class ---

struct WarpSmem {
  int Pidx[kWarpCap];
  int hk[2 * kWarpCap];
  short hv[2 * kWarpCap];
  uint32_t A[kWarpCap * 5];
  uint32_t al[4];
  int cnt;
};

__global__ void __launch_bounds__(kSW * 32) search_warp_kernel(SA a) {
  __shared__ WarpSmem sm[kSW];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  WarpSmem &S = sm[wib];
  const int64_t gw = (int64_t)blockIdx.x * kSW + wib;
  uint32_t *stk = a.stack + gw * a.stack_stride;
  unsigned long long colored = 0, branched = 0, nodes = 0, don = 0;
  const int hmask = 2 * kWarpCap - 1;
  const int64_t nroots = *a.nroots;
  for (;;) {
    __syncwarp();
    int idx = 0;
    if (lane == 0) idx = *(volatile int32_t *)a.err ? INT_MAX : atomicAdd(a.next, 1);
    idx = __shfl_sync(FULL, idx, 0);
    if (idx >= nroots) break;
    const int u = a.roots[idx];
    const int g = a.ogid ? a.ogid[u] : 0;
    int om = read_best(a.best, g);
    if (a.ocore[u] < om) continue;
    if (lane == 0) S.cnt = 0;
    for (int i = lane; i < 2 * kWarpCap; i += 32) S.hk[i] = -1;
    for (int i = lane; i < kWarpCap; i += 32) S.Pidx[i] = INT_MIN;
    __syncwarp();
    load_P(a, u, om, S.Pidx, kWarpCap, &S.cnt, lane, 32);
    __syncwarp();
    const int p = S.cnt;
    if (p > kWarpCap) {
      if (lane == 0) atomicExch(a.err, kDevCheck);
      break;
    }
    if (p < om || p == 0) continue;
    int np2 = 32;
    while (np2 < p) np2 <<= 1;
    bitonic_desc<false>(S.Pidx, np2, lane, 32);
    for (int i = lane; i < p; i += 32) hash_insert(S.hk, S.hv, hmask, S.Pidx[i], i);
    const int W = (p + 31) >> 5, Ws = W | 1;
    for (int i = lane; i < p * Ws; i += 32) S.A[i] = 0;
    __syncwarp();
    build_rows(a, S.Pidx, p, HashLookup{S.hk, S.hv, hmask}, S.A, Ws, 0, 1, a.counters + 4);
    __syncwarp();
    symmetrize<true>(S.A, Ws, W, p, 0, 1);
    __syncwarp();
    // alive set = all p vertices; (omega-1)-core of G[P]
    if (lane < 4) S.al[lane] = (lane < W) ? ((lane == W - 1 && (p & 31)) ? ((1u << (p & 31)) - 1u) : FULL) : 0u;
    __syncwarp();
    om = read_best(a.best, g);
    if (a.neigh_cores) {
      for (;;) {
        // lanes own rows k*32 + lane; row i's live bit is bit (i & 31) of word i >> 5
        uint32_t rm[4] = {0u, 0u, 0u, 0u};
#pragma unroll
        for (int k = 0; k < 4; k++) {
          if (k < W) {
            int i = k * 32 + lane;
            bool live = i < p && ((S.al[k] >> lane) & 1u);
            int deg = 0;
            if (live)
              for (int w = 0; w < W; w++) deg += __popc(S.A[i * Ws + w] & S.al[w]);
            rm[k] = __ballot_sync(FULL, live && deg < om - 1);
          }
        }
        __syncwarp();
        bool ch = (rm[0] | rm[1] | rm[2] | rm[3]) != 0;
        if (lane < 4) {
          uint32_t mine = lane == 0 ? rm[0] : lane == 1 ? rm[1] : lane == 2 ? rm[2] : rm[3];
          S.al[lane] &= ~mine;
        }
        __syncwarp();
        if (!ch) break;
      }
    }
    Bits<1> al;
    al.w[0] = (lane < 4) ? S.al[lane] : 0u;
    if (a.neigh_cores && bcount(al) < om) continue;
    colored++;
    Bits<1> B;
    color_ise<1, true>(S.A, Ws, W, al, om - 1, B);
    if (!bany(B)) continue;
    branched++;
    Bits<1> C;
    bzero(C);
    Root r{u, g, S.Pidx, p};
    dfs<1, true>(a, r, S.A, Ws, W, stk, 1, al, B, C, om, (Pool<1> *)nullptr, nodes, don,
                 a.tasks ? a.budget_warp : 0);
  }
  if (lane == 0) {
    atomicAdd(a.counters + 0, colored);
    atomicAdd(a.counters + 1, branched);
    atomicAdd(a.counters + 2, nodes);
  }
}

// ----------------------------------------------------------- block class ---

template <int WPL, bool SM, int PC = 1024 * WPL>
struct BlockLayout {
  static constexpr int PCAP = PC;
  static constexpr int HCAP = 4 * PCAP;  // load factor 1/4: short probes
  static constexpr int WMAX = 32 * WPL;                 // alive / removal words (one per lane)
  static constexpr int WSMAX = ((PCAP + 31) / 32) | 1;  // largest matrix row stride, W | 1
  // bytes: Pidx, hk, hv, alive/rm words, pool, control, matrix
  static constexpr size_t off_P = 0;
  static constexpr size_t off_hk = off_P + PCAP * 4;
  static constexpr size_t off_hv = off_hk + HCAP * 4;
  static constexpr size_t off_al = off_hv + HCAP * 2;
  static constexpr size_t off_rm = off_al + WMAX * 4;
  static constexpr size_t off_pool = off_rm + WMAX * 4;
  static constexpr size_t off_ctl = off_pool + ((sizeof(Pool<WPL>) + 15) / 16) * 16;
  static constexpr size_t off_bm = off_ctl + 64;                        // kBitmapWords words
  static constexpr size_t off_pre = off_bm + (size_t)kBitmapWords * 4;  // kBitmapWords uint16
  static constexpr size_t off_A = off_pre + (size_t)kBitmapWords * 2;
  static constexpr size_t bytes = off_A + (SM ? (size_t)PCAP * WSMAX * 4 : 0);
};

// The warps of a block search one root (or one task) together: warps that
// hold work run the depth-first Branch and hand untried branches to idle
// warps through the block's pool; the call returns when the pool is empty
// and every warp is idle.  All warps of the block call it.
template <int WPL, bool SM>
__device__ void block_search(const SA &a, const Root &r, const uint32_t *A, int Ws, int W, uint32_t *stk,
                             Pool<WPL> *pool, bool have, Bits<WPL> P, Bits<WPL> B, Bits<WPL> C, int cs, int wat,
                             unsigned long long &nodes, unsigned long long &don, long long budget) {
  const int lane = threadIdx.x & 31;
  const int g = r.g;
  long long waited = 0;
  int lastbeat = -1;
  for (;;) {
    if (have) {
      dfs<WPL, SM>(a, r, A, Ws, W, stk, cs, P, B, C, wat, pool, nodes, don, budget);
      have = false;
      if (lane == 0) {
        if (pool_lock(pool, a.err, a.spin)) {
          pool->idle++;
          pool_unlock(pool);
        }
      }
      __syncwarp();
    }
    int got = 0;
    if (lane == 0) {
      if (pool_lock(pool, a.err, a.spin)) {
        if (pool->count > 0) {
          got = pool->count--;
          pool->idle--;
        } else if (pool->idle == kBW) {
          got = -1;
        }
        if (got <= 0) pool_unlock(pool);
      } else {
        got = -1;
      }
    }
    got = __shfl_sync(FULL, got, 0);
    if (got < 0) break;
    if (got == 0) {
      int beat = *(volatile int *)&pool->beat;
      if (beat != lastbeat) {
        lastbeat = beat;
        waited = 0;
      }
      if (__shfl_sync(FULL, (++waited > a.spin || (lane == 0 && *(volatile int32_t *)a.err)) ? 1 : 0, 0)) {
        if (lane == 0) atomicExch(a.err, kDevTimeout);
        break;
      }
      __nanosleep(128);
      continue;
    }
    // copy the task while still holding the lock (lane 0 holds it)
    const int slot = got - 1;
#pragma unroll
    for (int k = 0; k < WPL; k++) {
      C.w[k] = pool->C[slot][k * 32 + lane];
      P.w[k] = pool->P[slot][k * 32 + lane];
    }
    cs = pool->csize[slot];
    __syncwarp();
    if (lane == 0) pool_unlock(pool);
    __syncwarp();
    if constexpr (WPL == 1 && SM) {
      // while the block spills, pooled subproblems go to the queue as tasks
      int sp = 0, rec = -1, t = -1;
      if (lane == 0 && budget > 0 && *(volatile int *)&pool->spill == 1) {
        sp = 1;
        rec = *(volatile int *)&pool->rec;
        t = reserve_tasks(a, 1);
      }
      sp = __shfl_sync(FULL, sp, 0);
      if (sp) {
        t = __shfl_sync(FULL, t, 0);
        rec = __shfl_sync(FULL, rec, 0);
        if (t >= 0) {
          write_task(a, t, rec, cs, C, P);
          if (lane == 0 && pool_lock(pool, a.err, a.spin)) {
            pool->idle++;
            pool_unlock(pool);
          }
          __syncwarp();
          continue;
        }
      }
    }
    int om2 = read_best(a.best, g);
    color_ise<WPL, SM>(A, Ws, W, P, om2 - cs, B);
    wat = om2;
    have = bany(B);
    if (!have && lane == 0) {
      if (pool_lock(pool, a.err, a.spin)) {
        pool->idle++;
        pool_unlock(pool);
      }
    }
    __syncwarp();
  }
}

// PC: candidate capacity of the shared-memory layout.  The kMidCap layout
// fits two blocks per SM; its roots with more candidates go to the overflow
// list, which the 1,024-candidate launch then searches.
template <int WPL, bool SM, int PC>
__global__ void __launch_bounds__(kBT, (SM && PC <= kMidCap) ? 2 : 1) search_block_kernel(SA a) {
  using L = BlockLayout<WPL, SM, PC>;
  extern __shared__ __align__(16) unsigned char smem[];
  int *Pidx = (int *)(smem + L::off_P);
  int *hk = (int *)(smem + L::off_hk);
  short *hv = (short *)(smem + L::off_hv);
  uint32_t *al = (uint32_t *)(smem + L::off_al);
  uint32_t *rm = (uint32_t *)(smem + L::off_rm);
  Pool<WPL> *pool = (Pool<WPL> *)(smem + L::off_pool);
  int *ctl = (int *)(smem + L::off_ctl);  // [0] root idx, [1] omega, [2] count, [3] flag, [4] go, [5] error
  uint32_t *A = SM ? (uint32_t *)(smem + L::off_A) : (a.gmat + (int64_t)blockIdx.x * a.gmat_stride);
  uint32_t *bm = (uint32_t *)(smem + L::off_bm);
  uint16_t *pre = (uint16_t *)(smem + L::off_pre);
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  uint32_t *stk = a.stack + ((int64_t)blockIdx.x * kBW + wid) * a.stack_stride;
  unsigned long long colored = 0, branched = 0, nodes = 0, don = 0;
  const int hmask = L::HCAP - 1;
  const int64_t nroots = *a.nroots;
  const int64_t npr = *a.np_count;
  for (int i = tid; i < kBitmapWords; i += kBT) bm[i] = 0u;  // each root clears the bits it set

  for (;;) {
    __syncthreads();
    if (tid == 0) {
      ctl[0] = atomicAdd(a.next, 1);
      ctl[2] = 0;
      ctl[5] = *(volatile int32_t *)a.err;
      ctl[6] = 0;  // the row builder's group counter
    }
    __syncthreads();
    const int idx = ctl[0];
    if (idx >= nroots || ctl[5]) break;
    const int u = a.roots[idx];
    const int g = a.ogid ? a.ogid[u] : 0;
    if (tid == 0) ctl[1] = *(volatile int32_t *)(a.best + g);
    __syncthreads();
    int om = ctl[1];
    if (a.ocore[u] < om) continue;
    // the later ranks (u, n') fit the bitmap: member lookups by bitmap,
    // otherwise by hash table
    const int base = u + 1;
    const bool use_bm = a.use_bitmap && ((npr - base + 31) >> 5) <= kBitmapWords;
    if (!use_bm)
      for (int i = tid; i < L::HCAP; i += kBT) hk[i] = -1;
    for (int i = tid; i < L::PCAP; i += kBT) Pidx[i] = INT_MIN;
    __syncthreads();
    load_P(a, u, om, Pidx, L::PCAP, &ctl[2], tid, kBT);
    __syncthreads();
    const int p = ctl[2];
    if (p > L::PCAP) {
      if (a.overflow) {
        if (tid == 0) a.overflow[atomicAdd((unsigned long long *)a.noverflow, 1ull)] = u;
        continue;
      }
      if (tid == 0) atomicExch(a.err, kDevUnsupported);
      break;
    }
    if (p < om || p == 0) continue;
    const int wwin = (int)((npr - base + 31) >> 5);
    if (use_bm) {
      // P in any order: its bits, the prefix counts, and then every member
      // moves to its index in decreasing-rank order, which the counts give
      // (the hash table's space, unused on this path, holds the list)
      int *tmp = hk;
      for (int i = tid; i < p; i += kBT) {
        const int y = Pidx[i];
        atomicOr(&bm[(y - base) >> 5], 1u << ((y - base) & 31));
        tmp[i] = y;
      }
      __syncthreads();
      // pre[w] = members in words [0, w): each thread counts a contiguous
      // chunk of words, the warps' totals are scanned in rm[], then each
      // thread writes its chunk's prefixes
      const int per = (wwin + kBT - 1) / kBT;
      const int w0 = min(wwin, tid * per), w1 = min(wwin, w0 + per);
      int mine = 0;
      for (int w = w0; w < w1; w++) mine += __popc(bm[w]);
      int incl = mine;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += y;
      }
      if (lane == 31) rm[wid] = (uint32_t)incl;
      __syncthreads();
      int before = 0;
      for (int w = 0; w < wid; w++) before += (int)rm[w];
      int run = before + incl - mine;
      for (int w = w0; w < w1; w++) {
        pre[w] = (uint16_t)run;
        run += __popc(bm[w]);
      }
      __syncthreads();
      const BitmapLookup at{bm, pre, base, p};
      for (int i = tid; i < p; i += kBT) Pidx[at(tmp[i])] = tmp[i];
    } else {
      int np2 = 32;
      while (np2 < p) np2 <<= 1;
      bitonic_desc<true>(Pidx, np2, tid, kBT);
      for (int i = tid; i < p; i += kBT) hash_insert(hk, hv, hmask, Pidx[i], i);
    }
    const int W = (p + 31) >> 5, Ws = W | 1;
    for (int64_t i = tid; i < (int64_t)p * Ws; i += kBT) A[i] = 0;
    if (!SM) __threadfence();
    __syncthreads();
    if (use_bm)
      build_rows(a, Pidx, p, BitmapLookup{bm, pre, base, p}, A, Ws, wid, kBW, a.counters + 5, &ctl[6]);
    else
      build_rows(a, Pidx, p, HashLookup{hk, hv, hmask}, A, Ws, wid, kBW, a.counters + 5, &ctl[6]);
    if (!SM) __threadfence();
    __syncthreads();
    if (use_bm)
      for (int i = tid; i < p; i += kBT) {
        const int r = Pidx[i] - base;
        atomicAnd(&bm[r >> 5], ~(1u << (r & 31)));
      }
    symmetrize<SM>(A, Ws, W, p, wid, kBW);
    if (!SM) __threadfence();
    __syncthreads();
    for (int w = tid; w < L::WMAX; w += kBT)
      al[w] = (w < W) ? ((w == W - 1 && (p & 31)) ? ((1u << (p & 31)) - 1u) : FULL) : 0u;
    if (tid == 0) ctl[1] = *(volatile int32_t *)(a.best + g);
    __syncthreads();
    om = ctl[1];
    if (a.neigh_cores) {
      // (omega-1)-core of G[P]: drop rows with fewer than omega-1 live neighbours
      for (;;) {
        for (int k = wid; k < W; k += kBW) {
          int i = k * 32 + lane;
          int deg = 0;
          bool live = i < p && ((al[k] >> lane) & 1u);
          if (live)
            for (int w = 0; w < W; w++) deg += __popc(rw<SM>(A, (int64_t)i * Ws + w) & al[w]);
          unsigned m = __ballot_sync(FULL, live && deg < om - 1);
          if (lane == 0) rm[k] = m;
        }
        if (tid == 0) ctl[3] = 0;
        __syncthreads();
        for (int k = tid; k < W; k += kBT)
          if (rm[k]) {
            al[k] &= ~rm[k];
            ctl[3] = 1;
          }
        __syncthreads();
        if (!ctl[3]) break;
        __syncthreads();
      }
    }
    // colouring test and the search, started by warp 0
    Root r{u, g, Pidx, p};
    Bits<WPL> P, B, C;
    bzero(C);
    int cs = 1, wat = om;
    bool have = false;
    if (wid == 0) {
#pragma unroll
      for (int k = 0; k < WPL; k++) P.w[k] = al[k * 32 + lane];
      int go = 0;
      if (!a.neigh_cores || bcount(P) >= om) {
        colored++;
        color_ise<WPL, SM>(A, Ws, W, P, om - 1, B);
        go = bany(B) ? 1 : 0;
        if (go) branched++;
      }
      have = go != 0;
      if (lane == 0) {
        ctl[4] = go;
        pool->lock = 0;
        pool->count = 0;
        pool->idle = kBW - 1;
        pool->beat = 0;
        pool->spent = 0;
        pool->spill = 0;
        pool->rec = -1;
      }
    }
    __syncthreads();
    if (!ctl[4]) continue;
    block_search<WPL, SM>(a, r, A, Ws, W, stk, pool, have, P, B, C, cs, wat, nodes, don,
                          (SM && WPL == 1 && a.tasks) ? a.budget_block : 0);
    __syncthreads();
  }
  if (lane == 0) {
    atomicAdd(a.counters + 0, colored);
    atomicAdd(a.counters + 1, branched);
    atomicAdd(a.counters + 2, nodes);
    atomicAdd(a.counters + 3, don);
  }
}


// The task queue: tasks of spilled roots, searched by whole blocks.  A block
// takes the next task, loads its root's matrix and P list into shared
// memory when the root changes, and searches it like a block worker; past
// its node budget, while the queue is short, it spills again.  The kernel
// ends when the queue is empty and no block holds a task (a block counts
// itself in `active` before it looks for a task and leaves it only after
// its spilled tasks are visible).
template <int PC>
__global__ void __launch_bounds__(kBT, (PC <= kMidCap) ? 2 : 1) branch_task_kernel(SA a) {
  using L = BlockLayout<1, true, PC>;  // PC >= every record's p
  extern __shared__ __align__(16) unsigned char smem[];
  int *Pidx = (int *)(smem + L::off_P);
  Pool<1> *pool = (Pool<1> *)(smem + L::off_pool);
  int *ctl = (int *)(smem + L::off_ctl);
  uint32_t *A = (uint32_t *)(smem + L::off_A);
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  uint32_t *stk = a.stack + ((int64_t)blockIdx.x * kBW + wid) * a.stack_stride;
  unsigned long long nodes = 0, don = 0;
  int loaded = -1;
  for (;;) {
    __syncthreads();
    Bits<1> C, P;
    bzero(C);
    bzero(P);
    if (wid == 0) {
      int got = -1;
      if (lane == 0) {
        long long waited = 0;
        int last = -1;
        atomicAdd(a.active, 1);
        __threadfence();
        for (;;) {
          if (*(volatile int32_t *)a.err) break;
          const int tail = *(volatile int32_t *)a.ntasks, head = *(volatile int32_t *)a.task_next;
          if (head < tail) {
            if (atomicCAS(a.task_next, head, head + 1) == head) {
              got = head;
              break;
            }
            continue;
          }
          // nothing queued: stand down and wait for work or for the end (no
          // block holds a task and the queue is empty)
          atomicSub(a.active, 1);
          __threadfence();
          bool done = false, work = false;
          while (!done && !work) {
            if (*(volatile int32_t *)a.err) {
              done = true;
              break;
            }
            const int act = *(volatile int32_t *)a.active;
            __threadfence();
            const int tail2 = *(volatile int32_t *)a.ntasks, head2 = *(volatile int32_t *)a.task_next;
            if (head2 < tail2) {
              work = true;
            } else if (act == 0) {
              done = true;
            } else {
              const int prog = *(volatile int32_t *)a.progress + tail2;
              if (prog != last) {
                last = prog;
                waited = 0;
              }
              if (++waited > a.spin) {
                atomicExch(a.err, kDevTimeout);
                done = true;
              }
              __nanosleep(512);
            }
          }
          if (done) break;
          atomicAdd(a.active, 1);
          __threadfence();
        }
        if (got >= 0) {
          // the slot's words are written before its word reads 2*lap+1
          const int slot = got & (a.task_cap - 1);
          const int lap2 = 2 * (got / a.task_cap);
          long long w = 0;
          while (*(volatile int32_t *)(a.ready + slot) != lap2 + 1) {
            if (++w > a.spin) {
              atomicExch(a.err, kDevTimeout);
              break;
            }
            __nanosleep(64);
          }
          __threadfence();
        }
      }
      got = __shfl_sync(FULL, got, 0);
      if (got >= 0) {
        const uint32_t *tk = a.tasks + (int64_t)(got & (a.task_cap - 1)) * kTaskWords;
        C.w[0] = __ldcg(tk + 2 + lane);
        P.w[0] = __ldcg(tk + 34 + lane);
        const int cs1 = (int)__ldcg(tk + 1), rec1 = (int)__ldcg(tk + 0);
        __syncwarp();
        if (lane == 0) {
          __threadfence();
          // free the slot for the next lap's writer
          atomicExch(a.ready + (got & (a.task_cap - 1)), 2 * (got / a.task_cap) + 2);
          ctl[1] = cs1;
          ctl[2] = rec1;
        }
      }
      if (lane == 0) {
        ctl[0] = got;
        ctl[3] = *(volatile int32_t *)a.err;
      }
    }
    __syncthreads();
    const int t = ctl[0];
    if (t < 0) break;
    const int cs0 = ctl[1], rec = ctl[2];
    if (cs0 == 0 || ctl[3]) {  // empty task (or giving up)
      __syncthreads();
      if (tid == 0) {
        __threadfence();
        atomicSub(a.active, 1);
      }
      continue;
    }
    RootRec rr;
    {
      const int *rp = (const int *)(a.recs + rec);
      rr.u = __ldcg(rp + 0);
      rr.g = __ldcg(rp + 1);
      rr.p = __ldcg(rp + 2);
      rr.W = __ldcg(rp + 3);
      rr.Ws = __ldcg(rp + 4);
      rr.off = __ldcg((const long long *)(rp + 6));
    }
    if (rec != loaded) {
      const uint32_t *sm = a.arena + rr.off;
      for (int i = tid; i < rr.p * rr.Ws; i += kBT) A[i] = __ldcg(sm + i);
      const int *sp = (const int *)(sm + (int64_t)rr.p * rr.Ws);
      for (int i = tid; i < rr.p; i += kBT) Pidx[i] = __ldcg(sp + i);
      loaded = rec;
    }
    __syncthreads();
    Root r{rr.u, rr.g, Pidx, rr.p};
    Bits<1> B;
    bzero(B);
    int cs = cs0, wat = 0;
    bool have = false;
    if (wid == 0) {
      wat = read_best(a.best, rr.g);
      color_ise<1, true>(A, rr.Ws, rr.W, P, wat - cs, B);
      have = bany(B);
      if (lane == 0) {
        ctl[4] = have ? 1 : 0;
        pool->lock = 0;
        pool->count = 0;
        pool->idle = kBW - 1;
        pool->beat = 0;
        pool->spent = 0;
        pool->spill = 0;
        pool->rec = rec;
      }
    }
    __syncthreads();
    if (ctl[4]) block_search<1, true>(a, r, A, rr.Ws, rr.W, stk, pool, have, P, B, C, cs, wat, nodes, don,
                                      a.budget_block);
    __syncthreads();
    if (tid == 0) {
      __threadfence();
      atomicSub(a.active, 1);
    }
  }
  if (lane == 0) {
    atomicAdd(a.counters + 2, nodes);
    atomicAdd(a.counters + 3, don);
  }
}

}  // namespace

int launch_search(mc_graph *g, const Pruned &pg, int no_neigh_cores, int no_split, int split_nodes,
                  long long spin_limit, SearchCounters *cnt, int layout, int no_bitmap) {
  // Persistent kernels with fixed grids; the root counts are read on the
  // device (pg.d_counts), and sizes are bounded by K(G) >= |N+(u)|, so the
  // launches need no host synchronisation.
  void *p;
  MC_TRY(ws_get(g, "se.ctr", 16 * sizeof(unsigned long long), &p));
  // [0..5] colored, branched, nodes, donations, row entries read by warp
  // workers, by block workers; [8..9] four root queue heads; [10] arena
  // words used; [11..13] records, task tail, task head, blocks holding a
  // task, heartbeat; [14] roots left to the 1,024-candidate launch
  unsigned long long *ctr = (unsigned long long *)p;
  int32_t *next = (int32_t *)(ctr + 8);
  MC_CUDA_TRY(cudaMemsetAsync(ctr, 0, 16 * sizeof(unsigned long long), g->stream));
  SA a{};
  a.np_count = pg.d_counts;
  a.use_bitmap = no_bitmap ? 0 : 1;
  a.orow = pg.orow;
  a.ocol = pg.ocol;
  a.ocore = pg.ocore;
  a.oold = pg.oold;
  a.ogid = pg.ogid;
  a.best = g->best;
  a.lock = g->lock;
  a.wit = g->wit;
  a.voff = g->gid ? g->voff : nullptr;
  a.err = g->err;
  a.spin = spin_limit;
  a.neigh_cores = no_neigh_cores ? 0 : 1;
  a.counters = ctr;
  // |P| <= |N+(u)| <= K(u) <= K(G); roots above kBigCap are not in any of
  // the lists launched here (single graphs solve them as induced subgraphs;
  // a batch with such a graph is refused before anything is launched)
  if (g->count > 1 && g->max_core > kBigCap) return MC_ERR_UNSUPPORTED;
  const int kbound = std::min(std::max(g->max_core, 1), kBigCap);
  const int wmax = g->warp_max_used;
  if (!no_split) {
    // queue sizes grow with the graph (a small graph gets a small queue; a
    // full queue only stops further spills)
    const long long arena_words = std::min<long long>(kArenaWords, std::max<long long>(1ll << 18, 4 * g->nnz));
    const int rec_cap = (int)std::min<int64_t>(kRecCap, std::max<int64_t>(1024, g->n));
    int task_cap = 1 << 12;
    while (task_cap < kTaskCap && (int64_t)task_cap < 4 * g->n) task_cap <<= 1;
    MC_TRY(ws_get(g, "se.arena", (size_t)arena_words * 4, &p));
    a.arena = (uint32_t *)p;
    a.arena_cap = arena_words;
    a.arena_used = ctr + 10;
    MC_TRY(ws_get(g, "se.recs", (size_t)rec_cap * sizeof(RootRec), &p));
    a.recs = (RootRec *)p;
    a.rec_cap = rec_cap;
    a.nrec = (int32_t *)(ctr + 11);
    MC_TRY(ws_get(g, "se.tasks", (size_t)task_cap * kTaskWords * 4, &p));
    a.tasks = (uint32_t *)p;
    MC_TRY(ws_get(g, "se.ready", (size_t)task_cap * 4, &p));
    a.ready = (int32_t *)p;
    MC_CUDA_TRY(cudaMemsetAsync(a.ready, 0, (size_t)task_cap * 4, g->stream));
    a.task_cap = task_cap;
    a.ntasks = a.nrec + 1;
    a.task_next = a.nrec + 2;
    a.active = a.nrec + 3;
    a.progress = a.nrec + 4;
    a.queue_gate = 0;
    a.budget_warp = split_nodes > 0 ? split_nodes : kSpillNodes;
    a.budget_block = 4 * a.budget_warp;
  }
  // Block workers (shared-memory matrices): a 512-candidate launch first,
  // then a 1,024-candidate launch over the roots it could not hold; the task
  // kernel shares the large layout and its stack buffer.
  using LB = BlockLayout<1, true>;
  using LM = BlockLayout<1, true, kMidCap>;
  const size_t smem_b = LB::bytes, smem_m = LM::bytes;
  MC_CUDA_TRY(cudaFuncSetAttribute(search_block_kernel<1, true, 1024>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)smem_b));
  MC_CUDA_TRY(cudaFuncSetAttribute(search_block_kernel<1, true, kMidCap>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)smem_m));
  MC_CUDA_TRY(cudaFuncSetAttribute(branch_task_kernel<1024>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_b));
  MC_CUDA_TRY(cudaFuncSetAttribute(branch_task_kernel<kMidCap>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)smem_m));
  int per_sm_b = 0, per_sm_t = 0, per_sm_m = 0, per_sm_tm = 0;
  MC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_b, search_block_kernel<1, true, 1024>, kBT, smem_b));
  MC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_t, branch_task_kernel<1024>, kBT, smem_b));
  MC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_tm, branch_task_kernel<kMidCap>, kBT, smem_m));
  MC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_m, search_block_kernel<1, true, kMidCap>, kBT,
                                                            smem_m));
  per_sm_b = std::min(per_sm_b, per_sm_t);
  if (per_sm_b < 1 || per_sm_m < 1 || per_sm_tm < 1) return MC_ERR_CUDA;
  // grids (and the stacks sized by them) shrink for small graphs: a block
  // per 64 vertices at most, a warp per four vertices in the warp class
  const int64_t small_cap = std::max<int64_t>(1, (g->n + 63) / 64);
  const int blocks_b = (int)std::min<int64_t>((int64_t)g->sm_count * per_sm_b, small_cap);
  const int blocks_m = (int)std::min<int64_t>((int64_t)g->sm_count * per_sm_m, small_cap);
  // the task kernel takes the mid layout (two blocks per SM) when no record
  // can hold more than kMidCap candidates (p <= K(G))
  const bool task_mid = kbound <= kMidCap;
  const int blocks_t =
      task_mid ? (int)std::min<int64_t>((int64_t)g->sm_count * per_sm_tm, small_cap) : blocks_b;
  const int64_t stride_b = (int64_t)(std::min(kbound, 1024) + 2) * (64 + 2);
  const int64_t stride_m = (int64_t)(std::min(kbound, kMidCap) + 2) * (64 + 2);
  uint32_t *stk_b = nullptr;
  if (kbound > wmax || !no_split) {
    MC_TRY(ws_get(g, "se.stk_b", (size_t)std::max(blocks_b, blocks_t) * kBW * stride_b * 4, &p));
    stk_b = (uint32_t *)p;
  }

  // block class first (largest trees), then big, then warp class, then the
  // tasks the first and last of these published; events 8-12 time each
  MC_TRY(record_event(g, 8));
  if (kbound > wmax) {
    a.gmat = nullptr;
    a.roots = pg.roots_block;
    a.nroots = pg.d_counts + 4;
    a.next = next + 0;
    const bool wide_only = layout == 1 && kbound > kMidCap;
    if (wide_only) {
      // every block-class root in the 1,024-candidate layout
      a.stack = stk_b;
      a.stack_stride = stride_b;
      search_block_kernel<1, true, 1024><<<blocks_b, kBT, smem_b, g->stream>>>(a);
      g_launches++;
      MC_CUDA_TRY(cudaGetLastError());
    } else {
      if (kbound > kMidCap) {
        MC_TRY(ws_get(g, "se.ovf", (size_t)std::max<int64_t>(g->n, 1) * 4, &p));
        a.overflow = (int32_t *)p;
        a.noverflow = (int64_t *)(ctr + 14);
      }
      MC_TRY(ws_get(g, "se.stk_m", (size_t)blocks_m * kBW * stride_m * 4, &p));
      a.stack = (uint32_t *)p;
      a.stack_stride = stride_m;
      search_block_kernel<1, true, kMidCap><<<blocks_m, kBT, smem_m, g->stream>>>(a);
      g_launches++;
      MC_CUDA_TRY(cudaGetLastError());
      if (kbound > kMidCap) {
        a.roots = a.overflow;
        a.nroots = a.noverflow;
        a.next = next + 3;
        a.overflow = nullptr;
        a.noverflow = nullptr;
        a.stack = stk_b;
        a.stack_stride = stride_b;
        search_block_kernel<1, true, 1024><<<blocks_b, kBT, smem_b, g->stream>>>(a);
        g_launches++;
        MC_CUDA_TRY(cudaGetLastError());
      }
    }
  }
  MC_TRY(record_event(g, 9));
  if (kbound > 1024) {
    using L = BlockLayout<4, false>;
    const size_t smem = L::bytes;
    MC_CUDA_TRY(cudaFuncSetAttribute(search_block_kernel<4, false, 4096>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
    const int blocks = g->sm_count;
    const int pmax = kbound;
    a.stack_stride = (int64_t)(pmax + 2) * (64 * 4 + 2);
    MC_TRY(ws_get(g, "se.stk_g", (size_t)blocks * kBW * a.stack_stride * 4, &p));
    a.stack = (uint32_t *)p;
    const int Wm = (pmax + 31) / 32;
    a.gmat_stride = (int64_t)pmax * (Wm | 1) + 64;
    MC_TRY(ws_get(g, "se.gmat", (size_t)blocks * a.gmat_stride * 4, &p));
    a.gmat = (uint32_t *)p;
    a.roots = pg.roots_big;
    a.nroots = pg.d_counts + 5;
    a.next = next + 1;
    search_block_kernel<4, false, 4096><<<blocks, kBT, smem, g->stream>>>(a);
    g_launches++;
    MC_CUDA_TRY(cudaGetLastError());
  }
  MC_TRY(record_event(g, 10));
  {
    int per_sm = 0;
    MC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, search_warp_kernel, kSW * 32, 0));
    if (per_sm < 1) return MC_ERR_CUDA;
    const int blocks = (int)std::min<int64_t>((int64_t)g->sm_count * per_sm,
                                              std::max<int64_t>(1, (g->n + 4 * kSW - 1) / (4 * kSW)));
    const int pmax = std::min(kbound, kWarpCap);
    a.stack_stride = (int64_t)(pmax + 2) * (64 + 2);
    MC_TRY(ws_get(g, "se.stk_w", (size_t)blocks * kSW * a.stack_stride * 4, &p));
    a.stack = (uint32_t *)p;
    a.roots = pg.roots_small;
    a.nroots = pg.d_counts + 3;
    a.next = next + 2;
    search_warp_kernel<<<blocks, kSW * 32, 0, g->stream>>>(a);
    g_launches++;
    MC_CUDA_TRY(cudaGetLastError());
  }
  MC_TRY(record_event(g, 11));
  if (!no_split) {
    a.stack_stride = stride_b;
    a.stack = stk_b;
    a.queue_gate = 2 * blocks_t;
    if (task_mid)
      branch_task_kernel<kMidCap><<<blocks_t, kBT, smem_m, g->stream>>>(a);
    else
      branch_task_kernel<1024><<<blocks_t, kBT, smem_b, g->stream>>>(a);
    g_launches++;
    MC_CUDA_TRY(cudaGetLastError());
  }
  MC_TRY(record_event(g, 12));
  cnt->d_counters = ctr;
  return MC_OK;
}

int read_search_counters(mc_graph *g, SearchCounters *cnt) {
  unsigned long long *h = (unsigned long long *)g->h_small;
  MC_CUDA_TRY(cudaMemcpyAsync(h, cnt->d_counters, 13 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, g->stream));
  MC_CUDA_TRY(cudaStreamSynchronize(g->stream));
  cnt->roots_colored = h[0];
  cnt->roots_branched = h[1];
  cnt->nodes = h[2];
  cnt->donations = h[3];
  cnt->entries = h[4] + h[5];
  cnt->entries_block = h[5];
  cnt->tasks = (unsigned long long)((const int32_t *)(h + 11))[1];
  return MC_OK;
}

}  // namespace mc
