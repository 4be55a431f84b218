// Stable LSD radix sort of (uint32 key, int32 value) pairs, descending by
// key: four passes of 8-bit digits; equal keys keep their input order.
//
// Each pass: a block histogram of its 2,048-item tile (digit-major table
// digit * blocks + block), an exclusive scan of that table (every digit's
// items of earlier blocks, and of larger digits, come first), and a stable
// scatter -- each warp owns 256 consecutive items of the tile, warp offsets
// come from a per-warp digit count, and within a warp the items are ranked
// 32 at a time in order (lanes of equal digit found by __match_any_sync).
// The values must be distinct indices in [0, n): the result is checked.
#include <algorithm>

#include "mc_internal.cuh"
#include "scan.cuh"

namespace mc {

namespace {

constexpr int kRT = 256;
constexpr int kRW = kRT / 32;
constexpr int kRItems = 8;               // chunks of 32 items per warp
constexpr int kRTile = kRT * kRItems;    // items per block
constexpr int kRWarpItems = 32 * kRItems;

__device__ __forceinline__ int digit_desc(uint32_t k, int shift) { return 255 - (int)((k >> shift) & 255u); }

__global__ void __launch_bounds__(kRT) radix_hist_kernel(int64_t n, const uint32_t *__restrict__ keys, int shift,
                                                         int64_t nblocks, int64_t *__restrict__ hist) {
  __shared__ int cnt[256];
  for (int i = threadIdx.x; i < 256; i += kRT) cnt[i] = 0;
  __syncthreads();
  const int64_t base = blockIdx.x * (int64_t)kRTile;
  for (int j = 0; j < kRItems; j++) {
    const int64_t i = base + (int64_t)j * kRT + threadIdx.x;
    if (i < n) atomicAdd(&cnt[digit_desc(keys[i], shift)], 1);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < 256; d += kRT) hist[(int64_t)d * nblocks + blockIdx.x] = cnt[d];
}

__global__ void __launch_bounds__(kRT) radix_scatter_kernel(int64_t n, const uint32_t *__restrict__ kin,
                                                            const int32_t *__restrict__ vin, uint32_t *__restrict__ kout,
                                                            int32_t *__restrict__ vout, int shift, int64_t nblocks,
                                                            const int64_t *__restrict__ off) {
  __shared__ int wcnt[kRW][256];
  __shared__ int64_t boff[256];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  for (int i = threadIdx.x; i < kRW * 256; i += kRT) (&wcnt[0][0])[i] = 0;
  for (int d = threadIdx.x; d < 256; d += kRT) boff[d] = off[(int64_t)d * nblocks + blockIdx.x];
  __syncthreads();
  const int64_t wbase = blockIdx.x * (int64_t)kRTile + (int64_t)w * kRWarpItems;
  // per-warp digit counts
  for (int c = 0; c < kRItems; c++) {
    const int64_t i = wbase + c * 32 + lane;
    if (i < n) atomicAdd(&wcnt[w][digit_desc(kin[i], shift)], 1);
  }
  __syncthreads();
  // exclusive scan over the warps, per digit (in place)
  for (int d = threadIdx.x; d < 256; d += kRT) {
    int run = 0;
    for (int x = 0; x < kRW; x++) {
      const int c = wcnt[x][d];
      wcnt[x][d] = run;
      run += c;
    }
  }
  __syncthreads();
  // rank 32 items at a time, in order; wcnt[w][d] is the next slot of digit
  // d for this warp
  for (int c = 0; c < kRItems; c++) {
    const int64_t i = wbase + c * 32 + lane;
    const bool ok = i < n;
    const uint32_t k = ok ? kin[i] : 0u;
    const int d = ok ? digit_desc(k, shift) : 256;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const int r = __popc(peers & lt);
    int64_t pos = 0;
    if (ok) pos = boff[d] + wcnt[w][d] + r;
    __syncwarp();
    if (ok && r == 0) wcnt[w][d] += __popc(peers);
    __syncwarp();
    if (ok) {
      kout[pos] = k;
      vout[pos] = vin[i];
    }
  }
}

// The result is checked: keys non-increasing, values a permutation of
// [0, n) (the callers sort indices); a failure sets the device error word.
__global__ void sort_check_kernel(int64_t n, const uint32_t *__restrict__ keys, const int32_t *__restrict__ vals,
                                  int32_t *__restrict__ seen, int32_t *err) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = vals[i];
    bool bad = (i + 1 < n && keys[i] < keys[i + 1]) || v < 0 || v >= n;
    if (!bad) bad = atomicExch(seen + v, 1) != 0;
    if (bad) atomicExch(err, kDevCheck);
  }
}

struct HistF {
  const int64_t *h;
  __device__ int64_t operator()(int64_t i) const { return h[i]; }
};
struct HistG {
  int64_t *off;
  __device__ void operator()(int64_t i, int64_t excl, int64_t) const { off[i] = excl; }
};

}  // namespace

int radix_sort_desc(mc_graph *g, uint32_t *keys, int32_t *vals, uint32_t *ktmp, int32_t *vtmp, int64_t n) {
  if (n <= 1) return MC_OK;
  const int64_t nb = (n + kRTile - 1) / kRTile;
  void *p;
  MC_TRY(ws_get(g, "rs.hist", (size_t)nb * 256 * 8, &p));
  int64_t *hist = (int64_t *)p;
  MC_TRY(ws_get(g, "rs.off", (size_t)nb * 256 * 8, &p));
  int64_t *off = (int64_t *)p;
  uint32_t *ka = keys, *kb = ktmp;
  int32_t *va = vals, *vb = vtmp;
  for (int shift = 0; shift < 32; shift += 8) {
    radix_hist_kernel<<<(unsigned)nb, kRT, 0, g->stream>>>(n, ka, shift, nb, hist);
    g_launches++;
    MC_CUDA_TRY(cudaGetLastError());
    MC_TRY(device_scan(g, nb * 256, HistF{hist}, HistG{off}, nullptr, "rs.scan"));
    radix_scatter_kernel<<<(unsigned)nb, kRT, 0, g->stream>>>(n, ka, va, kb, vb, shift, nb, off);
    g_launches++;
    MC_CUDA_TRY(cudaGetLastError());
    std::swap(ka, kb);
    std::swap(va, vb);
  }
  // four passes: the result is back in keys / vals; ktmp serves as the
  // permutation check's marks
  MC_CUDA_TRY(cudaMemsetAsync(ktmp, 0, (size_t)n * 4, g->stream));
  sort_check_kernel<<<(unsigned)std::min<int64_t>((n + 255) / 256, (int64_t)g->sm_count * 8), 256, 0, g->stream>>>(
      n, keys, vals, (int32_t *)ktmp, g->err);
  g_launches++;
  MC_CUDA_TRY(cudaGetLastError());
  return MC_OK;
}

}  // namespace mc
