// Device-wide exclusive scan of a generated int64 sequence (reduce-then-scan,
// three launches).  The input is a functor f(i) -> int64, so flags and counts
// need not be materialised.
#pragma once

#include "mc_internal.cuh"

namespace mc {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

template <class F>
__global__ void scan_reduce_kernel(int64_t n, F f, int64_t *__restrict__ bsum) {
  __shared__ int64_t red[kScanThreads / 32];
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  int64_t s = 0;
#pragma unroll
  for (int j = 0; j < kScanItems; j++) {
    int64_t i = base + (int64_t)j * kScanThreads + threadIdx.x;
    if (i < n) s += f(i);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t t = 0;
    for (int w = 0; w < kScanThreads / 32; w++) t += red[w];
    bsum[blockIdx.x] = t;
  }
}

// exclusive scan of bsum[0..nb) in place by one block; bsum[nb] = total
__global__ void scan_blocks_kernel(int64_t nb, int64_t *bsum);

template <class F, class G>
__global__ void scan_apply_kernel(int64_t n, F f, const int64_t *__restrict__ bsum, G g) {
  __shared__ int64_t wsum[kScanThreads / 32 + 1];
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  // each thread owns kScanItems consecutive items
  int64_t vals[kScanItems];
  int64_t tsum = 0;
#pragma unroll
  for (int j = 0; j < kScanItems; j++) {
    int64_t i = base + (int64_t)threadIdx.x * kScanItems + j;
    vals[j] = (i < n) ? f(i) : 0;
    tsum += vals[j];
  }
  int64_t incl = tsum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int64_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) wsum[wid] = incl;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t t = 0;
    for (int w = 0; w < kScanThreads / 32; w++) {
      int64_t x = wsum[w];
      wsum[w] = t;
      t += x;
    }
  }
  __syncthreads();
  int64_t run = bsum[blockIdx.x] + wsum[wid] + incl - tsum;
#pragma unroll
  for (int j = 0; j < kScanItems; j++) {
    int64_t i = base + (int64_t)threadIdx.x * kScanItems + j;
    if (i < n) g(i, run, vals[j]);
    run += vals[j];
  }
}

// Exclusive scan: for i in [0, n), g(i, sum_{j<i} f(j), f(i)).  Writes the
// total to *d_total (device).  bsum: workspace of at least nblocks+1 int64.
template <class F, class G>
int device_scan(mc_graph *gr, int64_t n, F f, G g, int64_t *d_total, const char *ws_name) {
  if (n <= 0) {
    if (d_total) {
      cudaError_t e = cudaMemsetAsync(d_total, 0, sizeof(int64_t), gr->stream);
      if (e != cudaSuccess) return MC_ERR_CUDA;
    }
    return MC_OK;
  }
  const int64_t nb = (n + kScanTile - 1) / kScanTile;
  void *p;
  MC_TRY(ws_get(gr, ws_name, (nb + 1) * sizeof(int64_t), &p));
  int64_t *bsum = (int64_t *)p;
  scan_reduce_kernel<<<(unsigned)nb, kScanThreads, 0, gr->stream>>>(n, f, bsum);
  scan_blocks_kernel<<<1, 1024, 0, gr->stream>>>(nb, bsum);
  scan_apply_kernel<<<(unsigned)nb, kScanThreads, 0, gr->stream>>>(n, f, bsum, g);
  g_launches += 3;
  if (d_total) {
    cudaError_t e = cudaMemcpyAsync(d_total, bsum + nb, sizeof(int64_t), cudaMemcpyDeviceToDevice, gr->stream);
    if (e != cudaSuccess) return MC_ERR_CUDA;
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? MC_OK : MC_ERR_CUDA;
}

}  // namespace mc
