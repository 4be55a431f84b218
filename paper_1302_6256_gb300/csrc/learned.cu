// Learned vertex ordering: per-vertex features and a 6 -> 64 -> 64 -> 1 MLP
// (ReLU, BF16 weights, FP32 accumulation, FP32 master weights and Adam).
// The score only orders the search's roots and seeds the heuristic; omega
// stays exact whatever the network predicts.
//
// Features of vertex v (d = degree, K = core number, Kmax = K(G), Dmax =
// maximum degree, c = number of neighbours with K >= K(v), Q = the first
// min(8, c) of those neighbours in increasing id):
//   f0 = log1p(d) / log1p(Dmax)        f3 = (chi + 1) / 9, chi = colours of
//   f1 = K(v) / Kmax                        the greedy colouring of G[Q] in
//   f2 = t / 28, t = edges among Q          increasing id (a bound on a
//                                           clique through v inside Q + v)
//   f4 = c / max(d, 1)                 f5 = log1p(c) / log1p(Dmax)
// Eight lanes per vertex, four vertices per warp in flight: a pass over the
// row (c and Q), the 28 pairs of Q each found by binary search in the
// shorter of the two rows, the colouring with one colour class per lane,
// and the network with eight hidden units per lane.
//
// Parameters, flat fp32 (4673): W1[64][6], b1[64], W2[64][64], b2[64],
// w3[64], b3.  Loss: binary cross-entropy on the logit s with weight
// pos_weight on positive labels, averaged over the rows.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "mc_internal.cuh"

namespace mc {

constexpr int kF = 6, kH = 64;
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kH * kF, kOffW2 = kOffB1 + kH, kOffB2 = kOffW2 + kH * kH,
              kOffW3 = kOffB2 + kH, kOffB3 = kOffW3 + kH, kParams = kOffB3 + 1;

}  // namespace mc

struct mc_mlp {
  cudaStream_t stream = nullptr;
  int device = 0, sm_count = 0;
  float *master = nullptr;   // fp32 master parameters
  uint16_t *wbf = nullptr;   // bf16 copies of the weights (all parameters, same layout)
  float *grad = nullptr, *m = nullptr, *v = nullptr;
  float *loss = nullptr;     // device scalar
  float *buf = nullptr;      // staging for host inputs
  size_t buf_bytes = 0;
  int64_t step = 0;
  void *h_small = nullptr;
};

namespace mc {
namespace {

__device__ __forceinline__ float bf16_to_f32(uint16_t h) { return __uint_as_float(((uint32_t)h) << 16); }

// round to nearest even
__host__ __device__ __forceinline__ uint16_t f32_to_bf16(float f) {
#ifdef __CUDA_ARCH__
  uint32_t x = __float_as_uint(f);
#else
  uint32_t x;
  memcpy(&x, &f, 4);
#endif
  if ((x & 0x7f800000u) == 0x7f800000u) return (uint16_t)(x >> 16);  // inf / nan
  uint32_t r = x + 0x7fffu + ((x >> 16) & 1u);
  return (uint16_t)(r >> 16);
}

constexpr int kQ = 8;  // neighbours of the triangle and colouring features

// Sub-warp primitive over the 8 lanes of a group (mask gm covers them).
__device__ __forceinline__ unsigned group_ballot(unsigned gm, bool x, int grp) {
  return (__ballot_sync(gm, x) >> (grp * 8)) & 0xFFu;
}

__device__ __forceinline__ bool in_row(const int64_t *__restrict__ rp, const int32_t *__restrict__ ci, int x, int y) {
  int64_t lo = rp[x], hi = rp[x + 1];
  const int64_t end = hi;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (ci[mid] < y) lo = mid + 1; else hi = mid;
  }
  return lo < end && ci[lo] == y;
}

// The six features of vertex v, computed by the 8 lanes of one group (all
// 8 call with the same v; every lane of the group returns them).  qs: 8
// ints of shared memory for this group.
__device__ void vertex_features(const int64_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                const int32_t *__restrict__ core, float kmax, float ldmax, int64_t v, int *qs,
                                float f[kF]) {
  const int lane = threadIdx.x & 31, grp = lane >> 3, gl = lane & 7;
  const unsigned gm = 0xFFu << (grp * 8);
  const unsigned below = (1u << gl) - 1u;
  const int kv = core[v];
  const int64_t e0 = rp[v], e1 = rp[v + 1];
  int c = 0;
  for (int64_t eb = e0; eb < e1; eb += 8) {
    const int64_t e = eb + gl;
    int u = -1;
    bool ok = false;
    if (e < e1) {
      u = ci[e];
      ok = core[u] >= kv;
    }
    const unsigned m = group_ballot(gm, ok, grp);
    if (ok) {
      const int pos = c + __popc(m & below);
      if (pos < kQ) qs[pos] = u;
    }
    c += __popc(m);
  }
  __syncwarp(gm);
  const int q = min(c, kQ);
  // the q(q-1)/2 pairs i < j, bit p of `pairs` for pair p (row-major over i)
  uint32_t pairs = 0u;
  for (int p = gl; p < q * (q - 1) / 2; p += 8) {
    int i = 0, r = p;
    while (r >= q - 1 - i) {
      r -= q - 1 - i;
      i++;
    }
    const int x = qs[i], y = qs[i + 1 + r];
    // binary search in the shorter row
    const bool adj = (rp[x + 1] - rp[x] <= rp[y + 1] - rp[y]) ? in_row(rp, ci, x, y) : in_row(rp, ci, y, x);
    if (adj) pairs |= 1u << p;
  }
  pairs = __reduce_or_sync(gm, pairs);
  const int t = __popc(pairs);
  // row gl of G[Q]: member j is adjacent to member gl if pair (min, max) is set
  uint32_t row = 0u;
  if (gl < q)
    for (int j = 0; j < q; j++) {
      if (j == gl) continue;
      const int a = min(gl, j), b = max(gl, j);
      const int pid = a * q - a * (a + 1) / 2 + (b - a - 1);
      if ((pairs >> pid) & 1u) row |= 1u << j;
    }
  // greedy colouring in index order: lane gl holds colour class gl; member
  // i joins the first class with none of its neighbours
  uint32_t cls = 0u;
  for (int i = 0; i < q; i++) {
    const uint32_t ai = __shfl_sync(gm, row, i, 8);
    const unsigned clash = group_ballot(gm, (cls & ai) != 0u, grp);
    const int k = __ffs(~clash) - 1;
    if (gl == k) cls |= 1u << i;
  }
  const int chi = __popc(group_ballot(gm, cls != 0u, grp));
  const float d = (float)(e1 - e0);
  f[0] = log1pf(d) / ldmax;
  f[1] = (float)kv / kmax;
  f[2] = (float)t / (float)(kQ * (kQ - 1) / 2);
  f[3] = (float)(chi + 1) / (float)(kQ + 1);
  f[4] = (float)c / fmaxf(d, 1.f);
  f[5] = log1pf((float)c) / ldmax;
}

// features of every vertex (list == nullptr) or of list[0 .. *count)
__global__ void __launch_bounds__(256) features_kernel(int64_t n, const int32_t *__restrict__ list,
                                                       const int64_t *__restrict__ count,
                                                       const int64_t *__restrict__ rp,
                                                       const int32_t *__restrict__ ci,
                                                       const int32_t *__restrict__ core, float kmax, float ldmax,
                                                       float *__restrict__ f) {
  __shared__ int qs[8][4][kQ];
  const int lane = threadIdx.x & 31, grp = lane >> 3, gl = lane & 7;
  const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t total = list ? *count : n;
  for (int64_t b = w0 * 4; b < total; b += nw * 4) {
    const int64_t r = b + grp;
    if (r >= total) continue;  // the whole group skips
    const int64_t v = list ? list[r] : r;
    float x[kF];
    vertex_features(rp, ci, core, kmax, ldmax, v, qs[threadIdx.x >> 5][grp], x);
    if (gl == 0) {
#pragma unroll
      for (int i = 0; i < kF; i++) f[v * kF + i] = x[i];
    }
  }
}

// The network in shared memory, laid out for a group of eight lanes per
// row: lane gl owns hidden units gl, gl + 8, ..., gl + 56; the first two
// layers are stored input-major so a group's reads of one input's weights
// are consecutive words.
struct MlpSmem {
  float w1t[kF][kH];  // w1t[i][j] = W1[j][i]
  float b1[kH];
  float w2t[kH][kH];  // w2t[k][j] = W2[j][k]
  float b2[kH];
  float w3[kH];
  float b3;
};

__device__ void load_mlp(const uint16_t *__restrict__ wbf, const float *__restrict__ master, MlpSmem &S) {
  for (int e = threadIdx.x; e < kH * kF; e += blockDim.x) {
    const int j = e / kF, i = e % kF;
    S.w1t[i][j] = bf16_to_f32(wbf[kOffW1 + e]);
  }
  for (int e = threadIdx.x; e < kH * kH; e += blockDim.x) {
    const int j = e / kH, k = e % kH;
    S.w2t[k][j] = bf16_to_f32(wbf[kOffW2 + e]);
  }
  for (int j = threadIdx.x; j < kH; j += blockDim.x) {
    S.b1[j] = master[kOffB1 + j];  // biases stay fp32
    S.b2[j] = master[kOffB2 + j];
    S.w3[j] = bf16_to_f32(wbf[kOffW3 + j]);
  }
  if (threadIdx.x == 0) S.b3 = master[kOffB3];
  __syncthreads();
}

// The logit of one row x (every lane of the group holds x), by the 8 lanes
// of a group.
__device__ __forceinline__ float mlp_logit_group(const MlpSmem &S, const float x[kF]) {
  const int lane = threadIdx.x & 31, grp = lane >> 3, gl = lane & 7;
  const unsigned gm = 0xFFu << (grp * 8);
  float h[8];
#pragma unroll
  for (int t = 0; t < 8; t++) {
    const int j = gl + 8 * t;
    float z = S.b1[j];
#pragma unroll
    for (int i = 0; i < kF; i++) z = fmaf(S.w1t[i][j], x[i], z);
    h[t] = fmaxf(z, 0.f);
  }
  float z[8];
#pragma unroll
  for (int t = 0; t < 8; t++) z[t] = S.b2[gl + 8 * t];
#pragma unroll
  for (int tk = 0; tk < 8; tk++) {
#pragma unroll
    for (int src = 0; src < 8; src++) {
      const float hk = __shfl_sync(gm, h[tk], src, 8);
      const int k = src + 8 * tk;
#pragma unroll
      for (int t = 0; t < 8; t++) z[t] = fmaf(S.w2t[k][gl + 8 * t], hk, z[t]);
    }
  }
  float sum = 0.f;
#pragma unroll
  for (int t = 0; t < 8; t++) sum = fmaf(S.w3[gl + 8 * t], fmaxf(z[t], 0.f), sum);
#pragma unroll
  for (int o = 4; o > 0; o >>= 1) sum += __shfl_xor_sync(gm, sum, o, 8);
  return sum + S.b3;
}

// weights into shared memory as fp32 (from the bf16 copies)
__device__ __forceinline__ void load_weights(const uint16_t *__restrict__ wbf, const float *__restrict__ master,
                                             float *sw) {
  for (int i = threadIdx.x; i < kParams; i += blockDim.x) {
    const bool is_bias = (i >= kOffB1 && i < kOffW2) || (i >= kOffB2 && i < kOffW3) || i == kOffB3;
    sw[i] = is_bias ? master[i] : bf16_to_f32(wbf[i]);  // biases stay fp32
  }
  __syncthreads();
}

// logits of n feature rows, eight lanes per row
__global__ void __launch_bounds__(256) forward_kernel(int64_t n, const float *__restrict__ feat,
                                                      const uint16_t *__restrict__ wbf,
                                                      const float *__restrict__ master, float *__restrict__ out) {
  __shared__ MlpSmem S;
  load_mlp(wbf, master, S);
  const int lane = threadIdx.x & 31, grp = lane >> 3, gl = lane & 7;
  const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t b = w0 * 4; b < n; b += nw * 4) {
    const int64_t r = b + grp;
    if (r >= n) continue;
    float x[kF];
#pragma unroll
    for (int i = 0; i < kF; i++) x[i] = feat[r * kF + i];
    const float s = mlp_logit_group(S, x);
    if (gl == 0) out[r] = s;
  }
}

// Learned scores of list[0 .. *count): features and logit fused, eight
// lanes per vertex; the n x 6 feature rows never reach memory.
__global__ void __launch_bounds__(256) score_kernel(const int32_t *__restrict__ list, const int64_t *__restrict__ count,
                                                    const int64_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                                    const int32_t *__restrict__ core, float kmax, float ldmax,
                                                    const uint16_t *__restrict__ wbf, const float *__restrict__ master,
                                                    float *__restrict__ score) {
  __shared__ MlpSmem S;
  __shared__ int qs[8][4][kQ];
  load_mlp(wbf, master, S);
  const int lane = threadIdx.x & 31, grp = lane >> 3, gl = lane & 7;
  const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t total = *count;
  for (int64_t b = w0 * 4; b < total; b += nw * 4) {
    const int64_t r = b + grp;
    if (r >= total) continue;
    const int v = list[r];
    float x[kF];
    vertex_features(rp, ci, core, kmax, ldmax, v, qs[threadIdx.x >> 5][grp], x);
    const float s = mlp_logit_group(S, x);
    if (gl == 0) score[v] = s;
  }
}

// Gradient of the mean weighted BCE over rows, accumulated into grad (fp32).
// Each block accumulates its rows' contributions in shared memory and adds
// them to the global gradient once.
constexpr int kGT = 128;
struct GradSmem {
  float sw[kParams];
  float sg[kParams];
  float sh1[kGT][kH + 1];  // this tile's hidden activations
  float sd2[kGT][kH + 1];  // d loss / d z2, then d loss / d z1
  float sx[kGT][kF];
  float sloss;
};
__global__ void __launch_bounds__(kGT) grad_kernel(int64_t n, const float *__restrict__ feat,
                                                   const float *__restrict__ label, float pos_weight,
                                                   const uint16_t *__restrict__ wbf, const float *__restrict__ master,
                                                   float *__restrict__ grad, float *__restrict__ loss) {
  extern __shared__ __align__(16) unsigned char gsm_raw[];
  GradSmem &S = *reinterpret_cast<GradSmem *>(gsm_raw);
  float *sw = S.sw, *sg = S.sg;
  auto &sh1 = S.sh1;
  auto &sd2 = S.sd2;
  auto &sx = S.sx;
  float &sloss = S.sloss;
  load_weights(wbf, master, sw);
  for (int i = threadIdx.x; i < kParams; i += blockDim.x) sg[i] = 0.f;
  if (threadIdx.x == 0) sloss = 0.f;
  __syncthreads();
  const float inv_n = 1.f / (float)n;
  const int t = threadIdx.x;
  for (int64_t base = (int64_t)blockIdx.x * kGT; base < n; base += (int64_t)gridDim.x * kGT) {
    const int64_t r = base + t;
    const bool valid = r < n;
    float x[kF], h1[kH];
#pragma unroll
    for (int i = 0; i < kF; i++) x[i] = valid ? feat[r * kF + i] : 0.f;
    // forward keeping z2 signs in sd2 as a scratch
    float s = sw[kOffB3];
#pragma unroll
    for (int j = 0; j < kH; j++) {
      float z = sw[kOffB1 + j];
#pragma unroll
      for (int i = 0; i < kF; i++) z = fmaf(sw[kOffW1 + j * kF + i], x[i], z);
      h1[j] = fmaxf(z, 0.f);
    }
    float z2[kH];
    for (int j = 0; j < kH; j++) {
      float z = sw[kOffB2 + j];
#pragma unroll
      for (int k = 0; k < kH; k++) z = fmaf(sw[kOffW2 + j * kH + k], h1[k], z);
      z2[j] = z;
      s = fmaf(sw[kOffW3 + j], fmaxf(z, 0.f), s);
    }
    // d loss / d s for weighted BCE with logits, mean over rows
    float gs = 0.f;
    if (valid) {
      const float y = label[r];
      const float w = y > 0.5f ? pos_weight : 1.f;
      const float sig = 1.f / (1.f + expf(-s));
      gs = w * (sig - y) * inv_n;
      // loss = w * (log(1 + e^s) - y s), computed stably
      const float l = w * (fmaxf(s, 0.f) + log1pf(expf(-fabsf(s))) - y * s);
      atomicAdd(&sloss, l * inv_n);
    }
    atomicAdd(&sg[kOffB3], gs);
    for (int j = 0; j < kH; j++) {
      const float a2 = fmaxf(z2[j], 0.f);
      sd2[t][j] = (z2[j] > 0.f) ? gs * sw[kOffW3 + j] : 0.f;
      z2[j] = a2 * gs;  // d loss / d w3_j contribution
    }
#pragma unroll
    for (int k = 0; k < kH; k++) sh1[t][k] = h1[k];
#pragma unroll
    for (int i = 0; i < kF; i++) sx[t][i] = x[i];
    // d loss / d h1_k = sum_j d2_j W2[j][k]; back through the first ReLU
    float d1[kH];
    for (int k = 0; k < kH; k++) d1[k] = 0.f;
    for (int j = 0; j < kH; j++) {
      const float dj = sd2[t][j];
      if (dj != 0.f)
#pragma unroll
        for (int k = 0; k < kH; k++) d1[k] = fmaf(dj, sw[kOffW2 + j * kH + k], d1[k]);
    }
    // reuse z2 storage: w3 gradient contributions
    for (int j = 0; j < kH; j++) atomicAdd(&sg[kOffW3 + j], z2[j]);
    __syncthreads();
    // W2 and b2: each thread owns entries (j, k), summing over the tile's rows
    for (int e = t; e < kH * kH; e += kGT) {
      const int j = e / kH, k = e % kH;
      float acc = 0.f;
      for (int q = 0; q < kGT; q++) acc = fmaf(sd2[q][j], sh1[q][k], acc);
      sg[kOffW2 + e] += acc;
    }
    if (t < kH) {
      float acc = 0.f;
      for (int q = 0; q < kGT; q++) acc += sd2[q][t];
      sg[kOffB2 + t] += acc;
    }
    __syncthreads();
    // first layer: d z1_k = d1_k [h1_k > 0]; W1 and b1 summed over the tile
#pragma unroll
    for (int k = 0; k < kH; k++) sd2[t][k] = (h1[k] > 0.f) ? d1[k] : 0.f;
    __syncthreads();
    for (int e = t; e < kH * kF; e += kGT) {
      const int k = e / kF, i = e % kF;
      float acc = 0.f;
      for (int q = 0; q < kGT; q++) acc = fmaf(sd2[q][k], sx[q][i], acc);
      sg[kOffW1 + e] += acc;
    }
    if (t < kH) {
      float acc = 0.f;
      for (int q = 0; q < kGT; q++) acc += sd2[q][t];
      sg[kOffB1 + t] += acc;
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < kParams; i += blockDim.x) atomicAdd(grad + i, sg[i]);
  if (threadIdx.x == 0 && loss) atomicAdd(loss, sloss);
}

__global__ void adam_kernel(float *__restrict__ master, uint16_t *__restrict__ wbf, const float *__restrict__ grad,
                            float *__restrict__ m, float *__restrict__ v, float lr, float b1, float b2, float eps,
                            float c1, float c2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kParams; i += gridDim.x * blockDim.x) {
    const float g = grad[i];
    const float mi = b1 * m[i] + (1.f - b1) * g;
    const float vi = b2 * v[i] + (1.f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    const float p = master[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    master[i] = p;
    wbf[i] = f32_to_bf16(p);
  }
}

__global__ void round_kernel(const float *__restrict__ master, uint16_t *__restrict__ wbf) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kParams; i += gridDim.x * blockDim.x)
    wbf[i] = f32_to_bf16(master[i]);
}

uint64_t splitmix(uint64_t z) {
  z += 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

int stage(mc_mlp *m, const void *src, size_t bytes, const void **dev) {
  if (is_device_ptr(src)) {
    *dev = src;
    return MC_OK;
  }
  if (m->buf_bytes < bytes) {
    if (m->buf) {
      MC_CUDA_TRY(cudaStreamSynchronize(m->stream));
      cudaFree(m->buf);
    }
    m->buf = nullptr;
    m->buf_bytes = 0;
    MC_CUDA_TRY(cudaMalloc(&m->buf, bytes));
    m->buf_bytes = bytes;
  }
  MC_CUDA_TRY(cudaMemcpyAsync(m->buf, src, bytes, cudaMemcpyHostToDevice, m->stream));
  *dev = m->buf;
  return MC_OK;
}

// ------------------------------------------- the learned form of a solve ---

// Vertices that can still be in a clique larger than their graph's current
// bound (K(v) >= best), appended to list (warp-aggregated); *count holds the
// number (zeroed by the caller).
__global__ void subset_kernel(int64_t n, const int32_t *__restrict__ core, const int32_t *__restrict__ gid,
                              const int32_t *__restrict__ best, const int32_t *__restrict__ kfloor,
                              int32_t *__restrict__ list, unsigned long long *__restrict__ count) {
  const int kf = kfloor ? *kfloor : 0;
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t b = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) & ~(int64_t)31; b < n; b += stride) {
    const int64_t v = b + lane;
    bool in = false;
    if (v < n) in = core[v] >= max(best[gid ? gid[v] : 0], kf);
    const unsigned m = __ballot_sync(0xffffffffu, in);
    if (!m) continue;
    unsigned long long at = 0;
    if (lane == 0) at = atomicAdd(count, (unsigned long long)__popc(m));
    at = __shfl_sync(0xffffffffu, at, 0);
    if (in) list[at + __popc(m & lt)] = (int32_t)v;
  }
}

__global__ void fill_kernel(int64_t n, float x, float *__restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = x;
}

// Histogram of the core numbers (bins 0..kmax).
__global__ void core_hist_kernel(int64_t n, const int32_t *__restrict__ core, int kmax, unsigned int *__restrict__ hist) {
  extern __shared__ unsigned int sh[];
  const bool local = kmax < 8192;
  if (local) {
    for (int i = threadIdx.x; i <= kmax; i += blockDim.x) sh[i] = 0;
    __syncthreads();
  }
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int k = min(core[v], kmax);
    atomicAdd(local ? &sh[k] : &hist[k], 1u);
  }
  if (local) {
    __syncthreads();
    for (int i = threadIdx.x; i <= kmax; i += blockDim.x)
      if (sh[i]) atomicAdd(&hist[i], sh[i]);
  }
}

// The core floor of the scored subset: the smallest k such that at most
// `budget` vertices have K(v) >= k (at least the top shell, K(G)).
__global__ void core_floor_kernel(const unsigned int *__restrict__ hist, int kmax, long long budget,
                                  int32_t *__restrict__ kfloor) {
  if (threadIdx.x != 0) return;
  long long above = 0;
  int k = kmax;
  above = hist[kmax];
  while (k > 0 && above + (long long)hist[k - 1] <= budget) {
    k--;
    above += hist[k];
  }
  *kfloor = k;
}

// Selection key of a scored vertex: the score's order as an unsigned
// integer (larger score, larger key; raised to at least 1) in the high
// word, and the complement of the vertex id in the low word, so keys are
// unique and ties go to the smaller id.
__device__ __forceinline__ unsigned long long seed_key(float s, int v) {
  const uint32_t b = __float_as_uint(s);
  const uint32_t k = max((b & 0x80000000u) ? ~b : (b | 0x80000000u), 1u);
  return ((unsigned long long)k << 32) | (unsigned long long)(0xFFFFFFFFu - (uint32_t)v);
}

struct SelectCtl {
  unsigned long long prefix, mask;  // key bits fixed so far
  long long need;                   // keys still to take at or below the prefix
  long long taken;                  // keys collected
  int all;                          // fewer keys than k: take every key
  int pad;
  unsigned int hist[256];
};

__global__ void select_init_kernel(SelectCtl *ctl, int k) {
  if (threadIdx.x == 0) ctl->need = k;
}

// one 8-bit digit of the k-th largest key: histogram of the keys that match
// the prefix so far
__global__ void select_hist_kernel(const int32_t *__restrict__ list, const unsigned long long *__restrict__ count,
                                   const float *__restrict__ score, SelectCtl *ctl, int shift) {
  __shared__ unsigned int h[256];
  for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0;
  __syncthreads();
  const unsigned long long prefix = ctl->prefix, mask = ctl->mask;
  const int64_t total = (int64_t)*count;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < total; r += (int64_t)gridDim.x * blockDim.x) {
    const int v = list[r];
    const unsigned long long key = seed_key(score[v], v);
    if ((key & mask) == prefix) atomicAdd(&h[(key >> shift) & 255ull], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 256; i += blockDim.x)
    if (h[i]) atomicAdd(&ctl->hist[i], h[i]);
}

__global__ void select_pick_kernel(SelectCtl *ctl, int shift) {
  if (threadIdx.x != 0 || ctl->all) return;
  long long acc = 0;
  int b = 255;
  for (; b >= 0; b--) {
    if (acc + (long long)ctl->hist[b] >= ctl->need) break;
    acc += ctl->hist[b];
  }
  if (b < 0) {  // fewer matching keys than needed: only on the first digit
    ctl->all = 1;
  } else {
    ctl->need -= acc;
    ctl->prefix |= (unsigned long long)b << shift;
    ctl->mask |= 255ull << shift;
  }
  for (int i = 0; i < 256; i++) ctl->hist[i] = 0;
}

__global__ void select_collect_kernel(const int32_t *__restrict__ list, const unsigned long long *__restrict__ count,
                                      const float *__restrict__ score, SelectCtl *ctl, int k,
                                      unsigned long long *__restrict__ keys) {
  const unsigned long long thr = ctl->all ? 0ull : ctl->prefix;
  const int64_t total = (int64_t)*count;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < total; r += (int64_t)gridDim.x * blockDim.x) {
    const int v = list[r];
    const unsigned long long key = seed_key(score[v], v);
    if (key >= thr) {
      const long long at = atomicAdd((unsigned long long *)&ctl->taken, 1ull);
      if (at < k) keys[at] = key;
    }
  }
}

// the collected keys in decreasing order -> seed vertices; -1 pads the
// slots past the number collected
constexpr int kMaxSeeds = 1024;
__global__ void __launch_bounds__(1024) select_sort_kernel(const SelectCtl *ctl, int k,
                                                           const unsigned long long *__restrict__ keys,
                                                           int32_t *__restrict__ seeds) {
  __shared__ unsigned long long a[kMaxSeeds];
  const int got = (int)(ctl->taken < (long long)k ? ctl->taken : (long long)k);
  for (int i = threadIdx.x; i < kMaxSeeds; i += blockDim.x) a[i] = i < got ? keys[i] : 0ull;
  __syncthreads();
  for (int len = 2; len <= kMaxSeeds; len <<= 1) {
    for (int j = len >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < kMaxSeeds; i += blockDim.x) {
        const int x = i ^ j;
        if (x > i) {
          const unsigned long long p = a[i], q = a[x];
          const bool desc = (i & len) == 0;
          if (desc ? (p < q) : (p > q)) {
            a[i] = q;
            a[x] = p;
          }
        }
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < k; i += blockDim.x)
    seeds[i] = i < got ? (int32_t)(0xFFFFFFFFu - (uint32_t)(a[i] & 0xFFFFFFFFull)) : -1;
}

// Batches: the j best-scored vertices of every graph among those that can
// beat its bound, one warp per graph (j rounds of a warp maximum, each
// below the last key taken).  seeds[g * j + r], -1 where a graph has fewer.
__global__ void graph_seeds_kernel(int32_t count, const int64_t *__restrict__ voff, const int32_t *__restrict__ core,
                                   const int32_t *__restrict__ best, const float *__restrict__ score, int j,
                                   int32_t *__restrict__ seeds) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t g = w0; g < count; g += nw) {
    const int64_t v0 = voff[g], v1 = voff[g + 1];
    const int bg = best[g];
    unsigned long long last = ~0ull;
    for (int r = 0; r < j; r++) {
      unsigned long long mx = 0ull;
      for (int64_t v = v0 + lane; v < v1; v += 32) {
        if (core[v] < bg) continue;
        const unsigned long long key = seed_key(score[v], (int)v);
        if (key < last && key > mx) mx = key;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long y = __shfl_xor_sync(0xffffffffu, mx, o);
        if (y > mx) mx = y;
      }
      if (lane == 0) seeds[g * j + r] = mx ? (int32_t)(0xFFFFFFFFu - (uint32_t)(mx & 0xFFFFFFFFull)) : -1;
      last = mx;
      if (!mx) last = 0ull;
    }
  }
}

}  // namespace

// Scores of the vertices that can still be in a clique larger than their
// graph's current bound -- for one graph, of at most kLearnedBudget of them,
// those of highest core number.  The other vertices get the lowest score
// (they are read only as candidates of a seeded growth, which then takes
// them last).
constexpr long long kLearnedBudget = 1ll << 22;
int learned_scores(mc_graph *g, const mc_mlp *m, float *score) {
  if (g->n == 0) return MC_OK;
  void *p;
  MC_TRY(ws_get(g, "ln.list", (size_t)g->n * 4, &p));
  int32_t *list = (int32_t *)p;
  MC_TRY(ws_get(g, "ln.ctl", 64 + sizeof(SelectCtl), &p));
  unsigned long long *count = (unsigned long long *)p;
  int32_t *kfloor = (int32_t *)((char *)p + 8);
  MC_CUDA_TRY(cudaMemsetAsync(count, 0, 16, g->stream));
  const int blocks = (int)std::min<int64_t>((g->n + 255) / 256, (int64_t)g->sm_count * 8);
  if (g->count == 1 && g->n > kLearnedBudget) {
    // one graph: score at most kLearnedBudget vertices, those of highest
    // core number (a vertex of core number K is in no clique above K + 1)
    const int kmax = std::max(g->max_core, 0);
    MC_TRY(ws_get(g, "ln.hist", (size_t)(kmax + 2) * 4, &p));
    unsigned int *hist = (unsigned int *)p;
    MC_CUDA_TRY(cudaMemsetAsync(hist, 0, (size_t)(kmax + 2) * 4, g->stream));
    const size_t shm = kmax < 8192 ? (size_t)(kmax + 1) * 4 : 0;
    core_hist_kernel<<<blocks, 256, shm, g->stream>>>(g->n, g->core, kmax, hist);
    core_floor_kernel<<<1, 32, 0, g->stream>>>(hist, kmax, kLearnedBudget, kfloor);
    g_launches += 2;
  }
  subset_kernel<<<blocks, 256, 0, g->stream>>>(g->n, g->core, g->gid, g->best, kfloor, list, count);
  fill_kernel<<<blocks, 256, 0, g->stream>>>(g->n, -INFINITY, score);
  g_launches += 2;
  const float kmax = (float)std::max(g->max_core, 1);
  const float ldmax = log1pf((float)std::max(g->max_degree, 1));
  const int sblocks = g->sm_count * 8;
  score_kernel<<<sblocks, 256, 0, g->stream>>>(list, (const int64_t *)count, g->row_ptr, g->col_idx, g->core, kmax,
                                               ldmax, m->wbf, m->master, score);
  g_launches++;
  MC_CUDA_TRY(cudaGetLastError());
  return MC_OK;
}

// Seeds of the learned heuristic: for one graph the k best-scored vertices
// of the subset that learned_scores scored (exact selection by 8-bit digits
// of a unique 64-bit key, best first); for a batch the k best of every
// graph.  Writes seeds (k or count * k slots, -1 for missing ones).
int learned_seeds(mc_graph *g, const float *score, int32_t k, int32_t *seeds) {
  if (g->n == 0 || k <= 0) return MC_OK;
  void *p;
  if (g->count > 1) {
    const int blocks = (int)std::min<int64_t>(((int64_t)g->count * 32 + 255) / 256, (int64_t)g->sm_count * 16);
    graph_seeds_kernel<<<blocks, 256, 0, g->stream>>>(g->count, g->voff, g->core, g->best, score, k, seeds);
    g_launches++;
    MC_CUDA_TRY(cudaGetLastError());
    return MC_OK;
  }
  if (k > kMaxSeeds) return MC_ERR_ARG;
  MC_TRY(ws_get(g, "ln.list", (size_t)g->n * 4, &p));
  const int32_t *list = (const int32_t *)p;
  MC_TRY(ws_get(g, "ln.ctl", 64 + sizeof(SelectCtl), &p));
  const unsigned long long *count = (const unsigned long long *)p;
  SelectCtl *ctl = (SelectCtl *)((char *)p + 64);
  MC_TRY(ws_get(g, "ln.keys", (size_t)kMaxSeeds * 8, &p));
  unsigned long long *keys = (unsigned long long *)p;
  MC_CUDA_TRY(cudaMemsetAsync(ctl, 0, sizeof(SelectCtl), g->stream));
  select_init_kernel<<<1, 32, 0, g->stream>>>(ctl, k);
  g_launches++;
  const int blocks = g->sm_count * 4;
  for (int shift = 56; shift >= 0; shift -= 8) {
    select_hist_kernel<<<blocks, 256, 0, g->stream>>>(list, count, score, ctl, shift);
    select_pick_kernel<<<1, 32, 0, g->stream>>>(ctl, shift);
    g_launches += 2;
  }
  select_collect_kernel<<<blocks, 256, 0, g->stream>>>(list, count, score, ctl, k, keys);
  select_sort_kernel<<<1, 1024, 0, g->stream>>>(ctl, k, keys, seeds);
  g_launches += 2;
  MC_CUDA_TRY(cudaGetLastError());
  return MC_OK;
}

}  // namespace mc

using namespace mc;

extern "C" {

int mc_mlp_create(uint64_t seed, void *cuda_stream, mc_mlp **out) {
  if (!out) return MC_ERR_ARG;
  *out = nullptr;
  mc_mlp *m = new mc_mlp();
  m->stream = (cudaStream_t)cuda_stream;
  auto fail = [&](int rc) {
    cudaFree(m->master); cudaFree(m->wbf); cudaFree(m->grad); cudaFree(m->m); cudaFree(m->v); cudaFree(m->loss);
    if (m->h_small) cudaFreeHost(m->h_small);
    delete m;
    return rc;
  };
  if (cudaGetDevice(&m->device) != cudaSuccess) return fail(MC_ERR_CUDA);
  cudaDeviceGetAttribute(&m->sm_count, cudaDevAttrMultiProcessorCount, m->device);
  if (cudaMalloc(&m->master, kParams * 4) != cudaSuccess || cudaMalloc(&m->wbf, kParams * 2) != cudaSuccess ||
      cudaMalloc(&m->grad, kParams * 4) != cudaSuccess || cudaMalloc(&m->m, kParams * 4) != cudaSuccess ||
      cudaMalloc(&m->v, kParams * 4) != cudaSuccess || cudaMalloc(&m->loss, 16) != cudaSuccess ||
      cudaMallocHost(&m->h_small, 4096) != cudaSuccess)
    return fail(MC_ERR_OOM);
  // He-uniform initial weights from a counter-based generator, zero biases
  std::vector<float> p(kParams, 0.f);
  uint64_t ctr = seed * 0x9E3779B97F4A7C15ULL + 1;
  auto uni = [&]() { return (double)(splitmix(ctr++) >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0; };
  for (int i = 0; i < kH * kF; i++) p[kOffW1 + i] = (float)(uni() * std::sqrt(6.0 / kF));
  for (int i = 0; i < kH * kH; i++) p[kOffW2 + i] = (float)(uni() * std::sqrt(6.0 / kH));
  for (int i = 0; i < kH; i++) p[kOffW3 + i] = (float)(uni() * std::sqrt(6.0 / kH));
  if (cudaMemcpyAsync(m->master, p.data(), kParams * 4, cudaMemcpyHostToDevice, m->stream) != cudaSuccess)
    return fail(MC_ERR_CUDA);
  cudaMemsetAsync(m->m, 0, kParams * 4, m->stream);
  cudaMemsetAsync(m->v, 0, kParams * 4, m->stream);
  round_kernel<<<(kParams + 255) / 256, 256, 0, m->stream>>>(m->master, m->wbf);
  g_launches++;
  if (cudaStreamSynchronize(m->stream) != cudaSuccess) return fail(MC_ERR_CUDA);
  *out = m;
  return MC_OK;
}

void mc_mlp_free(mc_mlp *m) {
  if (!m) return;
  cudaStreamSynchronize(m->stream);
  cudaFree(m->master); cudaFree(m->wbf); cudaFree(m->grad); cudaFree(m->m); cudaFree(m->v); cudaFree(m->loss);
  cudaFree(m->buf);
  if (m->h_small) cudaFreeHost(m->h_small);
  delete m;
}

int mc_mlp_num_params(void) { return kParams; }

int mc_mlp_get_params(mc_mlp *m, float *out) {
  if (!m || !out) return MC_ERR_ARG;
  MC_CUDA_TRY(cudaMemcpyAsync(out, m->master, kParams * 4, cudaMemcpyDefault, m->stream));
  MC_CUDA_TRY(cudaStreamSynchronize(m->stream));
  return MC_OK;
}

int mc_mlp_set_params(mc_mlp *m, const float *in) {
  if (!m || !in) return MC_ERR_ARG;
  MC_CUDA_TRY(cudaMemcpyAsync(m->master, in, kParams * 4, cudaMemcpyDefault, m->stream));
  MC_CUDA_TRY(cudaMemsetAsync(m->m, 0, kParams * 4, m->stream));
  MC_CUDA_TRY(cudaMemsetAsync(m->v, 0, kParams * 4, m->stream));
  round_kernel<<<(kParams + 255) / 256, 256, 0, m->stream>>>(m->master, m->wbf);
  g_launches++;
  m->step = 0;
  MC_CUDA_TRY(cudaStreamSynchronize(m->stream));
  return MC_OK;
}

int mc_features(mc_graph *g, float *feat_out) {
  if (!g || (g->n > 0 && !feat_out)) return MC_ERR_ARG;
  if (g->n == 0) return MC_OK;
  if (!g->cores_valid) MC_TRY(launch_core_numbers(g, kDefaultSpinLimit));
  float *dst = feat_out;
  void *p = nullptr;
  const bool dev_out = is_device_ptr(feat_out);
  if (!dev_out) {
    MC_TRY(ws_get(g, "ln.feat", (size_t)g->n * kF * 4, &p));
    dst = (float *)p;
  }
  const float kmax = (float)std::max(g->max_core, 1);
  const float ldmax = log1pf((float)std::max(g->max_degree, 1));
  const int blocks = (int)std::min<int64_t>((g->n * 32 + 255) / 256, (int64_t)g->sm_count * 16);
  features_kernel<<<blocks, 256, 0, g->stream>>>(g->n, nullptr, nullptr, g->row_ptr, g->col_idx, g->core, kmax,
                                                 ldmax, dst);
  g_launches++;
  MC_CUDA_TRY(cudaGetLastError());
  if (!dev_out) MC_CUDA_TRY(cudaMemcpyAsync(feat_out, dst, (size_t)g->n * kF * 4, cudaMemcpyDeviceToHost, g->stream));
  MC_CUDA_TRY(cudaStreamSynchronize(g->stream));
  return MC_OK;
}

int mc_mlp_forward(mc_mlp *m, const float *feat, int64_t n, float *score_out) {
  if (!m || n < 0 || (n > 0 && (!feat || !score_out))) return MC_ERR_ARG;
  if (n == 0) return MC_OK;
  const void *df;
  MC_TRY(stage(m, feat, (size_t)n * kF * 4, &df));
  float *out = score_out;
  const bool dev_out = is_device_ptr(score_out);
  float *tmp = nullptr;
  if (!dev_out) {
    MC_CUDA_TRY(cudaMallocAsync((void **)&tmp, (size_t)n * 4, m->stream));
    out = tmp;
  }
  const int blocks = (int)std::min<int64_t>((n * 32 + 255) / 256, (int64_t)m->sm_count * 16);
  forward_kernel<<<blocks, 256, 0, m->stream>>>(n, (const float *)df, m->wbf, m->master, out);
  g_launches++;
  MC_CUDA_TRY(cudaGetLastError());
  if (!dev_out) {
    MC_CUDA_TRY(cudaMemcpyAsync(score_out, tmp, (size_t)n * 4, cudaMemcpyDeviceToHost, m->stream));
    MC_CUDA_TRY(cudaFreeAsync(tmp, m->stream));
  }
  MC_CUDA_TRY(cudaStreamSynchronize(m->stream));
  return MC_OK;
}

static int run_grad(mc_mlp *m, const float *feat, const float *label, int64_t n, float pos_weight) {
  const void *df, *dl;
  // features and labels are staged separately (labels after the features)
  if (is_device_ptr(feat) && is_device_ptr(label)) {
    df = feat;
    dl = label;
  } else {
    const size_t fb = (size_t)n * kF * 4, lb = (size_t)n * 4;
    if (m->buf_bytes < fb + lb) {
      if (m->buf) {
        MC_CUDA_TRY(cudaStreamSynchronize(m->stream));
        cudaFree(m->buf);
      }
      m->buf = nullptr;
      m->buf_bytes = 0;
      MC_CUDA_TRY(cudaMalloc(&m->buf, fb + lb));
      m->buf_bytes = fb + lb;
    }
    MC_CUDA_TRY(cudaMemcpyAsync(m->buf, feat, fb, cudaMemcpyDefault, m->stream));
    MC_CUDA_TRY(cudaMemcpyAsync((char *)m->buf + fb, label, lb, cudaMemcpyDefault, m->stream));
    df = m->buf;
    dl = (char *)m->buf + fb;
  }
  MC_CUDA_TRY(cudaMemsetAsync(m->grad, 0, kParams * 4, m->stream));
  MC_CUDA_TRY(cudaMemsetAsync(m->loss, 0, 4, m->stream));
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((n + kGT - 1) / kGT, (int64_t)m->sm_count * 4));
  MC_CUDA_TRY(cudaFuncSetAttribute(grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(GradSmem)));
  grad_kernel<<<blocks, kGT, sizeof(GradSmem), m->stream>>>(n, (const float *)df, (const float *)dl, pos_weight, m->wbf,
                                                            m->master, m->grad, m->loss);
  g_launches++;
  MC_CUDA_TRY(cudaGetLastError());
  return MC_OK;
}

int mc_mlp_gradient(mc_mlp *m, const float *feat, const float *label, int64_t n, float pos_weight, float *grad_out,
                    float *loss_out) {
  if (!m || n <= 0 || !feat || !label || !grad_out) return MC_ERR_ARG;
  MC_TRY(run_grad(m, feat, label, n, pos_weight));
  MC_CUDA_TRY(cudaMemcpyAsync(grad_out, m->grad, kParams * 4, cudaMemcpyDefault, m->stream));
  float *hl = (float *)m->h_small;
  MC_CUDA_TRY(cudaMemcpyAsync(hl, m->loss, 4, cudaMemcpyDeviceToHost, m->stream));
  MC_CUDA_TRY(cudaStreamSynchronize(m->stream));
  if (loss_out) *loss_out = *hl;
  return MC_OK;
}

int mc_mlp_train_step(mc_mlp *m, const float *feat, const float *label, int64_t n, float pos_weight, float lr,
                      float *loss_out) {
  if (!m || n <= 0 || !feat || !label || !(lr > 0.f)) return MC_ERR_ARG;
  MC_TRY(run_grad(m, feat, label, n, pos_weight));
  m->step++;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)m->step), c2 = 1.f - powf(b2, (float)m->step);
  adam_kernel<<<(kParams + 255) / 256, 256, 0, m->stream>>>(m->master, m->wbf, m->grad, m->m, m->v, lr, b1, b2, 1e-8f,
                                                            c1, c2);
  g_launches++;
  MC_CUDA_TRY(cudaGetLastError());
  float *hl = (float *)m->h_small;
  MC_CUDA_TRY(cudaMemcpyAsync(hl, m->loss, 4, cudaMemcpyDeviceToHost, m->stream));
  MC_CUDA_TRY(cudaStreamSynchronize(m->stream));
  if (loss_out) *loss_out = *hl;
  return MC_OK;
}

}  // extern "C"
