// Learned vertex ordering: per-vertex features and a 6 -> 64 -> 64 -> 1 MLP
// (ReLU, BF16 weights, FP32 accumulation, FP32 master weights and Adam).
// The score only orders the search's roots and seeds the heuristic; omega
// stays exact whatever the network predicts.
//
// Features of vertex v (d = degree, K = core number, Kmax = K(G), Dmax =
// maximum degree, c = number of neighbours with K >= K(v)):
//   f0 = log1p(d) / log1p(Dmax)        f3 = max_{u in N(v)} K(u) / Kmax
//   f1 = K(v) / Kmax                   f4 = mean_{u in N(v)} K(u) / Kmax
//   f2 = log1p(c) / log1p(Dmax)        f5 = c / max(d, 1)
// All are one pass over the CSR (warp per vertex).
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

__global__ void features_kernel(int64_t n, const int64_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                const int32_t *__restrict__ core, float kmax, float ldmax, float *__restrict__ f) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t v = w0; v < n; v += nw) {
    const int kv = core[v];
    const int64_t e0 = rp[v], e1 = rp[v + 1];
    int c = 0, mx = 0;
    long long sum = 0;
    for (int64_t e = e0 + lane; e < e1; e += 32) {
      const int k = core[ci[e]];
      c += k >= kv ? 1 : 0;
      mx = max(mx, k);
      sum += k;
    }
    c = dev::warp_sum(c);
    mx = dev::warp_max(mx);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (lane == 0) {
      const float d = (float)(e1 - e0);
      float *o = f + v * kF;
      o[0] = log1pf(d) / ldmax;
      o[1] = (float)kv / kmax;
      o[2] = log1pf((float)c) / ldmax;
      o[3] = (float)mx / kmax;
      o[4] = d > 0 ? (float)((double)sum / (double)d) / kmax : 0.f;
      o[5] = (float)c / fmaxf(d, 1.f);
    }
  }
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

// forward for one row: returns the logit; h1 in registers
__device__ __forceinline__ float forward_row(const float *sw, const float *x, float *h1) {
#pragma unroll
  for (int j = 0; j < kH; j++) {
    float z = sw[kOffB1 + j];
#pragma unroll
    for (int i = 0; i < kF; i++) z = fmaf(sw[kOffW1 + j * kF + i], x[i], z);
    h1[j] = fmaxf(z, 0.f);
  }
  float s = sw[kOffB3];
  for (int j = 0; j < kH; j++) {
    float z = sw[kOffB2 + j];
#pragma unroll
    for (int k = 0; k < kH; k++) z = fmaf(sw[kOffW2 + j * kH + k], h1[k], z);
    s = fmaf(sw[kOffW3 + j], fmaxf(z, 0.f), s);
  }
  return s;
}

__global__ void __launch_bounds__(256) forward_kernel(int64_t n, const float *__restrict__ feat,
                                                      const uint16_t *__restrict__ wbf,
                                                      const float *__restrict__ master, float *__restrict__ out) {
  __shared__ float sw[kParams];
  load_weights(wbf, master, sw);
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
    float x[kF], h1[kH];
#pragma unroll
    for (int i = 0; i < kF; i++) x[i] = feat[r * kF + i];
    out[r] = forward_row(sw, x, h1);
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

}  // namespace
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
  features_kernel<<<blocks, 256, 0, g->stream>>>(g->n, g->row_ptr, g->col_idx, g->core, kmax, ldmax, dst);
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
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, (int64_t)m->sm_count * 8);
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
