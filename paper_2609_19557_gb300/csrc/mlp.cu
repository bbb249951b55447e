// Learned inner-solve controller: the MLP 16 -> 64 -> 64 -> 2 (GELU hidden
// layers) that proposes the inner tolerance factor rho_in (in place of Eq.
// inner-tolerance-factor) and the primal weight carried into the next inner
// solve (in place of the restart value of Eq. primal-weight-update).  BF16
// weights, FP32 arithmetic.  Hand-written inference and training kernels:
// forward (with the pre-activations kept for the backward pass), weighted
// squared-error gradient, backward (per-block partial gradients, reduced in
// a fixed order: deterministic), and Adam on FP32 master weights that
// refreshes the BF16 copy.  Sizes are tiny (5,378 parameters), so every
// kernel keeps the whole network in shared memory.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <string>

#include "../../include/pdnqp.h"

namespace pdq {
namespace {

constexpr int kIn = 16, kHid = 64, kOut = 2;
// Parameter layout (row-major, out x in): W1[64][16], b1[64], W2[64][64],
// b2[64], W3[2][64], b3[2].
constexpr int oW1 = 0, oB1 = oW1 + kHid * kIn, oW2 = oB1 + kHid, oB2 = oW2 + kHid * kHid, oW3 = oB2 + kHid,
              oB3 = oW3 + kOut * kHid, kParams = oB3 + kOut;
constexpr int kCache = 2 * kHid;       // z1, z2 per sample
constexpr int kSamplesPerBlock = 16;   // samples handled by one block
constexpr int kMaxGradBlocks = 1 << 16;  // partial-gradient rows (batches up to 1,048,576 samples)

static thread_local std::string g_mlp_err;

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_d(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

__device__ __forceinline__ void load_params(float *w, const __nv_bfloat16 *wb) {
  for (int p = threadIdx.x; p < kParams; p += blockDim.x) w[p] = __bfloat162float(wb[p]);
  __syncthreads();
}

// One block of kHid threads, kSamplesPerBlock samples per block.
__global__ void __launch_bounds__(kHid) k_mlp_forward(const __nv_bfloat16 *wb, const float *x, int B, float *y,
                                                      float *cache) {
  __shared__ float w[kParams];
  __shared__ float xs[kIn], h1[kHid], h2[kHid];
  load_params(w, wb);
  const int j = threadIdx.x;
  const int s0 = blockIdx.x * kSamplesPerBlock;
  for (int s = s0; s < s0 + kSamplesPerBlock && s < B; ++s) {
    if (j < kIn) xs[j] = x[(size_t)s * kIn + j];
    __syncthreads();
    float z1 = w[oB1 + j];
    for (int i = 0; i < kIn; ++i) z1 += w[oW1 + j * kIn + i] * xs[i];
    h1[j] = gelu(z1);
    __syncthreads();
    float z2 = w[oB2 + j];
    for (int k = 0; k < kHid; ++k) z2 += w[oW2 + j * kHid + k] * h1[k];
    h2[j] = gelu(z2);
    if (cache) {
      cache[(size_t)s * kCache + j] = z1;
      cache[(size_t)s * kCache + kHid + j] = z2;
    }
    __syncthreads();
    if (j < kOut) {
      float o = w[oB3 + j];
      for (int k = 0; k < kHid; ++k) o += w[oW3 + j * kHid + k] * h2[k];
      y[(size_t)s * kOut + j] = o;
    }
    __syncthreads();
  }
}

// Weighted squared error L = sum_s w_s ||y_s - t_s||^2 / sum_s w_s and its
// gradient dL/dy (single block, fixed order).
__global__ void __launch_bounds__(256) k_mlp_wmse(const float *y, const float *t, const float *wt, int B, float *dy,
                                                  float *loss) {
  __shared__ double red[2][256];
  double a = 0.0, sw = 0.0;
  for (int s = threadIdx.x; s < B; s += blockDim.x) {
    const double ws = wt ? (double)wt[s] : 1.0;
    sw += ws;
    for (int o = 0; o < kOut; ++o) {
      const double e = (double)y[(size_t)s * kOut + o] - (double)t[(size_t)s * kOut + o];
      a += ws * e * e;
    }
  }
  red[0][threadIdx.x] = a;
  red[1][threadIdx.x] = sw;
  __syncthreads();
  if (threadIdx.x == 0) {
    double A = 0.0, W = 0.0;
    for (int k = 0; k < (int)blockDim.x; ++k) {
      A += red[0][k];
      W += red[1][k];
    }
    red[0][0] = A;
    red[1][0] = W > 0.0 ? W : 1.0;
    if (loss) *loss = (float)(A / red[1][0]);
  }
  __syncthreads();
  const float inv = (float)(2.0 / red[1][0]);
  for (int s = threadIdx.x; s < B; s += blockDim.x) {
    const float ws = wt ? wt[s] : 1.0f;
    for (int o = 0; o < kOut; ++o)
      dy[(size_t)s * kOut + o] = inv * ws * (y[(size_t)s * kOut + o] - t[(size_t)s * kOut + o]);
  }
}

// Backward pass: block b accumulates the gradient of its samples (thread j
// owns the rows j of W1, W2, entries j of b1, b2 and column j of W3, so no
// two threads write the same accumulator) and writes it to part[b].
__global__ void __launch_bounds__(kHid) k_mlp_backward(const __nv_bfloat16 *wb, const float *x, const float *cache,
                                                       const float *dy, int B, float *part) {
  __shared__ float w[kParams];
  __shared__ float g[kParams];
  __shared__ float xs[kIn], h1[kHid], dz2[kHid], dys[kOut];
  load_params(w, wb);
  for (int p = threadIdx.x; p < kParams; p += blockDim.x) g[p] = 0.0f;
  __syncthreads();
  const int j = threadIdx.x;
  const int s0 = blockIdx.x * kSamplesPerBlock;
  for (int s = s0; s < s0 + kSamplesPerBlock && s < B; ++s) {
    if (j < kIn) xs[j] = x[(size_t)s * kIn + j];
    if (j < kOut) dys[j] = dy[(size_t)s * kOut + j];
    const float z1 = cache[(size_t)s * kCache + j], z2 = cache[(size_t)s * kCache + kHid + j];
    h1[j] = gelu(z1);
    __syncthreads();
    const float h2j = gelu(z2);
    // Output layer.
    float dh2 = 0.0f;
    for (int o = 0; o < kOut; ++o) {
      g[oW3 + o * kHid + j] += dys[o] * h2j;
      dh2 += w[oW3 + o * kHid + j] * dys[o];
    }
    if (j < kOut) g[oB3 + j] += dys[j];
    const float d2 = dh2 * gelu_d(z2);
    dz2[j] = d2;
    __syncthreads();
    // Second hidden layer.
    for (int k = 0; k < kHid; ++k) g[oW2 + j * kHid + k] += d2 * h1[k];
    g[oB2 + j] += d2;
    float dh1 = 0.0f;
    for (int r = 0; r < kHid; ++r) dh1 += w[oW2 + r * kHid + j] * dz2[r];
    const float d1 = dh1 * gelu_d(z1);
    // First hidden layer.
    for (int i = 0; i < kIn; ++i) g[oW1 + j * kIn + i] += d1 * xs[i];
    g[oB1 + j] += d1;
    __syncthreads();
  }
  __syncthreads();
  for (int p = threadIdx.x; p < kParams; p += blockDim.x) part[(size_t)blockIdx.x * kParams + p] = g[p];
}

// grad[p] = sum over blocks of part[b][p] in block order.
__global__ void k_mlp_grad_reduce(const float *part, int nb, float *grad) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= kParams) return;
  float a = 0.0f;
  for (int b = 0; b < nb; ++b) a += part[(size_t)b * kParams + p];
  grad[p] = a;
}

// Adam (Kingma & Ba) on the FP32 master weights; the BF16 copy is refreshed
// by round-to-nearest-even.
__global__ void k_mlp_adam(float *w, __nv_bfloat16 *wb, const float *g, float *m, float *v, float lr, float b1,
                           float b2, float eps, float c1, float c2) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= kParams) return;
  const float gp = g[p];
  const float mp = b1 * m[p] + (1.0f - b1) * gp;
  const float vp = b2 * v[p] + (1.0f - b2) * gp * gp;
  m[p] = mp;
  v[p] = vp;
  const float wp = w[p] - lr * (mp / c1) / (sqrtf(vp / c2) + eps);
  w[p] = wp;
  wb[p] = __float2bfloat16_rn(wp);
}

__global__ void k_mlp_to_bf16(const float *w, __nv_bfloat16 *wb, int n) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < n) wb[p] = __float2bfloat16_rn(w[p]);
}

int fail(const char *msg) {
  g_mlp_err = msg;
  return PDNQP_ERR_ARG;
}
int check_launch(const char *what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    g_mlp_err = std::string(what) + ": " + cudaGetErrorString(e);
    return PDNQP_ERR_CUDA;
  }
  return 0;
}
int blocks_for(int B) { return (B + kSamplesPerBlock - 1) / kSamplesPerBlock; }

}  // namespace
}  // namespace pdq

extern "C" {

int pdnqp_mlp_param_count(void) { return pdq::kParams; }

int pdnqp_mlp_forward(const uint16_t *w_bf16, const float *x, int batch, float *y, float *cache, void *stream) {
  using namespace pdq;
  if (!w_bf16 || !x || !y || batch < 0) return fail("NULL argument or negative batch");
  if (batch == 0) return 0;
  k_mlp_forward<<<blocks_for(batch), kHid, 0, (cudaStream_t)stream>>>((const __nv_bfloat16 *)w_bf16, x, batch, y,
                                                                       cache);
  return check_launch("k_mlp_forward");
}

int pdnqp_mlp_wmse(const float *y, const float *target, const float *weight, int batch, float *dy, float *loss,
                   void *stream) {
  using namespace pdq;
  if (!y || !target || !dy || batch < 0) return fail("NULL argument or negative batch");
  if (batch == 0) return 0;
  k_mlp_wmse<<<1, 256, 0, (cudaStream_t)stream>>>(y, target, weight, batch, dy, loss);
  return check_launch("k_mlp_wmse");
}

int pdnqp_mlp_backward(const uint16_t *w_bf16, const float *x, const float *cache, const float *dy, int batch,
                       float *grad, float *scratch, void *stream) {
  using namespace pdq;
  if (!w_bf16 || !x || !cache || !dy || !grad || !scratch || batch < 0) return fail("NULL argument");
  const int nb = blocks_for(batch);
  if (nb > kMaxGradBlocks) return fail("batch too large (at most 65536 x 16 samples)");
  cudaStream_t s = (cudaStream_t)stream;
  if (batch == 0) return cudaMemsetAsync(grad, 0, sizeof(float) * kParams, s) == cudaSuccess ? 0 : PDNQP_ERR_CUDA;
  k_mlp_backward<<<nb, kHid, 0, s>>>((const __nv_bfloat16 *)w_bf16, x, cache, dy, batch, scratch);
  int rc = check_launch("k_mlp_backward");
  if (rc) return rc;
  k_mlp_grad_reduce<<<(kParams + 255) / 256, 256, 0, s>>>(scratch, nb, grad);
  return check_launch("k_mlp_grad_reduce");
}

int pdnqp_mlp_adam(float *w, uint16_t *w_bf16, const float *grad, float *m, float *v, int step, float lr, float beta1,
                   float beta2, float eps, void *stream) {
  using namespace pdq;
  if (!w || !w_bf16 || !grad || !m || !v || step < 1) return fail("NULL argument or step < 1");
  const float c1 = 1.0f - powf(beta1, (float)step), c2 = 1.0f - powf(beta2, (float)step);
  k_mlp_adam<<<(kParams + 255) / 256, 256, 0, (cudaStream_t)stream>>>(w, (__nv_bfloat16 *)w_bf16, grad, m, v, lr,
                                                                     beta1, beta2, eps, c1, c2);
  return check_launch("k_mlp_adam");
}

int pdnqp_mlp_to_bf16(const float *w, uint16_t *w_bf16, int count, void *stream) {
  using namespace pdq;
  if (!w || !w_bf16 || count < 0) return fail("NULL argument");
  if (count == 0) return 0;
  k_mlp_to_bf16<<<(count + 255) / 256, 256, 0, (cudaStream_t)stream>>>(w, (__nv_bfloat16 *)w_bf16, count);
  return check_launch("k_mlp_to_bf16");
}

const char *pdnqp_mlp_last_error(void) { return pdq::g_mlp_err.c_str(); }

}  // extern "C"
