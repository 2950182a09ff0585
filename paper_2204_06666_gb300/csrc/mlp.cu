// The tuner network: a 3-layer perceptron 16 -> 64 -> 64 -> 4 (ReLU after the hidden layers, linear
// output), FP32, with hand-written forward, mean-squared-error backward and Adam kernels.  It is not in
// the paper: it is the learned-knob subsystem built around the method (it predicts the partition size
// of Eq. 1/2, the slab width cap and the lanes per row).
//
// Parameters are one flat array in this order (row-major): W1 (64x16), b1 (64), W2 (64x64), b2 (64),
// W3 (4x64), b3 (4) -- 5,508 floats.  A batch X is B x 16 row-major, targets T and outputs B x 4.
// Every reduction (over the batch for weight gradients, over the outputs for the loss) runs in a fixed
// order, so gradients and training runs are bit-reproducible.  The kernels are tiny; they are written
// for clarity and determinism, one thread per output element.
#include <cuda_runtime.h>

#include <cstdint>

#include "plan_internal.h"

namespace ehyb {
namespace {

constexpr int D0 = 16, D1 = 64, D2 = 64, D3 = 4;
constexpr int OW1 = 0, OB1 = OW1 + D1 * D0, OW2 = OB1 + D1, OB2 = OW2 + D2 * D1, OW3 = OB2 + D2, OB3 = OW3 + D3 * D2;
constexpr int NPARAM = OB3 + D3;
static_assert(NPARAM == 5508, "parameter count");

// out[b][o] = act(sum_i W[o][i] in[b][i] + bias[o]); z (pre-activation) kept for the backward pass
__global__ void dense_forward(const float* __restrict__ W, const float* __restrict__ bias, const float* __restrict__ in,
                              int B, int K, int N, float* __restrict__ z, float* __restrict__ out, int relu) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= B * N) return;
  const int b = t / N, o = t - b * N;
  float s = bias[o];
  for (int i = 0; i < K; ++i) s = fmaf(W[o * K + i], in[b * K + i], s);
  if (z) z[t] = s;
  out[t] = (relu && s < 0.0f) ? 0.0f : s;
}

// d_out[b][j] = 2 (out - T) / (B * 4); per-sample squared errors for the loss
__global__ void mse_grad(const float* __restrict__ out, const float* __restrict__ T, int B, float* __restrict__ dout,
                         float* __restrict__ sq) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= B * D3) return;
  const float e = out[t] - T[t];
  dout[t] = 2.0f * e / (float)(B * D3);
  sq[t] = e * e;
}

// loss = sum(sq) / (B * 4), one block, fixed order
__global__ void loss_reduce(const float* __restrict__ sq, int count, float* loss) {
  __shared__ double ws[32];
  double v = 0.0;
  for (int i = threadIdx.x; i < count; i += blockDim.x) v += (double)sq[i];
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += ws[w];
    *loss = (float)(s / (double)count);
  }
}

// gW[o][i] = sum_b dz[b][o] in[b][i]; gb[o] = sum_b dz[b][o]   (thread per weight, batch order fixed)
__global__ void dense_wgrad(const float* __restrict__ dz, const float* __restrict__ in, int B, int K, int N,
                            float* __restrict__ gW, float* __restrict__ gb) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < N * K) {
    const int o = t / K, i = t - o * K;
    float s = 0.0f;
    for (int b = 0; b < B; ++b) s = fmaf(dz[b * N + o], in[b * K + i], s);
    gW[t] = s;
  } else if (t < N * K + N) {
    const int o = t - N * K;
    float s = 0.0f;
    for (int b = 0; b < B; ++b) s += dz[b * N + o];
    gb[o] = s;
  }
}

// din[b][i] = (sum_o dz[b][o] W[o][i]) * [z_in[b][i] > 0]   (back through the previous ReLU)
__global__ void dense_igrad(const float* __restrict__ dz, const float* __restrict__ W, const float* __restrict__ z_in,
                            int B, int K, int N, float* __restrict__ din) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= B * K) return;
  const int b = t / K, i = t - b * K;
  float s = 0.0f;
  for (int o = 0; o < N; ++o) s = fmaf(dz[b * N + o], W[o * K + i], s);
  din[t] = z_in[t] > 0.0f ? s : 0.0f;
}

__global__ void adam_kernel(float* p, float* m, float* v, const float* __restrict__ g, int count, float lr,
                            float b1, float b2, float eps, float c1, float c2) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= count) return;
  const float gi = g[t];
  const float mi = b1 * m[t] + (1.0f - b1) * gi;
  const float vi = b2 * v[t] + (1.0f - b2) * gi * gi;
  m[t] = mi;
  v[t] = vi;
  p[t] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

inline int nblk(int64_t work) { return (int)((work + 255) / 256); }

struct Ws {  // activations of one batch, carved from the caller's workspace
  float *z1, *h1, *z2, *h2, *out, *dout, *sq, *d2, *d1;
};

Ws carve(void* ws, int B) {
  float* f = (float*)ws;
  Ws w;
  w.z1 = f; f += (size_t)B * D1;
  w.h1 = f; f += (size_t)B * D1;
  w.z2 = f; f += (size_t)B * D2;
  w.h2 = f; f += (size_t)B * D2;
  w.out = f; f += (size_t)B * D3;
  w.dout = f; f += (size_t)B * D3;
  w.sq = f; f += (size_t)B * D3;
  w.d2 = f; f += (size_t)B * D2;
  w.d1 = f;
  return w;
}

void forward(const float* P, const float* X, int B, const Ws& w, float* out, cudaStream_t s) {
  dense_forward<<<nblk((int64_t)B * D1), 256, 0, s>>>(P + OW1, P + OB1, X, B, D0, D1, w.z1, w.h1, 1);
  dense_forward<<<nblk((int64_t)B * D2), 256, 0, s>>>(P + OW2, P + OB2, w.h1, B, D1, D2, w.z2, w.h2, 1);
  dense_forward<<<nblk((int64_t)B * D3), 256, 0, s>>>(P + OW3, P + OB3, w.h2, B, D2, D3, nullptr, out, 0);
}

}  // namespace
}  // namespace ehyb

using namespace ehyb;

extern "C" int32_t ehyb_mlp_param_count(void) { return NPARAM; }

extern "C" int64_t ehyb_mlp_workspace_bytes(int32_t batch) {
  if (batch < 0) return -1;
  return (int64_t)batch * (2 * D1 + 2 * D2 + 3 * D3 + D2 + D1) * (int64_t)sizeof(float);
}

extern "C" ehyb_status_t ehyb_mlp_forward(const float* params, const float* X, int32_t batch, float* out,
                                          void* workspace, void* stream) {
  if (!params || !X || !out || batch < 0 || (batch > 0 && !workspace)) return EHYB_ERR_INVALID_ARG;
  if (batch == 0) return EHYB_OK;
  Ws w = carve(workspace, batch);
  forward(params, X, batch, w, out, (cudaStream_t)stream);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? EHYB_OK : cuda_error_status(e, "mlp forward");
}

extern "C" ehyb_status_t ehyb_mlp_loss_grad(const float* params, const float* X, const float* T, int32_t batch,
                                            float* grad, float* loss, void* workspace, void* stream) {
  if (!params || !X || !T || !grad || !loss || batch <= 0 || !workspace) return EHYB_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  Ws w = carve(workspace, batch);
  const int B = batch;
  forward(params, X, B, w, w.out, s);
  mse_grad<<<nblk((int64_t)B * D3), 256, 0, s>>>(w.out, T, B, w.dout, w.sq);
  loss_reduce<<<1, 256, 0, s>>>(w.sq, B * D3, loss);
  // layer 3
  dense_wgrad<<<nblk((int64_t)D3 * D2 + D3), 256, 0, s>>>(w.dout, w.h2, B, D2, D3, grad + OW3, grad + OB3);
  dense_igrad<<<nblk((int64_t)B * D2), 256, 0, s>>>(w.dout, params + OW3, w.z2, B, D2, D3, w.d2);
  // layer 2
  dense_wgrad<<<nblk((int64_t)D2 * D1 + D2), 256, 0, s>>>(w.d2, w.h1, B, D1, D2, grad + OW2, grad + OB2);
  dense_igrad<<<nblk((int64_t)B * D1), 256, 0, s>>>(w.d2, params + OW2, w.z1, B, D1, D2, w.d1);
  // layer 1
  dense_wgrad<<<nblk((int64_t)D1 * D0 + D1), 256, 0, s>>>(w.d1, X, B, D0, D1, grad + OW1, grad + OB1);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? EHYB_OK : cuda_error_status(e, "mlp backward");
}

extern "C" ehyb_status_t ehyb_mlp_adam(float* params, float* m, float* v, const float* grad, int32_t step, float lr,
                                       float beta1, float beta2, float eps, void* stream) {
  if (!params || !m || !v || !grad || step < 1) return EHYB_ERR_INVALID_ARG;
  const float c1 = 1.0f - powf(beta1, (float)step), c2 = 1.0f - powf(beta2, (float)step);
  adam_kernel<<<nblk(NPARAM), 256, 0, (cudaStream_t)stream>>>(params, m, v, grad, NPARAM, lr, beta1, beta2, eps, c1,
                                                              c2);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? EHYB_OK : cuda_error_status(e, "mlp adam");
}
