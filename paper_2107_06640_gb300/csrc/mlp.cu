// Friction-guess network: training kernels (forward + backward + Adam), FP32.
//
// The network maps per-solve features of the rate-and-state Newton problem to
// a guess of x* = ln |V| (see rupture.cu for the features):
//   x = (f - mu)/sd,  h1 = tanh(W1 x + b1),  h2 = tanh(W2 h1 + b2),
//   y = w3 . h2 + b3,  guess = x_a + shift + scale * y.
// Parameter vector layout (MLP_NPARAM floats): W1[H][IN], b1[H], W2[H][H],
// b2[H], w3[H], b3, mu[IN], sd[IN], shift, scale.  Only W1..b3 are trained;
// mu/sd/shift/scale are fixed from the captured samples.  A sample row is
// [f_0 .. f_5, z] with z = x* - x_a; the loss is mean((y - (z-shift)/scale)^2).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "kernels.cuh"

namespace adg {

constexpr int kTrainable = MLP_IN * MLP_H + MLP_H + MLP_H * MLP_H + MLP_H + MLP_H + 1;

__global__ void __launch_bounds__(128) mlp_grad_kernel(const float* __restrict__ P, const float* __restrict__ rows,
                                                        int64_t row0, int64_t n, float inv_n, float* __restrict__ grad,
                                                        double* __restrict__ loss) {
  __shared__ float sg[kTrainable];
  __shared__ float sl[128];
  for (int i = threadIdx.x; i < kTrainable; i += blockDim.x) sg[i] = 0.f;
  __syncthreads();
  const float* W1 = P;
  const float* b1 = W1 + MLP_IN * MLP_H;
  const float* W2 = b1 + MLP_H;
  const float* b2 = W2 + MLP_H * MLP_H;
  const float* w3 = b2 + MLP_H;
  const float* b3 = w3 + MLP_H;
  const float* mu = b3 + 1;
  const float* sd = mu + MLP_IN;
  const float* osc = sd + MLP_IN;
  float* gW1 = sg;
  float* gb1 = gW1 + MLP_IN * MLP_H;
  float* gW2 = gb1 + MLP_H;
  float* gb2 = gW2 + MLP_H * MLP_H;
  float* gw3 = gb2 + MLP_H;
  float* gb3 = gw3 + MLP_H;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  float lval = 0.f;
  if (i < n) {
    const float* r = rows + (row0 + i) * (MLP_IN + 1);
    float x[MLP_IN], h1[MLP_H], h2[MLP_H];
    for (int k = 0; k < MLP_IN; ++k) x[k] = (r[k] - mu[k]) / sd[k];
    for (int j = 0; j < MLP_H; ++j) {
      float s = b1[j];
      for (int k = 0; k < MLP_IN; ++k) s += W1[j * MLP_IN + k] * x[k];
      h1[j] = tanhf(s);
    }
    float y = b3[0];
    for (int j = 0; j < MLP_H; ++j) {
      float s = b2[j];
      for (int k = 0; k < MLP_H; ++k) s += W2[j * MLP_H + k] * h1[k];
      h2[j] = tanhf(s);
      y += w3[j] * h2[j];
    }
    const float t = (r[MLP_IN] - osc[0]) / osc[1];
    const float res = y - t;
    lval = res * res;
    const float dy = 2.f * res * inv_n;
    atomicAdd(gb3, dy);
    float dh1[MLP_H];
    for (int j = 0; j < MLP_H; ++j) dh1[j] = 0.f;
    for (int k = 0; k < MLP_H; ++k) {
      atomicAdd(&gw3[k], dy * h2[k]);
      const float da2 = dy * w3[k] * (1.f - h2[k] * h2[k]);
      atomicAdd(&gb2[k], da2);
      for (int j = 0; j < MLP_H; ++j) {
        atomicAdd(&gW2[k * MLP_H + j], da2 * h1[j]);
        dh1[j] += W2[k * MLP_H + j] * da2;
      }
    }
    for (int j = 0; j < MLP_H; ++j) {
      const float da1 = dh1[j] * (1.f - h1[j] * h1[j]);
      atomicAdd(&gb1[j], da1);
      for (int k = 0; k < MLP_IN; ++k) atomicAdd(&gW1[j * MLP_IN + k], da1 * x[k]);
    }
  }
  sl[threadIdx.x] = lval;
  __syncthreads();
  for (int s = 64; s > 0; s >>= 1) {
    if (threadIdx.x < s) sl[threadIdx.x] += sl[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(loss, (double)sl[0] * inv_n);
  for (int k = threadIdx.x; k < kTrainable; k += blockDim.x) atomicAdd(&grad[k], sg[k]);
}

__global__ void adam_kernel(float* P, const float* g, float* m, float* v, float lr, float b1, float b2, float eps,
                            float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kTrainable) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  P[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

int mlp_trainable() { return kTrainable; }

// grad (kTrainable floats) and loss (double) must be zeroed by the caller.
int launch_mlp_grad(const float* P, const float* rows, int64_t row0, int64_t n, int64_t n_norm, float* grad,
                    double* loss, void* stream) {
  if (n <= 0) return 0;
  const unsigned grid = (unsigned)((n + 127) / 128);
  mlp_grad_kernel<<<grid, 128, 0, (cudaStream_t)stream>>>(P, rows, row0, n, 1.f / (float)n_norm, grad, loss);
  return (int)cudaGetLastError();
}

int launch_adam(float* P, const float* g, float* m, float* v, float lr, int step, void* stream) {
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  adam_kernel<<<(kTrainable + 255) / 256, 256, 0, (cudaStream_t)stream>>>(P, g, m, v, lr, b1, b2, 1e-8f, c1, c2);
  return (int)cudaGetLastError();
}

}  // namespace adg
