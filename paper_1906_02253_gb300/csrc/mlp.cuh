// Learned hit proposal network: layout of its FP32 parameter buffer and its forward pass.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

namespace kfgb {

constexpr int kMlpIn = 14, kMlpHid = 64;
constexpr int kMlpW1 = 0;
constexpr int kMlpB1 = kMlpW1 + kMlpHid * kMlpIn;
constexpr int kMlpW2 = kMlpB1 + kMlpHid;
constexpr int kMlpB2 = kMlpW2 + kMlpHid * kMlpHid;
constexpr int kMlpW3 = kMlpB2 + kMlpHid;
constexpr int kMlpB3 = kMlpW3 + kMlpHid;
constexpr int kMlpParams = kMlpB3 + 1;              // 5185 weights
constexpr int kMlpMean = kMlpParams;                // normaliser: mean[14], sd[14]
constexpr int kMlpSd = kMlpMean + kMlpIn;
constexpr int kMlpParamsAll = kMlpSd + kMlpIn;      // 5213 floats

// Logit of raw features f (standardised here) with parameters w (shared or global memory).
__device__ __forceinline__ float mlp_logit(const float* w, const float* f) {
  float x[kMlpIn];
#pragma unroll
  for (int i = 0; i < kMlpIn; ++i) x[i] = (f[i] - w[kMlpMean + i]) / w[kMlpSd + i];
  float h1[kMlpHid];
#pragma unroll
  for (int j = 0; j < kMlpHid; ++j) {
    float z = w[kMlpB1 + j];
#pragma unroll
    for (int i = 0; i < kMlpIn; ++i) z += w[kMlpW1 + j * kMlpIn + i] * x[i];
    h1[j] = fmaxf(z, 0.f);
  }
  float out = w[kMlpB3];
  for (int j = 0; j < kMlpHid; ++j) {
    float z = w[kMlpB2 + j];
#pragma unroll
    for (int i = 0; i < kMlpHid; ++i) z += w[kMlpW2 + j * kMlpHid + i] * h1[i];
    out += w[kMlpW3 + j] * fmaxf(z, 0.f);
  }
  return out;
}

int launch_mlp_forward(const float* params, const float* feats, int n, float* logits, cudaStream_t st);
int launch_mlp_loss_grad(const float* params, const float* feats, const float* labels, int n, float* grad, float* loss,
                         cudaStream_t st);
int launch_mlp_adam(float* params, const float* grad, float* m, float* v, int t, float lr, float b1, float b2, float eps,
                    cudaStream_t st);

}  // namespace kfgb
