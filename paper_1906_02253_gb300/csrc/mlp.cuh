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

// Transposed copy of the parameters for the finder's warp-level inference (same size and the same
// offsets for b1, b2, W3, b3 and the normaliser): W1T[14][64] at kMlpW1 and W2T[64][64] at kMlpW2,
// input-major, so that lane j reads hidden units 2j, 2j+1 of one input as one 8-byte word of a
// contiguous row.
int launch_mlp_transpose(const float* params, float* wt, cudaStream_t st);

// First hidden layer of one (candidate, hit) pair from the owner's 12 normalised candidate features,
// for hidden units 2*lane and 2*lane + 1 (wt: transposed parameters). Summation in input order.
__device__ __forceinline__ float2 mlp_layer1_base(const float* __restrict__ wt, const float* x, int lane) {
  float2 a = __ldg(reinterpret_cast<const float2*>(wt + kMlpB1) + lane);
#pragma unroll
  for (int i = 0; i < 12; ++i) {
    const float2 w = __ldg(reinterpret_cast<const float2*>(wt + kMlpW1 + i * kMlpHid) + lane);
    a.x = fmaf(w.x, x[i], a.x);
    a.y = fmaf(w.y, x[i], a.y);
  }
  return a;
}

// Logit of one pair evaluated by the whole warp (every lane passes the same values): the first
// layer from its 12-input partial sum `base` plus the two normalised pulls x12, x13; lane j holds
// hidden units 2j, 2j+1 of both layers, the first layer reaches every lane through shuffles, the
// output is summed by a butterfly. Every lane returns the logit.
__device__ __forceinline__ float mlp_logit_warp(const float* __restrict__ wt, float2 base, float x12, float x13,
                                                int lane) {
  const float2 w12 = __ldg(reinterpret_cast<const float2*>(wt + kMlpW1 + 12 * kMlpHid) + lane);
  const float2 w13 = __ldg(reinterpret_cast<const float2*>(wt + kMlpW1 + 13 * kMlpHid) + lane);
  const float a0 = fmaxf(fmaf(w13.x, x13, fmaf(w12.x, x12, base.x)), 0.f);
  const float a1 = fmaxf(fmaf(w13.y, x13, fmaf(w12.y, x12, base.y)), 0.f);
  float2 z = __ldg(reinterpret_cast<const float2*>(wt + kMlpB2) + lane);
#pragma unroll
  for (int src = 0; src < 32; ++src) {
    const float u = __shfl_sync(0xffffffffu, a0, src), v = __shfl_sync(0xffffffffu, a1, src);
    const float2 wu = __ldg(reinterpret_cast<const float2*>(wt + kMlpW2 + (2 * src) * kMlpHid) + lane);
    const float2 wv = __ldg(reinterpret_cast<const float2*>(wt + kMlpW2 + (2 * src + 1) * kMlpHid) + lane);
    z.x = fmaf(wv.x, v, fmaf(wu.x, u, z.x));
    z.y = fmaf(wv.y, v, fmaf(wu.y, u, z.y));
  }
  const float2 w3 = __ldg(reinterpret_cast<const float2*>(wt + kMlpW3) + lane);
  float part = w3.x * fmaxf(z.x, 0.f) + w3.y * fmaxf(z.y, 0.f);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  return __ldg(wt + kMlpB3) + part;
}

int launch_mlp_forward(const float* params, const float* feats, int n, float* logits, cudaStream_t st);
int launch_mlp_loss_grad(const float* params, const float* feats, const float* labels, int n, float* grad, float* loss,
                         cudaStream_t st);
int launch_mlp_adam(float* params, const float* grad, float* m, float* v, int t, float lr, float b1, float b2, float eps,
                    cudaStream_t st);

}  // namespace kfgb
