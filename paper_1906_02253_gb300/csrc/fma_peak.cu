// FP32 throughput probe for the roofline of the ALU-bound kernels: every thread runs eight
// independent chains of fused multiply-adds, so the FMA pipe stays busy; the caller times the
// launch. One FMA counts as two flops.
#include "../../include/kfgb.h"

namespace kfgb {

constexpr int kFmaChains = 8;
constexpr int kFmaUnroll = 16;

__global__ void __launch_bounds__(256) k_fma_peak(float* __restrict__ sink, int iters, float a, float b) {
  float v[kFmaChains];
#pragma unroll
  for (int j = 0; j < kFmaChains; ++j) v[j] = static_cast<float>(threadIdx.x + j) * 1e-7f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kFmaUnroll; ++u) {
#pragma unroll
      for (int j = 0; j < kFmaChains; ++j) v[j] = fmaf(v[j], a, b);
    }
  }
  float acc = 0.f;
#pragma unroll
  for (int j = 0; j < kFmaChains; ++j) acc += v[j];
  if (acc == 12345.678f) sink[blockIdx.x] = acc;  // keeps the chains live; practically never true
}

int launch_fma_peak(float* sink, int blocks, int iters, cudaStream_t st, long long* flops) {
  k_fma_peak<<<blocks, 256, 0, st>>>(sink, iters, 0.999999f, 1e-7f);
  *flops = 2LL * kFmaChains * kFmaUnroll * static_cast<long long>(iters) * 256LL * blocks;
  return cudaGetLastError() == cudaSuccess ? KF_OK : KF_ERR_CUDA;
}

}  // namespace kfgb
