// Accuracy probe of the hand-written trigonometry on the Kalman path (measurement only, not on
// the path): evaluates sincos_small, atan_small and half_angle on caller-given arguments with the
// same code and compiler flags as the finder and the fit, so that a test can compare them with
// the CUDA library's functions and with FP64 values.
#include "../../include/kfgb.h"
#include "kf_math.cuh"

namespace kfgb {

__global__ void k_math_probe(int fn, const float* __restrict__ a, const float* __restrict__ b, int n,
                             float* __restrict__ o0, float* __restrict__ o1, float* __restrict__ o2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    float r0 = 0.f, r1 = 0.f, r2 = 0.f;
    if (fn == KF_PROBE_SINCOS) {
      sincos_small(a[i], r0, r1);
    } else if (fn == KF_PROBE_ATAN_SMALL) {
      r0 = atan_small(a[i], b[i]);
    } else {
      half_angle(a[i], r0, r1, r2);
    }
    o0[i] = r0;
    o1[i] = r1;
    o2[i] = r2;
  }
}

int launch_math_probe(int fn, const float* a, const float* b, int n, float* o0, float* o1, float* o2,
                      cudaStream_t st) {
  const int blocks = (n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024;
  k_math_probe<<<blocks, 256, 0, st>>>(fn, a, b, n, o0, o1, o2);
  return cudaGetLastError() == cudaSuccess ? KF_OK : KF_ERR_CUDA;
}

}  // namespace kfgb
