// Learned hit proposal: an MLP 14 -> 64 -> 64 -> 1 (ReLU) scoring (predicted candidate, hit)
// pairs, trained on the GPU with these kernels (binary cross-entropy with logits, Adam). The
// network is not in the paper; the features and the pruning rule are described in kfgb.h.
//
// Parameter buffer (FP32): W1[64][14], b1[64], W2[64][64], b2[64], W3[64], b3, then the feature
// normaliser mean[14], sd[14] (KF_MLP_PARAMS weights + 28).
#include "mlp.cuh"

namespace kfgb {

// Inference: one thread per sample, weights staged in shared memory.
__global__ void __launch_bounds__(128) k_mlp_forward(const float* __restrict__ params, const float* __restrict__ feats,
                                                     int n, float* __restrict__ logits) {
  __shared__ float w[kMlpParamsAll];
  for (int i = threadIdx.x; i < kMlpParamsAll; i += blockDim.x) w[i] = params[i];
  __syncthreads();
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  float x[kMlpIn];
#pragma unroll
  for (int i = 0; i < kMlpIn; ++i) x[i] = feats[static_cast<size_t>(s) * kMlpIn + i];
  logits[s] = mlp_logit(w, x);
}

// Transposed copy for the finder (layout in mlp.cuh).
__global__ void k_mlp_transpose(const float* __restrict__ w, float* __restrict__ wt) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kMlpParamsAll; i += gridDim.x * blockDim.x) {
    float v;
    if (i < kMlpB1) {  // W1T[in][j] = W1[j][in]
      const int in = i / kMlpHid, j = i % kMlpHid;
      v = w[kMlpW1 + j * kMlpIn + in];
    } else if (i >= kMlpW2 && i < kMlpB2) {  // W2T[in][o] = W2[o][in]
      const int in = (i - kMlpW2) / kMlpHid, o = (i - kMlpW2) % kMlpHid;
      v = w[kMlpW2 + o * kMlpHid + in];
    } else {
      v = w[i];
    }
    wt[i] = v;
  }
}

int launch_mlp_transpose(const float* params, float* wt, cudaStream_t st) {
  k_mlp_transpose<<<(kMlpParamsAll + 255) / 256, 256, 0, st>>>(params, wt);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

// Loss and gradient summed over the samples of a block of kGradBlock threads (one sample each):
// activations and their gradients in shared memory (rows padded to 65 words), then each thread
// reduces a stripe of parameters over the block's samples and adds it to the global sums.
constexpr int kGradBlock = 64;
constexpr int kPad = kMlpHid + 1;

__global__ void __launch_bounds__(kGradBlock) k_mlp_loss_grad(const float* __restrict__ params,
                                                              const float* __restrict__ feats,
                                                              const float* __restrict__ labels, int n,
                                                              float* __restrict__ grad, float* __restrict__ loss) {
  extern __shared__ __align__(16) float sm[];
  float* w = sm;                               // kMlpParamsAll
  float* xs = w + kMlpParamsAll;               // [kGradBlock][kMlpIn]
  float* h1 = xs + kGradBlock * kMlpIn;        // [kGradBlock][kPad]
  float* h2 = h1 + kGradBlock * kPad;
  float* d1 = h2 + kGradBlock * kPad;
  float* d2 = d1 + kGradBlock * kPad;
  float* dz = d2 + kGradBlock * kPad;          // [kGradBlock]
  __shared__ float red[kGradBlock];
  for (int i = threadIdx.x; i < kMlpParamsAll; i += blockDim.x) w[i] = params[i];
  __syncthreads();
  const int b = threadIdx.x;
  const int s = blockIdx.x * kGradBlock + b;
  const bool valid = s < n;
  float lsum = 0.f;
  {
    float* x = xs + b * kMlpIn;
#pragma unroll
    for (int i = 0; i < kMlpIn; ++i) {
      const float f = valid ? feats[static_cast<size_t>(s) * kMlpIn + i] : 0.f;
      x[i] = (f - w[kMlpMean + i]) / w[kMlpSd + i];
    }
    float* a1 = h1 + b * kPad;
    for (int j = 0; j < kMlpHid; ++j) {
      float z = w[kMlpB1 + j];
#pragma unroll
      for (int i = 0; i < kMlpIn; ++i) z += w[kMlpW1 + j * kMlpIn + i] * x[i];
      a1[j] = fmaxf(z, 0.f);
    }
    float* a2 = h2 + b * kPad;
    float z3 = w[kMlpB3];
    for (int j = 0; j < kMlpHid; ++j) {
      float z = w[kMlpB2 + j];
      for (int i = 0; i < kMlpHid; ++i) z += w[kMlpW2 + j * kMlpHid + i] * a1[i];
      a2[j] = fmaxf(z, 0.f);
      z3 += w[kMlpW3 + j] * a2[j];
    }
    const float y = valid ? labels[s] : 0.f;
    const float g = valid ? 1.f / (1.f + expf(-z3)) - y : 0.f;
    if (valid) lsum = fmaxf(z3, 0.f) - z3 * y + log1pf(expf(-fabsf(z3)));
    dz[b] = g;
    float* e2 = d2 + b * kPad;
    for (int j = 0; j < kMlpHid; ++j) e2[j] = a2[j] > 0.f ? g * w[kMlpW3 + j] : 0.f;
    float* e1 = d1 + b * kPad;
    for (int i = 0; i < kMlpHid; ++i) {
      float acc = 0.f;
      for (int j = 0; j < kMlpHid; ++j) acc += e2[j] * w[kMlpW2 + j * kMlpHid + i];
      e1[i] = a1[i] > 0.f ? acc : 0.f;
    }
  }
  red[b] = lsum;
  __syncthreads();
  for (int p = threadIdx.x; p < kMlpParams; p += blockDim.x) {
    float acc = 0.f;
    if (p < kMlpB1) {
      const int j = p / kMlpIn, i = p % kMlpIn;
      for (int k = 0; k < kGradBlock; ++k) acc += d1[k * kPad + j] * xs[k * kMlpIn + i];
    } else if (p < kMlpW2) {
      const int j = p - kMlpB1;
      for (int k = 0; k < kGradBlock; ++k) acc += d1[k * kPad + j];
    } else if (p < kMlpB2) {
      const int j = (p - kMlpW2) / kMlpHid, i = (p - kMlpW2) % kMlpHid;
      for (int k = 0; k < kGradBlock; ++k) acc += d2[k * kPad + j] * h1[k * kPad + i];
    } else if (p < kMlpW3) {
      const int j = p - kMlpB2;
      for (int k = 0; k < kGradBlock; ++k) acc += d2[k * kPad + j];
    } else if (p < kMlpB3) {
      const int j = p - kMlpW3;
      for (int k = 0; k < kGradBlock; ++k) acc += dz[k] * h2[k * kPad + j];
    } else {
      for (int k = 0; k < kGradBlock; ++k) acc += dz[k];
    }
    atomicAdd(grad + p, acc);
  }
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int k = 0; k < kGradBlock; ++k) t += red[k];
    atomicAdd(loss, t);
  }
}

__global__ void k_mlp_scale(float* grad, float* loss, float inv_n) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p <= kMlpParams; p += gridDim.x * blockDim.x) {
    if (p < kMlpParams) grad[p] *= inv_n;
    else *loss *= inv_n;
  }
}

// Adam (Kingma and Ba) on the weights; moments m, v; step t >= 1.
__global__ void k_mlp_adam(float* params, const float* grad, float* m, float* v, int t, float lr, float b1, float b2,
                           float eps) {
  const float c1 = 1.f - powf(b1, static_cast<float>(t)), c2 = 1.f - powf(b2, static_cast<float>(t));
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < kMlpParams; p += gridDim.x * blockDim.x) {
    const float g = grad[p];
    const float mp = b1 * m[p] + (1.f - b1) * g;
    const float vp = b2 * v[p] + (1.f - b2) * g * g;
    m[p] = mp;
    v[p] = vp;
    params[p] -= lr * (mp / c1) / (sqrtf(vp / c2) + eps);
  }
}

size_t mlp_grad_smem() {
  return sizeof(float) * (kMlpParamsAll + kGradBlock * kMlpIn + 4 * kGradBlock * kPad + kGradBlock);
}

int launch_mlp_forward(const float* params, const float* feats, int n, float* logits, cudaStream_t st) {
  if (n == 0) return 0;
  k_mlp_forward<<<(n + 127) / 128, 128, 0, st>>>(params, feats, n, logits);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int launch_mlp_loss_grad(const float* params, const float* feats, const float* labels, int n, float* grad, float* loss,
                         cudaStream_t st) {
  static int attr_set[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return -3;
  const size_t smem = mlp_grad_smem();
  if (!attr_set[dev]) {
    if (cudaFuncSetAttribute(k_mlp_loss_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)) !=
        cudaSuccess)
      return -3;
    attr_set[dev] = 1;
  }
  if (cudaMemsetAsync(grad, 0, sizeof(float) * kMlpParams, st) != cudaSuccess) return -3;
  if (cudaMemsetAsync(loss, 0, sizeof(float), st) != cudaSuccess) return -3;
  if (n > 0) k_mlp_loss_grad<<<(n + kGradBlock - 1) / kGradBlock, kGradBlock, smem, st>>>(params, feats, labels, n, grad, loss);
  k_mlp_scale<<<8, 256, 0, st>>>(grad, loss, n > 0 ? 1.f / n : 0.f);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int launch_mlp_adam(float* params, const float* grad, float* m, float* v, int t, float lr, float b1, float b2, float eps,
                    cudaStream_t st) {
  k_mlp_adam<<<(kMlpParams + 255) / 256, 256, 0, st>>>(params, grad, m, v, t, lr, b1, b2, eps);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

}  // namespace kfgb
