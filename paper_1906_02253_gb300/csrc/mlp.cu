// Learned hit proposal: an MLP 14 -> 64 -> 64 -> 1 (ReLU) scoring (predicted candidate, hit)
// pairs, trained on the GPU with these kernels (binary cross-entropy with logits, Adam). The
// network is not in the paper; the features and the pruning rule are described in kfgb.h.
//
// Parameter buffer (FP32): W1[64][14], b1[64], W2[64][64], b2[64], W3[64], b3, then the feature
// normaliser mean[14], sd[14] (KF_MLP_PARAMS weights + 28).
#include <algorithm>

#include "mlp.cuh"
#include "tc.cuh"

namespace kfgb {

// Inference on the tensor cores (tcgen05): a persistent CTA of 256 threads takes tiles of 128
// samples, two threads per sample (each half of the columns). Per tile: standardised inputs -> X tile (128 x 16); D1 = X W1^T
// in tensor memory; h1 = relu(D1 + b1) -> H tile (128 x 64); D2 = H W2^T; logit = b3 + sum_j W3[j]
// relu(D2[j] + b2[j]) on the CUDA cores. Every operand is three bf16 tiles (hi, mid, lo; tc.cuh).
// Shared memory (bytes): X, W1, W2 and H, then b1, b2, W3, mean, sd, b3, the mbarrier and the
// tensor-memory base; 128 tensor-memory columns (D1 at 0, D2 at 64).
namespace fwd {
constexpr uint32_t X_T = 4096, W1_T = 2048, W2_T = 8192, H_T = 16384;  // bytes of one tile
constexpr uint32_t X = 0, W1 = X + 3 * X_T, W2 = W1 + 3 * W1_T, H = W2 + 3 * W2_T, B1 = H + 3 * H_T, B2 = B1 + 256,
                   W3 = B2 + 256, MEAN = W3 + 256, SD = MEAN + 64, PART = SD + 64, B3 = PART + 1024, BAR = B3 + 8,
                   TMEM = BAR + 8, BYTES = TMEM + 8;
constexpr uint32_t kCols = 128;
}  // namespace fwd
constexpr int kTcM = 128;   // samples per tile (the MMA's M)
constexpr int kTcK1 = 16;   // the 14 inputs padded to one MMA K step
constexpr int kFwdCtasPerSm = 2;

// Loads W1 (64 x 16, inputs 14 and 15 zero) and W2 (64 x 64) as the MMAs' B operands in the
// K-major core-matrix layout, by all threads of the block.
__device__ __forceinline__ void stage_weights_b(const float* __restrict__ params, unsigned char* w1, uint32_t w1_t,
                                                unsigned char* w2, uint32_t w2_t) {
  for (int item = threadIdx.x; item < kMlpHid * 2; item += blockDim.x) {
    const int j = item >> 1, c = item & 1;
    float v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int i = 8 * c + e;
      v[e] = i < kMlpIn ? params[kMlpW1 + j * kMlpIn + i] : 0.f;
    }
    tc::store8_split(w1, w1_t, tc::kmajor_off(j, c, kTcK1), v);
  }
  for (int item = threadIdx.x; item < kMlpHid * 8; item += blockDim.x) {
    const int o = item >> 3, c = item & 7;
    float v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = params[kMlpW2 + o * kMlpHid + 8 * c + e];
    tc::store8_split(w2, w2_t, tc::kmajor_off(o, c, kMlpHid), v);
  }
}

// Two threads per sample: thread t takes sample t % 128 of the tile and half h = t / 128 of its
// columns. Warps w and w + 4 read the same tensor-memory lanes (32 (w % 4) ..), each its half of a
// 64-column accumulator; every branch around a tensor-memory load is uniform within a warp.
constexpr int kTcThreads = 2 * 128;

// Raw features [8 h, 8 h + 8) of sample r (zeros past n and past the 14 inputs), loaded ahead of
// their tile.
__device__ __forceinline__ void fetch_half(const float* __restrict__ feats, int r, int n, int half, float2* f) {
  const float2* f2 = reinterpret_cast<const float2*>(feats + static_cast<size_t>(r) * kMlpIn);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int k = 4 * half + i;
    f[i] = (r < n && k < kMlpIn / 2) ? __ldg(f2 + k) : make_float2(0.f, 0.f);
  }
}

// Standardised inputs [8 h, 8 h + 8) into x[8] (zero past n and for the padding inputs 14, 15).
__device__ __forceinline__ void standardise_half(const float2* f, bool valid, int half, const float* mean,
                                                 const float* sd, float* x) {
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int k = 8 * half + 2 * i;
    x[2 * i] = (valid && k < kMlpIn) ? (f[i].x - mean[k]) / sd[k] : 0.f;
    x[2 * i + 1] = (valid && k + 1 < kMlpIn) ? (f[i].y - mean[k + 1]) / sd[k + 1] : 0.f;
  }
}

// One MMA operand in shared memory: the first of its three tiles (shared-window address), the
// tile size, the descriptor's leading and stride byte offsets, and the byte advance per K = 16 step.
struct Operand {
  uint32_t base, tile, lbo, sbo, step;
};

// K-major operand (tc.cuh layout) of a tile with kt columns, starting at column block c0.
__device__ __forceinline__ Operand kmajor(uint32_t base, uint32_t tile, int kt, int c0 = 0) {
  return Operand{base + 128u * c0, tile, 128u, static_cast<uint32_t>(kt / 8 * 128), 256u};
}

// The same tile read MN-major (its rows become K, its columns M or N): 8-column blocks are 128 B
// apart (stride byte offset), 8-row groups kt / 8 * 128 B apart (leading byte offset).
__device__ __forceinline__ Operand mnmajor(uint32_t base, uint32_t tile, int kt) {
  const uint32_t g = static_cast<uint32_t>(kt / 8 * 128);
  return Operand{base, tile, g, 128u, 2u * g};
}

// D = A B^T over k_steps steps of K = 16 as the six products of the three-part split (hi*hi,
// hi*mid, mid*hi, hi*lo, lo*hi, mid*mid); one thread issues, the mbarrier receives the
// completion; the first product overwrites D unless accumulate is set.
__device__ __forceinline__ void mma_split(uint32_t d, const Operand& A, const Operand& B, int k_steps, uint32_t idesc,
                                          uint64_t* bar, bool accumulate = false) {
  constexpr int kPa[6] = {0, 0, 1, 0, 2, 1}, kPb[6] = {0, 1, 0, 2, 0, 1};
  tc::fence_after_sync();
  for (int k = 0; k < k_steps; ++k) {
#pragma unroll
    for (int p = 0; p < 6; ++p) {
      const uint64_t ad = tc::smem_desc(A.base + A.tile * kPa[p] + A.step * k, A.lbo, A.sbo);
      const uint64_t bd = tc::smem_desc(B.base + B.tile * kPb[p] + B.step * k, B.lbo, B.sbo);
      tc::mma_bf16(d, ad, bd, idesc, (k > 0 || p > 0 || accumulate) ? 1u : 0u);
    }
  }
  tc::mma_commit(bar);
}

__global__ void __launch_bounds__(kTcThreads) k_mlp_forward(const float* __restrict__ params,
                                                            const float* __restrict__ feats, int n,
                                                            float* __restrict__ logits) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* S = smem_raw + ((1024 - (tc::smem_u32(smem_raw) & 1023)) & 1023);
  const uint32_t sb = tc::smem_u32(S);
  float* b1 = reinterpret_cast<float*>(S + fwd::B1);
  float* b2 = reinterpret_cast<float*>(S + fwd::B2);
  float* w3 = reinterpret_cast<float*>(S + fwd::W3);
  float* mean = reinterpret_cast<float*>(S + fwd::MEAN);
  float* sd = reinterpret_cast<float*>(S + fwd::SD);
  float* part = reinterpret_cast<float*>(S + fwd::PART);  // [2][128] output-layer partial sums
  uint64_t* bar = reinterpret_cast<uint64_t*>(S + fwd::BAR);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(S + fwd::TMEM);
  const int t = threadIdx.x, warp = t >> 5, row = t & (kTcM - 1), half = t >> 7;

  stage_weights_b(params, S + fwd::W1, fwd::W1_T, S + fwd::W2, fwd::W2_T);
  for (int i = t; i < kMlpHid; i += blockDim.x) {
    b1[i] = params[kMlpB1 + i];
    b2[i] = params[kMlpB2 + i];
    w3[i] = params[kMlpW3 + i];
  }
  if (t < kMlpIn) {
    mean[t] = params[kMlpMean + t];
    sd[t] = params[kMlpSd + t];
  }
  const float b3 = params[kMlpB3];
  if (warp == 0) tc::tmem_alloc(tmem_slot, fwd::kCols);
  if (t == 0) tc::mbar_init(bar, 1);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  const uint32_t lane_base = tmem + (static_cast<uint32_t>((warp & 3) * 32) << 16) + 32u * half;
  constexpr uint32_t idesc = tc::idesc_bf16_f32(kTcM, kMlpHid);
  uint32_t phase = 0;
  bool failed = false;

  const int n_tiles = (n + kTcM - 1) / kTcM;
  float2 fin[4];  // this thread's half of the raw features of its sample in the next tile
  fetch_half(feats, blockIdx.x * kTcM + row, n, half, fin);
  for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int r = tile * kTcM + row;
    {
      float x[8];
      standardise_half(fin, r < n, half, mean, sd, x);
      tc::store8_split(S + fwd::X, fwd::X_T, tc::kmajor_off(row, half, kTcK1), x);
    }
    tc::fence_proxy_async();
    __syncthreads();
    if (t == 0)
      mma_split(tmem, kmajor(sb + fwd::X, fwd::X_T, kTcK1), kmajor(sb + fwd::W1, fwd::W1_T, kTcK1), 1, idesc, bar);
    fetch_half(feats, (tile + gridDim.x) * kTcM + row, n, half, fin);  // in flight during this tile's MMAs
    bool ok = tc::mbar_wait(bar, phase);
    phase ^= 1u;
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
    tc::fence_after_sync();
    // h1 columns [32 h, 32 h + 32) -> the H tile
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      float v[16];
      tc::tmem_ld16(lane_base + 16 * q, v);
#pragma unroll
      for (int i = 0; i < 16; ++i) v[i] = fmaxf(v[i] + b1[32 * half + 16 * q + i], 0.f);
      tc::store8_split(S + fwd::H, fwd::H_T, tc::kmajor_off(row, 4 * half + 2 * q, kMlpHid), v);
      tc::store8_split(S + fwd::H, fwd::H_T, tc::kmajor_off(row, 4 * half + 2 * q + 1, kMlpHid), v + 8);
    }
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    if (t == 0)
      mma_split(tmem + 64, kmajor(sb + fwd::H, fwd::H_T, kMlpHid), kmajor(sb + fwd::W2, fwd::W2_T, kMlpHid), 4, idesc,
                bar);
    ok = tc::mbar_wait(bar, phase);
    phase ^= 1u;
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
    tc::fence_after_sync();
    float acc = 0.f;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      float v[16];
      tc::tmem_ld16(lane_base + 64 + 16 * q, v);
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int j = 32 * half + 16 * q + i;
        acc = fmaf(w3[j], fmaxf(v[i] + b2[j], 0.f), acc);
      }
    }
    part[half * kTcM + row] = acc;
    tc::fence_before_sync();
    __syncthreads();
    if (half == 0 && r < n) logits[r] = b3 + part[row] + part[kTcM + row];
  }
  if (failed) {
    // A tensor-core wait gave up: this block's remaining samples get NaN logits; the MMA in
    // flight gets one more bounded wait before the tensor memory is released.
    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
      const int r = tile * kTcM + row;
      if (half == 0 && r < n) logits[r] = __int_as_float(0x7fc00000);
    }
    tc::mbar_wait(bar, phase ^ 1u);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, fwd::kCols);
  }
}

// The finder's A fragments of both hidden layers (layout in mlp.cuh): entry i holds, for row tile
// m and K step s, lane l's four f16x2 words (rows 16 m + l / 4 and + 8, columns 16 s + 2 (l % 4)
// and + 8; zero beyond the 14 inputs of the first layer), hi or scaled lo part.
__global__ void k_mlp_fragments(const float* __restrict__ w, uint4* __restrict__ frag) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kFragWords; i += gridDim.x * blockDim.x) {
    const int part = i & 1, lane = (i >> 1) % 32;
    int m, s, ld;
    const float* W;
    if (i < kFragL2) {
      m = (i >> 1) / 32;
      s = 0;
      W = w + kMlpW1;
      ld = kMlpIn;
    } else {
      const int j = ((i - kFragL2) >> 1) / 32;
      m = j / 4;
      s = j % 4;
      W = w + kMlpW2;
      ld = kMlpHid;
    }
    const int r = 16 * m + lane / 4, c = 16 * s + 2 * (lane % 4);
    const int rr[4] = {r, r + 8, r, r + 8}, cc[4] = {c, c, c + 8, c + 8};
    unsigned word[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float v0 = cc[q] < ld ? W[rr[q] * ld + cc[q]] : 0.f;
      const float v1 = cc[q] + 1 < ld ? W[rr[q] * ld + cc[q] + 1] : 0.f;
      unsigned h, l;
      split_f16x2(v0, v1, h, l);
      word[q] = part ? l : h;
    }
    frag[i] = make_uint4(word[0], word[1], word[2], word[3]);
  }
}

int launch_mlp_fragments(const float* params, uint4* frag, cudaStream_t st) {
  k_mlp_fragments<<<(kFragWords + 255) / 256, 256, 0, st>>>(params, frag);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

// The finder's scoring outside the finder: warp w of the grid takes rows 8w .. 8w + 7, lane l the
// features of row 8w + l / 4 in its operand columns, standardised as the finder standardises its
// candidate features and pulls; lanes 0-3 write the logits of rows 8w + 2l, 8w + 2l + 1.
__global__ void k_mlp_finder_scores(const uint4* __restrict__ frag, const float* __restrict__ prm,
                                    const float* __restrict__ feats, int n, float* __restrict__ logits) {
  const int lane = threadIdx.x & 31;
  const long long r0 = (static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x) / 32 * 8;
  if (r0 >= n) return;  // whole warps leave together (r0 is the same for the warp's lanes)
  const long long row = r0 + (lane >> 2);
  const int t = lane & 3;
  const int cols[4] = {2 * t, 2 * t + 1, 2 * t + 8, 2 * t + 9};
  float x[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int c = cols[q];
    x[q] = (row < n && c < kMlpIn) ? (feats[row * kMlpIn + c] - prm[kMlpMean + c]) / prm[kMlpSd + c] : 0.f;
  }
  const float2 l2 = mlp_logit8(frag, prm, x, lane);
  if (lane < 4) {
    if (r0 + 2 * lane < n) logits[r0 + 2 * lane] = l2.x;
    if (r0 + 2 * lane + 1 < n) logits[r0 + 2 * lane + 1] = l2.y;
  }
}

int launch_mlp_finder_scores(const float* params, const float* feats, int n, float* logits, uint4* frag,
                             cudaStream_t st) {
  if (launch_mlp_fragments(params, frag, st) != 0) return -3;
  if (n == 0) return 0;
  const long long warps = (static_cast<long long>(n) + 7) / 8;
  k_mlp_finder_scores<<<static_cast<unsigned>((warps + 7) / 8), 256, 0, st>>>(frag, params, feats, n, logits);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

// Loss and gradient on the tensor cores: a persistent CTA of 256 threads per SM takes tiles of 128
// samples, two threads per sample (each half of the columns), and runs per tile
//   D1 = X W1^T -> h1 = relu(D1 + b1);  D2 = H1 W2^T -> z3 = b3 + W3 . relu(D2 + b2),
//   g = sigmoid(z3) - y, e2 = g W3 [z2 > 0];  D3 = E2 W2 -> e1 = D3 [h1 > 0];
//   Dg += [E2 | E1]^T [H1 | X | 1]   (accumulated in tensor memory over all the CTA's tiles),
// so that Dg holds dW2 (rows 0-63, columns 0-63), dW1 (rows 64-127, columns 64-77), db2 and db1
// (column 80). dW3, db3 and the loss are summed in registers. Shared memory (bytes; each operand
// three tiles, hi, mid, lo): the sample x [e2 | e1] tile (128 x 128, K-major; read MN-major as the
// A operand of the gradient MMA), the sample x [h1 | x | 1 | 0] tile (128 x 96: the A operand of
// the first two MMAs, MN-major the B operand of the gradient MMA), W1 and W2 (W2 read MN-major is
// W2^T for the third MMA); tensor memory: D1 then D3 at column 0, D2 at 64, Dg at 128.
namespace grd {
constexpr uint32_t E_T = 32768, XH_T = 24576, W1_T = 2048, W2_T = 8192;  // bytes of one tile
constexpr uint32_t E = 0, XH = E + 3 * E_T, W1 = XH + 3 * XH_T, W2 = W1 + 3 * W1_T, B1 = W2 + 3 * W2_T,
                   B2 = B1 + 256, W3 = B2 + 256, MEAN = W3 + 256, SD = MEAN + 64, RED = SD + 64, PART = RED + 272,
                   B3 = PART + 1024, BAR = B3 + 8, TMEM = BAR + 8, BYTES = TMEM + 8;
// The allocation leaves room past W2's lo tile, so that no reading of the MN-major W2 operand's
// offsets can leave the block's shared memory.
constexpr uint32_t ALLOC = 208896;
static_assert(BYTES <= ALLOC && W2 + 2 * W2_T + 13568 <= ALLOC, "shared-memory layout");
constexpr uint32_t kCols = 256, kColD2 = 64, kColG = 128;
constexpr int kXhK = 96, kEK = 128, kGN = 96;
}  // namespace grd

// Instruction descriptor bits 15 and 16: A, B MN-major.
constexpr uint32_t kAmn = 1u << 15, kBmn = 1u << 16;

__global__ void __launch_bounds__(kTcThreads) k_mlp_loss_grad(const float* __restrict__ params,
                                                              const float* __restrict__ feats,
                                                              const float* __restrict__ labels, int n,
                                                              float* __restrict__ grad, float* __restrict__ loss) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* S = smem_raw + ((1024 - (tc::smem_u32(smem_raw) & 1023)) & 1023);
  const uint32_t sb = tc::smem_u32(S);
  float* b1 = reinterpret_cast<float*>(S + grd::B1);
  float* b2 = reinterpret_cast<float*>(S + grd::B2);
  float* w3 = reinterpret_cast<float*>(S + grd::W3);
  float* mean = reinterpret_cast<float*>(S + grd::MEAN);
  float* sd = reinterpret_cast<float*>(S + grd::SD);
  float* red = reinterpret_cast<float*>(S + grd::RED);    // dW3[64], db3, loss
  float* part = reinterpret_cast<float*>(S + grd::PART);  // [2][128] output-layer partial sums
  uint64_t* bar = reinterpret_cast<uint64_t*>(S + grd::BAR);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(S + grd::TMEM);
  const int t = threadIdx.x, warp = t >> 5, row = t & (kTcM - 1), half = t >> 7;
  const int hc = 32 * half;  // this thread's first column of a 64-column accumulator

  stage_weights_b(params, S + grd::W1, grd::W1_T, S + grd::W2, grd::W2_T);
  for (int i = t; i < kMlpHid; i += blockDim.x) {
    b1[i] = params[kMlpB1 + i];
    b2[i] = params[kMlpB2 + i];
    w3[i] = params[kMlpW3 + i];
  }
  if (t < kMlpIn) {
    mean[t] = params[kMlpMean + t];
    sd[t] = params[kMlpSd + t];
  }
  if (t < 66) red[t] = 0.f;
  {  // constant columns of this row of the [h1 | x | 1 | 0] tile: 80 (one) and 81-95 (zero)
    float c[8] = {half == 0 ? 1.f : 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    tc::store8_split(S + grd::XH, grd::XH_T, tc::kmajor_off(row, 10 + half, grd::kXhK), c);
  }
  const float b3 = params[kMlpB3];
  if (warp == 0) tc::tmem_alloc(tmem_slot, grd::kCols);
  if (t == 0) tc::mbar_init(bar, 1);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  const uint32_t lane_base = tmem + (static_cast<uint32_t>((warp & 3) * 32) << 16);
  constexpr uint32_t id_kk = tc::idesc_bf16_f32(kTcM, kMlpHid);
  constexpr uint32_t id_kmn = id_kk | kBmn;
  constexpr uint32_t id_grad = tc::idesc_bf16_f32(kTcM, grd::kGN) | kAmn | kBmn;
  uint32_t phase = 0;
  bool failed = false;
  float acc3[32];  // dW3 partial sums of this thread's 32 hidden units
#pragma unroll
  for (int j = 0; j < 32; ++j) acc3[j] = 0.f;
  float gsum = 0.f, lsum = 0.f;

  const int n_tiles = (n + kTcM - 1) / kTcM;
  int done_tiles = 0;
  float2 fin[4];  // this thread's half of the raw features, and the label, of its sample in the next tile
  fetch_half(feats, blockIdx.x * kTcM + row, n, half, fin);
  float yin = blockIdx.x * kTcM + row < n ? labels[blockIdx.x * kTcM + row] : 0.f;
  for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++done_tiles) {
    const int r = tile * kTcM + row;
    const bool valid = r < n;
    {  // inputs -> columns 64-79 of the [h1 | x | 1 | 0] tile
      float x[8];
      standardise_half(fin, valid, half, mean, sd, x);
      tc::store8_split(S + grd::XH, grd::XH_T, tc::kmajor_off(row, 8 + half, grd::kXhK), x);
    }
    const float y = yin;
    {
      const int rn = (tile + gridDim.x) * kTcM + row;  // in flight during this tile's MMAs
      fetch_half(feats, rn, n, half, fin);
      yin = rn < n ? labels[rn] : 0.f;
    }
    tc::fence_proxy_async();
    __syncthreads();
    if (t == 0)
      mma_split(tmem, kmajor(sb + grd::XH, grd::XH_T, grd::kXhK, 8), kmajor(sb + grd::W1, grd::W1_T, kTcK1), 1,
                id_kk, bar);
    bool ok = tc::mbar_wait(bar, phase);
    phase ^= 1u;
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
    tc::fence_after_sync();
    // h1 -> columns [hc, hc + 32) of the [h1 | x | 1 | 0] tile; mask1 = [h1 > 0]
    unsigned mask1 = 0u;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      float v[16];
      tc::tmem_ld16(lane_base + hc + 16 * q, v);
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        v[i] = fmaxf(v[i] + b1[hc + 16 * q + i], 0.f);
        if (v[i] > 0.f) mask1 |= 1u << (16 * q + i);
      }
      tc::store8_split(S + grd::XH, grd::XH_T, tc::kmajor_off(row, 4 * half + 2 * q, grd::kXhK), v);
      tc::store8_split(S + grd::XH, grd::XH_T, tc::kmajor_off(row, 4 * half + 2 * q + 1, grd::kXhK), v + 8);
    }
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    if (t == 0)
      mma_split(tmem + grd::kColD2, kmajor(sb + grd::XH, grd::XH_T, grd::kXhK),
                kmajor(sb + grd::W2, grd::W2_T, kMlpHid), 4, id_kk, bar);
    ok = tc::mbar_wait(bar, phase);
    phase ^= 1u;
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
    tc::fence_after_sync();
    {  // logit from the two halves' partial sums
      float acc = 0.f;
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        float v[16];
        tc::tmem_ld16(lane_base + grd::kColD2 + hc + 16 * q, v);
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int j = hc + 16 * q + i;
          acc = fmaf(w3[j], fmaxf(v[i] + b2[j], 0.f), acc);
        }
      }
      part[half * kTcM + row] = acc;
    }
    __syncthreads();
    const float z3 = b3 + part[row] + part[kTcM + row];
    const float g = valid ? 1.f / (1.f + expf(-z3)) - y : 0.f;
    if (half == 0) {
      if (valid) lsum += fmaxf(z3, 0.f) - z3 * y + log1pf(expf(-fabsf(z3)));
      gsum += g;
    }
    // e2 -> columns [hc, hc + 32) of the [e2 | e1] tile; dW3 partial sums
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      float v[16];
      tc::tmem_ld16(lane_base + grd::kColD2 + hc + 16 * q, v);
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const float a2 = fmaxf(v[i] + b2[hc + 16 * q + i], 0.f);
        acc3[16 * q + i] = fmaf(g, a2, acc3[16 * q + i]);
        v[i] = a2 > 0.f ? g * w3[hc + 16 * q + i] : 0.f;
      }
      tc::store8_split(S + grd::E, grd::E_T, tc::kmajor_off(row, 4 * half + 2 * q, grd::kEK), v);
      tc::store8_split(S + grd::E, grd::E_T, tc::kmajor_off(row, 4 * half + 2 * q + 1, grd::kEK), v + 8);
    }
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    // D3 = E2 W2: W2's K-major tile (rows o, columns i) read MN-major is W2^T (n = i, k = o).
    if (t == 0)
      mma_split(tmem, kmajor(sb + grd::E, grd::E_T, grd::kEK), mnmajor(sb + grd::W2, grd::W2_T, kMlpHid), 4, id_kmn,
                bar);
    ok = tc::mbar_wait(bar, phase);
    phase ^= 1u;
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
    tc::fence_after_sync();
    // e1 -> columns 64 + [hc, hc + 32) of the [e2 | e1] tile
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      float v[16];
      tc::tmem_ld16(lane_base + hc + 16 * q, v);
#pragma unroll
      for (int i = 0; i < 16; ++i) v[i] = (mask1 >> (16 * q + i)) & 1u ? v[i] : 0.f;
      tc::store8_split(S + grd::E, grd::E_T, tc::kmajor_off(row, 8 + 4 * half + 2 * q, grd::kEK), v);
      tc::store8_split(S + grd::E, grd::E_T, tc::kmajor_off(row, 9 + 4 * half + 2 * q, grd::kEK), v + 8);
    }
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    // Dg += [e2 | e1]^T [h1 | x | 1 | 0]: both tiles read MN-major, K = the tile's 128 samples.
    if (t == 0)
      mma_split(tmem + grd::kColG, mnmajor(sb + grd::E, grd::E_T, grd::kEK), mnmajor(sb + grd::XH, grd::XH_T, grd::kXhK),
                kTcM / 16, id_grad, bar, done_tiles > 0);
    ok = tc::mbar_wait(bar, phase);
    phase ^= 1u;
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
    tc::fence_after_sync();
  }
  if (failed) {
    // A tensor-core wait gave up: the loss becomes NaN and this block adds no gradient; the MMA in
    // flight gets one more bounded wait before the tensor memory is released.
    if (t == 0) atomicAdd(loss, __int_as_float(0x7fc00000));
    tc::mbar_wait(bar, phase ^ 1u);
  } else if (done_tiles > 0) {
#pragma unroll
    for (int j = 0; j < 32; ++j) atomicAdd(&red[hc + j], acc3[j]);
    if (half == 0) {
      atomicAdd(&red[64], gsum);
      atomicAdd(&red[65], lsum);
    }
    // Dg row `row` (warp-uniform branches): dW2 row j = row, columns [hc, hc + 32), and db2[j]
    // (column 80, half 0); or dW1 row i = row - 64 (columns 64-77, half 0) and db1[i] (half 1).
    float v[16];
    if (row < kMlpHid) {
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        tc::tmem_ld16(lane_base + grd::kColG + hc + 16 * q, v);
#pragma unroll
        for (int i = 0; i < 16; ++i) atomicAdd(grad + kMlpW2 + row * kMlpHid + hc + 16 * q + i, v[i]);
      }
      if (half == 0) {
        tc::tmem_ld16(lane_base + grd::kColG + 80, v);
        atomicAdd(grad + kMlpB2 + row, v[0]);
      }
    } else if (half == 0) {
      tc::tmem_ld16(lane_base + grd::kColG + 64, v);
#pragma unroll
      for (int k = 0; k < kMlpIn; ++k) atomicAdd(grad + kMlpW1 + (row - kMlpHid) * kMlpIn + k, v[k]);
    } else {
      tc::tmem_ld16(lane_base + grd::kColG + 80, v);
      atomicAdd(grad + kMlpB1 + row - kMlpHid, v[0]);
    }
    __syncthreads();
    if (t < kMlpHid) atomicAdd(grad + kMlpW3 + t, red[t]);
    if (t == kMlpHid) atomicAdd(grad + kMlpB3, red[64]);
    if (t == kMlpHid + 1) atomicAdd(loss, red[65]);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, grd::kCols);
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

// Number of SMs of the current device and, once per device, the kernel's shared-memory opt-in.
static int tc_prepare(const void* kernel, int smem, int* sms) {
  static int sm_count[64] = {0};
  static int smem_set[2][64] = {{0}};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return -3;
  if (!sm_count[dev] && cudaDeviceGetAttribute(&sm_count[dev], cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return -3;
  const int which = kernel == reinterpret_cast<const void*>(k_mlp_forward) ? 0 : 1;
  if (smem > smem_set[which][dev]) {
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) return -3;
    smem_set[which][dev] = smem;
  }
  *sms = sm_count[dev];
  return 0;
}

int launch_mlp_forward(const float* params, const float* feats, int n, float* logits, cudaStream_t st) {
  if (n == 0) return 0;
  const int smem = static_cast<int>(fwd::BYTES) + 1024;
  int sms = 0;
  if (tc_prepare(reinterpret_cast<const void*>(k_mlp_forward), smem, &sms) != 0) return -3;
  const int tiles = (n + kTcM - 1) / kTcM;
  k_mlp_forward<<<std::min(tiles, kFwdCtasPerSm * sms), kTcThreads, smem, st>>>(params, feats, n, logits);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int launch_mlp_loss_grad(const float* params, const float* feats, const float* labels, int n, float* grad, float* loss,
                         cudaStream_t st) {
  const int smem = static_cast<int>(grd::ALLOC) + 1024;
  int sms = 0;
  if (tc_prepare(reinterpret_cast<const void*>(k_mlp_loss_grad), smem, &sms) != 0) return -3;
  if (cudaMemsetAsync(grad, 0, sizeof(float) * kMlpParams, st) != cudaSuccess) return -3;
  if (cudaMemsetAsync(loss, 0, sizeof(float), st) != cudaSuccess) return -3;
  const int tiles = (n + kTcM - 1) / kTcM;
  if (n > 0) k_mlp_loss_grad<<<std::min(tiles, sms), kTcThreads, smem, st>>>(params, feats, labels, n, grad, loss);
  k_mlp_scale<<<8, 256, 0, st>>>(grad, loss, n > 0 ? 1.f / n : 0.f);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int launch_mlp_adam(float* params, const float* grad, float* m, float* v, int t, float lr, float b1, float b2, float eps,
                    cudaStream_t st) {
  k_mlp_adam<<<(kMlpParams + 255) / 256, 256, 0, st>>>(params, grad, m, v, t, lr, b1, b2, eps);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

}  // namespace kfgb
