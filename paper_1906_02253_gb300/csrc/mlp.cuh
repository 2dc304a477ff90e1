// Learned hit proposal network: layout of its FP32 parameter buffer and its forward pass.
#pragma once

#include <cuda_fp16.h>
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

// The finder scores its (candidate, hit) pairs on the tensor cores, 16 pairs at a time per warp,
// with warp-level MMAs of shape m16n8k16 (fp16 operands, FP32 accumulation). A pair is a row of the
// 16 x 16 input tile (14 features, two zero columns); the first layer is X W1^T (K = 16, eight
// 8-column tiles of hidden units), the second H1 W2^T (K = 64 in four steps, eight column tiles),
// and the output layer an FP32 dot product. Every operand is split into two fp16 parts, v = hi +
// 2^-11 lo with hi = f16(v) and lo = f16(2^11 (v - hi)) (lo is scaled so that it stays a normal
// fp16 number), which leaves |v - hi - 2^-11 lo| <= 2^-22 |v| for |v| >= 2^-14. Each product A B is
// accumulated as hi hi in one FP32 accumulator and hi lo + lo hi in a second, combined as
// D + 2^-11 E; the dropped 2^-22 lo lo and the two splits leave at most ~3 2^-22 of each product, a
// few FP32 roundings. Operands must stay below the fp16 range (65504): the features are
// standardised and the chi2 cut bounds the pulls, so they and the hidden units of a trained
// network are far below it.
//
// The weights' parts are laid out once per launch as the B fragments of the MMA, so that each lane
// loads both parts of one (K step, column tile) as one 16-byte word and a warp one contiguous
// 512-byte run. Lane l (g = l / 4, t = l % 4) holds, for hidden unit n = 8 * tile + g, the weights
// of inputs k = 16 * step + {2t, 2t + 1} (words x: hi, z: lo) and {2t + 8, 2t + 9} (words y: hi,
// w: lo), two fp16 each, the lower input in the low half. Entries (uint4):
//   layer 1: kFragL1 + tile * 32 + lane
//   layer 2: kFragL2 + (step * 8 + tile) * 32 + lane
constexpr int kFragL1 = 0;
constexpr int kFragL2 = kFragL1 + 8 * 32;
constexpr int kFragWords = kFragL2 + 4 * 8 * 32;  // 1280 entries, 20 KiB
constexpr float kLoScale = 2048.f, kLoUnscale = 1.f / 2048.f;

// Writes the fragments of params (KF_MLP_BUFFER floats) to frag (kFragWords entries).
int launch_mlp_fragments(const float* params, uint4* frag, cudaStream_t st);

// The two fp16 parts of (x0, x1), each packed as one f16x2 word with x0 in the low half.
__device__ __forceinline__ void split_f16x2(float x0, float x1, unsigned& hi, unsigned& lo) {
  const __half2 h = __floats2half2_rn(x0, x1);
  const float2 hf = __half22float2(h);
  const __half2 l = __floats2half2_rn((x0 - hf.x) * kLoScale, (x1 - hf.y) * kLoScale);
  hi = *reinterpret_cast<const unsigned*>(&h);
  lo = *reinterpret_cast<const unsigned*>(&l);
}

// D += A B for one m16n8k16 tile: A as four f16x2 words (rows g and g + 8, columns 2t, 2t + 1 and
// 2t + 8, 2t + 9 in the order (g, lo), (g + 8, lo), (g, hi), (g + 8, hi)), B two words (inputs
// 2t, 2t + 1 and 2t + 8, 2t + 9 of column g), D rows g (d[0], d[1]) and g + 8 (d[2], d[3]),
// columns 2t, 2t + 1.
__device__ __forceinline__ void mma_m16n8k16(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
  asm("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// One K step of a split product: d += A_hi B_hi, e += A_hi B_lo + A_lo B_hi (b: the fragment).
__device__ __forceinline__ void mma_split(float (&d)[4], float (&e)[4], const unsigned (&ahi)[4],
                                          const unsigned (&alo)[4], uint4 b) {
  mma_m16n8k16(e, alo, b.x, b.y);
  mma_m16n8k16(e, ahi, b.z, b.w);
  mma_m16n8k16(d, ahi, b.x, b.y);
}

// Logits of 16 pairs evaluated together by the warp (every lane takes part). Lane l (g = l / 4,
// t = l % 4) passes the normalised features of rows g (xa) and g + 8 (xb) in columns 2t, 2t + 1,
// 2t + 8, 2t + 9 (zero beyond column 13) and receives their logits (la, lb). prm: the network's
// FP32 parameters (biases, output layer), frag: the fragments of its hidden layers.
__device__ __forceinline__ void mlp_logit16(const uint4* __restrict__ frag, const float* __restrict__ prm,
                                            const float (&xa)[4], const float (&xb)[4], int lane, float& la,
                                            float& lb) {
  const int t = lane & 3;
  unsigned a1h[4], a1l[4];
  split_f16x2(xa[0], xa[1], a1h[0], a1l[0]);
  split_f16x2(xb[0], xb[1], a1h[1], a1l[1]);
  split_f16x2(xa[2], xa[3], a1h[2], a1l[2]);
  split_f16x2(xb[2], xb[3], a1h[3], a1l[3]);
  // First layer, column tiles 2s and 2s + 1 at a time: their ReLU outputs are the A operand of
  // the second layer's K step s (the accumulator layout of two column tiles is the operand layout
  // of one K step), split at once.
  unsigned a2h[4][4], a2l[4][4];
#pragma unroll
  for (int s = 0; s < 4; ++s) {
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const int nt = 2 * s + half;
      const float b0 = __ldg(prm + kMlpB1 + 8 * nt + 2 * t), b1 = __ldg(prm + kMlpB1 + 8 * nt + 2 * t + 1);
      float d[4] = {b0, b1, b0, b1}, e[4] = {0.f, 0.f, 0.f, 0.f};
      mma_split(d, e, a1h, a1l, __ldg(frag + kFragL1 + nt * 32 + lane));
      split_f16x2(fmaxf(fmaf(e[0], kLoUnscale, d[0]), 0.f), fmaxf(fmaf(e[1], kLoUnscale, d[1]), 0.f),
                  a2h[s][2 * half], a2l[s][2 * half]);
      split_f16x2(fmaxf(fmaf(e[2], kLoUnscale, d[2]), 0.f), fmaxf(fmaf(e[3], kLoUnscale, d[3]), 0.f),
                  a2h[s][2 * half + 1], a2l[s][2 * half + 1]);
    }
  }
  // Second layer, one column tile at a time, folded into the output layer's sums of rows g, g + 8
  // (not unrolled: the loads of one tile at a time stay in flight).
  float sa = 0.f, sb = 0.f;
#pragma unroll 1
  for (int nt = 0; nt < 8; ++nt) {
    const float b0 = __ldg(prm + kMlpB2 + 8 * nt + 2 * t), b1 = __ldg(prm + kMlpB2 + 8 * nt + 2 * t + 1);
    float d[4] = {b0, b1, b0, b1}, e[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int s = 0; s < 4; ++s) mma_split(d, e, a2h[s], a2l[s], __ldg(frag + kFragL2 + (s * 8 + nt) * 32 + lane));
    const float w0 = __ldg(prm + kMlpW3 + 8 * nt + 2 * t), w1 = __ldg(prm + kMlpW3 + 8 * nt + 2 * t + 1);
    sa = fmaf(w1, fmaxf(fmaf(e[1], kLoUnscale, d[1]), 0.f), fmaf(w0, fmaxf(fmaf(e[0], kLoUnscale, d[0]), 0.f), sa));
    sb = fmaf(w1, fmaxf(fmaf(e[3], kLoUnscale, d[3]), 0.f), fmaf(w0, fmaxf(fmaf(e[2], kLoUnscale, d[2]), 0.f), sb));
  }
  // The four lanes of a row hold its 64 terms.
  sa += __shfl_xor_sync(0xffffffffu, sa, 1);
  sb += __shfl_xor_sync(0xffffffffu, sb, 1);
  sa += __shfl_xor_sync(0xffffffffu, sa, 2);
  sb += __shfl_xor_sync(0xffffffffu, sb, 2);
  const float b3 = __ldg(prm + kMlpB3);
  la = b3 + sa;
  lb = b3 + sb;
}

int launch_mlp_forward(const float* params, const float* feats, int n, float* logits, cudaStream_t st);
int launch_mlp_loss_grad(const float* params, const float* feats, const float* labels, int n, float* grad, float* loss,
                         cudaStream_t st);
int launch_mlp_adam(float* params, const float* grad, float* m, float* v, int t, float lr, float b1, float b2, float eps,
                    cudaStream_t st);

}  // namespace kfgb
