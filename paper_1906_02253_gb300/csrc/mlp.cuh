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

// The finder scores its (candidate, hit) pairs on the tensor cores, 8 pairs at a time per warp,
// with warp-level MMAs of shape m16n8k16 (fp16 operands, FP32 accumulation) in which the pairs are
// the 8 columns and the network's weights the 16-row A operand: layer 1 is W1 X^T (four 16-row
// tiles of hidden units, K = 16 inputs: 14 features and two zeros), layer 2 W2 H1 (four row tiles,
// K = 64 in four steps), and the output layer an FP32 dot product. Layer 1's accumulator tiles
// become layer 2's B operand by an 8 x 8 transpose in registers (movmatrix). Every operand is split
// into two fp16 parts, v = hi + 2^-11 lo with hi = f16(v) and lo = f16(2^11 (v - hi)) (lo is scaled
// so that it stays a normal fp16 number), which leaves |v - hi - 2^-11 lo| <= 2^-22 |v| for
// |v| >= 2^-14. Each product A B is accumulated as hi hi in one FP32 accumulator and hi lo + lo hi
// in a second, combined as D + 2^-11 E; the dropped 2^-22 lo lo and the two splits leave at most
// ~3 2^-22 of each product, a few FP32 roundings. Operands must stay below the fp16 range (65504):
// the features are standardised and the chi2 cut bounds the pulls, so they and the hidden units of
// a trained network are far below it.
//
// The weights' parts are laid out once per launch as the A fragments of the MMA: lane l (g = l / 4,
// t = l % 4) of (row tile m, K step s) holds rows r = 16 m + g and r + 8, columns c = 16 s + 2t and
// c + 8, as the words (W[r][c], W[r][c + 1]), (W[r + 8][c], ...), (W[r][c + 8], ...), (W[r + 8][c + 8],
// ...) of two fp16 each (zero beyond the 14 inputs of the first layer), hi in one 16-byte entry and
// lo in the next:
//   layer 1: kFragL1 + (m * 32 + lane) * 2 + part
//   layer 2: kFragL2 + ((m * 4 + s) * 32 + lane) * 2 + part
constexpr int kFragL1 = 0;
constexpr int kFragL2 = kFragL1 + 4 * 32 * 2;
constexpr int kFragWords = kFragL2 + 16 * 32 * 2;  // 1280 entries, 20 KiB
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

// D += A B for one m16n8k16 tile: A as the four f16x2 words of the layout above, B two words (lane
// l: column g = l / 4, rows 2t, 2t + 1 and 2t + 8, 2t + 9), D rows g (d[0], d[1]) and g + 8 (d[2],
// d[3]), columns 2t, 2t + 1.
__device__ __forceinline__ void mma_m16n8k16(float (&d)[4], uint4 a, unsigned b0, unsigned b1) {
  asm("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a.x), "r"(a.y), "r"(a.z), "r"(a.w), "r"(b0), "r"(b1));
}

// One K step of a split product: d += A_hi B_hi, e += A_hi B_lo + A_lo B_hi.
__device__ __forceinline__ void mma_split(float (&d)[4], float (&e)[4], uint4 ahi, uint4 alo, const unsigned (&bhi)[2],
                                          const unsigned (&blo)[2]) {
  mma_m16n8k16(e, alo, bhi[0], bhi[1]);
  mma_m16n8k16(e, ahi, blo[0], blo[1]);
  mma_m16n8k16(d, ahi, bhi[0], bhi[1]);
}

// Transpose of an 8 x 8 matrix of 16-bit values held as one word per lane (lane l: row l / 4,
// columns 2 (l % 4), 2 (l % 4) + 1).
__device__ __forceinline__ unsigned transpose8x8(unsigned v) {
  unsigned r;
  asm("movmatrix.sync.aligned.m8n8.trans.b16 %0, %1;" : "=r"(r) : "r"(v));
  return r;
}

// Logits of 8 pairs evaluated together by the warp (every lane takes part). Lane l (g = l / 4,
// t = l % 4) passes the normalised features of pair g in columns 2t, 2t + 1, 2t + 8, 2t + 9 (zero
// beyond column 13) and receives the logits of pairs 2t and 2t + 1. prm: the network's FP32
// parameters (biases, output layer), frag: the fragments of its hidden layers, in global memory
// (read through the read-only path) or, with SMEM, in shared memory.
template <bool SMEM = false>
__device__ __forceinline__ float2 mlp_logit8(const uint4* __restrict__ frag, const float* __restrict__ prm,
                                             const float (&x)[4], int lane) {
  const int g = lane >> 2;
  unsigned xh[2], xl[2];
  split_f16x2(x[0], x[1], xh[0], xl[0]);
  split_f16x2(x[2], x[3], xh[1], xl[1]);
  // Layer 1, row tile m: its ReLU outputs (hidden units 16 m + g, + 8 of pairs 2t, 2t + 1),
  // transposed, are layer 2's B operand of K step m.
  unsigned hh[4][2], hl[4][2];
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    const float b0 = __ldg(prm + kMlpB1 + 16 * m + g), b1 = __ldg(prm + kMlpB1 + 16 * m + g + 8);
    float d[4] = {b0, b0, b1, b1}, e[4] = {0.f, 0.f, 0.f, 0.f};
    const uint4* f = frag + kFragL1 + (m * 32 + lane) * 2;
    mma_split(d, e, SMEM ? f[0] : __ldg(f), SMEM ? f[1] : __ldg(f + 1), xh, xl);
    unsigned th, tl, uh, ul;
    split_f16x2(fmaxf(fmaf(e[0], kLoUnscale, d[0]), 0.f), fmaxf(fmaf(e[1], kLoUnscale, d[1]), 0.f), th, tl);
    split_f16x2(fmaxf(fmaf(e[2], kLoUnscale, d[2]), 0.f), fmaxf(fmaf(e[3], kLoUnscale, d[3]), 0.f), uh, ul);
    hh[m][0] = transpose8x8(th);
    hl[m][0] = transpose8x8(tl);
    hh[m][1] = transpose8x8(uh);
    hl[m][1] = transpose8x8(ul);
  }
  // Layer 2, row tile m, folded into the output layer's sums of pairs 2t, 2t + 1 (not unrolled:
  // the loads of one tile at a time stay in flight).
  float s0 = 0.f, s1 = 0.f;
#pragma unroll 1
  for (int m = 0; m < 4; ++m) {
    const float b0 = __ldg(prm + kMlpB2 + 16 * m + g), b1 = __ldg(prm + kMlpB2 + 16 * m + g + 8);
    float d[4] = {b0, b0, b1, b1}, e[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint4* f = frag + kFragL2 + ((m * 4 + k) * 32 + lane) * 2;
      mma_split(d, e, SMEM ? f[0] : __ldg(f), SMEM ? f[1] : __ldg(f + 1), hh[k], hl[k]);
    }
    const float w0 = __ldg(prm + kMlpW3 + 16 * m + g), w1 = __ldg(prm + kMlpW3 + 16 * m + g + 8);
    s0 = fmaf(w1, fmaxf(fmaf(e[2], kLoUnscale, d[2]), 0.f), fmaf(w0, fmaxf(fmaf(e[0], kLoUnscale, d[0]), 0.f), s0));
    s1 = fmaf(w1, fmaxf(fmaf(e[3], kLoUnscale, d[3]), 0.f), fmaf(w0, fmaxf(fmaf(e[1], kLoUnscale, d[1]), 0.f), s1));
  }
  // The eight lanes of a column (t fixed) hold its 64 terms.
#pragma unroll
  for (int o = 4; o < 32; o <<= 1) {
    s0 += __shfl_xor_sync(0xffffffffu, s0, o);
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
  }
  const float b3 = __ldg(prm + kMlpB3);
  return make_float2(b3 + s0, b3 + s1);
}

int launch_mlp_forward(const float* params, const float* feats, int n, float* logits, cudaStream_t st);
int launch_mlp_loss_grad(const float* params, const float* feats, const float* labels, int n, float* grad, float* loss,
                         cudaStream_t st);
int launch_mlp_adam(float* params, const float* grad, float* m, float* v, int t, float lr, float b1, float b2, float eps,
                    cudaStream_t st);

}  // namespace kfgb
