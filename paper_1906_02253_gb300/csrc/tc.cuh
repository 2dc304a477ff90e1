// Fifth-generation tensor cores (tcgen05) for the learned proposal's dense layers: inline PTX for
// tensor-memory allocation, MMA issue from one thread, completion through a shared-memory
// mbarrier, and tensor-memory loads, plus the shared-memory matrix and instruction descriptors.
//
// Operand layout (no swizzle, K-major): a tile of R rows x Kt bf16 columns is stored as 8 x 8
// core matrices of 128 contiguous bytes (8 rows of 16 bytes); element (r, k) sits at byte
//   (r / 8) * SBO + (k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2,   SBO = Kt / 8 * 128,
// so the core matrices of one 8-row group follow each other along K (leading byte offset 128) and
// the 8-row groups follow each other (stride byte offset SBO). One MMA consumes K = 16 (two core
// matrices); the k-th step starts 256 * k bytes further.
//
// FP32-faithful products from bf16 operands: v = hi + mid + lo with hi = bf16(v), mid =
// bf16(v - hi), lo = bf16(v - hi - mid) leaves |v - hi - mid - lo| <= 2^-27 |v|; A * B is
// accumulated in FP32 as hi*hi + hi*mid + mid*hi + hi*lo + lo*hi + mid*mid (six MMAs into the same
// accumulator; the dropped terms are below 2^-26 of the product), which is at least as accurate as
// an FP32 dot product summed in order. Each operand occupies three equal consecutive tiles: hi,
// mid, lo.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace kfgb {
namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor: start address, leading and stride byte offsets (16-byte
// units, 14 bits each), descriptor version 1 (bits 46-47), no base offset, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return static_cast<uint64_t>((addr >> 4) & 0x3FFFu) | (static_cast<uint64_t>((lbo >> 4) & 0x3FFFu) << 16) |
         (static_cast<uint64_t>((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), A and B bf16 (bits 7-9 and
// 10-12 = 1), both K-major (bits 15, 16 = 0), N / 8 in bits 17-22, M / 16 in bits 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(n >> 3) << 17) |
         (static_cast<uint32_t>(m >> 4) << 24);
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// Waits for the mbarrier phase with the given parity to complete; gives up after limit_ns and
// returns false.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint64_t limit_ns = 1000000000ull) {
  const uint32_t a = smem_u32(bar);
  const uint64_t t0 = global_ns();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if (global_ns() - t0 > limit_ns) return false;
  }
}

// Tensor-memory allocation by one whole warp; the column base is written to *dst.
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t base, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(base), "r"(ncols) : "memory");
}

// D (tensor memory) = A * B^T (+ D when accumulate), A from adesc (M x 16), B from bdesc (N x 16).
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// The mbarrier receives one arrival when every MMA issued before by this thread has completed.
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// 16 consecutive FP32 columns of this thread's tensor-memory lane (warp w of a warpgroup reads
// lanes 32 w .. 32 w + 31); the load completes before the values are returned.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint32_t pack_bf16(__nv_bfloat16 a, __nv_bfloat16 b) {
  return static_cast<uint32_t>(__bfloat16_as_ushort(a)) | (static_cast<uint32_t>(__bfloat16_as_ushort(b)) << 16);
}

// Splits 8 consecutive values into their hi, mid and lo bf16 parts and stores them as one 16-byte
// row of a core matrix at byte offset off of each of the three tiles (tile_bytes apart from t0).
__device__ __forceinline__ void store8_split(unsigned char* t0, uint32_t tile_bytes, uint32_t off, const float* v) {
  uint32_t h[4], m[4], l[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    __nv_bfloat16 p[3][2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const float x = v[2 * i + e];
      p[0][e] = __float2bfloat16_rn(x);
      const float r1 = x - __bfloat162float(p[0][e]);
      p[1][e] = __float2bfloat16_rn(r1);
      p[2][e] = __float2bfloat16_rn(r1 - __bfloat162float(p[1][e]));
    }
    h[i] = pack_bf16(p[0][0], p[0][1]);
    m[i] = pack_bf16(p[1][0], p[1][1]);
    l[i] = pack_bf16(p[2][0], p[2][1]);
  }
  *reinterpret_cast<uint4*>(t0 + off) = make_uint4(h[0], h[1], h[2], h[3]);
  *reinterpret_cast<uint4*>(t0 + tile_bytes + off) = make_uint4(m[0], m[1], m[2], m[3]);
  *reinterpret_cast<uint4*>(t0 + 2 * tile_bytes + off) = make_uint4(l[0], l[1], l[2], l[3]);
}

// Byte offset of row r, core-matrix column c (elements 8c .. 8c + 7) in a K-major tile of Kt columns.
__host__ __device__ constexpr uint32_t kmajor_off(int r, int c, int kt) {
  return static_cast<uint32_t>((r >> 3) * (kt / 8) * 128 + c * 128 + (r & 7) * 16);
}

}  // namespace tc
}  // namespace kfgb
