// Probe of the bounded wait that the tensor-core kernels use for MMA completion (measurement only,
// not on the path): one warp waits on a shared-memory mbarrier that receives no arrival, with the
// caller's limit, then on the same barrier after its one expected arrival. A test checks that the
// first wait gives up after the limit and returns (no hang, the context stays usable) and that the
// second completes.
#include "../../include/kfgb.h"
#include "tc.cuh"

namespace kfgb {

__global__ void k_wait_probe(unsigned long long limit_ns, long long* __restrict__ out) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) tc::mbar_init(&bar, 1);
  __syncwarp();
  const uint64_t t0 = tc::global_ns();
  const bool first = tc::mbar_wait(&bar, 0, limit_ns);
  const uint64_t t1 = tc::global_ns();
  __syncwarp();
  if (threadIdx.x == 0) {
    uint64_t state;
    asm volatile("mbarrier.arrive.shared::cta.b64 %0, [%1];" : "=l"(state) : "r"(tc::smem_u32(&bar)) : "memory");
    (void)state;
  }
  __syncwarp();
  const bool second = tc::mbar_wait(&bar, 0, limit_ns);
  if (threadIdx.x == 0) {
    out[0] = first ? 1 : 0;
    out[1] = second ? 1 : 0;
    out[2] = static_cast<long long>(t1 - t0);
  }
}

int launch_wait_probe(int limit_us, long long* out, cudaStream_t st) {
  k_wait_probe<<<1, 32, 0, st>>>(1000ull * static_cast<unsigned long long>(limit_us), out);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

}  // namespace kfgb
