// Combinatorial Kalman-filter track finding, host side and plain instances: the seed states,
// launch plans (capacity, block size, adaptive capacity), the allocation-free scratch and the
// dispatch of the compiled instances. The kernel itself is in find_kernel.cuh.
#include "find_kernel.cuh"

namespace kfgb {

// Seed states, one thread per seed: the circle seed of the three hits and the filter over them
// (update with hit 1, propagate and update through hits 2 and 3). Written structure-of-arrays
// as kSeedWords words per seed (p[6], C[21], chi2; chi2 < 0 marks a failed seed, whose outputs
// are written here).
__global__ void __launch_bounds__(128) k_seed_states(DevGeom G, const __grid_constant__ DevMat M, FindArgs A) {
  const int seed = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = A.n_seeds;
  if (seed >= n) return;
  int ids[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) ids[k] = A.seed_hits[static_cast<size_t>(k) * n + seed];
  const int ev = A.seed_event[seed];
  const bool removed = A.seed_keep && A.seed_keep[seed] == 0;
  bool ok = !removed && ids[0] >= 0 && ids[1] >= 0 && ids[2] >= 0 && ev >= 0 && ev < A.n_events;
  Cand c;
  int ss[3] = {0, 0, 0};
  if (ok) {
    float xs[3], ys[3], zs[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float2 h = A.hits[ids[k]];
      ss[k] = A.hit_surface[ids[k]];
      ok = ok && ss[k] >= 0 && ss[k] < G.n_surf;
      if (ok) hit_xyz(G, ss[k], h.x, h.y, xs[k], ys[k], zs[k]);
    }
    ok = ok && seed_from_hits(G, xs, ys, zs, ss[0], c.p, c.C);
  }
  c.chi2 = 0.f;
  for (int k = 0; k < 3 && ok; ++k) {
    if (k > 0) {
      const float w = -kCurvF * start_field(G, c.p) * c.p[3];
      float st, ct, bz;
      sincos_small(c.p[5], st, ct);
      Prop pr;
      ok = path_to_surface(G, ss[k], c.p, w, st, ct, pr) && step_field(G, ss[k], c.p, st, ct, pr, bz);
      ok = ok && apply_propagation(G, M, ss[k], c.p, c.C, pr, st, ct, bz);
      if (!ok) break;
    }
    const float2 h = A.hits[ids[k]];
    c.chi2 += update_exact(G, ss[k], c, h.x, h.y);
  }
  float* out = A.seed_state + seed;
  if (ok) {
#pragma unroll
    for (int i = 0; i < 6; ++i) out[static_cast<size_t>(i) * n] = c.p[i];
#pragma unroll
    for (int i = 0; i < 21; ++i) out[static_cast<size_t>(6 + i) * n] = c.C[i];
    out[static_cast<size_t>(27) * n] = c.chi2;
    A.seed_surf[seed] = ss[2];
  } else {
    out[static_cast<size_t>(27) * n] = -1.f;
    if (!A.hits_out) return;  // seed states alone (kf_seed_states): no track outputs
    const float nanf_ = __int_as_float(0x7fc00000);
    for (int k = 0; k < A.lmax; ++k) A.hits_out[static_cast<size_t>(k) * n + seed] = -1;
    A.nhits_out[seed] = 0;
    A.chi2_out[seed] = nanf_;
    for (int i = 0; i < 6; ++i) A.state_out[static_cast<size_t>(i) * n + seed] = nanf_;
    for (int i = 0; i < 21; ++i) A.cov_out[static_cast<size_t>(i) * n + seed] = nanf_;
    A.status_out[seed] = removed ? 2 : 1;
  }
}

// The learned instances' launch and occupancy come from find_learned.cu.
#define KF_LEARNED_INSTANCE(KC, FEAT)                                                                    \
  extern template int find_occupancy<KC, true, FEAT>(int, size_t, int*);                                 \
  extern template void find_launch_kernel<KC, true, FEAT>(const DevGeom&, const DevMat&, const FindArgs&, int, \
                                                          int, size_t, cudaStream_t);
KF_LEARNED_INSTANCE(1, 0) KF_LEARNED_INSTANCE(1, kFeatAll) KF_LEARNED_INSTANCE(2, 0) KF_LEARNED_INSTANCE(2, kFeatAll)
KF_LEARNED_INSTANCE(4, 0) KF_LEARNED_INSTANCE(4, kFeatAll) KF_LEARNED_INSTANCE(6, 0) KF_LEARNED_INSTANCE(6, kFeatAll)
KF_LEARNED_INSTANCE(8, 0) KF_LEARNED_INSTANCE(8, kFeatAll) KF_LEARNED_INSTANCE(16, 0) KF_LEARNED_INSTANCE(16, kFeatAll)
#undef KF_LEARNED_INSTANCE

// Compile-time choice of capacity, mode (plain or learned proposal) and instance (plain, one
// option alone, every option), dispatched from the runtime plan.
template <int KC, bool L, int FEAT>
struct FindKernel {
  static constexpr int kc = KC;
  static constexpr bool learned = L;
  static constexpr int feat = FEAT;
};

// The compiled instance that covers the options in use.
static int compiled_features(bool learned, int feat) {
  if (feat == 0) return 0;
  if (learned) return kFeatAll;
  return (feat == kFeatSteer || feat == kFeatMaterial || feat == kFeatField) ? feat : kFeatAll;
}

template <int KC, class F>
static int dispatch_mode(bool learned, int feat, F&& f) {
  if (learned) return feat == 0 ? f(FindKernel<KC, true, 0>{}) : f(FindKernel<KC, true, kFeatAll>{});
  if (feat == 0) return f(FindKernel<KC, false, 0>{});
  if (feat == kFeatSteer) return f(FindKernel<KC, false, kFeatSteer>{});
  if (feat == kFeatMaterial) return f(FindKernel<KC, false, kFeatMaterial>{});
  if (feat == kFeatField) return f(FindKernel<KC, false, kFeatField>{});
  return f(FindKernel<KC, false, kFeatAll>{});
}

template <class F>
static int dispatch_find(int kc, bool learned, int feat, F&& f) {
  switch (kc) {
    case 1: return dispatch_mode<1>(learned, feat, f);
    case 2: return dispatch_mode<2>(learned, feat, f);
    case 4: return dispatch_mode<4>(learned, feat, f);
    case 6: return dispatch_mode<6>(learned, feat, f);
    case 8: return dispatch_mode<8>(learned, feat, f);
    case 16: return dispatch_mode<16>(learned, feat, f);
    default: return KF_ERR_ARG;
  }
}

// ------------------------------------------------------------------------------------------------

static int pick_kc(int need) {
  static const int caps[] = {1, 2, 4, 6, 8, 16};
  for (int c : caps)
    if (c >= need) return c;
  return -1;
}

int plan_find(int n_seeds, const KfFindParams* p, int sms, int features, FindPlan* plan) {
  if (!p || n_seeds < 0 || sms <= 0) return KF_ERR_ARG;
  if (p->k_max < 1 || p->k_max > KF_MAX_K || p->max_miss < 0 || p->lmax < 4 || p->lmax > KF_MAX_LMAX) return KF_ERR_ARG;
  if (!(p->chi2_cut > 0.f)) return KF_ERR_ARG;
  const bool learned = p->mlp != nullptr && p->top_n > 0;
  if (p->top_n < 0 || p->top_n > KF_MAX_K) return KF_ERR_ARG;
  if (!(p->score_margin >= 0.f) || !(p->score_margin < 3.4e38f)) return KF_ERR_ARG;
  if (p->window_ranking != 0 && p->window_ranking != 1) return KF_ERR_ARG;
  if (p->block_threads != 0 && (p->block_threads < 32 || p->block_threads > 256 || p->block_threads % 32))
    return KF_ERR_ARG;
  if (p->blocks_per_sm < 0) return KF_ERR_ARG;
  if (learned && p->block_threads > kFindMaxBlockLearned) return KF_ERR_CAPACITY;
  if (p->k_capacity < 0 || p->k_capacity > KF_MAX_K) return KF_ERR_ARG;
  const int kc = pick_kc(std::max(learned ? std::max(p->k_max, p->top_n) : p->k_max, p->k_capacity));
  if (kc < 0) return KF_ERR_ARG;
  // Adaptive capacity: a first pass at the smallest compiled capacity >= the requested one, when
  // that is below the full capacity (and, with the learned proposal, holds top_n).
  const int ac = p->adaptive_capacity;
  if (ac < 0 || ac > KF_MAX_K) return KF_ERR_ARG;
  int kc1 = ac > 0 ? pick_kc(ac) : 0;
  if (kc1 >= kc || (learned && p->top_n > kc1)) kc1 = 0;
  // Resident blocks per SM for a block size (shared memory and registers), cached per (device,
  // capacity, mode, block size, lmax) so later calls, e.g. inside a stream capture, only launch.
  const int feat = compiled_features(learned, features);
  const int fi = feat == 0 ? 0 : feat == kFeatSteer ? 1 : feat == kFeatMaterial ? 2 : feat == kFeatField ? 3 : 4;
  static int occ_cache[16][6][2][5][8][32] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 16) return KF_ERR_ARG;
  auto occupancy = [&](int kcx, int blk, size_t* smem_out, int* occ_out) {
    const int ki = kcx == 1 ? 0 : kcx == 2 ? 1 : kcx == 4 ? 2 : kcx == 6 ? 3 : kcx == 8 ? 4 : 5;
    size_t sm = 0;
    dispatch_find(kcx, learned, feat, [&](auto k) {
      sm = block_smem_base<decltype(k)::kc, decltype(k)::learned>() +
           warp_smem_bytes<decltype(k)::kc, decltype(k)::learned>(p->lmax) * (blk / 32);
      return KF_OK;
    });
    *smem_out = sm;
    *occ_out = 0;
    if (sm > 227 * 1024) return KF_OK;
    int& cached = occ_cache[dev][ki][learned][fi][blk / 32 - 1][p->lmax];
    if (cached == 0) {
      int o = 0;
      const int rc = dispatch_find(kcx, learned, feat, [&](auto k) {
        return find_occupancy<decltype(k)::kc, decltype(k)::learned, decltype(k)::feat>(blk, sm, &o);
      });
      if (rc != KF_OK) return rc;
      cached = o > 0 ? o : -1;
    }
    *occ_out = cached > 0 ? cached : 0;
    return KF_OK;
  };
  // Block size (the caller's, or the one that keeps the most warps resident per SM), persistent
  // grid and shared memory of the instance with capacity kcx.
  auto choose = [&](int kcx, int* block_out, int* grid_out, size_t* smem_out) {
    int block = p->block_threads;
    size_t smem = 0;
    int occ = 0;
    if (block != 0) {
      const int rc = occupancy(kcx, block, &smem, &occ);
      if (rc != KF_OK) return rc;
    } else {
      int best_warps = 0;
      for (int blk = learned ? kFindMaxBlockLearned : 256; blk >= 64; blk -= 32) {
        size_t sm = 0;
        int o = 0;
        const int rc = occupancy(kcx, blk, &sm, &o);
        if (rc != KF_OK) return rc;
        if (o * blk / 32 > best_warps) {
          best_warps = o * blk / 32;
          block = blk;
          smem = sm;
          occ = o;
        }
      }
    }
    if (occ < 1) return KF_ERR_CAPACITY;
    int bps = p->blocks_per_sm;
    if (bps == 0 || bps > occ) bps = occ;
    const long long groups_per_block = static_cast<long long>(block / 32) * (32 / kcx);
    const long long want = (static_cast<long long>(n_seeds) + groups_per_block - 1) / groups_per_block;
    *block_out = block;
    *grid_out = static_cast<int>(std::max(1LL, std::min<long long>(static_cast<long long>(sms) * bps, want)));
    *smem_out = smem;
    return KF_OK;
  };
  int rc = choose(kc, &plan->block, &plan->grid, &plan->smem);
  if (rc != KF_OK) return rc;
  plan->kc1 = kc1;
  plan->block1 = plan->grid1 = 0;
  plan->smem1 = 0;
  if (kc1 > 0) {
    rc = choose(kc1, &plan->block1, &plan->grid1, &plan->smem1);
    if (rc != KF_OK) return rc;
  }
  plan->kc = kc;
  plan->learned = learned;
  plan->feat = feat;
  auto up = [](size_t v) { return (v + 255) / 256 * 256; };
  plan->off_state = 256;  // after the work counters
  plan->off_surf = up(plan->off_state + static_cast<size_t>(kSeedWords) * n_seeds * sizeof(float));
  plan->off_mlp = up(plan->off_surf + static_cast<size_t>(n_seeds) * sizeof(int));
  plan->ws_bytes = learned ? up(plan->off_mlp + static_cast<size_t>(kFragWords) * sizeof(uint4)) : plan->off_mlp;
  plan->off_ovf = 0;
  if (kc1 > 0) {
    plan->off_ovf = plan->ws_bytes;
    plan->ws_bytes = up(plan->off_ovf + static_cast<size_t>(n_seeds) * sizeof(int));
  }
  return KF_OK;
}

int launch_seed_states(const DevGeom& G, const DevMat& M, const FindArgs& A, cudaStream_t stream) {
  k_seed_states<<<(A.n_seeds + 127) / 128, 128, 0, stream>>>(G, M, A);
  return cudaGetLastError() == cudaSuccess ? KF_OK : KF_ERR_CUDA;
}

// ------------------------------------------------------------------------------------------------
// Scratch of the allocation-free entry point (kf_find_tracks_static): the work counter, the seed
// states for at most KF_STATIC_MAX_SEEDS seeds and the learned proposal's weight fragments,
// laid out as plan_find lays out a caller's workspace. A fixed array in the library: every GPU that loads the library holds it until the
// process exits. In host code g_find_scratch only names the array; its device address comes from
// cudaGetSymbolAddress, looked up once per device.
constexpr size_t static_scratch_bytes() {
  return (((256 + static_cast<size_t>(kSeedWords) * KF_STATIC_MAX_SEEDS * sizeof(float) + 255) / 256 * 256 +
           static_cast<size_t>(KF_STATIC_MAX_SEEDS) * sizeof(int) + 255) /
              256 * 256 +
          static_cast<size_t>(kFragWords) * sizeof(uint4) + 255) /
         256 * 256;
}
static_assert(static_scratch_bytes() == KF_STATIC_SCRATCH_BYTES, "header and library disagree on the scratch size");
static __device__ __align__(256) unsigned char g_find_scratch[static_scratch_bytes()];

int static_scratch(void** ptr) {
  static void* addr[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return KF_ERR_CUDA;
  if (addr[dev] == nullptr) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_find_scratch) != cudaSuccess || p == nullptr) return KF_ERR_CUDA;
    addr[dev] = p;
  }
  *ptr = addr[dev];
  return KF_OK;
}

int launch_find(const DevGeom& G, const DevMat& M, FindArgs& A, const FindPlan& plan, void* ws, cudaStream_t stream) {
  char* base = static_cast<char*>(ws);
  A.counter = reinterpret_cast<int*>(base);
  A.seed_state = reinterpret_cast<float*>(base + plan.off_state);
  A.seed_surf = reinterpret_cast<int*>(base + plan.off_surf);
  A.mlp_frag = nullptr;
  if (plan.learned) {
    uint4* frag = reinterpret_cast<uint4*>(base + plan.off_mlp);
    if (launch_mlp_fragments(A.mlp, frag, stream) != 0) return KF_ERR_CUDA;
    A.mlp_frag = frag;
  }
  // Work counters: [0] the (first) pass's seed queue, [1] the second pass's, [2] the overflow count.
  if (cudaMemsetAsync(A.counter, 0, 3 * sizeof(int), stream) != cudaSuccess) return KF_ERR_CUDA;
  A.detect = 0;
  A.ovf_list = A.ovf_count = nullptr;
  A.seed_list = A.seed_list_count = nullptr;
  k_seed_states<<<(A.n_seeds + 127) / 128, 128, 0, stream>>>(G, M, A);
  if (plan.kc1 > 0) {
    // First pass at the smaller capacity; its overflowing seeds go to the second pass.
    FindArgs A1 = A;
    A1.detect = 1;
    A1.ovf_list = reinterpret_cast<int*>(base + plan.off_ovf);
    A1.ovf_count = A.counter + 2;
    dispatch_find(plan.kc1, plan.learned, plan.feat, [&](auto k) {
      find_launch_kernel<decltype(k)::kc, decltype(k)::learned, decltype(k)::feat>(G, M, A1, plan.grid1, plan.block1,
                                                                                  plan.smem1, stream);
      return KF_OK;
    });
    A.counter = A.counter + 1;
    A.seed_list = A1.ovf_list;
    A.seed_list_count = A1.ovf_count;
  }
  dispatch_find(plan.kc, plan.learned, plan.feat, [&](auto k) {
    find_launch_kernel<decltype(k)::kc, decltype(k)::learned, decltype(k)::feat>(G, M, A, plan.grid, plan.block,
                                                                                plan.smem, stream);
    return KF_OK;
  });
  return cudaGetLastError() == cudaSuccess ? KF_OK : KF_ERR_CUDA;
}

}  // namespace kfgb
