// Combinatorial Kalman-filter track finding (paper Sec. 2 and Sec. 4): a beam search per seed
// that keeps the k_max best candidates, stepping outward surface by surface, with hits picked
// through binned search windows. Seeds run in parallel with no hit marking between them
// (Sec. 3.2).
//
// Design. One thread per seed in a persistent grid: each warp takes 32 consecutive seeds from an
// atomic work counter (seeds of one event and nearby direction sit next to each other, so a
// warp's windows touch neighbouring bins and reuse cached hits). A thread keeps its seed's
// candidates in a structure-of-arrays workspace (two buffers, current and next, 32 words per
// candidate, word-major so a warp's accesses to the same word coalesce) and the ranking keys
// of the next step in registers. Each parent is propagated once; its passing hits are kept as a
// sorted top-k list; children are updated only when they enter the next step's top k, in
// ranking order, so a parent's remaining children are skipped once one is rejected. A per-step
// trace (parent slot, hit id) is backtracked at the end for the best candidate's hit list.
#include <algorithm>

#include "find_launch.cuh"

namespace kfgb {

constexpr int kWords = 32;
constexpr int kHitBits = 27;  // trace entry: parent slot << 27 | (hit id + 1)

// Ranking key: more hits first, then lower total chi2, then parent rank, then kind (0 hit child,
// 1 miss child, 2 carried), then hit id.
struct Key {
  int nh;
  float c2;
  int pk;   // parent rank << 2 | kind
  int hit;
};

__device__ __forceinline__ bool key_less(const Key& a, const Key& b) {
  if (a.nh != b.nh) return a.nh > b.nh;
  if (a.c2 != b.c2) return a.c2 < b.c2;
  if (a.pk != b.pk) return a.pk < b.pk;
  return a.hit < b.hit;
}

template <int KC>
struct NextList {
  Key k[KC];
  int slot[KC];
  int n;
};

// Would `e` enter a list of capacity cap holding n entries?
template <int KC>
__device__ __forceinline__ bool next_accepts(const NextList<KC>& L, int cap, const Key& e) {
  if (L.n < cap) return true;
  bool acc = false;
#pragma unroll
  for (int i = 0; i < KC; ++i)
    if (i == cap - 1) acc = key_less(e, L.k[i]);
  return acc;
}

// Storage slot the accepted entry will occupy: a fresh one, or the evicted worst's.
template <int KC>
__device__ __forceinline__ int next_slot_for(const NextList<KC>& L, int cap) {
  if (L.n < cap) return L.n;
  int s = 0;
#pragma unroll
  for (int i = 0; i < KC; ++i)
    if (i == cap - 1) s = L.slot[i];
  return s;
}

template <int KC>
__device__ __forceinline__ void next_insert(NextList<KC>& L, int cap, const Key& e, int slot) {
  const int p0 = L.n < cap ? L.n : cap - 1;
  if (L.n < cap) ++L.n;
  bool placed = false;
#pragma unroll
  for (int i = KC - 1; i >= 0; --i) {
    if (i > p0 || placed) continue;
    if (i > 0 && key_less(e, L.k[i - 1])) {
      L.k[i] = L.k[i - 1];
      L.slot[i] = L.slot[i - 1];
    } else {
      L.k[i] = e;
      L.slot[i] = slot;
      placed = true;
    }
  }
}

// A parent's passing hits, sorted by (chi2, hit id), at most cap of them.
template <int KC>
struct HitList {
  float c2[KC];
  int hit[KC];
  int n;
};

template <int KC>
__device__ __forceinline__ void hits_insert(HitList<KC>& L, int cap, float c2, int hit) {
  if (L.n == cap) {
    bool better = false;
#pragma unroll
    for (int i = 0; i < KC; ++i)
      if (i == cap - 1) better = (c2 < L.c2[i]) || (c2 == L.c2[i] && hit < L.hit[i]);
    if (!better) return;
  }
  const int p0 = L.n < cap ? L.n : cap - 1;
  if (L.n < cap) ++L.n;
  bool placed = false;
#pragma unroll
  for (int i = KC - 1; i >= 0; --i) {
    if (i > p0 || placed) continue;
    if (i > 0 && ((c2 < L.c2[i - 1]) || (c2 == L.c2[i - 1] && hit < L.hit[i - 1]))) {
      L.c2[i] = L.c2[i - 1];
      L.hit[i] = L.hit[i - 1];
    } else {
      L.c2[i] = c2;
      L.hit[i] = hit;
      placed = true;
    }
  }
}

struct Cand {
  float p[6];
  float C[21];
  float chi2;
  int nh, nm, stopped, surf;
};

__device__ __forceinline__ float* rec(float* cand, int KC, int buf, int slot, int nt, int tid) {
  return cand + (static_cast<size_t>(buf * KC + slot) * kWords) * nt + tid;
}

__device__ __forceinline__ void store_cand(float* r, int nt, const Cand& c) {
#pragma unroll
  for (int i = 0; i < 6; ++i) r[static_cast<size_t>(i) * nt] = c.p[i];
#pragma unroll
  for (int i = 0; i < 21; ++i) r[static_cast<size_t>(6 + i) * nt] = c.C[i];
  r[static_cast<size_t>(27) * nt] = c.chi2;
  r[static_cast<size_t>(28) * nt] = __int_as_float(c.nh);
  r[static_cast<size_t>(29) * nt] = __int_as_float(c.nm);
  r[static_cast<size_t>(30) * nt] = __int_as_float(c.stopped);
  r[static_cast<size_t>(31) * nt] = __int_as_float(c.surf);
}

__device__ __forceinline__ void load_cand(const float* r, int nt, Cand& c) {
#pragma unroll
  for (int i = 0; i < 6; ++i) c.p[i] = r[static_cast<size_t>(i) * nt];
#pragma unroll
  for (int i = 0; i < 21; ++i) c.C[i] = r[static_cast<size_t>(6 + i) * nt];
  c.chi2 = r[static_cast<size_t>(27) * nt];
  c.nh = __float_as_int(r[static_cast<size_t>(28) * nt]);
  c.nm = __float_as_int(r[static_cast<size_t>(29) * nt]);
  c.stopped = __float_as_int(r[static_cast<size_t>(30) * nt]);
  c.surf = __float_as_int(r[static_cast<size_t>(31) * nt]);
}

// Next surface outward and the path to it: the next barrel layer beyond the candidate's radius
// (accepted if crossed within its z extent) and the next disk beyond |z| in the direction of
// motion (accepted if crossed within its r extent); the nearer accepted one. -1 if none.
__device__ __forceinline__ int next_surface(const DevGeom& G, const float* p, Prop& best) {
  const float w = -kCurvF * G.bz * p[3];
  const float rho = sqrtf(p[0] * p[0] + p[1] * p[1]);
  float st, ct;
  sincosf(p[5], &st, &ct);
  const float cot = ct / st;
  int sel = -1;
  for (int i = 0; i < G.n_barrel; ++i) {
    const int s = G.barrel_order[i];
    if (G.r_or_z[s] > rho + 0.01f) {
      Prop pr;
      if (path_to_cylinder(p, w, G.r_or_z[s], pr)) {
        const float z = p[2] + pr.s * cot;
        if (z >= G.lo[s] && z <= G.hi[s]) {
          sel = s;
          best = pr;
        }
      }
      break;
    }
  }
  const int nd = cot > 0.f ? G.n_dpos : (cot < 0.f ? G.n_dneg : 0);
  for (int i = 0; i < nd; ++i) {
    const int s = cot > 0.f ? G.dpos_order[i] : G.dneg_order[i];
    const float Z = G.r_or_z[s];
    if ((cot > 0.f && Z > p[2] + 0.01f) || (cot < 0.f && Z < p[2] - 0.01f)) {
      Prop pr;
      if (path_to_disk(p, w, Z, pr)) {
        float x, y, z;
        prop_position(p, pr, cot, x, y, z);
        const float r = sqrtf(x * x + y * y);
        if (r >= G.lo[s] && r <= G.hi[s] && (sel < 0 || pr.s < best.s)) {
          sel = s;
          best = pr;
        }
      }
      break;
    }
  }
  return sel;
}

// Every hit of surface si in event ev with chi2 below the cut for the predicted state (p, C),
// through the padded bounding box of the chi2 ellipse turned into bin ranges.
template <int KC>
__device__ __forceinline__ void search_window(const DevGeom& G, const FindArgs& A, int ev, int si, const float* p,
                                              const float* C, int cap, HitList<KC>& out) {
  out.n = 0;
  Meas m;
  float rho;
  meas_setup(G, si, p, m, rho);
  Innov in;
  innovation(G, C, m, in);
  const float cut = A.chi2_cut;
  const float rref = G.type[si] == 0 ? G.r_or_z[si] : rho;
  const float dphi = sqrtf(cut * in.s00) / rref * (1.f + 1e-4f) + 1e-5f;
  const float d2 = sqrtf(cut * in.s11) * (1.f + 1e-4f) + 1e-4f;
  const float phip = atan2f(p[1], p[0]);
  const float c2 = G.type[si] == 0 ? p[2] : rho;
  const int nphi = G.n_phi[si], n2 = G.n_2nd[si];
  int pb0, npb;
  if (!(dphi < kPiF * (1.f - 2.f / nphi))) {
    pb0 = 0;
    npb = nphi;
  } else {
    pb0 = phi_bin(G, si, wrap_pi(phip - dphi));
    const int pb1 = phi_bin(G, si, wrap_pi(phip + dphi));
    npb = ((pb1 - pb0) % nphi + nphi) % nphi + 1;
  }
  const int zb0 = second_bin(G, si, c2 - d2);
  const int zb1 = second_bin(G, si, c2 + d2);
  const float det = in.s00 * in.s11 - in.s01 * in.s01;
  const float inv = 1.f / det;
  const float i00 = in.s11 * inv, i01 = -in.s01 * inv, i11 = in.s00 * inv;
  const int* off = A.bin_off + static_cast<size_t>(ev * G.n_surf + si) * (G.n_bins + 1);
  for (int k = 0; k < npb; ++k) {
    int pb = pb0 + k;
    if (pb >= nphi) pb -= nphi;
    const int a = __ldg(off + pb * n2 + zb0);
    const int b = __ldg(off + pb * n2 + zb1 + 1);
    for (int q = a; q < b; ++q) {
      const float2 h = __ldg(A.sorted_hits + q);
      meas_residual(G, si, p, rho, h.x, h.y, m);
      const float c = m.r0 * (i00 * m.r0 + i01 * m.r1) + m.r1 * (i01 * m.r0 + i11 * m.r1);
      if (c < cut) hits_insert<KC>(out, cap, c, __ldg(A.sorted_ids + q));
    }
  }
}

__device__ __forceinline__ float kf_step_update(const DevGeom& G, int si, Cand& c, float phi_h, float v) {
  Meas m;
  float rho;
  meas_setup(G, si, c.p, m, rho);
  meas_residual(G, si, c.p, rho, phi_h, v, m);
  Innov in;
  innovation(G, c.C, m, in);
  return kalman_update(c.p, c.C, in, m.r0, m.r1);
}

template <int KC>
__device__ __forceinline__ void find_one_seed(const DevGeom& G, const FindArgs& A, int seed, int tid) {
    const int nt = A.nt;
    const int cap = A.k_max;
    const float nanf_ = __int_as_float(0x7fc00000);
    const int n = A.n_seeds;
    // ---- seed fit ------------------------------------------------------------------------
    int ids[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) ids[k] = A.seed_hits[static_cast<size_t>(k) * n + seed];
    const int ev = A.seed_event[seed];
    Cand c;
    bool ok = ids[0] >= 0 && ids[1] >= 0 && ids[2] >= 0 && ev >= 0 && ev < A.n_events;
    if (ok) {
      float xs[3], ys[3], zs[3];
      int ss[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float2 h = A.hits[ids[k]];
        ss[k] = A.hit_surface[ids[k]];
        ok &= ss[k] >= 0 && ss[k] < G.n_surf;
        if (ok) hit_xyz(G, ss[k], h.x, h.y, xs[k], ys[k], zs[k]);
      }
      ok = ok && seed_from_hits(G, xs, ys, zs, ss[0], c.p, c.C);
      c.chi2 = 0.f;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        if (!ok) break;
        if (k > 0) {
          const float w = -kCurvF * G.bz * c.p[3];
          Prop pr;
          ok = G.type[ss[k]] == 0 ? path_to_cylinder(c.p, w, G.r_or_z[ss[k]], pr)
                                  : path_to_disk(c.p, w, G.r_or_z[ss[k]], pr);
          if (ok) ok = apply_propagation(G, ss[k], c.p, c.C, pr);
          if (!ok) break;
        }
        const float2 h = A.hits[ids[k]];
        c.chi2 += kf_step_update(G, ss[k], c, h.x, h.y);
      }
      c.surf = ss[2];
    }
    if (!ok) {
      for (int k = 0; k < A.lmax; ++k) A.hits_out[static_cast<size_t>(k) * n + seed] = -1;
      A.nhits_out[seed] = 0;
      A.chi2_out[seed] = nanf_;
      for (int i = 0; i < 6; ++i) A.state_out[static_cast<size_t>(i) * n + seed] = nanf_;
      for (int i = 0; i < 21; ++i) A.cov_out[static_cast<size_t>(i) * n + seed] = nanf_;
      A.status_out[seed] = 1;
      return;
    }
    c.nh = 3;
    c.nm = 0;
    c.stopped = 0;
    store_cand(rec(A.cand, KC, 0, 0, nt, tid), nt, c);
    int ncur = 1;
    unsigned long long cur_slots = 0ull;  // storage slot of rank r in bits [4r, 4r+4)
    int cur = 0;
    int nsteps = 0;
    bool any_active = true;
    // ---- steps ---------------------------------------------------------------------------
    for (int step = 0; step < A.lmax - 3 && any_active; ++step) {
      NextList<KC> L;
      L.n = 0;
      const int nxt = cur ^ 1;
      int* trace_step = A.trace + static_cast<size_t>(step) * KC * nt + tid;
      for (int r = 0; r < ncur; ++r) {
        const int pslot = static_cast<int>((cur_slots >> (4 * r)) & 0xFull);
        float* prec = rec(A.cand, KC, cur, pslot, nt, tid);
        load_cand(prec, nt, c);
        int kind = 2;  // carried unless a child is produced
        HitList<KC> H;
        H.n = 0;
        int si = -1;
        if (!c.stopped) {
          Prop pr;
          si = next_surface(G, c.p, pr);
          if (si >= 0 && apply_propagation(G, si, c.p, c.C, pr)) {
            search_window<KC>(G, A, ev, si, c.p, c.C, cap, H);
            kind = H.n > 0 ? 0 : (c.nm < A.max_miss ? 1 : 2);
          } else {
            si = -1;
          }
        }
        if (kind == 0) {
          if (H.n > 1) store_cand(prec, nt, c);  // the prediction, for the other children
          const float parent_chi2 = c.chi2;
          const int parent_nh = c.nh;
#pragma unroll
          for (int j = 0; j < KC; ++j) {
            if (j >= H.n) break;
            const Key e{parent_nh + 1, parent_chi2 + H.c2[j], (r << 2) | 0, H.hit[j]};
            if (!next_accepts<KC>(L, cap, e)) break;
            if (j > 0) load_cand(prec, nt, c);
            const int hid = H.hit[j];
            const float2 h = __ldg(A.hits + hid);
            kf_step_update(G, si, c, h.x, h.y);
            c.chi2 = e.c2;
            c.nh = parent_nh + 1;
            c.surf = si;
            const int ns = next_slot_for<KC>(L, cap);
            store_cand(rec(A.cand, KC, nxt, ns, nt, tid), nt, c);
            trace_step[static_cast<size_t>(ns) * nt] = (pslot << kHitBits) | (hid + 1);
            next_insert<KC>(L, cap, e, ns);
          }
        } else {
          const Key e{c.nh, c.chi2, (r << 2) | kind, -1};
          if (next_accepts<KC>(L, cap, e)) {
            if (kind == 1) {
              c.nm += 1;
              c.surf = si;
            } else {
              if (!c.stopped) load_cand(prec, nt, c);  // undo the prediction
              c.stopped = 1;
            }
            const int ns = next_slot_for<KC>(L, cap);
            store_cand(rec(A.cand, KC, nxt, ns, nt, tid), nt, c);
            trace_step[static_cast<size_t>(ns) * nt] = pslot << kHitBits;
            next_insert<KC>(L, cap, e, ns);
          }
        }
      }
      // Promote the next list.
      ncur = L.n;
      cur_slots = 0ull;
      any_active = false;
#pragma unroll
      for (int i = 0; i < KC; ++i) {
        if (i < L.n) {
          cur_slots |= static_cast<unsigned long long>(L.slot[i]) << (4 * i);
          any_active |= (L.k[i].pk & 3) != 2;
        }
      }
      cur ^= 1;
      nsteps = step + 1;
    }
    // ---- output: best candidate, hit list by backtracking ----------------------------------
    int slot = static_cast<int>(cur_slots & 0xFull);
    load_cand(rec(A.cand, KC, cur, slot, nt, tid), nt, c);
    for (int k = A.lmax - 1; k >= 3 + nsteps; --k) A.hits_out[static_cast<size_t>(k) * n + seed] = -1;
    for (int step = nsteps - 1; step >= 0; --step) {
      const int e = A.trace[(static_cast<size_t>(step) * KC + slot) * nt + tid];
      const int hit = (e & ((1 << kHitBits) - 1)) - 1;
      A.hits_out[static_cast<size_t>(3 + step) * n + seed] = hit;
      slot = e >> kHitBits;
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) A.hits_out[static_cast<size_t>(k) * n + seed] = ids[k];
    A.nhits_out[seed] = c.nh;
    A.chi2_out[seed] = c.chi2;
#pragma unroll
    for (int i = 0; i < 6; ++i) A.state_out[static_cast<size_t>(i) * n + seed] = c.p[i];
#pragma unroll
    for (int i = 0; i < 21; ++i) A.cov_out[static_cast<size_t>(i) * n + seed] = c.C[i];
    A.status_out[seed] = 0;
}

template <int KC>
__global__ void __launch_bounds__(128) k_find_tracks(DevGeom G, FindArgs A) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  for (;;) {
    int base = 0;
    if (lane == 0) base = atomicAdd(A.counter, 32);
    base = __shfl_sync(0xffffffffu, base, 0);
    if (base >= A.n_seeds) break;
    const int seed = base + lane;
    if (seed < A.n_seeds) find_one_seed<KC>(G, A, seed, tid);
    __syncwarp();
  }
}

template __global__ void k_find_tracks<1>(DevGeom, FindArgs);
template __global__ void k_find_tracks<2>(DevGeom, FindArgs);
template __global__ void k_find_tracks<4>(DevGeom, FindArgs);
template __global__ void k_find_tracks<8>(DevGeom, FindArgs);
template __global__ void k_find_tracks<16>(DevGeom, FindArgs);

}  // namespace kfgb

namespace kfgb {

int plan_find(int n_seeds, const KfFindParams* p, int sms, FindPlan* plan) {
  if (!p || n_seeds < 0 || sms <= 0) return KF_ERR_ARG;
  if (p->k_max < 1 || p->k_max > KF_MAX_K || p->max_miss < 0 || p->lmax < 3 || p->lmax > KF_MAX_LMAX) return KF_ERR_ARG;
  if (!(p->chi2_cut > 0.f)) return KF_ERR_ARG;
  const int block = p->block_threads == 0 ? 128 : p->block_threads;
  if (block < 32 || block > 128 || block % 32) return KF_ERR_ARG;
  int kc = 1;
  while (kc < p->k_max) kc *= 2;
  int bps = p->blocks_per_sm;
  if (bps < 0) return KF_ERR_ARG;
  // Occupancy per (device, capacity, block size), queried once so later calls (for instance
  // inside a stream capture) only launch.
  static int occ_cache[16][5][5] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 16) return KF_ERR_ARG;
  const int ki = kc == 1 ? 0 : kc == 2 ? 1 : kc == 4 ? 2 : kc == 8 ? 3 : 4;
  const int bi = block / 32 - 1;
  if (bps == 0 && occ_cache[dev][ki][bi] > 0) bps = occ_cache[dev][ki][bi];
  if (bps == 0) {
    cudaError_t e = cudaSuccess;
    switch (kc) {
      case 1: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_find_tracks<1>, block, 0); break;
      case 2: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_find_tracks<2>, block, 0); break;
      case 4: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_find_tracks<4>, block, 0); break;
      case 8: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_find_tracks<8>, block, 0); break;
      default: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_find_tracks<16>, block, 0); break;
    }
    if (e != cudaSuccess || bps < 1) bps = 1;
    occ_cache[dev][ki][bi] = bps;
  }
  const long long want = (static_cast<long long>(n_seeds) + block - 1) / block;
  const int grid = static_cast<int>(std::max(1LL, std::min<long long>(static_cast<long long>(sms) * bps, want)));
  plan->kc = kc;
  plan->block = block;
  plan->grid = grid;
  plan->nt = grid * block;
  const size_t align = 256;
  auto up = [&](size_t v) { return (v + align - 1) / align * align; };
  plan->off_cand = align;
  const size_t cand_bytes = 2ull * kc * kWords * plan->nt * sizeof(float);
  plan->off_trace = up(plan->off_cand + cand_bytes);
  const size_t trace_bytes = static_cast<size_t>(p->lmax) * kc * plan->nt * sizeof(int);
  plan->ws_bytes = up(plan->off_trace + trace_bytes);
  return KF_OK;
}

int launch_find(const DevGeom& G, FindArgs& A, const FindPlan& plan, void* ws, cudaStream_t stream) {
  char* base = static_cast<char*>(ws);
  A.counter = reinterpret_cast<int*>(base);
  A.cand = reinterpret_cast<float*>(base + plan.off_cand);
  A.trace = reinterpret_cast<int*>(base + plan.off_trace);
  A.nt = plan.nt;
  if (cudaMemsetAsync(A.counter, 0, sizeof(int), stream) != cudaSuccess) return KF_ERR_CUDA;
  switch (plan.kc) {
    case 1: k_find_tracks<1><<<plan.grid, plan.block, 0, stream>>>(G, A); break;
    case 2: k_find_tracks<2><<<plan.grid, plan.block, 0, stream>>>(G, A); break;
    case 4: k_find_tracks<4><<<plan.grid, plan.block, 0, stream>>>(G, A); break;
    case 8: k_find_tracks<8><<<plan.grid, plan.block, 0, stream>>>(G, A); break;
    default: k_find_tracks<16><<<plan.grid, plan.block, 0, stream>>>(G, A); break;
  }
  return cudaGetLastError() == cudaSuccess ? KF_OK : KF_ERR_CUDA;
}

}  // namespace kfgb
