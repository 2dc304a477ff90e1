// Seed cleaning and duplicate-track removal (paper Sec. 3.2: seeds of the same particle are
// cleaned before finding, using hit identity and the seed's direction; Sec. 4: duplicate tracks
// from several seeds per particle, removed after finding).
//
// Both are decided item by item against the items that share a hit with it, through an inverted
// index hit -> items (counts, an exclusive scan over the hits, then a fill with atomics). The
// order of the items under a hit depends on the fill, the decisions do not: every candidate is
// checked and the rules compare (index, quality), never the order of discovery.
#include <cstddef>

#include "../../include/kfgb.h"
#include "kf_math.cuh"

namespace kfgb {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 2 * kScanThreads;  // counts per scan block

// Items reference hits through lists[k * n + i], k < m (-1: none).
__global__ void k_count_users(const int* __restrict__ lists, int n, int m, int n_hits, int* __restrict__ count) {
  const long long t = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= static_cast<long long>(n) * m) return;
  const int h = lists[t];
  if (h >= 0 && h < n_hits) atomicAdd(count + h, 1);
}

__device__ __forceinline__ int block_exclusive_scan(int v, int* warp_sums, int& total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int u = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += u;
  }
  if (lane == 31) warp_sums[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
    int w = lane < nw ? warp_sums[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += u;
    }
    if (lane < nw) warp_sums[lane] = w;  // inclusive over warps
  }
  __syncthreads();
  total = warp_sums[(blockDim.x >> 5) - 1];
  const int r = incl - v + (wid > 0 ? warp_sums[wid - 1] : 0);
  __syncthreads();
  return r;
}

// Sum of each block's kScanItems counts.
__global__ void __launch_bounds__(kScanThreads) k_scan_sums(const int* __restrict__ count, int n, int* __restrict__ bsum) {
  __shared__ int ws[32];
  const long long base = static_cast<long long>(blockIdx.x) * kScanItems + 2 * threadIdx.x;
  const int v = (base < n ? count[base] : 0) + (base + 1 < n ? count[base + 1] : 0);
  int total;
  block_exclusive_scan(v, ws, total);
  if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

// Exclusive scan of the block sums, one block looping over them.
__global__ void __launch_bounds__(kScanThreads) k_scan_carry(int* __restrict__ bsum, int nb) {
  __shared__ int ws[32];
  int carry = 0;
  for (int b0 = 0; b0 < nb; b0 += kScanThreads) {
    const int b = b0 + static_cast<int>(threadIdx.x);
    const int v = b < nb ? bsum[b] : 0;
    int total;
    const int ex = block_exclusive_scan(v, ws, total);
    if (b < nb) bsum[b] = carry + ex;
    carry += total;
  }
}

// off[i] = sum of count[< i]; off[n] = total.
__global__ void __launch_bounds__(kScanThreads) k_scan_apply(const int* __restrict__ count, int n,
                                                             const int* __restrict__ bsum, int* __restrict__ off) {
  __shared__ int ws[32];
  const long long base = static_cast<long long>(blockIdx.x) * kScanItems + 2 * threadIdx.x;
  const int a = base < n ? count[base] : 0, b = base + 1 < n ? count[base + 1] : 0;
  int total;
  const int ex = block_exclusive_scan(a + b, ws, total) + bsum[blockIdx.x];
  if (base < n) off[base] = ex;
  if (base + 1 < n) off[base + 1] = ex + a;
  if (base + 1 == n || base + 2 == n) off[n] = ex + a + b;  // the thread holding the last count
  if (n == 0 && blockIdx.x == 0 && threadIdx.x == 0) off[0] = 0;
}

__global__ void k_fill_users(const int* __restrict__ lists, int n, int m, int n_hits, const int* __restrict__ off,
                             int* __restrict__ cursor, int* __restrict__ users) {
  const long long t = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= static_cast<long long>(n) * m) return;
  const int h = lists[t];
  if (h >= 0 && h < n_hits) users[off[h] + atomicAdd(cursor + h, 1)] = static_cast<int>(t % n);
}

// Direction (phi, theta) of each seed from its three hits (the seed state at hit 1), NaN when the
// hits give no seed.
__global__ void k_seed_dirs(DevGeom G, const float2* __restrict__ hits, const int* __restrict__ hit_surface,
                            const int* __restrict__ seed_hits, int n, int n_hits, float2* __restrict__ dir) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float xs[3], ys[3], zs[3];
  int s1 = 0;
  bool ok = true;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int h = seed_hits[static_cast<size_t>(k) * n + i];
    ok = ok && h >= 0 && h < n_hits;
    if (!ok) break;
    const int s = hit_surface[h];
    ok = s >= 0 && s < G.n_surf;
    if (!ok) break;
    if (k == 0) s1 = s;
    const float2 hv = hits[h];
    hit_xyz(G, s, hv.x, hv.y, xs[k], ys[k], zs[k]);
  }
  float p[6], C[21];
  ok = ok && seed_from_hits(G, xs, ys, zs, s1, p, C);
  const float nan = __int_as_float(0x7fc00000);
  dir[i] = ok ? make_float2(p[4], p[5]) : make_float2(nan, nan);
}

__device__ __forceinline__ bool directions_agree(float2 a, float2 b, float dphi, float dtheta) {
  return fabsf(wrap_pi(a.x - b.x)) < dphi && fabsf(a.y - b.y) < dtheta;
}

// Seed j is removed when a seed i < j of the same event shares a hit with it and their directions
// agree.
__global__ void k_clean_seeds(const int* __restrict__ seed_hits, const int* __restrict__ seed_event,
                              const float2* __restrict__ dir, const int* __restrict__ off,
                              const int* __restrict__ users, int n, int n_hits, float dphi, float dtheta,
                              int* __restrict__ keep) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const float2 dj = dir[j];
  const int ej = seed_event[j];
  int k_out = 1;
  if (dj.x == dj.x) {
    for (int k = 0; k < 3 && k_out; ++k) {
      const int h = seed_hits[static_cast<size_t>(k) * n + j];
      if (h < 0 || h >= n_hits) continue;
      for (int u = off[h]; u < off[h + 1]; ++u) {
        const int i = users[u];
        if (i < j && seed_event[i] == ej && directions_agree(dir[i], dj, dphi, dtheta)) {
          k_out = 0;
          break;
        }
      }
    }
  }
  keep[j] = k_out;
}

// Track j is removed when a better track i of the same event (more hits, then lower chi2, then
// lower index) with agreeing final direction holds more than half of j's hits.
__global__ void k_remove_duplicates(const int* __restrict__ lists, const int* __restrict__ nhits,
                                    const float* __restrict__ chi2, const float* __restrict__ state,
                                    const int* __restrict__ event, const int* __restrict__ off,
                                    const int* __restrict__ users, int n, int lmax, int n_hits, float dphi,
                                    float dtheta, int* __restrict__ keep) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const float2 dj = make_float2(state[static_cast<size_t>(4) * n + j], state[static_cast<size_t>(5) * n + j]);
  const int ej = event[j], nj = nhits[j];
  const float cj = chi2[j];
  int own = 0;
  for (int k = 0; k < lmax; ++k) own += lists[static_cast<size_t>(k) * n + j] >= 0;
  int k_out = 1;
  for (int k = 0; k < lmax && k_out; ++k) {
    const int h = lists[static_cast<size_t>(k) * n + j];
    if (h < 0 || h >= n_hits) continue;
    for (int u = off[h]; u < off[h + 1] && k_out; ++u) {
      const int i = users[u];
      if (i == j || event[i] != ej) continue;
      const int ni = nhits[i];
      const float ci_ = chi2[i];
      const bool better = ni != nj ? ni > nj : (ci_ != cj ? ci_ < cj : i < j);
      if (!better) continue;
      // checked once: at the first of j's hits that i also holds
      bool first = true;
      for (int k2 = 0; k2 < k && first; ++k2) {
        const int h2 = lists[static_cast<size_t>(k2) * n + j];
        if (h2 < 0 || h2 >= n_hits) continue;
        for (int u2 = off[h2]; u2 < off[h2 + 1]; ++u2)
          if (users[u2] == i) {
            first = false;
            break;
          }
      }
      if (!first) continue;
      const float2 di = make_float2(state[static_cast<size_t>(4) * n + i], state[static_cast<size_t>(5) * n + i]);
      if (!directions_agree(di, dj, dphi, dtheta)) continue;
      int shared = 0;
      for (int a = 0; a < lmax; ++a) {
        const int ha = lists[static_cast<size_t>(a) * n + j];
        if (ha < 0) continue;
        for (int b = 0; b < lmax; ++b)
          if (lists[static_cast<size_t>(b) * n + i] == ha) {
            ++shared;
            break;
          }
      }
      if (2 * shared > own) k_out = 0;
    }
  }
  keep[j] = k_out;
}

// ------------------------------------------------------------------------------------------------

size_t dup_workspace_bytes(int n, int m, int n_hits) {
  auto up = [](size_t v) { return (v + 255) / 256 * 256; };
  const size_t nb = (static_cast<size_t>(n_hits) + kScanItems - 1) / kScanItems + 1;
  return up(static_cast<size_t>(n_hits) * 4) * 2 + up((static_cast<size_t>(n_hits) + 1) * 4) + up(nb * 4) +
         up(static_cast<size_t>(n) * m * 4) + up(static_cast<size_t>(n) * 8);
}

// Inverted index hit -> items of lists (m per item) in the workspace; returns off/users pointers
// and the per-item float2 scratch.
static int build_users(const int* lists, int n, int m, int n_hits, void* ws, cudaStream_t st, const int** off_out,
                       const int** users_out, float2** dir_out) {
  auto up = [](size_t v) { return (v + 255) / 256 * 256; };
  char* p = static_cast<char*>(ws);
  int* count = reinterpret_cast<int*>(p);
  p += up(static_cast<size_t>(n_hits) * 4);
  int* cursor = reinterpret_cast<int*>(p);
  p += up(static_cast<size_t>(n_hits) * 4);
  int* off = reinterpret_cast<int*>(p);
  p += up((static_cast<size_t>(n_hits) + 1) * 4);
  const int nb = (n_hits + kScanItems - 1) / kScanItems;
  int* bsum = reinterpret_cast<int*>(p);
  p += up((static_cast<size_t>(nb) + 1) * 4);
  int* users = reinterpret_cast<int*>(p);
  p += up(static_cast<size_t>(n) * m * 4);
  *dir_out = reinterpret_cast<float2*>(p);
  if (cudaMemsetAsync(count, 0, static_cast<size_t>(n_hits) * 4, st) != cudaSuccess) return KF_ERR_CUDA;
  if (cudaMemsetAsync(cursor, 0, static_cast<size_t>(n_hits) * 4, st) != cudaSuccess) return KF_ERR_CUDA;
  const long long refs = static_cast<long long>(n) * m;
  const int tb = 256;
  if (refs > 0) k_count_users<<<static_cast<int>((refs + tb - 1) / tb), tb, 0, st>>>(lists, n, m, n_hits, count);
  if (nb > 0) {
    k_scan_sums<<<nb, kScanThreads, 0, st>>>(count, n_hits, bsum);
    k_scan_carry<<<1, kScanThreads, 0, st>>>(bsum, nb);
    k_scan_apply<<<nb, kScanThreads, 0, st>>>(count, n_hits, bsum, off);
  } else if (cudaMemsetAsync(off, 0, 4, st) != cudaSuccess) {
    return KF_ERR_CUDA;
  }
  if (refs > 0) k_fill_users<<<static_cast<int>((refs + tb - 1) / tb), tb, 0, st>>>(lists, n, m, n_hits, off, cursor, users);
  *off_out = off;
  *users_out = users;
  return cudaGetLastError() == cudaSuccess ? KF_OK : KF_ERR_CUDA;
}

int launch_clean_seeds(const DevGeom& G, const float2* hits, const int* hit_surface, const int* seed_hits,
                       const int* seed_event, int n, int n_hits, float dphi, float dtheta, int* keep, void* ws,
                       cudaStream_t st) {
  const int* off;
  const int* users;
  float2* dir;
  int rc = build_users(seed_hits, n, 3, n_hits, ws, st, &off, &users, &dir);
  if (rc != KF_OK) return rc;
  const int tb = 128, nbk = (n + tb - 1) / tb;
  k_seed_dirs<<<nbk, tb, 0, st>>>(G, hits, hit_surface, seed_hits, n, n_hits, dir);
  k_clean_seeds<<<nbk, tb, 0, st>>>(seed_hits, seed_event, dir, off, users, n, n_hits, dphi, dtheta, keep);
  return cudaGetLastError() == cudaSuccess ? KF_OK : KF_ERR_CUDA;
}

int launch_remove_duplicates(const int* track_hits, const int* nhits, const float* chi2, const float* state,
                             const int* event, int n, int lmax, int n_hits, float dphi, float dtheta, int* keep,
                             void* ws, cudaStream_t st) {
  const int* off;
  const int* users;
  float2* dir;
  int rc = build_users(track_hits, n, lmax, n_hits, ws, st, &off, &users, &dir);
  if (rc != KF_OK) return rc;
  const int tb = 128;
  k_remove_duplicates<<<(n + tb - 1) / tb, tb, 0, st>>>(track_hits, nhits, chi2, state, event, off, users, n, lmax,
                                                         n_hits, dphi, dtheta, keep);
  return cudaGetLastError() == cudaSuccess ? KF_OK : KF_ERR_CUDA;
}

}  // namespace kfgb
