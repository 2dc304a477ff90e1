// Hit index build: per (event, surface) slab, a counting sort of the hits by bin
// (phi-bin * n_2nd + second-bin), ascending hit id within a bin. This is the binned hit
// structure behind the per-layer search windows (paper Sec. 3.1) and the reuse of hit data by
// nearby seeds (Sec. 3.2).
//
// One CTA per slab, everything staged in shared memory: the bin of each hit (u16), the bin
// histogram and its exclusive scan, then an unstable scatter of local hit numbers by shared
// atomics, then a per-bin insertion sort that restores ascending id (bins hold a handful of
// hits), then a coalesced gather-write of the sorted hits and ids and, when asked for, of each
// hit's direction (cos phi, sin phi) so that the search computes residual angles without trig.
// Global traffic per hit: one 8-byte read (plus an L2 re-read in the gather) and a 12-byte write
// (20 bytes with directions).
#include "kf_math.cuh"

namespace kfgb {

__global__ void __launch_bounds__(512) k_build_hit_index(DevGeom G, const float2* __restrict__ hits,
                                                         const int* __restrict__ slab_off, int n_slabs,
                                                         int cap, int* __restrict__ bin_off,
                                                         float2* __restrict__ sorted_hits,
                                                         int* __restrict__ sorted_ids, float2* __restrict__ sorted_dir,
                                                         int* __restrict__ d_status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nb = G.n_bins;
  int* hist = reinterpret_cast<int*>(smem_raw);                       // [nb + 1]
  unsigned short* bin = reinterpret_cast<unsigned short*>(hist + nb + 1);  // [cap]
  unsigned short* order = bin + cap;                                  // [cap]
  __shared__ int warp_sums[32];

  for (int sl = blockIdx.x; sl < n_slabs; sl += gridDim.x) {
    const int si = sl % G.n_surf;
    const int h0 = slab_off[sl];
    const int n = slab_off[sl + 1] - h0;
    int* out = bin_off + static_cast<size_t>(sl) * (nb + 1);
    if (n > cap || n < 0) {
      for (int b = threadIdx.x; b <= nb; b += blockDim.x) out[b] = h0;
      if (threadIdx.x == 0 && d_status) atomicOr(d_status, 1);
      __syncthreads();
      continue;
    }
    const int nbs = G.n_phi[si] * G.n_2nd[si];
    const int n2 = G.n_2nd[si];
    for (int b = threadIdx.x; b <= nb; b += blockDim.x) hist[b] = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const float2 h = hits[h0 + i];
      const int b = phi_bin(G, si, h.x) * n2 + second_bin(G, si, h.y);
      bin[i] = static_cast<unsigned short>(b);
      atomicAdd(&hist[b], 1);
    }
    __syncthreads();
    // Exclusive scan of hist[0, nbs) in place: each thread scans a contiguous chunk.
    const int per = (nbs + blockDim.x - 1) / blockDim.x;
    const int b0 = min(nbs, static_cast<int>(threadIdx.x) * per), b1 = min(nbs, b0 + per);
    int local = 0;
    for (int b = b0; b < b1; ++b) local += hist[b];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int incl = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    if (lane == 31) warp_sums[wid] = incl;
    __syncthreads();
    if (wid == 0) {
      const int nw = blockDim.x >> 5;
      int v = lane < nw ? warp_sums[lane] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
      }
      if (lane < nw) warp_sums[lane] = v;  // inclusive over warps
    }
    __syncthreads();
    int run = incl - local + (wid > 0 ? warp_sums[wid - 1] : 0);
    for (int b = b0; b < b1; ++b) {
      const int c = hist[b];
      hist[b] = run;
      run += c;
    }
    __syncthreads();
    for (int b = threadIdx.x; b <= nb; b += blockDim.x) out[b] = h0 + (b < nbs ? hist[b] : n);
    __syncthreads();
    // Unstable scatter: hist[b] becomes the end of bin b.
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const int pos = atomicAdd(&hist[bin[i]], 1);
      order[pos] = static_cast<unsigned short>(i);
    }
    __syncthreads();
    // Restore ascending hit id inside each bin.
    for (int b = threadIdx.x; b < nbs; b += blockDim.x) {
      const int e = hist[b];
      const int s = b > 0 ? hist[b - 1] : 0;
      for (int i = s + 1; i < e; ++i) {
        const unsigned short v = order[i];
        int j = i - 1;
        while (j >= s && order[j] > v) {
          order[j + 1] = order[j];
          --j;
        }
        order[j + 1] = v;
      }
    }
    __syncthreads();
    for (int p = threadIdx.x; p < n; p += blockDim.x) {
      const int i = order[p];
      const float2 h = hits[h0 + i];
      sorted_hits[h0 + p] = h;
      sorted_ids[h0 + p] = h0 + i;
      if (sorted_dir) {
        float s, c;
        sincosf(h.x, &s, &c);
        sorted_dir[h0 + p] = make_float2(c, s);
      }
    }
    __syncthreads();
  }
}

}  // namespace kfgb
