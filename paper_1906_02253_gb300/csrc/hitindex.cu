// Hit index build: per (event, surface) slab, a counting sort of the hits by bin
// (phi-bin * n_2nd + second-bin), ordered within a bin by (phi sub-bin, hit id). This is the binned
// hit structure behind the per-layer search windows (paper Sec. 3.1) and the reuse of hit data by
// nearby seeds (Sec. 3.2).
//
// One CTA per slab, everything staged in shared memory: the bin (u16) and phi sub-bin (u8) of each
// hit, the bin histogram and its exclusive scan, then an unstable scatter of local hit numbers by
// shared atomics. Each bin's sub-bin counts give its sub-bin offsets; the output pass puts the hit
// at unstable position p of bin [s, e) at s + its rank by (sub-bin, id) among the bin's hits (bins
// hold a handful of hits) and writes the sorted hits, ids and, when asked for, each hit's 16-byte
// search record (cos phi, sin phi, second coordinate, id), so that the search reads one aligned
// record per hit and computes residual angles without trig. The ranks replace a per-bin insertion
// sort, which took 43% of the kernel (one lane per bin, dependent shared loads, lanes diverging
// with the bin sizes).
// Global traffic per hit: one 8-byte read (plus an L2 re-read in the output pass) and a 12-byte
// write (28 bytes with search records).
#include "kf_math.cuh"

namespace kfgb {

static_assert(kPhiSub == 8, "sub-bin offsets are written as eight 16-bit counts");

__global__ void __launch_bounds__(1024, 2) k_build_hit_index(DevGeom G, const float2* __restrict__ hits,
                                                         const int* __restrict__ slab_off, int n_slabs,
                                                         int cap, int* __restrict__ bin_off,
                                                         float2* __restrict__ sorted_hits,
                                                         int* __restrict__ sorted_ids, float4* __restrict__ sorted_rec,
                                                         uint4* __restrict__ sub_off, int* __restrict__ d_status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nb = G.n_bins;
  int* hist = reinterpret_cast<int*>(smem_raw);                       // [nb + 1]
  unsigned short* bin = reinterpret_cast<unsigned short*>(hist + nb + 1);  // [cap]
  unsigned short* order = bin + cap;                                  // [cap]
  unsigned char* sub = reinterpret_cast<unsigned char*>(order + cap);  // [cap]
  __shared__ int warp_sums[32];

  for (int sl = blockIdx.x; sl < n_slabs; sl += gridDim.x) {
    const int si = sl % G.n_surf;
    const int h0 = slab_off[sl];
    const int n = slab_off[sl + 1] - h0;
    int* out = bin_off + static_cast<size_t>(sl) * (nb + 1);
    uint4* sout = sub_off ? sub_off + static_cast<size_t>(sl) * nb : nullptr;
    if (n > cap || n < 0) {
      for (int b = threadIdx.x; b <= nb; b += blockDim.x) out[b] = h0;
      if (sout)
        for (int b = threadIdx.x; b < nb; b += blockDim.x) sout[b] = make_uint4(0u, 0u, 0u, 0u);
      if (threadIdx.x == 0 && d_status) atomicOr(d_status, 1);
      __syncthreads();
      continue;
    }
    const int nbs = G.n_phi[si] * G.n_2nd[si];
    const int n2 = G.n_2nd[si];
    for (int b = threadIdx.x; b <= nb; b += blockDim.x) hist[b] = 0;
    __syncthreads();
    // Four hits per thread per iteration, their loads issued together.
    for (int i0 = threadIdx.x; i0 < n; i0 += 4 * blockDim.x) {
      float2 hv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int i = i0 + u * blockDim.x;
        hv[u] = i < n ? __ldg(hits + h0 + i) : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int i = i0 + u * blockDim.x;
        if (i < n) {
          const int pb = phi_bin(G, si, hv[u].x);
          const int b = pb * n2 + second_bin(G, si, hv[u].y);
          bin[i] = static_cast<unsigned short>(b);
          sub[i] = static_cast<unsigned char>(sub_of(phi_fine(G, si, hv[u].x), pb));
          atomicAdd(&hist[b], 1);
        }
      }
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
    // Sub-bin offsets of each bin (hit counts of its sub-bins, cumulated).
    if (sout) {
      for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        unsigned long long c03 = 0, c47 = 0;  // 16-bit hit counts of sub-bins 0-3 and 4-7
        if (b < nbs) {
          const int e = hist[b];
          const int s = b > 0 ? hist[b - 1] : 0;
          for (int i = s; i < e; ++i) {
            const unsigned sv = sub[order[i]];
            const unsigned long long inc = 1ull << (16 * (sv & 3));
            if (sv < 4) c03 += inc;
            else c47 += inc;
          }
        }
        unsigned cum[kPhiSub];
        unsigned run = 0;
#pragma unroll
        for (int j = 0; j < kPhiSub; ++j) {
          run += static_cast<unsigned>(((j < 4 ? c03 : c47) >> (16 * (j & 3))) & 0xffffull);
          cum[j] = run;
        }
        sout[b] = make_uint4(cum[0] | (cum[1] << 16), cum[2] | (cum[3] << 16), cum[4] | (cum[5] << 16),
                             cum[6] | (cum[7] << 16));
      }
    }
    // Gather: the hit at (unstable) position p of bin [s, e) goes to s + its rank by (sub-bin, id)
    // among the bin's hits; four per thread per iteration with their loads issued together.
    for (int p0 = threadIdx.x; p0 < n; p0 += 4 * blockDim.x) {
      int iv[4], dv[4];
      float2 hv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int p = p0 + u * blockDim.x;
        iv[u] = 0;
        dv[u] = 0;
        if (p < n) {
          const int v = order[p];
          const int b = bin[v];
          const int s = b > 0 ? hist[b - 1] : 0, e = hist[b];
          const unsigned kv = (static_cast<unsigned>(sub[v]) << 16) | static_cast<unsigned>(v);
          int rank = 0;
          for (int q = s; q < e; ++q) {
            const unsigned w = order[q];
            rank += ((static_cast<unsigned>(sub[w]) << 16) | w) < kv;
          }
          iv[u] = v;
          dv[u] = s + rank;
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) hv[u] = p0 + u * static_cast<int>(blockDim.x) < n ? __ldg(hits + h0 + iv[u]) : make_float2(0.f, 0.f);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int p = p0 + u * blockDim.x;
        if (p < n) {
          const int d = h0 + dv[u];
          sorted_hits[d] = hv[u];
          sorted_ids[d] = h0 + iv[u];
          if (sorted_rec) {
            float s, c;
            sincosf(hv[u].x, &s, &c);
            sorted_rec[d] = make_float4(c, s, hv[u].y, __int_as_float(h0 + iv[u]));
          }
        }
      }
    }
    __syncthreads();
  }
}

}  // namespace kfgb
