// Kalman-filter track fit over known hit sequences (paper Sec. 2: track fitting as the first
// vectorised use of the filter). One thread per track in a persistent grid striding over all
// tracks of all events; the state (6) and the packed covariance (21) stay in registers through
// all surfaces; track hit ids are read as structure-of-arrays (coalesced), hits gathered by id.
#include "kf_math.cuh"

namespace kfgb {

__global__ void __launch_bounds__(256) k_fit_tracks(DevGeom G, const __grid_constant__ DevMat M,
                                                    const float2* __restrict__ hits,
                                                    const int* __restrict__ hit_surface,
                                                    const int* __restrict__ track_hits, int n_tracks, int lmax,
                                                    float* __restrict__ state_out, float* __restrict__ cov_out,
                                                    float* __restrict__ chi2_out, int* __restrict__ ndof_out,
                                                    int* __restrict__ status_out) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n_tracks; t += gridDim.x * blockDim.x) {
  float p[6], C[21];
  int status = 0;
  float chi2 = 0.f;
  int nh = 0;
  int id[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) id[k] = track_hits[static_cast<size_t>(k) * n_tracks + t];
  if (id[0] < 0 || id[1] < 0 || id[2] < 0) {
    status = 3;
  } else {
    float xs[3], ys[3], zs[3];
    int s1 = 0;
    bool surf_ok = true;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float2 h = hits[id[k]];
      const int si = hit_surface[id[k]];
      surf_ok &= si >= 0 && si < G.n_surf;
      if (k == 0) s1 = si;
      if (surf_ok) hit_xyz(G, si, h.x, h.y, xs[k], ys[k], zs[k]);
    }
    if (!surf_ok || !seed_from_hits(G, xs, ys, zs, s1, p, C)) {
      status = 1;
    } else {
      // Two-stage prefetch: entry k + 2 of the hit list and hit k + 1 (its coordinates and surface)
      // are loaded while step k computes.
      auto list_at = [&](int k) {
        return k < 3 ? id[k] : (k < lmax ? track_hits[static_cast<size_t>(k) * n_tracks + t] : -1);
      };
      int hid = id[0];
      float2 h = hits[hid];
      int si = hit_surface[hid];
      int hid_n = id[1];
      int hid_nn = list_at(2);
      for (int k = 0; k < lmax; ++k) {
        float2 h_n = make_float2(0.f, 0.f);
        int si_n = -1;
        if (hid_n >= 0) {
          h_n = hits[hid_n];
          si_n = hit_surface[hid_n];
        }
        const int hid_3 = list_at(k + 3);
        if (hid < 0) {
          hid = hid_n, h = h_n, si = si_n, hid_n = hid_nn, hid_nn = hid_3;
          continue;
        }
        if (si < 0 || si >= G.n_surf) {
          status = 2;
          break;
        }
        if (k > 0) {
          const float w = -kCurvF * start_field(G, p) * p[3];
          float st, ct, bz;
          sincos_small(p[5], st, ct);
          Prop pr;
          const bool ok = path_to_surface(G, si, p, w, st, ct, pr) && step_field(G, si, p, st, ct, pr, bz);
          if (!ok || !apply_propagation(G, M, si, p, C, pr, st, ct, bz)) {
            status = 2;
            break;
          }
        }
        Meas m;
        float rho;
        meas_setup(G, si, p, m, rho);
        meas_residual(G, si, p, rho, h.x, h.y, m);
        Innov in;
        innovation(G, C, m, in);
        chi2 += kalman_update(p, C, in, m.r0, m.r1);
        ++nh;
        hid = hid_n, h = h_n, si = si_n, hid_n = hid_nn, hid_nn = hid_3;
      }
    }
  }
  const float nanf_ = __int_as_float(0x7fc00000);
#pragma unroll
  for (int i = 0; i < 6; ++i) state_out[static_cast<size_t>(i) * n_tracks + t] = status == 0 ? p[i] : nanf_;
#pragma unroll
  for (int i = 0; i < 21; ++i) cov_out[static_cast<size_t>(i) * n_tracks + t] = status == 0 ? C[i] : nanf_;
  chi2_out[t] = status == 0 ? chi2 : nanf_;
  // ndof counts every valid entry of the list, as the oracle does.
  int nvalid = nh;
  if (status != 0) {
    nvalid = 0;
    for (int k = 0; k < lmax; ++k) nvalid += track_hits[static_cast<size_t>(k) * n_tracks + t] >= 0;
  }
  ndof_out[t] = 2 * nvalid - 5;
  status_out[t] = status;
  }
}

}  // namespace kfgb
