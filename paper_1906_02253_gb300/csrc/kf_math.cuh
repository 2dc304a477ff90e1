// FP32 device math of the Kalman-filter hot path: helix propagation to a barrel cylinder or an
// endcap disk, surface-projected Jacobian and covariance transport C' = J C J^T + Q with
// thin-layer multiple scattering, 2D hit measurement and the Kalman update, seed from three hits.
//
// The paper (arXiv:1906.02253, Sec. 1-2) names the traditional Kalman filter and prints no
// formulas; these are the textbook ones for a helix in a uniform field Bz (Sec. 4: 3.8 T) with
// state (x, y, z, kappa = q/pT, phi, theta) and transverse arc length s as path parameter,
// signed curvature omega = -k Bz kappa. Written for FP32 accuracy: positions advance by small
// increments computed from half-angle sines, the crossing is found by Newton steps on a
// residual assembled from small terms, the small-angle derivatives use series.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace kfgb {

constexpr int kMaxSurf = 64;
constexpr float kPiF = 3.14159265358979323846f;
constexpr float kTwoPiF = 6.28318530717958647692f;
constexpr float kCurvF = 0.00299792458f;  // GeV / (T cm)
constexpr int kPhiSub = 8;                 // phi sub-bins per phi bin (KF_PHI_SUB)
constexpr int kRegions = 5;                // tracking regions of the steering (KF_N_REGIONS)

// Geometry as the kernels see it: passed by value, so it lives in the constant bank.
struct DevGeom {
  float bz, sigma_rphi, sigma_2nd;
  float prior[5];
  int n_surf, n_barrel, n_dpos, n_dneg;
  int n_bins;
  int type[kMaxSurf];
  float r_or_z[kMaxSurf], lo[kMaxSurf], hi[kMaxSurf], x0[kMaxSurf];
  int n_phi[kMaxSurf], n_2nd[kMaxSurf];
  float sphi[kMaxSurf], s2[kMaxSurf];        // FP32 bin scales, rounded once from FP64 on the host
  float sphi_sub[kMaxSurf];                  // FP32 scale of the fine phi index (n_phi * kPhiSub bins)
  signed char barrel_order[kMaxSurf];        // barrel surfaces by increasing radius
  signed char dpos_order[kMaxSurf];          // disks at z > 0 by increasing z
  signed char dneg_order[kMaxSurf];          // disks at z < 0 by decreasing z
  signed char ord[kMaxSurf];                 // index of each surface in its order list above
  float barrel_r[kMaxSurf];                  // radius of barrel_order[i]
  float dpos_z[kMaxSurf], dneg_z[kMaxSurf];  // z of dpos_order[i], dneg_order[i]
  int ms_on;  // multiple scattering
  // Parametrised solenoid field (field_on): Bz(r, z) = bz (1 + fz2 z^2 + fr2 r^2); else bz.
  int field_on;
  float fz2, fr2;
  // Region steering of the finder (steer = 1) or the geometric next-surface rule (steer = 0).
  int steer;
  float c_barrel, c_endcap;
  int steer_n[kRegions];
  signed char steer_list[kRegions][kMaxSurf];  // surfaces of each region, in traversal order
  signed char steer_pos[kRegions][kMaxSurf];   // position of each surface in each list, -1 if absent
};

// Material map and energy loss, a separate launch parameter (read from the constant bank; not in
// the finder's shared-memory geometry copy): x/X0 of surface s at kMatNodes points over its extent.
constexpr int kMatNodes = 8;
struct DevMat {
  int map_on;
  float eloss, mass;  // GeV per unit x/X0 (0: none); particle mass, GeV
  float node[kMaxSurf][kMatNodes];
};

// Packed symmetric 6x6 index, i <= j (upper triangle, row-major).
__host__ __device__ constexpr int ci(int i, int j) { return i <= j ? i * (11 - i) / 2 + j : j * (11 - j) / 2 + i; }

__device__ __forceinline__ float wrap_pi(float a) {
  if (a > kPiF) a -= kTwoPiF;
  if (a <= -kPiF) a += kTwoPiF;
  return a;
}

// sin and cos of state angles and half helix steps by the Cody-Waite reduction (W. J. Cody
// and W. Waite, Software Manual for the Elementary Functions, 1980): x = k pi/2 + r with k =
// rint(2x/pi) and r = ((x - k P1) - k P2) - k P3, pi/2 = P1 + P2 + P3 split into FP32 parts (each
// step one fused multiply-add), |r| <= pi/4 up to rounding; then the Taylor series of sin r to r^9
// and of cos r to r^10 (truncation below 3e-9 at pi/4) and the quadrant rotation by k mod 4. The
// fused reduction keeps r accurate while k is exact in FP32; beyond |x| = 1e5 (no state angle or
// helix step comes near) the result is NaN.
__device__ __forceinline__ void sincos_small(float x, float& s, float& c) {
  if (!(fabsf(x) <= 1e5f)) x = __int_as_float(0x7fc00000);
  const float k = rintf(x * 0.636619747f);  // 2/pi
  float r = fmaf(-k, 1.57079637f, x);
  r = fmaf(-k, -4.37113883e-08f, r);
  r = fmaf(-k, -1.71512451e-15f, r);
  const float r2 = r * r;
  const float sr = fmaf(r * r2, -1.f / 6.f + r2 * (1.f / 120.f + r2 * (-1.f / 5040.f + r2 * (1.f / 362880.f))), r);
  const float cr =
      fmaf(r2, -0.5f + r2 * (1.f / 24.f + r2 * (-1.f / 720.f + r2 * (1.f / 40320.f + r2 * (-1.f / 3628800.f)))), 1.f);
  const int q = static_cast<int>(k) & 3;  // quadrant (two's complement for k < 0)
  const float ss = (q & 1) ? cr : sr, cc = (q & 1) ? sr : cr;
  s = (q & 2) ? -ss : ss;
  c = ((q + 1) & 2) ? -cc : cc;
}

// atan(a / b) for b > 0 and |a| < 0.05 b: its series to t^7 (next term below 2e-11 relative).
__device__ __forceinline__ float atan_small(float a, float b) {
  const float t = a / b, t2 = t * t;
  return t * (1.f + t2 * (-1.f / 3.f + t2 * (1.f / 5.f + t2 * (-1.f / 7.f))));
}

// sin(D/2), cos(D/2) and q = sin(D/2)/(D/2); then f1 = sin(D)/D = q cos(D/2) and
// f2 = (1 - cos D)/D = q sin(D/2).
// Below |D/2| = 0.1 (every step of a track above ~0.1 GeV over a few cm) the Taylor series are
// exact to FP32 (next terms < 3e-11 relative) and cost a few FMAs instead of a range-reduced
// sincos.
__device__ __forceinline__ void half_angle(float D, float& q, float& sh, float& ch) {
  const float h = 0.5f * D;
  if (fabsf(h) < 0.1f) {
    const float h2 = h * h;
    q = 1.f + h2 * (-1.f / 6.f + h2 * (1.f / 120.f + h2 * (-1.f / 5040.f)));
    sh = h * q;
    ch = 1.f + h2 * (-0.5f + h2 * (1.f / 24.f + h2 * (-1.f / 720.f)));
  } else {
    sincos_small(h, sh, ch);
    q = sh / h;
  }
}

// Derivatives d f1/dD and d f2/dD (series below |D| = 0.5, where the closed forms cancel).
__device__ __forceinline__ void helix_dfd(float D, float f1, float q, float cosD, float& d1, float& d2) {
  if (fabsf(D) < 0.5f) {
    const float D2 = D * D;
    d1 = D * (-1.f / 3.f + D2 * (1.f / 30.f + D2 * (-1.f / 840.f + D2 * (1.f / 45360.f))));
    d2 = 0.5f + D2 * (-1.f / 8.f + D2 * (1.f / 144.f + D2 * (-1.f / 5760.f)));
  } else {
    d1 = (cosD - f1) / D;
    d2 = f1 - 0.5f * q * q;
  }
}

struct Prop {
  float s;        // transverse path to the surface
  float f1, f2;   // helix functions at D = omega s
  float q, sh, ch;
  float c0, s0;   // cos, sin of phi at the start
};

__device__ __forceinline__ void prop_eval(Prop& pr, float w) {
  half_angle(w * pr.s, pr.q, pr.sh, pr.ch);
  pr.f1 = pr.q * pr.ch;
  pr.f2 = pr.q * pr.sh;
}

// Smallest s > 0 reaching radius R from state p, by Newton steps on
// g(s) = (rho0^2 - R^2) + 2 p0.dp(s) + |dp(s)|^2, started from the root of its second-order
// expansion dp = s t0 + (omega s^2 / 2) n0: (1 + omega B) s^2 + 2 A s + (rho0^2 - R^2) = 0 with
// A = p0.t0, B = p0.n0 (t0, n0 the unit direction and its left normal).
__device__ __forceinline__ bool path_to_cylinder(const float* p, float w, float R, Prop& pr) {
  sincos_small(p[4], pr.s0, pr.c0);
  const float x0 = p[0], y0 = p[1];
  const float rho0 = sqrtf(x0 * x0 + y0 * y0);
  const float d0 = (rho0 - R) * (rho0 + R);
  const float A = x0 * pr.c0 + y0 * pr.s0;
  const float B = y0 * pr.c0 - x0 * pr.s0;
  const float disc2 = A * A - (1.f + w * B) * d0;
  const float den2 = disc2 >= 0.f ? A + sqrtf(disc2) : -1.f;
  if (den2 > 0.f) {
    pr.s = -d0 / den2;  // near root of the second-order expansion (also when 1 + omega B <= 0)
  } else {
    const float disc = A * A - d0;  // straight line
    if (!(disc >= 0.f)) return false;
    const float den = A + sqrtf(disc);
    if (!(den > 0.f)) return false;
    pr.s = -d0 / den;
  }
  if (!(pr.s > 0.f)) return false;
  // At most 12 Newton steps; the helix functions are evaluated once per pass, the last pass at the
  // final s (one evaluation site keeps the code short).
  bool done = false;
#pragma unroll 1
  for (int it = 0;; ++it) {
    prop_eval(pr, w);
    if (done || it == 12) break;
    const float dx = pr.s * (pr.c0 * pr.f1 - pr.s0 * pr.f2);
    const float dy = pr.s * (pr.s0 * pr.f1 + pr.c0 * pr.f2);
    const float g = d0 + 2.f * (x0 * dx + y0 * dy) + (dx * dx + dy * dy);
    const float cD = 1.f - 2.f * pr.sh * pr.sh, sD = 2.f * pr.sh * pr.ch;
    const float tx = pr.c0 * cD - pr.s0 * sD, ty = pr.s0 * cD + pr.c0 * sD;
    const float gp = 2.f * ((x0 + dx) * tx + (y0 + dy) * ty);
    if (!(gp > 0.f)) return false;
    const float ds = g / gp;
    pr.s -= ds;
    done = fabsf(ds) <= 2e-7f * pr.s;
  }
  return pr.s > 0.f;
}

// Path to the plane z = Z; reached only within half a turn in the transverse plane
// (|omega s| < pi): beyond that the particle would be coming back inward.
__device__ __forceinline__ bool path_to_disk(const float* p, float w, float Z, float st, float ct, Prop& pr) {
  if (ct == 0.f) return false;
  pr.s = (Z - p[2]) * st / ct;
  if (!(pr.s > 0.f)) return false;
  if (!(fabsf(w * pr.s) < kPiF)) return false;
  sincos_small(p[4], pr.s0, pr.c0);
  prop_eval(pr, w);
  return true;
}

// Position reached after path s (used to test a crossing against the surface extent).
__device__ __forceinline__ void prop_position(const float* p, const Prop& pr, float cot, float& x, float& y,
                                              float& z) {
  x = p[0] + pr.s * (pr.c0 * pr.f1 - pr.s0 * pr.f2);
  y = p[1] + pr.s * (pr.s0 * pr.f1 + pr.c0 * pr.f2);
  z = p[2] + pr.s * cot;
}

// Bz at (x, y, z) of the parametrised field.
__device__ __forceinline__ float field_at(const DevGeom& G, float x, float y, float z) {
  return G.bz * (1.f + G.fz2 * z * z + G.fr2 * (x * x + y * y));
}

// Field at the start of a step from state p (the field that decides which surface is next).
__device__ __forceinline__ float start_field(const DevGeom& G, const float* p) {
  return G.field_on ? field_at(G, p[0], p[1], p[2]) : G.bz;
}

__device__ __forceinline__ bool path_to_surface(const DevGeom& G, int si, const float* p, float w, float st, float ct,
                                                Prop& pr) {
  return G.type[si] == 0 ? path_to_cylinder(p, w, G.r_or_z[si], pr) : path_to_disk(p, w, G.r_or_z[si], st, ct, pr);
}

// Field of the step to surface si, whose path in the field at the start is in pr: uniform field,
// that field; parametrised field, the field at the midpoint of the chord p + (s/2) (cos phi,
// sin phi, cot theta), with the path solved again in it. False when that path misses the surface.
__device__ __forceinline__ bool step_field(const DevGeom& G, int si, const float* p, float st, float ct, Prop& pr,
                                           float& bz) {
  if (!G.field_on) {
    bz = G.bz;
    return true;
  }
  const float h = 0.5f * pr.s;
  bz = field_at(G, p[0] + h * pr.c0, p[1] + h * pr.s0, p[2] + h * ct / st);
  return path_to_surface(G, si, p, -kCurvF * bz * p[3], st, ct, pr);
}

__device__ __forceinline__ float highland_var(float p, float x_over_x0) {
  const float t0 = 0.0136f / p * sqrtf(x_over_x0) * (1.f + 0.038f * logf(x_over_x0));
  return t0 * t0;
}

// x/X0 of surface si at second coordinate v: linear between the map's nodes, clamped at the ends.
__device__ __forceinline__ float material_at(const DevMat& M, const DevGeom& G, int si, float v) {
  float u = (v - G.lo[si]) / (G.hi[si] - G.lo[si]) * static_cast<float>(kMatNodes - 1);
  u = fminf(fmaxf(u, 0.f), static_cast<float>(kMatNodes - 1));
  const int k = min(static_cast<int>(floorf(u)), kMatNodes - 2);
  const float a = M.node[si][k], b = M.node[si][k + 1];
  return a + (u - static_cast<float>(k)) * (b - a);
}

// Move state p and covariance C along the helix by pr.s onto surface `si`; C' = J C J^T + Q where
// J = (I - t g^T / g^T t) J_s: J_s at fixed s, t = d(state)/ds, g = gradient of the surface; then
// the mean energy loss in the layer (kappa scaled by p/p', its row and column of C by
// (p/p')^3 E'/E). st, ct: sin and cos of the polar angle p[5] (unchanged by the propagation); bz:
// the field of the step (step_field; its gradient is not propagated into C). EXTRAS = false: a
// variant for geometries without material map and energy loss (the surfaces' x/X0 only).
template <bool EXTRAS = true>
__device__ __forceinline__ bool apply_propagation(const DevGeom& G, const DevMat& M, int si, float* p, float* C,
                                                  const Prop& pr, float st, float ct, float bz) {
  const float a = -kCurvF * bz;  // d omega / d kappa
  const float w = a * p[3];
  const float s = pr.s;
  const float D = w * s;
  const float cot = ct / st;
  const float dx = s * (pr.c0 * pr.f1 - pr.s0 * pr.f2);
  const float dy = s * (pr.s0 * pr.f1 + pr.c0 * pr.f2);
  const float cD = 1.f - 2.f * pr.sh * pr.sh, sD = 2.f * pr.sh * pr.ch;
  float d1, d2;
  helix_dfd(D, pr.f1, pr.q, cD, d1, d2);
  // Jacobian at fixed s.
  const float Jxp = -dy, Jyp = dx;
  const float Jxk = a * s * s * (pr.c0 * d1 - pr.s0 * d2);
  const float Jyk = a * s * s * (pr.s0 * d1 + pr.c0 * d2);
  const float Jzt = -s / (st * st);
  const float Jpk = a * s;
  // New state.
  p[0] += dx;
  p[1] += dy;
  p[2] += s * cot;
  p[4] = wrap_pi(p[4] + D);
  const float tx = pr.c0 * cD - pr.s0 * sD, ty = pr.s0 * cD + pr.c0 * sD;
  // Rows of J_s C for the changed rows 0, 1, 2, 4.
  float R0[6], R1[6], R2[6], R4[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    R0[k] = C[ci(0, k)] + Jxk * C[ci(3, k)] + Jxp * C[ci(4, k)];
    R1[k] = C[ci(1, k)] + Jyk * C[ci(3, k)] + Jyp * C[ci(4, k)];
    R2[k] = C[ci(2, k)] + Jzt * C[ci(5, k)];
    R4[k] = C[ci(4, k)] + Jpk * C[ci(3, k)];
  }
  const float c33 = C[ci(3, 3)], c34 = C[ci(3, 4)], c35 = C[ci(3, 5)], c55 = C[ci(5, 5)];
  // C1 = (J_s C) J_s^T, upper triangle.
  C[ci(0, 0)] = R0[0] + Jxk * R0[3] + Jxp * R0[4];
  C[ci(0, 1)] = R0[1] + Jyk * R0[3] + Jyp * R0[4];
  C[ci(0, 2)] = R0[2] + Jzt * R0[5];
  C[ci(0, 3)] = R0[3];
  C[ci(0, 4)] = R0[4] + Jpk * R0[3];
  C[ci(0, 5)] = R0[5];
  C[ci(1, 1)] = R1[1] + Jyk * R1[3] + Jyp * R1[4];
  C[ci(1, 2)] = R1[2] + Jzt * R1[5];
  C[ci(1, 3)] = R1[3];
  C[ci(1, 4)] = R1[4] + Jpk * R1[3];
  C[ci(1, 5)] = R1[5];
  C[ci(2, 2)] = R2[2] + Jzt * R2[5];
  C[ci(2, 3)] = R2[3];
  C[ci(2, 4)] = R2[4] + Jpk * R2[3];
  C[ci(2, 5)] = R2[5];
  C[ci(3, 4)] = c34 + Jpk * c33;
  C[ci(4, 4)] = R4[4] + Jpk * R4[3];
  C[ci(4, 5)] = R4[5];
  (void)c35;
  (void)c55;
  // Projection onto the surface: with gh = g / (g.t), v = C1 gh, alpha = gh.v,
  // C' = C1 - t v^T - v t^T + alpha t t^T  (t3 = t5 = 0).
  const float t[6] = {tx, ty, cot, 0.f, w, 0.f};
  float g0, g1, g2;
  if (G.type[si] == 0) {
    const float gt = p[0] * tx + p[1] * ty;
    if (!(gt != 0.f)) return false;
    g0 = p[0] / gt;
    g1 = p[1] / gt;
    g2 = 0.f;
  } else {
    if (!(cot != 0.f)) return false;
    g0 = 0.f;
    g1 = 0.f;
    g2 = 1.f / cot;
  }
  float v[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) v[i] = C[ci(i, 0)] * g0 + C[ci(i, 1)] * g1 + C[ci(i, 2)] * g2;
  const float alpha = g0 * v[0] + g1 * v[1] + g2 * v[2];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
#pragma unroll
    for (int j = i; j < 6; ++j) {
      if (i == 3 || i == 5) {
        if (j == 3 || j == 5) continue;
      }
      C[ci(i, j)] += -t[i] * v[j] - v[i] * t[j] + alpha * t[i] * t[j];
    }
  }
  // Thin-layer multiple scattering (Highland, beta = 1) in (kappa, phi, theta) and the mean energy
  // loss, with the material at the crossing.
  float xx0 = G.x0[si];
  if (EXTRAS && M.map_on) xx0 = material_at(M, G, si, G.type[si] == 0 ? p[2] : sqrtf(p[0] * p[0] + p[1] * p[1]));
  const bool ms = G.ms_on && xx0 > 0.f, el = EXTRAS && M.eloss > 0.f && xx0 > 0.f;
  if (ms || el) {
    float cos_a;
    if (G.type[si] == 0) {
      const float r = sqrtf(p[0] * p[0] + p[1] * p[1]);
      cos_a = st * (p[0] * tx + p[1] * ty) / r;
    } else {
      cos_a = ct;
    }
    const float kap = p[3];
    const float pm = 1.f / (fabsf(kap) * st);
    if (ms) {
      const float var = highland_var(pm, xx0 / fabsf(cos_a));
      C[ci(5, 5)] += var;
      C[ci(4, 4)] += var / (st * st);
      C[ci(3, 5)] += -kap * cot * var;
      C[ci(3, 3)] += kap * kap * cot * cot * var;
    }
    if (el) {
      const float m = M.mass, e = sqrtf(pm * pm + m * m);
      const float e1 = e - M.eloss * xx0 / fabsf(cos_a);
      if (!(e1 > m)) return false;  // stopped in the layer
      const float ratio = pm / sqrtf((e1 - m) * (e1 + m));
      const float gk = ratio * ratio * ratio * (e1 / e);
      p[3] = kap * ratio;
#pragma unroll
      for (int j = 0; j < 6; ++j) C[ci(3, j)] *= (j == 3 ? gk * gk : gk);
    }
  }
  return true;
}

// Measurement model of one hit on surface si for state p: residuals r0 (transverse, cm), r1
// (z or r), and the two rows of H restricted to (x, y, z).
struct Meas {
  float r0, r1;
  float h0[3], h1[3];
};

// Predicted position azimuth and the H rows; residuals are filled by meas_residual.
__device__ __forceinline__ void meas_setup(const DevGeom& G, int si, const float* p, Meas& m, float& rho) {
  const float x = p[0], y = p[1];
  const float rho2 = x * x + y * y;
  rho = sqrtf(rho2);
  if (G.type[si] == 0) {
    const float R = G.r_or_z[si];
    m.h0[0] = -R * y / rho2;
    m.h0[1] = R * x / rho2;
    m.h0[2] = 0.f;
    m.h1[0] = 0.f;
    m.h1[1] = 0.f;
    m.h1[2] = 1.f;
  } else {
    m.h0[0] = -y / rho;
    m.h0[1] = x / rho;
    m.h0[2] = 0.f;
    m.h1[0] = x / rho;
    m.h1[1] = y / rho;
    m.h1[2] = 0.f;
  }
}

// Residual of hit (phi_h, v): the angle phi_h - phi_pred comes from the hit direction rotated
// into the predicted position's frame, which avoids subtracting two rounded azimuths.
__device__ __forceinline__ void meas_residual(const DevGeom& G, int si, const float* p, float rho, float phi_h,
                                              float v, Meas& m) {
  float sh, ch;
  sincos_small(phi_h, sh, ch);
  const float x = p[0], y = p[1];
  const float dphi = atan2f(x * sh - y * ch, x * ch + y * sh);
  if (G.type[si] == 0) {
    m.r0 = G.r_or_z[si] * dphi;
    m.r1 = v - p[2];
  } else {
    m.r0 = rho * dphi;
    m.r1 = v - rho;
  }
}

// Innovation covariance S = H C H^T + V (2x2) and the columns C H^T.
struct Innov {
  float ch0[6], ch1[6];
  float s00, s01, s11;
};

__device__ __forceinline__ void innovation(const DevGeom& G, const float* C, const Meas& m, Innov& in) {
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    in.ch0[i] = C[ci(i, 0)] * m.h0[0] + C[ci(i, 1)] * m.h0[1] + C[ci(i, 2)] * m.h0[2];
    in.ch1[i] = C[ci(i, 0)] * m.h1[0] + C[ci(i, 1)] * m.h1[1] + C[ci(i, 2)] * m.h1[2];
  }
  in.s00 = m.h0[0] * in.ch0[0] + m.h0[1] * in.ch0[1] + m.h0[2] * in.ch0[2] + G.sigma_rphi * G.sigma_rphi;
  in.s01 = m.h0[0] * in.ch1[0] + m.h0[1] * in.ch1[1] + m.h0[2] * in.ch1[2];
  in.s11 = m.h1[0] * in.ch1[0] + m.h1[1] * in.ch1[1] + m.h1[2] * in.ch1[2] + G.sigma_2nd * G.sigma_2nd;
}

// True when S is a covariance (positive definite); otherwise no hit can be compatible.
__device__ __forceinline__ bool innovation_ok(const Innov& in) {
  const float det = in.s00 * in.s11 - in.s01 * in.s01;
  return det > 0.f && in.s00 > 0.f;
}

// Kalman update: K = C H^T S^-1, p += K r, C -= K (H C). Returns the predicted chi2.
__device__ __forceinline__ float kalman_update(float* p, float* C, const Innov& in, float r0, float r1) {
  const float det = in.s00 * in.s11 - in.s01 * in.s01;
  const float inv = 1.f / det;
  const float i00 = in.s11 * inv, i01 = -in.s01 * inv, i11 = in.s00 * inv;
  const float chi2 = r0 * (i00 * r0 + i01 * r1) + r1 * (i01 * r0 + i11 * r1);
  float k0[6], k1[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    k0[i] = in.ch0[i] * i00 + in.ch1[i] * i01;
    k1[i] = in.ch0[i] * i01 + in.ch1[i] * i11;
  }
#pragma unroll
  for (int i = 0; i < 6; ++i) p[i] += k0[i] * r0 + k1[i] * r1;
  p[4] = wrap_pi(p[4]);
#pragma unroll
  for (int i = 0; i < 6; ++i) {
#pragma unroll
    for (int j = i; j < 6; ++j) C[ci(i, j)] -= k0[i] * in.ch0[j] + k1[i] * in.ch1[j];
  }
  return chi2;
}

// Hit position in space.
__device__ __forceinline__ void hit_xyz(const DevGeom& G, int si, float phi_h, float v, float& x, float& y,
                                        float& z) {
  float sh, ch;
  sincos_small(phi_h, sh, ch);
  if (G.type[si] == 0) {
    const float R = G.r_or_z[si];
    x = R * ch;
    y = R * sh;
    z = v;
  } else {
    x = v * ch;
    y = v * sh;
    z = G.r_or_z[si];
  }
}

// Seed from three hits: curvature of the circle through them (4 * area / product of sides,
// signed by the turning direction), azimuth at hit 1 = chord direction 1->3 minus half the turning
// angle, arc length 1->3 from the chord, cot(theta) from z over that arc. The prior sits on the
// tangent space of hit 1's surface.
__device__ __forceinline__ bool seed_from_hits(const DevGeom& G, const float* xs, const float* ys, const float* zs,
                                               int si1, float* p, float* C) {
  const float ax = xs[1] - xs[0], ay = ys[1] - ys[0];
  const float bx = xs[2] - xs[0], by = ys[2] - ys[0];
  const float cx = xs[2] - xs[1], cy = ys[2] - ys[1];
  const float la = sqrtf(ax * ax + ay * ay), lb = sqrtf(bx * bx + by * by), lc = sqrtf(cx * cx + cy * cy);
  const float cross = ax * by - ay * bx;  // twice the signed area; > 0 turning left
  if (!(la > 0.f && lb > 0.f && lc > 0.f)) return false;
  const float w = 2.f * cross / (la * lb * lc);
  // Turning angle between hits 1 and 3 and arc length.
  const float hw = 0.5f * lb * w;
  if (!(fabsf(hw) < 1.f)) return false;
  const float half = asinf(hw);                 // half the turning angle
  float s13;
  if (fabsf(hw) < 1e-3f) s13 = lb * (1.f + hw * hw * (1.f / 6.f));
  else s13 = 2.f * half / w;
  const float phi = wrap_pi(atan2f(by, bx) - half);
  const float theta = atan2f(s13, zs[2] - zs[0]);
  p[0] = xs[0];
  p[1] = ys[0];
  p[2] = zs[0];
  p[3] = -w / (kCurvF * (G.field_on ? field_at(G, xs[0], ys[0], zs[0]) : G.bz));  // the field at hit 1
  p[4] = phi;
  p[5] = theta;
#pragma unroll
  for (int i = 0; i < 21; ++i) C[i] = 0.f;
  const float rho = sqrtf(xs[0] * xs[0] + ys[0] * ys[0]);
  const float ux = -ys[0] / rho, uy = xs[0] / rho;  // transverse direction along the surface
  const float su2 = G.prior[0] * G.prior[0], s22 = G.prior[1] * G.prior[1];
  C[ci(0, 0)] = su2 * ux * ux;
  C[ci(0, 1)] = su2 * ux * uy;
  C[ci(1, 1)] = su2 * uy * uy;
  if (G.type[si1] == 0) {
    C[ci(2, 2)] = s22;
  } else {
    const float rx = xs[0] / rho, ry = ys[0] / rho;
    C[ci(0, 0)] += s22 * rx * rx;
    C[ci(0, 1)] += s22 * rx * ry;
    C[ci(1, 1)] += s22 * ry * ry;
  }
  C[ci(3, 3)] = G.prior[2] * G.prior[2];
  C[ci(4, 4)] = G.prior[3] * G.prior[3];
  C[ci(5, 5)] = G.prior[4] * G.prior[4];
  return true;
}

// Hit-index bins by the FP32 rule, every operation separately rounded.
__device__ __forceinline__ int phi_bin(const DevGeom& G, int si, float phi) {
  const float a = __fmul_rn(__fadd_rn(phi, kPiF), G.sphi[si]);
  const float f = floorf(a);
  const int k = (f >= 0.f) ? (f > 1e8f ? 100000000 : static_cast<int>(f)) : -1;
  return min(max(k, 0), G.n_phi[si] - 1);
}

// Fine phi index (n_phi * kPhiSub bins) by the same rule; the sub-bin of a hit in phi-bin pb is
// clamp(fine - pb * kPhiSub, 0, kPhiSub - 1), non-decreasing in phi within the bin.
__device__ __forceinline__ int phi_fine(const DevGeom& G, int si, float phi) {
  const float a = __fmul_rn(__fadd_rn(phi, kPiF), G.sphi_sub[si]);
  const float f = floorf(a);
  const int k = (f >= 0.f) ? (f > 1e8f ? 100000000 : static_cast<int>(f)) : -1;
  return min(max(k, 0), G.n_phi[si] * kPhiSub - 1);
}

__device__ __forceinline__ int sub_of(int fine, int pb) { return min(max(fine - pb * kPhiSub, 0), kPhiSub - 1); }

__device__ __forceinline__ int second_bin(const DevGeom& G, int si, float v) {
  const float a = __fmul_rn(__fsub_rn(v, G.lo[si]), G.s2[si]);
  const float f = floorf(a);
  const int k = (f >= 0.f) ? (f > 1e8f ? 100000000 : static_cast<int>(f)) : -1;
  return min(max(k, 0), G.n_2nd[si] - 1);
}

}  // namespace kfgb
