// FP64 CPU oracle for Kalman-filter track fitting and combinatorial track finding.
//
// TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check and the benchmark's CPU
// baseline leg may load this library. It shares no code with the CUDA path.
//
// What it follows. The paper (Sec. 1, Sec. 2) adapts the traditional Kalman filter to track
// fitting and combinatorial track finding, propagates layer to layer (Sec. 3.1), accounts for
// multiple scattering from the detector material (Sec. 3.1), uses a constant 3.8 T field
// (Sec. 4), selects hits through per-layer search windows and scores candidates (Sec. 4),
// and processes seeds in parallel without marking used hits (Sec. 3.2). It prints no formulas,
// so every formula below is the textbook one, written out plainly:
//   * helix motion in a uniform field Bz, state (x, y, z, kappa = q/pT, phi, theta), transverse
//     arc length s as the path parameter, signed curvature omega = -k*Bz*kappa;
//   * crossing of a cylinder by circle-circle intersection, of a disk by z = z0 + s*cot(theta);
//   * Jacobian of the fixed-s map, projected onto the surface (I - t g^T / g^T t);
//   * covariance transport C' = J C J^T + Q, Q from the Highland formula (PDG, beta = 1);
//   * extended Kalman update with 2D hits (barrel: r*phi and z; disk: r*phi and r);
//   * hit binning with the FP32 rounding rule below; beam search keeping K candidates;
//   * the options the paper describes (Sec. 3.1, Sec. 3.2): region steering lists, an r-z material
//     map with mean energy loss, a parametrised solenoid field (one helix per step in the field at
//     the chord's midpoint), seed cleaning and duplicate-track removal by hit identity and
//     direction; and the learned hit proposal's network (forward and backward, FP64).
// Full 6x6 matrices in FP64; nothing is blocked, fused or reordered.
//
// Parity unpinned (the paper prints no numbers): the prior widths, the candidate ranking key,
// the barrel half-lengths and disk extents, the efficiency definition, the cleaning and removal
// cuts, and the synthetic material map and field coefficients are readings of the text, not values
// it gives.

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <thread>
#include <unordered_map>
#include <vector>

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr double kCurv = 0.00299792458;  // GeV/(T cm)

// ------------------------------------------------------------------------------------------
// Geometry as the oracle sees it (FP32 numbers are the canonical geometry, upcast here).
// ------------------------------------------------------------------------------------------
}  // namespace

extern "C" {
struct OrSurface {
  int type;  // 0 barrel cylinder radius r_or_z, z in [lo, hi]; 1 disk at z = r_or_z, r in [lo, hi]
  float r_or_z, lo, hi, x_over_x0;
  int n_phi, n_2nd;
};
struct OrGeom {
  float bz;
  int n_surf;
  const OrSurface* surf;
  float sigma_rphi, sigma_2nd;
  float prior[5];  // sd of u, second coordinate, kappa, phi, theta at the first hit
  // Material and energy loss (Sec. 3.1: material tables indexed in r-z; energy loss): x/X0 of
  // surface s at 8 points spread evenly over its extent (z on barrels, r on disks), interpolated
  // linearly at the crossing (null: the surface's x_over_x0); scattering switch; mean ionisation
  // loss eloss GeV per unit of x/X0 crossed (0: none) for a particle of mass `mass` GeV.
  int ms_off;
  const float* material;
  float eloss, mass;
  // Parametrised solenoid field (Sec. 3.1: constant or parametrised field): Bz(r, z) = bz (1 +
  // field_z2 z^2 + field_r2 r^2), cm^-2; both zero: uniform. The radial component is neglected.
  float field_z2, field_r2;
};
constexpr int kMatNodes = 8;
// Region steering of the finder (Sec. 3.1 tracking regions): five regions in eta (0 barrel, 1/2
// +z/-z transition, 3/4 +z/-z endcap), each with its ordered list of surfaces.
struct OrSteering {
  float c_barrel, c_endcap;
  int n[5];
  int surf[5][64];
};
struct OrFindParams {
  float chi2_cut;
  int k_max;
  int max_miss;
  int brute_force;  // 1: scan every hit on the surface instead of the binned window
};
}

namespace {

using Vec6 = double[6];
using Mat6 = double[6][6];

struct State {
  double p[6];     // x, y, z, kappa, phi, theta
  double C[6][6];  // covariance
};

inline double wrap_angle(double a) {
  a = std::fmod(a, 2.0 * kPi);
  if (a > kPi) a -= 2.0 * kPi;
  if (a <= -kPi) a += 2.0 * kPi;
  return a;
}

inline double omega_of(double bz, double kappa) { return -kCurv * bz * kappa; }

inline bool field_map(const OrGeom& g) { return g.field_z2 != 0.0f || g.field_r2 != 0.0f; }

// Bz at (x, y, z).
inline double field_at(const OrGeom& g, double x, double y, double z) {
  return static_cast<double>(g.bz) *
         (1.0 + static_cast<double>(g.field_z2) * z * z + static_cast<double>(g.field_r2) * (x * x + y * y));
}

// Field at the start of a step from state p (the field that decides which surface is next).
inline double start_field(const OrGeom& g, const double* p) {
  return field_map(g) ? field_at(g, p[0], p[1], p[2]) : static_cast<double>(g.bz);
}

// ---- helix at fixed transverse path s -------------------------------------------------------
// f1 = sin(D)/D, f2 = (1-cos D)/D with D = omega*s; position change
//   dx = s*(cos(phi) f1 - sin(phi) f2),  dy = s*(sin(phi) f1 + cos(phi) f2).
inline void helix_f(double D, double& f1, double& f2) {
  if (D == 0.0) {
    f1 = 1.0;
    f2 = 0.0;
  } else {
    const double h = std::sin(0.5 * D);
    f1 = std::sin(D) / D;
    f2 = 2.0 * h * h / D;
  }
}
// derivatives df1/dD, df2/dD
inline void helix_df(double D, double& d1, double& d2) {
  if (std::fabs(D) < 1e-3) {
    const double D2 = D * D;
    d1 = -D / 3.0 + D * D2 / 30.0 - D * D2 * D2 / 840.0;
    d2 = 0.5 - D2 / 8.0 + D2 * D2 / 144.0;
  } else {
    const double h = std::sin(0.5 * D);
    d1 = (D * std::cos(D) - std::sin(D)) / (D * D);
    d2 = (D * std::sin(D) - 2.0 * h * h) / (D * D);
  }
}

void helix_at(double bz, const double* p0, double s, double* p1) {
  const double w = omega_of(bz, p0[3]);
  double f1, f2;
  helix_f(w * s, f1, f2);
  const double c = std::cos(p0[4]), sn = std::sin(p0[4]);
  p1[0] = p0[0] + s * (c * f1 - sn * f2);
  p1[1] = p0[1] + s * (sn * f1 + c * f2);
  p1[2] = p0[2] + s * std::cos(p0[5]) / std::sin(p0[5]);
  p1[3] = p0[3];
  p1[4] = wrap_angle(p0[4] + w * s);
  p1[5] = p0[5];
}

// Smallest s > 0 at which the helix reaches radius R; false when it does not.
bool path_to_cylinder(double bz, const double* p0, double R, double& s_out) {
  const double x = p0[0], y = p0[1], phi = p0[4];
  const double w = omega_of(bz, p0[3]);
  const double c = std::cos(phi), sn = std::sin(phi);
  if (std::fabs(w) < 1e-9) {  // straight line
    const double a = x * c + y * sn;
    const double disc = a * a + R * R - (x * x + y * y);
    if (disc < 0.0) return false;
    const double s = -a + std::sqrt(disc);
    if (!(s > 1e-9)) return false;
    s_out = s;
    return true;
  }
  // Circle of the helix: centre (x - sin(phi)/w, y + cos(phi)/w), radius 1/|w|.
  const double cx = x - sn / w, cy = y + c / w;
  const double rc = 1.0 / std::fabs(w);
  const double d = std::hypot(cx, cy);
  if (d == 0.0) return false;
  const double a = (R * R - rc * rc + d * d) / (2.0 * d);
  const double h2 = R * R - a * a;
  if (h2 < 0.0) return false;
  const double hh = std::sqrt(h2);
  const double ux = cx / d, uy = cy / d;
  double best = -1.0;
  for (int sgn = -1; sgn <= 1; sgn += 2) {
    const double px = a * ux - sgn * hh * uy;
    const double py = a * uy + sgn * hh * ux;
    // On the helix, (p - centre) = (sin(psi), -cos(psi)) / w with psi = phi + w*s.
    const double psi = std::atan2(w * (px - cx), -w * (py - cy));
    double dpsi = std::fmod(psi - phi, 2.0 * kPi);
    if (w > 0) {
      if (dpsi <= 0) dpsi += 2.0 * kPi;
    } else {
      if (dpsi >= 0) dpsi -= 2.0 * kPi;
    }
    const double s = dpsi / w;
    if (s > 1e-9 && (best < 0 || s < best)) best = s;
  }
  if (best < 0) return false;
  s_out = best;
  return true;
}

// Path to the plane z = Z. A track is followed for at most half a turn in the transverse plane
// (|omega s| < pi), as the generator follows particles: beyond that it would be coming back
// inward, and the disk is not reached.
bool path_to_disk(double bz, const double* p0, double Z, double& s_out) {
  const double cot = std::cos(p0[5]) / std::sin(p0[5]);
  if (cot == 0.0) return false;
  const double s = (Z - p0[2]) / cot;
  if (!(s > 1e-9)) return false;
  if (!(std::fabs(omega_of(bz, p0[3]) * s) < kPi)) return false;
  s_out = s;
  return true;
}

// Jacobian d(state at s)/d(state at 0) at fixed s.
void jacobian_fixed_s(double bz, const double* p0, double s, Mat6 J) {
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) J[i][j] = (i == j) ? 1.0 : 0.0;
  const double dwdk = -kCurv * bz;
  const double w = dwdk * p0[3];
  const double D = w * s;
  double f1, f2, d1, d2;
  helix_f(D, f1, f2);
  helix_df(D, d1, d2);
  const double c = std::cos(p0[4]), sn = std::sin(p0[4]);
  const double dx = s * (c * f1 - sn * f2), dy = s * (sn * f1 + c * f2);
  J[0][4] = -dy;
  J[1][4] = dx;
  J[0][3] = dwdk * s * s * (c * d1 - sn * d2);
  J[1][3] = dwdk * s * s * (sn * d1 + c * d2);
  const double st = std::sin(p0[5]);
  J[2][5] = -s / (st * st);
  J[4][3] = dwdk * s;
}

void matmul(const Mat6 A, const Mat6 B, Mat6 out) {
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) {
      double acc = 0.0;
      for (int k = 0; k < 6; ++k) acc += A[i][k] * B[k][j];
      out[i][j] = acc;
    }
}

void transpose(const Mat6 A, Mat6 out) {
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) out[i][j] = A[j][i];
}

double highland(double p, double x_over_x0) {
  return 0.0136 / p * std::sqrt(x_over_x0) * (1.0 + 0.038 * std::log(x_over_x0));
}

// x/X0 of surface si at second coordinate v (linear between the map's nodes, clamped at the ends).
double material_at(const OrGeom& g, int si, double v) {
  const OrSurface& S = g.surf[si];
  if (!g.material) return S.x_over_x0;
  double u = (v - S.lo) / (static_cast<double>(S.hi) - S.lo) * (kMatNodes - 1);
  u = std::min(std::max(u, 0.0), static_cast<double>(kMatNodes - 1));
  const int k = std::min(static_cast<int>(std::floor(u)), kMatNodes - 2);
  const float* nd = g.material + static_cast<size_t>(si) * kMatNodes;
  return nd[k] + (u - k) * (static_cast<double>(nd[k + 1]) - nd[k]);
}

// Propagate to surface `si`: state moves along the helix, covariance by J C J^T with J
// projected onto the surface, plus multiple-scattering noise of the material at the crossing,
// then the mean energy loss in it: |p| -> p' with E' = E - eloss x/X0 / |cos a| (direction kept),
// kappa scaled by p/p' and the kappa row and column of C by d kappa'/d kappa = (p/p')^3 E'/E (the
// loss taken as fixed; its dependence on theta and on the crossing angle is not propagated).
// With a parametrised field the step is a helix in the field at the midpoint of its chord: the path
// in the field at the start gives the chord p + (s/2) (cos phi, sin phi, cot theta) to its
// midpoint, and the path is solved again in the field there (Bz's gradient is not propagated
// into the covariance).
bool path_to_surface(const OrGeom& g, double bz, const double* p0, int si, double& s) {
  const OrSurface& S = g.surf[si];
  return (S.type == 0) ? path_to_cylinder(bz, p0, S.r_or_z, s) : path_to_disk(bz, p0, S.r_or_z, s);
}

bool step_field(const OrGeom& g, const double* p0, int si, double& bz, double& s) {
  bz = start_field(g, p0);
  if (!path_to_surface(g, bz, p0, si, s)) return false;
  if (!field_map(g)) return true;
  const double h = 0.5 * s;
  bz = field_at(g, p0[0] + h * std::cos(p0[4]), p0[1] + h * std::sin(p0[4]),
                p0[2] + h * std::cos(p0[5]) / std::sin(p0[5]));
  return path_to_surface(g, bz, p0, si, s);
}

bool propagate(const OrGeom& g, const State& in, int si, State& out, Mat6* jac_out = nullptr,
               double* s_used = nullptr) {
  const OrSurface& S = g.surf[si];
  double s, bz;
  if (!step_field(g, in.p, si, bz, s)) return false;
  helix_at(bz, in.p, s, out.p);
  Mat6 Js, J;
  jacobian_fixed_s(bz, in.p, s, Js);
  // Direction of motion along s at the crossing and the surface gradient.
  const double w = omega_of(bz, in.p[3]);
  const double t[6] = {std::cos(out.p[4]), std::sin(out.p[4]), std::cos(out.p[5]) / std::sin(out.p[5]), 0.0, w, 0.0};
  double gr[6] = {0, 0, 0, 0, 0, 0};
  if (S.type == 0) {
    gr[0] = out.p[0];
    gr[1] = out.p[1];
  } else {
    gr[2] = 1.0;
  }
  double gt = 0.0;
  for (int i = 0; i < 6; ++i) gt += gr[i] * t[i];
  if (gt == 0.0) return false;
  Mat6 P;
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) P[i][j] = (i == j ? 1.0 : 0.0) - t[i] * gr[j] / gt;
  matmul(P, Js, J);
  Mat6 JC, Jt;
  matmul(J, in.C, JC);
  transpose(J, Jt);
  matmul(JC, Jt, out.C);
  // Thin-layer multiple scattering and energy loss at the crossing.
  const double xx0 = material_at(g, si, S.type == 0 ? out.p[2] : std::hypot(out.p[0], out.p[1]));
  const bool ms = !g.ms_off && xx0 > 0.0, el = g.eloss > 0.0f && xx0 > 0.0;
  if (ms || el) {
    const double kap = out.p[3], th = out.p[5];
    const double sth = std::sin(th), cth = std::cos(th);
    double cos_a;
    if (S.type == 0) {
      const double r = std::hypot(out.p[0], out.p[1]);
      cos_a = sth * (out.p[0] * std::cos(out.p[4]) + out.p[1] * std::sin(out.p[4])) / r;
    } else {
      cos_a = cth;
    }
    const double p = 1.0 / (std::fabs(kap) * sth);
    if (ms) {
      const double t0 = highland(p, xx0 / std::fabs(cos_a));
      const double v = t0 * t0;
      const double cot = cth / sth;
      out.C[5][5] += v;
      out.C[4][4] += v / (sth * sth);
      out.C[3][5] += -kap * cot * v;
      out.C[5][3] += -kap * cot * v;
      out.C[3][3] += kap * kap * cot * cot * v;
    }
    if (el) {
      const double m = g.mass, e = std::sqrt(p * p + m * m);
      const double e1 = e - static_cast<double>(g.eloss) * xx0 / std::fabs(cos_a);
      if (!(e1 > m)) return false;  // stopped in the layer
      const double p1 = std::sqrt(e1 * e1 - m * m), ratio = p / p1;
      const double gk = ratio * ratio * ratio * e1 / e;
      out.p[3] = kap * ratio;
      for (int i = 0; i < 6; ++i) {
        out.C[3][i] *= gk;
        out.C[i][3] *= gk;
      }
    }
  }
  if (jac_out)
    for (int i = 0; i < 6; ++i)
      for (int j = 0; j < 6; ++j) (*jac_out)[i][j] = J[i][j];
  if (s_used) *s_used = s;
  return true;
}

// ---- measurement ----------------------------------------------------------------------------
struct Meas {
  double r[2];     // residual
  double H[2][6];  // measurement Jacobian
  double V[2];     // hit variances
};

void measure(const OrGeom& g, int si, const double* p, float hphi, float hsecond, Meas& m) {
  const OrSurface& S = g.surf[si];
  const double x = p[0], y = p[1];
  const double rho2 = x * x + y * y, rho = std::sqrt(rho2);
  const double phip = std::atan2(y, x);
  const double dphi = wrap_angle(static_cast<double>(hphi) - phip);
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 6; ++j) m.H[i][j] = 0.0;
  m.V[0] = static_cast<double>(g.sigma_rphi) * g.sigma_rphi;
  m.V[1] = static_cast<double>(g.sigma_2nd) * g.sigma_2nd;
  if (S.type == 0) {
    const double R = S.r_or_z;
    m.r[0] = R * dphi;
    m.r[1] = static_cast<double>(hsecond) - p[2];
    m.H[0][0] = -R * y / rho2;
    m.H[0][1] = R * x / rho2;
    m.H[1][2] = 1.0;
  } else {
    m.r[0] = rho * dphi;
    m.r[1] = static_cast<double>(hsecond) - rho;
    m.H[0][0] = -y / rho;
    m.H[0][1] = x / rho;
    m.H[1][0] = x / rho;
    m.H[1][1] = y / rho;
  }
}

// S = H C H^T + V; returns chi2 = r^T S^-1 r and fills S.
double chi2_of(const Meas& m, const Mat6 C, double Sm[2][2]) {
  double HC[2][6];
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 6; ++j) {
      double acc = 0.0;
      for (int k = 0; k < 6; ++k) acc += m.H[i][k] * C[k][j];
      HC[i][j] = acc;
    }
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) {
      double acc = 0.0;
      for (int k = 0; k < 6; ++k) acc += HC[i][k] * m.H[j][k];
      Sm[i][j] = acc;
    }
  Sm[0][0] += m.V[0];
  Sm[1][1] += m.V[1];
  const double det = Sm[0][0] * Sm[1][1] - Sm[0][1] * Sm[1][0];
  if (!(det > 0.0) || !(Sm[0][0] > 0.0)) return HUGE_VAL;  // not a covariance: no hit is compatible
  const double i00 = Sm[1][1] / det, i01 = -Sm[0][1] / det, i11 = Sm[0][0] / det;
  return m.r[0] * (i00 * m.r[0] + i01 * m.r[1]) + m.r[1] * (i01 * m.r[0] + i11 * m.r[1]);
}

// Kalman update: K = C H^T S^-1, p += K r, C -= K H C. Returns the predicted chi2.
double kf_update(const Meas& m, State& st) {
  double Sm[2][2];
  const double chi2 = chi2_of(m, st.C, Sm);
  const double det = Sm[0][0] * Sm[1][1] - Sm[0][1] * Sm[1][0];
  const double Si[2][2] = {{Sm[1][1] / det, -Sm[0][1] / det}, {-Sm[1][0] / det, Sm[0][0] / det}};
  double CHt[6][2];
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 2; ++j) {
      double acc = 0.0;
      for (int k = 0; k < 6; ++k) acc += st.C[i][k] * m.H[j][k];
      CHt[i][j] = acc;
    }
  double K[6][2];
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 2; ++j) K[i][j] = CHt[i][0] * Si[0][j] + CHt[i][1] * Si[1][j];
  for (int i = 0; i < 6; ++i) st.p[i] += K[i][0] * m.r[0] + K[i][1] * m.r[1];
  st.p[4] = wrap_angle(st.p[4]);
  double HC[2][6];
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 6; ++j) {
      double acc = 0.0;
      for (int k = 0; k < 6; ++k) acc += m.H[i][k] * st.C[k][j];
      HC[i][j] = acc;
    }
  Mat6 Cn;
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) Cn[i][j] = st.C[i][j] - (K[i][0] * HC[0][j] + K[i][1] * HC[1][j]);
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) st.C[i][j] = 0.5 * (Cn[i][j] + Cn[j][i]);
  return chi2;
}

// ---- hits -------------------------------------------------------------------------------------
void hit_position(const OrGeom& g, int si, float hphi, float hsecond, double* xyz) {
  const OrSurface& S = g.surf[si];
  const double ph = hphi;
  if (S.type == 0) {
    xyz[0] = S.r_or_z * std::cos(ph);
    xyz[1] = S.r_or_z * std::sin(ph);
    xyz[2] = hsecond;
  } else {
    xyz[0] = static_cast<double>(hsecond) * std::cos(ph);
    xyz[1] = static_cast<double>(hsecond) * std::sin(ph);
    xyz[2] = S.r_or_z;
  }
}

// Seed state at hit 1 from the circle through three hits (transverse plane) and the
// straight line in (arc length, z); prior covariance on the tangent space of hit 1's surface.
bool seed_state(const OrGeom& g, const float* hits, const int* hsurf, const int* ids, State& st) {
  double P[3][3];
  for (int i = 0; i < 3; ++i) hit_position(g, hsurf[ids[i]], hits[2 * ids[i]], hits[2 * ids[i] + 1], P[i]);
  const double x1 = P[0][0], y1 = P[0][1], x2 = P[1][0], y2 = P[1][1], x3 = P[2][0], y3 = P[2][1];
  const double D = 2.0 * (x1 * (y2 - y3) + x2 * (y3 - y1) + x3 * (y1 - y2));
  const double cross = (x2 - x1) * (y3 - y2) - (y2 - y1) * (x3 - x2);
  double w = 0.0, phi, s13;
  const double scale = std::max({std::fabs(x1), std::fabs(y1), std::fabs(x3), std::fabs(y3), 1.0});
  if (std::fabs(D) > 1e-12 * scale * scale) {
    const double a1 = x1 * x1 + y1 * y1, a2 = x2 * x2 + y2 * y2, a3 = x3 * x3 + y3 * y3;
    const double cx = (a1 * (y2 - y3) + a2 * (y3 - y1) + a3 * (y1 - y2)) / D;
    const double cy = (a1 * (x3 - x2) + a2 * (x1 - x3) + a3 * (x2 - x1)) / D;
    const double rc = std::hypot(x1 - cx, y1 - cy);
    w = (cross > 0 ? 1.0 : -1.0) / rc;
    // Direction of motion at hit 1: (cos phi, sin phi) = w * (-(y1 - cy), x1 - cx).
    phi = std::atan2(w * (x1 - cx), -w * (y1 - cy));
    const double ax = x1 - cx, ay = y1 - cy, bx = x3 - cx, by = y3 - cy;
    const double swept = std::atan2(ax * by - ay * bx, ax * bx + ay * by);
    s13 = swept / w;
    if (s13 <= 0) s13 += 2.0 * kPi / std::fabs(w);
  } else {
    phi = std::atan2(y3 - y1, x3 - x1);
    s13 = std::hypot(x3 - x1, y3 - y1);
  }
  if (!(s13 > 0)) return false;
  const double theta = std::atan2(s13, P[2][2] - P[0][2]);
  st.p[0] = x1;
  st.p[1] = y1;
  st.p[2] = P[0][2];
  st.p[3] = -w / (kCurv * start_field(g, P[0]));  // the field at hit 1
  st.p[4] = phi;
  st.p[5] = theta;
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) st.C[i][j] = 0.0;
  const OrSurface& S = g.surf[hsurf[ids[0]]];
  const double pp = std::atan2(y1, x1);
  const double eu[3] = {-std::sin(pp), std::cos(pp), 0.0};
  const double su = g.prior[0], s2 = g.prior[1];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) st.C[i][j] += su * su * eu[i] * eu[j];
  if (S.type == 0) {
    st.C[2][2] += s2 * s2;
  } else {
    const double er[3] = {std::cos(pp), std::sin(pp), 0.0};
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) st.C[i][j] += s2 * s2 * er[i] * er[j];
  }
  st.C[3][3] = static_cast<double>(g.prior[2]) * g.prior[2];
  st.C[4][4] = static_cast<double>(g.prior[3]) * g.prior[3];
  st.C[5][5] = static_cast<double>(g.prior[4]) * g.prior[4];
  return true;
}

void pack_cov(const Mat6 C, float* out21, double* out21d) {
  int k = 0;
  for (int i = 0; i < 6; ++i)
    for (int j = i; j < 6; ++j, ++k) {
      if (out21) out21[k] = static_cast<float>(C[i][j]);
      if (out21d) out21d[k] = C[i][j];
    }
}

template <class F>
void parallel_for(long long n, int n_threads, F&& f) {
  int nt = n_threads > 0 ? n_threads : static_cast<int>(std::thread::hardware_concurrency());
  nt = static_cast<int>(std::max<long long>(1, std::min<long long>(nt, n)));
  if (nt <= 1) {
    for (long long i = 0; i < n; ++i) f(i);
    return;
  }
  std::atomic<long long> next(0);
  std::vector<std::thread> pool;
  for (int t = 0; t < nt; ++t)
    pool.emplace_back([&]() {
      for (;;) {
        const long long i0 = next.fetch_add(64);
        if (i0 >= n) break;
        const long long i1 = std::min(n, i0 + 64);
        for (long long i = i0; i < i1; ++i) f(i);
      }
    });
  for (auto& th : pool) th.join();
}

// ---- hit binning: FP32, every operation rounded to nearest, no contraction -----------------
// phi-bin = clamp(floor((phi + pi_f) * sphi), 0, n_phi - 1) with sphi = (float)(n_phi / 2pi);
// 2nd-bin = clamp(floor((v - lo_f) * s2), 0, n_2nd - 1) with s2 = (float)(n_2nd / (hi_f - lo_f)).
// The build flags forbid FMA contraction so each float operation rounds on its own.
// Phi sub-bins (kSub per phi bin): fine = clamp(floor((phi + pi_f) * sphi_sub), 0, n_phi*kSub - 1)
// with sphi_sub = (float)(n_phi * kSub / 2pi), sub = clamp(fine - phi_bin * kSub, 0, kSub - 1).
constexpr int kSub = 8;

struct BinRule {
  float pi_f, sphi, sphi_sub, lo, s2;
  int n_phi, n_2nd;
  explicit BinRule(const OrSurface& S) {
    pi_f = static_cast<float>(kPi);
    sphi = static_cast<float>(static_cast<double>(S.n_phi) / (2.0 * kPi));
    sphi_sub = static_cast<float>(static_cast<double>(S.n_phi) * kSub / (2.0 * kPi));
    lo = S.lo;
    s2 = static_cast<float>(static_cast<double>(S.n_2nd) / (static_cast<double>(S.hi) - static_cast<double>(S.lo)));
    n_phi = S.n_phi;
    n_2nd = S.n_2nd;
  }
  int phi_bin(float phi) const {
    const float a = phi + pi_f;
    const float b = a * sphi;
    const float f = std::floor(b);
    const int k = (f >= 0.0f) ? (f > 1e8f ? 100000000 : static_cast<int>(f)) : -1;  // NaN -> -1
    return std::min(std::max(k, 0), n_phi - 1);
  }
  int fine_bin(float phi) const {
    const float a = phi + pi_f;
    const float b = a * sphi_sub;
    const float f = std::floor(b);
    const int k = (f >= 0.0f) ? (f > 1e8f ? 100000000 : static_cast<int>(f)) : -1;  // NaN -> -1
    return std::min(std::max(k, 0), n_phi * kSub - 1);
  }
  int sub_bin(float phi) const { return std::min(std::max(fine_bin(phi) - phi_bin(phi) * kSub, 0), kSub - 1); }
  int second_bin(float v) const {
    const float a = v - lo;
    const float b = a * s2;
    const float f = std::floor(b);
    const int k = (f >= 0.0f) ? (f > 1e8f ? 100000000 : static_cast<int>(f)) : -1;  // NaN -> -1
    return std::min(std::max(k, 0), n_2nd - 1);
  }
};

int max_bins(const OrGeom& g) {
  int m = 0;
  for (int s = 0; s < g.n_surf; ++s) m = std::max(m, g.surf[s].n_phi * g.surf[s].n_2nd);
  return m;
}

struct Index {
  int nb = 0;                   // bins per slab (max over surfaces)
  std::vector<long long> off;   // [(e*n_surf+s)*(nb+1) + b]: global position of bin b's first hit
  std::vector<float> sorted;    // [n_hits][2]
  std::vector<int> ids;         // [n_hits] original hit id
  std::vector<unsigned short> sub;  // [(e*n_surf+s)*nb + b][kSub]: hits of bin b with sub-bin <= j
};

// Counting sort per (event, surface) slab by (bin, phi sub-bin), bin = phi_bin * n_2nd +
// second_bin; within a (bin, sub-bin), ascending hit id. Slabs keep their position in the hit
// array.
void build_index(const OrGeom& g, const float* hits, const long long* slab_off, int n_events, Index& ix) {
  ix.nb = max_bins(g);
  const long long n_slabs = static_cast<long long>(n_events) * g.n_surf;
  const long long n_hits = slab_off[n_slabs];
  ix.off.assign(n_slabs * (ix.nb + 1), 0);
  ix.sorted.assign(2 * n_hits, 0.0f);
  ix.ids.assign(n_hits, 0);
  ix.sub.assign(static_cast<size_t>(n_slabs) * ix.nb * kSub, 0);
  for (long long sl = 0; sl < n_slabs; ++sl) {
    const int si = static_cast<int>(sl % g.n_surf);
    const OrSurface& S = g.surf[si];
    const BinRule br(S);
    const long long h0 = slab_off[sl], h1 = slab_off[sl + 1];
    // key = bin * kSub + sub-bin: a counting sort on it orders bins, and sub-bins within a bin
    std::vector<long long> count(static_cast<size_t>(ix.nb) * kSub + 1, 0);
    std::vector<int> key(h1 - h0);
    for (long long h = h0; h < h1; ++h) {
      const int b = br.phi_bin(hits[2 * h]) * S.n_2nd + br.second_bin(hits[2 * h + 1]);
      key[h - h0] = b * kSub + br.sub_bin(hits[2 * h]);
      count[key[h - h0] + 1]++;
    }
    std::vector<long long> start(static_cast<size_t>(ix.nb) * kSub + 1);
    start[0] = h0;
    for (size_t k = 0; k + 1 < start.size(); ++k) start[k + 1] = start[k] + count[k + 1];
    long long* o = &ix.off[sl * (ix.nb + 1)];
    for (int b = 0; b <= ix.nb; ++b) o[b] = start[static_cast<size_t>(b) * kSub];
    unsigned short* sb = &ix.sub[static_cast<size_t>(sl) * ix.nb * kSub];
    for (int b = 0; b < ix.nb; ++b)
      for (int j = 0; j < kSub; ++j)
        sb[b * kSub + j] = static_cast<unsigned short>(start[static_cast<size_t>(b) * kSub + j + 1] - o[b]);
    std::vector<long long> cursor(start.begin(), start.end() - 1);
    for (long long h = h0; h < h1; ++h) {  // ascending id keeps equal keys in id order
      const long long pos = cursor[key[h - h0]]++;
      ix.sorted[2 * pos] = hits[2 * h];
      ix.sorted[2 * pos + 1] = hits[2 * h + 1];
      ix.ids[pos] = static_cast<int>(h);
    }
  }
}

// ---- finding ----------------------------------------------------------------------------------
struct Cand {
  State st;
  int n_hits = 0, n_miss = 0;
  double chi2 = 0.0;
  int surf = -1;
  int pos = -1;  // position of surf in the steering list of the seed's region
  bool stopped = false;
  std::vector<int> hits;  // hit id per step, -1 = miss
};

// Next surface outward from a candidate: the next barrel layer beyond its radius (accepted if
// the crossing lies within the layer's z extent) and the next disk beyond |z| in the direction
// of motion (accepted if the crossing radius is within the disk); the nearer accepted one wins.
int next_surface(const OrGeom& g, const State& st, double* s_next) {
  const double rho = std::hypot(st.p[0], st.p[1]);
  const double z = st.p[2];
  const double cot = std::cos(st.p[5]) / std::sin(st.p[5]);
  int best = -1;
  double best_s = 0.0;
  int nb = -1;
  for (int s = 0; s < g.n_surf; ++s) {
    const OrSurface& S = g.surf[s];
    if (S.type == 0 && S.r_or_z > rho + 0.01 && (nb < 0 || S.r_or_z < g.surf[nb].r_or_z)) nb = s;
  }
  const double bz = start_field(g, st.p);
  if (nb >= 0) {
    double s;
    if (path_to_cylinder(bz, st.p, g.surf[nb].r_or_z, s)) {
      double q[6];
      helix_at(bz, st.p, s, q);
      if (q[2] >= g.surf[nb].lo && q[2] <= g.surf[nb].hi) {
        best = nb;
        best_s = s;
      }
    }
  }
  int nd = -1;
  for (int s = 0; s < g.n_surf; ++s) {
    const OrSurface& S = g.surf[s];
    if (S.type != 1) continue;
    if ((cot > 0 && S.r_or_z > z + 0.01) || (cot < 0 && S.r_or_z < z - 0.01)) {
      if (nd < 0 || std::fabs(S.r_or_z) < std::fabs(g.surf[nd].r_or_z)) nd = s;
    }
  }
  if (nd >= 0) {
    double s;
    if (path_to_disk(bz, st.p, g.surf[nd].r_or_z, s)) {
      double q[6];
      helix_at(bz, st.p, s, q);
      const double r = std::hypot(q[0], q[1]);
      if (r >= g.surf[nd].lo && r <= g.surf[nd].hi && (best < 0 || s < best_s)) {
        best = nd;
        best_s = s;
      }
    }
  }
  if (s_next) *s_next = best_s;
  return best;
}

struct Found {
  int hit;
  double chi2;
};

// ---- learned hit proposal: MLP 14 -> 64 -> 64 -> 1 (ReLU), FP64 -------------------------------
// Weight layout (shared with the CUDA path as data only): W1[64][14], b1[64], W2[64][64], b2[64],
// W3[64], b3; features are standardised by (x - mean) / sd before the first layer.
constexpr int kIn = 14, kHid = 64;
constexpr int kW1 = 0, kB1 = kW1 + kHid * kIn, kW2 = kB1 + kHid, kB2 = kW2 + kHid * kHid, kW3 = kB2 + kHid,
              kB3 = kW3 + kHid, kNParam = kB3 + 1;

struct Mlp {
  const double* w = nullptr;   // kNParam weights
  const double* mean = nullptr;
  const double* sd = nullptr;
  int top_n = 0;               // 0: plain finding
  double margin = 0.0;         // > 0: score margin rule (below)
  bool window = false;         // rank every hit of the window before the chi2 cut (below)
};

double mlp_forward(const double* w, const double* xs, double* h1 = nullptr, double* h2 = nullptr) {
  double a1[kHid], a2[kHid];
  for (int j = 0; j < kHid; ++j) {
    double z = w[kB1 + j];
    for (int i = 0; i < kIn; ++i) z += w[kW1 + j * kIn + i] * xs[i];
    a1[j] = z > 0.0 ? z : 0.0;
  }
  for (int j = 0; j < kHid; ++j) {
    double z = w[kB2 + j];
    for (int i = 0; i < kHid; ++i) z += w[kW2 + j * kHid + i] * a1[i];
    a2[j] = z > 0.0 ? z : 0.0;
  }
  double out = w[kB3];
  for (int j = 0; j < kHid; ++j) out += w[kW3 + j] * a2[j];
  if (h1) std::memcpy(h1, a1, sizeof(a1));
  if (h2) std::memcpy(h2, a2, sizeof(a2));
  return out;
}

// Binary cross-entropy with logits of one sample; adds its gradient (scaled by `scale`) to g.
double mlp_loss_grad(const double* w, const double* xs, double y, double scale, double* g) {
  double h1[kHid], h2[kHid];
  const double z = mlp_forward(w, xs, h1, h2);
  const double loss = std::max(z, 0.0) - z * y + std::log1p(std::exp(-std::fabs(z)));
  const double dz = (1.0 / (1.0 + std::exp(-z)) - y) * scale;
  g[kB3] += dz;
  double d2[kHid];
  for (int j = 0; j < kHid; ++j) {
    g[kW3 + j] += dz * h2[j];
    d2[j] = h2[j] > 0.0 ? dz * w[kW3 + j] : 0.0;
  }
  double d1[kHid];
  for (int i = 0; i < kHid; ++i) d1[i] = 0.0;
  for (int j = 0; j < kHid; ++j) {
    g[kB2 + j] += d2[j];
    for (int i = 0; i < kHid; ++i) {
      g[kW2 + j * kHid + i] += d2[j] * h1[i];
      d1[i] += d2[j] * w[kW2 + j * kHid + i];
    }
  }
  for (int j = 0; j < kHid; ++j) {
    const double dj = h1[j] > 0.0 ? d1[j] : 0.0;
    g[kB1 + j] += dj;
    for (int i = 0; i < kIn; ++i) g[kW1 + j * kIn + i] += dj * xs[i];
  }
  return loss;
}

// Features of a (predicted candidate, hit) pair: the predicted state, log of the covariance
// diagonal, and the two residuals over the square roots of the innovation variances.
void pair_features(const OrGeom& g, int si, const State& pred, float hphi, float h2, double* f) {
  Meas m;
  measure(g, si, pred.p, hphi, h2, m);
  double Sm[2][2];
  chi2_of(m, pred.C, Sm);
  for (int i = 0; i < 6; ++i) f[i] = pred.p[i];
  for (int i = 0; i < 6; ++i) f[6 + i] = std::log(pred.C[i][i] + 1e-12);
  f[12] = m.r[0] / std::sqrt(Sm[0][0]);
  f[13] = m.r[1] / std::sqrt(Sm[1][1]);
}

double mlp_score(const Mlp& mlp, const double* f) {
  double xs[kIn];
  for (int i = 0; i < kIn; ++i) xs[i] = (f[i] - mlp.mean[i]) / mlp.sd[i];
  return mlp_forward(mlp.w, xs);
}

struct PairSink {
  const int* hit_sim = nullptr;
  int seed_track = -1;
  std::vector<float> features;  // [n][14]
  std::vector<float> labels;
};

struct Ctx {
  const OrGeom* g;
  const float* hits;
  const int* hsurf;
  const long long* slab_off;
  const Index* ix;
  OrFindParams prm;
  Mlp mlp;
  const OrSteering* steer = nullptr;  // region steering, or null for the geometric rule
  long long n_hits = 0;  // hits of the batch and events: a seed outside them fails
  int n_events = 0;
};

// Whether the helix from st reaches surface s within its extent (the acceptance used by the
// geometric rule: barrel z extent; disk r extent, the disk path rule included).
bool reaches(const OrGeom& g, const State& st, int s) {
  const OrSurface& S = g.surf[s];
  double len, q[6];
  const double bz = start_field(g, st.p);
  if (S.type == 0) {
    if (!path_to_cylinder(bz, st.p, S.r_or_z, len)) return false;
    helix_at(bz, st.p, len, q);
    return q[2] >= S.lo && q[2] <= S.hi;
  }
  if (!path_to_disk(bz, st.p, S.r_or_z, len)) return false;
  helix_at(bz, st.p, len, q);
  const double r = std::hypot(q[0], q[1]);
  return r >= S.lo && r <= S.hi;
}

// Region of a seed from its third hit (phi, v) on surface s3: (z, rho) = (v, R) on a barrel and
// (Z, v) on a disk; barrel if |z| <= c_barrel * rho, transition if |z| <= c_endcap * rho, else
// endcap, +z side for z > 0. The products are FP32 (no contraction in this build), as the
// steering defines them.
int seed_region(const OrGeom& g, const OrSteering& sg, int s3, float v) {
  const OrSurface& S = g.surf[s3];
  const float z = S.type == 0 ? v : S.r_or_z;
  const float rho = S.type == 0 ? S.r_or_z : v;
  const float az = std::fabs(z);
  const float lb = sg.c_barrel * rho;
  if (az <= lb) return 0;
  const float le = sg.c_endcap * rho;
  return (az <= le ? 1 : 3) + (z > 0.0f ? 0 : 1);
}

// Next surface of a steered candidate: the first surface of its region's list after position
// pos that it reaches; -1 at the end of the list.
int next_steered(const OrGeom& g, const OrSteering& sg, int region, int pos, const State& st, int* newpos) {
  for (int q = pos + 1; q < sg.n[region]; ++q) {
    if (reaches(g, st, sg.surf[region][q])) {
      *newpos = q;
      return sg.surf[region][q];
    }
  }
  return -1;
}

// All hits of surface si in event ev whose chi2 against the predicted state is below the cut.
// Binned: the window is the bounding box of the chi2 ellipse, padded, turned into bin ranges by
// the same FP32 rule as the index; brute force: every hit of the surface. box (optional): the hits
// inside the bounding box itself, |r_i| <= sqrt(cut S_ii) for both residuals, with their chi2 (a
// superset of out).
void search_hits(const Ctx& cx, int ev, int si, const State& pred, std::vector<Found>& out,
                 long long* scanned = nullptr, long long* window_hits = nullptr, std::vector<Found>* box = nullptr) {
  out.clear();
  if (box) box->clear();
  const OrGeom& g = *cx.g;
  const OrSurface& S = g.surf[si];
  const long long sl = static_cast<long long>(ev) * g.n_surf + si;
  const double cut = cx.prm.chi2_cut;
  auto try_hit = [&](float hphi, float h2, int id) {
    Meas m;
    measure(g, si, pred.p, hphi, h2, m);
    double Sm[2][2];
    const double c2 = chi2_of(m, pred.C, Sm);
    if (scanned) ++*scanned;
    if (c2 < cut) out.push_back({id, c2});
    if (box && std::fabs(m.r[0]) <= std::sqrt(cut * Sm[0][0]) && std::fabs(m.r[1]) <= std::sqrt(cut * Sm[1][1]))
      box->push_back({id, c2});
  };
  if (cx.prm.brute_force) {
    for (long long h = cx.slab_off[sl]; h < cx.slab_off[sl + 1]; ++h) try_hit(cx.hits[2 * h], cx.hits[2 * h + 1], static_cast<int>(h));
    return;
  }
  // Window half-widths from the diagonal of S.
  Meas m0;
  measure(g, si, pred.p, 0.0f, 0.0f, m0);
  double Sm[2][2];
  chi2_of(m0, pred.C, Sm);
  const double x = pred.p[0], y = pred.p[1];
  const double rho = std::hypot(x, y);
  const double rref = (S.type == 0) ? static_cast<double>(S.r_or_z) : rho;
  double dphi = std::sqrt(cut * Sm[0][0]) / rref;
  dphi = dphi * (1.0 + 1e-4) + 1e-5;
  double d2 = std::sqrt(cut * Sm[1][1]);
  d2 = d2 * (1.0 + 1e-4) + 1e-4;
  const double phip = std::atan2(y, x);
  const double c2 = (S.type == 0) ? pred.p[2] : rho;
  const BinRule br(S);
  int pb0, npb;
  if (!(dphi < kPi * (1.0 - 2.0 / S.n_phi))) {
    pb0 = 0;
    npb = S.n_phi;
  } else {
    pb0 = br.phi_bin(static_cast<float>(wrap_angle(phip - dphi)));
    const int pb1 = br.phi_bin(static_cast<float>(wrap_angle(phip + dphi)));
    npb = ((pb1 - pb0) % S.n_phi + S.n_phi) % S.n_phi + 1;
  }
  const int zb0 = br.second_bin(static_cast<float>(std::max(c2 - d2, -1e30)));
  const int zb1 = br.second_bin(static_cast<float>(std::min(c2 + d2, 1e30)));
  const long long* o = &cx.ix->off[sl * (cx.ix->nb + 1)];
  for (int k = 0; k < npb; ++k) {
    const int pb = (pb0 + k) % S.n_phi;
    const long long a = o[pb * S.n_2nd + zb0], b = o[pb * S.n_2nd + zb1 + 1];
    for (long long q = a; q < b; ++q) try_hit(cx.ix->sorted[2 * q], cx.ix->sorted[2 * q + 1], cx.ix->ids[q]);
  }
  if (window_hits) {
    // Hits of the window limited to the phi sub-bins its phi range touches in its first and last
    // phi bins (a count only: the search above scans whole bins).
    int flo = 0, fhi = S.n_phi * kSub - 1;
    if (npb < S.n_phi) {
      flo = br.fine_bin(static_cast<float>(wrap_angle(phip - dphi)));
      fhi = br.fine_bin(static_cast<float>(wrap_angle(phip + dphi)));
    }
    const unsigned short* sb = &cx.ix->sub[static_cast<size_t>(sl) * cx.ix->nb * kSub];
    for (int k = 0; k < npb; ++k) {
      const int pb = (pb0 + k) % S.n_phi;
      const int slo = k == 0 ? std::min(std::max(flo - pb * kSub, 0), kSub - 1) : 0;
      const int shi = k == npb - 1 ? std::min(std::max(fhi - pb * kSub, 0), kSub - 1) : kSub - 1;
      for (int zb = zb0; zb <= zb1; ++zb) {
        const int b = pb * S.n_2nd + zb;
        *window_hits += sb[b * kSub + shi] - (slo > 0 ? sb[b * kSub + slo - 1] : 0);
      }
    }
  }
}

struct Child {
  int parent;
  int hit;       // -1: miss child or carried candidate
  int kind;      // 0 hit child, 1 miss child, 2 carried
  int n_hits;
  double chi2;   // total
  double chi2_hit;
};

bool child_less(const Child& a, const Child& b) {
  if (a.n_hits != b.n_hits) return a.n_hits > b.n_hits;
  if (a.chi2 != b.chi2) return a.chi2 < b.chi2;
  if (a.parent != b.parent) return a.parent < b.parent;
  if (a.kind != b.kind) return a.kind < b.kind;
  return a.hit < b.hit;
}

struct Counters {
  long long n_prop = 0, n_chi2 = 0, n_upd = 0, n_scan = 0, n_win = 0, n_mlp = 0;
};

// Beam search for one seed. Returns false if the seed could not be formed.
bool find_one(const Ctx& cx, const int* seed_ids, int ev, int lmax, Cand& best, Counters& cnt,
              PairSink* sink = nullptr) {
  const OrGeom& g = *cx.g;
  if (ev < 0 || ev >= cx.n_events) return false;
  for (int k = 0; k < 3; ++k) {
    const int id = seed_ids[k];
    if (id < 0 || id >= cx.n_hits || cx.hsurf[id] < 0 || cx.hsurf[id] >= g.n_surf) return false;
  }
  Cand c0;
  if (!seed_state(g, cx.hits, cx.hsurf, seed_ids, c0.st)) return false;
  // Fit the seed hits: update with hit 1, then propagate + update through hits 2, 3.
  for (int k = 0; k < 3; ++k) {
    const int id = seed_ids[k];
    const int si = cx.hsurf[id];
    if (k > 0) {
      State pr;
      if (!propagate(g, c0.st, si, pr)) return false;
      c0.st = pr;
      cnt.n_prop++;
    }
    Meas m;
    measure(g, si, c0.st.p, cx.hits[2 * id], cx.hits[2 * id + 1], m);
    c0.chi2 += kf_update(m, c0.st);
    cnt.n_chi2++;
    cnt.n_upd++;
    c0.hits.push_back(id);
    c0.surf = si;
  }
  c0.n_hits = 3;
  int region = 0;
  if (cx.steer) {
    const int id3 = seed_ids[2];
    region = seed_region(g, *cx.steer, c0.surf, cx.hits[2 * id3 + 1]);
    for (int q = 0; q < cx.steer->n[region]; ++q)
      if (cx.steer->surf[region][q] == c0.surf) c0.pos = q;
  }
  std::vector<Cand> cands{c0};
  std::vector<Found> found, box;
  std::vector<Child> pool;
  std::vector<State> pred;
  for (int step = 3; step < lmax; ++step) {
    bool any_active = false;
    for (const Cand& c : cands) any_active |= !c.stopped;
    if (!any_active) break;
    pool.clear();
    pred.assign(cands.size(), State());
    std::vector<int> pred_surf(cands.size(), -1), pred_pos(cands.size(), -1);
    for (int ci = 0; ci < static_cast<int>(cands.size()); ++ci) {
      const Cand& c = cands[ci];
      if (c.stopped) {
        pool.push_back({ci, -1, 2, c.n_hits, c.chi2, 0.0});
        continue;
      }
      int np = -1;
      const int si = cx.steer ? next_steered(g, *cx.steer, region, c.pos, c.st, &np) : next_surface(g, c.st, nullptr);
      if (si < 0 || !propagate(g, c.st, si, pred[ci])) {
        pool.push_back({ci, -1, 2, c.n_hits, c.chi2, 0.0});
        continue;
      }
      cnt.n_prop++;
      pred_surf[ci] = si;
      pred_pos[ci] = np;
      search_hits(cx, ev, si, pred[ci], found, &cnt.n_scan, &cnt.n_win, cx.mlp.top_n > 0 && cx.mlp.window ? &box : nullptr);
      cnt.n_chi2 += static_cast<long long>(found.size());
      if (sink) {  // training pairs: every passing (candidate, hit) pair, labelled by truth
        double f[kIn];
        for (const Found& fd : found) {
          pair_features(g, si, pred[ci], cx.hits[2 * fd.hit], cx.hits[2 * fd.hit + 1], f);
          for (int i = 0; i < kIn; ++i) sink->features.push_back(static_cast<float>(f[i]));
          sink->labels.push_back(sink->hit_sim[fd.hit] == sink->seed_track ? 1.f : 0.f);
        }
      }
      const bool margin_rule = cx.mlp.margin > 0.0;
      if (cx.mlp.top_n > 0 && cx.mlp.window) {
        // Learned proposal ranking the window before the chi2 cut: when the window (the bounding
        // box of the chi2 ellipse) holds more than top_n hits (with a score margin, two or more),
        // only its top_n by MLP score (ties: lower hit id) go on to the cut, with a margin only
        // those of them that score within the margin of the best; otherwise every passing hit
        // makes a child.
        if (static_cast<int>(box.size()) > (margin_rule ? 1 : cx.mlp.top_n)) {
          std::vector<std::pair<double, int>> sc;
          double f[kIn];
          for (const Found& fd : box) {
            pair_features(g, si, pred[ci], cx.hits[2 * fd.hit], cx.hits[2 * fd.hit + 1], f);
            sc.push_back({mlp_score(cx.mlp, f), fd.hit});
            cnt.n_mlp++;
          }
          std::sort(sc.begin(), sc.end(), [](const std::pair<double, int>& a, const std::pair<double, int>& b) {
            return a.first != b.first ? a.first > b.first : a.second < b.second;
          });
          std::vector<Found> kept;
          for (int k = 0; k < cx.mlp.top_n && k < static_cast<int>(sc.size()); ++k) {
            if (margin_rule && k > 0 && sc[k].first < sc[0].first - cx.mlp.margin) break;
            for (const Found& fd : box)
              if (fd.hit == sc[k].second && fd.chi2 < cx.prm.chi2_cut) kept.push_back(fd);
          }
          found.swap(kept);
        }
      } else if (cx.mlp.top_n > 0 && static_cast<int>(found.size()) > (margin_rule ? 1 : cx.mlp.top_n)) {
        // Learned proposal: rank the passing hits by MLP score (ties: lower hit id) and keep the
        // top_n; with a score margin, only those of them that score within the margin of the best
        // (the best is always kept), so a window whose best hit stands out keeps one child.
        std::vector<std::pair<double, int>> sc;
        double f[kIn];
        for (const Found& fd : found) {
          pair_features(g, si, pred[ci], cx.hits[2 * fd.hit], cx.hits[2 * fd.hit + 1], f);
          sc.push_back({mlp_score(cx.mlp, f), fd.hit});
          cnt.n_mlp++;
        }
        std::sort(sc.begin(), sc.end(), [](const std::pair<double, int>& a, const std::pair<double, int>& b) {
          return a.first != b.first ? a.first > b.first : a.second < b.second;
        });
        std::vector<Found> kept;
        for (int k = 0; k < cx.mlp.top_n && k < static_cast<int>(sc.size()); ++k) {
          if (margin_rule && k > 0 && sc[k].first < sc[0].first - cx.mlp.margin) break;
          for (const Found& fd : found)
            if (fd.hit == sc[k].second) kept.push_back(fd);
        }
        found.swap(kept);
      }
      if (!found.empty()) {
        for (const Found& f : found) pool.push_back({ci, f.hit, 0, c.n_hits + 1, c.chi2 + f.chi2, f.chi2});
      } else if (c.n_miss < cx.prm.max_miss) {
        pool.push_back({ci, -1, 1, c.n_hits, c.chi2, 0.0});
      } else {
        pool.push_back({ci, -1, 2, c.n_hits, c.chi2, 0.0});
      }
    }
    std::sort(pool.begin(), pool.end(), child_less);
    if (static_cast<int>(pool.size()) > cx.prm.k_max) pool.resize(cx.prm.k_max);
    std::vector<Cand> next;
    next.reserve(pool.size());
    for (const Child& ch : pool) {
      const Cand& par = cands[ch.parent];
      Cand n = par;
      if (ch.kind == 2) {
        n.stopped = true;
      } else {
        n.st = pred[ch.parent];
        n.surf = pred_surf[ch.parent];
        n.pos = pred_pos[ch.parent];
        if (ch.kind == 0) {
          Meas m;
          measure(g, n.surf, n.st.p, cx.hits[2 * ch.hit], cx.hits[2 * ch.hit + 1], m);
          kf_update(m, n.st);
          cnt.n_upd++;
          n.n_hits += 1;
          n.chi2 = ch.chi2;
          n.hits.push_back(ch.hit);
        } else {
          n.n_miss += 1;
          n.hits.push_back(-1);
        }
      }
      next.push_back(std::move(n));
    }
    cands.swap(next);
  }
  best = cands.front();
  return true;
}

}  // namespace

// ================================================================================================
extern "C" {

int or_version() { return 1; }

// Propagate one state (p[6], full C[36] row-major) to surface `surf`. Outputs the new state,
// covariance, the projected Jacobian J[36] and the path s. Returns 0, or -1 if not reached.
int or_propagate(const OrGeom* g, const double* p, const double* C, int surf, double* p_out, double* C_out,
                 double* J_out, double* s_out) {
  State in, out;
  for (int i = 0; i < 6; ++i) in.p[i] = p[i];
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) in.C[i][j] = C ? C[6 * i + j] : 0.0;
  Mat6 J;
  double s;
  if (!propagate(*g, in, surf, out, &J, &s)) return -1;
  for (int i = 0; i < 6; ++i) p_out[i] = out.p[i];
  if (C_out)
    for (int i = 0; i < 6; ++i)
      for (int j = 0; j < 6; ++j) C_out[6 * i + j] = out.C[i][j];
  if (J_out)
    for (int i = 0; i < 6; ++i)
      for (int j = 0; j < 6; ++j) J_out[6 * i + j] = J[i][j];
  if (s_out) *s_out = s;
  return 0;
}

// Position of the helix at fixed transverse path s (no surface), for finite-difference tests.
void or_helix_at(const OrGeom* g, const double* p, double s, double* p_out) {
  helix_at(start_field(*g, p), p, s, p_out);
}

// Seed state + prior from three hit ids.
int or_seed(const OrGeom* g, const float* hits, const int* hsurf, const int* ids, double* p_out, double* C_out) {
  State st;
  if (!seed_state(*g, hits, hsurf, ids, st)) return -1;
  for (int i = 0; i < 6; ++i) p_out[i] = st.p[i];
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) C_out[6 * i + j] = st.C[i][j];
  return 0;
}

// Fit tracks over known hit sequences. track_hits is [n][lmax] row-major, -1 padded (the
// entries equal to -1 are skipped, e.g. misses of a found track; the first three entries are
// the seed hits). Outputs per track: p[6], C packed upper-triangle [21] (row-major
// i<=j), chi2 total, ndof = 2N-5, status (0 ok, 1 seed failed, 2 propagation failed, 3 < 3 hits).
// Optional per-hit outputs [n][lmax]: predicted chi2 and the two normalised predicted residuals.
void or_fit(const OrGeom* g, const float* hits, const int* hsurf, const int* track_hits, long long n, int lmax,
            int n_threads, double* p_out, double* C_out, double* chi2_out, int* ndof_out, int* status_out,
            double* hit_chi2, double* hit_pull) {
  parallel_for(n, n_threads, [&](long long t) {
    const int* th = track_hits + t * lmax;
    int nh = 0;
    for (int k = 0; k < lmax; ++k) nh += th[k] >= 0;
    if (hit_chi2)
      for (int k = 0; k < lmax; ++k) hit_chi2[t * lmax + k] = -1.0;
    State st{};
    int status = 0;
    double chi2 = 0.0;
    if (nh < 3 || th[0] < 0 || th[1] < 0 || th[2] < 0) {
      status = 3;
    } else if (!seed_state(*g, hits, hsurf, th, st)) {
      status = 1;
    } else {
      for (int k = 0; k < lmax; ++k) {
        const int id = th[k];
        if (id < 0) continue;
        const int si = hsurf[id];
        if (k > 0) {
          State pr;
          if (!propagate(*g, st, si, pr)) {
            status = 2;
            break;
          }
          st = pr;
        }
        Meas m;
        measure(*g, si, st.p, hits[2 * id], hits[2 * id + 1], m);
        if (hit_pull) {
          double Sm[2][2];
          chi2_of(m, st.C, Sm);
          hit_pull[(t * lmax + k) * 2 + 0] = m.r[0] / std::sqrt(Sm[0][0]);
          hit_pull[(t * lmax + k) * 2 + 1] = m.r[1] / std::sqrt(Sm[1][1]);
        }
        const double c2 = kf_update(m, st);
        if (hit_chi2) hit_chi2[t * lmax + k] = c2;
        chi2 += c2;
      }
    }
    for (int i = 0; i < 6; ++i) p_out[6 * t + i] = status == 0 ? st.p[i] : NAN;
    pack_cov(st.C, nullptr, C_out + 21 * t);
    if (status != 0)
      for (int i = 0; i < 21; ++i) C_out[21 * t + i] = NAN;
    chi2_out[t] = status == 0 ? chi2 : NAN;
    ndof_out[t] = 2 * nh - 5;
    status_out[t] = status;
  });
}

// Hit index. bin_off is [n_events*n_surf][nb+1] (nb = max n_phi*n_2nd), absolute positions
// into sorted_hits[n_hits][2] / sorted_ids[n_hits].
int or_index_bins(const OrGeom* g) { return max_bins(*g); }

void or_build_index(const OrGeom* g, const float* hits, const long long* slab_off, int n_events, long long* bin_off,
                    float* sorted_hits, int* sorted_ids, unsigned short* sub_off) {
  Index ix;
  build_index(*g, hits, slab_off, n_events, ix);
  std::memcpy(bin_off, ix.off.data(), sizeof(long long) * ix.off.size());
  std::memcpy(sorted_hits, ix.sorted.data(), sizeof(float) * ix.sorted.size());
  std::memcpy(sorted_ids, ix.ids.data(), sizeof(int) * ix.ids.size());
  if (sub_off) std::memcpy(sub_off, ix.sub.data(), sizeof(unsigned short) * ix.sub.size());
}

// Bin of one value by the FP32 rule (tests compare it with the index).
void or_bin_of(const OrGeom* g, int surf, float phi, float second, int* phi_bin, int* second_bin) {
  const BinRule br(g->surf[surf]);
  *phi_bin = br.phi_bin(phi);
  *second_bin = br.second_bin(second);
}

// Hits passing the chi2 cut on surface `surf` of event `ev` for a predicted state (p, full C),
// by the binned window (brute=0) or by scanning every hit (brute=1). Returns the count written
// (at most cap), ids and chi2 in scan order.
int or_search(const OrGeom* g, const float* hits, const int* hsurf, const long long* slab_off, int n_events,
              const double* p, const double* C, int ev, int surf, float chi2_cut, int brute, int cap, int* ids_out,
              double* chi2_out) {
  Index ix;
  if (!brute) build_index(*g, hits, slab_off, n_events, ix);
  Ctx cx{g, hits, hsurf, slab_off, &ix, {chi2_cut, 1, 0, brute}};
  State st;
  for (int i = 0; i < 6; ++i) st.p[i] = p[i];
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) st.C[i][j] = C[6 * i + j];
  std::vector<Found> found;
  search_hits(cx, ev, surf, st, found);
  const int n = std::min(cap, static_cast<int>(found.size()));
  for (int i = 0; i < n; ++i) {
    ids_out[i] = found[i].hit;
    chi2_out[i] = found[i].chi2;
  }
  return static_cast<int>(found.size());
}

// Kalman update of one state (p[6], full C[36]) with hit (phi, second) on surface `surf`.
// Writes the updated state and covariance; returns the predicted chi2.
double or_update(const OrGeom* g, const double* p, const double* C, int surf, float hphi, float hsecond,
                 double* p_out, double* C_out) {
  State st;
  for (int i = 0; i < 6; ++i) st.p[i] = p[i];
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) st.C[i][j] = C[6 * i + j];
  Meas m;
  measure(*g, surf, st.p, hphi, hsecond, m);
  const double chi2 = kf_update(m, st);
  for (int i = 0; i < 6; ++i) p_out[i] = st.p[i];
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) C_out[6 * i + j] = st.C[i][j];
  return chi2;
}

// Next surface rule, for tests.
int or_next_surface(const OrGeom* g, const double* p, double* s_out) {
  State st;
  for (int i = 0; i < 6; ++i) st.p[i] = p[i];
  return next_surface(*g, st, s_out);
}

// Combinatorial finding from seeds (3 hit ids each, [n][3]) with seed_event[n]. With mlp_w set and
// top_n > 0, the learned proposal keeps only the top_n passing hits by MLP score of each window
// that has more; with score_margin > 0, of each window with two or more passing hits, the hits
// among its top_n that score within score_margin of its best; with window != 0, the top_n by score
// of every hit in the window's box go on to the chi2 cut when the box holds more than top_n hits
// (with score_margin > 0: two or more hits, and only those of the top_n within the margin of the
// best). Outputs per
// seed: hits_out[n][lmax] (path order, -1 = miss or none), n_hits, chi2 total, p[6], C[21],
// status (0 ok, 1 seed failed). steering: region steering lists, or null for the geometric
// next-surface rule. counters[6] += propagations, chi2 evaluations that passed the
// cut, Kalman updates, hits whose chi2 was evaluated (whole bins of the windows), hits of the
// windows limited to the phi sub-bins their phi range touches, network evaluations of the learned
// proposal.
void or_find(const OrGeom* g, const float* hits, const int* hsurf, const long long* slab_off, int n_events,
             const int* seeds, const int* seed_event, long long n, int lmax, const OrFindParams* prm, int n_threads,
             int* hits_out, int* nhits_out, double* chi2_out, double* p_out, double* C_out, int* status_out,
             long long* counters, const double* mlp_w, const double* mlp_mean, const double* mlp_sd, int top_n,
             const OrSteering* steering, double score_margin, int window) {
  Index ix;
  if (!prm->brute_force) build_index(*g, hits, slab_off, n_events, ix);
  Ctx cx{g, hits, hsurf, slab_off, &ix, *prm,
         Mlp{mlp_w, mlp_mean, mlp_sd, mlp_w ? top_n : 0, score_margin, window != 0}, steering};
  cx.n_hits = slab_off[static_cast<long long>(n_events) * g->n_surf];
  cx.n_events = n_events;
  std::atomic<long long> c_prop(0), c_chi2(0), c_upd(0), c_scan(0), c_win(0), c_mlp(0);
  parallel_for(n, n_threads, [&](long long i) {
    Cand best;
    Counters cnt;
    const bool ok = find_one(cx, seeds + 3 * i, seed_event[i], lmax, best, cnt);
    for (int k = 0; k < lmax; ++k) hits_out[i * lmax + k] = (ok && k < static_cast<int>(best.hits.size())) ? best.hits[k] : -1;
    nhits_out[i] = ok ? best.n_hits : 0;
    chi2_out[i] = ok ? best.chi2 : NAN;
    for (int k = 0; k < 6; ++k) p_out[6 * i + k] = ok ? best.st.p[k] : NAN;
    pack_cov(best.st.C, nullptr, C_out + 21 * i);
    status_out[i] = ok ? 0 : 1;
    c_prop += cnt.n_prop;
    c_chi2 += cnt.n_chi2;
    c_scan += cnt.n_scan;
    c_win += cnt.n_win;
    c_upd += cnt.n_upd;
    c_mlp += cnt.n_mlp;
  });
  if (counters) {
    counters[0] += c_prop.load();
    counters[1] += c_chi2.load();
    counters[2] += c_upd.load();
    counters[3] += c_scan.load();
    counters[4] += c_win.load();
    counters[5] += c_mlp.load();
  }
}

// ---- learned proposal: training pairs and the FP64 MLP ----------------------------------------
int or_mlp_nparams() { return kNParam; }

// Plain finding over the given seeds, returning every passing (candidate, hit) pair seen: features
// [n][14] (float) and label 1 if the hit belongs to the seed's simulated track. Returns the number
// of pairs (at most cap are written).
long long or_find_pairs(const OrGeom* g, const float* hits, const int* hsurf, const long long* slab_off, int n_events,
                        const int* seeds, const int* seed_event, const int* seed_track, const int* hit_sim, long long n,
                        int lmax, const OrFindParams* prm, int n_threads, long long cap, float* features, float* labels) {
  Index ix;
  build_index(*g, hits, slab_off, n_events, ix);
  Ctx cx{g, hits, hsurf, slab_off, &ix, *prm, Mlp{}};
  cx.n_hits = slab_off[static_cast<long long>(n_events) * g->n_surf];
  cx.n_events = n_events;
  std::vector<PairSink> sinks(n);
  parallel_for(n, n_threads, [&](long long i) {
    sinks[i].hit_sim = hit_sim;
    sinks[i].seed_track = seed_track[i];
    Cand best;
    Counters cnt;
    find_one(cx, seeds + 3 * i, seed_event[i], lmax, best, cnt, &sinks[i]);
  });
  long long k = 0;
  for (long long i = 0; i < n; ++i) {
    const long long m = static_cast<long long>(sinks[i].labels.size());
    for (long long j = 0; j < m && k < cap; ++j, ++k) {
      std::memcpy(features + kIn * k, sinks[i].features.data() + kIn * j, sizeof(float) * kIn);
      labels[k] = sinks[i].labels[j];
    }
  }
  return k;
}

// Features of one (predicted state p[6], covariance C[36] row-major, hit) pair, as the learned
// proposal sees them: p, log(C_ii + 1e-12), residuals over sqrt(S_ii).
void or_pair_features(const OrGeom* g, int surf, const double* p, const double* C, float hphi, float h2, double* f) {
  State st;
  for (int i = 0; i < 6; ++i) st.p[i] = p[i];
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) st.C[i][j] = C[6 * i + j];
  pair_features(*g, surf, st, hphi, h2, f);
}

// MLP on standardised features xs[n][14]: logits[n].
void or_mlp_forward(const double* w, const double* xs, long long n, double* logits) {
  for (long long i = 0; i < n; ++i) logits[i] = mlp_forward(w, xs + kIn * i);
}

// Mean binary cross-entropy with logits over the batch and its gradient grad[kNParam].
double or_mlp_loss_grad(const double* w, const double* xs, const double* y, long long n, double* grad) {
  for (int i = 0; i < kNParam; ++i) grad[i] = 0.0;
  double loss = 0.0;
  for (long long i = 0; i < n; ++i) loss += mlp_loss_grad(w, xs + kIn * i, y[i], 1.0 / n, grad);
  return loss / n;
}

// One Adam step (Kingma and Ba): m, v moments; step t >= 1.
void or_adam(double* w, const double* grad, double* m, double* v, int t, double lr, double b1, double b2, double eps) {
  const double c1 = 1.0 - std::pow(b1, t), c2 = 1.0 - std::pow(b2, t);
  for (int i = 0; i < kNParam; ++i) {
    m[i] = b1 * m[i] + (1.0 - b1) * grad[i];
    v[i] = b2 * v[i] + (1.0 - b2) * grad[i] * grad[i];
    w[i] -= lr * (m[i] / c1) / (std::sqrt(v[i] / c2) + eps);
  }
}

// ---- seed cleaning and duplicate-track removal (Sec. 3.2 and Sec. 4 readings) -----------------
// Seed parameters (kappa, phi, theta) from the circle through the three hits and the line through
// hits 1 and 3 (the seed state at hit 1); NaN when the hits give no seed.
void or_seed_params(const OrGeom* g, const float* hits, const int* hsurf, const int* seeds, long long n,
                    double* out) {
  for (long long i = 0; i < n; ++i) {
    State st;
    const bool ok = seeds[3 * i] >= 0 && seeds[3 * i + 1] >= 0 && seeds[3 * i + 2] >= 0 &&
                    seed_state(*g, hits, hsurf, seeds + 3 * i, st);
    out[3 * i] = ok ? st.p[3] : NAN;
    out[3 * i + 1] = ok ? st.p[4] : NAN;
    out[3 * i + 2] = ok ? st.p[5] : NAN;
  }
}

// Seeds i < j of the same event are duplicates when they share a hit and their directions agree
// (|d phi| < dphi, |d theta| < dtheta); a seed with a duplicate of lower index is removed
// (keep = 0). The rule depends on no processing order. params: or_seed_params.
void or_clean_seeds(const int* seeds, const int* seed_event, const double* params, long long n, double dphi,
                    double dtheta, int* keep) {
  std::unordered_map<int, std::vector<long long>> users;  // hit -> seeds using it
  for (long long i = 0; i < n; ++i)
    for (int k = 0; k < 3; ++k)
      if (seeds[3 * i + k] >= 0) users[seeds[3 * i + k]].push_back(i);
  for (long long j = 0; j < n; ++j) {
    keep[j] = 1;
    if (!(params[3 * j + 1] == params[3 * j + 1])) continue;  // no seed: nothing to compare
    for (int k = 0; k < 3 && keep[j]; ++k) {
      const int h = seeds[3 * j + k];
      if (h < 0) continue;
      for (long long i : users[h]) {
        if (i >= j || seed_event[i] != seed_event[j]) continue;
        const double a = std::fabs(wrap_angle(params[3 * i + 1] - params[3 * j + 1]));
        const double b = std::fabs(params[3 * i + 2] - params[3 * j + 2]);
        if (a < dphi && b < dtheta) {
          keep[j] = 0;
          break;
        }
      }
    }
  }
}

// Found tracks (hits[n][lmax], -1 = none; n_hits, chi2, final phi and theta): track j is removed
// (keep = 0) when a better track i of the same event (more hits, then lower chi2, then lower
// index) with |d phi| < dphi and |d theta| < dtheta holds more than half of j's hits.
void or_remove_duplicates(const int* hits, const int* n_hits, const double* chi2, const double* phi,
                          const double* theta, const int* track_event, long long n, int lmax, double dphi,
                          double dtheta, int* keep) {
  std::unordered_map<int, std::vector<long long>> users;
  for (long long i = 0; i < n; ++i)
    for (int k = 0; k < lmax; ++k)
      if (hits[i * lmax + k] >= 0) users[hits[i * lmax + k]].push_back(i);
  auto better = [&](long long i, long long j) {
    if (n_hits[i] != n_hits[j]) return n_hits[i] > n_hits[j];
    if (chi2[i] != chi2[j]) return chi2[i] < chi2[j];
    return i < j;
  };
  for (long long j = 0; j < n; ++j) {
    keep[j] = 1;
    int own = 0;
    std::unordered_map<long long, int> shared;
    for (int k = 0; k < lmax; ++k) {
      const int h = hits[j * lmax + k];
      if (h < 0) continue;
      ++own;
      for (long long i : users[h])
        if (i != j && track_event[i] == track_event[j]) ++shared[i];
    }
    for (const auto& kv : shared) {
      const long long i = kv.first;
      if (2 * kv.second <= own || !better(i, j)) continue;
      if (std::fabs(wrap_angle(phi[i] - phi[j])) < dphi && std::fabs(theta[i] - theta[j]) < dtheta) {
        keep[j] = 0;
        break;
      }
    }
  }
}

}  // extern "C"
