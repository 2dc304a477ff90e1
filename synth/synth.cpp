// Seeded synthetic event generator for the Kalman-filter tracking workloads.
//
// Input generation only. It simulates charged particles from the origin in a uniform
// solenoid field (turning-angle helix parametrisation, charge-signed), finds their
// crossings with barrel cylinders and endcap disks by a safeguarded Newton/bisection
// root search, applies Highland multiple-scattering kicks as exact rotations of the
// momentum direction, smears the crossings into 2D hits and adds uniform noise hits.
// None of the track fit's arithmetic lives here: no state covariance, no Jacobian,
// no Kalman gain, no hit binning. Both the FP64 oracle and the CUDA path consume the
// FP32 hits this file writes.
//
// Random numbers: xoshiro256** (Blackman & Vigna) seeded through SplitMix64, one
// stream per (run seed, event index), Gaussian deviates by Box-Muller in FP64.

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr double kCurv = 0.00299792458;  // GeV / (T cm): pT = kCurv * B * radius

uint64_t splitmix64(uint64_t& x) {
  uint64_t z = (x += 0x9e3779b97f4a7c15ULL);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

struct Rng {
  uint64_t s[4];
  bool have_spare = false;
  double spare = 0.0;
  Rng(uint64_t seed, uint64_t stream) {
    uint64_t x = seed * 0x9e3779b97f4a7c15ULL ^ (stream + 0x632be59bd9b4e019ULL);
    for (int i = 0; i < 4; ++i) s[i] = splitmix64(x);
  }
  static uint64_t rotl(uint64_t v, int k) { return (v << k) | (v >> (64 - k)); }
  uint64_t next() {
    const uint64_t result = rotl(s[1] * 5, 7) * 9;
    const uint64_t t = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= t;
    s[3] = rotl(s[3], 45);
    return result;
  }
  double uniform() { return (next() >> 11) * 0x1.0p-53; }  // [0, 1)
  double gauss() {
    if (have_spare) {
      have_spare = false;
      return spare;
    }
    double u1 = uniform();
    while (u1 <= 0.0) u1 = uniform();
    const double u2 = uniform();
    const double mag = std::sqrt(-2.0 * std::log(u1));
    spare = mag * std::sin(2.0 * kPi * u2);
    have_spare = true;
    return mag * std::cos(2.0 * kPi * u2);
  }
};

}  // namespace

extern "C" {

struct SynthSurface {
  int type;        // 0 = barrel cylinder of radius r_or_z, 1 = disk at z = r_or_z
  double r_or_z;
  double lo, hi;   // barrel: z extent; disk: radial extent
  double x_over_x0;
};

struct SynthParams {
  int n_events;
  int tracks_lo, tracks_hi;  // per-event track count, uniform integer in [lo, hi]
  double pt_lo, pt_hi;       // GeV
  double eta_max;
  double bz;                 // tesla
  double sigma_rphi;         // cm, transverse smear
  double sigma_2nd;          // cm, z smear on barrels, r smear on disks
  double noise_frac;         // noise hits per surface = round(frac * signal hits on it)
  uint64_t seed;
  int ms_on;                 // apply multiple-scattering kicks
  int smear_on;              // smear hits (0: hits at exact crossings)
  int record_truth;          // keep true states at every crossing
  int n_threads;
  // Material map and mean energy loss (optional): x/X0 of surface s at kMatNodes points spread
  // evenly over its extent (z on barrels, r on disks), interpolated linearly at the crossing
  // (null: the surface's x_over_x0 everywhere); mean ionisation loss eloss GeV per unit of x/X0
  // crossed (0: none) for a particle of mass `mass` GeV.
  const double* material;    // [n_surf][kMatNodes] or null
  double eloss;
  double mass;
  // Module overlaps: with this probability a crossing leaves a second hit of the same particle
  // on the surface (an overlapping module; smeared independently).
  double overlap_frac;
  // Non-uniform solenoid field (optional): Bz(r, z) = bz (1 + field_z2 z^2 + field_r2 r^2), cm^-2;
  // the radial component is neglected. With either coefficient non-zero, particles are moved in
  // helix substeps of at most kFieldStep cm of transverse path, each with Bz at its midpoint.
  double field_z2, field_r2;
};
constexpr int kMatNodes = 8;
constexpr double kFieldStep = 0.5;

}  // extern "C"

namespace {

struct Particle {
  double x, y, z;
  double px, py, pz;
  int q;
};

struct Crossing {
  int surf;
  double x, y, z;
  double px, py, pz;  // momentum arriving at the surface
};

// Helix by turning angle psi >= 0 from the current point. For Bz > 0 a positive charge
// turns clockwise seen from +z, so the momentum azimuth is phi0 - h*psi with h = q*sign(Bz).
struct Helix {
  double x0, y0, z0, phi0, pt, cot_theta, rho;  // rho = bending radius [cm]
  int h;
  Helix(const Particle& p, double bz) {
    x0 = p.x;
    y0 = p.y;
    z0 = p.z;
    pt = std::hypot(p.px, p.py);
    phi0 = std::atan2(p.py, p.px);
    cot_theta = p.pz / pt;
    rho = pt / (kCurv * std::fabs(bz));
    h = (bz >= 0 ? p.q : -p.q);
  }
  void at(double psi, double& x, double& y, double& z) const {
    const double phi = phi0 - h * psi;
    x = x0 + h * rho * (std::sin(phi0) - std::sin(phi));
    y = y0 + h * rho * (std::cos(phi) - std::cos(phi0));
    z = z0 + rho * psi * cot_theta;
  }
  double radial_sq_minus(double psi, double R) const {
    double x, y, z;
    at(psi, x, y, z);
    return x * x + y * y - R * R;
  }
  // d/dpsi of x^2 + y^2
  double d_radial_sq(double psi) const {
    double x, y, z;
    at(psi, x, y, z);
    const double phi = phi0 - h * psi;
    return 2.0 * rho * (x * std::cos(phi) + y * std::sin(phi));
  }
};

// Smallest psi > 0 where the helix reaches radius R (R above the current radius), or -1.
double cross_cylinder(const Helix& hx, double R) {
  const double r0sq = hx.x0 * hx.x0 + hx.y0 * hx.y0;
  if (r0sq >= R * R) return -1.0;
  // Straight-line first guess for the transverse distance, turned into an angle.
  const double a = hx.x0 * std::cos(hx.phi0) + hx.y0 * std::sin(hx.phi0);
  const double line = -a + std::sqrt(a * a + R * R - r0sq);
  double hi = std::min(line / hx.rho, kPi);
  double lo = 0.0;
  int expand = 0;
  while (hx.radial_sq_minus(hi, R) < 0.0) {
    lo = hi;
    hi = std::min(hi * 1.5 + 1e-12, kPi);
    if (hi >= kPi && hx.radial_sq_minus(hi, R) < 0.0) return -1.0;
    if (++expand > 200) return -1.0;
  }
  // Newton steps kept inside the bracket [lo, hi]; bisection when a step leaves it.
  double psi = 0.5 * (lo + hi);
  for (int it = 0; it < 200; ++it) {
    const double f = hx.radial_sq_minus(psi, R);
    if (f < 0.0) lo = psi; else hi = psi;
    const double df = hx.d_radial_sq(psi);
    double next = (df != 0.0) ? psi - f / df : 0.5 * (lo + hi);
    if (!(next > lo && next < hi)) next = 0.5 * (lo + hi);
    if (std::fabs(next - psi) <= 1e-16 * std::max(1.0, psi) || hi - lo <= 1e-17) {
      psi = next;
      break;
    }
    psi = next;
  }
  return psi;
}

double cross_disk(const Helix& hx, double Z) {
  if (hx.cot_theta == 0.0) return -1.0;
  const double psi = (Z - hx.z0) / (hx.rho * hx.cot_theta);
  return (psi > 0.0 && psi < kPi) ? psi : -1.0;
}

struct TrackOut {
  std::vector<Crossing> cross;
  std::vector<std::array<double, 6>> truth_in, truth_out;  // (x,y,z,kappa,phi,theta)
};

std::array<double, 6> state_of(const Particle& p) {
  const double pt = std::hypot(p.px, p.py);
  return {p.x, p.y, p.z, p.q / pt, std::atan2(p.py, p.px), std::atan2(pt, p.pz)};
}

// Highland width for a unit-charge particle with beta = 1.
double highland(double p, double x_over_x0) {
  return 0.0136 / p * std::sqrt(x_over_x0) * (1.0 + 0.038 * std::log(x_over_x0));
}

void kick(Particle& p, double normal_cos, double x_over_x0, Rng& rng) {
  const double pmag = std::sqrt(p.px * p.px + p.py * p.py + p.pz * p.pz);
  const double t = x_over_x0 / std::max(std::fabs(normal_cos), 1e-6);
  const double theta0 = highland(pmag, t);
  const double a1 = rng.gauss() * theta0;
  const double a2 = rng.gauss() * theta0;
  double d[3] = {p.px / pmag, p.py / pmag, p.pz / pmag};
  // e1: azimuthal unit vector, e2 = d x e1 completes the right-handed frame.
  double e1[3] = {-d[1], d[0], 0.0};
  double n1 = std::hypot(e1[0], e1[1]);
  if (n1 < 1e-12) {
    e1[0] = 1.0;
    e1[1] = 0.0;
    n1 = 1.0;
  }
  e1[0] /= n1;
  e1[1] /= n1;
  const double e2[3] = {d[1] * e1[2] - d[2] * e1[1], d[2] * e1[0] - d[0] * e1[2],
                        d[0] * e1[1] - d[1] * e1[0]};
  const double alpha = std::sqrt(a1 * a1 + a2 * a2);
  if (alpha > 0.0) {
    const double c1 = a1 / alpha, c2 = a2 / alpha;
    const double ca = std::cos(alpha), sa = std::sin(alpha);
    for (int i = 0; i < 3; ++i) d[i] = ca * d[i] + sa * (c1 * e1[i] + c2 * e2[i]);
    const double nd = std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    for (int i = 0; i < 3; ++i) d[i] /= nd;
  }
  p.px = pmag * d[0];
  p.py = pmag * d[1];
  p.pz = pmag * d[2];
}

// x/X0 of surface s at second coordinate v (linear between the map's nodes, clamped at the ends).
double material_at(const SynthParams& prm, const SynthSurface& S, int s, double v) {
  if (!prm.material) return S.x_over_x0;
  double u = (v - S.lo) / (S.hi - S.lo) * (kMatNodes - 1);
  u = std::min(std::max(u, 0.0), static_cast<double>(kMatNodes - 1));
  const int k = std::min(static_cast<int>(std::floor(u)), kMatNodes - 2);
  const double* nd = prm.material + static_cast<size_t>(s) * kMatNodes;
  return nd[k] + (u - k) * (nd[k + 1] - nd[k]);
}

double field_at(const SynthParams& prm, double x, double y, double z) {
  return prm.bz * (1.0 + prm.field_z2 * z * z + prm.field_r2 * (x * x + y * y));
}

// Earliest crossing of a surface within turning angle psi_max along the helix (the next barrel
// layer beyond the current radius whose crossing lies within its z extent, and the nearer disk
// in the direction of motion within its r extent): best (turning angle) and its surface, or -1.
int first_crossing(const Helix& hx, const Particle& p, const std::vector<SynthSurface>& surf,
                   const std::vector<int>& barrel_order, const std::vector<int>& disk_pos,
                   const std::vector<int>& disk_neg, double psi_max, double& best) {
  const double rho_now = std::hypot(p.x, p.y);
  best = -1.0;
  int best_surf = -1;
  for (int s : barrel_order) {
    const SynthSurface& S = surf[s];
    if (S.r_or_z <= rho_now + 1e-9) continue;
    const double psi = cross_cylinder(hx, S.r_or_z);
    if (psi <= 0.0 || psi > psi_max) break;  // cannot reach this radius (in range), nor any larger one
    double x, y, z;
    hx.at(psi, x, y, z);
    if (z >= S.lo && z <= S.hi) {
      best = psi;
      best_surf = s;
      break;
    }
  }
  const std::vector<int>& disks = (hx.cot_theta >= 0.0) ? disk_pos : disk_neg;
  for (int s : disks) {
    const SynthSurface& S = surf[s];
    if (std::fabs(S.r_or_z) <= std::fabs(p.z) + 1e-9) continue;
    const double psi = cross_disk(hx, S.r_or_z);
    if (psi <= 0.0 || psi > psi_max) continue;
    if (best >= 0.0 && psi >= best) break;
    double x, y, z;
    hx.at(psi, x, y, z);
    const double r = std::hypot(x, y);
    if (r >= S.lo && r <= S.hi) {
      best = psi;
      best_surf = s;
      break;
    }
  }
  return best_surf;
}

// Move the particle along the helix by turning angle psi.
void advance(Particle& p, const Helix& hx, double psi) {
  double x, y, z;
  hx.at(psi, x, y, z);
  const double phi = hx.phi0 - hx.h * psi;
  p.x = x;
  p.y = y;
  p.z = z;
  p.px = hx.pt * std::cos(phi);
  p.py = hx.pt * std::sin(phi);
}

// Scattering and energy loss at a crossing of surface `si` (the particle is on it); false when
// the particle stops in the layer.
bool interact(Particle& p, int si, const std::vector<SynthSurface>& surf, const SynthParams& prm, Rng& rng) {
  const SynthSurface& S = surf[si];
  const double x = p.x, y = p.y, z = p.z;
  const double xx0 = material_at(prm, S, si, S.type == 0 ? z : std::hypot(x, y));
  if ((prm.ms_on && xx0 > 0.0) || prm.eloss > 0.0) {
    const double pmag = std::sqrt(p.px * p.px + p.py * p.py + p.pz * p.pz);
    double ncos;
    if (S.type == 0) {
      const double r = std::hypot(x, y);
      ncos = (p.px * x + p.py * y) / (pmag * r);
    } else {
      ncos = p.pz / pmag;
    }
    if (prm.ms_on && xx0 > 0.0) kick(p, ncos, xx0, rng);
    if (prm.eloss > 0.0 && xx0 > 0.0) {
      // Mean ionisation loss over the path through the layer; the direction is kept.
      const double e = std::sqrt(pmag * pmag + prm.mass * prm.mass);
      const double e1 = e - prm.eloss * xx0 / std::max(std::fabs(ncos), 1e-6);
      if (!(e1 > prm.mass)) return false;  // stopped in the layer
      const double f = std::sqrt(e1 * e1 - prm.mass * prm.mass) / pmag;
      p.px *= f;
      p.py *= f;
      p.pz *= f;
    }
  }
  return true;
}

void simulate_track(Particle p, const std::vector<SynthSurface>& surf, const std::vector<int>& barrel_order,
                    const std::vector<int>& disk_pos, const std::vector<int>& disk_neg, const SynthParams& prm,
                    Rng& rng, TrackOut& out) {
  const int max_steps = static_cast<int>(surf.size());
  const bool stepped = prm.field_z2 != 0.0 || prm.field_r2 != 0.0;
  for (int step = 0; step < max_steps; ++step) {
    int best_surf = -1;
    if (!stepped) {
      // Uniform field: the exact helix to the next crossing.
      Helix hx(p, prm.bz);
      double best;
      best_surf = first_crossing(hx, p, surf, barrel_order, disk_pos, disk_neg, kPi, best);
      if (best_surf < 0) return;
      advance(p, hx, best);
    } else {
      // Non-uniform field: substeps of at most kFieldStep cm transverse path, each a helix with
      // the field at its midpoint (second order); the crossing is solved on the substep's helix.
      // A particle is followed for at most half a turn between crossings, and not at all when
      // the helix of the local field reaches no surface (it has left the detector).
      {
        double best;
        const Helix hl(p, field_at(prm, p.x, p.y, p.z));
        if (first_crossing(hl, p, surf, barrel_order, disk_pos, disk_neg, kPi, best) < 0) return;
      }
      double turned = 0.0;
      for (int sub = 0; sub < 100000 && best_surf < 0; ++sub) {
        const Helix h0(p, field_at(prm, p.x, p.y, p.z));
        double xm, ym, zm;
        h0.at(0.5 * kFieldStep / h0.rho, xm, ym, zm);
        const Helix hx(p, field_at(prm, xm, ym, zm));
        const double psi_sub = std::min(kFieldStep / hx.rho, kPi - turned);
        if (!(psi_sub > 0.0)) return;
        double best;
        best_surf = first_crossing(hx, p, surf, barrel_order, disk_pos, disk_neg, psi_sub, best);
        advance(p, hx, best_surf >= 0 ? best : psi_sub);
        turned += best_surf >= 0 ? best : psi_sub;
      }
      if (best_surf < 0) return;
    }
    Crossing c{best_surf, p.x, p.y, p.z, p.px, p.py, p.pz};
    if (prm.record_truth) out.truth_in.push_back(state_of(p));
    if (!interact(p, best_surf, surf, prm, rng)) return;
    if (prm.record_truth) out.truth_out.push_back(state_of(p));
    out.cross.push_back(c);
  }
}

struct EventOut {
  int n_tracks = 0;
  std::vector<int> track_q;
  std::vector<double> track_init;  // pt, eta, phi per track
  std::vector<int> track_nhits;
  std::vector<int> track_hits;     // [n_tracks][lmax], event-local hit index, -1 pad
  std::vector<int> track_surf;     // [n_tracks][lmax]
  std::vector<double> truth_in, truth_out;  // [n_tracks][lmax][6]
  std::vector<float> hits;         // (phi, z|r) pairs, grouped by surface
  std::vector<int> hit_surface, hit_sim;
  std::vector<int> surf_count;     // hits per surface
};

float wrap_phi_f(double phi) {
  while (phi >= kPi) phi -= 2.0 * kPi;
  while (phi < -kPi) phi += 2.0 * kPi;
  return static_cast<float>(phi);
}

void generate_event(int e, int n_tracks, const std::vector<SynthSurface>& surf, const SynthParams& prm, int lmax,
                    EventOut& ev) {
  Rng rng(prm.seed, static_cast<uint64_t>(e) + 1);
  const int ns = static_cast<int>(surf.size());
  std::vector<int> barrel, dpos, dneg;
  for (int s = 0; s < ns; ++s) {
    if (surf[s].type == 0) barrel.push_back(s);
    else if (surf[s].r_or_z > 0) dpos.push_back(s);
    else dneg.push_back(s);
  }
  std::sort(barrel.begin(), barrel.end(), [&](int a, int b) { return surf[a].r_or_z < surf[b].r_or_z; });
  std::sort(dpos.begin(), dpos.end(), [&](int a, int b) { return surf[a].r_or_z < surf[b].r_or_z; });
  std::sort(dneg.begin(), dneg.end(), [&](int a, int b) { return surf[a].r_or_z > surf[b].r_or_z; });

  ev.n_tracks = n_tracks;
  ev.track_q.resize(n_tracks);
  ev.track_init.resize(3 * n_tracks);
  ev.track_nhits.assign(n_tracks, 0);
  ev.track_surf.assign(static_cast<size_t>(n_tracks) * lmax, -1);
  if (prm.record_truth) {
    ev.truth_in.assign(static_cast<size_t>(n_tracks) * lmax * 6, 0.0);
    ev.truth_out.assign(static_cast<size_t>(n_tracks) * lmax * 6, 0.0);
  }
  // Per surface: list of (phi, second coordinate, sim id, track, position in track).
  struct RawHit { float a, b; int sim, track, k; };
  std::vector<std::vector<RawHit>> per_surf(ns);
  TrackOut tout;
  for (int t = 0; t < n_tracks; ++t) {
    const int q = rng.uniform() < 0.5 ? -1 : 1;
    const double pt = prm.pt_lo + (prm.pt_hi - prm.pt_lo) * rng.uniform();
    const double eta = -prm.eta_max + 2.0 * prm.eta_max * rng.uniform();
    const double phi = -kPi + 2.0 * kPi * rng.uniform();
    ev.track_q[t] = q;
    ev.track_init[3 * t + 0] = pt;
    ev.track_init[3 * t + 1] = eta;
    ev.track_init[3 * t + 2] = phi;
    const double theta = 2.0 * std::atan(std::exp(-eta));
    Particle p{0.0, 0.0, 0.0, pt * std::cos(phi), pt * std::sin(phi), pt / std::tan(theta), q};
    tout.cross.clear();
    tout.truth_in.clear();
    tout.truth_out.clear();
    simulate_track(p, surf, barrel, dpos, dneg, prm, rng, tout);
    const int nh = std::min(static_cast<int>(tout.cross.size()), lmax);
    ev.track_nhits[t] = nh;
    for (int k = 0; k < nh; ++k) {
      const Crossing& c = tout.cross[k];
      const SynthSurface& S = surf[c.surf];
      ev.track_surf[static_cast<size_t>(t) * lmax + k] = c.surf;
      const double r = std::hypot(c.x, c.y);
      double phi_h = std::atan2(c.y, c.x);
      double second;
      if (S.type == 0) {
        if (prm.smear_on) phi_h += rng.gauss() * prm.sigma_rphi / S.r_or_z;
        second = c.z + (prm.smear_on ? rng.gauss() * prm.sigma_2nd : 0.0);
      } else {
        if (prm.smear_on) phi_h += rng.gauss() * prm.sigma_rphi / r;
        second = r + (prm.smear_on ? rng.gauss() * prm.sigma_2nd : 0.0);
      }
      per_surf[c.surf].push_back({wrap_phi_f(phi_h), static_cast<float>(second), t, t, k});
      if (prm.overlap_frac > 0.0 && rng.uniform() < prm.overlap_frac) {
        double phi2 = std::atan2(c.y, c.x), second2;
        if (S.type == 0) {
          if (prm.smear_on) phi2 += rng.gauss() * prm.sigma_rphi / S.r_or_z;
          second2 = c.z + (prm.smear_on ? rng.gauss() * prm.sigma_2nd : 0.0);
        } else {
          if (prm.smear_on) phi2 += rng.gauss() * prm.sigma_rphi / r;
          second2 = r + (prm.smear_on ? rng.gauss() * prm.sigma_2nd : 0.0);
        }
        per_surf[c.surf].push_back({wrap_phi_f(phi2), static_cast<float>(second2), t, -1, -1});
      }
      if (prm.record_truth) {
        for (int i = 0; i < 6; ++i) {
          ev.truth_in[(static_cast<size_t>(t) * lmax + k) * 6 + i] = tout.truth_in[k][i];
          ev.truth_out[(static_cast<size_t>(t) * lmax + k) * 6 + i] = tout.truth_out[k][i];
        }
      }
    }
  }
  // Noise hits, uniform over each surface.
  for (int s = 0; s < ns; ++s) {
    const int n_noise = static_cast<int>(std::llround(prm.noise_frac * per_surf[s].size()));
    const SynthSurface& S = surf[s];
    for (int i = 0; i < n_noise; ++i) {
      const double phi = -kPi + 2.0 * kPi * rng.uniform();
      double second;
      if (S.type == 0) {
        second = S.lo + (S.hi - S.lo) * rng.uniform();
      } else {
        second = std::sqrt(S.lo * S.lo + (S.hi * S.hi - S.lo * S.lo) * rng.uniform());
      }
      per_surf[s].push_back({wrap_phi_f(phi), static_cast<float>(second), -1, -1, -1});
    }
    // Shuffle within the surface (Fisher-Yates) so hit order carries no track order.
    auto& v = per_surf[s];
    for (int i = static_cast<int>(v.size()) - 1; i > 0; --i) {
      const int j = static_cast<int>(rng.uniform() * (i + 1));
      std::swap(v[i], v[std::min(j, i)]);
    }
  }
  ev.track_hits.assign(static_cast<size_t>(n_tracks) * lmax, -1);
  ev.surf_count.assign(ns, 0);
  int id = 0;
  for (int s = 0; s < ns; ++s) {
    ev.surf_count[s] = static_cast<int>(per_surf[s].size());
    for (const RawHit& h : per_surf[s]) {
      ev.hits.push_back(h.a);
      ev.hits.push_back(h.b);
      ev.hit_surface.push_back(s);
      ev.hit_sim.push_back(h.sim);
      if (h.track >= 0) ev.track_hits[static_cast<size_t>(h.track) * lmax + h.k] = id;
      ++id;
    }
  }
}

struct Batch {
  int lmax = 0, n_surf = 0;
  std::vector<EventOut> events;
};

}  // namespace

extern "C" {

// Generate a batch of events. Returns an opaque handle (nullptr on bad arguments).
void* synth_generate(const SynthParams* prm, const SynthSurface* surfaces, int n_surf, int lmax) {
  if (!prm || !surfaces || n_surf <= 0 || lmax <= 0 || prm->n_events <= 0) return nullptr;
  std::vector<SynthSurface> surf(surfaces, surfaces + n_surf);
  Batch* b = new Batch;
  b->lmax = lmax;
  b->n_surf = n_surf;
  b->events.resize(prm->n_events);
  std::vector<int> counts(prm->n_events);
  Rng count_rng(prm->seed, 0);
  for (int e = 0; e < prm->n_events; ++e) {
    const int span = prm->tracks_hi - prm->tracks_lo + 1;
    counts[e] = prm->tracks_lo + static_cast<int>(count_rng.uniform() * span);
  }
  int nt = prm->n_threads > 0 ? prm->n_threads : static_cast<int>(std::thread::hardware_concurrency());
  nt = std::max(1, std::min(nt, prm->n_events));
  std::vector<std::thread> pool;
  for (int w = 0; w < nt; ++w) {
    pool.emplace_back([&, w]() {
      for (int e = w; e < prm->n_events; e += nt) generate_event(e, counts[e], surf, *prm, lmax, b->events[e]);
    });
  }
  for (auto& t : pool) t.join();
  return b;
}

void synth_sizes(void* h, long long* n_hits, long long* n_tracks) {
  Batch* b = static_cast<Batch*>(h);
  long long nh = 0, ntr = 0;
  for (auto& e : b->events) {
    nh += static_cast<long long>(e.hit_surface.size());
    ntr += e.n_tracks;
  }
  *n_hits = nh;
  *n_tracks = ntr;
}

// Copy the batch out. Hit ids become global (event offsets added). Any pointer may be null.
//  hits[n_hits][2] f32, hit_surface[n_hits], hit_sim[n_hits] (global track id or -1),
//  slab_offsets[n_events*n_surf+1], track_event[n_tracks], track_q[n_tracks],
//  track_init[n_tracks][3] (pt, eta, phi), track_nhits[n_tracks],
//  track_hits[n_tracks][lmax], track_surf[n_tracks][lmax],
//  truth_in/out[n_tracks][lmax][6] (only when generated with record_truth).
void synth_copy(void* h, float* hits, int* hit_surface, int* hit_sim, long long* slab_offsets, int* track_event,
                int* track_q, double* track_init, int* track_nhits, int* track_hits, int* track_surf,
                double* truth_in, double* truth_out) {
  Batch* b = static_cast<Batch*>(h);
  const int lmax = b->lmax;
  long long hoff = 0, toff = 0;
  long long slab = 0;
  for (size_t e = 0; e < b->events.size(); ++e) {
    const EventOut& ev = b->events[e];
    const long long nh = static_cast<long long>(ev.hit_surface.size());
    if (hits) std::memcpy(hits + 2 * hoff, ev.hits.data(), sizeof(float) * 2 * nh);
    if (hit_surface) std::memcpy(hit_surface + hoff, ev.hit_surface.data(), sizeof(int) * nh);
    if (hit_sim)
      for (long long i = 0; i < nh; ++i) hit_sim[hoff + i] = ev.hit_sim[i] >= 0 ? static_cast<int>(ev.hit_sim[i] + toff) : -1;
    if (slab_offsets) {
      long long acc = hoff;
      for (int s = 0; s < b->n_surf; ++s) {
        slab_offsets[slab++] = acc;
        acc += ev.surf_count[s];
      }
    }
    for (int t = 0; t < ev.n_tracks; ++t) {
      const long long g = toff + t;
      if (track_event) track_event[g] = static_cast<int>(e);
      if (track_q) track_q[g] = ev.track_q[t];
      if (track_init)
        for (int i = 0; i < 3; ++i) track_init[3 * g + i] = ev.track_init[3 * t + i];
      if (track_nhits) track_nhits[g] = ev.track_nhits[t];
      for (int k = 0; k < lmax; ++k) {
        const int loc = ev.track_hits[static_cast<size_t>(t) * lmax + k];
        if (track_hits) track_hits[g * lmax + k] = loc >= 0 ? static_cast<int>(loc + hoff) : -1;
        if (track_surf) track_surf[g * lmax + k] = ev.track_surf[static_cast<size_t>(t) * lmax + k];
      }
      if (!ev.truth_in.empty()) {
        if (truth_in)
          std::memcpy(truth_in + g * lmax * 6, ev.truth_in.data() + static_cast<size_t>(t) * lmax * 6,
                      sizeof(double) * lmax * 6);
        if (truth_out)
          std::memcpy(truth_out + g * lmax * 6, ev.truth_out.data() + static_cast<size_t>(t) * lmax * 6,
                      sizeof(double) * lmax * 6);
      }
    }
    hoff += nh;
    toff += ev.n_tracks;
  }
  if (slab_offsets) slab_offsets[slab] = hoff;
}

void synth_free(void* h) { delete static_cast<Batch*>(h); }

// Helix crossing of a single particle, exposed for tests: starting at (x,y,z) with momentum
// (px,py,pz) and charge q, the smallest turning angle psi > 0 reaching cylinder R (type 0)
// or plane z = Z (type 1); writes the position and momentum there. Returns 0, or -1 if none.
int synth_cross(int type, double r_or_z, double bz, int q, const double* pos, const double* mom, double* pos_out,
                double* mom_out, double* psi_out) {
  Particle p{pos[0], pos[1], pos[2], mom[0], mom[1], mom[2], q};
  Helix hx(p, bz);
  const double psi = type == 0 ? cross_cylinder(hx, r_or_z) : cross_disk(hx, r_or_z);
  if (psi <= 0.0) return -1;
  hx.at(psi, pos_out[0], pos_out[1], pos_out[2]);
  const double phi = hx.phi0 - hx.h * psi;
  mom_out[0] = hx.pt * std::cos(phi);
  mom_out[1] = hx.pt * std::sin(phi);
  mom_out[2] = p.pz;
  if (psi_out) *psi_out = psi;
  return 0;
}

}  // extern "C"
