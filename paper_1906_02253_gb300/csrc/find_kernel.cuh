// Combinatorial Kalman-filter track finding (paper Sec. 2 and Sec. 4): a beam search per seed
// that keeps the k_max best candidates, stepping outward surface by surface, with hits picked
// through binned search windows. Seeds run in parallel with no hit marking between them
// (Sec. 3.2).
//
// Design: a warp owns floor(32 / KC) seeds with KC candidate slots each, one lane per slot, and
// keeps the candidates in shared memory (the geometry too, one copy per block). One step of all
// its seeds:
//  1. every lane with a live candidate picks the next surface and propagates it (state and
//     covariance in registers), then sets up its search window: the inverse innovation covariance
//     and up to kRows runs of sorted hit positions (one run per phi bin of the window);
//  2. the hits of all the warp's windows are flattened with a warp prefix sum and every lane
//     evaluates chi2 for every 32nd of them (full SIMT width whatever the window sizes); hits
//     below the cut are buffered in flattened order, so each owner's pairs form one contiguous
//     run, which the owner merges into its list of the k_max best by (total chi2, hit id);
//  3. per seed, each lane offers its children (hit children, miss child, carried candidate) as a
//     sorted list; k_max rounds of a tournament over the lists' heads (a segmented minimum by
//     shuffles) rank them, the child of rank j goes to slot j, and lane j materialises it (Kalman
//     update for a hit child) from its parent's record;
//  4. a seed whose candidates have all stopped writes its best track (backtracking a per-step
//     trace of parent slot and hit) and its lanes take the next seed from an atomic queue.
// The warps of a block vote once per step (block barrier), which keeps them in the same phase.
// Seeds are consumed in queue order, one event after another, so the warps of the GPU read the
// index of one or two events at a time through L2.
#pragma once

#include <algorithm>

#include "find_launch.cuh"
#include "mlp.cuh"

namespace kfgb {

constexpr int kWords = 32;      // candidate record: p[6], C[21], chi2, nh, nm, stopped, surf
constexpr int kHitBits = 27;    // trace entry: parent slot << 27 | (hit id + 1)
constexpr int kRows = 4;        // window runs (one per bin) per lane scanned cooperatively
constexpr int kPList = 128;     // buffered passing (candidate, hit) pairs per warp
constexpr unsigned kFull = 0xffffffffu;
static_assert(kPList >= 32, "the pair buffer holds one scan round");

// Geometry copy at the start of the block's shared memory.
constexpr size_t kGeomBytes = (sizeof(DevGeom) + 15) / 16 * 16;
static_assert(sizeof(DevGeom) % 4 == 0, "geometry is copied in 4-byte words");

template <int KC>
struct WarpSmem {
  float4 cand[kWords / 4][32];  // candidate records: words 4i..4i+3 of lane l at [i][l]
  float4 win_a[32];        // window of each lane: x, y, centre of the 2nd coordinate, transverse scale
  float4 win_b[32];        // S^-1 (00, 01, 11) and the far-hit threshold of window_chi2
  int2 rows[kRows][32];    // runs: (end of the run in the lane's flattened window, position - start)
  float hl_tot[KC][32];    // per lane: best passing hits, sorted by (total chi2, hit id)
  int hl_id[KC][32];
  int hl_pos[KC][32];
  unsigned long long tab_key[32];  // winner table of each group, by rank
  int tab_id[32];
  int tab_pos[32];
  union {
    struct {
      float c2[kPList];
      int id[kPList];
      int pos[kPList];
      int own[kPList];
    } pl;                               // buffered passing pairs (scan)
  } u;
};

// Learned instances of up to 4 slots hold the network's weight fragments in shared memory, after
// the geometry; the warps' areas follow.
template <int KC, bool LEARNED>
constexpr bool kFragInSmem = LEARNED && KC <= 4;
template <int KC, bool LEARNED>
__host__ __device__ constexpr size_t block_smem_base() {
  return kGeomBytes + (kFragInSmem<KC, LEARNED> ? static_cast<size_t>(kFragWords) * sizeof(uint4) : 0);
}

// Learned proposal: the floor of its log-variance features, log(1e-12).
constexpr float kLogFloor = -27.631021f;

// Learned proposal, per warp: the network score of each kept hit.
template <int KC>
struct WarpLearned {
  float hl_sc[KC][32];
  float2 box[32];  // window ranking: half-widths sqrt(cut S_00), sqrt(cut S_11) of each lane's window
  float pl_sc[kPList];  // score of each buffered pair being ranked
};

template <int KC, bool LEARNED>
__host__ __device__ size_t warp_smem_bytes(int lmax) {
  return (sizeof(WarpSmem<KC>) + static_cast<size_t>(lmax - 3) * 32 * sizeof(int) +
          (LEARNED ? sizeof(WarpLearned<KC>) : 0) + 15) / 16 * 16;
}

__device__ __forceinline__ bool before(float t, int id, float u, int uid) { return t < u || (t == u && id < uid); }

// Insert into a lane's kept list ordered by (score descending, hit id ascending), capacity cap.
template <int KC>
__device__ __forceinline__ void hl_insert_scored(WarpSmem<KC>& W, WarpLearned<KC>& L, int lane, int& n, int cap,
                                                 float sc, float tot, int id, int pos) {
  if (n == cap) {
    const float ls = L.hl_sc[cap - 1][lane];
    const int li = W.hl_id[cap - 1][lane];
    if (!(sc > ls || (sc == ls && id < li))) return;
    n = cap - 1;
  }
  int i = n;
  while (i > 0) {
    const float ps = L.hl_sc[i - 1][lane];
    const int pi = W.hl_id[i - 1][lane];
    if (!(sc > ps || (sc == ps && id < pi))) break;
    L.hl_sc[i][lane] = ps;
    W.hl_tot[i][lane] = W.hl_tot[i - 1][lane];
    W.hl_id[i][lane] = pi;
    W.hl_pos[i][lane] = W.hl_pos[i - 1][lane];
    --i;
  }
  L.hl_sc[i][lane] = sc;
  W.hl_tot[i][lane] = tot;
  W.hl_id[i][lane] = id;
  W.hl_pos[i][lane] = pos;
  ++n;
}

// Reorder a lane's kept list by (total chi2, hit id) and keep at most cap entries.
template <int KC>
__device__ __forceinline__ void hl_sort_by_chi2(WarpSmem<KC>& W, int lane, int& n, int cap) {
  for (int i = 1; i < n; ++i) {
    const float c = W.hl_tot[i][lane];
    const int id = W.hl_id[i][lane], pos = W.hl_pos[i][lane];
    int j = i;
    while (j > 0 && before(c, id, W.hl_tot[j - 1][lane], W.hl_id[j - 1][lane])) {
      W.hl_tot[j][lane] = W.hl_tot[j - 1][lane];
      W.hl_id[j][lane] = W.hl_id[j - 1][lane];
      W.hl_pos[j][lane] = W.hl_pos[j - 1][lane];
      --j;
    }
    W.hl_tot[j][lane] = c;
    W.hl_id[j][lane] = id;
    W.hl_pos[j][lane] = pos;
  }
  if (n > cap) n = cap;
}

struct Cand {
  float p[6];
  float C[21];
  float chi2;
  int nh, nm, stopped, surf;  // surf: (position in the steering list + 1) << 8 | surface id
};

template <int KC>
__device__ __forceinline__ void load_cand(const WarpSmem<KC>& W, int col, Cand& c) {
  float v[kWords];
#pragma unroll
  for (int i = 0; i < kWords / 4; ++i) {
    const float4 q = W.cand[i][col];
    v[4 * i] = q.x;
    v[4 * i + 1] = q.y;
    v[4 * i + 2] = q.z;
    v[4 * i + 3] = q.w;
  }
#pragma unroll
  for (int i = 0; i < 6; ++i) c.p[i] = v[i];
#pragma unroll
  for (int i = 0; i < 21; ++i) c.C[i] = v[6 + i];
  c.chi2 = v[27];
  c.nh = __float_as_int(v[28]);
  c.nm = __float_as_int(v[29]);
  c.stopped = __float_as_int(v[30]);
  c.surf = __float_as_int(v[31]);
}

template <int KC>
__device__ __forceinline__ void store_cand(WarpSmem<KC>& W, int col, const Cand& c) {
  float v[kWords];
#pragma unroll
  for (int i = 0; i < 6; ++i) v[i] = c.p[i];
#pragma unroll
  for (int i = 0; i < 21; ++i) v[6 + i] = c.C[i];
  v[27] = c.chi2;
  v[28] = __int_as_float(c.nh);
  v[29] = __int_as_float(c.nm);
  v[30] = __int_as_float(c.stopped);
  v[31] = __int_as_float(c.surf);
#pragma unroll
  for (int i = 0; i < kWords / 4; ++i) W.cand[i][col] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
}

// Word w of lane col's candidate record.
template <int KC>
__device__ __forceinline__ float& cand_word(WarpSmem<KC>& W, int w, int col) {
  return reinterpret_cast<float*>(&W.cand[w >> 2][col])[w & 3];
}
template <int KC>
__device__ __forceinline__ float cand_word(const WarpSmem<KC>& W, int w, int col) {
  return reinterpret_cast<const float*>(&W.cand[w >> 2][col])[w & 3];
}

// Full-range angle, out of line: only hits far from the prediction in azimuth need it.
static __device__ __noinline__ float atan2_cold(float a, float b) { return atan2f(a, b); }

// Residual angle phi_hit - phi_pred from the hit direction (c, s) rotated into the frame of the
// predicted position (x, y).
__device__ __forceinline__ float resid_angle(float x, float y, float c, float s) {
  const float a = x * s - y * c, b = x * c + y * s;
  if (b > 0.f && fabsf(a) < 0.05f * b) return atan_small(a, b);
  return atan2_cold(a, b);
}

// chi2 of a hit's search record against a window (wa: x, y, centre of the 2nd coordinate,
// transverse scale R; wb: S^-1 00, 01, 11 and the far-hit threshold t). With a = rho sin(dphi),
// b = rho cos(dphi) (rho the predicted transverse radius), chi2 >= R^2 dphi^2 / S_00 >=
// R^2 sin^2(dphi) / S_00 (the minimum over the second residual, then |dphi| >= |sin dphi|). Hits
// outside the series range of the angle are rejected (infinite chi2) when that bound reaches
// 1.002 x the cut, i.e. when a^2 >= t (a^2 + b^2) with t = 1.002 cut S_00 / R^2; the others get
// the full-range angle.
__device__ __forceinline__ float window_chi2(const float4& wa, const float4& wb, const float4& h, float& r0, float& r1) {
  const float a = wa.x * h.y - wa.y * h.x, b = wa.x * h.x + wa.y * h.y;
  float dphi;
  if (b > 0.f && fabsf(a) < 0.05f * b) {
    dphi = atan_small(a, b);
  } else {
    const float a2 = a * a;
    if (a2 >= wb.w * (a2 + b * b)) {
      r0 = r1 = 0.f;
      return __int_as_float(0x7f800000);
    }
    dphi = atan2_cold(a, b);
  }
  r0 = wa.w * dphi;
  r1 = h.z - wa.z;
  return r0 * (wb.x * r0 + wb.y * r1) + r1 * (wb.y * r0 + wb.z * r1);
}

// Kalman update of candidate c on surface si with the hit of search record h.
__device__ __forceinline__ void update_with(const DevGeom& G, int si, Cand& c, const float4& h) {
  Meas m;
  float rho;
  meas_setup(G, si, c.p, m, rho);
  const float dphi = resid_angle(c.p[0], c.p[1], h.x, h.y);
  if (G.type[si] == 0) {
    m.r0 = G.r_or_z[si] * dphi;
    m.r1 = h.z - c.p[2];
  } else {
    m.r0 = rho * dphi;
    m.r1 = h.z - rho;
  }
  Innov in;
  innovation(G, c.C, m, in);
  kalman_update(c.p, c.C, in, m.r0, m.r1);
}

__device__ __forceinline__ float update_exact(const DevGeom& G, int si, Cand& c, float phi_h, float v) {
  Meas m;
  float rho;
  meas_setup(G, si, c.p, m, rho);
  meas_residual(G, si, c.p, rho, phi_h, v, m);
  Innov in;
  innovation(G, c.C, m, in);
  return kalman_update(c.p, c.C, in, m.r0, m.r1);
}

// Insert (tot, id, pos) into lane's list sorted by (total chi2, hit id), capacity cap (holding n).
template <int KC>
__device__ __forceinline__ void hl_insert(WarpSmem<KC>& W, int lane, int& n, int cap, float tot, int id, int pos) {
  if (n == cap) {
    if (!before(tot, id, W.hl_tot[cap - 1][lane], W.hl_id[cap - 1][lane])) return;
    n = cap - 1;
  }
  int i = n;
  while (i > 0) {
    const float pc = W.hl_tot[i - 1][lane];
    const int pi = W.hl_id[i - 1][lane];
    if (!before(tot, id, pc, pi)) break;
    W.hl_tot[i][lane] = pc;
    W.hl_id[i][lane] = pi;
    W.hl_pos[i][lane] = W.hl_pos[i - 1][lane];
    --i;
  }
  W.hl_tot[i][lane] = tot;
  W.hl_id[i][lane] = id;
  W.hl_pos[i][lane] = pos;
  ++n;
}

// Barrel s is certainly crossed outside its z extent: the transverse path to radius R is at least
// R - rho (a straight line), so z moves by at least (R - rho) cot theta before the crossing.
__device__ __forceinline__ bool barrel_beyond_z(const DevGeom& G, int s, const float* p, float rho, float cot) {
  const float dz = (G.r_or_z[s] - rho) * cot;
  return (cot > 0.f && p[2] + dz > G.hi[s]) || (cot < 0.f && p[2] + dz < G.lo[s]);
}

// Whether the helix from state p reaches disk s within its r extent and half a turn, and the path
// to it. st, ct: sin and cos of the polar angle p[5].
__device__ __forceinline__ bool reach_disk(const DevGeom& G, const float* p, float w, int s, float st, float ct,
                                           float cot, Prop& pr) {
  if (!path_to_disk(p, w, G.r_or_z[s], st, ct, pr)) return false;
  float x, y, z;
  prop_position(p, pr, cot, x, y, z);
  const float r = sqrtf(x * x + y * y);
  return r >= G.lo[s] && r <= G.hi[s];
}

// Whether the helix from state p reaches surface s within its extent (barrel: z extent; disk:
// reach_disk), and the path to it.
__device__ __forceinline__ bool reach_surface(const DevGeom& G, const float* p, float w, int s, float st, float ct,
                                              float cot, Prop& pr) {
  if (G.type[s] == 0) {
    // z moves monotonically along the helix: past the z extent and moving away, it stays out; a
    // steering list's later barrel layers are passed over by the bound without a crossing search.
    if ((cot >= 0.f && p[2] > G.hi[s]) || (cot <= 0.f && p[2] < G.lo[s])) return false;
    if (barrel_beyond_z(G, s, p, sqrtf(p[0] * p[0] + p[1] * p[1]), cot)) return false;
    if (!path_to_cylinder(p, w, G.r_or_z[s], pr)) return false;
    const float z = p[2] + pr.s * cot;
    return z >= G.lo[s] && z <= G.hi[s];
  }
  return reach_disk(G, p, w, s, st, ct, cot, pr);
}

// Region of a seed from its third hit h on surface s3 (KfSteering): (z, rho) = (z, R) on a barrel,
// (Z, r) on a disk; barrel if |z| <= c_barrel rho, transition if |z| <= c_endcap rho, else endcap,
// +z side for z > 0 (regions 0 barrel, 1/2 transition, 3/4 endcap).
__device__ __forceinline__ int seed_region(const DevGeom& G, int s3, float2 h) {
  const bool barrel = G.type[s3] == 0;
  const float z = barrel ? h.y : G.r_or_z[s3];
  const float rho = barrel ? G.r_or_z[s3] : h.y;
  const float az = fabsf(z);
  if (az <= __fmul_rn(G.c_barrel, rho)) return 0;
  return (az <= __fmul_rn(G.c_endcap, rho) ? 1 : 3) + (z > 0.f ? 0 : 1);
}

// Next surface of a candidate and the path to it; -1 if none. With region steering: the next
// surface of the region's list after position pos that the candidate reaches (its position goes
// to newpos). Geometric rule: the next barrel layer beyond the candidate's radius (accepted if
// crossed within its z extent) and the next disk beyond |z| in the direction of motion (accepted if
// crossed within its r extent and half a turn), the nearer one; the layer lists are sorted, so
// each "next" is a lower bound, searched from the candidate's current surface `cur`. The barrel
// candidate of the geometric rule is tried in straight-line code; disks and steering lists go
// through one loop (a single further copy of the path solvers in the code).
// STEER = false: the geometric rule only; FLD = false: the uniform field only.
template <bool STEER, bool FLD>
__device__ __forceinline__ int next_surface(const DevGeom& G, const float* p, int cur, int region, int pos, float st,
                                            float ct, Prop& best, int& newpos) {
  const float w = -kCurvF * (FLD ? start_field(G, p) : G.bz) * p[3];
  const float cot = ct / st;
  const bool steer = STEER && G.steer != 0;
  int sb = -1, sd = -1;  // geometric candidates: next barrel layer, next disk
  if (!steer) {
    const float rho = sqrtf(p[0] * p[0] + p[1] * p[1]);
    const bool cur_ok = cur >= 0 && cur < G.n_surf;
    const float lim = rho + 0.01f;  // first barrel radius above lim
    int i = (cur_ok && G.type[cur] == 0) ? max(0, static_cast<int>(G.ord[cur])) : 0;
    while (i > 0 && G.barrel_r[i - 1] > lim) --i;
    while (i < G.n_barrel && !(G.barrel_r[i] > lim)) ++i;
    if (i < G.n_barrel) sb = G.barrel_order[i];
    if (cot > 0.f || cot < 0.f) {
      const bool fwd = cot > 0.f;
      const int nd = fwd ? G.n_dpos : G.n_dneg;
      const float* zs = fwd ? G.dpos_z : G.dneg_z;
      const float zlo = p[2] + 0.01f, zhi = p[2] - 0.01f;  // first disk beyond z in the direction of motion
      int j = (cur_ok && G.type[cur] != 0 && ((G.r_or_z[cur] > 0.f) == fwd)) ? max(0, static_cast<int>(G.ord[cur])) : 0;
      while (j > 0 && (fwd ? zs[j - 1] > zlo : zs[j - 1] < zhi)) --j;
      while (j < nd && !(fwd ? zs[j] > zlo : zs[j] < zhi)) ++j;
      if (j < nd) sd = fwd ? G.dpos_order[j] : G.dneg_order[j];
    }
  }
  int sel = -1;
  if (!steer) {
    if (sb >= 0) {
      Prop pr;
      if (path_to_cylinder(p, w, G.r_or_z[sb], pr)) {
        const float z = p[2] + pr.s * cot;
        if (z >= G.lo[sb] && z <= G.hi[sb]) {
          sel = sb;
          best = pr;
        }
      }
    }
    if (sd < 0) return sel;
    if (!STEER) {  // the disk candidate of the geometric rule
      Prop pr;
      if (reach_disk(G, p, w, sd, st, ct, cot, pr) && (sel < 0 || pr.s < best.s)) {
        sel = sd;
        best = pr;
      }
      return sel;
    }
  }
  const int q1 = steer ? G.steer_n[region] : 2;
#pragma unroll 1
  for (int q = steer ? pos + 1 : 1; q < q1; ++q) {
    const int s = steer ? G.steer_list[region][q] : sd;
    if (s < 0) continue;
    Prop pr;
    if (!reach_surface(G, p, w, s, st, ct, cot, pr)) continue;
    if (steer) {
      best = pr;
      newpos = q;
      return s;
    }
    if (sel < 0 || pr.s < best.s) {
      sel = s;
      best = pr;
    }
  }
  return sel;
}

// Words per seed of the seed states k_seed_states writes (p[6], C[21], chi2).
constexpr int kSeedWords = 28;

// A fresh seed's state (fitted by k_seed_states, structure of arrays with stride n) into the
// candidate record of `lane`; false for a failed seed. Out of line: once per seed.
template <int KC>
__device__ __noinline__ bool load_seed(WarpSmem<KC>& W, int lane, const float* in, int surf_word, int n) {
  const float chi2 = in[static_cast<size_t>(27) * n];
  if (!(chi2 >= 0.f)) return false;
  for (int i = 0; i < 27; ++i) cand_word(W, i, lane) = in[static_cast<size_t>(i) * n];
  cand_word(W, 27, lane) = chi2;
  cand_word(W, 28, lane) = __int_as_float(3);  // hits
  cand_word(W, 29, lane) = __int_as_float(0);  // misses
  cand_word(W, 30, lane) = __int_as_float(0);  // stopped
  cand_word(W, 31, lane) = __int_as_float(surf_word);
  return true;
}

// Output of a finished seed: the best candidate (slot 0 of the group at gbase) and its hit list,
// backtracked through the per-step trace of (parent slot, hit id + 1). Out of line: once per seed.
template <int KC>
__device__ __noinline__ void write_track(const WarpSmem<KC>& W, const int* trace, int gbase, int step, int seed, int n,
                                         int lmax, const int* seed_hits, int* hits_out, int* nhits_out,
                                         float* chi2_out, float* state_out, float* cov_out, int* status_out) {
  int sl = 0;
  for (int st = step - 1; st >= 0; --st) {
    const int e = trace[st * 32 + gbase + sl];
    hits_out[static_cast<size_t>(3 + st) * n + seed] = (e & ((1 << kHitBits) - 1)) - 1;
    sl = e >> kHitBits;
  }
  for (int k = 3 + step; k < lmax; ++k) hits_out[static_cast<size_t>(k) * n + seed] = -1;
  for (int k = 0; k < 3; ++k) hits_out[static_cast<size_t>(k) * n + seed] = seed_hits[static_cast<size_t>(k) * n + seed];
  nhits_out[seed] = __float_as_int(cand_word(W, 28, gbase));
  chi2_out[seed] = cand_word(W, 27, gbase);
  for (int i = 0; i < 6; ++i) state_out[static_cast<size_t>(i) * n + seed] = cand_word(W, i, gbase);
  for (int i = 0; i < 21; ++i) cov_out[static_cast<size_t>(i) * n + seed] = cand_word(W, 6 + i, gbase);
  status_out[seed] = 0;
}

// Packed ranking key: (63 - hits) << 58 | chi2 bits << 26 | (parent slot << 2 | kind) << 20.
// For chi2 >= 0 its IEEE bits order like its value (a rounding-negative chi2 ranks as 0); the hit
// id breaks remaining ties.
__device__ __forceinline__ unsigned long long pack_key(int nh, float c2, int pk) {
  return (static_cast<unsigned long long>(63 - nh) << 58) |
         (static_cast<unsigned long long>(__float_as_uint(fmaxf(c2, 0.f))) << 26) |
         (static_cast<unsigned long long>(pk) << 20);
}

// Options compiled into an instance (FEAT bits): region steering, material map and energy loss,
// parametrised field. Without them the geometric next-surface rule, the surfaces' x/X0 and the
// uniform field are compiled in alone; each option left out keeps its code out of the kernel.
constexpr int kFeatSteer = 1, kFeatMaterial = 2, kFeatField = 4, kFeatAll = 7;

// Blocks of the learned instances hold at most 192 threads: at two blocks per SM that leaves them
// 168 registers, which their scoring and score-ordered lists need (capped at 128, as the plain
// instances are for 256-thread blocks, they spilled ~150 bytes per thread and ran 21-29% slower).
constexpr int kFindMaxBlockLearned = 192;
template <int KC, bool LEARNED, int FEAT>
__global__ void __launch_bounds__(LEARNED ? kFindMaxBlockLearned : 256, 2) k_find_tracks(const __grid_constant__ DevGeom Gp,
                                                        const __grid_constant__ DevMat M, FindArgs A) {
  extern __shared__ __align__(16) unsigned char smem[];
  {
    // Geometry into shared memory: lanes index it by their own surface, which would serialise
    // constant-bank loads.
    const int* src = reinterpret_cast<const int*>(&Gp);
    int* dst = reinterpret_cast<int*>(smem);
    for (int i = threadIdx.x; i < static_cast<int>(sizeof(DevGeom) / 4); i += blockDim.x) dst[i] = src[i];
    // The learned instances of up to 4 slots keep the network's weight fragments (20 KiB) next to
    // it: their scoring reads them from shared memory instead of through L1 (7% faster on the
    // barrel + disk workload; larger instances have no room left for two blocks per SM).
    if constexpr (kFragInSmem<KC, LEARNED>) {
      uint4* fdst = reinterpret_cast<uint4*>(smem + kGeomBytes);
      for (int i = threadIdx.x; i < kFragWords; i += blockDim.x) fdst[i] = __ldg(A.mlp_frag + i);
    }
    __syncthreads();
  }
  const DevGeom& G = *reinterpret_cast<const DevGeom*>(smem);
  constexpr bool STEER = (FEAT & kFeatSteer) != 0, MAT = (FEAT & kFeatMaterial) != 0, FLD = (FEAT & kFeatField) != 0;
  constexpr int NS = 32 / KC;
  const int lane = threadIdx.x & 31;
  const int wid = threadIdx.x >> 5;
  const size_t wbytes = warp_smem_bytes<KC, LEARNED>(A.lmax);
  unsigned char* wbase = smem + block_smem_base<KC, LEARNED>() + wid * wbytes;
  WarpSmem<KC>& W = *reinterpret_cast<WarpSmem<KC>*>(wbase);
  int* trace = reinterpret_cast<int*>(wbase + sizeof(WarpSmem<KC>));  // [step][32]
  WarpLearned<KC>& WL = *reinterpret_cast<WarpLearned<KC>*>(wbase + sizeof(WarpSmem<KC>) +
                                                            static_cast<size_t>(A.lmax - 3) * 32 * sizeof(int));
  const float* __restrict__ wmlp = A.mlp;  // network parameters (biases, output layer, normaliser)
  // Capacity of a lane's list during the scan; a first pass of adaptive capacity (detect) keeps at
  // most its own slots (a lane with more passing hits makes its seed overflow anyway). With the
  // learned proposal a first pass runs only when top_n fits its slots, so a lane's list holds
  // exactly its children.
  const int keep = LEARNED ? A.top_n : (A.detect ? min(A.k_max, KC) : A.k_max);
  const bool detect = A.detect != 0;
  const bool margin_on = LEARNED && A.score_margin > 0.f;
  const bool window_rank = LEARNED && A.window_rank != 0;  // rank the window's box before the cut
  const int grp = lane / KC, slot = lane % KC;
  const bool in_grp = grp < NS;
  const int gbase = in_grp ? grp * KC : lane;
  const unsigned gmask = in_grp ? (((KC >= 32) ? kFull : ((1u << KC) - 1u)) << gbase) : (1u << lane);
  const int cap = A.k_max;
  const int n = A.n_seeds;
  const int max_steps = A.lmax - 3;
  const float cut = A.chi2_cut;

  int seed = -1, ev = 0, step = 0, region = 0;
  bool exhausted = !in_grp;
  bool valid = false;

  for (;;) {
    // ---- refill: a group without a seed takes the next one --------------------------------
    const bool want = !exhausted && seed < 0;
    int s = -1;
    // Seeds removed by cleaning (their outputs written by the seed-state kernel) are passed over
    // here rather than costing the group a step each.
    if (want && slot == 0) {
      s = atomicAdd(A.counter, 1);
      if (A.seed_list)  // second pass of adaptive capacity: the first pass's overflowing seeds
        s = s < min(*A.seed_list_count, n) ? A.seed_list[s] : n;
      else if (A.seed_keep)
        while (s < n && A.seed_keep[s] == 0) s = atomicAdd(A.counter, 1);
    }
    s = __shfl_sync(kFull, s, gbase);
    bool fresh = false;
    if (want) {
      if (s >= n || s < 0) {  // (a list entry outside the seeds, e.g. from a workspace shared by
        exhausted = true;     // overlapping calls, ends the group instead of reading out of bounds)
      } else {
        seed = s;
        step = 0;
        valid = false;
        fresh = true;
        ev = A.seed_event[seed];
      }
    }
    // One block-wide vote per step: the block's warps stay in step with each other, so the SM
    // fetches the code of one or two phases at a time (the kernel is larger than the instruction
    // cache); the block ends when none of its warps has a seed. This holds for the learned
    // instances too: with warps voting on their own they drift apart, and the larger learned
    // kernel then stalls on instruction fetch (twice as often per issued instruction), which costs
    // more than the barrier's wait for a warp that is scoring.
    if (!__syncthreads_or(seed >= 0)) break;

    // ---- a fresh group loads its seed state into slot 0 ------------------------------------
    int failed = 0;
    if (fresh && slot == 0) {
      // Candidate surface word: (position in the region's list + 1) << 8 | surface.
      const int s3 = A.seed_surf[seed];
      int pos = -1;
      if (STEER && G.steer && s3 >= 0 && s3 < G.n_surf) {
        region = seed_region(G, s3, A.hits[A.seed_hits[static_cast<size_t>(2) * n + seed]]);
        pos = G.steer_pos[region][s3];
      }
      valid = load_seed(W, lane, A.seed_state + seed, STEER ? ((pos + 1) << 8) | (s3 & 255) : s3, n);
      failed = !valid;  // a failed seed's outputs were written by the seed-state kernel
    }
    failed = __shfl_sync(kFull, failed, gbase);
    if (STEER) region = __shfl_sync(kFull, region, gbase);
    if (fresh && failed) {
      seed = -1;
      valid = false;
    }
    const bool on = seed >= 0;

    // ---- 1. propagation and window set-up -------------------------------------------------
    Cand c;
    int kind = 3;  // 0 hit children, 1 miss child, 2 carried, 3 empty slot
    // Window: phi bins pb0 .. pb0 + npb - 1 (wrapping), 2nd bins zb0 .. zb1, fine phi range
    // [flo, fhi]; its runs are enumerated from the cursor (row, zrun), row == npb when done.
    int si = -1, npb = 0, pb0 = 0, zb0 = 0, zb1 = 0, flo = 0, fhi = 0, hl_n = 0, row = 0, zrun = 0, newpos = -1;
    bool scored = false;  // learned: this lane's kept hits carry network scores
    float s00v = 1.f, s11v = 1.f;  // innovation variances of this lane's window
    if (on && valid) {
      load_cand(W, lane, c);
      kind = 2;
      if (!c.stopped) {
        Prop pr;
        float st, ct;
        sincos_small(c.p[5], st, ct);
        si = next_surface<STEER, FLD>(G, c.p, STEER ? c.surf & 255 : c.surf, region, STEER ? (c.surf >> 8) - 1 : -1,
                                      st, ct, pr, newpos);
        float bz = G.bz;
        if (si >= 0 && (!FLD || step_field(G, si, c.p, st, ct, pr, bz)) &&
            apply_propagation<MAT>(G, M, si, c.p, c.C, pr, st, ct, bz)) {
          kind = 1;
          Meas m;
          float rho;
          meas_setup(G, si, c.p, m, rho);
          Innov in;
          innovation(G, c.C, m, in);
          if (innovation_ok(in)) {
            const float det = in.s00 * in.s11 - in.s01 * in.s01;
            const float inv = 1.f / det;
            const bool barrel = G.type[si] == 0;
            const float rref = barrel ? G.r_or_z[si] : rho;
            const float cz = barrel ? c.p[2] : rho;
            W.win_a[lane] = make_float4(c.p[0], c.p[1], cz, rref);
            W.win_b[lane] = make_float4(in.s11 * inv, -in.s01 * inv, in.s00 * inv, 1.002f * cut * in.s00 / (rref * rref));
            if (LEARNED && window_rank) WL.box[lane] = make_float2(sqrtf(cut * in.s00), sqrtf(cut * in.s11));
            s00v = in.s00;
            s11v = in.s11;
            const float dphi = sqrtf(cut * in.s00) / rref * (1.f + 1e-4f) + 1e-5f;
            const float d2 = sqrtf(cut * in.s11) * (1.f + 1e-4f) + 1e-4f;
            const int nphi = G.n_phi[si];
            if (!(dphi < kPiF * (1.f - 2.f / nphi))) {
              pb0 = 0;
              npb = nphi;
              flo = 0;
              fhi = nphi * kPhiSub - 1;
            } else {
              const float phip = atan2f(c.p[1], c.p[0]);
              const float plo = wrap_pi(phip - dphi), phi_ = wrap_pi(phip + dphi);
              pb0 = phi_bin(G, si, plo);
              const int pb1 = phi_bin(G, si, phi_);
              int dp = pb1 - pb0;  // both in [0, nphi)
              if (dp < 0) dp += nphi;
              npb = dp + 1;
              flo = phi_fine(G, si, plo);
              fhi = phi_fine(G, si, phi_);
            }
            zb0 = second_bin(G, si, cz - d2);
            zb1 = second_bin(G, si, cz + d2);
            zrun = zb0;
          }
        } else {
          si = -1;
        }
      }
    }

    // ---- 2. cooperative chi2 over every window hit of the warp ------------------------------
    // Passes: every lane lists its next kRows runs of sorted positions (one per (phi bin, 2nd bin)
    // of its window, limited to the sub-bins its phi range touches; a phi bin whose sub-bins are
    // all in gives one run over its 2nd bins); the runs of the warp are flattened with a prefix
    // sum and scanned in rounds of 32 hits; passes repeat while any lane has runs left.
    const size_t slab = static_cast<size_t>(ev * G.n_surf + (si >= 0 ? si : 0));
    const int* off = A.bin_off + slab * (G.n_bins + 1);
    const unsigned short* sub = A.sub_off + slab * G.n_bins * kPhiSub;
    const int nphi = si >= 0 ? G.n_phi[si] : 1, n2 = si >= 0 ? G.n_2nd[si] : 1;
    int np = 0;      // buffered pairs
    int my_cnt = 0;  // buffered pairs of this lane's window: one contiguous run of the buffer
    int npass = 0;   // passing hits of this lane's window (a detecting pass counts beyond its list)
    // Buffered passing pairs go to their owner's list: the k_max best by (total chi2, hit id)
    // (plain), or, with the learned proposal, the top_n best by network score. A pair is scored
    // only when its owner has more passing hits than top_n (with a score margin, two or more);
    // otherwise every hit is kept anyway. A flush in the middle of the scan (buffer full) scores
    // all its pairs. The pairs to score are evaluated by the warp on the tensor cores, 8 at a
    // time; then each owner inserts its own (the kept list is ordered by (score, hit id), so the
    // order of insertion does not matter).
    auto flush = [&](int count, bool final_flush) {
      int run = my_cnt;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(kFull, run, o);
        if (lane >= o) run += v;
      }
      const int start = run - my_cnt;
      if (LEARNED) {
        const bool need = !final_flush || scored || hl_n + my_cnt > (margin_on ? 1 : keep);
        const unsigned needmask = __ballot_sync(kFull, need && my_cnt > 0);
        if (needmask) {
          // Every lane's raw candidate features (predicted state, log covariance diagonal) and the
          // square roots of its innovation variances; an owner's reach the rows of its pairs by
          // shuffles.
          float fe[kMlpIn];
#pragma unroll
          for (int i = 0; i < 6; ++i) fe[i] = c.p[i];
#pragma unroll
          for (int i = 0; i < 6; ++i) fe[6 + i] = logf(c.C[ci(i, i)] + 1e-12f);
          // On a disk z is fixed by the surface: after the projection onto it the z variance is
          // exactly zero, and in FP32 what is left is rounding residue of the projected terms
          // (up to ~1e-7 cm^2, far above the 1e-12 floor), so the feature takes the exact value.
          // On a barrel the x or y variance nears zero for crossings close to an axis, where the
          // residue may be negative: the floor also stands in for a NaN there (fmaxf drops it).
          if (si >= 0 && G.type[si] != 0) fe[8] = kLogFloor;
          fe[6] = fmaxf(fe[6], kLogFloor);
          fe[7] = fmaxf(fe[7], kLogFloor);
          fe[12] = sqrtf(s00v);
          fe[13] = sqrtf(s11v);
#pragma unroll
          for (int i = 0; i < 12; ++i) fe[i] = (fe[i] - __ldg(wmlp + kMlpMean + i)) / __ldg(wmlp + kMlpSd + i);
          // The pairs to score: the runs of the owners in needmask, numbered owner by owner.
          const int ncnt = ((needmask >> lane) & 1u) ? my_cnt : 0;
          int ninc = ncnt;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(kFull, ninc, o);
            if (lane >= o) ninc += v;
          }
          const int nexc = ninc - ncnt;
          const int total_sc = __shfl_sync(kFull, ninc, 31);
          const int t4 = lane & 3;
          for (int r0 = 0; r0 < total_sc; r0 += 8) {
            // Pair lane / 4 of this tile: its features in this lane's operand columns 2 t4,
            // 2 t4 + 1, 2 t4 + 8, 2 t4 + 9.
            const int j = r0 + (lane >> 2);
            int o = 0;
#pragma unroll
            for (int bit = 16; bit > 0; bit >>= 1) {
              const int v = __shfl_sync(kFull, ninc, o + bit - 1);
              if (v <= j) o += bit;
            }
            o = min(o, 31);
            const int k = __shfl_sync(kFull, start, o) + j - __shfl_sync(kFull, nexc, o);
            float f[12];
#pragma unroll
            for (int i = 0; i < 12; ++i) f[i] = __shfl_sync(kFull, fe[i], o);
            const float d12 = __shfl_sync(kFull, fe[12], o), d13 = __shfl_sync(kFull, fe[13], o);
            const bool real = j < total_sc;
            float x12 = 0.f, x13 = 0.f;
            if (real && t4 == 2) {
              const float4 hr = __ldg(A.sorted_rec + W.u.pl.pos[k]);
              float q0, q1;
              window_chi2(W.win_a[o], W.win_b[o], hr, q0, q1);
              x12 = (q0 / d12 - __ldg(wmlp + kMlpMean + 12)) / __ldg(wmlp + kMlpSd + 12);
              x13 = (q1 / d13 - __ldg(wmlp + kMlpMean + 13)) / __ldg(wmlp + kMlpSd + 13);
            }
            const float x[4] = {!real ? 0.f : t4 == 0 ? f[0] : t4 == 1 ? f[2] : t4 == 2 ? f[4] : f[6],
                                !real ? 0.f : t4 == 0 ? f[1] : t4 == 1 ? f[3] : t4 == 2 ? f[5] : f[7],
                                !real ? 0.f : t4 == 0 ? f[8] : t4 == 1 ? f[10] : t4 == 2 ? x12 : 0.f,
                                !real ? 0.f : t4 == 0 ? f[9] : t4 == 1 ? f[11] : t4 == 2 ? x13 : 0.f};
            const int kr = real ? k : -1;
            float2 l2;
            if constexpr (kFragInSmem<KC, LEARNED>)
              l2 = mlp_logit8<true>(reinterpret_cast<const uint4*>(smem + kGeomBytes), wmlp, x, lane);
            else
              l2 = mlp_logit8<false>(A.mlp_frag, wmlp, x, lane);
            // lanes 0-3 hold the logits of pairs 2 t4, 2 t4 + 1 of the tile (computed by lanes 8 t4, 8 t4 + 4)
            const int k0 = __shfl_sync(kFull, kr, 8 * t4), k1 = __shfl_sync(kFull, kr, 8 * t4 + 4);
            if (lane < 4) {
              if (k0 >= 0) WL.pl_sc[k0] = l2.x;
              if (k1 >= 0) WL.pl_sc[k1] = l2.y;
            }
          }
          __syncwarp();
          if ((needmask >> lane) & 1u)
            for (int k = start; k < start + my_cnt; ++k)
              hl_insert_scored(W, WL, lane, hl_n, keep, WL.pl_sc[k], c.chi2 + W.u.pl.c2[k], W.u.pl.id[k],
                               W.u.pl.c2[k] < cut ? W.u.pl.pos[k] : ~W.u.pl.pos[k]);
        }
        if (!need) {  // kept unconditionally (at most top_n of them)
          for (int k = start; k < start + my_cnt; ++k) {
            W.hl_tot[hl_n][lane] = c.chi2 + W.u.pl.c2[k];
            W.hl_id[hl_n][lane] = W.u.pl.id[k];
            W.hl_pos[hl_n][lane] = W.u.pl.c2[k] < cut ? W.u.pl.pos[k] : ~W.u.pl.pos[k];
            ++hl_n;
          }
        }
        scored = scored || (need && my_cnt > 0);
      } else {
        for (int k = start; k < start + my_cnt; ++k)
          hl_insert(W, lane, hl_n, keep, c.chi2 + W.u.pl.c2[k], W.u.pl.id[k], W.u.pl.pos[k]);
        npass += my_cnt;
      }
      my_cnt = 0;
    };
    for (;;) {
      int T = 0;
#pragma unroll
      for (int k = 0; k < kRows; ++k) {
        int a = 0, b = 0;
        if (row < npb) {
          int pb = pb0 + row;
          if (pb >= nphi) pb -= nphi;
          const int slo = row == 0 ? sub_of(flo, pb) : 0;
          const int shi = row == npb - 1 ? sub_of(fhi, pb) : kPhiSub - 1;
          if (slo == 0 && shi == kPhiSub - 1) {
            a = __ldg(off + pb * n2 + zb0);
            b = __ldg(off + pb * n2 + zb1 + 1);
            ++row;
          } else {
            const int bb = pb * n2 + zrun;
            const int s0 = __ldg(off + bb);
            a = s0 + (slo > 0 ? __ldg(sub + bb * kPhiSub + slo - 1) : 0);
            b = s0 + __ldg(sub + bb * kPhiSub + shi);
            if (++zrun > zb1) {
              zrun = zb0;
              ++row;
            }
          }
        }
        W.rows[k][lane] = make_int2(T + (b - a), a - T);
        T += b - a;
      }
      const bool more = __any_sync(kFull, row < npb);
      int incl = T;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += v;
      }
      const int total = __shfl_sync(kFull, incl, 31);
      const int excl = incl - T;
      __syncwarp();
      // Rounds of 32 hits; the buffer is merged after the last round of each pass (pairs of one
      // pass are in owner order, so each owner's pairs are one run of the buffer), or earlier when
      // it could not take another round.
      for (int q0 = 0;; q0 += 32) {
        if (q0 < total) {
          // Owner of hit q (binary search over the inclusive prefix), its position in the index
          // (the run of the owner's list it falls in) and its search record.
          const int q = q0 + lane;
          int owner = 0;
#pragma unroll
          for (int bit = 16; bit > 0; bit >>= 1) {
            const int v = __shfl_sync(kFull, incl, owner + bit - 1);
            if (v <= q) owner += bit;
          }
          owner = min(owner, 31);
          const int o = q - __shfl_sync(kFull, excl, owner);
          int adj = W.rows[kRows - 1][owner].y;
#pragma unroll
          for (int r = kRows - 2; r >= 0; --r) {
            const int2 rr = W.rows[r][owner];
            if (o < rr.x) adj = rr.y;
          }
          const int pos = o + adj;
          float c2v = __int_as_float(0x7f800000);
          int hid = 0;
          bool inbox = false;
          if (q < total) {
            const float4 h = __ldg(A.sorted_rec + pos);
            float r0, r1;
            c2v = window_chi2(W.win_a[owner], W.win_b[owner], h, r0, r1);
            hid = __float_as_int(h.w);
            // Window ranking buffers every hit of the box of the chi2 ellipse (a hit rejected by the
            // angular pre-test, c2v infinite, lies outside it).
            if (LEARNED && window_rank) {
              const float2 bx = WL.box[owner];
              inbox = c2v < __int_as_float(0x7f800000) && fabsf(r0) <= bx.x && fabsf(r1) <= bx.y;
            }
          }
          const bool pass = (LEARNED && window_rank) ? inbox : c2v < cut;
          const unsigned m = __ballot_sync(kFull, pass);
          // passing hits of this lane's own runs in this round
          const int lo = excl - q0, hi = incl - q0;
          if (hi > 0 && lo < 32) {
            const unsigned lom = lo <= 0 ? kFull : (kFull << lo);
            const unsigned him = hi >= 32 ? kFull : ((1u << hi) - 1u);
            my_cnt += __popc(m & lom & him);
          }
          if (pass) {
            const int k = np + __popc(m & ((1u << lane) - 1u));
            W.u.pl.c2[k] = c2v;
            W.u.pl.id[k] = hid;
            W.u.pl.pos[k] = pos;
            if (LEARNED) W.u.pl.own[k] = owner;
          }
          np += __popc(m);
        }
        const bool last = q0 + 32 >= total;
        if (last || np > kPList - 32) {
          __syncwarp();
          flush(np, last && !more);
          np = 0;
          __syncwarp();
        }
        if (last) break;
      }
      if (!more) break;
      __syncwarp();
    }
    // With the learned proposal the kept hits are reordered by chi2 for the ranking below; with a
    // score margin, the scored ones (kept in score order) are first cut to those within the margin
    // of the best.
    if (LEARNED && margin_on && scored) {
      const float floor_sc = WL.hl_sc[0][lane] - A.score_margin;
      int k = 1;
      while (k < hl_n && !(WL.hl_sc[k][lane] < floor_sc)) ++k;
      hl_n = min(hl_n, k);
    }
    // Window ranking: of the kept hits of the box, those failing the chi2 cut (position stored
    // inverted) make no child.
    if (LEARNED && window_rank && hl_n > 0) {
      int m = 0;
      for (int k = 0; k < hl_n; ++k) {
        if (W.hl_pos[k][lane] < 0) continue;
        W.hl_tot[m][lane] = W.hl_tot[k][lane];
        W.hl_id[m][lane] = W.hl_id[k][lane];
        W.hl_pos[m][lane] = W.hl_pos[k][lane];
        ++m;
      }
      hl_n = m;
    }
    if (LEARNED && hl_n > 0) hl_sort_by_chi2(W, lane, hl_n, cap);
    // Outcome of each propagated candidate; keep the prediction for its children.
    if (kind == 1) {
      kind = hl_n > 0 ? 0 : (c.nm < A.max_miss ? 1 : 2);
      if (kind != 2) {
        c.surf = STEER ? ((newpos + 1) << 8) | si : si;
        store_cand(W, lane, c);
      }
    }
    __syncwarp();

    // ---- 3. selection of the k_max best children of each seed -----------------------------
    // Each lane offers its children in ranking order (hit children by total chi2, or one miss or
    // carried child) as a list whose head key is in a register; k_max rounds of a tournament
    // over the group's heads (a segmented minimum by shuffles) give the seed's children in rank
    // order, and the child of rank j goes to the group's slot j. Keys of different lanes differ
    // (they carry the slot), so the order is the same total order as comparing all children.
    // In a detecting pass a seed whose children outnumber the slots overflows: its group takes no
    // part in the selection and the seed goes to the second pass (its children all fit otherwise,
    // and keeping them all is what the full capacity does).
    int nch = (on && kind != 3) ? (kind == 0 ? (detect && !LEARNED ? npass : hl_n) : 1) : 0;
    // Rounds: the most children any group of the warp has, up to k_max.
    int tot = nch;
#pragma unroll
    for (int off = 1; off < KC; off <<= 1) {
      const int v = __shfl_down_sync(kFull, tot, off);
      if (slot + off < KC) tot += v;
    }
    const bool ovf = detect && __shfl_sync(kFull, tot, gbase) > KC;
    if (ovf) nch = 0;
    const int rounds =
        min(cap, static_cast<int>(__reduce_max_sync(kFull, in_grp && slot == 0 && !ovf ? tot : 0)));
    unsigned long long mk = ~0ull, nk = ~0ull;  // this lane's head key and the one after it
    if (nch > 0) mk = kind == 0 ? pack_key(c.nh + 1, W.hl_tot[0][lane], slot << 2) : pack_key(c.nh, c.chi2, (slot << 2) | kind);
    if (nch > 1) nk = pack_key(c.nh + 1, W.hl_tot[1][lane], slot << 2);
    int head = 0;
    W.tab_key[lane] = ~0ull;
    __syncwarp();
#pragma unroll 1
    for (int r = 0; r < rounds; ++r) {
      unsigned long long m = mk;
#pragma unroll
      for (int off = 1; off < KC; off <<= 1) {
        const unsigned long long v = __shfl_down_sync(kFull, m, off);
        if (slot + off < KC) m = v < m ? v : m;
      }
      const unsigned long long gm = __shfl_sync(kFull, m, gbase);
      if (in_grp && mk != ~0ull && mk == gm) {
        W.tab_key[gbase + r] = mk;
        W.tab_id[gbase + r] = kind == 0 ? W.hl_id[head][lane] : -1;
        W.tab_pos[gbase + r] = kind == 0 ? W.hl_pos[head][lane] : 0;
        ++head;
        mk = nk;
        nk = head + 1 < nch ? pack_key(c.nh + 1, W.hl_tot[head + 1][lane], slot << 2) : ~0ull;
      }
    }
    __syncwarp();
    int w_par = 0, w_kind = 3, w_id = -1, w_pos = 0, w_nh = 0;
    float w_c2 = 0.f;
    if (on) {
      const unsigned long long mk = W.tab_key[lane];
      if (mk != ~0ull) {
        const int pk = static_cast<int>((mk >> 20) & 63ull);
        w_par = pk >> 2;
        w_kind = pk & 3;
        w_id = W.tab_id[lane];
        w_pos = W.tab_pos[lane];
        w_nh = 63 - static_cast<int>(mk >> 58);
        w_c2 = __uint_as_float(static_cast<unsigned>((mk >> 26) & 0xffffffffull));
      }
    }

    // ---- materialise: lane j takes the j-th winner ----------------------------------------
    Cand nc;
    const bool won = on && w_kind != 3;
    if (won) {
      load_cand(W, gbase + w_par, nc);
      if (w_kind == 0) {
        const float4 h = __ldg(A.sorted_rec + w_pos);
        update_with(G, STEER ? nc.surf & 255 : nc.surf, nc, h);
        nc.chi2 = w_c2;
        nc.nh = w_nh;
      } else if (w_kind == 1) {
        nc.nm += 1;
      } else {
        nc.stopped = 1;
      }
    }
    __syncwarp();
    if (won) {
      store_cand(W, lane, nc);
      trace[step * 32 + lane] = (w_par << kHitBits) | (w_kind == 0 ? w_id + 1 : 0);
    }
    if (on) valid = won;
    __syncwarp();

    // ---- 4. finished seeds write their best track -----------------------------------------
    if (on) ++step;
    const unsigned live = __ballot_sync(kFull, on && won && !nc.stopped);
    const bool done = on && (((live & gmask) == 0u) || step >= max_steps);
    if (done && slot == 0) {
      if (ovf) {
        const int at = atomicAdd(A.ovf_count, 1);
        if (at < n) A.ovf_list[at] = seed;  // the list holds n entries (each seed appends once)
      } else
        write_track(W, trace, gbase, step, seed, n, A.lmax, A.seed_hits, A.hits_out, A.nhits_out, A.chi2_out,
                    A.state_out, A.cov_out, A.status_out);
    }
    __syncwarp();
    if (done) {
      seed = -1;
      valid = false;
    }
  }
}

// Launch and occupancy of one instance. The learned instances are compiled in their own
// translation unit (find_learned.cu), the plain ones where they are dispatched (find.cu), so that
// the code of one kind does not change how the compiler allocates the other's registers.
template <int KC, bool L, int FEAT>
int find_occupancy(int block, size_t smem, int* bps) {
  static int attr_set[16] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 16) return KF_ERR_CUDA;
  if (static_cast<int>(smem) > attr_set[dev]) {
    if (cudaFuncSetAttribute(k_find_tracks<KC, L, FEAT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(smem)) != cudaSuccess)
      return KF_ERR_CUDA;
    attr_set[dev] = static_cast<int>(smem);
  }
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, k_find_tracks<KC, L, FEAT>, block, smem) != cudaSuccess)
    return KF_ERR_CUDA;
  return KF_OK;
}

template <int KC, bool L, int FEAT>
void find_launch_kernel(const DevGeom& G, const DevMat& M, const FindArgs& A, int grid, int block, size_t smem,
                        cudaStream_t stream) {
  k_find_tracks<KC, L, FEAT><<<grid, block, smem, stream>>>(G, M, A);
}

}  // namespace kfgb
