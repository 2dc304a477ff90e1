// Launch plan and argument block of the finder kernel, shared by find.cu and the C ABI layer.
#pragma once

#include <cstddef>

#include "../../include/kfgb.h"
#include "kf_math.cuh"

namespace kfgb {

struct FindArgs {
  const int* bin_off;
  const float2* sorted_hits;
  const int* sorted_ids;
  const float4* sorted_rec;  // (cos phi, sin phi, second coordinate, id bits) per sorted hit
  const unsigned short* sub_off;  // per bin: hits with phi sub-bin <= j, j < kPhiSub
  const float2* hits;
  const int* hit_surface;
  const int* seed_hits;
  const int* seed_event;
  int n_seeds;
  int n_events;  // events in the index; seeds naming another event fail (status 1)
  float chi2_cut;
  int k_max, max_miss, lmax;
  const float* mlp;    // learned proposal parameters (KF_MLP_BUFFER floats) or null
  const uint4* mlp_frag;  // their hidden layers as tensor-core fragments in the workspace (set by launch_find)
  const int* seed_keep;  // seeds with 0 are skipped (status 2), or null
  int top_n;         // > 0 with mlp: keep the top_n passing hits by score
  float score_margin;  // > 0: of those, only the ones within this margin of the window's best score
  int window_rank;     // 1: rank every hit of the window's box, then apply the chi2 cut to the top_n
  int* hits_out;
  int* nhits_out;
  float* chi2_out;
  float* state_out;
  float* cov_out;
  int* status_out;
  // Workspace: the work counter (zeroed before each launch) and the fitted seed states.
  int* counter;
  float* seed_state;  // [28][n_seeds]: p[6], C[21], chi2 (< 0: failed seed)
  int* seed_surf;     // [n_seeds]: surface of the third seed hit
  // Adaptive capacity (plain finding): a first pass at a smaller capacity (detect = 1) finishes the
  // seeds whose children never outnumber its slots, which then have exactly the results of the
  // full capacity, and lists the others in ovf_list (*ovf_count of them) without writing their
  // outputs; the second pass takes its seeds from that list (seed_list, *seed_list_count).
  int detect;
  int* ovf_list;
  int* ovf_count;
  const int* seed_list;
  const int* seed_list_count;
};

// Candidate capacity kc (smallest compiled capacity >= k_max), persistent grid, shared memory,
// workspace layout.
struct FindPlan {
  int kc, block, grid;
  bool learned;
  int feat;  // options compiled into the instance: 1 steering, 2 material map and energy loss, 4 field
  size_t smem;
  size_t off_state, off_surf, off_mlp, ws_bytes;
  // Adaptive capacity: the first pass's capacity (0 = a single pass), launch and shared memory,
  // and the overflow list's place in the workspace.
  int kc1, block1, grid1;
  size_t smem1, off_ovf;
};

// general: the geometry or the parameters use region steering, the material map, energy loss or
// the parametrised field.
int plan_find(int n_seeds, const KfFindParams* p, int sms, int features, FindPlan* plan);
inline int find_features(const DevGeom& G, const DevMat& M) {
  return (G.steer != 0 ? 1 : 0) | ((M.map_on != 0 || M.eloss > 0.f) ? 2 : 0) | (G.field_on != 0 ? 4 : 0);
}
int launch_find(const DevGeom& G, const DevMat& M, FindArgs& A, const FindPlan& plan, void* ws, cudaStream_t stream);
// The seed-state kernel alone (A.hits_out null: failed seeds get chi2 = -1 only).
int launch_seed_states(const DevGeom& G, const DevMat& M, const FindArgs& A, cudaStream_t stream);
// Device address of the library's fixed finder scratch on the current device (looked up on the
// first call per device; no allocation).
int static_scratch(void** ptr);

}  // namespace kfgb
