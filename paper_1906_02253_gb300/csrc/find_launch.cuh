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
  const float2* hits;
  const int* hit_surface;
  const int* seed_hits;
  const int* seed_event;
  int n_seeds;
  int n_events;  // events in the index; seeds naming another event fail (status 1)
  float chi2_cut;
  int k_max, max_miss, lmax;
  int* hits_out;
  int* nhits_out;
  float* chi2_out;
  float* state_out;
  float* cov_out;
  int* status_out;
  int* counter;  // work counter, zeroed before each launch
  float* cand;   // [2][KC][32][nt] candidate records, word-major
  int* trace;    // [lmax][KC][nt] parent slot and hit per step
  int nt;        // threads in the grid
};

// Template capacity kc (power of two >= k_max), persistent grid, workspace layout.
struct FindPlan {
  int kc, block, grid, nt;
  size_t off_cand, off_trace, ws_bytes;
};

int plan_find(int n_seeds, const KfFindParams* p, int sms, FindPlan* plan);
int launch_find(const DevGeom& G, FindArgs& A, const FindPlan& plan, void* ws, cudaStream_t stream);

}  // namespace kfgb
