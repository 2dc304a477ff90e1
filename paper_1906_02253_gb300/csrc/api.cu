// C ABI of the library (declared in include/kfgb.h): argument checks, geometry packing into the
// kernels' by-value struct, launch configuration. Nothing here allocates device memory or
// synchronises; every launch goes to the caller's stream.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "../../include/kfgb.h"
#include "kf_math.cuh"
#include "mlp.cuh"

namespace kfgb {

__global__ void k_build_hit_index(DevGeom G, const float2* hits, const int* slab_off, int n_slabs, int cap,
                                  int* bin_off, float2* sorted_hits, int* sorted_ids, float4* sorted_rec,
                                  uint4* sub_off, int* d_status);
__global__ void k_fit_tracks(DevGeom G, const __grid_constant__ DevMat M, const float2* hits, const int* hit_surface,
                             const int* track_hits,
                             int n_tracks, int lmax, float* state_out, float* cov_out, float* chi2_out, int* ndof_out,
                             int* status_out);

size_t dup_workspace_bytes(int n, int m, int n_hits);
int launch_clean_seeds(const DevGeom& G, const float2* hits, const int* hit_surface, const int* seed_hits,
                       const int* seed_event, int n, int n_hits, float dphi, float dtheta, int* keep, void* ws,
                       cudaStream_t st);
int launch_fma_peak(float* sink, int blocks, int iters, cudaStream_t st, long long* flops);
int launch_math_probe(int fn, const float* a, const float* b, int n, float* o0, float* o1, float* o2,
                      cudaStream_t st);
int launch_wait_probe(int limit_us, long long* out, cudaStream_t st);
int launch_mlp_finder_scores(const float* params, const float* feats, int n, float* logits, uint4* frag,
                             cudaStream_t st);
static_assert(KF_MLP_FRAG_BYTES == kFragWords * sizeof(uint4), "header and library disagree on the fragment size");
int launch_remove_duplicates(const int* track_hits, const int* nhits, const float* chi2, const float* state,
                             const int* event, int n, int lmax, int n_hits, float dphi, float dtheta, int* keep,
                             void* ws, cudaStream_t st);

}  // namespace kfgb

#include "find_launch.cuh"

namespace kfgb {

static int pack_geometry(const KfGeometry* g, DevGeom* d) {
  if (!g || !g->surf || g->n_surf <= 0 || g->n_surf > kMaxSurf) return KF_ERR_ARG;
  if (!(std::isfinite(g->bz)) || g->bz == 0.f) return KF_ERR_ARG;
  if (!(g->sigma_rphi > 0.f) || !(g->sigma_2nd > 0.f)) return KF_ERR_ARG;
  std::memset(d, 0, sizeof(*d));
  d->bz = g->bz;
  d->sigma_rphi = g->sigma_rphi;
  d->sigma_2nd = g->sigma_2nd;
  for (int i = 0; i < 5; ++i) {
    if (!(g->prior[i] > 0.f)) return KF_ERR_ARG;
    d->prior[i] = g->prior[i];
  }
  d->n_surf = g->n_surf;
  d->ms_on = g->ms_off ? 0 : 1;
  if (!std::isfinite(g->field_z2) || !std::isfinite(g->field_r2)) return KF_ERR_ARG;
  d->field_on = (g->field_z2 != 0.f || g->field_r2 != 0.f) ? 1 : 0;
  d->fz2 = g->field_z2;
  d->fr2 = g->field_r2;
  int nb = 0;
  for (int s = 0; s < g->n_surf; ++s) {
    const KfSurface& S = g->surf[s];
    if (S.type != KF_BARREL && S.type != KF_DISK) return KF_ERR_ARG;
    if (S.n_phi < 1 || S.n_2nd < 1 || S.n_phi * S.n_2nd > 65536) return KF_ERR_ARG;
    if (!(S.hi > S.lo) || !(S.x_over_x0 >= 0.f)) return KF_ERR_ARG;
    if (S.type == KF_BARREL && !(S.r_or_z > 0.f)) return KF_ERR_ARG;
    d->type[s] = S.type;
    d->r_or_z[s] = S.r_or_z;
    d->lo[s] = S.lo;
    d->hi[s] = S.hi;
    d->x0[s] = S.x_over_x0;
    d->n_phi[s] = S.n_phi;
    d->n_2nd[s] = S.n_2nd;
    d->sphi[s] = static_cast<float>(static_cast<double>(S.n_phi) / (2.0 * 3.14159265358979323846));
    d->sphi_sub[s] =
        static_cast<float>(static_cast<double>(S.n_phi) * KF_PHI_SUB / (2.0 * 3.14159265358979323846));
    d->s2[s] = static_cast<float>(static_cast<double>(S.n_2nd) / (static_cast<double>(S.hi) - static_cast<double>(S.lo)));
    nb = std::max(nb, S.n_phi * S.n_2nd);
  }
  d->n_bins = nb;
  int ib = 0, ip = 0, in = 0;
  signed char idx[kMaxSurf];
  for (int s = 0; s < g->n_surf; ++s) idx[s] = static_cast<signed char>(s);
  std::sort(idx, idx + g->n_surf, [&](signed char a, signed char b) { return g->surf[a].r_or_z < g->surf[b].r_or_z; });
  for (int k = 0; k < g->n_surf; ++k) {
    const int s = idx[k];
    if (g->surf[s].type == KF_BARREL) d->barrel_order[ib++] = static_cast<signed char>(s);
    else if (g->surf[s].r_or_z > 0.f) d->dpos_order[ip++] = static_cast<signed char>(s);
  }
  for (int k = g->n_surf - 1; k >= 0; --k) {
    const int s = idx[k];
    if (g->surf[s].type == KF_DISK && g->surf[s].r_or_z < 0.f) d->dneg_order[in++] = static_cast<signed char>(s);
  }
  d->n_barrel = ib;
  d->n_dpos = ip;
  d->n_dneg = in;
  for (int s = 0; s < kMaxSurf; ++s) d->ord[s] = -1;
  for (int i = 0; i < ib; ++i) {
    d->ord[d->barrel_order[i]] = static_cast<signed char>(i);
    d->barrel_r[i] = d->r_or_z[d->barrel_order[i]];
  }
  for (int i = 0; i < ip; ++i) {
    d->ord[d->dpos_order[i]] = static_cast<signed char>(i);
    d->dpos_z[i] = d->r_or_z[d->dpos_order[i]];
  }
  for (int i = 0; i < in; ++i) {
    d->ord[d->dneg_order[i]] = static_cast<signed char>(i);
    d->dneg_z[i] = d->r_or_z[d->dneg_order[i]];
  }
  return KF_OK;
}

// Material map and energy loss of the geometry into their launch parameter.
static int pack_material(const KfGeometry* g, DevMat* m) {
  std::memset(m, 0, sizeof(*m));
  if (!(g->eloss >= 0.f) || !std::isfinite(g->eloss)) return KF_ERR_ARG;
  if (g->eloss > 0.f && !(g->mass > 0.f)) return KF_ERR_ARG;
  m->eloss = g->eloss;
  m->mass = g->mass;
  if (g->material) {
    for (int s = 0; s < g->n_surf; ++s)
      for (int k = 0; k < kMatNodes; ++k) {
        const float v = g->material[s * kMatNodes + k];
        if (!(v >= 0.f) || !std::isfinite(v)) return KF_ERR_ARG;
        m->node[s][k] = v;
      }
    m->map_on = 1;
  }
  return KF_OK;
}

// Region steering tables into the kernels' geometry (steer = 0 without them).
static int pack_steering(const KfSteering* st, DevGeom* d) {
  d->steer = 0;
  d->c_barrel = d->c_endcap = 0.f;
  std::memset(d->steer_n, 0, sizeof(d->steer_n));
  std::memset(d->steer_list, -1, sizeof(d->steer_list));
  std::memset(d->steer_pos, -1, sizeof(d->steer_pos));
  if (!st) return KF_OK;
  if (!(st->c_barrel >= 0.f) || !(st->c_endcap >= st->c_barrel) || !std::isfinite(st->c_endcap)) return KF_ERR_ARG;
  for (int r = 0; r < KF_N_REGIONS; ++r) {
    if (st->n[r] < 0 || st->n[r] > KF_MAX_SURF) return KF_ERR_ARG;
    for (int q = 0; q < st->n[r]; ++q) {
      const int s = st->surf[r][q];
      if (s < 0 || s >= d->n_surf || d->steer_pos[r][s] >= 0) return KF_ERR_ARG;  // in range, listed once
      d->steer_list[r][q] = static_cast<signed char>(s);
      d->steer_pos[r][s] = static_cast<signed char>(q);
    }
    d->steer_n[r] = st->n[r];
  }
  d->steer = 1;
  d->c_barrel = st->c_barrel;
  d->c_endcap = st->c_endcap;
  return KF_OK;
}

static int sm_count() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  return n;
}

static int launch_status() {
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? KF_OK : KF_ERR_CUDA;
}

}  // namespace kfgb

namespace {

struct EventPair {
  cudaEvent_t a = nullptr, b = nullptr;
  EventPair() {
    cudaEventCreate(&a);
    cudaEventCreate(&b);
  }
  ~EventPair() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
};

// Median of three timed runs after one untimed run; negative on a launch error.
template <class F>
float time_config(cudaStream_t st, F&& run) {
  EventPair ev;
  if (run() != KF_OK) return -1.f;
  float t[3];
  for (int i = 0; i < 3; ++i) {
    cudaEventRecord(ev.a, st);
    if (run() != KF_OK) return -1.f;
    cudaEventRecord(ev.b, st);
    if (cudaEventSynchronize(ev.b) != cudaSuccess) return -1.f;
    cudaEventElapsedTime(&t[i], ev.a, ev.b);
  }
  std::sort(t, t + 3);
  return t[1];
}

}  // namespace

using namespace kfgb;

extern "C" {

int kf_index_bins(const KfGeometry* geom) {
  DevGeom G;
  const int rc = pack_geometry(geom, &G);
  return rc == KF_OK ? G.n_bins : rc;
}

int kf_build_hit_index(const KfGeometry* geom, const float* hits, const int* slab_offsets, int n_events,
                       int max_slab_hits, const KfHitIndex* index, int* d_status, kf_stream_t stream) {
  DevGeom G;
  int rc = pack_geometry(geom, &G);
  if (rc != KF_OK) return rc;
  if (!slab_offsets || !index || n_events < 0 || max_slab_hits < 0) return KF_ERR_ARG;
  if (max_slab_hits > KF_MAX_SLAB_HITS) return KF_ERR_CAPACITY;
  if (index->n_events != n_events || index->n_bins != G.n_bins) return KF_ERR_ARG;
  if (n_events == 0) return KF_OK;
  if (!index->bin_off || !index->sorted_hits || !index->sorted_ids || (!hits && max_slab_hits > 0)) return KF_ERR_ARG;
  if ((reinterpret_cast<size_t>(index->sorted_rec) & 15) || (reinterpret_cast<size_t>(index->sub_off) & 15))
    return KF_ERR_ARG;
  const int n_slabs = n_events * G.n_surf;
  const int cap = std::max(2, (max_slab_hits + 1) & ~1);
  const size_t smem = static_cast<size_t>(G.n_bins + 1) * sizeof(int) + 2 * static_cast<size_t>(cap) * sizeof(unsigned short) +
                      static_cast<size_t>(cap) * sizeof(unsigned char);
  // Raise the kernel's dynamic shared memory limit once per device (and only when a larger slab
  // needs it), so later calls, e.g. inside a stream capture, make no attribute call.
  static int smem_set[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return KF_ERR_CUDA;
  if (static_cast<int>(smem) > smem_set[dev]) {
    if (cudaFuncSetAttribute(k_build_hit_index, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(smem)) != cudaSuccess)
      return KF_ERR_CUDA;
    smem_set[dev] = static_cast<int>(smem);
  }
  k_build_hit_index<<<n_slabs, 1024, smem, reinterpret_cast<cudaStream_t>(stream)>>>(
      G, reinterpret_cast<const float2*>(hits), slab_offsets, n_slabs, cap, index->bin_off,
      reinterpret_cast<float2*>(index->sorted_hits), index->sorted_ids, reinterpret_cast<float4*>(index->sorted_rec),
      reinterpret_cast<uint4*>(index->sub_off), d_status);
  return launch_status();
}

int kf_fit_tracks(const KfGeometry* geom, const float* hits, const int* hit_surface, const int* track_hits,
                  int n_tracks, int lmax, float* state_out, float* cov_out, float* chi2_out, int* ndof_out,
                  int* status_out, int block_threads, kf_stream_t stream) {
  DevGeom G;
  int rc = pack_geometry(geom, &G);
  if (rc != KF_OK) return rc;
  DevMat M;
  rc = pack_material(geom, &M);
  if (rc != KF_OK) return rc;
  if (n_tracks < 0 || lmax < 3 || lmax > KF_MAX_LMAX) return KF_ERR_ARG;
  if (block_threads == 0) block_threads = 128;
  if (block_threads < 32 || block_threads > 256 || block_threads % 32) return KF_ERR_ARG;
  if (n_tracks == 0) return KF_OK;
  if (!hits || !hit_surface || !track_hits || !state_out || !cov_out || !chi2_out || !ndof_out || !status_out)
    return KF_ERR_ARG;
  // Persistent grid: as many blocks as stay resident, each thread striding over the tracks.
  static int occ_cache[64][8] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return KF_ERR_CUDA;
  int& occ = occ_cache[dev][block_threads / 32 - 1];
  if (occ == 0) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_fit_tracks, block_threads, 0) != cudaSuccess || occ < 1)
      occ = 1;
  }
  const long long want = (static_cast<long long>(n_tracks) + block_threads - 1) / block_threads;
  const int grid = static_cast<int>(std::min<long long>(want, static_cast<long long>(sm_count()) * occ));
  k_fit_tracks<<<grid, block_threads, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
      G, M, reinterpret_cast<const float2*>(hits), hit_surface, track_hits, n_tracks, lmax, state_out, cov_out, chi2_out,
      ndof_out, status_out);
  return launch_status();
}

size_t kf_find_workspace_size(int n_seeds, const KfFindParams* params) {
  FindPlan plan;
  if (plan_find(n_seeds, params, sm_count(), 7, &plan) != KF_OK) return 0;
  return plan.ws_bytes;
}

}  // extern "C"

namespace kfgb {

// Argument checks, geometry packing, launch plan and kernel arguments of a finder call, shared by
// kf_find_tracks and kf_find_tracks_static (which differ only in where the scratch lives).
// Returns KF_OK with *empty set when there is nothing to launch (no seeds).
static int prepare_find(const KfGeometry* geom, const KfHitIndex* index, const float* hits, const int* hit_surface,
                        const int* seed_hits, const int* seed_event, int n_seeds, const KfFindParams* params,
                        int* hits_out, int* nhits_out, float* chi2_out, float* state_out, float* cov_out,
                        int* status_out, int max_seeds, DevGeom* G, DevMat* M, FindPlan* plan, FindArgs* A,
                        bool* empty) {
  *empty = false;
  int rc = pack_geometry(geom, G);
  if (rc != KF_OK) return rc;
  if (!params || !index || n_seeds < 0) return KF_ERR_ARG;
  rc = pack_steering(params->steering, G);
  if (rc != KF_OK) return rc;
  rc = pack_material(geom, M);
  if (rc != KF_OK) return rc;
  if (max_seeds >= 0 && n_seeds > max_seeds) return KF_ERR_CAPACITY;
  rc = plan_find(n_seeds, params, sm_count(), find_features(*G, *M), plan);
  if (rc != KF_OK) return rc;
  if (n_seeds == 0) {
    *empty = true;
    return KF_OK;
  }
  if (index->n_bins != G->n_bins || !index->bin_off || !index->sorted_hits || !index->sorted_ids ||
      !index->sorted_rec || (reinterpret_cast<size_t>(index->sorted_rec) & 15) || !index->sub_off)
    return KF_ERR_ARG;
  if (!hits || !hit_surface || !seed_hits || !seed_event || !hits_out || !nhits_out || !chi2_out || !state_out ||
      !cov_out || !status_out)
    return KF_ERR_ARG;
  A->bin_off = index->bin_off;
  A->sorted_hits = reinterpret_cast<const float2*>(index->sorted_hits);
  A->sorted_ids = index->sorted_ids;
  A->sorted_rec = reinterpret_cast<const float4*>(index->sorted_rec);
  A->sub_off = index->sub_off;
  A->hits = reinterpret_cast<const float2*>(hits);
  A->hit_surface = hit_surface;
  A->seed_hits = seed_hits;
  A->seed_event = seed_event;
  A->n_seeds = n_seeds;
  A->n_events = index->n_events;
  A->chi2_cut = params->chi2_cut;
  A->k_max = params->k_max;
  A->max_miss = params->max_miss;
  A->lmax = params->lmax;
  A->hits_out = hits_out;
  A->nhits_out = nhits_out;
  A->chi2_out = chi2_out;
  A->state_out = state_out;
  A->cov_out = cov_out;
  A->status_out = status_out;
  A->mlp = params->mlp;
  A->top_n = params->mlp ? params->top_n : 0;
  A->score_margin = params->mlp ? params->score_margin : 0.f;
  A->window_rank = params->mlp ? params->window_ranking : 0;
  A->seed_keep = params->seed_keep;
  return KF_OK;
}

}  // namespace kfgb

extern "C" {

int kf_find_tracks(const KfGeometry* geom, const KfHitIndex* index, const float* hits, const int* hit_surface,
                   const int* seed_hits, const int* seed_event, int n_seeds, const KfFindParams* params,
                   int* hits_out, int* nhits_out, float* chi2_out, float* state_out, float* cov_out,
                   int* status_out, void* workspace, size_t workspace_bytes, kf_stream_t stream) {
  DevGeom G;
  DevMat M;
  FindPlan plan;
  FindArgs A;
  bool empty = false;
  const int rc = prepare_find(geom, index, hits, hit_surface, seed_hits, seed_event, n_seeds, params, hits_out,
                              nhits_out, chi2_out, state_out, cov_out, status_out, -1, &G, &M, &plan, &A, &empty);
  if (rc != KF_OK || empty) return rc;
  if (!workspace || workspace_bytes < plan.ws_bytes || (reinterpret_cast<size_t>(workspace) & 255)) return KF_ERR_ARG;
  return launch_find(G, M, A, plan, workspace, reinterpret_cast<cudaStream_t>(stream));
}

int kf_seed_states(const KfGeometry* geom, const float* hits, const int* hit_surface, const int* seed_hits,
                   const int* seed_event, int n_seeds, int n_events, float* state_out, int* surf_out,
                   kf_stream_t stream) {
  DevGeom G;
  int rc = pack_geometry(geom, &G);
  if (rc != KF_OK) return rc;
  DevMat M;
  rc = pack_material(geom, &M);
  if (rc != KF_OK) return rc;
  if (n_seeds < 0 || n_events < 0) return KF_ERR_ARG;
  if (n_seeds == 0) return KF_OK;
  if (!hits || !hit_surface || !seed_hits || !seed_event || !state_out || !surf_out) return KF_ERR_ARG;
  FindArgs A;
  std::memset(&A, 0, sizeof(A));
  A.hits = reinterpret_cast<const float2*>(hits);
  A.hit_surface = hit_surface;
  A.seed_hits = seed_hits;
  A.seed_event = seed_event;
  A.n_seeds = n_seeds;
  A.n_events = n_events;
  A.lmax = 4;
  A.seed_state = state_out;
  A.seed_surf = surf_out;
  return launch_seed_states(G, M, A, reinterpret_cast<cudaStream_t>(stream));
}

int kf_mlp_forward(const float* params, const float* features, int n, float* logits, kf_stream_t stream) {
  if (n < 0 || (n > 0 && (!params || !features || !logits))) return KF_ERR_ARG;
  if (reinterpret_cast<size_t>(features) & 7) return KF_ERR_ARG;  // rows are read as float pairs
  return launch_mlp_forward(params, features, n, logits, reinterpret_cast<cudaStream_t>(stream));
}

int kf_mlp_finder_scores(const float* params, const float* features, int n, float* logits, void* workspace,
                         kf_stream_t stream) {
  if (n < 0 || !params || !workspace || (n > 0 && (!features || !logits))) return KF_ERR_ARG;
  if (reinterpret_cast<size_t>(workspace) & 15) return KF_ERR_ARG;  // fragments are 16-byte words
  return launch_mlp_finder_scores(params, features, n, logits, static_cast<uint4*>(workspace),
                                  reinterpret_cast<cudaStream_t>(stream)) == 0
             ? KF_OK
             : KF_ERR_CUDA;
}

int kf_mlp_loss_grad(const float* params, const float* features, const float* labels, int n, float* grad,
                     float* loss, kf_stream_t stream) {
  if (n < 0 || !params || !grad || !loss || (n > 0 && (!features || !labels))) return KF_ERR_ARG;
  if (reinterpret_cast<size_t>(features) & 7) return KF_ERR_ARG;  // rows are read as float pairs
  return launch_mlp_loss_grad(params, features, labels, n, grad, loss, reinterpret_cast<cudaStream_t>(stream));
}

int kf_mlp_adam(float* params, const float* grad, float* m, float* v, int step, float lr, float beta1, float beta2,
                float eps, kf_stream_t stream) {
  if (!params || !grad || !m || !v || step < 1 || !(lr > 0.f) || !(eps > 0.f)) return KF_ERR_ARG;
  return launch_mlp_adam(params, grad, m, v, step, lr, beta1, beta2, eps, reinterpret_cast<cudaStream_t>(stream));
}

// Allocation-free finding: the library's fixed scratch array replaces the caller's workspace.
int kf_find_tracks_static(const KfGeometry* geom, const KfHitIndex* index, const float* hits,
                          const int* hit_surface, const int* seed_hits, const int* seed_event, int n_seeds,
                          const KfFindParams* params, int* hits_out, int* nhits_out, float* chi2_out,
                          float* state_out, float* cov_out, int* status_out, kf_stream_t stream) {
  DevGeom G;
  DevMat M;
  FindPlan plan;
  FindArgs A;
  bool empty = false;
  if (params && params->adaptive_capacity != 0) return KF_ERR_ARG;  // the scratch holds no overflow list
  int rc = prepare_find(geom, index, hits, hit_surface, seed_hits, seed_event, n_seeds, params, hits_out, nhits_out,
                        chi2_out, state_out, cov_out, status_out, KF_STATIC_MAX_SEEDS, &G, &M, &plan, &A, &empty);
  if (rc != KF_OK) return rc;
  if (plan.ws_bytes > KF_STATIC_SCRATCH_BYTES) return KF_ERR_CAPACITY;
  if (empty) return KF_OK;
  void* scratch = nullptr;
  rc = static_scratch(&scratch);
  if (rc != KF_OK) return rc;
  return launch_find(G, M, A, plan, scratch, reinterpret_cast<cudaStream_t>(stream));
}

// ---- autotuners: time each configuration with CUDA events on the caller's stream ---------------


int kf_autotune_find(const KfGeometry* geom, const KfHitIndex* index, const float* hits, const int* hit_surface,
                     const int* seed_hits, const int* seed_event, int n_seeds, KfFindParams* params, int* hits_out,
                     int* nhits_out, float* chi2_out, float* state_out, float* cov_out, int* status_out,
                     void* workspace, size_t workspace_bytes, float* best_ms, kf_stream_t stream) {
  if (!params || !best_ms || n_seeds <= 0) return KF_ERR_ARG;
  const cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int need = std::max(params->k_max, params->mlp ? params->top_n : 0);
  static const int caps[] = {1, 2, 4, 6, 8, 16};
  int cap_opts[2] = {0, 0}, n_cap = 0;
  for (int c : caps)
    if (c >= need && n_cap < 2) cap_opts[n_cap++] = c;
  // With k_max > 4 adaptive capacities 2 and 4 are tried too, those that hold top_n with the
  // learned proposal (a configuration whose workspace does not fit the caller's fails and is
  // passed over).
  const bool learned = params->mlp && params->top_n > 0;
  int ad_opts[3] = {0, 0, 0}, n_ad = 1;
  if (params->k_max > 4)
    for (int a : {2, 4})
      if (!learned || params->top_n <= a) ad_opts[n_ad++] = a;
  KfFindParams best = *params;
  float best_t = -1.f;
  for (int ci2 = 0; ci2 < n_cap; ++ci2) {
    for (int blk = 64; blk <= 256; blk += 32) {
      for (int ai = 0; ai < n_ad; ++ai) {
        KfFindParams p = *params;
        p.block_threads = blk;
        p.k_capacity = cap_opts[ci2];
        p.blocks_per_sm = 0;
        p.adaptive_capacity = ad_opts[ai];
        const float t = time_config(st, [&]() {
          return kf_find_tracks(geom, index, hits, hit_surface, seed_hits, seed_event, n_seeds, &p, hits_out,
                                nhits_out, chi2_out, state_out, cov_out, status_out, workspace, workspace_bytes, stream);
        });
        if (t >= 0.f && (best_t < 0.f || t < best_t)) {
          best_t = t;
          best = p;
        }
      }
    }
  }
  if (best_t < 0.f) return KF_ERR_CUDA;
  *params = best;
  *best_ms = best_t;
  return KF_OK;
}

int kf_autotune_fit(const KfGeometry* geom, const float* hits, const int* hit_surface, const int* track_hits,
                    int n_tracks, int lmax, float* state_out, float* cov_out, float* chi2_out, int* ndof_out,
                    int* status_out, int* block_threads, float* best_ms, kf_stream_t stream) {
  if (!block_threads || !best_ms || n_tracks <= 0) return KF_ERR_ARG;
  const cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  float best_t = -1.f;
  int best_b = 0;
  for (int blk = 64; blk <= 256; blk += 32) {
    const float t = time_config(st, [&]() {
      return kf_fit_tracks(geom, hits, hit_surface, track_hits, n_tracks, lmax, state_out, cov_out, chi2_out, ndof_out,
                           status_out, blk, stream);
    });
    if (t >= 0.f && (best_t < 0.f || t < best_t)) {
      best_t = t;
      best_b = blk;
    }
  }
  if (best_t < 0.f) return KF_ERR_CUDA;
  *block_threads = best_b;
  *best_ms = best_t;
  return KF_OK;
}

size_t kf_dedup_workspace_size(int n_items, int refs_per_item, int n_hits) {
  if (n_items < 0 || refs_per_item < 1 || n_hits < 0) return 0;
  return dup_workspace_bytes(n_items, refs_per_item, n_hits);
}

int kf_clean_seeds(const KfGeometry* geom, const float* hits, const int* hit_surface, int n_hits, const int* seed_hits,
                   const int* seed_event, int n_seeds, float dphi, float dtheta, int* keep_out, void* workspace,
                   size_t workspace_bytes, kf_stream_t stream) {
  DevGeom G;
  const int rc = pack_geometry(geom, &G);
  if (rc != KF_OK) return rc;
  if (n_seeds < 0 || n_hits < 0 || !(dphi >= 0.f) || !(dtheta >= 0.f)) return KF_ERR_ARG;
  if (n_seeds == 0) return KF_OK;
  if (!hits || !hit_surface || !seed_hits || !seed_event || !keep_out || !workspace) return KF_ERR_ARG;
  if (workspace_bytes < dup_workspace_bytes(n_seeds, 3, n_hits) || (reinterpret_cast<size_t>(workspace) & 255))
    return KF_ERR_ARG;
  return launch_clean_seeds(G, reinterpret_cast<const float2*>(hits), hit_surface, seed_hits, seed_event, n_seeds,
                            n_hits, dphi, dtheta, keep_out, workspace, reinterpret_cast<cudaStream_t>(stream));
}

int kf_remove_duplicates(const int* track_hits, const int* nhits, const float* chi2, const float* state,
                         const int* track_event, int n_tracks, int lmax, int n_hits, float dphi, float dtheta,
                         int* keep_out, void* workspace, size_t workspace_bytes, kf_stream_t stream) {
  if (n_tracks < 0 || n_hits < 0 || lmax < 1 || lmax > KF_MAX_LMAX || !(dphi >= 0.f) || !(dtheta >= 0.f))
    return KF_ERR_ARG;
  if (n_tracks == 0) return KF_OK;
  if (!track_hits || !nhits || !chi2 || !state || !track_event || !keep_out || !workspace) return KF_ERR_ARG;
  if (static_cast<long long>(n_tracks) * lmax > 0x7fffffffLL) return KF_ERR_CAPACITY;
  if (workspace_bytes < dup_workspace_bytes(n_tracks, lmax, n_hits) || (reinterpret_cast<size_t>(workspace) & 255))
    return KF_ERR_ARG;
  return launch_remove_duplicates(track_hits, nhits, chi2, state, track_event, n_tracks, lmax, n_hits, dphi, dtheta,
                                  keep_out, workspace, reinterpret_cast<cudaStream_t>(stream));
}

int kf_fp32_fma_probe(float* sink, int blocks, int iters, long long* flops, kf_stream_t stream) {
  if (!sink || !flops || blocks <= 0 || iters <= 0) return KF_ERR_ARG;
  return launch_fma_peak(sink, blocks, iters, reinterpret_cast<cudaStream_t>(stream), flops);
}

int kf_math_probe(int fn, const float* a, const float* b, int n, float* o0, float* o1, float* o2, kf_stream_t stream) {
  if (fn < KF_PROBE_SINCOS || fn > KF_PROBE_HALF_ANGLE || n < 0) return KF_ERR_ARG;
  if (n == 0) return KF_OK;
  if (!a || !o0 || !o1 || !o2 || (fn == KF_PROBE_ATAN_SMALL && !b)) return KF_ERR_ARG;
  return launch_math_probe(fn, a, b, n, o0, o1, o2, reinterpret_cast<cudaStream_t>(stream));
}

int kf_wait_probe(int limit_us, long long* out, kf_stream_t stream) {
  if (limit_us < 1 || limit_us > 1000000 || !out) return KF_ERR_ARG;
  return launch_wait_probe(limit_us, out, reinterpret_cast<cudaStream_t>(stream));
}

const char* kf_status_string(int status) {
  switch (status) {
    case KF_OK: return "ok";
    case KF_ERR_ARG: return "invalid argument";
    case KF_ERR_CAPACITY: return "size above a compiled capacity";
    case KF_ERR_CUDA: return "CUDA launch error";
    case KF_ERR_TIMEOUT: return "bounded device wait ran out";
    default: return "unknown status";
  }
}

}  // extern "C"
