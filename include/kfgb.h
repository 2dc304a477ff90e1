/*
 * kfgb: Kalman-filter track fitting and combinatorial track finding on the GPU (sm_103a).
 *
 * C ABI over caller-owned device buffers. Every entry point is asynchronous on the given CUDA
 * stream, allocates nothing, synchronises nothing and returns a status code at launch time:
 *   KF_OK (0) launched; KF_ERR_ARG invalid argument (nothing launched); KF_ERR_CAPACITY a size
 *   above a compiled limit (nothing launched); KF_ERR_CUDA a CUDA launch error.
 * Conditions found on the device (propagation failures, capacity overflow inside a kernel) are
 * written to per-track status arrays and to an optional device status word (see each call); no
 * kernel traps or asserts. All float data are IEEE FP32.
 *
 * Method. The paper (arXiv:1906.02253, Sec. 1-2) adapts the traditional Kalman filter to track
 * fitting and to combinatorial track finding: tracks are propagated layer to layer (Sec. 3.1) in
 * a constant 3.8 T field (Sec. 4), multiple scattering from the detector material enters the
 * prediction (Sec. 3.1), hits are selected through per-layer search windows and candidates are
 * scored and kept per seed (Sec. 4), and seeds are processed in parallel without marking used
 * hits (Sec. 3.2). The formulas are the textbook ones; the state is (x, y, z, kappa = q/pT, phi,
 * theta) in cm, 1/GeV and rad, with a 6x6 covariance stored as its upper triangle, row-major:
 * element (i, j), i <= j, at index i*(11-i)/2 + j ("packed 21").
 */
#ifndef KFGB_H
#define KFGB_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* kf_stream_t; /* a cudaStream_t; NULL = legacy default stream */

#define KF_OK 0
#define KF_ERR_ARG (-1)
#define KF_ERR_CAPACITY (-2)
#define KF_ERR_CUDA (-3)
#define KF_ERR_TIMEOUT (-4)

#define KF_BARREL 0
#define KF_DISK 1

#define KF_MAX_SURF 64       /* surfaces per geometry */
#define KF_MAX_LMAX 31       /* entries per track hit list */
#define KF_MAX_K 16          /* candidates kept per seed */
#define KF_MAX_SLAB_HITS 32768 /* hits per (event, surface) in the hit index */

/* One detection surface (the paper's per-layer description, Sec. 3.1, reduced to what the
 * fit and the search use). Barrel: cylinder of radius r_or_z, hits (phi, z) with z in [lo, hi].
 * Disk: plane z = r_or_z, hits (phi, r) with r in [lo, hi]. x_over_x0 is the material thickness
 * at normal incidence in radiation lengths (0: no scattering). n_phi x n_2nd index bins. */
typedef struct {
  int type;
  float r_or_z, lo, hi;
  float x_over_x0;
  int n_phi, n_2nd;
} KfSurface;

/* Geometry and resolution. surf is a HOST array of n_surf entries, read during the call only.
 * prior: standard deviations of the seed prior at the first hit: transverse position (cm),
 * second coordinate z or r (cm), kappa (1/GeV), phi (rad), theta (rad). */
typedef struct {
  float bz;
  int n_surf;
  const KfSurface* surf;
  float sigma_rphi, sigma_2nd;
  float prior[5];
  /* Material and energy loss (Sec. 3.1: material tables indexed in r-z, energy loss). ms_off: 1
   * turns multiple scattering off. material: NULL (each surface's x_over_x0 everywhere) or a host
   * array [n_surf][KF_MAT_NODES] of x/X0 at points spread evenly over the surface's extent (z on a
   * barrel, r on a disk), interpolated linearly at the crossing and clamped at the ends. eloss:
   * mean ionisation loss in GeV per unit of x/X0 crossed (0: none), taken along the path through
   * the layer, |p| -> p' with E' = E - eloss x/X0 / |cos a| for a particle of mass `mass` GeV,
   * direction kept; in the covariance kappa's row and column scale by (p/p')^3 E'/E. Zero-filled
   * fields keep the plain behaviour. */
  int ms_off;
  const float* material;
  float eloss, mass;
  /* Parametrised solenoid field (Sec. 3.1: constant or parametrised magnetic field): Bz(r, z) =
   * bz (1 + field_z2 z^2 + field_r2 r^2), cm^-2, radial component neglected. Each step between
   * surfaces is a helix in the field at the midpoint of its chord p + (s/2)(cos phi, sin phi,
   * cot theta), s the path in the field at the step's start (which also decides the next
   * surface); the field's gradient is not propagated into the covariance; a seed's kappa uses
   * the field at its first hit. Both zero (zero-filled): uniform field bz. Non-finite:
   * KF_ERR_ARG. */
  float field_z2, field_r2;
} KfGeometry;
#define KF_MAT_NODES 8

/* Hit index: per (event, surface) slab, hits sorted by bin (phi-bin * n_2nd + second-bin) and,
 * within a bin, by phi sub-bin and then ascending hit id. The phi sub-bin refines the phi bin
 * into KF_PHI_SUB equal parts: fine = clamp(floor((phi + pi_f) * (float)(n_phi * KF_PHI_SUB /
 * 2pi)), 0, n_phi * KF_PHI_SUB - 1) by the same FP32 rule as the bins, sub = clamp(fine -
 * phi-bin * KF_PHI_SUB, 0, KF_PHI_SUB - 1). All pointers are caller-owned device memory:
 *   bin_off     int [n_events * n_surf][n_bins + 1]: absolute position in sorted_* of the first
 *               hit of each bin; entry n_bins (and every bin beyond the surface's own count) is
 *               the slab end. n_bins = max over surfaces of n_phi * n_2nd.
 *   sorted_hits float [n_hits][2] and sorted_ids int [n_hits]: same slab ranges as the input.
 *   sorted_rec  float [n_hits][4], 16-byte aligned: the search record of each sorted hit,
 *               (cos phi, sin phi, second coordinate, hit id as int32 bits), so that a window scan
 *               reads one 16-byte record per hit. Optional for kf_build_hit_index (NULL: not
 *               written); required by kf_find_tracks.
 *   sub_off     uint16 [n_events * n_surf][n_bins][KF_PHI_SUB]: entry j of a bin = number of the
 *               bin's hits with sub-bin <= j (entry KF_PHI_SUB - 1 = the bin's count; zero for
 *               bins beyond the surface's own count). Optional for kf_build_hit_index (NULL: not
 *               written); required by kf_find_tracks, whose windows scan only the sub-bins their
 *               phi range touches. */
#define KF_PHI_SUB 8
typedef struct {
  int n_events;
  int n_bins;
  int* bin_off;
  float* sorted_hits;
  int* sorted_ids;
  float* sorted_rec;
  unsigned short* sub_off;
} KfHitIndex;

/* Steering of the finder by tracking region (Sec. 3.1: five regions in eta, each with the layers
 * its track finding traverses). Regions: 0 barrel, 1 +z transition, 2 -z transition, 3 +z endcap,
 * 4 -z endcap. A seed's region comes from its third hit, (z, rho) = (z, R) on a barrel and (Z, r)
 * on a disk: barrel if |z| <= c_barrel * rho, else transition if |z| <= c_endcap * rho, else
 * endcap; +z side when z > 0 (each product one FP32 multiplication, rounded to nearest). Its
 * candidates step through surf[region][0 .. n[region]-1], starting after the position of the
 * third hit's surface in that list (from the first entry if it is absent): at each step a
 * candidate moves to the next listed surface it reaches within the surface's extent (barrel: the
 * z extent; disk: the r extent, within half a turn), passing over surfaces it cannot reach; at the
 * end of its list it stops. Host memory, read during the call. */
#define KF_N_REGIONS 5
typedef struct {
  float c_barrel, c_endcap;
  int n[KF_N_REGIONS];
  signed char surf[KF_N_REGIONS][KF_MAX_SURF];
} KfSteering;

/* Finder settings. chi2_cut: hits with predicted chi2 below it make children; k_max: candidates
 * kept per seed (<= KF_MAX_K); max_miss: surfaces a candidate may cross without a hit; lmax:
 * length of each output hit list (3 seed hits + at most lmax-3 steps; 4 <= lmax <= KF_MAX_LMAX);
 * block_threads: threads per block (0 = the size keeping most warps resident; a multiple of 32,
 * <= 256; with the learned proposal <= 192, else KF_ERR_CAPACITY);
 * blocks_per_sm: resident blocks per SM for the persistent grid (0 = occupancy maximum). */
typedef struct {
  float chi2_cut;
  int k_max;
  int max_miss;
  int lmax;
  int block_threads;
  int blocks_per_sm;
  /* Learned hit proposal (not in the paper): NULL for plain finding, else a device buffer of
   * KF_MLP_BUFFER floats (see kf_mlp_forward), 4-byte aligned, unchanged while the call runs. With
   * top_n > 0, when more than top_n hits of a candidate's window pass the chi2 cut, only the top_n
   * with the highest network score (ties: lower hit id) make children. The finder evaluates the
   * network on the tensor cores, 8 pairs at a time per warp, with every operand split into two
   * fp16 parts, which keeps all but 3 2^-22 of each product (inputs and hidden units must stay
   * within the fp16 range, as they do for standardised features and a trained network); see
   * kf_mlp_finder_scores. */
  const float* mlp;
  int top_n;
  /* Candidate capacity of the compiled kernel (one of 1, 2, 4, 6, 8, 16, >= k_max and top_n);
   * 0 picks the smallest that fits. A larger capacity gives the same results. */
  int k_capacity;
  /* Region steering (see KfSteering), or NULL for the geometric rule: the next surface is the
   * nearer of the next barrel layer beyond the candidate's radius (crossed within its z extent)
   * and the next disk beyond |z| in the direction of motion (crossed within its r extent, within
   * half a turn). */
  const KfSteering* steering;
  /* Optional device int [n_seeds] (kf_clean_seeds' keep_out): seeds with 0 are not processed;
   * their outputs are empty (no hits, NaN state) with status 2. NULL: every seed. */
  const int* seed_keep;
  /* Learned proposal with a score margin (> 0; 0 keeps the top_n rule above): of a window with two
   * or more passing hits, only those among its top_n by score that score within score_margin (in
   * logit units) of its best make children, the best always. A window whose best hit stands out then
   * keeps one child. */
  float score_margin;
  /* Adaptive capacity (0 = off, the default): a first pass runs every seed with adaptive_capacity
   * candidate slots (rounded up to a compiled capacity), more seeds per warp, and finishes the
   * seeds whose children never outnumber those slots: keeping all of a step's children is what
   * k_max does then, so their results are those of the single pass. The other seeds are listed in
   * the workspace and found again, from their seed state, by a second pass at the full capacity.
   * Ignored when no smaller compiled capacity exists or, with the learned proposal, when top_n
   * exceeds the first pass's slots; KF_ERR_ARG outside [0, KF_MAX_K]. Pays where most seeds carry
   * few candidates (barrel + disk events with noise; the learned proposal's pruning). */
  int adaptive_capacity;
  /* Learned proposal ranking the window before the chi2 test (0 = off; 1 = on): the window is the
   * bounding box of the chi2 ellipse, |r_i| <= sqrt(chi2_cut S_ii) for both residuals; when it
   * holds more than top_n hits, only its top_n by score (ties: lower hit id) face the chi2 cut, else
   * every passing hit makes a child. With a score margin the box is ranked when it holds two or
   * more hits, and only those of its top_n within the margin of its best score face the cut.
   * Reading of "ranks and prunes each candidate's hit window before the exact chi2 and update" that
   * scores failing hits too; with window_ranking = 0 the rules apply to the passing hits. */
  int window_ranking;
} KfFindParams;

/* Build the hit index (the binned hit structure behind the per-layer search windows, Sec. 3.1,
 * and the hit-data reuse of Sec. 3.2).
 *   hits          device float [n_hits][2]: (phi, z) on barrels, (phi, r) on disks; phi in
 *                 [-pi, pi]. Hits of one event are contiguous and grouped by surface.
 *   slab_offsets  device int [n_events * n_surf + 1]: first hit id of slab (event e, surface s)
 *                 at index e * n_surf + s; non-decreasing; the last entry is n_hits.
 *   max_slab_hits host int: an upper bound of the largest slab (sets shared memory); must be
 *                 <= KF_MAX_SLAB_HITS, else KF_ERR_CAPACITY.
 *   index         host struct whose device arrays receive the result (index->n_events and
 *                 index->n_bins must match the geometry; kf_index_bins gives n_bins).
 *   d_status      optional device int, OR-ed with 1 if a slab exceeded max_slab_hits (its
 *                 bins are then left empty).
 * Bins follow the FP32 rule: phi-bin = clamp(floor((phi + pi_f) * sphi), 0, n_phi - 1) with
 * pi_f = (float)pi and sphi = (float)(n_phi / (2 pi)); second-bin = clamp(floor((v - lo) * s2),
 * 0, n_2nd - 1) with s2 = (float)(n_2nd / ((double)hi - (double)lo)); each FP32 operation rounds
 * to nearest on its own (no fused multiply-add); NaN goes to bin 0. */
int kf_build_hit_index(const KfGeometry* geom, const float* hits, const int* slab_offsets, int n_events,
                       int max_slab_hits, const KfHitIndex* index, int* d_status, kf_stream_t stream);

/* Bins per slab of the index for this geometry (max n_phi * n_2nd), or KF_ERR_ARG. */
int kf_index_bins(const KfGeometry* geom);

/* Fit tracks over known hit sequences (Kalman-filter track fitting, Sec. 2).
 *   hits, hit_surface  device float [n_hits][2] and int [n_hits] (surface of each hit).
 *   track_hits         device int [lmax][n_tracks] (structure of arrays: entry k of track t at
 *                      k * n_tracks + t): hit ids in path order; -1 entries are skipped (misses);
 *                      the first three must be hits, they seed the fit.
 * The seed state comes from the circle through the first three hits (transverse plane) and the
 * line through the first and third in (arc length, z), with the prior of the geometry on the
 * first hit's surface; the filter updates with hit 1, then propagates and updates through the
 * rest. Outputs (device, caller-owned), at the last hit:
 *   state_out float [6][n_tracks], cov_out float [21][n_tracks] (packed 21), chi2_out float
 *   [n_tracks] (sum of predicted chi2), ndof_out int [n_tracks] (2 * hits - 5), status_out int
 *   [n_tracks]: 0 ok, 1 seed failed, 2 a surface was not reached, 3 fewer than three seed hits.
 * The grid is persistent (a multiple of the SM count, each thread striding over tracks).
 * block_threads: 0 for the default (128), else a multiple of 32 up to 256. */
int kf_fit_tracks(const KfGeometry* geom, const float* hits, const int* hit_surface, const int* track_hits,
                  int n_tracks, int lmax, float* state_out, float* cov_out, float* chi2_out, int* ndof_out,
                  int* status_out, int block_threads, kf_stream_t stream);

/* Device workspace (bytes) kf_find_tracks needs for these parameters on the current device. */
size_t kf_find_workspace_size(int n_seeds, const KfFindParams* params);

/* Combinatorial track finding (Sec. 2 and Sec. 4): from each seed's three hits, fit the seed,
 * then step outward surface by surface. The next surface is the nearer of the next barrel layer
 * beyond the candidate's radius (if crossed inside its z extent) and the next disk beyond |z| in
 * the direction of motion (if crossed inside its r extent). At each step every candidate is
 * propagated (covariance with scattering noise), every hit in its search window with chi2 below
 * the cut becomes a child (updated); a candidate with no such hit becomes one miss child while
 * it has misses left, else it stops and is carried unchanged. The k_max best of all children and
 * carried candidates of the seed survive, ordered by more hits, then lower total chi2, then
 * parent rank, then child kind (hit, miss, carried), then hit id. Seeds run in parallel with no
 * hit marking across seeds (Sec. 3.2).
 *   hits, hit_surface  as for the fit (original hit ids); index built by kf_build_hit_index.
 *   seed_hits          device int [3][n_seeds] (structure of arrays), seed_event int [n_seeds]. A
 *                      seed with a negative hit id, a hit on no surface of the geometry or an event
 *                      outside [0, index->n_events) fails (status 1); hit ids must be below the
 *                      number of hits.
 *   workspace          device memory of kf_find_workspace_size bytes, 256-byte aligned, owned
 *                      by this call until its kernels finish: calls that can run at the same time
 *                      (other streams, other host threads) need workspaces of their own (sharing
 *                      one gives wrong results; the kernels keep their accesses in bounds).
 * Outputs (device): hits_out int [lmax][n_seeds] (best candidate's hit ids in path order, -1 for
 * a miss or no further step), nhits_out int, chi2_out float, state_out float [6][n_seeds],
 * cov_out float [21][n_seeds], status_out int (0 ok, 1 seed failed, 2 seed removed by seed_keep). */
int kf_find_tracks(const KfGeometry* geom, const KfHitIndex* index, const float* hits, const int* hit_surface,
                   const int* seed_hits, const int* seed_event, int n_seeds, const KfFindParams* params,
                   int* hits_out, int* nhits_out, float* chi2_out, float* state_out, float* cov_out,
                   int* status_out, void* workspace, size_t workspace_bytes, kf_stream_t stream);

/* Seed states alone (the first stage of kf_find_tracks; Sec. 2: each seed's track state from its
 * three hits). Per seed: the circle through the three hits and the line through hits 1 and 3 give
 * the state at hit 1 with the geometry's prior on hit 1's surface; the filter updates with hit 1,
 * then propagates and updates through hits 2 and 3, as the fit does.
 *   seed_hits, seed_event  as for kf_find_tracks; n_events: the batch's event count (a seed naming
 *                          another event fails).
 *   state_out  device float [28][n_seeds] (structure of arrays): p[6], packed C[21] at hit 3 and
 *              chi2 (sum of the three predicted chi2); chi2 = -1 marks a seed that failed (invalid
 *              hit id, event or surface, collinear hits, no crossing).
 *   surf_out   device int [n_seeds]: surface of hit 3 (set for seeds that did not fail).
 * Asynchronous on the stream; KF_ERR_ARG for a bad geometry, negative counts or null pointers. */
int kf_seed_states(const KfGeometry* geom, const float* hits, const int* hit_surface, const int* seed_hits,
                   const int* seed_event, int n_seeds, int n_events, float* state_out, int* surf_out,
                   kf_stream_t stream);

/* Seed cleaning and duplicate-track removal. Seeds and tracks of one event that share a hit are
 * compared through an inverted index hit -> items built in the workspace; the decisions depend on
 * no processing order.
 * kf_clean_seeds (Sec. 3.2: several seeds of one particle, e.g. from overlapping modules, are
 * removed before finding, by hit identity and seed direction): seed j is removed (keep_out[j] =
 * 0, else 1) when a seed i < j of the same event shares a hit with it and their directions at the
 * first hit agree, |d phi| < dphi and |d theta| < dtheta (the direction of the circle through the
 * three hits and of the line through hits 1 and 3, as the finder's seed state; a seed whose hits
 * give no state is kept).
 * kf_remove_duplicates (Sec. 4: duplicate tracks from several seeds per particle): track j is
 * removed when a better track i of the same event (more hits, then lower chi2, then lower index)
 * whose final direction agrees (state[4], state[5]: |d phi| < dphi, |d theta| < dtheta) holds
 * more than half of j's hits.
 *   seed_hits  device int [3][n_seeds]; track_hits device int [lmax][n_tracks] (-1: none), nhits,
 *              chi2, state [6][n_tracks] (the finder's outputs); *_event device int; hit ids < n_hits.
 *   workspace  device memory of kf_dedup_workspace_size(n_items, 3 or lmax, n_hits) bytes, 256-byte
 *              aligned (0 from the size function for invalid sizes).
 * Asynchronous on the stream. Returns KF_OK (nothing launched for zero items), KF_ERR_ARG (negative
 * counts, negative or NaN cuts, lmax outside 1..KF_MAX_LMAX, a null pointer, a small or misaligned
 * workspace, an invalid geometry), KF_ERR_CAPACITY (n_tracks * lmax above 2^31 - 1) or
 * KF_ERR_CUDA. */
size_t kf_dedup_workspace_size(int n_items, int refs_per_item, int n_hits);
int kf_clean_seeds(const KfGeometry* geom, const float* hits, const int* hit_surface, int n_hits, const int* seed_hits,
                   const int* seed_event, int n_seeds, float dphi, float dtheta, int* keep_out, void* workspace,
                   size_t workspace_bytes, kf_stream_t stream);
int kf_remove_duplicates(const int* track_hits, const int* nhits, const float* chi2, const float* state,
                         const int* track_event, int n_tracks, int lmax, int n_hits, float dphi, float dtheta,
                         int* keep_out, void* workspace, size_t workspace_bytes, kf_stream_t stream);

/* Learned hit proposal network (not in the paper): MLP 14 -> 64 -> 64 -> 1 with ReLU, scoring a
 * (predicted candidate, hit) pair from 14 features: the predicted state (x, y, z, kappa, phi,
 * theta), log(C_ii + 1e-12) of the six covariance diagonal terms (exact value on a disk, where the
 * z variance is zero after the projection onto the surface, so log(1e-12) whatever the rounding
 * residue; x and y floored at log(1e-12), as their rounding residue near an axis can be
 * negative), and the two residuals divided by the square roots of the
 * innovation variances. Parameter buffer, FP32, KF_MLP_BUFFER floats:
 * W1[64][14], b1[64], W2[64][64], b2[64], W3[64], b3 (KF_MLP_PARAMS weights), then the feature
 * normaliser mean[14], sd[14] (x -> (x - mean) / sd before the first layer). All pointers are
 * device memory. */
#define KF_MLP_IN 14
#define KF_MLP_HID 64
#define KF_MLP_PARAMS 5185
#define KF_MLP_BUFFER 5213

/* Logits of n feature rows (features float [n][14], raw, standardised inside; 8-byte aligned, else
 * KF_ERR_ARG). The two layers run on the tensor cores (tcgen05) with FP32-faithful products: each
 * operand is split into three bf16 parts, hi = bf16(v), mid = bf16(v - hi), lo = bf16(v - hi - mid),
 * and the six products hi*hi, hi*mid, mid*hi, hi*lo, lo*hi, mid*mid are accumulated in FP32. A tile
 * whose tensor-core wait gives up (one second) gets NaN logits. */
int kf_mlp_forward(const float* params, const float* features, int n, float* logits, kf_stream_t stream);

/* Logits of n feature rows evaluated exactly as the finder scores its (candidate, hit) pairs
 * (measurement only, not part of the path): the features standardised in FP32, the hidden layers
 * as warp-level tensor-core MMAs over 8 rows at a time with every operand split into two fp16
 * parts (hi = f16(v), lo = f16(2^11 (v - hi))) and FP32 accumulation, the output layer in FP32:
 * each product keeps all but 3 2^-22 of itself, and a logit lies within 2^-18 of the network
 * evaluated on the absolute values of its weights and inputs (in practice about 1e-6 of logits of
 * order 1). features float [n][14] (raw), logits float [n]; workspace: device memory of
 * KF_MLP_FRAG_BYTES bytes, 16-byte aligned, which receives the weights' tensor-core operands.
 * KF_ERR_ARG for n < 0, a null pointer or a misaligned workspace. */
#define KF_MLP_FRAG_BYTES 20480
int kf_mlp_finder_scores(const float* params, const float* features, int n, float* logits, void* workspace,
                         kf_stream_t stream);

/* Mean binary cross-entropy with logits over n samples (labels 0 or 1) and its gradient with
 * respect to the KF_MLP_PARAMS weights: grad float [KF_MLP_PARAMS] and loss float [1] are
 * overwritten. Features as for kf_mlp_forward (8-byte aligned). The forward layers, the
 * back-propagation through W2 and the weight gradients of W1, b1, W2, b2 run on the tensor cores
 * with the same FP32-faithful split; a tensor-core wait that gives up makes the loss NaN. */
int kf_mlp_loss_grad(const float* params, const float* features, const float* labels, int n, float* grad,
                     float* loss, kf_stream_t stream);

/* One Adam step (Kingma and Ba) on the weights of params with gradient grad and moments m, v
 * (float [KF_MLP_PARAMS] each, zero before step 1); step counts from 1. */
int kf_mlp_adam(float* params, const float* grad, float* m, float* v, int step, float lr, float beta1, float beta2,
                float eps, kf_stream_t stream);

/* Allocation-free track finding. The paper has no counterpart: this entry point exists for
 * callers that cannot allocate device memory while they reconstruct events, for example an
 * online trigger process that reserves all of its GPU memory at start-up and forbids any
 * allocation during event processing (to keep latency bounded and memory unfragmented), or a
 * plug-in running inside a host framework that owns the device memory pool. Such callers cannot
 * provide the workspace kf_find_tracks takes.
 *
 * Same arguments and results as kf_find_tracks, without workspace. The scratch (work counter, seed
 * states and, with the learned proposal, the network's weights as tensor-core operands) is a fixed
 * array inside
 * the library of KF_STATIC_SCRATCH_BYTES (about 7.3 MiB),
 * held on every GPU that loads the library until the process exits. At most KF_STATIC_MAX_SEEDS
 * seeds per call: more returns KF_ERR_CAPACITY and launches nothing (split the seeds into
 * chunks). Adaptive capacity needs workspace for its overflow list: params->adaptive_capacity must
 * be 0 here (else KF_ERR_ARG). The call allocates nothing and calls no allocating routine.
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress, with
 * that device current); make that first call before any stream capture. Every call uses the same
 * array and leaves its contents behind: calls whose kernels can overlap on the GPU (several
 * streams, several host threads) race and corrupt each other's results, so serialise them. */
#define KF_STATIC_MAX_SEEDS 65536
#define KF_STATIC_SCRATCH_BYTES 7622912
int kf_find_tracks_static(const KfGeometry* geom, const KfHitIndex* index, const float* hits,
                          const int* hit_surface, const int* seed_hits, const int* seed_event, int n_seeds,
                          const KfFindParams* params, int* hits_out, int* nhits_out, float* chi2_out,
                          float* state_out, float* cov_out, int* status_out, kf_stream_t stream);

/* Autotuner for the persistent finder (not in the paper): runs kf_find_tracks on the given seeds
 * (a calibration subset of the workload) for every block size 64..256 (step 32) and for the
 * smallest and the next compiled candidate capacity, and for k_max > 4 with adaptive capacity 2,
 * 4 (those holding top_n with the learned proposal) or none, times each run with CUDA events (the
 * stream is synchronised: do not call it during a stream capture), and writes the fastest block
 * size, capacity and adaptive capacity into params->block_threads, params->k_capacity and
 * params->adaptive_capacity; *best_ms receives its time. Every configuration gives the same results. Outputs as for kf_find_tracks; a
 * configuration whose workspace is larger than workspace_bytes is passed over (size the workspace
 * with an adaptive capacity set, which adds the same overflow list for 2 and 4, to let those
 * compete). */
int kf_autotune_find(const KfGeometry* geom, const KfHitIndex* index, const float* hits, const int* hit_surface,
                     const int* seed_hits, const int* seed_event, int n_seeds, KfFindParams* params, int* hits_out,
                     int* nhits_out, float* chi2_out, float* state_out, float* cov_out, int* status_out,
                     void* workspace, size_t workspace_bytes, float* best_ms, kf_stream_t stream);

/* Autotuner for the fit: times kf_fit_tracks for block sizes 64..256 (step 32) on the given tracks
 * and writes the fastest to *block_threads (synchronises the stream). */
int kf_autotune_fit(const KfGeometry* geom, const float* hits, const int* hit_surface, const int* track_hits,
                    int n_tracks, int lmax, float* state_out, float* cov_out, float* chi2_out, int* ndof_out,
                    int* status_out, int* block_threads, float* best_ms, kf_stream_t stream);

/* FP32 throughput probe (measurement only, not part of the path): launches `blocks` blocks of 256
 * threads, each running eight independent fused multiply-add chains for iters x 16 steps, on the
 * stream, and stores the launch's flop count (2 per FMA) in *flops. The caller times the launch
 * (CUDA events) to get the FP32 rate the ALU-bound kernels are compared with. sink: device float
 * [blocks] (practically never written). KF_ERR_ARG for non-positive sizes or null pointers. */
int kf_fp32_fma_probe(float* sink, int blocks, int iters, long long* flops, kf_stream_t stream);

/* Accuracy probe of the path's hand-written trigonometry (measurement only, not part of the path;
 * the same code and compiler flags as the finder and the fit). For i < n (device arrays):
 *   fn = KF_PROBE_SINCOS      o0 = sin a[i], o1 = cos a[i] (Cody-Waite reduction, Taylor series;
 *                             for |a| <= 1e5, else NaN);
 *   fn = KF_PROBE_ATAN_SMALL  o0 = atan(a[i] / b[i]) by its series, valid for b > 0, |a| < 0.05 b;
 *   fn = KF_PROBE_HALF_ANGLE  o0 = sin(h)/h, o1 = sin h, o2 = cos h for h = a[i] / 2 (the helix
 *                             step functions: series below |h| = 0.1, else the sincos above).
 * b may be NULL except for KF_PROBE_ATAN_SMALL; o1 and o2 receive 0 where unused. KF_ERR_ARG for
 * an unknown fn, n < 0 or a null pointer. */
#define KF_PROBE_SINCOS 0
#define KF_PROBE_ATAN_SMALL 1
#define KF_PROBE_HALF_ANGLE 2
int kf_math_probe(int fn, const float* a, const float* b, int n, float* o0, float* o1, float* o2, kf_stream_t stream);

/* Probe of the bounded wait that the tensor-core kernels use for MMA completion (measurement only,
 * not part of the path): one warp waits limit_us microseconds on a shared-memory mbarrier that
 * receives no arrival, then, after the barrier's one expected arrival, waits on it again. out:
 * device long long [3] = (1 if the first wait completed, 1 if the second completed, the first
 * wait's duration in ns); expected (0, 1, about limit_us * 1000). KF_ERR_ARG for limit_us outside
 * [1, 1000000] or a null pointer. */
int kf_wait_probe(int limit_us, long long* out, kf_stream_t stream);

/* Human-readable name of a status code. */
const char* kf_status_string(int status);

#ifdef __cplusplus
}
#endif
#endif /* KFGB_H */
