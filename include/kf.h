/*
 * kf.h - C ABI of the GB300 batched Kalman-filter track finder and fitter.
 *
 * The library implements the data-parallel core of the vectorized Kalman
 * filter tracking of Cerati et al., "Speeding up Particle Track
 * Reconstruction in the CMS Detector using a Vectorized and Parallelized
 * Kalman Filter Algorithm" (arXiv:1906.11744):
 *   - load hits and seeds (Sec. 3: the input conversion step of the build);
 *   - find tracks: combinatorial Kalman-filter building with per-seed
 *     candidate ranking (Sec. 2; candidate scores, Sec. 4.3);
 *   - seed cleaning before finding and duplicate removal after it: the two
 *     steps of duplicate handling on pT, eta, phi and shared hits (Sec. 4.2);
 *   - fit tracks: the Kalman re-fit of the built tracks (Sec. 5, "fitting");
 *   - the gradient of the summed fit chi2 with respect to layer alignment
 *     offsets, hit positions and seed parameters (adjoint of the fit).
 *
 * Track state p = (x, y, z, q/pT, phi, theta) in cm, GeV and rad; the
 * symmetric 6x6 covariance is stored as its 21-element upper triangle,
 * row-major: (0,0) (0,1) ... (0,5) (1,1) ... (1,5) (2,2) ... (5,5).
 * Structure-of-arrays buffers are [component][n] with n the number of seeds.
 *
 * Conventions for every call:
 *   - Return value: KF_OK (0) or a negative KF_ERR_* code; kf_last_error()
 *     gives a message.  No C++ exception crosses this boundary.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls are
 *     asynchronous on that stream unless stated otherwise.
 *   - `device_ptrs` = 1: the array arguments are device pointers read (or
 *     written) in stream order; 0: they are host pointers, copied inside the
 *     call (host-to-device before, device-to-host after; the call then
 *     synchronizes the stream before returning).
 *   - Input buffers stay owned by the caller; the context owns its device
 *     buffers, sized at load time (loads that grow a buffer allocate; later
 *     loads of equal or smaller size do not).
 *   - One context per host thread at a time.  Contexts are independent.
 *   - Errors raised inside kernels (capacity overflow) set a status word on
 *     the device; they are reported by the next call that synchronizes
 *     (kf_get_*, kf_sync).
 */
#ifndef KF_H_
#define KF_H_

#ifdef __cplusplus
extern "C" {
#endif

#define KF_OK 0
#define KF_ERR_ARG (-1)      /* invalid argument */
#define KF_ERR_CUDA (-2)     /* a CUDA runtime call failed */
#define KF_ERR_CAPACITY (-3) /* a size exceeds a documented limit */
#define KF_ERR_TIMEOUT (-4)  /* a bounded device-side loop gave up */
#define KF_ERR_STATE (-5)    /* calls made out of order */

#define KF_MAX_LAYERS 32       /* barrel layers */
#define KF_MAX_DISKS 16        /* endcap disks per side */
#define KF_MAX_CANDS 16        /* candidates kept per seed */
#define KF_MAX_EVENT_HITS (1 << 21) /* hits per event (21-bit hit index in ranking keys) */
#define KF_SEED_MAX_DETA 1.0f       /* largest eta window of seed cleaning */

/* Fit sources for kf_fit_tracks. */
#define KF_FIT_FOUND 0 /* hit lists produced by kf_find_tracks (kept tracks only after dedup) */
#define KF_FIT_GIVEN 1 /* caller hit lists */

/* Status values of kf_get_fit's status array. */
#define KF_FIT_OK 0
#define KF_FIT_SKIPPED 1   /* track removed as duplicate, not fitted */
#define KF_FIT_NO_CROSS (-1) /* propagation found no crossing of a hit's layer */
#define KF_FIT_FAR_SIDE (-2) /* a hit lies on the far half of the cylinder */

typedef struct kf_ctx kf_ctx;

/* Geometry (Sec. 3): concentric barrel cylinders in an axial field, uniform
 * or parameterized. */
typedef struct {
  int n_layers;                 /* 1..KF_MAX_LAYERS, radii increasing */
  float radius[KF_MAX_LAYERS];  /* cm */
  float x0[KF_MAX_LAYERS];      /* thickness in radiation lengths at normal incidence */
  float z_max;                  /* half-length of every layer, cm */
  float bz;                     /* field, tesla (0 = straight tracks) */
  float sigma_rphi;             /* hit resolution along r-phi, cm */
  float sigma_z;                /* hit resolution along z, cm */
  /* Mean ionization energy loss of each layer at normal incidence for
   * beta -> 1, GeV (>= 0; 0 = none).  Sec. 3: the material description also
   * serves energy loss.  Applied after each layer's scattering: dE = e f /
   * beta^2 with f = 1/|sin(theta) cos(phi - phi_p)| the scattering's path
   * factor (phi_p the position angle) and beta from the pion mass; dE is at
   * most (E - m)/2; q/pT is scaled by p/p' and the covariance carried through
   * the Jacobian of that map.  Straggling is not modelled. */
  float eloss[KF_MAX_LAYERS];
  /* Parameterized field (Sec. 3: the field may be constant or parameterized):
   * Bz(r, z) = bz (1 + field_cz z^2 + field_cr r^2), r^2 = x^2 + y^2, in cm^-2
   * (0, 0 = uniform).  Each propagation is a helix in the field at its starting
   * point; the covariance is carried by the Jacobian of that helix, and the
   * adjoint also differentiates the field's dependence on the starting point.
   * 1 + field_cz z^2 + field_cr r^2 must lie in [0.2, 5] for |z| <= z_max and
   * r <= the outermost radius (KF_ERR_ARG otherwise).  Duplicate kinematics
   * (pT, eta, phi0 cuts) use bz. */
  float field_cz;
  float field_cr;
  /* Endcap disks (Sec. 2: barrel layers and endcap disks, each event split
   * into eta regions).  n_disks planes per side at z = +-disk_z[k] (0 <
   * disk_z[0] < disk_z[1] < ...; a forward plan searches the barrel layers
   * before the disks, the order of a track's crossings when the disks lie
   * beyond the barrel's ends, |z| > z_max), covering disk_rmin <= r <=
   * disk_rmax, each disk_x0 radiation lengths thick with mean ionization loss
   * disk_eloss at normal incidence (GeV, >= 0).  Surfaces: barrel layers
   * 0..n_layers-1, the +z disks n_layers..n_layers+n_disks-1, then the -z
   * disks; a hit's layer index names its surface (n_surfaces = n_layers +
   * 2 n_disks).  On a disk: the measurement is (r-phi, r) with resolutions
   * sigma_rphi and sigma_r; propagation is the helix to the plane (transverse
   * arc s = (z_d - z) tan(theta) > 0, less than half a turn, in the field at
   * the starting point); scattering and energy loss take the path factor
   * 1/|cos(theta)|; hits carry no alignment.  Finding: a seed whose prior has
   * |eta| >= eta_barrel (a transition or endcap region) searches the barrel
   * layers after its seed and then the disks of its side in order of |z|;
   * along such a plan a surface that a candidate does not cross within its
   * bounds is passed (no hole, the candidate goes on).  Other seeds search
   * the barrel layers only, as without disks.  Seed hits lie on barrel
   * layers.  n_disks = 0: a barrel detector (the fields below are unused). */
  int n_disks;  /* 0..KF_MAX_DISKS */
  float disk_z[KF_MAX_DISKS];
  float disk_rmin, disk_rmax;  /* cm, 0 < disk_rmin < disk_rmax */
  float disk_x0;               /* radiation lengths at normal incidence, >= 0 */
  float disk_eloss;            /* GeV, >= 0 */
  float sigma_r;               /* radial hit resolution on a disk, cm, > 0 */
  float eta_barrel;            /* > 0 */
} kf_detector;

/* Algorithm settings (Sec. 2 and Sec. 4.3: windows, scores, duplicate cuts). */
typedef struct {
  int max_cands;          /* candidates kept per seed, 1..KF_MAX_CANDS */
  int max_holes;          /* layers without a hit allowed per candidate */
  float chi2_cut;         /* a hit is compatible if its chi2 is below this */
  float dup_shared_frac;  /* duplicate if shared hits > frac * min(nA, nB) */
  int n_eta_bins;         /* hit grid per layer: eta bins (1..256) ... */
  int n_phi_bins;         /* ... times phi bins */
  int lanes_per_seed;     /* 0 = automatic; else one of 4, 6, 8, 10, 12, 16 and >= max_cands */
  int block_threads;      /* 0 = automatic (128); multiple of 32, <= 256 */
  int persistent;         /* 1 = persistent work-queue launch, 0 = one warp per seed tile */
  int per_event;          /* 1 = bin, find and remove duplicates with one launch per event
                             (the plain form); 0 = one launch per step over the whole batch */
  int ckpt_stride;        /* hits between forward checkpoints of the adjoint (0 = 1; 1..8) */
  int find_regcap;        /* 0 = finding kernel at the compiler's register count (blocks <= 256
                             threads); 1 = at most 102 registers, five blocks per SM (blocks
                             <= 128 threads).  The results are identical. */
  /* Kinematic criteria (Sec. 4.2 names pT, eta and phi).  For two states A, B:
   * eta = -ln tan(theta/2); phi0 = the direction of motion at the point of the
   * helix closest to the z axis (the same for every state along a helix);
   * k = q/pT.  A and B are close when |eta_A - eta_B| < deta,
   * |phi0_A - phi0_B| (on the circle) < dphi and
   * ||k_A| - |k_B|| <= dpt * max(|k_A|, |k_B|); a cut of 0 is not applied. */
  float dup_deta;         /* duplicate removal: a pair over the shared-hit fraction is a */
  float dup_dphi;         /* duplicate only if its found states are also close (all 0: the */
  float dup_dpt;          /* shared fraction alone); each >= 0 */
  int seed_clean;         /* 1 = seed cleaning before finding: visit each event's seeds by index
                             and drop a seed that is close to a kept one and shares at least
                             seed_min_shared of its three hits with it.  A dropped seed gives an
                             empty track (n_found 0, keep 0). */
  float seed_deta;        /* seed cleaning cuts: 0 < seed_deta <= KF_SEED_MAX_DETA, */
  float seed_dphi;        /* seed_dphi >= 0, */
  float seed_dpt;         /* seed_dpt >= 0 */
  int seed_min_shared;    /* 0..3 */
  int resolve_max_rounds; /* 0 = the resolution rounds of seed cleaning and duplicate removal run
                             until every decision is taken (at most items + 4 rounds, always
                             enough); > 0 = give up after that many rounds: the next synchronizing
                             call returns KF_ERR_TIMEOUT, and flags of undecided items are not
                             valid (a latency bound on the device-side loop) */
} kf_config;

/* Create a context for a detector and configuration.  Allocates nothing on
 * the device yet.  Errors: KF_ERR_ARG for out-of-range fields. */
int kf_create(const kf_detector* det, const kf_config* cfg, kf_ctx** out);

/* Release every device buffer, graph and stream-independent resource. */
int kf_destroy(kf_ctx* ctx);

/* Load hits of n_events events.
 * ev_offsets: HOST array [n_events+1], CSR offsets into the hit arrays.
 * x, y, z: float [n_hits] global positions (cm); layer: int [n_hits] in
 * [0, n_surfaces): a barrel layer or an endcap disk (kf_detector).  A hit is referred to by its index within its event
 * (0 .. ev_offsets[e+1]-ev_offsets[e]-1), in the order given here.
 * Loading hits unloads the seeds (their hit indices refer to the previous
 * hits): call kf_load_seeds again before finding, fitting, tuning or a graph
 * replay, which return KF_ERR_STATE until then.
 * Errors: KF_ERR_ARG, KF_ERR_CAPACITY (an event above KF_MAX_EVENT_HITS). */
int kf_load_hits(kf_ctx* ctx, int n_events, const int* ev_offsets, const float* x,
                 const float* y, const float* z, const int* layer, int device_ptrs, void* stream);

/* Load seeds: prior state at the first seed hit and three seed hits.
 * ev_offsets: HOST array [n_events+1] (same n_events as the hits).
 * params: float [6][n_seeds]; cov: float [21][n_seeds]; seed_hits: int
 * [3][n_seeds] event-local hit indices on increasing barrel layers. */
int kf_load_seeds(kf_ctx* ctx, int n_events, const int* ev_offsets, const float* params,
                  const float* cov, const int* seed_hits, int device_ptrs, void* stream);

/* Material map (the r-z material description of Sec. 3, per barrel layer):
 * x0_map float [n_layers][n_z], the thickness in radiation lengths at normal
 * incidence at n_z z nodes spread evenly over [-z_max, z_max]; between nodes
 * the thickness is linear in z, beyond the ends constant, and the scattering
 * of a layer uses it at the state's z.  n_z = 0 (x0_map may be NULL) returns
 * to the per-layer x0 of the detector.  2 <= n_z <= KF_MAX_MATERIAL_NODES;
 * host values must be finite and >= 0 (device arrays are not checked).  A
 * captured graph keeps the material it was captured with: this call drops the
 * graph (capture again).  Errors: KF_ERR_ARG. */
#define KF_MAX_MATERIAL_NODES 4096
int kf_set_material(kf_ctx* ctx, int n_z, const float* x0_map, int device_ptrs, void* stream);

/* Layer alignment offsets float [n_layers][2] = (a_rphi, a_z) in cm.  A hit
 * on layer L is used after rotating it by -a_rphi/R_L about z and shifting
 * z by -a_z.  Zero after kf_create. */
int kf_set_alignment(kf_ctx* ctx, const float* offsets, int device_ptrs, void* stream);

/* Bin hits, clean the seeds (with seed_clean) and run the combinatorial
 * Kalman-filter finding for every (kept) seed (Sec. 2): seed fit over the
 * three seed hits, then per surface of the seed's region plan (barrel
 * layers; then the disks of its side for a forward seed) propagation,
 * covariance transport, chi2 of every compatible hit, per-seed top-N ranking,
 * update and multiple scattering.  Asynchronous.  Errors of seed cleaning (more than 16
 * lower-index duplicates of one seed: KF_ERR_CAPACITY) surface at the next
 * synchronizing call. */
int kf_find_tracks(kf_ctx* ctx, void* stream);

/* Duplicate removal over the found tracks of each event (Sec. 4.2): shared
 * hits over dup_shared_frac and the kinematic pre-cuts dup_deta, dup_dphi,
 * dup_dpt; an empty track (a cleaned seed) is never kept.  Asynchronous.
 * Requires kf_find_tracks. */
int kf_remove_duplicates(kf_ctx* ctx, void* stream);

/* Kalman re-fit from each seed's prior over a hit list.
 * source = KF_FIT_FOUND: the found tracks (only kept ones once duplicates
 * were removed); KF_FIT_GIVEN: hit_lists int [n_seeds][max_len]
 * (event-local indices on increasing layers) with n_hits int [n_seeds].
 * The result is the state after the last hit, before its scattering.
 * Asynchronous (host hit lists are copied before the call returns). */
int kf_fit_tracks(kf_ctx* ctx, int source, const int* hit_lists, const int* n_hits, int max_len,
                  int device_ptrs, void* stream);

/* Gradient of the summed chi2 of the last kf_fit_tracks (tracks with status
 * KF_FIT_OK) with respect to the alignment offsets (g_align float
 * [n_layers][2]), hit positions (g_hits float [n_hits][3], global hit order,
 * may be NULL) and seed parameters (g_seed float [6][n_seeds], may be NULL):
 * the adjoint of the fit, one thread per track.  Forward states are kept
 * every ckpt_stride hits and recomputed in between; ckpt_stride (1..8) must
 * satisfy hits per track <= 32 * ckpt_stride (KF_ERR_CAPACITY otherwise).
 * Disk hits contribute to g_hits (their x and y; z is 0) and not to g_align
 * (disks carry no alignment). */
int kf_fit_adjoint(kf_ctx* ctx, float* g_align, float* g_hits, float* g_seed, int device_ptrs,
                   void* stream);

/* Copy out the found tracks.  hits int [n_seeds][n_surfaces] (n_surfaces =
 * n_layers + 2 n_disks; event-local indices in search order, -1 padded),
 * n_found int [n_seeds], chi2 float [n_seeds], params
 * float [6][n_seeds], cov float [21][n_seeds], keep uint8 [n_seeds] (1 when
 * duplicate removal did not run).  Any pointer may be NULL. */
int kf_get_tracks(kf_ctx* ctx, int* hits, int* n_found, float* chi2, float* params, float* cov,
                  unsigned char* keep, int device_ptrs, void* stream);

/* Copy out the fit results: params float [6][n_seeds], cov float
 * [21][n_seeds], chi2 float [n_seeds], status int [n_seeds] (KF_FIT_*). */
int kf_get_fit(kf_ctx* ctx, float* params, float* cov, float* chi2, int* status, int device_ptrs,
               void* stream);

/* Capture find + duplicate removal + fit (+ the adjoint of the fit if
 * with_adjoint, its gradients kept in the context for kf_get_gradient) on
 * the stream into a CUDA graph owned by the context; kf_launch_graph replays
 * it.  stream must not be the legacy default stream.  The graph holds the
 * buffer addresses, sizes and event offsets of the capture: loads between
 * replays may change the values of hits and seeds, but kf_launch_graph
 * returns KF_ERR_STATE (capture again) when a load since the capture changed
 * a size or an event offset or moved a buffer, or when the seeds were not
 * loaded again after the hits. */
int kf_capture_graph(kf_ctx* ctx, int with_adjoint, void* stream);
int kf_launch_graph(kf_ctx* ctx, void* stream);

/* Copy out the gradients kept by a graph with the adjoint (or by the last
 * kf_fit_adjoint called with host pointers): g_align float [n_layers][2],
 * g_hits float [n_hits][3], g_seed float [6][n_seeds]; any may be NULL. */
int kf_get_gradient(kf_ctx* ctx, float* g_align, float* g_hits, float* g_seed, int device_ptrs, void* stream);

/* Time every lanes-per-seed (4..16, >= max_cands) / block-size (32, 64, 128,
 * 256 threads: candidate tiles of that many lanes) / register-budget /
 * launch-form choice of the finding kernel on the loaded inputs and keep the
 * fastest in the context.  Synchronous.  results (may be NULL) receives up to
 * max_results rows of 5 floats (lanes, threads, persistent, register cap, ms). */
int kf_autotune(kf_ctx* ctx, float* results, int max_results, int* n_results, void* stream);

/* Counters of the last kf_find_tracks, synchronous (8 values):
 * [0] candidate-layer steps (a live candidate propagated, transported and
 * window-searched on one layer), [1] hit-children updated, [2] hits whose
 * chi2 was evaluated, [3] seeds built (those kept by seed cleaning), [4]
 * hole-children (scattering only),
 * [5] propagations run in double (crossings with cos(angle to the radial
 * direction) < 0.2), [6] predictions without a positive definite measurement
 * covariance (no hit searched; expected 0), [7] seeds redone by the careful
 * pass (their candidates met such a crossing). */
int kf_get_counters(kf_ctx* ctx, long long* counters8, void* stream);

/* The same counters and those of the endcap disks, synchronous: the first n
 * (1..KF_N_COUNTERS) of [0..7] as kf_get_counters, [8] the candidate-layer
 * steps onto endcap disks (a part of [0]), [9] the hit-children updated on
 * disks (a part of [1]), [10] the hole-children on disks (a part of [4]).
 * Errors: KF_ERR_ARG (n out of range). */
#define KF_N_COUNTERS 11
int kf_get_counters_n(kf_ctx* ctx, long long* counters, int n, void* stream);

/* Stage timing: with enable = 1, CUDA events are recorded around the
 * binning, finding, duplicate removal, fit, adjoint and seed-cleaning
 * launches of the batched form (also inside a captured graph).
 * kf_get_stage_ms (synchronous) returns the durations of the last completed
 * run: ms6 = {bin, find, dedup, fit, adjoint, seed clean} (find excludes seed
 * cleaning); a stage that did not run reads -1. */
int kf_set_stage_timing(kf_ctx* ctx, int enable);
int kf_get_stage_ms(kf_ctx* ctx, float* ms6, void* stream);

/* Number of kernel nodes in the captured graph (launches per replay). */
int kf_graph_kernel_count(kf_ctx* ctx, int* n_kernels);

/* Wait for the stream and report a sticky device-side error, if any. */
int kf_sync(kf_ctx* ctx, void* stream);

/* Message of the last error on this context (static storage, never NULL). */
const char* kf_last_error(const kf_ctx* ctx);

/* Limits of kf_remove_duplicates_noalloc (one event per call). */
#define KF_NOALLOC_MAX_TRACKS 16384
#define KF_NOALLOC_MAX_HITS 262144

/* Duplicate removal for ONE event without any device allocation.
 *
 * The paper has no counterpart to this entry point; it exists for callers that
 * cannot allocate device memory at all -- code running inside a host framework
 * that owns every device allocation through its own pool, a trigger-style
 * pipeline where cudaMalloc/cudaFree are banned from the hot path because
 * they synchronize the device, or a plugin held to another library's fixed
 * memory budget.  It needs no kf_ctx (creating one allocates).
 *
 * Same definition as kf_remove_duplicates with the shared-hit criterion
 * alone: the kinematic pre-cuts (dup_deta, dup_dphi, dup_dpt of kf_config)
 * are not applied here.  Inputs and the output are device pointers owned by
 * the caller, read and written in stream order:
 *   hits     int   [n_tracks][n_layers] event-local hit indices, -1 padded;
 *            every used index must lie in [0, n_hits);
 *   n_found  int   [n_tracks] hits per track (<= n_layers);
 *   chi2     float [n_tracks] chi2 sums (ordering key);
 *   keep     uint8 [n_tracks] output, 1 = kept;
 *   status   int   [1] output (may be NULL): 0, or a nonzero device-side
 *            status when a table of the kernel overflowed; written by every
 *            call that returns KF_OK, n_tracks = 0 included.
 * Scratch lives in a fixed static device array (about 4.2 MB, present on every
 * device that loads the library until the process exits).  The first call on a
 * device looks up that array's device address (with the device current); make
 * that first call before any stream capture.  Every call shares the array, so
 * calls whose kernels overlap on the GPU race: order them on one stream.
 * Returns KF_ERR_CAPACITY when n_tracks > KF_NOALLOC_MAX_TRACKS or n_hits >
 * KF_NOALLOC_MAX_HITS (nothing is launched), KF_ERR_ARG for a bad argument,
 * KF_ERR_CUDA when the address lookup or a launch fails.  Asynchronous. */
int kf_remove_duplicates_noalloc(int n_tracks, int n_layers, int n_hits, const int* hits,
                                 const int* n_found, const float* chi2, float dup_shared_frac,
                                 unsigned char* keep, int* status, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* KF_H_ */
