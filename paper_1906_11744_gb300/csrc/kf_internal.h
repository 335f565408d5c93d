// Internal launch interface between the C ABI layer and the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "kf_common.cuh"

namespace kfg {

// Device-side status word values (sticky; read by kf_sync / kf_get_*).
enum : int {
  ST_OK = 0,
  ST_DEDUP_PARTNERS = 1,   // a track shares hits with more tracks than the partner table holds
  ST_DEDUP_CONFLICTS = 2,  // more higher-priority conflicts than the conflict table holds
  ST_DEDUP_ROUNDS = 3,     // the resolution loop hit its iteration bound
  ST_SEED_CONFLICTS = 4,   // seed cleaning: more lower-index duplicates than the conflict table holds
  ST_SEED_ROUNDS = 5,      // seed cleaning: the resolution loop hit its iteration bound
};

// Seeds of an event are taken in order of their polar angle, counting-sorted
// into SEED_THETA_BINS equal bins of [0, pi] (the order within a bin is
// arbitrary).
constexpr int SEED_THETA_BINS = 1024;
__device__ __forceinline__ int seed_theta_bin(float theta) {
  return min(max((int)(theta * ((float)SEED_THETA_BINS / PI_F)), 0), SEED_THETA_BINS - 1);
}

struct FindParams {
  DevGeom g;
  const float* hx;
  const float* hy;
  const float* hz;
  const int* hlayer;
  const int* hit_off;        // [n_events + 1]
  const float4* hb;          // binned hits (x, y, z, event-local index as int bits)
  const unsigned* bin_off;   // [n_events * n_layers * n_bins + 1] global offsets into hb
  const float* eta_edges;    // [KF_MAX_LAYERS][MAX_ETA_BINS + 1] z edges of the eta bins
  const unsigned char* eta_lut;  // [KF_MAX_LAYERS][ETA_LUT] first guess of the eta bin
  const float* sp;           // seed params [6][ns]
  const float* sc;           // seed cov [21][ns]
  const int* sh;             // seed hits [3][ns]
  const int* seed_event;     // [ns]
  const Align4* align;       // [n_layers]
  int ns;                    // seed stride
  int s_begin, s_end;        // seed range of this launch
  const int* order;          // [ns] order of the seeds within each event (or null)
  const int* seed_off;       // [n_events + 1]
  const int* kept_cnt;       // [n_events] seeds left by seed cleaning (or null: every seed);
                             // with it, order lists each event's kept seeds first
  int* out_hits;             // [ns][n_layers]
  int* out_n;                // [ns]
  float* out_chi2;           // [ns]
  float* out_p;              // [6][ns]
  float* out_C;              // [21][ns]
  unsigned* queue;           // [3] work counters of the main and careful passes and the
                             // number of listed seeds (zeroed before the launch)
  int* tangent_list;         // [ns] seeds the main pass left to the careful pass
  float* sfit;               // [29][ns] seed kernel: the state the first layer's children come
                             // from (p, C), the seed's chi2 sum, the first layer's counts
  unsigned long long* skeys; // [max_cands][ns] seed kernel: the first layer's children (keys)
  unsigned char* sflag;      // [ns] seed kernel: bit 1 near-tangent crossing, bit 2 carried,
                             // bits 3-7 number of children
  unsigned long long* counters;  // [8], see kf_get_counters
  int persistent;
};

struct BinParams {
  DevGeom g;
  const float* hx;
  const float* hy;
  const float* hz;
  const int* hlayer;
  const int* hit_off;
  int n_events;
  int h_begin, h_end;     // hit range of this launch
  const float* eta_edges; // [KF_MAX_LAYERS][MAX_ETA_BINS + 1]
  const unsigned char* eta_lut;  // [KF_MAX_LAYERS][ETA_LUT]
  unsigned* cnt;          // [n_bins_total + 1] counts, then offsets
  unsigned* key;          // [n_hits]
  unsigned* rank;         // [n_hits]
  float4* hb;             // [n_hits]
  float4* grouped;        // [n_hits] hits grouped by (event, layer) (layer-grouped form)
  unsigned* gtab;         // bin_group_elems(): bucket counts, bases (+ total), cursors of the
                          // (event, layer, chunk of eta rows) buckets
};

struct DedupParams {
  const int* out_hits;   // [ns][L]
  const int* out_n;
  const float* out_chi2;
  const int* hit_off;
  const int* seed_off;   // [n_events + 1]
  const int* seed_event; // [ns] (batched launch)
  int L;
  int ns;
  float frac;
  int e_begin;           // first event of this launch (one block per event)
  unsigned* hit_cnt;     // [n_hits + n_events]
  int* owners;           // [ns * L]
  int* conf;             // [ns * DEDUP_CONF_CAP]
  int* n_conf;           // [ns]
  unsigned char* state;  // [ns]
  unsigned char* keep;   // [ns]
  int* status;
  // Kinematic pre-cuts (null trk_p: none): a pair is a duplicate only if its
  // states trk_p [6][ns] are also close in eta, phi0 and pT (a cut <= 0 is off).
  const float* trk_p = nullptr;
  float kb = 0.f;        // h = kb * q/pT
  float deta = 0.f, dphi = 0.f, dpt = 0.f;
  int max_rounds = 0;    // resolution rounds before giving up (0: until settled)
};

struct SeedCleanParams {
  float kb;              // h = kb * q/pT
  const float* sp;       // seed params [6][ns]
  const float* sc;       // seed cov [21][ns]
  const int* sh;         // seed hits [3][ns]
  const int* seed_off;   // [n_events + 1]
  const int* seed_event; // [ns]
  const int* order;      // [ns] the theta order of each event's seeds
  int ns;
  int L;
  float deta, dphi, dpt; // cuts (deta > 0; dphi, dpt <= 0: not applied)
  int min_shared;        // seed hits shared, at least
  float4* kin;           // [ns] by position in order: (eta, phi0, |q/pT|, theta bin as int bits)
  int4* kseed;           // [ns] by position: (seed, its three hits)
  int* conf;             // [ns * DEDUP_CONF_CAP] by position: positions of the lower-index duplicates
  int* n_conf;           // [ns] by position
  unsigned char* state;  // [ns] by position
  int* list;             // [ns] per event (at its positions): the positions with conflicts
  int* list_cnt;         // [n_events]
  int* clean_order;      // [ns] per event: the kept seeds in theta order, then the dropped ones
  int* kept_cnt;         // [n_events]
  // outputs written for a dropped seed: an empty track, not kept
  int* out_hits;         // [ns][L]
  int* out_n;
  float* out_chi2;
  float* out_p;          // [6][ns]
  float* out_C;          // [21][ns]
  unsigned char* keep;   // [ns]
  int* status;
  int max_rounds = 0;    // resolution rounds before giving up (0: until settled)
};

// The adjoint redoes in double only the steps closer to tangent than this
// (its tolerance is looser than the fit's; the fit's threshold is 0.5).
constexpr float ADJOINT_CAREFUL_COS = 0.2f;
constexpr unsigned CAREFUL_DBL_BIT = 0x80000000u;  // careful_list entry: a crossing below ADJOINT_CAREFUL_COS

constexpr int DEDUP_PARTNER_CAP = 32;
constexpr int DEDUP_CONF_CAP = 16;

struct FitParams {
  DevGeom g;
  const float* hx;
  const float* hy;
  const float* hz;
  const int* hlayer;
  const int* hit_off;
  const float* sp;
  const float* sc;
  const int* seed_event;
  const Align4* align;
  int ns;
  const int* lists;       // [ns][max_len]
  const int* n_list;      // [ns]
  int max_len;
  const unsigned char* keep;  // may be null
  // false: the FP32 pass runs beside duplicate removal and fits every track
  // (keep is still being written); launch_fit_unkept clears the removed
  // tracks' outputs afterwards, and the careful pass reads keep as usual
  bool keep_in_main = true;
  float* fit_p;           // [6][ns]
  float* fit_C;           // [21][ns]
  float* fit_chi2;        // [ns]
  int* fit_status;        // [ns]
  int* careful_list;      // [ns] positions (in order) of the tracks refitted with double-precision steps;
                          // the careful pass adds CAREFUL_DBL_BIT where the adjoint needs double steps
  unsigned* careful_count;  // zeroed before the launch
  unsigned char* careful_flag;  // [ns] by track: 1 for the tracks of careful_list, else 0
  int* dbl_list;          // [ns] positions of the careful tracks with CAREFUL_DBL_BIT, packed
  unsigned* dbl_count;    // their number (zeroed before the careful pass)
  float* ckpt;            // [ckpt_slices][27][ns] by position: states before every ckpt_stride-th hit, or null
  int ckpt_stride;
  int ckpt_slices;        // checkpoints per track the buffer holds
  // Tracks of each window of 4,096 by decreasing hit count (duplicates
  // last): position i of the fit and of the adjoint takes track order[i], so
  // that a warp's tracks run about the same number of steps.
  int* order;             // [ns] written by launch_fit_main
};

constexpr int MAX_CKPT = KF_MAX_LAYERS;  // checkpoints per track at most
// Checkpoints per track for tracks of up to max_len hits.
inline int ckpt_slices_for(int max_len, int stride) {
  const int n = (max_len + stride - 1) / stride;
  return n < MAX_CKPT ? n : MAX_CKPT;
}
constexpr int DEFAULT_CKPT_STRIDE = 1;
constexpr int MAX_CKPT_STRIDE = 8;

struct AdjParams {
  DevGeom g;
  const float* hx;
  const float* hy;
  const float* hz;
  const int* hlayer;
  const int* hit_off;
  const float* sp;
  const float* sc;
  const int* seed_event;
  const Align4* align;
  int ns;
  int n_hits;
  const int* lists;
  const int* n_list;
  int max_len;
  const unsigned char* keep;   // may be null
  const int* fit_status;       // tracks with a status other than KF_FIT_OK are skipped
  int stride;                  // checkpoint stride
  float* g_hits;               // [n_hits][3] (required: the alignment gradient is summed from it)
  float* g_seed;               // [6][ns] or null
  float* g_align;              // [n_layers][2]
  double* g_align_acc;         // [2 * KF_MAX_LAYERS] accumulator
  const int* careful_list;     // positions of the tracks the fit flagged as near-tangent ...
  const unsigned* careful_count;
  const unsigned char* careful_flag;  // ... and their per-track flag
  const int* dbl_list;         // the careful tracks whose adjoint needs double steps, packed
  const unsigned* dbl_count;
  const float* ckpt;           // the fit's checkpoints [slices][27][ns] by position
  const int* order;            // the fit's track order (position -> track)
};

// kf_adjoint.cu
// Adjoint: zero the accumulators, the FP32 pass and the passes over the
// fit's careful list (independent: either order or concurrently), then the
// alignment gradient from its double-precision sums.
cudaError_t launch_adjoint_begin(const AdjParams& P, cudaStream_t st);
cudaError_t launch_adjoint_pass(const AdjParams& P, bool careful, cudaStream_t st);
cudaError_t launch_adjoint_end(const AdjParams& P, cudaStream_t st);
bool adjoint_stride_ok(int stride, int max_len);
// kf_find.cu
// Finding: the main pass (gives up and lists seeds that meet a near-tangent
// crossing), then the careful pass over the listed seeds (persistent, any
// grid; the count is read on the device).
cudaError_t launch_find_main(const FindParams& P, int lanes, int regcap, int threads, int grid_cap,
                             cudaStream_t st);
cudaError_t launch_find_careful(const FindParams& P, int lanes, int grid, cudaStream_t st);
// Per event, the seeds sorted by theta (params row 5) into order[].
cudaError_t launch_seed_order(const float* theta, const int* seed_off, int n_events, int* order, cudaStream_t st);
size_t find_smem_bytes(int threads, int n_layers, int n_eta);
bool find_lanes_supported(int lanes);
// Sets the dynamic shared-memory limit of the kernel variant (must run
// outside stream capture) and reports resident blocks per SM.
cudaError_t find_prepare(int lanes, int regcap, int threads, const DevGeom& g, int* blocks_per_sm);
// The disk variants (kf_find_disk.cu), called by the entry points above for a
// detector with endcap disks.
cudaError_t find_prepare_disk(int lanes, int regcap, int threads, const DevGeom& g, int* blocks_per_sm);
cudaError_t launch_find_main_disk(const FindParams& P, int lanes, int regcap, int threads, int grid_cap,
                                  cudaStream_t st);
cudaError_t launch_find_careful_disk(const FindParams& P, int lanes, int grid, cudaStream_t st);
// kf_bin.cu
cudaError_t launch_bin(const BinParams& P, size_t bin_begin, size_t n_bins, unsigned first_pos, int max_event_hits,
                       unsigned* scan_tmp, size_t scan_tmp_elems, cudaStream_t st);
size_t scan_tmp_elems(size_t n);
// Exclusive scan of cnt[0..n) in place plus add; cnt[n] = total + add.
// tmp: scan_tmp_elems(n) entries.
cudaError_t scan_exclusive_inplace(unsigned* cnt, size_t n, unsigned add, unsigned* tmp, size_t tmp_elems,
                                   cudaStream_t st);
size_t bin_group_elems(int n_events, int n_layers, int n_eta, int n_phi);
// kf_dedup.cu
cudaError_t launch_dedup(const DedupParams& P, int n_events, cudaStream_t st);
// Whole batch: hit_cnt holds n_hits + n_events + 1 entries; scan_tmp
// scan_tmp_elems(n_hits + n_events) entries.
cudaError_t launch_dedup_batched(const DedupParams& P, int n_events, int n_hits, unsigned* scan_tmp,
                                 size_t scan_tmp_elems, cudaStream_t st);
// Seed cleaning of the seeds at positions [pos_begin, pos_end) of the theta
// order, which are those of events [e_begin, e_begin + n_events).
cudaError_t launch_seed_clean(const SeedCleanParams& P, int pos_begin, int pos_end, int e_begin, int n_events,
                              cudaStream_t st);
// kf_fit.cu: the FP32 pass (flags and lists near-tangent tracks) and the
// careful pass over the list; launch_fit runs both.
cudaError_t launch_fit_main(const FitParams& P, cudaStream_t st);
cudaError_t launch_fit_careful(const FitParams& P, cudaStream_t st);
cudaError_t launch_fit(const FitParams& P, cudaStream_t st);
// After a main pass with keep_in_main false: the removed tracks' outputs
// zeroed and their status KF_FIT_SKIPPED, as the main pass would have left them.
cudaError_t launch_fit_unkept(const FitParams& P, cudaStream_t st);

}  // namespace kfg
