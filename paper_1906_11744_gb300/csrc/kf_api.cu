// C ABI (include/kf.h): context, device buffers, launches, CUDA graph and
// autotuner.  The calls follow the paper's problem statement: load hits and
// seeds (Sec. 3), find tracks (Sec. 2), remove duplicates (Sec. 4.2), fit
// tracks (Sec. 5).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "kf_internal.h"

using namespace kfg;

namespace {

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

}  // namespace

struct kf_ctx {
  kf_detector det;
  kf_config cfg;
  DevGeom g;
  int lanes = 0, threads = 0, persistent = 1, per_event = 0, regcap = 0;
  int num_sms = 0;
  int blocks_per_sm = 1;
  int n_events = 0, n_hits = 0, n_seeds = 0, n_seed_events = -1, max_event_hits = 0;
  std::vector<int> hit_off_h, seed_off_h;
  size_t n_bins_total = 0;
  // inputs
  DevBuf hx, hy, hz, hlayer, hit_off, seed_off, sp, sc, sh, seed_event, align_raw, align4, eta_edges, eta_lut;
  // binning
  DevBuf hb, bin_cnt, bin_key, bin_rank, scan_tmp, bin_grouped, bin_gtab;
  // finding
  DevBuf out_hits, out_n, out_chi2, out_p, out_C, keep, queue, counters, status, tangent, seed_order, check;
  DevBuf sfit, sflag, skeys, x0map;
  // duplicate removal scratch (the conflict lists also serve seed cleaning)
  DevBuf dd_hit_cnt, dd_owners, dd_conf, dd_nconf, dd_state, dd_scan_tmp;
  // seed cleaning
  DevBuf sc_kin, sc_seed, clean_order, kept_cnt, sc_list, sc_list_cnt;
  // fit
  DevBuf given_lists, given_n, fit_p, fit_C, fit_chi2, fit_status, careful_list, careful_count, careful_flag, ckpt;
  DevBuf fit_order, dbl_list;
  bool want_ckpt = false;
  int given_max_len = 0;
  bool found = false, deduped = false, fitted = false;
  int fit_source = KF_FIT_FOUND;
  FitParams last_fit;
  DevBuf adj_align_acc, adj_align, adj_hits, adj_seed;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  // What the captured graph baked in: the device address of every buffer and
  // the loaded sizes and event offsets.  A replay after a load that moved a
  // buffer or changed a size is refused.
  std::vector<void*> graph_bufs;
  std::vector<int> graph_hit_off, graph_seed_off;
  int graph_n_seeds = -1;
  int stage_timing = 0;
  cudaEvent_t ev[12] = {};  // start/end of bin, find, dedup, fit, adjoint, seed cleaning
  // Side stream (highest priority) for the careful passes that run beside
  // the main passes; fork/join events.
  cudaStream_t side = nullptr;
  // Inside a graph capture with the adjoint: kf_fit_tracks leaves the fit's
  // careful pass to kf_fit_adjoint, which runs it on the side stream before
  // the careful adjoint, beside the FP32 adjoint (which needs neither).
  bool defer_careful_fit = false, careful_fit_pending = false;
  // Inside a graph capture: kf_fit_tracks runs beside duplicate removal (its
  // FP32 pass fits every found track; the caller then clears the removed ones)
  // and always leaves its careful pass for later.
  bool fit_beside_dedup = false;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  std::string err = "";
};

namespace {

int fail(kf_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

#define CK(call)                                                                         \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return fail(ctx, KF_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

cudaError_t grow(DevBuf& b, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (b.bytes >= bytes) return cudaSuccess;
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
  cudaError_t e = cudaMalloc(&b.p, bytes);
  if (e == cudaSuccess) b.bytes = bytes;
  return e;
}

template <class T>
T* ptr(const DevBuf& b) {
  return reinterpret_cast<T*>(b.p);
}

void release(DevBuf& b) {
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
}

cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// Copy n bytes into a device buffer from a host or device source.
cudaError_t put(void* dst, const void* src, size_t n, int device_ptrs, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  return cudaMemcpyAsync(dst, src, n, device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st);
}

cudaError_t get(void* dst, const void* src, size_t n, int device_ptrs, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  return cudaMemcpyAsync(dst, src, n, device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st);
}

// Input checks on the device (after the copies; works for host and device
// arrays alike): any value outside [0, hi) sets *bad.
__global__ void k_check_range(const int* v, int n, int hi, int* bad) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    if (v[i] < 0 || v[i] >= hi) *bad = 1;
}
// Seed hit indices (three per seed, [3][n]) against their event's hit count;
// the hits must lie on barrel layers (*bad = 2 otherwise).
__global__ void k_check_seed_hits(const int* sh, const int* seed_event, const int* hit_off, const int* hlayer,
                                  int n_layers, int n, int* bad) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
    const int e = seed_event[s];
    const int nh = hit_off[e + 1] - hit_off[e];
    for (int k = 0; k < 3; ++k) {
      const int h = sh[(size_t)k * n + s];
      if (h < 0 || h >= nh) *bad = 1;
      else if (hlayer[hit_off[e] + h] >= n_layers) atomicMax(bad, 2);
    }
  }
}

// Event of every seed from the seed offsets (binary search).
__global__ void k_seed_event(const int* seed_off, int n_events, int n, int* out) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  int lo = 0, hi = n_events - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (seed_off[mid] <= s) lo = mid; else hi = mid - 1;
  }
  out[s] = lo;
}

__global__ void k_align(const float* off, const DevGeom g, Align4* out) {
  const int l = threadIdx.x;
  if (l >= g.n_layers) return;
  const float R = g.radius[l];
  const float ar = off ? off[2 * l] : 0.f, az = off ? off[2 * l + 1] : 0.f;
  float s, c;
  sincosf(-ar / R, &s, &c);
  out[l] = Align4{c, s, ar / R, az};
}

bool supported_lanes(int lanes) { return find_lanes_supported(lanes); }

int auto_lanes(int n) {
  const int opts[] = {4, 6, 8, 10, 12, 16};
  for (int o : opts)
    if (o >= n) return o;
  return 16;
}

}  // namespace

static int check_status(kf_ctx* ctx, cudaStream_t st) {
  int h = 0;
  CK(cudaMemcpyAsync(&h, ctx->status.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (h == ST_OK) return KF_OK;
  CK(cudaMemsetAsync(ctx->status.p, 0, sizeof(int), st));
  CK(cudaStreamSynchronize(st));
  switch (h) {
    case ST_DEDUP_PARTNERS: return fail(ctx, KF_ERR_CAPACITY, "duplicate removal: partner table overflow");
    case ST_DEDUP_CONFLICTS: return fail(ctx, KF_ERR_CAPACITY, "duplicate removal: conflict table overflow");
    case ST_DEDUP_ROUNDS: return fail(ctx, KF_ERR_TIMEOUT, "duplicate removal: resolution did not settle");
    case ST_SEED_CONFLICTS: return fail(ctx, KF_ERR_CAPACITY, "seed cleaning: conflict table overflow");
    case ST_SEED_ROUNDS: return fail(ctx, KF_ERR_TIMEOUT, "seed cleaning: resolution did not settle");
    default: return fail(ctx, KF_ERR_CUDA, "unknown device status");
  }
}
static int check_status_sync(kf_ctx* ctx, cudaStream_t st) { return check_status(ctx, st); }

extern "C" {

const char* kf_last_error(const kf_ctx* ctx) {
  if (!ctx) return "null context";
  return ctx->err.c_str();
}

int kf_create(const kf_detector* det, const kf_config* cfg, kf_ctx** out) {
  kf_ctx* ctx = nullptr;
  if (!det || !cfg || !out) return KF_ERR_ARG;
  *out = nullptr;
  if (det->n_layers < 1 || det->n_layers > KF_MAX_LAYERS) return KF_ERR_ARG;
  for (int l = 0; l < det->n_layers; ++l) {
    if (!(det->radius[l] > 0.f) || (l > 0 && !(det->radius[l] > det->radius[l - 1]))) return KF_ERR_ARG;
    if (!(det->x0[l] >= 0.f)) return KF_ERR_ARG;
    if (!(det->eloss[l] >= 0.f) || !std::isfinite(det->eloss[l])) return KF_ERR_ARG;
  }
  if (!(det->z_max > 0.f) || !(det->sigma_rphi > 0.f) || !(det->sigma_z > 0.f) || !std::isfinite(det->bz))
    return KF_ERR_ARG;
  if (det->n_disks < 0 || det->n_disks > KF_MAX_DISKS) return KF_ERR_ARG;
  if (det->n_disks > 0) {
    for (int k = 0; k < det->n_disks; ++k)
      if (!(det->disk_z[k] > 0.f) || !std::isfinite(det->disk_z[k]) ||
          (k > 0 && !(det->disk_z[k] > det->disk_z[k - 1])))
        return KF_ERR_ARG;
    if (!(det->disk_rmin > 0.f) || !(det->disk_rmax > det->disk_rmin) || !std::isfinite(det->disk_rmax) ||
        !(det->disk_x0 >= 0.f) || !std::isfinite(det->disk_x0) || !(det->disk_eloss >= 0.f) ||
        !std::isfinite(det->disk_eloss) || !(det->sigma_r > 0.f) || !std::isfinite(det->sigma_r) ||
        !(det->eta_barrel > 0.f) || !std::isfinite(det->eta_barrel))
      return KF_ERR_ARG;
  }
  {  // the field factor at the corners of the detector's (r, z) box (monotone in r^2 and z^2)
    const double zm = det->n_disks > 0 ? std::max(det->z_max, det->disk_z[det->n_disks - 1]) : det->z_max;
    const double rm = det->n_disks > 0 ? std::max(det->radius[det->n_layers - 1], det->disk_rmax)
                                       : det->radius[det->n_layers - 1];
    const double z2 = zm * zm, r2 = rm * rm;
    if (!std::isfinite(det->field_cz) || !std::isfinite(det->field_cr)) return KF_ERR_ARG;
    for (int c = 0; c < 4; ++c) {
      const double f = 1.0 + det->field_cz * ((c & 1) ? z2 : 0.0) + det->field_cr * ((c & 2) ? r2 : 0.0);
      if (!(f >= 0.2 && f <= 5.0)) return KF_ERR_ARG;
    }
  }
  if (cfg->max_cands < 1 || cfg->max_cands > KF_MAX_CANDS || cfg->max_holes < 0 || !(cfg->chi2_cut > 0.f) ||
      !(cfg->dup_shared_frac >= 0.f) || cfg->n_eta_bins < 1 || cfg->n_eta_bins > MAX_ETA_BINS ||
      cfg->n_phi_bins < 1 ||
      (size_t)cfg->n_eta_bins * cfg->n_phi_bins > (1u << 24))
    return KF_ERR_ARG;
  int lanes = cfg->lanes_per_seed ? cfg->lanes_per_seed : auto_lanes(cfg->max_cands);
  if (!supported_lanes(lanes) || lanes < cfg->max_cands) return KF_ERR_ARG;
  int threads = cfg->block_threads ? cfg->block_threads : 128;
  if (threads < 32 || threads > 256 || threads % 32) return KF_ERR_ARG;
  if (cfg->find_regcap < 0 || cfg->find_regcap > 1 || (cfg->find_regcap && threads > 128)) return KF_ERR_ARG;
  auto cut_ok = [](float c) { return c >= 0.f && std::isfinite(c); };
  if (!cut_ok(cfg->dup_deta) || !cut_ok(cfg->dup_dphi) || !cut_ok(cfg->dup_dpt)) return KF_ERR_ARG;
  if (cfg->seed_clean < 0 || cfg->seed_clean > 1 || cfg->resolve_max_rounds < 0) return KF_ERR_ARG;
  if (cfg->seed_clean && (!(cfg->seed_deta > 0.f) || !(cfg->seed_deta <= KF_SEED_MAX_DETA) ||
                          !cut_ok(cfg->seed_dphi) || !cut_ok(cfg->seed_dpt) || cfg->seed_min_shared < 0 ||
                          cfg->seed_min_shared > 3))
    return KF_ERR_ARG;
  ctx = new kf_ctx();
  ctx->det = *det;
  ctx->cfg = *cfg;
  ctx->lanes = lanes;
  ctx->threads = threads;
  ctx->persistent = cfg->persistent ? 1 : 0;
  ctx->per_event = cfg->per_event ? 1 : 0;
  ctx->regcap = cfg->find_regcap;
  DevGeom& g = ctx->g;
  std::memset(&g, 0, sizeof(g));
  g.n_layers = det->n_layers;
  g.max_cands = cfg->max_cands;
  g.max_holes = cfg->max_holes;
  g.n_eta = cfg->n_eta_bins;
  g.n_phi = cfg->n_phi_bins;
  g.z_max = det->z_max;
  g.kb = -KCURV * det->bz;
  g.fcz = det->field_cz;
  g.fcr = det->field_cr;
  g.vr = det->sigma_rphi * det->sigma_rphi;
  g.vz = det->sigma_z * det->sigma_z;
  g.chi2_cut = cfg->chi2_cut;
  g.phi_scale = (float)cfg->n_phi_bins / TWO_PI_F;
  g.eta_lut_scale = (float)ETA_LUT / (2.f * det->z_max);
  g.n_disks = det->n_disks;
  g.n_surf = det->n_layers + 2 * det->n_disks;
  g.n_plan = det->n_layers + det->n_disks;
  if (det->n_disks > 0) {
    for (int k = 0; k < det->n_disks; ++k) g.disk_z[k] = det->disk_z[k];
    g.disk_rmin = det->disk_rmin;
    g.disk_rmax = det->disk_rmax;
    g.disk_x0 = det->disk_x0;
    g.disk_eloss = det->disk_eloss;
    g.vrr = det->sigma_r * det->sigma_r;
    g.disk_rscale = (float)cfg->n_eta_bins / (det->disk_rmax - det->disk_rmin);
    g.eta_barrel = det->eta_barrel;
  }
  for (int l = 0; l < det->n_layers; ++l) {
    g.radius[l] = det->radius[l];
    g.x0[l] = det->x0[l];
    g.eloss[l] = det->eloss[l];
    g.eta_max[l] = asinhf(det->z_max / det->radius[l]);
    g.eta_scale[l] = (float)cfg->n_eta_bins / (2.f * g.eta_max[l]);
    g.r_inv[l] = 1.f / det->radius[l];
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = find_prepare(ctx->lanes, ctx->regcap, ctx->threads, ctx->g, &ctx->blocks_per_sm);
  if (e == cudaSuccess) e = grow(ctx->align4, sizeof(Align4) * KF_MAX_LAYERS);
  if (e == cudaSuccess) {
    // z edges of the eta bins per layer: edge_k = R sinh(-eta_max + k * 2 eta_max / n_eta)
    std::vector<float> edges((size_t)KF_MAX_LAYERS * (MAX_ETA_BINS + 1), 0.f);
    for (int l = 0; l < det->n_layers; ++l) {
      const double R = det->radius[l], em = std::asinh((double)det->z_max / R);
      for (int k = 0; k <= cfg->n_eta_bins; ++k)
        edges[(size_t)l * (MAX_ETA_BINS + 1) + k] =
            (float)(R * std::sinh(-em + 2.0 * em * k / cfg->n_eta_bins));
    }
    e = grow(ctx->eta_edges, sizeof(float) * edges.size());
    if (e == cudaSuccess)
      e = cudaMemcpy(ctx->eta_edges.p, edges.data(), sizeof(float) * edges.size(), cudaMemcpyHostToDevice);
    // first guess of the bin per uniform z cell: the bin of the cell's lower end
    std::vector<unsigned char> lut((size_t)KF_MAX_LAYERS * ETA_LUT, 0);
    for (int l = 0; l < det->n_layers; ++l) {
      const float* ed = edges.data() + (size_t)l * (MAX_ETA_BINS + 1);
      int b = 0;
      for (int c = 0; c < ETA_LUT; ++c) {
        const float z = -det->z_max + (float)c / g.eta_lut_scale;
        while (b < cfg->n_eta_bins - 1 && z >= ed[b + 1]) ++b;
        lut[(size_t)l * ETA_LUT + c] = (unsigned char)b;
      }
    }
    if (e == cudaSuccess) e = grow(ctx->eta_lut, lut.size());
    if (e == cudaSuccess) e = cudaMemcpy(ctx->eta_lut.p, lut.data(), lut.size(), cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) e = grow(ctx->queue, 64);
  if (e == cudaSuccess) {
    int least = 0, greatest = 0;
    e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&ctx->side, cudaStreamNonBlocking, greatest);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = grow(ctx->counters, 8 * KF_N_COUNTERS);
  if (e == cudaSuccess) e = grow(ctx->status, 64);
  if (e == cudaSuccess) {
    k_align<<<1, KF_MAX_LAYERS>>>(nullptr, g, ptr<Align4>(ctx->align4));
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemset(ctx->status.p, 0, 64);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    kf_destroy(ctx);
    return KF_ERR_CUDA;
  }
  if (ctx->blocks_per_sm < 1) ctx->blocks_per_sm = 1;
  *out = ctx;
  return KF_OK;
}

// Every device buffer of a context.
static std::vector<DevBuf*> all_bufs(kf_ctx* ctx) {
  return {&ctx->hx, &ctx->hy, &ctx->hz, &ctx->hlayer, &ctx->hit_off, &ctx->seed_off, &ctx->sp,
                    &ctx->sc, &ctx->sh, &ctx->seed_event, &ctx->align_raw, &ctx->align4, &ctx->eta_edges, &ctx->eta_lut, &ctx->hb,
                    &ctx->bin_cnt, &ctx->bin_key, &ctx->bin_rank, &ctx->scan_tmp, &ctx->bin_grouped, &ctx->bin_gtab, &ctx->out_hits,
                    &ctx->out_n, &ctx->out_chi2, &ctx->out_p, &ctx->out_C, &ctx->keep, &ctx->queue, &ctx->tangent, &ctx->seed_order, &ctx->check,
                    &ctx->counters, &ctx->status, &ctx->dd_hit_cnt, &ctx->dd_owners, &ctx->dd_conf,
                    &ctx->dd_nconf, &ctx->dd_state, &ctx->dd_scan_tmp, &ctx->given_lists, &ctx->given_n, &ctx->fit_p,
                    &ctx->fit_C, &ctx->fit_chi2, &ctx->fit_status, &ctx->careful_list,
                    &ctx->careful_count, &ctx->adj_align_acc, &ctx->adj_align, &ctx->adj_hits,
                    &ctx->adj_seed, &ctx->careful_flag, &ctx->ckpt, &ctx->sc_kin, &ctx->sc_seed,
                    &ctx->clean_order, &ctx->kept_cnt, &ctx->sc_list, &ctx->sc_list_cnt, &ctx->sfit,
                    &ctx->sflag, &ctx->skeys, &ctx->x0map, &ctx->fit_order, &ctx->dbl_list};
}

int kf_destroy(kf_ctx* ctx) {
  if (!ctx) return KF_ERR_ARG;
  for (cudaEvent_t& e : ctx->ev)
    if (e) cudaEventDestroy(e);
  if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
  if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
  if (ctx->side) cudaStreamDestroy(ctx->side);
  if (ctx->exec) cudaGraphExecDestroy(ctx->exec);
  if (ctx->graph) cudaGraphDestroy(ctx->graph);
  for (DevBuf* b : all_bufs(ctx)) release(*b);
  delete ctx;
  return KF_OK;
}

int kf_load_hits(kf_ctx* ctx, int n_events, const int* ev_offsets, const float* x, const float* y,
                 const float* z, const int* layer, int device_ptrs, void* stream) {
  if (!ctx) return KF_ERR_ARG;
  if (n_events < 1 || !ev_offsets || !x || !y || !z || !layer)
    return fail(ctx, KF_ERR_ARG, "kf_load_hits: null argument or n_events < 1");
  if (ev_offsets[0] != 0) return fail(ctx, KF_ERR_ARG, "kf_load_hits: ev_offsets[0] must be 0");
  for (int e = 0; e < n_events; ++e) {
    const long long n = (long long)ev_offsets[e + 1] - ev_offsets[e];
    if (n < 0) return fail(ctx, KF_ERR_ARG, "kf_load_hits: decreasing ev_offsets");
    if (n > KF_MAX_EVENT_HITS) return fail(ctx, KF_ERR_CAPACITY, "kf_load_hits: event above KF_MAX_EVENT_HITS");
  }
  const int n = ev_offsets[n_events];
  const size_t nb = (size_t)ctx->g.n_eta * ctx->g.n_phi;
  const size_t n_bins = (size_t)n_events * ctx->g.n_surf * nb;
  if (n_bins >= 0xFFFFFFFFull) return fail(ctx, KF_ERR_CAPACITY, "kf_load_hits: too many hit-grid cells");
  cudaStream_t st = S(stream);
  CK(grow(ctx->hx, sizeof(float) * n));
  CK(grow(ctx->hy, sizeof(float) * n));
  CK(grow(ctx->hz, sizeof(float) * n));
  CK(grow(ctx->hlayer, sizeof(int) * n));
  CK(grow(ctx->hit_off, sizeof(int) * (n_events + 1)));
  CK(grow(ctx->hb, sizeof(float4) * n));
  CK(grow(ctx->bin_key, sizeof(unsigned) * n));
  CK(grow(ctx->bin_rank, sizeof(unsigned) * n));
  CK(grow(ctx->bin_cnt, sizeof(unsigned) * (n_bins + 1)));
  CK(grow(ctx->scan_tmp, sizeof(unsigned) * scan_tmp_elems(n_bins)));
  CK(grow(ctx->bin_grouped, sizeof(float4) * n));
  CK(grow(ctx->bin_gtab, sizeof(unsigned) * bin_group_elems(n_events, ctx->g.n_surf, ctx->g.n_eta, ctx->g.n_phi)));
  CK(grow(ctx->dd_hit_cnt, sizeof(unsigned) * ((size_t)n + n_events + 1)));
  CK(grow(ctx->dd_scan_tmp, sizeof(unsigned) * scan_tmp_elems((size_t)n + n_events)));
  CK(put(ctx->hx.p, x, sizeof(float) * n, device_ptrs, st));
  CK(put(ctx->hy.p, y, sizeof(float) * n, device_ptrs, st));
  CK(put(ctx->hz.p, z, sizeof(float) * n, device_ptrs, st));
  CK(put(ctx->hlayer.p, layer, sizeof(int) * n, device_ptrs, st));
  ctx->hit_off_h.assign(ev_offsets, ev_offsets + n_events + 1);
  CK(cudaMemcpyAsync(ctx->hit_off.p, ctx->hit_off_h.data(), sizeof(int) * (n_events + 1),
                     cudaMemcpyHostToDevice, st));
  ctx->found = ctx->deduped = ctx->fitted = false;
  // Seed hit indices were checked against the previous hit offsets: the seeds
  // must be loaded again before finding, fitting or tuning.
  ctx->n_seed_events = -1;
  // Layer indices checked on the device (the caller's buffers are in use until
  // the synchronization below).
  int bad = 0;
  CK(grow(ctx->check, 64));
  CK(cudaMemsetAsync(ctx->check.p, 0, sizeof(int), st));
  if (n > 0) {
    k_check_range<<<std::min((n + 255) / 256, 4 * ctx->num_sms), 256, 0, st>>>(ptr<int>(ctx->hlayer), n,
                                                                               ctx->g.n_surf, ptr<int>(ctx->check));
    CK(cudaGetLastError());
  }
  CK(cudaMemcpyAsync(&bad, ctx->check.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (bad) {
    ctx->n_events = 0;
    ctx->n_hits = -1;
    return fail(ctx, KF_ERR_ARG, "kf_load_hits: layer index out of range");
  }
  ctx->n_events = n_events;
  ctx->n_hits = n;
  ctx->n_bins_total = n_bins;
  ctx->max_event_hits = 0;
  for (int e = 0; e < n_events; ++e)
    ctx->max_event_hits = std::max(ctx->max_event_hits, ev_offsets[e + 1] - ev_offsets[e]);
  return KF_OK;
}

int kf_load_seeds(kf_ctx* ctx, int n_events, const int* ev_offsets, const float* params, const float* cov,
                  const int* seed_hits, int device_ptrs, void* stream) {
  if (!ctx) return KF_ERR_ARG;
  if (n_events < 1 || !ev_offsets || !params || !cov || !seed_hits)
    return fail(ctx, KF_ERR_ARG, "kf_load_seeds: null argument");
  if (n_events != ctx->n_events) return fail(ctx, KF_ERR_STATE, "kf_load_seeds: load hits of the same events first");
  if (ev_offsets[0] != 0) return fail(ctx, KF_ERR_ARG, "kf_load_seeds: ev_offsets[0] must be 0");
  for (int e = 0; e < n_events; ++e)
    if (ev_offsets[e + 1] < ev_offsets[e]) return fail(ctx, KF_ERR_ARG, "kf_load_seeds: decreasing ev_offsets");
  const int n = ev_offsets[n_events];
  cudaStream_t st = S(stream);
  const int L = ctx->g.n_surf;  // hit-list row: one entry per surface at most
  CK(grow(ctx->sp, sizeof(float) * 6 * (size_t)n));
  CK(grow(ctx->sc, sizeof(float) * 21 * (size_t)n));
  CK(grow(ctx->sh, sizeof(int) * 3 * (size_t)n));
  CK(grow(ctx->seed_event, sizeof(int) * (size_t)n));
  CK(grow(ctx->seed_off, sizeof(int) * (n_events + 1)));
  CK(grow(ctx->out_hits, sizeof(int) * (size_t)n * L));
  CK(grow(ctx->out_n, sizeof(int) * (size_t)n));
  CK(grow(ctx->tangent, sizeof(int) * (size_t)n));
  CK(grow(ctx->seed_order, sizeof(int) * (size_t)n));
  CK(grow(ctx->sfit, sizeof(float) * 29 * (size_t)n));
  CK(grow(ctx->sflag, (size_t)n));
  CK(grow(ctx->skeys, sizeof(unsigned long long) * ctx->g.max_cands * (size_t)n));
  CK(grow(ctx->out_chi2, sizeof(float) * (size_t)n));
  CK(grow(ctx->out_p, sizeof(float) * 6 * (size_t)n));
  CK(grow(ctx->out_C, sizeof(float) * 21 * (size_t)n));
  CK(grow(ctx->keep, (size_t)n));
  CK(grow(ctx->dd_owners, sizeof(int) * (size_t)n * L));
  CK(grow(ctx->dd_conf, sizeof(int) * (size_t)n * DEDUP_CONF_CAP));
  CK(grow(ctx->dd_nconf, sizeof(int) * (size_t)n));
  CK(grow(ctx->dd_state, (size_t)n));
  CK(grow(ctx->fit_p, sizeof(float) * 6 * (size_t)n));
  CK(grow(ctx->fit_C, sizeof(float) * 21 * (size_t)n));
  CK(grow(ctx->fit_chi2, sizeof(float) * (size_t)n));
  CK(grow(ctx->fit_status, sizeof(int) * (size_t)n));
  CK(grow(ctx->careful_list, sizeof(int) * (size_t)n));
  CK(grow(ctx->careful_count, 64));
  CK(grow(ctx->careful_flag, (size_t)n));
  CK(grow(ctx->fit_order, sizeof(int) * (size_t)n));
  CK(grow(ctx->dbl_list, sizeof(int) * (size_t)n));
  if (ctx->cfg.seed_clean) {
    CK(grow(ctx->sc_kin, sizeof(float4) * (size_t)n));
    CK(grow(ctx->sc_seed, sizeof(int4) * (size_t)n));
    CK(grow(ctx->clean_order, sizeof(int) * (size_t)n));
    CK(grow(ctx->kept_cnt, sizeof(int) * (size_t)n_events));
    CK(grow(ctx->sc_list, sizeof(int) * (size_t)n));
    CK(grow(ctx->sc_list_cnt, sizeof(int) * (size_t)n_events));
  }
  CK(put(ctx->sp.p, params, sizeof(float) * 6 * (size_t)n, device_ptrs, st));
  CK(put(ctx->sc.p, cov, sizeof(float) * 21 * (size_t)n, device_ptrs, st));
  CK(put(ctx->sh.p, seed_hits, sizeof(int) * 3 * (size_t)n, device_ptrs, st));
  ctx->seed_off_h.assign(ev_offsets, ev_offsets + n_events + 1);
  CK(cudaMemcpyAsync(ctx->seed_off.p, ctx->seed_off_h.data(), sizeof(int) * (n_events + 1),
                     cudaMemcpyHostToDevice, st));
  if (n > 0) {
    k_seed_event<<<(n + 255) / 256, 256, 0, st>>>(ptr<int>(ctx->seed_off), n_events, n, ptr<int>(ctx->seed_event));
    CK(cudaGetLastError());
    CK(launch_seed_order(ptr<float>(ctx->sp) + 5 * (size_t)n, ptr<int>(ctx->seed_off), n_events,
                         ptr<int>(ctx->seed_order), st));
  }
  CK(cudaMemsetAsync(ctx->keep.p, 1, (size_t)n, st));
  ctx->found = ctx->deduped = ctx->fitted = false;
  // Seed hit indices checked on the device against their event's hits.
  int bad = 0;
  CK(grow(ctx->check, 64));
  CK(cudaMemsetAsync(ctx->check.p, 0, sizeof(int), st));
  if (n > 0) {
    k_check_seed_hits<<<std::min((n + 255) / 256, 4 * ctx->num_sms), 256, 0, st>>>(
        ptr<int>(ctx->sh), ptr<int>(ctx->seed_event), ptr<int>(ctx->hit_off), ptr<int>(ctx->hlayer),
        ctx->g.n_layers, n, ptr<int>(ctx->check));
    CK(cudaGetLastError());
  }
  CK(cudaMemcpyAsync(&bad, ctx->check.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (bad) {
    ctx->n_seed_events = -1;
    return fail(ctx, KF_ERR_ARG, bad == 1 ? "kf_load_seeds: seed hit index out of range"
                                          : "kf_load_seeds: seed hits must lie on barrel layers");
  }
  ctx->n_seeds = n;
  ctx->n_seed_events = n_events;
  return KF_OK;
}

int kf_set_material(kf_ctx* ctx, int n_z, const float* x0_map, int device_ptrs, void* stream) {
  if (!ctx) return KF_ERR_ARG;
  if (n_z == 0) {
    ctx->g.x0map = nullptr;
    ctx->g.n_z = 0;
    ctx->g.z_node_inv = 0.f;
  } else {
    if (n_z < 2 || n_z > KF_MAX_MATERIAL_NODES || !x0_map)
      return fail(ctx, KF_ERR_ARG, "kf_set_material: 2 <= n_z <= KF_MAX_MATERIAL_NODES and a map are required");
    const size_t n = (size_t)ctx->g.n_layers * n_z;
    if (!device_ptrs)
      for (size_t i = 0; i < n; ++i)
        if (!(x0_map[i] >= 0.f) || !std::isfinite(x0_map[i]))
          return fail(ctx, KF_ERR_ARG, "kf_set_material: thickness must be finite and >= 0");
    cudaStream_t st = S(stream);
    CK(grow(ctx->x0map, sizeof(float) * n));
    CK(put(ctx->x0map.p, x0_map, sizeof(float) * n, device_ptrs, st));
    if (!device_ptrs) CK(cudaStreamSynchronize(st));
    ctx->g.x0map = ptr<float>(ctx->x0map);
    ctx->g.n_z = n_z;
    ctx->g.z_node_inv = (float)(n_z - 1) / (2.f * ctx->g.z_max);
  }
  // the graph's kernels hold the old geometry
  if (ctx->exec) { cudaGraphExecDestroy(ctx->exec); ctx->exec = nullptr; }
  if (ctx->graph) { cudaGraphDestroy(ctx->graph); ctx->graph = nullptr; }
  return KF_OK;
}

int kf_set_alignment(kf_ctx* ctx, const float* offsets, int device_ptrs, void* stream) {
  if (!ctx) return KF_ERR_ARG;
  cudaStream_t st = S(stream);
  const int L = ctx->g.n_layers;
  CK(grow(ctx->align_raw, sizeof(float) * 2 * KF_MAX_LAYERS));
  if (offsets) CK(put(ctx->align_raw.p, offsets, sizeof(float) * 2 * L, device_ptrs, st));
  k_align<<<1, KF_MAX_LAYERS, 0, st>>>(offsets ? ptr<float>(ctx->align_raw) : nullptr, ctx->g,
                                       ptr<Align4>(ctx->align4));
  CK(cudaGetLastError());
  if (!device_ptrs) CK(cudaStreamSynchronize(st));
  return KF_OK;
}

static void stage_mark(kf_ctx* ctx, int i, cudaStream_t st) {
  if (!ctx->stage_timing || !ctx->ev[i]) return;
  // Inside stream capture an external record becomes an event-record node;
  // outside capture it is a plain record.
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(st, &cs);
  if (cs == cudaStreamCaptureStatusActive) cudaEventRecordWithFlags(ctx->ev[i], st, cudaEventRecordExternal);
  else cudaEventRecord(ctx->ev[i], st);
}

// Work on ctx->side after everything enqueued so far on st (fork), and st
// after everything enqueued on ctx->side (join).  Inside a stream capture the
// side stream joins the capture and becomes a parallel branch of the graph.
static cudaError_t fork_side(kf_ctx* ctx, cudaStream_t st) {
  cudaError_t e = cudaEventRecord(ctx->ev_fork, st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->side, ctx->ev_fork, 0);
  return e;
}
static cudaError_t join_side(kf_ctx* ctx, cudaStream_t st) {
  cudaError_t e = cudaEventRecord(ctx->ev_join, ctx->side);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ctx->ev_join, 0);
  return e;
}

static FindParams find_params(kf_ctx* ctx) {
  FindParams P;
  P.g = ctx->g;
  P.hx = ptr<float>(ctx->hx);
  P.hy = ptr<float>(ctx->hy);
  P.hz = ptr<float>(ctx->hz);
  P.hlayer = ptr<int>(ctx->hlayer);
  P.hit_off = ptr<int>(ctx->hit_off);
  P.hb = ptr<float4>(ctx->hb);
  P.bin_off = ptr<unsigned>(ctx->bin_cnt);
  P.eta_edges = ptr<float>(ctx->eta_edges);
  P.eta_lut = ptr<unsigned char>(ctx->eta_lut);
  P.sp = ptr<float>(ctx->sp);
  P.sc = ptr<float>(ctx->sc);
  P.sh = ptr<int>(ctx->sh);
  P.seed_event = ptr<int>(ctx->seed_event);
  P.align = ptr<Align4>(ctx->align4);
  P.ns = ctx->n_seeds;
  P.s_begin = 0;
  P.s_end = ctx->n_seeds;
  P.out_hits = ptr<int>(ctx->out_hits);
  P.out_n = ptr<int>(ctx->out_n);
  P.out_chi2 = ptr<float>(ctx->out_chi2);
  P.out_p = ptr<float>(ctx->out_p);
  P.out_C = ptr<float>(ctx->out_C);
  P.queue = ptr<unsigned>(ctx->queue);
  P.tangent_list = ptr<int>(ctx->tangent);
  P.sfit = ptr<float>(ctx->sfit);
  P.sflag = ptr<unsigned char>(ctx->sflag);
  P.skeys = ptr<unsigned long long>(ctx->skeys);
  P.order = ptr<int>(ctx->seed_order);
  P.seed_off = ptr<int>(ctx->seed_off);
  P.kept_cnt = nullptr;
  P.counters = ptr<unsigned long long>(ctx->counters);
  P.persistent = ctx->persistent;
  return P;
}

static SeedCleanParams clean_params(kf_ctx* ctx) {
  SeedCleanParams C;
  C.kb = ctx->g.kb;
  C.sp = ptr<float>(ctx->sp);
  C.sc = ptr<float>(ctx->sc);
  C.sh = ptr<int>(ctx->sh);
  C.seed_off = ptr<int>(ctx->seed_off);
  C.seed_event = ptr<int>(ctx->seed_event);
  C.order = ptr<int>(ctx->seed_order);
  C.ns = ctx->n_seeds;
  C.L = ctx->g.n_surf;
  C.deta = ctx->cfg.seed_deta;
  C.dphi = ctx->cfg.seed_dphi;
  C.dpt = ctx->cfg.seed_dpt;
  C.min_shared = ctx->cfg.seed_min_shared;
  C.kin = ptr<float4>(ctx->sc_kin);
  C.kseed = ptr<int4>(ctx->sc_seed);
  C.conf = ptr<int>(ctx->dd_conf);
  C.n_conf = ptr<int>(ctx->dd_nconf);
  C.state = ptr<unsigned char>(ctx->dd_state);
  C.list = ptr<int>(ctx->sc_list);
  C.list_cnt = ptr<int>(ctx->sc_list_cnt);
  C.clean_order = ptr<int>(ctx->clean_order);
  C.kept_cnt = ptr<int>(ctx->kept_cnt);
  C.out_hits = ptr<int>(ctx->out_hits);
  C.out_n = ptr<int>(ctx->out_n);
  C.out_chi2 = ptr<float>(ctx->out_chi2);
  C.out_p = ptr<float>(ctx->out_p);
  C.out_C = ptr<float>(ctx->out_C);
  C.keep = ptr<unsigned char>(ctx->keep);
  C.status = ptr<int>(ctx->status);
  C.max_rounds = ctx->cfg.resolve_max_rounds;
  return C;
}

static BinParams bin_params(kf_ctx* ctx) {
  BinParams B;
  B.g = ctx->g;
  B.hx = ptr<float>(ctx->hx);
  B.hy = ptr<float>(ctx->hy);
  B.hz = ptr<float>(ctx->hz);
  B.hlayer = ptr<int>(ctx->hlayer);
  B.hit_off = ptr<int>(ctx->hit_off);
  B.n_events = ctx->n_events;
  B.h_begin = 0;
  B.h_end = ctx->n_hits;
  B.cnt = ptr<unsigned>(ctx->bin_cnt);
  B.key = ptr<unsigned>(ctx->bin_key);
  B.rank = ptr<unsigned>(ctx->bin_rank);
  B.hb = ptr<float4>(ctx->hb);
  B.grouped = ptr<float4>(ctx->bin_grouped);
  B.gtab = ptr<unsigned>(ctx->bin_gtab);
  B.eta_edges = ptr<float>(ctx->eta_edges);
  B.eta_lut = ptr<unsigned char>(ctx->eta_lut);
  return B;
}

// Blocks of the careful pass over the seeds the main pass gave up (a few
// percent, 12 per block and round; two blocks fit an SM): enough for all of
// them in about one round, at most two blocks per SM.
static int careful_grid(const kf_ctx* ctx, int n_seeds) {
  return std::max(1, std::min(2 * ctx->num_sms, (n_seeds / 50 + 11) / 12));
}

int kf_find_tracks(kf_ctx* ctx, void* stream) {
  if (!ctx) return KF_ERR_ARG;
  if (ctx->n_hits < 0 || ctx->n_seed_events != ctx->n_events || ctx->n_events < 1)
    return fail(ctx, KF_ERR_STATE, "kf_find_tracks: load hits and seeds first");
  cudaStream_t st = S(stream);
  const size_t cells = (size_t)ctx->g.n_surf * ctx->g.n_eta * ctx->g.n_phi;
  CK(cudaMemsetAsync(ctx->counters.p, 0, 8 * KF_N_COUNTERS, st));
  CK(cudaMemsetAsync(ctx->keep.p, 1, (size_t)ctx->n_seeds, st));
  const int grid_cap = ctx->num_sms * ctx->blocks_per_sm;
  if (!ctx->per_event) {
    BinParams B = bin_params(ctx);
    stage_mark(ctx, 0, st);
    CK(launch_bin(B, 0, ctx->n_bins_total, 0u, ctx->max_event_hits, ptr<unsigned>(ctx->scan_tmp),
                  ctx->scan_tmp.bytes / sizeof(unsigned), st));
    stage_mark(ctx, 1, st);
    FindParams P = find_params(ctx);
    if (ctx->cfg.seed_clean) {
      stage_mark(ctx, 10, st);
      CK(launch_seed_clean(clean_params(ctx), 0, ctx->n_seeds, 0, ctx->n_events, st));
      stage_mark(ctx, 11, st);
      P.order = ptr<int>(ctx->clean_order);
      P.kept_cnt = ptr<int>(ctx->kept_cnt);
    }
    CK(cudaMemsetAsync(ctx->queue.p, 0, 64, st));
    stage_mark(ctx, 2, st);
    CK(launch_find_main(P, ctx->lanes, ctx->regcap, ctx->threads, grid_cap, st));
    CK(launch_find_careful(P, ctx->lanes, careful_grid(ctx, P.s_end - P.s_begin), st));
    stage_mark(ctx, 3, st);
  } else {
    for (int e = 0; e < ctx->n_events; ++e) {
      BinParams B = bin_params(ctx);
      B.h_begin = ctx->hit_off_h[e];
      B.h_end = ctx->hit_off_h[e + 1];
      CK(launch_bin(B, (size_t)e * cells, cells, (unsigned)ctx->hit_off_h[e],
                    ctx->hit_off_h[e + 1] - ctx->hit_off_h[e], ptr<unsigned>(ctx->scan_tmp),
                    ctx->scan_tmp.bytes / sizeof(unsigned), st));
      FindParams P = find_params(ctx);
      P.s_begin = ctx->seed_off_h[e];
      P.s_end = ctx->seed_off_h[e + 1];
      if (ctx->cfg.seed_clean) {
        CK(launch_seed_clean(clean_params(ctx), P.s_begin, P.s_end, e, 1, st));
        P.order = ptr<int>(ctx->clean_order);
        P.kept_cnt = ptr<int>(ctx->kept_cnt);
      }
      CK(cudaMemsetAsync(ctx->queue.p, 0, 64, st));
      CK(launch_find_main(P, ctx->lanes, ctx->regcap, ctx->threads, grid_cap, st));
      CK(launch_find_careful(P, ctx->lanes, careful_grid(ctx, P.s_end - P.s_begin), st));
    }
  }
  ctx->found = true;
  ctx->deduped = false;
  return KF_OK;
}

int kf_remove_duplicates(kf_ctx* ctx, void* stream) {
  if (!ctx) return KF_ERR_ARG;
  if (!ctx->found) return fail(ctx, KF_ERR_STATE, "kf_remove_duplicates: run kf_find_tracks first");
  cudaStream_t st = S(stream);
  DedupParams D;
  D.out_hits = ptr<int>(ctx->out_hits);
  D.out_n = ptr<int>(ctx->out_n);
  D.out_chi2 = ptr<float>(ctx->out_chi2);
  D.hit_off = ptr<int>(ctx->hit_off);
  D.seed_off = ptr<int>(ctx->seed_off);
  D.seed_event = ptr<int>(ctx->seed_event);
  D.L = ctx->g.n_surf;
  D.ns = ctx->n_seeds;
  D.frac = ctx->cfg.dup_shared_frac;
  D.e_begin = 0;
  D.hit_cnt = ptr<unsigned>(ctx->dd_hit_cnt);
  D.owners = ptr<int>(ctx->dd_owners);
  D.conf = ptr<int>(ctx->dd_conf);
  D.n_conf = ptr<int>(ctx->dd_nconf);
  D.state = ptr<unsigned char>(ctx->dd_state);
  D.keep = ptr<unsigned char>(ctx->keep);
  D.status = ptr<int>(ctx->status);
  D.max_rounds = ctx->cfg.resolve_max_rounds;
  if (ctx->cfg.dup_deta > 0.f || ctx->cfg.dup_dphi > 0.f || ctx->cfg.dup_dpt > 0.f) {
    D.trk_p = ptr<float>(ctx->out_p);
    D.kb = ctx->g.kb;
    D.deta = ctx->cfg.dup_deta;
    D.dphi = ctx->cfg.dup_dphi;
    D.dpt = ctx->cfg.dup_dpt;
  }
  if (!ctx->per_event) {
    stage_mark(ctx, 4, st);
    CK(launch_dedup_batched(D, ctx->n_events, ctx->n_hits, ptr<unsigned>(ctx->dd_scan_tmp),
                            ctx->dd_scan_tmp.bytes / sizeof(unsigned), st));
    stage_mark(ctx, 5, st);
  } else {
    for (int e = 0; e < ctx->n_events; ++e) {
      D.e_begin = e;
      CK(launch_dedup(D, 1, st));
    }
  }
  ctx->deduped = true;
  return KF_OK;
}

int kf_fit_tracks(kf_ctx* ctx, int source, const int* hit_lists, const int* n_hits, int max_len,
                  int device_ptrs, void* stream) {
  if (!ctx) return KF_ERR_ARG;
  if (ctx->n_seeds < 0 || ctx->n_seed_events != ctx->n_events)
    return fail(ctx, KF_ERR_STATE, "kf_fit_tracks: load hits and seeds first");
  cudaStream_t st = S(stream);
  FitParams F;
  F.g = ctx->g;
  F.hx = ptr<float>(ctx->hx);
  F.hy = ptr<float>(ctx->hy);
  F.hz = ptr<float>(ctx->hz);
  F.hlayer = ptr<int>(ctx->hlayer);
  F.hit_off = ptr<int>(ctx->hit_off);
  F.sp = ptr<float>(ctx->sp);
  F.sc = ptr<float>(ctx->sc);
  F.seed_event = ptr<int>(ctx->seed_event);
  F.align = ptr<Align4>(ctx->align4);
  F.ns = ctx->n_seeds;
  F.fit_p = ptr<float>(ctx->fit_p);
  F.fit_C = ptr<float>(ctx->fit_C);
  F.fit_chi2 = ptr<float>(ctx->fit_chi2);
  F.fit_status = ptr<int>(ctx->fit_status);
  F.careful_list = ptr<int>(ctx->careful_list);
  F.careful_count = ptr<unsigned>(ctx->careful_count);
  F.careful_flag = ptr<unsigned char>(ctx->careful_flag);
  F.order = ptr<int>(ctx->fit_order);
  F.dbl_list = ptr<int>(ctx->dbl_list);
  F.dbl_count = ptr<unsigned>(ctx->careful_count) + 1;
  F.ckpt_stride = ctx->cfg.ckpt_stride > 0 ? ctx->cfg.ckpt_stride : DEFAULT_CKPT_STRIDE;
  F.ckpt = nullptr;
  F.ckpt_slices = 0;
  if (source == KF_FIT_FOUND) {
    if (!ctx->found) return fail(ctx, KF_ERR_STATE, "kf_fit_tracks: no found tracks");
    F.lists = ptr<int>(ctx->out_hits);
    F.n_list = ptr<int>(ctx->out_n);
    F.max_len = ctx->g.n_surf;
    F.keep = ctx->deduped || ctx->fit_beside_dedup ? ptr<unsigned char>(ctx->keep) : nullptr;
    F.keep_in_main = !ctx->fit_beside_dedup;
  } else if (source == KF_FIT_GIVEN) {
    if (!hit_lists || !n_hits || max_len < 1) return fail(ctx, KF_ERR_ARG, "kf_fit_tracks: missing hit lists");
    const size_t n = (size_t)ctx->n_seeds;
    if (!device_ptrs) {
      for (size_t s = 0; s < n; ++s) {
        if (n_hits[s] < 1 || n_hits[s] > max_len) return fail(ctx, KF_ERR_ARG, "kf_fit_tracks: bad hit count");
        const int e = (int)(std::upper_bound(ctx->seed_off_h.begin(), ctx->seed_off_h.end(), (int)s) -
                            ctx->seed_off_h.begin()) - 1;
        const int nh = ctx->hit_off_h[e + 1] - ctx->hit_off_h[e];
        for (int k = 0; k < n_hits[s]; ++k) {
          const int h = hit_lists[s * max_len + k];
          if (h < 0 || h >= nh) return fail(ctx, KF_ERR_ARG, "kf_fit_tracks: hit index out of range");
        }
      }
    }
    CK(grow(ctx->given_lists, sizeof(int) * n * max_len));
    CK(grow(ctx->given_n, sizeof(int) * n));
    CK(put(ctx->given_lists.p, hit_lists, sizeof(int) * n * max_len, device_ptrs, st));
    CK(put(ctx->given_n.p, n_hits, sizeof(int) * n, device_ptrs, st));
    F.lists = ptr<int>(ctx->given_lists);
    F.n_list = ptr<int>(ctx->given_n);
    F.max_len = max_len;
    F.keep = nullptr;
    ctx->given_max_len = max_len;
    if (!device_ptrs) CK(cudaStreamSynchronize(st));
  } else {
    return fail(ctx, KF_ERR_ARG, "kf_fit_tracks: unknown source");
  }
  if (ctx->want_ckpt) {  // checkpoints for the adjoint
    F.ckpt_slices = ckpt_slices_for(F.max_len, F.ckpt_stride);
    CK(grow(ctx->ckpt, sizeof(float) * (size_t)F.ckpt_slices * 27 * (size_t)ctx->n_seeds));
    F.ckpt = ptr<float>(ctx->ckpt);
  }
  stage_mark(ctx, 6, st);
  if (ctx->defer_careful_fit || ctx->fit_beside_dedup) {
    CK(launch_fit_main(F, st));
    ctx->careful_fit_pending = true;
  } else {
    CK(launch_fit(F, st));
    ctx->careful_fit_pending = false;
  }
  stage_mark(ctx, 7, st);
  ctx->last_fit = F;
  ctx->fitted = true;
  ctx->fit_source = source;
  return KF_OK;
}

int kf_fit_adjoint(kf_ctx* ctx, float* g_align, float* g_hits, float* g_seed, int device_ptrs, void* stream) {
  if (!ctx) return KF_ERR_ARG;
  if (!ctx->fitted) return fail(ctx, KF_ERR_STATE, "kf_fit_adjoint: run kf_fit_tracks first");
  if (!g_align) return fail(ctx, KF_ERR_ARG, "kf_fit_adjoint: g_align is required");
  const int stride = ctx->cfg.ckpt_stride > 0 ? ctx->cfg.ckpt_stride : DEFAULT_CKPT_STRIDE;
  if (!adjoint_stride_ok(stride, ctx->last_fit.max_len))
    return fail(ctx, KF_ERR_CAPACITY, "kf_fit_adjoint: ckpt_stride must be 1..8 with hits per track <= 32 * stride");
  cudaStream_t st = S(stream);
  if (!ctx->last_fit.ckpt) {  // the last fit kept no checkpoints: refit with them (same lists)
    ctx->want_ckpt = true;
    ctx->last_fit.ckpt_stride = stride;
    ctx->last_fit.ckpt_slices = ckpt_slices_for(ctx->last_fit.max_len, stride);
    CK(grow(ctx->ckpt, sizeof(float) * (size_t)ctx->last_fit.ckpt_slices * 27 * (size_t)ctx->n_seeds));
    ctx->last_fit.ckpt = ptr<float>(ctx->ckpt);
    CK(launch_fit_main(ctx->last_fit, st));
    ctx->careful_fit_pending = true;
  }
  const FitParams& F = ctx->last_fit;
  const size_t ns = (size_t)ctx->n_seeds, nh = (size_t)ctx->n_hits;
  CK(grow(ctx->adj_align_acc, sizeof(double) * 2 * KF_MAX_LAYERS));
  CK(grow(ctx->adj_align, sizeof(float) * 2 * KF_MAX_LAYERS));
  // The hit gradient is always formed (the alignment gradient is summed from
  // it); without a device array from the caller it goes to the context.
  const bool own_hits = !(device_ptrs && g_hits);
  if (own_hits) CK(grow(ctx->adj_hits, sizeof(float) * 3 * nh));
  if (!device_ptrs && g_seed) CK(grow(ctx->adj_seed, sizeof(float) * 6 * ns));
  AdjParams A;
  A.g = ctx->g;
  A.hx = F.hx;
  A.hy = F.hy;
  A.hz = F.hz;
  A.hlayer = F.hlayer;
  A.hit_off = F.hit_off;
  A.sp = F.sp;
  A.sc = F.sc;
  A.seed_event = F.seed_event;
  A.align = F.align;
  A.ns = F.ns;
  A.n_hits = ctx->n_hits;
  A.lists = F.lists;
  A.n_list = F.n_list;
  A.max_len = F.max_len;
  A.keep = F.keep;
  A.fit_status = F.fit_status;
  A.stride = stride;
  A.g_hits = own_hits ? ptr<float>(ctx->adj_hits) : g_hits;
  A.g_seed = g_seed ? (device_ptrs ? g_seed : ptr<float>(ctx->adj_seed)) : nullptr;
  A.g_align = device_ptrs ? g_align : ptr<float>(ctx->adj_align);
  A.g_align_acc = ptr<double>(ctx->adj_align_acc);
  A.careful_list = F.careful_list;
  A.careful_count = F.careful_count;
  A.careful_flag = F.careful_flag;
  A.dbl_list = F.dbl_list;
  A.dbl_count = F.dbl_count;
  A.ckpt = F.ckpt;
  A.order = F.order;
  stage_mark(ctx, 8, st);
  CK(launch_adjoint_begin(A, st));
  CK(fork_side(ctx, st));
  // the careful tracks beside the FP32 pass: their fit (if still to run),
  // then their adjoint
  if (ctx->careful_fit_pending) CK(launch_fit_careful(F, ctx->side));
  ctx->careful_fit_pending = false;
  CK(launch_adjoint_pass(A, true, ctx->side));
  CK(launch_adjoint_pass(A, false, st));
  CK(join_side(ctx, st));
  CK(launch_adjoint_end(A, st));
  stage_mark(ctx, 9, st);
  if (!device_ptrs) {
    CK(cudaMemcpyAsync(g_align, A.g_align, sizeof(float) * 2 * ctx->g.n_layers, cudaMemcpyDeviceToHost, st));
    if (g_hits) CK(cudaMemcpyAsync(g_hits, A.g_hits, sizeof(float) * 3 * nh, cudaMemcpyDeviceToHost, st));
    if (g_seed) CK(cudaMemcpyAsync(g_seed, A.g_seed, sizeof(float) * 6 * ns, cudaMemcpyDeviceToHost, st));
    return check_status_sync(ctx, st);
  }
  return KF_OK;
}


int kf_sync(kf_ctx* ctx, void* stream) {
  if (!ctx) return KF_ERR_ARG;
  cudaStream_t st = S(stream);
  CK(cudaStreamSynchronize(st));
  return check_status(ctx, st);
}

int kf_get_tracks(kf_ctx* ctx, int* hits, int* n_found, float* chi2, float* params, float* cov,
                  unsigned char* keep, int device_ptrs, void* stream) {
  if (!ctx) return KF_ERR_ARG;
  if (!ctx->found) return fail(ctx, KF_ERR_STATE, "kf_get_tracks: run kf_find_tracks first");
  cudaStream_t st = S(stream);
  const size_t n = (size_t)ctx->n_seeds, L = (size_t)ctx->g.n_surf;
  if (hits) CK(get(hits, ctx->out_hits.p, sizeof(int) * n * L, device_ptrs, st));
  if (n_found) CK(get(n_found, ctx->out_n.p, sizeof(int) * n, device_ptrs, st));
  if (chi2) CK(get(chi2, ctx->out_chi2.p, sizeof(float) * n, device_ptrs, st));
  if (params) CK(get(params, ctx->out_p.p, sizeof(float) * 6 * n, device_ptrs, st));
  if (cov) CK(get(cov, ctx->out_C.p, sizeof(float) * 21 * n, device_ptrs, st));
  if (keep) CK(get(keep, ctx->keep.p, n, device_ptrs, st));
  if (!device_ptrs) return check_status(ctx, st);
  return KF_OK;
}

int kf_get_fit(kf_ctx* ctx, float* params, float* cov, float* chi2, int* status, int device_ptrs, void* stream) {
  if (!ctx) return KF_ERR_ARG;
  if (!ctx->fitted) return fail(ctx, KF_ERR_STATE, "kf_get_fit: run kf_fit_tracks first");
  cudaStream_t st = S(stream);
  const size_t n = (size_t)ctx->n_seeds;
  if (params) CK(get(params, ctx->fit_p.p, sizeof(float) * 6 * n, device_ptrs, st));
  if (cov) CK(get(cov, ctx->fit_C.p, sizeof(float) * 21 * n, device_ptrs, st));
  if (chi2) CK(get(chi2, ctx->fit_chi2.p, sizeof(float) * n, device_ptrs, st));
  if (status) CK(get(status, ctx->fit_status.p, sizeof(int) * n, device_ptrs, st));
  if (!device_ptrs) return check_status(ctx, st);
  return KF_OK;
}

int kf_get_counters(kf_ctx* ctx, long long* counters8, void* stream) { return kf_get_counters_n(ctx, counters8, 8, stream); }

int kf_get_counters_n(kf_ctx* ctx, long long* counters, int n, void* stream) {
  if (!ctx || !counters || n < 1 || n > KF_N_COUNTERS) return KF_ERR_ARG;
  cudaStream_t st = S(stream);
  CK(cudaMemcpyAsync(counters, ctx->counters.p, (size_t)n * sizeof(long long), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return KF_OK;
}

int kf_set_stage_timing(kf_ctx* ctx, int enable) {
  if (!ctx) return KF_ERR_ARG;
  if (enable)
    for (cudaEvent_t& e : ctx->ev)
      if (!e) CK(cudaEventCreate(&e));
  ctx->stage_timing = enable ? 1 : 0;
  return KF_OK;
}

int kf_get_stage_ms(kf_ctx* ctx, float* ms6, void* stream) {
  if (!ctx || !ms6) return KF_ERR_ARG;
  if (!ctx->stage_timing) return fail(ctx, KF_ERR_STATE, "kf_get_stage_ms: stage timing is off");
  CK(cudaStreamSynchronize(S(stream)));
  for (int k = 0; k < 6; ++k) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, ctx->ev[2 * k], ctx->ev[2 * k + 1]) != cudaSuccess) ms = -1.f;
    ms6[k] = ms;
  }
  cudaGetLastError();  // an event that never ran leaves a benign error
  return KF_OK;
}

int kf_graph_kernel_count(kf_ctx* ctx, int* n_kernels) {
  if (!ctx || !n_kernels) return KF_ERR_ARG;
  if (!ctx->graph) return fail(ctx, KF_ERR_STATE, "kf_graph_kernel_count: capture a graph first");
  size_t n = 0;
  CK(cudaGraphGetNodes(ctx->graph, nullptr, &n));
  std::vector<cudaGraphNode_t> nodes(n);
  CK(cudaGraphGetNodes(ctx->graph, nodes.data(), &n));
  int k = 0;
  for (size_t i = 0; i < n; ++i) {
    cudaGraphNodeType t;
    CK(cudaGraphNodeGetType(nodes[i], &t));
    if (t == cudaGraphNodeTypeKernel) ++k;
  }
  *n_kernels = k;
  return KF_OK;
}

int kf_capture_graph(kf_ctx* ctx, int with_adjoint, void* stream) {
  if (!ctx) return KF_ERR_ARG;
  cudaStream_t st = S(stream);
  if (!st) return fail(ctx, KF_ERR_ARG, "kf_capture_graph: capture needs a non-default stream");
  if (ctx->exec) { cudaGraphExecDestroy(ctx->exec); ctx->exec = nullptr; }
  if (ctx->graph) { cudaGraphDestroy(ctx->graph); ctx->graph = nullptr; }
  if (with_adjoint) {  // every buffer the captured work uses exists before capture starts
    ctx->want_ckpt = true;
    const int stride = ctx->cfg.ckpt_stride > 0 ? ctx->cfg.ckpt_stride : DEFAULT_CKPT_STRIDE;
    CK(grow(ctx->ckpt, sizeof(float) * (size_t)ckpt_slices_for(ctx->g.n_surf, stride) * 27 * (size_t)ctx->n_seeds));
    CK(grow(ctx->adj_align_acc, sizeof(double) * 2 * KF_MAX_LAYERS));
    CK(grow(ctx->adj_align, sizeof(float) * 2 * KF_MAX_LAYERS));
    CK(grow(ctx->adj_hits, sizeof(float) * 3 * (size_t)ctx->n_hits));
    CK(grow(ctx->adj_seed, sizeof(float) * 6 * (size_t)ctx->n_seeds));
  }
  CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  int rc = kf_find_tracks(ctx, stream);
  if (rc == KF_OK) {
    // Duplicate removal (short, latency-bound kernels) on the high-priority
    // side branch; beside it the fit's FP32 pass over every found track (it
    // removes few), whose removed tracks are cleared once both are done.
    cudaError_t fe = fork_side(ctx, st);
    const bool forked = fe == cudaSuccess;
    if (!forked) rc = fail(ctx, KF_ERR_CUDA, cudaGetErrorString(fe));
    if (rc == KF_OK) rc = kf_remove_duplicates(ctx, (void*)ctx->side);
    ctx->fit_beside_dedup = true;
    if (rc == KF_OK) rc = kf_fit_tracks(ctx, KF_FIT_FOUND, nullptr, nullptr, 0, 1, stream);
    ctx->fit_beside_dedup = false;
    if (forked) {  // the side branch rejoins the capture on every path
      fe = join_side(ctx, st);
      if (fe != cudaSuccess && rc == KF_OK) rc = fail(ctx, KF_ERR_CUDA, cudaGetErrorString(fe));
    }
    if (rc == KF_OK) {
      fe = launch_fit_unkept(ctx->last_fit, st);
      // the careful pass after the final keep flags: in the adjoint's side
      // branch with the adjoint, here without it
      if (fe == cudaSuccess && !with_adjoint) {
        fe = launch_fit_careful(ctx->last_fit, st);
        ctx->careful_fit_pending = false;
      }
      if (fe != cudaSuccess) rc = fail(ctx, KF_ERR_CUDA, cudaGetErrorString(fe));
    }
  }
  if (rc == KF_OK && with_adjoint)  // gradient into context buffers; kf_get_gradient reads them
    rc = kf_fit_adjoint(ctx, ptr<float>(ctx->adj_align), ptr<float>(ctx->adj_hits), ptr<float>(ctx->adj_seed), 1,
                        stream);
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(st, &graph);
  if (rc != KF_OK) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (e != cudaSuccess) return fail(ctx, KF_ERR_CUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e));
  ctx->graph = graph;
  CK(cudaGraphInstantiate(&ctx->exec, ctx->graph, cudaGraphInstantiateFlagUseNodePriority));
  ctx->graph_bufs.clear();
  for (DevBuf* b : all_bufs(ctx)) ctx->graph_bufs.push_back(b->p);
  ctx->graph_hit_off = ctx->hit_off_h;
  ctx->graph_seed_off = ctx->seed_off_h;
  ctx->graph_n_seeds = ctx->n_seeds;
  return KF_OK;
}

int kf_get_gradient(kf_ctx* ctx, float* g_align, float* g_hits, float* g_seed, int device_ptrs, void* stream) {
  if (!ctx) return KF_ERR_ARG;
  if (!ctx->adj_align.p) return fail(ctx, KF_ERR_STATE, "kf_get_gradient: no gradient computed");
  cudaStream_t st = S(stream);
  if (g_align) CK(get(g_align, ctx->adj_align.p, sizeof(float) * 2 * ctx->g.n_layers, device_ptrs, st));
  if (g_hits) {
    if (ctx->adj_hits.bytes < sizeof(float) * 3 * (size_t)ctx->n_hits)
      return fail(ctx, KF_ERR_STATE, "kf_get_gradient: no hit gradient kept");
    CK(get(g_hits, ctx->adj_hits.p, sizeof(float) * 3 * (size_t)ctx->n_hits, device_ptrs, st));
  }
  if (g_seed) {
    if (ctx->adj_seed.bytes < sizeof(float) * 6 * (size_t)ctx->n_seeds)
      return fail(ctx, KF_ERR_STATE, "kf_get_gradient: no seed gradient kept");
    CK(get(g_seed, ctx->adj_seed.p, sizeof(float) * 6 * (size_t)ctx->n_seeds, device_ptrs, st));
  }
  if (!device_ptrs) return check_status(ctx, st);
  return KF_OK;
}

int kf_launch_graph(kf_ctx* ctx, void* stream) {
  if (!ctx) return KF_ERR_ARG;
  if (!ctx->exec) return fail(ctx, KF_ERR_STATE, "kf_launch_graph: capture a graph first");
  if (ctx->n_seed_events != ctx->n_events || ctx->n_hits < 0)
    return fail(ctx, KF_ERR_STATE, "kf_launch_graph: load hits and seeds first");
  // The graph's kernels hold the buffer addresses, sizes and event offsets of
  // the capture: a load that reallocated a buffer or changed a size would make
  // them read freed memory or stale extents.
  bool same = ctx->hit_off_h == ctx->graph_hit_off && ctx->seed_off_h == ctx->graph_seed_off &&
              ctx->n_seeds == ctx->graph_n_seeds;
  const std::vector<DevBuf*> bufs = all_bufs(ctx);
  same = same && bufs.size() == ctx->graph_bufs.size();
  for (size_t i = 0; same && i < bufs.size(); ++i) same = bufs[i]->p == ctx->graph_bufs[i];
  if (!same)
    return fail(ctx, KF_ERR_STATE,
                "kf_launch_graph: a load since the capture changed the sizes or moved a buffer; capture again");
  CK(cudaGraphLaunch(ctx->exec, S(stream)));
  ctx->found = ctx->deduped = ctx->fitted = true;
  ctx->fit_source = KF_FIT_FOUND;
  return KF_OK;
}

int kf_autotune(kf_ctx* ctx, float* results, int max_results, int* n_results, void* stream) {
  if (!ctx) return KF_ERR_ARG;
  if (ctx->n_seed_events != ctx->n_events || ctx->n_events < 1)
    return fail(ctx, KF_ERR_STATE, "kf_autotune: load hits and seeds first");
  cudaStream_t st = S(stream);
  const int lane_opts[] = {4, 6, 8, 10, 12, 16};
  // candidate tiles of 32 to 256 threads (one lane per candidate slot)
  const int thread_opts[] = {32, 64, 128, 256};
  const int saved_lanes = ctx->lanes, saved_threads = ctx->threads, saved_pers = ctx->persistent,
            saved_bps = ctx->blocks_per_sm, saved_rc = ctx->regcap;
  float best = 1e30f;
  int best_l = saved_lanes, best_t = saved_threads, best_p = saved_pers, best_b = saved_bps,
      best_rc = saved_rc;
  int nr = 0;
  cudaEvent_t a, b;
  CK(cudaEventCreate(&a));
  CK(cudaEventCreate(&b));
  int rc = KF_OK;
  for (int lanes : lane_opts) {
    if (lanes < ctx->cfg.max_cands) continue;
    for (int threads : thread_opts)
    for (int regcap = 0; regcap < 2; ++regcap) {
      int bps = 1;
      if (find_prepare(lanes, regcap, threads, ctx->g, &bps) != cudaSuccess || bps < 1)
        continue;
      for (int pers = 0; pers < 2 && rc == KF_OK; ++pers) {
        ctx->lanes = lanes;
        ctx->threads = threads;
        ctx->persistent = pers;
        ctx->blocks_per_sm = bps;
        ctx->regcap = regcap;
        rc = kf_find_tracks(ctx, stream);  // warm-up
        if (rc != KF_OK) break;
        float tot = 0.f;
        for (int rep = 0; rep < 3 && rc == KF_OK; ++rep) {
          cudaEventRecord(a, st);
          rc = kf_find_tracks(ctx, stream);
          cudaEventRecord(b, st);
          cudaEventSynchronize(b);
          float ms = 0.f;
          cudaEventElapsedTime(&ms, a, b);
          tot += ms;
        }
        const float ms = tot / 3.f;
        if (results && nr < max_results) {
          results[5 * nr + 0] = (float)lanes;
          results[5 * nr + 1] = (float)threads;
          results[5 * nr + 2] = (float)pers;
          results[5 * nr + 3] = (float)regcap;
          results[5 * nr + 4] = ms;
        }
        ++nr;
        if (ms < best) {
          best = ms;
          best_l = lanes;
          best_t = threads;
          best_p = pers;
          best_b = bps;
          best_rc = regcap;
        }
      }
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  ctx->lanes = best_l;
  ctx->threads = best_t;
  ctx->persistent = best_p;
  ctx->blocks_per_sm = best_b;
  ctx->regcap = best_rc;
  CK(find_prepare(best_l, best_rc, best_t, ctx->g, &ctx->blocks_per_sm));
  if (n_results) *n_results = nr;
  if (rc != KF_OK) return rc;
  return KF_OK;
}

}  // extern "C"
