// Kalman re-fit of tracks (the paper's "fitting" step, Sec. 5): one thread
// per track, state and covariance in registers, from the seed prior placed at
// the first hit over the track's hits layer by layer.  The result is the
// state after the last hit, before its scattering, and the summed chi2 of the
// predicted residuals.
//
// Conditioning: where a track crosses a layer close to tangentially (the
// looper at the end of its reach), the propagation Jacobian grows like
// 1/cos(alpha) and the predicted covariance gains a large, nearly rank-one
// term that the update then removes again; FP32 loses the posterior there.
// A first FP32 pass fits every track and flags a track as soon as one of its
// crossings has cos(alpha) below CAREFUL_COS; a second pass refits only the
// flagged tracks, running those steps' propagation and update in double
// precision (a small fraction of tracks: loopers near their maximum radius).
// On a detector with endcap disks, a plane step along more than half a
// radian of the helix (a looper reaching a disk) flags its track the same
// way (PLANE_CAREFUL_PSI).
#include "kf_internal.h"

namespace kfg {

namespace {

constexpr float CAREFUL_COS = 0.5f;
constexpr int FIT_THREADS = 128;  // threads per block of the FP32 pass

// One Kalman step on an endcap disk in scalar type T (the plane, the (r-phi, r)
// measurement, the disk's scattering and loss).
template <class T>
__device__ __forceinline__ int disk_step(const DevGeom& g, T (&p)[6], T (&C)[21], bool first, bool last, int L,
                                         float mx, float my, float& chi2) {
  if (!first && !propagate_plane<T, true>(p, C, (T)plane_z(g, L), field_kb<T>(g, p))) return KF_FIT_NO_CROSS;
  DiskFrameT<T> d;
  make_frame_disk<T>(p, C, (T)g.vr, (T)g.vrr, d);
  T r0, r1;
  if (!residual_disk<T>(p, d.f, (T)mx, (T)my, r0, r1)) return KF_FIT_FAR_SIDE;
  chi2 += (float)chi2_of<T>(d.f, r0, r1);
  kf_update_disk<T>(p, C, d, r0, r1);
  if (!last) {
    add_ms_disk<T>(p, C, (T)g.disk_x0);
    add_eloss_ool<T, true, true>(p, C, (T)g.disk_eloss);
  }
  return KF_FIT_OK;
}

// One Kalman step in scalar type T: propagate (unless first), update with the
// corrected hit, scatter unless last.  Returns a KF_FIT_* status.  The fit
// takes the library's sine and cosine throughout (ACC).
template <class T, bool DISK>
__device__ __forceinline__ int fit_step(const DevGeom& g, float (&pf)[6], float (&Cf)[21], bool first,
                                        bool last, int L, float mx, float my, float mz, float& chi2) {
  T p[6], C[21];
#pragma unroll
  for (int k = 0; k < 6; ++k) p[k] = (T)pf[k];
#pragma unroll
  for (int k = 0; k < 21; ++k) C[k] = (T)Cf[k];
  if (DISK && is_disk(g, L)) {
    const int rc = disk_step<T>(g, p, C, first, last, L, mx, my, chi2);
    if (rc != KF_FIT_OK) return rc;
#pragma unroll
    for (int k = 0; k < 6; ++k) pf[k] = (float)p[k];
#pragma unroll
    for (int k = 0; k < 21; ++k) Cf[k] = (float)C[k];
    return KF_FIT_OK;
  }
  if (!first && propagate<T, true>(p, C, (T)g.radius[L], field_kb<T>(g, p), T(INFINITY)) != 1)
    return KF_FIT_NO_CROSS;
  FrameT<T> f;
  make_frame<T>(p, C, (T)g.vr, (T)g.vz, f);
  T r0, r1;
  if (!residual<T>(p, f, (T)mx, (T)my, (T)mz, r0, r1)) return KF_FIT_FAR_SIDE;
  chi2 += (float)chi2_of<T>(f, r0, r1);
  kf_update<T>(p, C, f, r0, r1);
  if (!last) {
    add_ms<T, true>(p, C, x0_at<T>(g, L, p[2]));
    add_eloss_ool<T, false, true>(p, C, (T)g.eloss[L]);
  }
#pragma unroll
  for (int k = 0; k < 6; ++k) pf[k] = (float)p[k];
#pragma unroll
  for (int k = 0; k < 21; ++k) Cf[k] = (float)C[k];
  return KF_FIT_OK;
}

// The fit's track order, per window of ORDER_WINDOW consecutive tracks: by
// decreasing hit count (tracks removed as duplicates count 0), so that a
// warp's tracks run about the same number of steps, while the per-track
// reads and writes of a window stay close together in time (they meet in L2).
// The order within a hit count is not fixed; no result depends on it.
constexpr int ORDER_WINDOW = 4096, ORDER_THREADS = 512, ORDER_BINS = 64;

__device__ __forceinline__ int order_key(const FitParams& P, int t) {
  if (P.keep && P.keep_in_main && !P.keep[t]) return 0;
  return min(max(P.n_list[t], 0), ORDER_BINS - 1);
}

// One block per window: counts per hit count, an exclusive prefix over the
// counts from the longest down, then each track's position (one shared-memory
// atomic per hit count and warp).
__global__ void __launch_bounds__(ORDER_THREADS) k_fit_order(const FitParams P) {
  static_assert(ORDER_BINS == 64, "two bins per lane");
  __shared__ unsigned cnt[ORDER_BINS], cur[ORDER_BINS];
  const int w0 = blockIdx.x * ORDER_WINDOW;
  const int w1 = min(P.ns, w0 + ORDER_WINDOW);
  for (int b = threadIdx.x; b < ORDER_BINS; b += blockDim.x) cnt[b] = 0u;
  __syncthreads();
  for (int t = w0 + threadIdx.x; t < w1; t += blockDim.x) atomicAdd(&cnt[order_key(P, t)], 1u);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  if (threadIdx.x < 32) {  // lane j: bins 63 - 2j and 62 - 2j
    const unsigned a = cnt[63 - 2 * lane], b = cnt[62 - 2 * lane];
    unsigned incl = a + b;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const unsigned v = __shfl_up_sync(0xffffffffu, incl, off);
      if (lane >= off) incl += v;
    }
    cur[63 - 2 * lane] = incl - a - b;
    cur[62 - 2 * lane] = incl - b;
  }
  __syncthreads();
  for (int r = 0; r < ORDER_WINDOW; r += ORDER_THREADS) {
    const int t = w0 + r + threadIdx.x;
    const int key = t < w1 ? order_key(P, t) : ORDER_BINS;  // ORDER_BINS: no track
    const unsigned same = __match_any_sync(0xffffffffu, key);
    if (key < ORDER_BINS) {
      const int leader = __ffs(same) - 1;
      unsigned pos = 0;
      if (lane == leader) pos = atomicAdd(&cur[key], (unsigned)__popc(same));
      pos = __shfl_sync(same, pos, leader) + __popc(same & ((1u << lane) - 1u));
      P.order[w0 + pos] = t;
    }
  }
}

// Track at position i of the fit's order; checkpoints go to column i.
// Returns, in the careful pass, whether a crossing of the track has
// cos(alpha) < ADJOINT_CAREFUL_COS (its adjoint then needs double steps).
// DISK: the detector has endcap disks (hits on surfaces >= n_layers take the
// plane step; they carry no alignment).
template <bool CAREFUL, bool DISK>
__device__ __forceinline__ bool fit_track(const FitParams& P, int i, int t) {
  if (!CAREFUL && P.careful_flag) P.careful_flag[t] = 0;  // set below if the track is left to the careful pass
  // removed as a duplicate: zero outputs (the careful pass reads the final
  // flags; the main pass only when they are written before it)
  if (P.keep && (CAREFUL || P.keep_in_main) && !P.keep[t]) {
#pragma unroll
    for (int k = 0; k < 6; ++k) P.fit_p[(size_t)k * P.ns + t] = 0.f;
#pragma unroll
    for (int k = 0; k < 21; ++k) P.fit_C[(size_t)k * P.ns + t] = 0.f;
    P.fit_chi2[t] = 0.f;
    P.fit_status[t] = KF_FIT_SKIPPED;
    return false;
  }
  const DevGeom& g = P.g;
  float p[6], C[21];
#pragma unroll
  for (int k = 0; k < 6; ++k) p[k] = P.sp[(size_t)k * P.ns + t];
#pragma unroll
  for (int k = 0; k < 21; ++k) C[k] = P.sc[(size_t)k * P.ns + t];
  // a loose prior: the careful pass runs the first steps in double
  const bool loose = loose_prior(C, g);
  if (!CAREFUL && loose) {
    P.careful_list[atomicAdd(P.careful_count, 1u)] = i;
    if (P.careful_flag) P.careful_flag[t] = 1;
    return false;
  }
  const int hoff = P.hit_off[P.seed_event[t]];
  const int n = P.n_list[t];
  const int* lst = P.lists + (size_t)t * P.max_len;
  float chi2 = 0.f;
  int status = KF_FIT_OK;
  bool adj_dbl = false;
#pragma unroll 1
  for (int k = 0; k < n && status == KF_FIT_OK; ++k) {
    if (P.ckpt && k % P.ckpt_stride == 0 && k / P.ckpt_stride < P.ckpt_slices) {  // state before hit k
      float* c = P.ckpt + (size_t)(k / P.ckpt_stride) * 27 * P.ns + i;
#pragma unroll
      for (int q = 0; q < 6; ++q) c[(size_t)q * P.ns] = p[q];
#pragma unroll
      for (int q = 0; q < 21; ++q) c[(size_t)(6 + q) * P.ns] = C[q];
    }
    const int hi = hoff + lst[k];
    const int L = P.hlayer[hi];
    const bool disk = DISK && is_disk(g, L);
    float mx, my, mz;
    if (disk) {
      mx = P.hx[hi];
      my = P.hy[hi];
      mz = P.hz[hi];
    } else {
      corrected_hit(P.align[L], P.hx[hi], P.hy[hi], P.hz[hi], mx, my, mz);
    }
    if (!CAREFUL && disk) {
      if (k > 0 && plane_careful(g, p, plane_z(g, L))) {  // a long arc onto the disk: the careful pass
        P.careful_list[atomicAdd(P.careful_count, 1u)] = i;
        if (P.careful_flag) P.careful_flag[t] = 1;
        return false;
      }
      status = disk_step<float>(g, p, C, k == 0, k + 1 == n, L, mx, my, chi2);
    } else if (!CAREFUL) {
      if (k > 0) {
        float cosa = 1.f;
        if (propagate<float, true>(p, C, g.radius[L], field_kb<float>(g, p), INFINITY, &cosa) != 1) {
          status = KF_FIT_NO_CROSS;
          break;
        }
        if (cosa < CAREFUL_COS) {  // leave the track to the careful pass
          P.careful_list[atomicAdd(P.careful_count, 1u)] = i;
          if (P.careful_flag) P.careful_flag[t] = 1;
          return false;
        }
      }
      Frame f;
      make_frame<float>(p, C, g.vr, g.vz, f);
      float r0, r1;
      if (!residual<float>(p, f, mx, my, mz, r0, r1)) { status = KF_FIT_FAR_SIDE; break; }
      chi2 += chi2_of<float>(f, r0, r1);
      kf_update<float>(p, C, f, r0, r1);
      if (k + 1 < n) {
        add_ms<float, true>(p, C, x0_at<float>(g, L, p[2]));
        add_eloss_ool<float, false, true>(p, C, g.eloss[L]);
      }
    } else {
      bool careful = false;
      if (k > 0 && !disk) {
        float zc, cosa;
        if (!crossing(p, g.radius[L], field_kb<float>(g, p), zc, cosa)) { status = KF_FIT_NO_CROSS; break; }
        careful = cosa < CAREFUL_COS;
        adj_dbl = adj_dbl || cosa < ADJOINT_CAREFUL_COS;
      } else if (k > 0) {  // a long arc onto a disk: in double here and in the adjoint
        careful = plane_careful(g, p, plane_z(g, L));
        adj_dbl = adj_dbl || careful;
      }
      if (loose && k < LOOSE_STEPS) careful = true;  // the first steps against a loose prior
      status = careful ? fit_step<double, DISK>(g, p, C, k == 0, k + 1 == n, L, mx, my, mz, chi2)
                       : fit_step<float, DISK>(g, p, C, k == 0, k + 1 == n, L, mx, my, mz, chi2);
    }
  }
#pragma unroll
  for (int k = 0; k < 6; ++k) P.fit_p[(size_t)k * P.ns + t] = p[k];
#pragma unroll
  for (int k = 0; k < 21; ++k) P.fit_C[(size_t)k * P.ns + t] = C[k];
  P.fit_chi2[t] = chi2;
  P.fit_status[t] = status;
  return adj_dbl;
}

template <bool DISK>
__global__ void __launch_bounds__(FIT_THREADS) k_fit(const FitParams P) {
  const int i = blockIdx.x * FIT_THREADS + threadIdx.x;
  if (i < P.ns) fit_track<false, DISK>(P, i, P.order[i]);
}

// Second pass over the flagged tracks (grid-stride over their list).  A
// track whose adjoint needs double steps gets CAREFUL_DBL_BIT in its entry
// and is listed in dbl_list.
template <bool DISK>
__global__ void __launch_bounds__(128) k_fit_careful(const FitParams P) {
  const unsigned n = *P.careful_count;
  for (unsigned j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    const unsigned v = (unsigned)P.careful_list[j];
    const int pos = (int)(v & ~CAREFUL_DBL_BIT);
    const bool dbl = fit_track<true, DISK>(P, pos, P.order[pos]);
    P.careful_list[j] = (int)(dbl ? (v | CAREFUL_DBL_BIT) : (v & ~CAREFUL_DBL_BIT));
    if (dbl) P.dbl_list[atomicAdd(P.dbl_count, 1u)] = pos;  // packed, so that few blocks hold them
  }
}

__global__ void __launch_bounds__(256) k_fit_unkept(const FitParams P) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= P.ns || P.keep[t]) return;
#pragma unroll
  for (int k = 0; k < 6; ++k) P.fit_p[(size_t)k * P.ns + t] = 0.f;
#pragma unroll
  for (int k = 0; k < 21; ++k) P.fit_C[(size_t)k * P.ns + t] = 0.f;
  P.fit_chi2[t] = 0.f;
  P.fit_status[t] = KF_FIT_SKIPPED;
}

}  // namespace

cudaError_t launch_fit_unkept(const FitParams& P, cudaStream_t st) {
  if (P.ns <= 0 || !P.keep) return cudaSuccess;
  k_fit_unkept<<<(P.ns + 255) / 256, 256, 0, st>>>(P);
  return cudaGetLastError();
}

cudaError_t launch_fit_main(const FitParams& P, cudaStream_t st) {
  if (P.ns <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(P.careful_count, 0, sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  k_fit_order<<<(P.ns + ORDER_WINDOW - 1) / ORDER_WINDOW, ORDER_THREADS, 0, st>>>(P);
  const int blocks = (P.ns + FIT_THREADS - 1) / FIT_THREADS;
  if (P.g.n_disks > 0) k_fit<true><<<blocks, FIT_THREADS, 0, st>>>(P);
  else k_fit<false><<<blocks, FIT_THREADS, 0, st>>>(P);
  return cudaGetLastError();
}

cudaError_t launch_fit_careful(const FitParams& P, cudaStream_t st) {
  if (P.ns <= 0) return cudaSuccess;
  // flagged tracks are a few percent of all, and their double-precision
  // steps are bound by the SM's FP64 rate: blocks of 32 threads, so that they
  // spread over many SMs; a grid for a twentieth of all tracks, striding over
  // however many there are
  const int threads = 32;
  const int careful_blocks = (P.ns / 20 + threads - 1) / threads + 1;
  cudaError_t e = cudaMemsetAsync(P.dbl_count, 0, sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  if (P.g.n_disks > 0) k_fit_careful<true><<<careful_blocks, threads, 0, st>>>(P);
  else k_fit_careful<false><<<careful_blocks, threads, 0, st>>>(P);
  return cudaGetLastError();
}

cudaError_t launch_fit(const FitParams& P, cudaStream_t st) {
  cudaError_t e = launch_fit_main(P, st);
  if (e == cudaSuccess) e = launch_fit_careful(P, st);
  return e;
}

}  // namespace kfg
