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
#include "kf_internal.h"

namespace kfg {

namespace {

constexpr float CAREFUL_COS = 0.5f;

// One Kalman step in scalar type T: propagate (unless first), update with the
// corrected hit, scatter unless last.  Returns a KF_FIT_* status.
template <class T>
__device__ __forceinline__ int fit_step(const DevGeom& g, float (&pf)[6], float (&Cf)[21], bool first,
                                        bool last, int L, float mx, float my, float mz, float& chi2) {
  T p[6], C[21];
#pragma unroll
  for (int k = 0; k < 6; ++k) p[k] = (T)pf[k];
#pragma unroll
  for (int k = 0; k < 21; ++k) C[k] = (T)Cf[k];
  if (!first && propagate<T>(p, C, (T)g.radius[L], (T)g.kb, T(INFINITY)) != 1) return KF_FIT_NO_CROSS;
  FrameT<T> f;
  make_frame<T>(p, C, (T)g.vr, (T)g.vz, f);
  T r0, r1;
  if (!residual<T>(p, f, (T)mx, (T)my, (T)mz, r0, r1)) return KF_FIT_FAR_SIDE;
  chi2 += (float)chi2_of<T>(f, r0, r1);
  kf_update<T>(p, C, f, r0, r1);
  if (!last) {
    add_ms<T>(p, C, x0_at<T>(g, L, p[2]));
    add_eloss_ool<T>(p, C, (T)g.eloss[L]);
  }
#pragma unroll
  for (int k = 0; k < 6; ++k) pf[k] = (float)p[k];
#pragma unroll
  for (int k = 0; k < 21; ++k) Cf[k] = (float)C[k];
  return KF_FIT_OK;
}

// Track at position i of the fit's order; checkpoints go to column i.
template <bool CAREFUL>
__device__ __forceinline__ void fit_track(const FitParams& P, int i) {
  const int t = P.order[i];
  if (!CAREFUL && P.careful_flag) P.careful_flag[t] = 0;  // set below if the track is left to the careful pass
  if (!CAREFUL && P.keep && !P.keep[t]) {  // removed as a duplicate: zero outputs
#pragma unroll
    for (int k = 0; k < 6; ++k) P.fit_p[(size_t)k * P.ns + t] = 0.f;
#pragma unroll
    for (int k = 0; k < 21; ++k) P.fit_C[(size_t)k * P.ns + t] = 0.f;
    P.fit_chi2[t] = 0.f;
    P.fit_status[t] = KF_FIT_SKIPPED;
    return;
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
    return;
  }
  const int hoff = P.hit_off[P.seed_event[t]];
  const int n = P.n_list[t];
  const int* lst = P.lists + (size_t)t * P.max_len;
  float chi2 = 0.f;
  float min_cos = 1.f;
  int status = KF_FIT_OK;
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
    float mx, my, mz;
    corrected_hit(P.align[L], P.hx[hi], P.hy[hi], P.hz[hi], mx, my, mz);
    if (!CAREFUL) {
      if (k > 0) {
        float cosa = 1.f;
        if (propagate<float>(p, C, g.radius[L], g.kb, INFINITY, &cosa) != 1) { status = KF_FIT_NO_CROSS; break; }
        if (cosa < CAREFUL_COS) {  // leave the track to the careful pass
          P.careful_list[atomicAdd(P.careful_count, 1u)] = i;
          if (P.careful_flag) P.careful_flag[t] = 1;
          return;
        }
      }
      Frame f;
      make_frame<float>(p, C, g.vr, g.vz, f);
      float r0, r1;
      if (!residual<float>(p, f, mx, my, mz, r0, r1)) { status = KF_FIT_FAR_SIDE; break; }
      chi2 += chi2_of<float>(f, r0, r1);
      kf_update<float>(p, C, f, r0, r1);
      if (k + 1 < n) {
        add_ms<float>(p, C, x0_at<float>(g, L, p[2]));
        add_eloss_ool<float>(p, C, g.eloss[L]);
      }
    } else {
      bool careful = false;
      if (k > 0) {
        float zc, cosa;
        if (!crossing(p, g.radius[L], g.kb, zc, cosa)) { status = KF_FIT_NO_CROSS; break; }
        careful = cosa < CAREFUL_COS;
        min_cos = fminf(min_cos, cosa);
      }
      if (loose && k < LOOSE_STEPS) careful = true;  // the first steps against a loose prior
      status = careful ? fit_step<double>(g, p, C, k == 0, k + 1 == n, L, mx, my, mz, chi2)
                       : fit_step<float>(g, p, C, k == 0, k + 1 == n, L, mx, my, mz, chi2);
    }
  }
#pragma unroll
  for (int k = 0; k < 6; ++k) P.fit_p[(size_t)k * P.ns + t] = p[k];
#pragma unroll
  for (int k = 0; k < 21; ++k) P.fit_C[(size_t)k * P.ns + t] = C[k];
  P.fit_chi2[t] = chi2;
  P.fit_status[t] = status;
  if (CAREFUL && P.careful_flag) P.careful_flag[t] = min_cos < ADJOINT_CAREFUL_COS ? 2 : 1;
}

__global__ void __launch_bounds__(128) k_fit(const FitParams P) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < P.ns) fit_track<false>(P, i);
}

// Second pass over the flagged tracks (grid-stride over their list).
__global__ void __launch_bounds__(128) k_fit_careful(const FitParams P) {
  const unsigned n = *P.careful_count;
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    fit_track<true>(P, P.careful_list[i]);
}

// The fit's track order: a counting sort by hit count, decreasing; tracks
// removed as duplicates count as 0 hits and come last.  Positions within a
// bin are taken by atomics (the order within a bin is not fixed; each track's
// results do not depend on it).
__device__ __forceinline__ int order_key(const FitParams& P, int t) {
  if (P.keep && !P.keep[t]) return 0;
  return min(max(P.n_list[t], 0), FIT_ORDER_BINS - 1);
}

constexpr int ORDER_THREADS = 256;

__global__ void __launch_bounds__(ORDER_THREADS) k_order_count(const FitParams P) {
  __shared__ unsigned h[FIT_ORDER_BINS];
  for (int b = threadIdx.x; b < FIT_ORDER_BINS; b += blockDim.x) h[b] = 0u;
  __syncthreads();
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < P.ns; t += gridDim.x * blockDim.x)
    atomicAdd(&h[order_key(P, t)], 1u);
  __syncthreads();
  for (int b = threadIdx.x; b < FIT_ORDER_BINS; b += blockDim.x)
    if (h[b]) atomicAdd(&P.order_hist[b], h[b]);
}

// One track per thread: position = (tracks in bins of more hits) + the
// track's place among its bin's tracks (one atomic per bin and warp).
__global__ void __launch_bounds__(ORDER_THREADS) k_order_scatter(const FitParams P) {
  static_assert(FIT_ORDER_BINS == 64, "two bins per lane");
  __shared__ unsigned base[FIT_ORDER_BINS];
  const int lane = threadIdx.x & 31;
  if (threadIdx.x < 32) {
    // lane j holds bins 63 - 2j and 62 - 2j; exclusive prefix over lanes
    const unsigned a = P.order_hist[63 - 2 * lane], b = P.order_hist[62 - 2 * lane];
    unsigned incl = a + b;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const unsigned v = __shfl_up_sync(0xffffffffu, incl, off);
      if (lane >= off) incl += v;
    }
    const unsigned excl = incl - a - b;
    base[63 - 2 * lane] = excl;
    base[62 - 2 * lane] = excl + a;
  }
  __syncthreads();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int key = t < P.ns ? order_key(P, t) : FIT_ORDER_BINS;  // FIT_ORDER_BINS: no track
  const unsigned same = __match_any_sync(0xffffffffu, key);
  if (key < FIT_ORDER_BINS) {
    const int leader = __ffs(same) - 1;
    unsigned off = 0;
    if (lane == leader) off = atomicAdd(&P.order_hist[FIT_ORDER_BINS + key], (unsigned)__popc(same));
    off = __shfl_sync(same, off, leader);
    const unsigned rank = __popc(same & ((1u << lane) - 1u));
    P.order[base[key] + off + rank] = t;
  }
}

}  // namespace

cudaError_t launch_fit_main(const FitParams& P, cudaStream_t st) {
  if (P.ns <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(P.order_hist, 0, sizeof(unsigned) * 2 * FIT_ORDER_BINS, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(P.careful_count, 0, sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int order_blocks = (P.ns + ORDER_THREADS - 1) / ORDER_THREADS;
  k_order_count<<<min(order_blocks, 4 * sms), ORDER_THREADS, 0, st>>>(P);
  k_order_scatter<<<order_blocks, ORDER_THREADS, 0, st>>>(P);
  const int threads = 128;
  const int blocks = (P.ns + threads - 1) / threads;
  k_fit<<<blocks, threads, 0, st>>>(P);
  return cudaGetLastError();
}

cudaError_t launch_fit_careful(const FitParams& P, cudaStream_t st) {
  if (P.ns <= 0) return cudaSuccess;
  // flagged tracks are a few percent of all: a grid sized for a twentieth of
  // them, striding over however many there are
  const int threads = 128;
  const int careful_blocks = (P.ns / 20 + threads - 1) / threads + 1;
  k_fit_careful<<<careful_blocks, threads, 0, st>>>(P);
  return cudaGetLastError();
}

cudaError_t launch_fit(const FitParams& P, cudaStream_t st) {
  cudaError_t e = launch_fit_main(P, st);
  if (e == cudaSuccess) e = launch_fit_careful(P, st);
  return e;
}

}  // namespace kfg
