// Combinatorial Kalman-filter track finding (the paper's "build" step, Sec. 2).
//
// Mapping: one seed per group of G lanes, one lane per candidate slot (G >=
// N = max_cands), 32/G seeds per warp processed in lockstep.  A candidate's
// state (6 parameters + 21 covariance terms) stays in its lane's registers
// across all layers.  The seed fit (three forced hits) and the first layer
// after it, where each seed has a single candidate, run before, one thread
// per seed (k_seed_fit): inside the group loop only one lane of each group
// would work on them.  The careful pass keeps the seed fit and the first
// layer in its loop (with double-precision steps where needed).  Per layer:
//   1. every live candidate propagates to the layer (closed-form helix, exact
//      Jacobian, sparse J C J^T) and builds its measurement frame;
//   2. it walks the eta x phi bins of a window that contains the whole
//      chi2 < cut ellipse (bounds padded by the FP32 error of the window
//      arithmetic), tests every hit there and keeps its own best N
//      hit-children in a sorted list in shared memory;
//   3. the group selects the N best children of all its candidates by their
//      64-bit ranking keys (more hits, lower chi2 sum, parent slot, hit
//      before hole, hit index): the children are packed into one shared
//      array, each lane ranks a few of them by counting smaller keys, and the
//      children of rank < N land in the slots of their rank;
//   4. each lane pulls its chosen parent's predicted state with warp shuffles,
//      applies the Kalman update for a hit-child and the scattering of the layer.
// Parent pointers and hit indices go to a per-group history in shared memory;
// the best candidate's hit list is rebuilt from it at the end.
//
// Endcap disks (the DISK variants, for a detector with disks): a seed's
// candidates search the surfaces of its region's plan (Sec. 2: the event is
// split into eta regions) -- the barrel layers after the seed, then for a
// forward seed the disks of its side; a disk is reached by the plane step and
// searched in an r x phi grid with the (r-phi, r) measurement; along a
// forward plan a surface not crossed within its bounds is passed (the
// candidate is carried on unchanged, neither a hole nor finished).  Their
// seed kernel fits the seed only; the plan's first surface is searched in the
// group loop.
//
// The kernel templates live in this header; kf_find.cu instantiates the
// barrel variants and kf_find_disk.cu the disk variants.
#pragma once

#include "kf_internal.h"

namespace kfg {

namespace {

constexpr int BACKUP_STRIDE = 28;  // 27 state floats, padded
// Shared memory per warp, for G lanes per seed: child lists [32 lanes][G + 1]
// u64 (at most N <= G hit children and the hole or carried child; the careful
// pass also keeps 27 floats of scratch there, so at least 14 entries); the
// packed children of each group [32][G + 1] u64, which between the propagation
// and the selection holds the state backup [32 lanes][28] float; selected
// children [32] u64; history [32 lanes][n_hist] int, one column per position
// of the longest search plan (n_layers, plus n_disks with endcap disks).
__host__ __device__ constexpr int list_stride(int G, bool careful) {
  return (careful && G + 1 < 14) ? 14 : G + 1;
}
__host__ __device__ constexpr int smem_list(int G, bool careful) { return 32 * list_stride(G, careful) * 8; }
__host__ __device__ constexpr int smem_gather(int G, bool careful) {
  return smem_list(G, careful) > 32 * BACKUP_STRIDE * 4 ? smem_list(G, careful) : 32 * BACKUP_STRIDE * 4;
}
constexpr int SMEM_SLOT = 32 * 8;
__host__ __device__ constexpr int smem_per_warp(int G, bool careful, int n_hist) {
  return smem_list(G, careful) + smem_gather(G, careful) + SMEM_SLOT + ((32 * n_hist * 4 + 15) / 16) * 16;
}
// The careful pass adds each lane's double-precision prediction [32][27] and
// the lanes' lists of a warp-wide window search [32][KF_MAX_CANDS] u64.
constexpr int SMEM_DSTATE = 32 * 27 * 8;
constexpr int SMEM_COOP = 32 * KF_MAX_CANDS * 8;
__host__ __device__ constexpr int smem_per_warp_k(int G, int n_hist, bool careful) {
  return smem_per_warp(G, careful, n_hist) + (careful ? SMEM_DSTATE + SMEM_COOP : 0);
}
// Shared memory per block ahead of the warps' areas: the z edges of the eta
// bins of every layer [n_layers][n_eta + 1].
__host__ __device__ constexpr int smem_edges(int n_layers, int n_eta) {
  return ((n_layers * (n_eta + 1) * 4 + 15) / 16) * 16;
}
// Window padding: relative and absolute slack on the chi2-ellipse bounds that
// covers the FP32 rounding of the window arithmetic and of the hit's own
// angle and eta-bin computation.
constexpr float WIN_REL = 1e-3f;
constexpr float WIN_PHI_ABS = 1.5e-5f;  // rad (includes the error of atan2_window, about 1e-6)
constexpr float WIN_Z_ABS = 1e-4f;    // cm
// Crossings closer to tangent than this (cos of the angle between direction
// and radial direction) are propagated in double: the FP32 error of the
// transported covariance grows as 1/cos^4 and near the turning radius of a
// looper it can leave the prediction without a positive definite S.  The
// main pass gives up a seed whose candidates meet such a crossing (after that
// layer its lanes go idle) and lists it; a careful pass after it (the same
// kernel with CAREFUL) redoes the listed seeds with those propagations in
// double, so that the double code and its registers stay out of the main
// pass.  The threshold for the finding is 0.2: on the PU-200 batch every
// threshold from 0.1 to 0.5 gives the oracle's hit lists for the most tangent
// loopers, and no prediction without a positive definite S, while the double
// work (FP64 runs at a small fraction of the FP32 rate) grows tenfold from 0.2
// to 0.5.  The number of seeds redone is counted (counter 7).  On such
// a layer the careful pass keeps the prediction in double (shared memory):
// the measurement frame (S, S^-1) is formed from it in double and only then
// rounded for the window search, and the children of that prediction are
// updated (and scattered) in double from it, as the re-fit's careful pass
// does, because the prediction carries a large nearly rank-one term that
// FP32 rounding of the covariance would turn indefinite.
constexpr float FIND_CAREFUL_COS = 0.2f;
constexpr int CAREFUL_THREADS = 128;

// Double-precision propagation of the state st[0..26] (p, then C) in place;
// st is the lane's child list in shared memory, unused at this point.  The
// double result also goes to dst[0..26].
// kb0, fcz, fcr: the field (DevGeom), taken at the state's position in double.
__device__ __noinline__ int careful_propagate(float* st, double* dst, float R, float kb0, float fcz, float fcr,
                                              float z_lim) {
  double p[6], C[21];
  for (int k = 0; k < 6; ++k) p[k] = st[k];
  for (int k = 0; k < 21; ++k) C[k] = st[6 + k];
  const double kb = (double)kb0 * fma((double)fcz, p[2] * p[2], fma((double)fcr, fma(p[0], p[0], p[1] * p[1]), 1.0));
  const int rc = propagate<double>(p, C, (double)R, kb, (double)z_lim);
  if (rc == 1) {
    for (int k = 0; k < 6; ++k) {
      st[k] = (float)p[k];
      dst[k] = p[k];
    }
    for (int k = 0; k < 21; ++k) {
      st[6 + k] = (float)C[k];
      dst[6 + k] = C[k];
    }
  }
  return rc;
}

// Measurement frame of a double-precision prediction, rounded.
__device__ __noinline__ Frame careful_frame(const double* dst, float vr, float vz) {
  double p[6], C[21];
  for (int k = 0; k < 6; ++k) p[k] = dst[k];
  for (int k = 0; k < 21; ++k) C[k] = dst[6 + k];
  FrameT<double> fd;
  make_frame<double>(p, C, (double)vr, (double)vz, fd);
  Frame f;
  f.su = (float)fd.su;
  f.cu = (float)fd.cu;
  for (int k = 0; k < 6; ++k) f.a0[k] = (float)fd.a0[k];
  f.s00 = (float)fd.s00;
  f.s11 = (float)fd.s11;
  f.si00 = (float)fd.si00;
  f.si01 = (float)fd.si01;
  f.si11 = (float)fd.si11;
  return f;
}

// A child of a double-precision prediction in[0..26]: the update with the
// corrected hit m (upd) and the scattering of the layer (ms; always after an
// update), in double; the result rounded to out[0..26].  Returns false for a
// hit on the far half (no update, no scattering); *dchi2 = the hit's chi2.
__device__ __noinline__ bool careful_child(const double* in, float* out, float mx, float my, float mz, bool upd,
                                           bool ms, const DevGeom& g, int l, float* dchi2) {
  const float vr = g.vr, vz = g.vz;
  double p[6], C[21];
  for (int k = 0; k < 6; ++k) p[k] = in[k];
  for (int k = 0; k < 21; ++k) C[k] = in[6 + k];
  bool ok = true;
  if (upd) {
    FrameT<double> f;
    make_frame<double>(p, C, (double)vr, (double)vz, f);
    double r0, r1;
    ok = residual<double>(p, f, (double)mx, (double)my, (double)mz, r0, r1);
    if (ok) {
      *dchi2 = (float)chi2_of<double>(f, r0, r1);
      kf_update<double>(p, C, f, r0, r1);
      ms = true;
    } else {
      ms = false;
    }
  }
  if (ms) {
    add_ms<double>(p, C, x0_at<double>(g, l, p[2]));
    add_eloss<double>(p, C, (double)g.eloss[l]);
  }
  for (int k = 0; k < 6; ++k) out[k] = (float)p[k];
  for (int k = 0; k < 21; ++k) out[6 + k] = (float)C[k];
  return ok;
}

// CAP = 0: blocks of up to 256 threads, registers at the compiler's choice;
// CAP = 1: blocks of up to 128 threads, five per SM (at most 102 registers).
// CAREFUL: the pass over the seeds the main pass listed (always persistent).
// Counters in P.queue: [0] main-pass work, [1] careful-pass work, [2] number
// of listed seeds.
// The eta-phi bins of the window that contains the chi2 < cut ellipse of the
// prediction p (frame f) on layer l: |r_rphi| < sqrt(cut S00) with
// r_rphi = R_hit sin(dphi) on the near half, |r_z| < sqrt(cut S11); rows
// [e0, e1] (none when S is not positive definite), columns [b0, b1) and, when
// the window wraps around phi = pi, [0, b2) as well.
struct Window {
  int e0, e1, b0, b1, b2;
};
// s_edges: the eta-bin edges of every layer in shared memory ([n_layers][n_eta
// + 1]), or null for the global table and its first-guess lookup.
__device__ __forceinline__ Window window_of(const FindParams& P, int l, float R, const float (&p)[6],
                                            const Frame& f, bool spd, const Align4& al,
                                            const float* s_edges = nullptr) {
  const DevGeom& g = P.g;
  // Bounds through hardware approximations (square root, quotient, window
  // centre angle): their errors are a few ulp, far inside the padding.
  const float w1 = sqrt_bound(g.chi2_cut * f.s00);
  const float w2 = sqrt_bound(g.chi2_cut * f.s11);
  // asin(x) for the usual small x by x + x^3/6 + 3x^5/40 (truncation below
  // 3e-9 relative for x < 0.05, far inside the padding)
  const float xr = w1 * g.r_inv[l];
  float dphi = (xr >= 1.f) ? 0.5f * PI_F
               : (xr < 0.05f ? xr * fmaf(xr * xr, fmaf(xr * xr, 0.075f, 1.f / 6.f), 1.f) : asinf(xr));
  dphi = fminf(dphi, 0.5f * PI_F) * (1.f + WIN_REL) + WIN_PHI_ABS;
  const float phic = atan2_window(p[1], p[0]) + al.dphi;
  const int nphi = g.n_phi, neta = g.n_eta;
  const int u0 = phi_bin_raw(phic - dphi, g.phi_scale);
  const int u1 = phi_bin_raw(phic + dphi, g.phi_scale);
  int span = u1 - u0 + 1, b0;
  if (span >= nphi) { span = nphi; b0 = 0; } else { b0 = wrap_bin(u0, nphi); }
  const float zc = p[2] + al.az;
  const float wz = w2 * (1.f + WIN_REL) + WIN_Z_ABS;
  Window w;
  if (s_edges) {
    const float* edges = s_edges + l * (neta + 1);
    const float ri = g.r_inv[l], em = g.eta_max[l], es = g.eta_scale[l];
    w.e0 = eta_bin_smem(zc - wz, ri, em, es, neta, edges);
    w.e1 = spd ? eta_bin_smem(zc + wz, ri, em, es, neta, edges) : w.e0 - 1;
  } else {
    const float* edges = P.eta_edges + (size_t)l * (MAX_ETA_BINS + 1);
    const unsigned char* lut = P.eta_lut + (size_t)l * ETA_LUT;
    w.e0 = eta_bin(zc - wz, neta, g.z_max, g.eta_lut_scale, lut, edges);
    w.e1 = spd ? eta_bin(zc + wz, neta, g.z_max, g.eta_lut_scale, lut, edges) : w.e0 - 1;
  }
  w.b0 = b0;
  w.b1 = min(b0 + span, nphi);
  w.b2 = b0 + span - nphi;  // > 0 when the window wraps
  return w;
}

// The r x phi bins of the window on an endcap disk that contains the chi2 <
// cut ellipse of the prediction p (frame f): with r_p = |p_xy| and a hit at
// radius r_h, angle dphi from the prediction, r0 = r_h sin(dphi) and r1 =
// r_h cos(dphi) - r_p; |r0| < w0 = sqrt(cut S00) and |r1| < w1 = sqrt(cut S11)
// on the near half (cos(dphi) > 0) give r_p - w1 < r_h < sqrt((r_p + w1)^2 +
// w0^2) and |sin(dphi)| < w0 / r_h < w0 / (r_p - w1).  Bounds padded as
// window_of's.
__device__ __forceinline__ Window window_disk(const FindParams& P, const float (&p)[6], const Frame& f, bool spd) {
  const DevGeom& g = P.g;
  const float w0 = sqrt_bound(g.chi2_cut * f.s00) * (1.f + WIN_REL) + WIN_Z_ABS;
  const float w1 = sqrt_bound(g.chi2_cut * f.s11) * (1.f + WIN_REL) + WIN_Z_ABS;
  const float rp = disk_r(p[0], p[1]);
  const float rlo = (rp - w1) * (1.f - WIN_REL) - WIN_Z_ABS;
  const float rhi = sqrtf(fmaf(rp + w1, rp + w1, w0 * w0)) * (1.f + WIN_REL) + WIN_Z_ABS;
  float dphi = 0.5f * PI_F;
  if (rlo > w0) {
    const float xr = w0 / rlo;
    dphi = xr < 0.05f ? xr * fmaf(xr * xr, fmaf(xr * xr, 0.075f, 1.f / 6.f), 1.f) : asinf(xr);
  }
  dphi = fminf(dphi, 0.5f * PI_F) * (1.f + WIN_REL) + WIN_PHI_ABS;
  const float phic = atan2_window(p[1], p[0]);
  const int nphi = g.n_phi;
  const int u0 = phi_bin_raw(phic - dphi, g.phi_scale);
  const int u1 = phi_bin_raw(phic + dphi, g.phi_scale);
  int span = u1 - u0 + 1, b0;
  if (span >= nphi) { span = nphi; b0 = 0; } else { b0 = wrap_bin(u0, nphi); }
  Window w;
  w.e0 = r_bin(g, rlo);
  w.e1 = spd ? r_bin(g, rhi) : w.e0 - 1;
  w.b0 = b0;
  w.b1 = min(b0 + span, nphi);
  w.b2 = b0 + span - nphi;
  return w;
}

// Tests every hit of the window (cell offsets off of the event and layer)
// against the prediction; the hits with chi2 < cut become children (ranking
// key: nf1 hits, chi2 sum + chi2, parent slot) in the candidate's ascending
// child list lst[0..cnt) of at most max_cands.  BATCH: hits loaded in batches
// of 8, so that their latencies overlap (near-tangent windows can hold
// thousands of hits).  DK: a disk's window (raw hit positions, (r-phi, r)
// residuals).
template <bool BATCH, bool DK = false>
__device__ __forceinline__ void scan_window(const FindParams& P, const unsigned* off, const Window& w,
                                            const Align4& al, const float (&p)[6], const Frame& f, int nf1,
                                            float chi2, int slot, unsigned long long* lst, int& cnt,
                                            unsigned& c_chi2) {
  const int nphi = P.g.n_phi, N = P.g.max_cands;
  const float cut = P.g.chi2_cut;
  const bool wrap = w.b2 > 0;
#pragma unroll 1
  for (int e = w.e0; e <= w.e1; e += 2) {
    // Offsets of up to two eta rows (each one or two phi ranges), all loaded
    // before any is used.
    const bool two = e + 1 <= w.e1;
    const unsigned* rA = off + (size_t)e * nphi;
    const unsigned* rB = rA + nphi;
    unsigned o0 = rA[w.b0], o1 = rA[w.b1];
    unsigned o2 = wrap ? rA[0] : 0u, o3 = wrap ? rA[w.b2] : 0u;
    unsigned o4 = two ? rB[w.b0] : 0u, o5 = two ? rB[w.b1] : 0u;
    unsigned o6 = (two && wrap) ? rB[0] : 0u, o7 = (two && wrap) ? rB[w.b2] : 0u;
    // chi2 of one hit; the compatible ones enter the sorted list
    auto consider = [&](const float4& h) {
      float r0, r1;
      c_chi2++;
      if constexpr (DK) {
        if (!residual_disk<float>(p, f, h.x, h.y, r0, r1)) return;
      } else {
        float mx, my, mz;
        corrected_hit(al, h.x, h.y, h.z, mx, my, mz);
        if (!residual<float>(p, f, mx, my, mz, r0, r1)) return;
      }
      const float c2 = chi2_of<float>(f, r0, r1);
      if (!(c2 < cut)) return;
      const unsigned long long key = make_key(nf1, chi2 + c2, slot, 0, __float_as_int(h.w));
      int pos;
      if (cnt < N) pos = cnt++;
      else if (key < lst[N - 1]) pos = N - 1;
      else return;
      while (pos > 0 && lst[pos - 1] > key) { lst[pos] = lst[pos - 1]; --pos; }
      lst[pos] = key;
    };
    if constexpr (BATCH) {
      constexpr int B = 8;
#pragma unroll 1
      for (int part = 0; part < 4; ++part) {
        const unsigned i0 = o0, i1 = o1;
        o0 = o2; o1 = o3; o2 = o4; o3 = o5; o4 = o6; o5 = o7;
#pragma unroll 1
        for (unsigned i = i0; i < i1; i += B) {
          float4 hh[B];
#pragma unroll
          for (int k = 0; k < B; ++k)
            if (i + k < i1) hh[k] = P.hb[i + k];
#pragma unroll
          for (int k = 0; k < B; ++k)
            if (i + k < i1) consider(hh[k]);
        }
      }
    } else {
      // one loop over the (up to four) ranges of the two rows
      const unsigned n0 = o1 - o0, n01 = n0 + (o3 - o2), n012 = n01 + (o5 - o4), tot = n012 + (o7 - o6);
#pragma unroll 1
      for (unsigned t = 0; t < tot; ++t) {
        const unsigned i = t < n0 ? o0 + t : t < n01 ? o2 + (t - n0) : t < n012 ? o4 + (t - n01) : o6 + (t - n012);
        consider(P.hb[i]);
      }
    }
  }
}

// Careful pass: a window of more than BIG_WINDOW_CELLS cells (near-tangent
// predictions can span thousands of hits) is searched by the whole warp
// instead of its lane alone.
constexpr int BIG_WINDOW_CELLS = 1024;
__device__ __forceinline__ int window_cells(const Window& w) {
  return (w.e1 - w.e0 + 1) * (w.b1 - w.b0 + max(w.b2, 0));
}

// The warp searches the window w of lane src (all 32 lanes call this with
// the same src; every argument is read from lane src): each lane tests every
// 32nd hit of each range and keeps its own best max_cands children in
// coop[lane * KF_MAX_CANDS ...]; then max_cands rounds of a warp minimum over
// the lists' heads hand the best keys, in order, to lst (lane src's list).
// Keys are unique, so the result is the single-lane search's.  Returns the
// number of children on every lane.
__device__ __noinline__ int coop_scan(const FindParams& P, int src, Window w, const unsigned* off, Align4 al,
                                      const float* p_src, Frame f, int nf1, float chi2, int slot,
                                      unsigned long long* coop, unsigned long long* lst, unsigned* c_chi2) {
  constexpr unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  w.e0 = __shfl_sync(FULL, w.e0, src);
  w.e1 = __shfl_sync(FULL, w.e1, src);
  w.b0 = __shfl_sync(FULL, w.b0, src);
  w.b1 = __shfl_sync(FULL, w.b1, src);
  w.b2 = __shfl_sync(FULL, w.b2, src);
  off = reinterpret_cast<const unsigned*>(__shfl_sync(FULL, reinterpret_cast<unsigned long long>(off), src));
  al.ca = __shfl_sync(FULL, al.ca, src);
  al.sa = __shfl_sync(FULL, al.sa, src);
  al.az = __shfl_sync(FULL, al.az, src);
  float p[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) p[k] = __shfl_sync(FULL, p_src[k], src);
  f.su = __shfl_sync(FULL, f.su, src);
  f.cu = __shfl_sync(FULL, f.cu, src);
  f.si00 = __shfl_sync(FULL, f.si00, src);
  f.si01 = __shfl_sync(FULL, f.si01, src);
  f.si11 = __shfl_sync(FULL, f.si11, src);
  nf1 = __shfl_sync(FULL, nf1, src);
  chi2 = __shfl_sync(FULL, chi2, src);
  slot = __shfl_sync(FULL, slot, src);
  const int nphi = P.g.n_phi, N = P.g.max_cands;
  const float cut = P.g.chi2_cut;
  unsigned long long* mine = coop + lane * KF_MAX_CANDS;
  int lc = 0;
  unsigned n_eval = 0;
  auto consider = [&](unsigned i) {
    const float4 h = P.hb[i];
    float mx, my, mz;
    corrected_hit(al, h.x, h.y, h.z, mx, my, mz);
    float r0, r1;
    ++n_eval;
    if (!residual<float>(p, f, mx, my, mz, r0, r1)) return;
    const float c2 = chi2_of<float>(f, r0, r1);
    if (!(c2 < cut)) return;
    const unsigned long long key = make_key(nf1, chi2 + c2, slot, 0, __float_as_int(h.w));
    int pos;
    if (lc < N) pos = lc++;
    else if (key < mine[N - 1]) pos = N - 1;
    else return;
    while (pos > 0 && mine[pos - 1] > key) { mine[pos] = mine[pos - 1]; --pos; }
    mine[pos] = key;
  };
#pragma unroll 1
  for (int e = w.e0; e <= w.e1; ++e) {
    const unsigned* row = off + (size_t)e * nphi;
    const unsigned a0 = row[w.b0], a1 = row[w.b1];
    const unsigned c0 = w.b2 > 0 ? row[0] : 0u, c1 = w.b2 > 0 ? row[w.b2] : 0u;
#pragma unroll 1
    for (unsigned i = a0 + lane; i < a1; i += 32) consider(i);
#pragma unroll 1
    for (unsigned i = c0 + lane; i < c1; i += 32) consider(i);
  }
  *c_chi2 += n_eval;
  // merge: the smallest head of the 32 lists, N times
  int head = 0, n = 0;
#pragma unroll 1
  for (; n < N; ++n) {
    const unsigned long long k = head < lc ? mine[head] : KEY_EMPTY;
    const unsigned hi = __reduce_min_sync(FULL, (unsigned)(k >> 32));
    const unsigned lo = __reduce_min_sync(FULL, (unsigned)(k >> 32) == hi ? (unsigned)k : 0xffffffffu);
    const unsigned long long m = ((unsigned long long)hi << 32) | lo;
    if (m == KEY_EMPTY) break;
    if (k == m) ++head;
    if (lane == src) lst[n] = m;
  }
  return n;
}

// Seed fit and first layer, one thread per seed of [s_begin, s_end).
// Seed fit: at the first seed hit the update of the prior, then for the
// second and third hit propagation, transport and update, with the
// scattering of each layer after its update.  First layer after the seed
// (the seed's single candidate): what the group loop does on a layer for one
// live candidate — propagation, window search and its children (hit children
// and the hole child, top max_cands by ranking key).  Outputs: sfit [28][ns]
// the state the children are taken from (the prediction on the first layer,
// or the unchanged state of a carried candidate) and the seed's chi2 sum;
// skeys [max_cands][ns] the children in ascending key order; sflag bit 1 a
// crossing closer to tangent than FIND_CAREFUL_COS (the main pass lists the
// seed for the careful pass without searching it), bit 2 the candidate is
// carried unchanged (no crossing, a far-side seed hit, or a stop), bits 3-7
// the number of children; sfit row 28 the first layer's counts (bits 0-29
// chi2 evaluations, bit 30 a candidate-layer step, bit 31 a prediction
// without positive definite S), which the main pass adds to its counters
// (so that they are dropped with the rest if it gives the seed up later).
// DISK: the seed fit only (the group loop searches the plan's first surface);
// sfit holds the fitted seed after its third layer's scattering, sflag bit 1
// a near-tangent seed step, bit 2 a seed fit that stopped (the candidate is
// finished).
constexpr int SEED_THREADS = 128;
template <bool DISK>
__global__ void __launch_bounds__(SEED_THREADS) k_seed_fit(const FindParams P) {
  __shared__ unsigned long long s_lst[SEED_THREADS][KF_MAX_CANDS];
  const int seed = P.s_begin + blockIdx.x * blockDim.x + threadIdx.x;
  unsigned c_steps = 0, c_chi2 = 0, c_npd = 0;
  if (seed < P.s_end) {
    const DevGeom& g = P.g;
    const size_t ns = (size_t)P.ns;
    const int N = g.max_cands;
    const int ev = P.seed_event[seed];
    const int hoff = P.hit_off[ev];
    float p[6], C[21];
#pragma unroll
    for (int k = 0; k < 6; ++k) p[k] = P.sp[k * ns + seed];
#pragma unroll
    for (int k = 0; k < 21; ++k) C[k] = P.sc[k * ns + seed];
    float chi2 = 0.f;
    bool finished = false, near = loose_prior(C, g);  // a loose prior: the careful pass fits the seed
    int l = 0;
#pragma unroll 1
    for (int it = 0; it < 3; ++it) {
      const int hi = hoff + P.sh[it * ns + seed];
      l = P.hlayer[hi];
      if (finished || near) continue;  // (l still walks to the third seed hit's layer)
      if (it != 0) {
        float q[6], J[6][6], cosa = 1.f;
        const int pr = prop_jacobian<float>(p, g.radius[l], field_kb<float>(g, p), INFINITY, q, J, &cosa);
        if (pr != 1) {
          finished = true;
          continue;
        }
        if (cosa < FIND_CAREFUL_COS) {
          near = true;
          continue;
        }
        transport<float>(J, C);
#pragma unroll
        for (int k = 0; k < 6; ++k) p[k] = q[k];
      }
      float mx, my, mz;
      corrected_hit(P.align[l], P.hx[hi], P.hy[hi], P.hz[hi], mx, my, mz);
      Frame f;
      make_frame<float>(p, C, g.vr, g.vz, f);
      float r0, r1;
      if (!residual<float>(p, f, mx, my, mz, r0, r1)) {
        finished = true;
        continue;
      }
      chi2 += chi2_of<float>(f, r0, r1);
      kf_update<float>(p, C, f, r0, r1);
      add_ms<float>(p, C, x0_at<float>(g, l, p[2]));
      add_eloss_ool<float>(p, C, g.eloss[l]);
    }
    // first layer after the seed
    unsigned long long* lst = s_lst[threadIdx.x];
    int cnt = 0;
    bool carried = true;
    const int L = g.n_layers, l1 = l + 1;
    if (DISK) {
      if (near) finished = false;
      carried = finished;
    } else if (!near && l1 < L) {
      unsigned long long tail = make_key(3, chi2, 0, 1, 0);
      if (!finished) {
        float bp[6], bC[21];  // state before the layer, kept for a stop
#pragma unroll
        for (int k = 0; k < 6; ++k) bp[k] = p[k];
#pragma unroll
        for (int k = 0; k < 21; ++k) bC[k] = C[k];
        const float R = g.radius[l1];
        float q[6], J[6][6], cosa = 1.f;
        const int pr = prop_jacobian<float>(p, R, field_kb<float>(g, p), g.z_max, q, J, &cosa);
        if (pr == 1 && cosa < FIND_CAREFUL_COS) {
          near = true;
        } else if (pr == 1) {
          transport<float>(J, C);
#pragma unroll
          for (int k = 0; k < 6; ++k) p[k] = q[k];
          carried = false;
          c_steps++;
          Frame f;
          make_frame<float>(p, C, g.vr, g.vz, f);
          const bool spd = f.s00 > 0.f && f.si00 > 0.f && f.si11 > 0.f;
          if (!spd) c_npd++;
          const Align4 al = P.align[l1];
          const Window w = window_of(P, l1, R, p, f, spd, al);
          const unsigned* off = P.bin_off + ((size_t)ev * L + l1) * ((size_t)g.n_eta * g.n_phi);
          scan_window<false>(P, off, w, al, p, f, 4, chi2, 0, lst, cnt, c_chi2);
          if (g.max_holes > 0) {
            // hole child
          } else if (cnt == 0) {  // no compatible hit and no hole allowed: stops unchanged
            tail = make_key(3, chi2, 0, 1, 0);
            carried = true;
#pragma unroll
            for (int k = 0; k < 6; ++k) p[k] = bp[k];
#pragma unroll
            for (int k = 0; k < 21; ++k) C[k] = bC[k];
          } else {
            tail = KEY_EMPTY;
          }
        }
      }
      if (!near && tail != KEY_EMPTY) {
        // the hole (or carried) child joins the hit children; the best N stay
        int pos;
        if (cnt < N) pos = cnt++;
        else if (tail < lst[N - 1]) pos = N - 1;
        else pos = -1;
        if (pos >= 0) {
          while (pos > 0 && lst[pos - 1] > tail) { lst[pos] = lst[pos - 1]; --pos; }
          lst[pos] = tail;
        }
      }
    }
    if (near) {
      cnt = 0;
      c_steps = c_chi2 = c_npd = 0;  // the careful pass redoes and counts the seed
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) P.sfit[k * ns + seed] = p[k];
#pragma unroll
    for (int k = 0; k < 21; ++k) P.sfit[(6 + k) * ns + seed] = C[k];
    P.sfit[27 * ns + seed] = chi2;
    P.sfit[28 * ns + seed] = __uint_as_float(min(c_chi2, (1u << 30) - 1u) | (c_steps << 30) | (c_npd << 31));
    for (int k = 0; k < cnt; ++k) P.skeys[k * ns + seed] = lst[k];
    P.sflag[seed] = (unsigned char)((near ? 2u : 0u) | (carried ? 4u : 0u) | ((unsigned)cnt << 3));
  }
}

// EL: the detector has energy loss (the main pass without it carries none of
// its code; the careful pass always does).  DISK: the detector has endcap
// disks (region plans, disk surfaces).
template <int G, int CAP, bool CAREFUL, bool EL, bool DISK = false>
__global__ void __launch_bounds__(CAP ? 128 : 256, CAP ? 5 : 1) k_find(const FindParams P) {
  constexpr int W = 32 / G;  // seeds per warp
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int grp = lane / G;
  const int gl = lane - grp * G;
  const int base = grp * G;
  const bool lane_used = grp < W;
  const DevGeom& g = P.g;
  const int L = g.n_layers;
  const int HL = DISK ? g.n_plan : L;  // history columns: positions of the longest plan
  const int S = DISK ? g.n_surf : L;   // surfaces (hit-list row, cell blocks per event)
  // the eta-bin edges of every layer, copied once per block
  float* const s_edges = reinterpret_cast<float*>(smem);
  for (int i = threadIdx.x; i < L * (g.n_eta + 1); i += blockDim.x) {
    const int l = i / (g.n_eta + 1);
    s_edges[i] = P.eta_edges[(size_t)l * (MAX_ETA_BINS + 1) + (i - l * (g.n_eta + 1))];
  }
  __syncthreads();
  constexpr int LS = list_stride(G, CAREFUL);
  constexpr int SL = smem_list(G, CAREFUL), SG = smem_gather(G, CAREFUL);
  unsigned char* ws = smem + smem_edges(L, g.n_eta) + (size_t)warp * smem_per_warp_k(G, HL, CAREFUL);
  double* const dst_warp = reinterpret_cast<double*>(ws + smem_per_warp(G, CAREFUL, HL));  // careful pass only
  unsigned long long* const coop_warp =
      reinterpret_cast<unsigned long long*>(ws + smem_per_warp(G, CAREFUL, HL) + SMEM_DSTATE);  // careful pass only
  unsigned long long* lst = reinterpret_cast<unsigned long long*>(ws) + lane * LS;
  unsigned long long* gather = reinterpret_cast<unsigned long long*>(ws + SL);
  float* bak = reinterpret_cast<float*>(gather) + lane * BACKUP_STRIDE;
  unsigned long long* slot = reinterpret_cast<unsigned long long*>(ws + SL + SG);
  int* hist = reinterpret_cast<int*>(ws + SL + SG + SMEM_SLOT);
  const int N = g.max_cands;
  const int n_seed_range = CAREFUL ? (int)P.queue[2] : P.s_end - P.s_begin;
  const int n_tasks = (n_seed_range + W - 1) / W;
  const int warps_per_block = blockDim.x >> 5;
  unsigned* const queue = P.queue + (CAREFUL ? 1 : 0);
  // Counters: per-warp sums in shared memory (lane 0 of the warp owns its
  // row), added to the global counters once when the warp ends.
  // per warp: counters 0-6, then (DISK) [8..10] the disk steps, updates, holes
  constexpr int NCNT = DISK ? 11 : 8;
  __shared__ unsigned long long s_cnt[8][NCNT];
  if (lane < NCNT) s_cnt[warp][lane] = 0ull;
  unsigned c_redo = 0;  // seeds given up (kept across tasks: not a per-task count)
  __syncwarp();


  int task;
  if (CAREFUL || P.persistent) {
    unsigned t = 0;
    if (lane == 0) t = atomicAdd(queue, 1u);
    task = (int)__shfl_sync(0xffffffffu, t, 0);
  } else {
    task = blockIdx.x * warps_per_block + warp;
  }

  while (task < n_tasks) {
    int seed;
    bool has_seed;
    if constexpr (CAREFUL) {
      const int j = task * W + grp;
      has_seed = lane_used && j < n_seed_range;
      seed = has_seed ? P.tangent_list[j] : 0;
    } else {
      const int j = P.s_begin + task * W + grp;
      has_seed = lane_used && (j < P.s_end);
      if (has_seed && P.kept_cnt) {  // after seed cleaning: the event's first kept_cnt positions
        const int e = P.seed_event[j];  // positions and seed indices share the event ranges
        has_seed = j - P.seed_off[e] < P.kept_cnt[e];
      }
      seed = has_seed && P.order ? P.order[j] : j;
    }
    // counters of this task (dropped for a seed given up)
    unsigned c_steps = 0, c_updates = 0, c_chi2 = 0, c_seeds = 0, c_holes = 0, c_careful = 0, c_npd = 0;
    unsigned c_dsteps = 0, c_dupdates = 0, c_dholes = 0;  // DISK: the steps, updates and holes on disks
    bool near = false, given_up = false;
    // main pass: the first layer's children, found by the seed kernel (this
    // lane's child and whether their parent was carried or propagated)
    unsigned long long first_key = KEY_EMPTY;
    int first_cls = 0;
    int ev = 0, hoff = 0;
    float p[6], C[21];
    float chi2 = 0.f;
    bool loose = false;  // careful pass: the seed's prior is loose (its steps in double)
    int nfound = 3, nholes = 0;
    bool finished = false;
    bool bdone = false;  // DISK: a forward candidate past the barrel's reach (it passed a barrel layer)
    bool occ = has_seed && gl == 0;
    int sh0 = 0, sh1 = 0, sh2 = 0, sl0 = 0, sl1 = 0, sl2 = 0;
    bool fwd = false, neg = false;  // the seed's region: forward (its side's disks after the barrel), -z side
    if (has_seed) {
      if constexpr (DISK) {
        const float th0 = P.sp[(size_t)5 * P.ns + seed];
        fwd = seed_forward(g, th0);
        neg = seed_eta_negative(th0);
      }
      ev = P.seed_event[seed];
      hoff = P.hit_off[ev];
      sh0 = P.sh[seed];
      sh1 = P.sh[(size_t)P.ns + seed];
      sh2 = P.sh[2 * (size_t)P.ns + seed];
      sl2 = P.hlayer[hoff + sh2];
      if constexpr (CAREFUL) {
        sl0 = P.hlayer[hoff + sh0];
        sl1 = P.hlayer[hoff + sh1];
#pragma unroll
        for (int k = 0; k < 6; ++k) p[k] = P.sp[(size_t)k * P.ns + seed];
#pragma unroll
        for (int k = 0; k < 21; ++k) C[k] = P.sc[(size_t)k * P.ns + seed];
        loose = loose_prior(C, g);
      } else {  // the fitted seed and its first layer
#pragma unroll
        for (int k = 0; k < 6; ++k) p[k] = P.sfit[(size_t)k * P.ns + seed];
#pragma unroll
        for (int k = 0; k < 21; ++k) C[k] = P.sfit[(size_t)(6 + k) * P.ns + seed];
        chi2 = P.sfit[(size_t)27 * P.ns + seed];
        const unsigned flag = P.sflag[seed];
        if (flag & 2u) given_up = true;
        if (DISK) {
          finished = (flag & 4u) != 0;  // the seed fit stopped
        } else {
          first_cls = (flag & 4u) ? 1 : 2;
          if (gl < (int)(flag >> 3)) first_key = P.skeys[(size_t)gl * P.ns + seed];
        }
      }
      if (gl == 0) c_seeds++;
    } else {
#pragma unroll
      for (int k = 0; k < 6; ++k) p[k] = 0.f;
#pragma unroll
      for (int k = 0; k < 21; ++k) C[k] = 0.f;
    }
    const int start = has_seed ? sl2 + 1 : L;           // first layer searched
    // iterations: the three seed hits (careful pass only; the main pass starts
    // from the fitted seed), then the positions of the plan
    int n_iter = has_seed && !given_up ? 3 + (L - start) + (fwd ? g.n_disks : 0) : 0;
    int it_end = __reduce_max_sync(0xffffffffu, n_iter);

#pragma unroll 1
    for (int it = CAREFUL ? 0 : 3; it < it_end; ++it) {
      const bool in_seed = CAREFUL && it < 3;
      const bool active = it < n_iter;
      const int pos = start + (it - 3);  // position in the plan (the history's column)
      const int l = in_seed ? (it == 0 ? sl0 : (it == 1 ? sl1 : sl2)) : (DISK ? plan_surface(g, pos, neg) : pos);
      const bool disk = DISK && !in_seed && is_disk(g, l);
      int cls = 0;  // 1 = carried unchanged, 2 = propagated with hit/hole children
      int cnt = 0;
      bool dbl = false;  // careful pass: the prediction of this layer is kept in double
      unsigned long long tail = KEY_EMPTY;
      // main pass: the first layer after the seed was searched by the seed kernel
      const bool pre = !CAREFUL && !DISK && it == 3;
      // after the window search: the hole child, or the stop of a candidate
      // without a compatible hit and without holes left
      auto after_scan = [&]() {
        if (nholes < g.max_holes) {
          tail = make_key(nfound, chi2, gl, 1, 0);
        } else if (cnt == 0) {
          // no compatible hit and no hole left: the candidate stops unchanged
          cls = 1;
          finished = true;
          tail = make_key(nfound, chi2, gl, 1, 0);
#pragma unroll
          for (int k = 0; k < 6; ++k) p[k] = bak[k];
#pragma unroll
          for (int k = 0; k < 21; ++k) C[k] = bak[6 + k];
        }
      };
      // careful pass: a window too large for one lane, searched by the warp
      // after this block (its window, frame, alignment and cell offsets)
      bool big = false;
      Window bw{};
      Frame bf{};
      Align4 bal{};
      const unsigned* boff = nullptr;
      if (active && occ && !pre) {
        if (finished) {
          cls = 1;
          tail = make_key(nfound, chi2, gl, 1, 0);
        } else {
          if (!in_seed && nholes >= g.max_holes) {  // only such a candidate can stop
#pragma unroll
            for (int k = 0; k < 6; ++k) bak[k] = p[k];
#pragma unroll
            for (int k = 0; k < 21; ++k) bak[6 + k] = C[k];
          }
          const float R = disk ? 0.f : g.radius[l];
          int pr = 1;
          if (disk) {
            // the plane step; a crossing outside the disk's radii is none
            float q[6], J[6][6];
            pr = prop_plane_jacobian<float>(p, plane_z(g, l), field_kb<float>(g, p), q, J) ? 1 : 0;
            if (pr == 1) {
              const float rr = disk_r(q[0], q[1]);
              if (!(rr >= g.disk_rmin && rr <= g.disk_rmax)) pr = 0;
            }
            if (pr == 1) {
              transport_plane<float>(J, C);
#pragma unroll
              for (int k = 0; k < 6; ++k) p[k] = q[k];
            }
          } else if (DISK && fwd && !in_seed && bdone) {
            pr = 0;  // it passed an earlier barrel layer, so it passes this one
          } else if (it != 0) {
            const float z_lim = in_seed ? INFINITY : g.z_max;
            float q[6], J[6][6], cosa = 1.f;
            pr = prop_jacobian<float>(p, R, field_kb<float>(g, p), z_lim, q, J, &cosa);
            if (CAREFUL && pr == 1 && (cosa < FIND_CAREFUL_COS || (in_seed && loose))) {
              float* st = reinterpret_cast<float*>(lst);
#pragma unroll
              for (int k = 0; k < 6; ++k) st[k] = p[k];
#pragma unroll
              for (int k = 0; k < 21; ++k) st[6 + k] = C[k];
              pr = careful_propagate(st, dst_warp + lane * 27, R, g.kb, g.fcz, g.fcr, z_lim);
              dbl = pr == 1;
              if (pr == 1) {
#pragma unroll
                for (int k = 0; k < 6; ++k) p[k] = st[k];
#pragma unroll
                for (int k = 0; k < 21; ++k) C[k] = st[6 + k];
              }
              c_careful++;
            } else if (pr == 1) {
              if (!CAREFUL && cosa < FIND_CAREFUL_COS) near = true;
              transport<float>(J, C);
#pragma unroll
              for (int k = 0; k < 6; ++k) p[k] = q[k];
            }
          }
          if (pr != 1) {
            // no crossing: on a forward plan the surface is passed (cls 3),
            // else the candidate has left the detector
            cls = fwd && !in_seed ? 3 : 1;
            finished = cls == 1;
            tail = make_key(nfound, chi2, gl, 1, 0);
          } else {
            cls = 2;
            if (!in_seed && disk) {
              c_steps++;
              c_dsteps++;
              DiskFrameT<float> d;
              make_frame_disk<float>(p, C, g.vr, g.vrr, d);
              const bool spd = d.f.s00 > 0.f && d.f.si00 > 0.f && d.f.si11 > 0.f;
              if (!spd) c_npd++;
              const Window w = window_disk(P, p, d.f, spd);
              const unsigned* off = P.bin_off + ((size_t)ev * S + l) * ((size_t)g.n_eta * g.n_phi);
              scan_window<CAREFUL, true>(P, off, w, Align4{1.f, 0.f, 0.f, 0.f}, p, d.f, nfound + 1, chi2, gl, lst,
                                         cnt, c_chi2);
              after_scan();
            } else if (!in_seed) {
              c_steps++;
              Frame f;
              if (CAREFUL && dbl) f = careful_frame(dst_warp + lane * 27, g.vr, g.vz);
              else make_frame<float>(p, C, g.vr, g.vz, f);
              // A prediction without a positive definite S searches no hits
              // (the careful propagation should leave none; counted).
              const bool spd = f.s00 > 0.f && f.si00 > 0.f && f.si11 > 0.f;
              if (!spd) c_npd++;
              const Align4 al = P.align[l];
              const Window w = window_of(P, l, R, p, f, spd, al, s_edges);
              const unsigned* off = P.bin_off + ((size_t)ev * S + l) * ((size_t)g.n_eta * g.n_phi);
              if (CAREFUL && window_cells(w) > BIG_WINDOW_CELLS) {
                big = true;
                bw = w;
                bf = f;
                bal = al;
                boff = off;
              } else {
                scan_window<CAREFUL>(P, off, w, al, p, f, nfound + 1, chi2, gl, lst, cnt, c_chi2);
                after_scan();
              }
            }
          }
        }
      }
      if constexpr (CAREFUL) {  // the large windows, one after another, by the whole warp
        unsigned pend = __ballot_sync(0xffffffffu, big);
        while (pend) {
          const int src = __ffs(pend) - 1;
          pend &= pend - 1;
          const int n = coop_scan(P, src, bw, boff, bal, p, bf, nfound + 1, chi2, gl, coop_warp, lst, &c_chi2);
          if (lane == src) cnt = n;
        }
        if (big) after_scan();
      }

      // Top-N of all children of each group (layers only; a group in its seed
      // fit keeps its single candidate).
      unsigned long long mine = KEY_EMPTY;
      int par = gl, p_holes = nholes, p_cls = cls;
      bool p_dbl = dbl;
      // The chosen hit's coordinates are loaded as soon as the child is known,
      // so that the load overlaps the state exchange.
      float hit_x = 0.f, hit_y = 0.f, hit_z = 0.f;
      auto fetch_hit = [&]() {
        if (active && mine != KEY_EMPTY && !key_nonhit(mine)) {
          const int hi = hoff + key_hit(mine);
          hit_x = __ldg(P.hx + hi);
          hit_y = __ldg(P.hy + hi);
          hit_z = __ldg(P.hz + hi);
        }
      };
      if constexpr (!CAREFUL) {
        // A group with a near-tangent crossing gives its seed up after this
        // layer (its lanes go idle) and lists it for the careful pass.
        const unsigned nb = __ballot_sync(0xffffffffu, near);
        if (lane_used && ((nb >> base) & ((1u << G) - 1u)) && !given_up) {
          given_up = true;
          n_iter = min(n_iter, it + 1);
        }
      }
      if (pre) {
        // the children of the seed's candidate, in rank order, one per lane;
        // every lane holds their parent's state already
        mine = lane_used ? first_key : KEY_EMPTY;
        fetch_hit();
        par = 0;
        p_holes = 0;
        p_cls = first_cls;
      } else if (DISK && __any_sync(0xffffffffu, active && !in_seed) &&
                 !__any_sync(0xffffffffu, active && !in_seed && occ && cls == 2)) {
        // Every candidate of the warp is carried unchanged (a surface passed
        // on a forward plan, or finished): the selection would keep each in
        // its slot -- the slots are in key order, and a carried child's key
        // (hits, chi2 sum, its own slot) keeps that order -- so it is skipped.
        mine = (active && occ) ? make_key(nfound, chi2, gl, 1, 0) : KEY_EMPTY;
      } else if (__any_sync(0xffffffffu, active && !in_seed)) {
        // Rank of each child = its position in its own sorted list + the
        // number of smaller keys in the other lists of the group (keys are
        // unique); the children of rank < N go to the slots of their rank.
        if (tail != KEY_EMPTY) lst[cnt++] = tail;
        // Pack the group's children into one array: exclusive prefix of the
        // list lengths over the group's lanes.
        int incl = cnt;
#pragma unroll
        for (int off = 1; off < G; off <<= 1) {
          const int v = __shfl_up_sync(0xffffffffu, incl, off);
          if (gl >= off) incl += v;
        }
        const int M = __shfl_sync(0xffffffffu, incl, min(base + G - 1, 31));
        unsigned long long* A = gather + base * LS;
        for (int j = 0, o = incl - cnt; j < cnt; ++j) A[o + j] = lst[j];
        // An odd count is padded with an empty key (never smaller), so that
        // the ranking reads two keys per 16-byte load.  The group's area holds
        // G (G + 1) keys, an even number, so an odd count leaves room for the
        // pad; it starts on a 16-byte boundary for the same reason.
        if (gl == G - 1 && (M & 1)) A[M] = KEY_EMPTY;
        slot[lane] = KEY_EMPTY;
        __syncwarp();
        // rank = number of smaller keys in the group (keys are unique)
        const ulonglong2* A2 = reinterpret_cast<const ulonglong2*>(A);
#pragma unroll 1
        for (int m = gl; m < M && lane_used; m += G) {
          const unsigned long long key = A[m];
          int rank = 0;
#pragma unroll 4
          for (int q = 0; q < (M + 1) / 2; ++q) {
            const ulonglong2 v = A2[q];
            rank += (v.x < key ? 1 : 0) + (v.y < key ? 1 : 0);
          }
          if (rank < N) slot[base + rank] = key;
        }
        __syncwarp();
        if (lane_used && gl < N) mine = slot[lane];
        fetch_hit();
        // Pull the parent's exported state (the prediction, or the unchanged
        // state of a carried candidate) through shared memory: every lane
        // writes its 27 values to the packed-children area (no longer read
        // after the selection; rows of 27 floats, so that the 32 lanes fall in
        // distinct banks), then reads its parent's row.
        par = (mine != KEY_EMPTY) ? key_parent(mine) : gl;
        const int src = lane_used ? base + par : lane;
        float* xs = reinterpret_cast<float*>(gather);
#pragma unroll
        for (int k = 0; k < 6; ++k) xs[lane * 27 + k] = p[k];
#pragma unroll
        for (int k = 0; k < 21; ++k) xs[lane * 27 + 6 + k] = C[k];
        p_holes = __shfl_sync(0xffffffffu, nholes, src);
        p_cls = __shfl_sync(0xffffffffu, cls, src);
        if constexpr (CAREFUL) p_dbl = __shfl_sync(0xffffffffu, (int)dbl, src) != 0;
        __syncwarp();
        if (active && !in_seed) {
#pragma unroll
          for (int k = 0; k < 6; ++k) p[k] = xs[src * 27 + k];
#pragma unroll
          for (int k = 0; k < 21; ++k) C[k] = xs[src * 27 + 6 + k];
        }
        __syncwarp();
      }

      if (active) {
        // What the lane does with its (new) candidate on this layer.
        bool do_update = false, do_ms = false;
        int hit = 0;
        if (in_seed) {
          do_update = occ && cls == 2;
          hit = it == 0 ? sh0 : (it == 1 ? sh1 : sh2);
        } else if (mine == KEY_EMPTY) {
          occ = false;
        } else {
          occ = true;
          nfound = key_nfound(mine);
          chi2 = key_chi2(mine);
          nholes = p_holes;
          if (!key_nonhit(mine)) {
            do_update = true;
            hit = key_hit(mine);
            finished = false;
            bdone = false;
          } else if (p_cls == 2) {
            nholes += 1;
            do_ms = true;
            finished = false;
            bdone = false;
            c_holes++;
            if (disk) c_dholes++;
          } else {
            finished = p_cls != 3;  // 3: the surface was passed, the search goes on
            bdone = DISK && p_cls == 3;
          }
          hist[(grp * HL + pos) * G + gl] = (par << 24) | (do_update ? hit + 1 : 0);
        }
        if (CAREFUL && p_dbl && (do_update || do_ms)) {
          // child of a double-precision prediction (the parent's, or the
          // lane's own in the seed fit)
          float mx = 0.f, my = 0.f, mz = 0.f;
          if (do_update) {
            const int hi = hoff + hit;
            corrected_hit(P.align[l], P.hx[hi], P.hy[hi], P.hz[hi], mx, my, mz);
          }
          float* st = reinterpret_cast<float*>(lst);
          float dchi2 = 0.f;
          const double* in = dst_warp + (in_seed ? lane : base + par) * 27;
          if (careful_child(in, st, mx, my, mz, do_update, do_ms, g, l, &dchi2)) {
            if (do_update) {
              if (in_seed) chi2 += dchi2;
              if (!in_seed) c_updates++;
            }
          } else {
            finished = true;  // far-side seed hit: the seed fit stops here
          }
#pragma unroll
          for (int k = 0; k < 6; ++k) p[k] = st[k];
#pragma unroll
          for (int k = 0; k < 21; ++k) C[k] = st[6 + k];
          do_update = do_ms = false;
        }
        if (do_update && CAREFUL && in_seed && it == 0 && loose) {
          // the first update against a loose prior in double
          const int hi = hoff + hit;
          float mx, my, mz;
          corrected_hit(P.align[l], P.hx[hi], P.hy[hi], P.hz[hi], mx, my, mz);
          if (!first_update_double(p, C, g, l, mx, my, mz, true, chi2)) finished = true;
          do_update = do_ms = false;
        }
        if (disk && do_update) {
          DiskFrameT<float> d;
          make_frame_disk<float>(p, C, g.vr, g.vrr, d);
          float r0, r1;
          if (residual_disk<float>(p, d.f, hit_x, hit_y, r0, r1)) {
            kf_update_disk<float>(p, C, d, r0, r1);
            do_ms = true;
            c_updates++;
            c_dupdates++;
          }
          do_update = false;
        }
        if (disk && do_ms) {
          add_ms_disk<float>(p, C, g.disk_x0);
          add_eloss_ool<float, true>(p, C, g.disk_eloss);
          do_ms = false;
        }
        if (do_update) {
          float mx, my, mz;
          if (in_seed) {
            const int hi = hoff + hit;
            hit_x = P.hx[hi];
            hit_y = P.hy[hi];
            hit_z = P.hz[hi];
          }
          corrected_hit(P.align[l], hit_x, hit_y, hit_z, mx, my, mz);
          Frame f;
          make_frame<float>(p, C, g.vr, g.vz, f);
          float r0, r1;
          if (residual<float>(p, f, mx, my, mz, r0, r1)) {
            if (in_seed) chi2 += chi2_of<float>(f, r0, r1);
            kf_update<float>(p, C, f, r0, r1);
            do_ms = true;
            if (!in_seed) c_updates++;
          } else {
            finished = true;  // far-side seed hit: the seed fit stops here
          }
        }
        if (do_ms) {
          add_ms<float>(p, C, x0_at<float>(g, l, p[2]));
          if constexpr (EL) add_eloss_ool<float>(p, C, g.eloss[l]);
        }
      }
      // A group whose candidates are all finished (carried unchanged) or
      // empty would only carry them on, each to its own slot, layer after
      // layer: its seed's search ends here (the backtrack starts from the
      // last layer searched), and the warp ends with its last live group.
      if (!in_seed) {
        const unsigned live = __ballot_sync(0xffffffffu, active && occ && !finished);
        if (lane_used && active && !((live >> base) & ((1u << G) - 1u))) n_iter = min(n_iter, it + 1);
        it_end = __reduce_max_sync(0xffffffffu, n_iter);
      }
      if constexpr (DISK) {
        // A forward candidate that passed a barrel layer passes every later
        // one: it moves outward from its last crossing, so a larger radius
        // comes later along the helix (or never), and |z|, already beyond
        // z_max, grows along it.  When every live candidate of the warp has
        // passed one, the warp goes on at the first disk of its plans; each
        // position skipped carries every candidate in its slot (what the
        // passes would do).
        if (!in_seed && __any_sync(0xffffffffu, lane_used && active && occ && !finished) &&
            !__any_sync(0xffffffffu, lane_used && active && occ && !finished && !bdone)) {
          const int first_disk = __reduce_min_sync(0xffffffffu, lane_used && active ? 3 + (L - start) : 0x7fffffff);
          if (first_disk > it + 1 && first_disk != 0x7fffffff) {
            for (int q = it + 1; q < first_disk; ++q)
              if (lane_used && q < n_iter) hist[(grp * HL + start + (q - 3)) * G + gl] = gl << 24;
            it = first_disk - 1;
          }
        }
      }
      __syncwarp();
    }

    if constexpr (!CAREFUL) {
      if (has_seed && gl == 0) {  // the first layer's counts, from the seed kernel
        const unsigned c = __float_as_uint(P.sfit[(size_t)28 * P.ns + seed]);
        c_chi2 += c & ((1u << 30) - 1u);
        c_steps += (c >> 30) & 1u;
        c_npd += c >> 31;
      }
    }
    if (given_up) {
      if (has_seed && gl == 0) {
        P.tangent_list[atomicAdd(P.queue + 2, 1u)] = seed;
        ++c_redo;
      }
      c_steps = c_updates = c_chi2 = c_seeds = c_holes = c_npd = 0;
      c_dsteps = c_dupdates = c_dholes = 0;
    }
    // Counters of the task: summed over the warp into its shared row.
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      c_steps += __shfl_xor_sync(0xffffffffu, c_steps, off);
      c_updates += __shfl_xor_sync(0xffffffffu, c_updates, off);
      c_chi2 += __shfl_xor_sync(0xffffffffu, c_chi2, off);
      c_seeds += __shfl_xor_sync(0xffffffffu, c_seeds, off);
      c_holes += __shfl_xor_sync(0xffffffffu, c_holes, off);
      c_careful += __shfl_xor_sync(0xffffffffu, c_careful, off);
      c_npd += __shfl_xor_sync(0xffffffffu, c_npd, off);
      if constexpr (DISK) {
        c_dsteps += __shfl_xor_sync(0xffffffffu, c_dsteps, off);
        c_dupdates += __shfl_xor_sync(0xffffffffu, c_dupdates, off);
        c_dholes += __shfl_xor_sync(0xffffffffu, c_dholes, off);
      }
    }
    if (lane == 0) {
      s_cnt[warp][0] += c_steps;
      s_cnt[warp][1] += c_updates;
      s_cnt[warp][2] += c_chi2;
      s_cnt[warp][3] += c_seeds;
      s_cnt[warp][4] += c_holes;
      s_cnt[warp][5] += c_careful;
      s_cnt[warp][6] += c_npd;
      if constexpr (DISK) {
        s_cnt[warp][NCNT - 3] += c_dsteps;
        s_cnt[warp][NCNT - 2] += c_dupdates;
        s_cnt[warp][NCNT - 1] += c_dholes;
      }
    }
    // The best candidate sits in slot 0: rebuild its hit list.
    if (has_seed && gl == 0 && !given_up) {
      int* oh = P.out_hits + (size_t)seed * S;
      int k = nfound - 1;
      int cur = 0;
      for (int q = start + n_iter - 4; q >= start; --q) {  // from the last plan position searched
        const int e = hist[(grp * HL + q) * G + cur];
        if (e & 0xFFFFFF) oh[k--] = (e & 0xFFFFFF) - 1;
        cur = e >> 24;
      }
      oh[0] = sh0;
      oh[1] = sh1;
      oh[2] = sh2;
      for (int j = nfound; j < S; ++j) oh[j] = -1;
      P.out_n[seed] = nfound;
      P.out_chi2[seed] = chi2;
#pragma unroll
      for (int q = 0; q < 6; ++q) P.out_p[(size_t)q * P.ns + seed] = p[q];
#pragma unroll
      for (int q = 0; q < 21; ++q) P.out_C[(size_t)q * P.ns + seed] = C[q];
    }
    __syncwarp();

    if (CAREFUL || P.persistent) {
      unsigned t = 0;
      if (lane == 0) t = atomicAdd(queue, 1u);
      task = (int)__shfl_sync(0xffffffffu, t, 0);
    } else {
      break;
    }
  }
  __syncwarp();
  if (lane < 7 && P.counters && s_cnt[warp][lane]) atomicAdd(&P.counters[lane], s_cnt[warp][lane]);
  if constexpr (DISK) {
    if (lane >= 8 && lane < NCNT && P.counters && s_cnt[warp][lane]) atomicAdd(&P.counters[lane], s_cnt[warp][lane]);
  }
  if (c_redo && P.counters) atomicAdd(&P.counters[7], (unsigned long long)c_redo);
}

// The main-pass kernel of a variant: DISK kernels carry the energy-loss code
// (the loss is tested at run time); barrel kernels with EL only when a layer
// has a loss.
template <int G, int CAP, bool DISK, bool EL>
__host__ auto main_kernel() {
  if constexpr (DISK) return k_find<G, CAP, false, true, true>;
  else return k_find<G, CAP, false, EL, false>;
}

// n_layers: barrel layers (the eta-edge table); n_hist: history columns (the
// longest plan).
template <int G, int CAP, bool DISK>
cudaError_t prepare_t(int threads, int n_layers, int n_hist, int n_eta, int* blocks_per_sm) {
  const size_t smem = smem_edges(n_layers, n_eta) + (size_t)(threads / 32) * smem_per_warp(G, false, n_hist);
  cudaError_t err =
      cudaFuncSetAttribute(main_kernel<G, CAP, DISK, false>(), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err == cudaSuccess && !DISK)
    err = cudaFuncSetAttribute(main_kernel<G, CAP, DISK, true>(), cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem);
  if (err == cudaSuccess)
    err = cudaFuncSetAttribute(k_find<G, 0, true, true, DISK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)(smem_edges(n_layers, n_eta) +
                                     (CAREFUL_THREADS / 32) * smem_per_warp_k(G, n_hist, true)));
  if (err != cudaSuccess) return err;
  cudaFuncAttributes fa;
  err = cudaFuncGetAttributes(&fa, main_kernel<G, CAP, DISK, false>());
  if (err != cudaSuccess) return err;
  if (threads > fa.maxThreadsPerBlock) {  // the launch bounds forbid this block size
    if (blocks_per_sm) *blocks_per_sm = 0;
    return cudaSuccess;
  }
  if (blocks_per_sm)
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, main_kernel<G, CAP, DISK, false>(), threads,
                                                        smem);
  return err;
}

template <int G, int CAP, bool DISK>
cudaError_t launch_main_t(const FindParams& P, int threads, int grid_cap, cudaStream_t st) {
  const int n_hist = DISK ? P.g.n_plan : P.g.n_layers;
  const size_t smem =
      smem_edges(P.g.n_layers, P.g.n_eta) + (size_t)(threads / 32) * smem_per_warp(G, false, n_hist);
  constexpr int W = 32 / G;
  const int n = P.s_end - P.s_begin;
  const int n_tasks = (n + W - 1) / W;
  const int wpb = threads / 32;
  int grid = (n_tasks + wpb - 1) / wpb;
  if (P.persistent && grid_cap > 0 && grid > grid_cap) grid = grid_cap;
  if (grid < 1) grid = 1;
  bool el = false;  // energy loss on any layer: the variant with its code
  for (int l = 0; l < P.g.n_layers; ++l) el = el || P.g.eloss[l] > 0.f;
  const auto kern = (DISK || !el) ? main_kernel<G, CAP, DISK, false>() : main_kernel<G, CAP, DISK, true>();
  kern<<<grid, threads, smem, st>>>(P);
  return cudaGetLastError();
}

template <int G, int CAP, bool DISK>
cudaError_t launch_careful_t(const FindParams& P, int grid, cudaStream_t st) {
  const int n_hist = DISK ? P.g.n_plan : P.g.n_layers;
  const size_t smem =
      smem_edges(P.g.n_layers, P.g.n_eta) + (size_t)(CAREFUL_THREADS / 32) * smem_per_warp_k(G, n_hist, true);
  k_find<G, 0, true, true, DISK><<<grid, CAREFUL_THREADS, smem, st>>>(P);
  return cudaGetLastError();
}

// Kernel variants: lanes per seed G x register budget CAP (regcap).
#define KF_FIND_DISPATCH(FN, ...)                                   \
  switch (lanes * 4 + (regcap ? 1 : 0)) {                          \
    case 4 * 4: return FN<4, 0>(__VA_ARGS__);                      \
    case 4 * 4 + 1: return FN<4, 1>(__VA_ARGS__);                  \
    case 6 * 4: return FN<6, 0>(__VA_ARGS__);                      \
    case 6 * 4 + 1: return FN<6, 1>(__VA_ARGS__);                  \
    case 8 * 4: return FN<8, 0>(__VA_ARGS__);                      \
    case 8 * 4 + 1: return FN<8, 1>(__VA_ARGS__);                  \
    case 10 * 4: return FN<10, 0>(__VA_ARGS__);                    \
    case 10 * 4 + 1: return FN<10, 1>(__VA_ARGS__);                \
    case 12 * 4: return FN<12, 0>(__VA_ARGS__);                    \
    case 12 * 4 + 1: return FN<12, 1>(__VA_ARGS__);                \
    case 16 * 4: return FN<16, 0>(__VA_ARGS__);                    \
    case 16 * 4 + 1: return FN<16, 1>(__VA_ARGS__);                \
    default: return cudaErrorInvalidValue;                         \
  }

}  // namespace

}  // namespace kfg
