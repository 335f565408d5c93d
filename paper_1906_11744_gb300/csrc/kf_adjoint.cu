// Adjoint of the Kalman re-fit: d(sum of chi2)/d(layer alignment offsets, hit
// positions, seed parameters), one thread per track.
//
// Forward: the fit of kf_fit.cu (prior at the first hit; per hit: propagate,
// tangent-frame measurement, chi2, update, scattering except after the last)
// writes the state (p, C) before every `stride`-th hit as a checkpoint.
// Reverse: for each segment from the last, the states before each step are
// recomputed from the segment's checkpoint, then the steps are reversed one
// by one:
//   * scattering C += Q(p): dQ/dp by forward-mode dual numbers (5 directions);
//   * update and chi2 with U = C H^T, S = H U + V, K = U S^-1,
//       p' = p + U S^-1 r,  C' = C - U S^-1 U^T,  chi2 = r^T S^-1 r,
//     reversed with the matrix identities dS^-1 = -S^-1 dS S^-1 (adjoints of
//     U, S^-1, r, H and C by hand);
//   * the measurement frame H(p) and residual r(p, m), m = R(-a_rphi/R_L) h - a_z e_z;
//   * propagation q = F(p), C' = J C J^T: Cbar <- J^T Cbar' J,
//     pbar <- J^T pbar' + sum_ij Jbar_ij dJ_ij/dp with Jbar = 2 Cbar' J C and
//     dJ/dp from the same propagation code run on dual numbers.
// The adjoint of the final state is zero: the objective is the chi2 sum.
// Tracks the fit flagged for a near-tangent crossing go to a second pass that
// keeps their adjoints in double and runs the near-tangent steps in double.
#include <type_traits>

#include "kf_dual.cuh"
#include "kf_internal.h"

namespace kfg {

namespace {

constexpr float ADJ_CAREFUL_COS = 0.5f;
constexpr int NDIR = 5;  // dual directions: x, y, q/pT, phi, theta
__device__ __forceinline__ int dir_param(int d) { return d < 2 ? d : d + 1; }

template <class S>
struct Hit {
  S mx, my, mz;   // corrected position
  S ca, sa, R;    // correction rotation and layer radius
  int L;
};

template <class S>
__device__ __forceinline__ Hit<S> load_hit(const AdjParams& P, int hi) {
  Hit<S> h;
  h.L = P.hlayer[hi];
  const Align4 a = P.align[h.L];
  const S x = (S)P.hx[hi], y = (S)P.hy[hi], z = (S)P.hz[hi];
  h.ca = (S)a.ca;
  h.sa = (S)a.sa;
  h.R = (S)P.g.radius[h.L];
  h.mx = kfma(h.ca, x, -h.sa * y);
  h.my = kfma(h.sa, x, h.ca * y);
  h.mz = z - (S)a.az;
  return h;
}

// One forward fit step (as kf_fit.cu).  Returns false if the step fails or,
// for float, when the crossing is near-tangent (the track then goes to the
// double-precision pass).
template <class S>
__device__ __forceinline__ int fwd_step(const DevGeom& g, S (&p)[6], S (&C)[21], const Hit<S>& h, bool first,
                                        bool last) {
  if (!first) {
    S cosa = S(1);
    if (propagate<S>(p, C, h.R, (S)g.kb, S(INFINITY), &cosa) != 1) return KF_FIT_NO_CROSS;
    if (sizeof(S) == 4 && cosa < S(ADJ_CAREFUL_COS)) return 99;
  }
  FrameT<S> f;
  make_frame<S>(p, C, (S)g.vr, (S)g.vz, f);
  S r0, r1;
  if (!residual<S>(p, f, h.mx, h.my, h.mz, r0, r1)) return KF_FIT_FAR_SIDE;
  kf_update<S>(p, C, f, r0, r1);
  if (!last) add_ms<S>(p, C, (S)g.x0[h.L]);
  return KF_FIT_OK;
}

// Reverse of one step.  In: the state before the step (p_in, C_in), the
// adjoints of the state after it (pb, Cb: Cb a full symmetric 6x6).  Out: pb,
// Cb replaced by the adjoints of the state before it; the hit and alignment
// gradients of this step in hb[3], ab[2].
template <class S>
__device__ __forceinline__ void rev_step(const DevGeom& g, const S (&p_in)[6], const S (&C_in)[21],
                                         const Hit<S>& h, bool first, bool last, S (&pb)[6], S (&Cb)[6][6],
                                         S (&hb)[3], S (&ab)[2]) {
  using D = Dual<S, NDIR>;
  // ---- forward recompute of the step
  S q[6], J[6][6], Cp[21];
  S dJ[6][6][NDIR];  // dJ_ij / d(direction)
#pragma unroll
  for (int k = 0; k < 21; ++k) Cp[k] = C_in[k];
  if (!first) {
    D pd[6], qd[6], Jd[6][6];
#pragma unroll
    for (int k = 0; k < 6; ++k) pd[k] = D::of(p_in[k]);
#pragma unroll
    for (int d = 0; d < NDIR; ++d) pd[dir_param(d)].d[d] = S(1);
    prop_jacobian<D>(pd, D::of(h.R), D::of((S)g.kb), D::of(S(INFINITY)), qd, Jd);
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      q[i] = qd[i].v;
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        if (JS(i, j) != 2) continue;
        J[i][j] = Jd[i][j].v;
#pragma unroll
        for (int d = 0; d < NDIR; ++d) dJ[i][j][d] = Jd[i][j].d[d];
      }
    }
    transport<S>(J, Cp);
  } else {
#pragma unroll
    for (int k = 0; k < 6; ++k) q[k] = p_in[k];
  }
  const S rho2 = kfma(q[0], q[0], q[1] * q[1]);
  const S irho = krsqrt(rho2);
  const S cu = q[0] * irho, su = q[1] * irho;
  S U[6][2];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    U[i][0] = kfma(-su, Cp[S6(i, 0)], cu * Cp[S6(i, 1)]);
    U[i][1] = Cp[S6(i, 2)];
  }
  const S s00 = kfma(-su, U[0][0], kfma(cu, U[1][0], (S)g.vr));
  const S s01 = U[2][0];
  const S s11 = Cp[S6(2, 2)] + (S)g.vz;
  const S idet = S(1) / kfma(s00, s11, -s01 * s01);
  const S si00 = s11 * idet, si01 = -s01 * idet, si11 = s00 * idet;
  const S r0 = kfma(-su, h.mx - q[0], cu * (h.my - q[1]));
  const S r1 = h.mz - q[2];
  const S sir0 = kfma(si00, r0, si01 * r1), sir1 = kfma(si01, r0, si11 * r1);
  S pu[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) pu[i] = q[i] + kfma(U[i][0], sir0, U[i][1] * sir1);

  // ---- reverse: scattering, C_out = C_upd + Q(p_upd)
  S pbu[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) pbu[i] = pb[i];
  if (!last) {
    D pd[6], q44, q55;
#pragma unroll
    for (int k = 0; k < 6; ++k) pd[k] = D::of(pu[k]);
#pragma unroll
    for (int d = 0; d < NDIR; ++d) pd[dir_param(d)].d[d] = S(1);
    ms_terms<D>(pd, D::of((S)g.x0[h.L]), q44, q55);
#pragma unroll
    for (int d = 0; d < NDIR; ++d)
      pbu[dir_param(d)] = kfma(Cb[4][4], q44.d[d], kfma(Cb[5][5], q55.d[d], pbu[dir_param(d)]));
  }
  // ---- reverse: update and chi2 (chi2 adjoint 1)
  const S w0 = [&] { S a = S(0); for (int i = 0; i < 6; ++i) a = kfma(U[i][0], pbu[i], a); return a; }();
  const S w1 = [&] { S a = S(0); for (int i = 0; i < 6; ++i) a = kfma(U[i][1], pbu[i], a); return a; }();
  // rbar = S^-1 w + 2 S^-1 r
  const S rb0 = kfma(si00, w0, si01 * w1) + S(2) * sir0;
  const S rb1 = kfma(si01, w0, si11 * w1) + S(2) * sir1;
  // Sibar = w r^T - U^T Cb U + r r^T   (2x2)
  S CbU[6][2];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    S a0 = S(0), a1 = S(0);
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      a0 = kfma(Cb[i][j], U[j][0], a0);
      a1 = kfma(Cb[i][j], U[j][1], a1);
    }
    CbU[i][0] = a0;
    CbU[i][1] = a1;
  }
  S UCU00 = S(0), UCU01 = S(0), UCU10 = S(0), UCU11 = S(0);
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    UCU00 = kfma(U[i][0], CbU[i][0], UCU00);
    UCU01 = kfma(U[i][0], CbU[i][1], UCU01);
    UCU10 = kfma(U[i][1], CbU[i][0], UCU10);
    UCU11 = kfma(U[i][1], CbU[i][1], UCU11);
  }
  const S Sib00 = w0 * r0 - UCU00 + r0 * r0, Sib01 = w0 * r1 - UCU01 + r0 * r1;
  const S Sib10 = w1 * r0 - UCU10 + r1 * r0, Sib11 = w1 * r1 - UCU11 + r1 * r1;
  // Sbar = -S^-1 Sibar S^-1
  const S t00 = kfma(si00, Sib00, si01 * Sib10), t01 = kfma(si00, Sib01, si01 * Sib11);
  const S t10 = kfma(si01, Sib00, si11 * Sib10), t11 = kfma(si01, Sib01, si11 * Sib11);
  const S Sb00 = -kfma(t00, si00, t01 * si01), Sb01 = -kfma(t00, si01, t01 * si11);
  const S Sb10 = -kfma(t10, si00, t11 * si01), Sb11 = -kfma(t10, si01, t11 * si11);
  // Ubar = pbu (S^-1 r)^T - 2 Cb U S^-1 + H^T Sbar
  S Ub[6][2];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    Ub[i][0] = pbu[i] * sir0 - S(2) * kfma(CbU[i][0], si00, CbU[i][1] * si01);
    Ub[i][1] = pbu[i] * sir1 - S(2) * kfma(CbU[i][0], si01, CbU[i][1] * si11);
  }
  Ub[0][0] = kfma(-su, Sb00, Ub[0][0]);
  Ub[0][1] = kfma(-su, Sb01, Ub[0][1]);
  Ub[1][0] = kfma(cu, Sb00, Ub[1][0]);
  Ub[1][1] = kfma(cu, Sb01, Ub[1][1]);
  Ub[2][0] += Sb10;
  Ub[2][1] += Sb11;
  // Hbar (row 0, columns x and y) = Sbar U^T + Ubar^T C_pred
  S Hb00 = kfma(Sb00, U[0][0], Sb01 * U[0][1]);
  S Hb01 = kfma(Sb00, U[1][0], Sb01 * U[1][1]);
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    Hb00 = kfma(Ub[i][0], Cp[S6(i, 0)], Hb00);
    Hb01 = kfma(Ub[i][0], Cp[S6(i, 1)], Hb01);
  }
  // Cbar_pred = Cb + sym(Ubar H), H row 0 = (-su, cu, 0..), row 1 = e_z
  S Cbp[6][6];
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int j = 0; j < 6; ++j) Cbp[i][j] = Cb[i][j];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    const S v0 = S(0.5) * -su * Ub[i][0], v1 = S(0.5) * cu * Ub[i][0], v2 = S(0.5) * Ub[i][1];
    Cbp[i][0] += v0; Cbp[0][i] += v0;
    Cbp[i][1] += v1; Cbp[1][i] += v1;
    Cbp[i][2] += v2; Cbp[2][i] += v2;
  }
  // pbar of the prediction: pass-through, residual, frame
  S pbp[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) pbp[i] = pbu[i];
  const S irho3 = irho * irho * irho;
  const S mq = kfma(h.mx, q[0], h.my * q[1]);
  pbp[0] = kfma(rb0, q[1] * mq * irho3, pbp[0]);
  pbp[1] = kfma(-rb0, q[0] * mq * irho3, pbp[1]);
  pbp[2] -= rb1;
  pbp[0] = kfma(Hb00, q[0] * q[1] * irho3, kfma(Hb01, q[1] * q[1] * irho3, pbp[0]));
  pbp[1] = kfma(-Hb00, q[0] * q[0] * irho3, kfma(-Hb01, q[0] * q[1] * irho3, pbp[1]));
  // hit and alignment
  const S mbx = -su * rb0, mby = cu * rb0, mbz = rb1;
  hb[0] = kfma(h.ca, mbx, h.sa * mby);
  hb[1] = kfma(-h.sa, mbx, h.ca * mby);
  hb[2] = mbz;
  const S alpha_b = kfma(-h.my, mbx, h.mx * mby);  // d/d(rotation angle)
  ab[0] = -alpha_b / h.R;                           // angle = -a_rphi / R
  ab[1] = -mbz;
  // ---- reverse: propagation
  if (first) {
#pragma unroll
    for (int i = 0; i < 6; ++i) pb[i] = pbp[i];
    return;
  }
  // Jbar = 2 Cbar' J C_in ; pbar_in = J^T pbar' + sum Jbar_ij dJ_ij/dp
  S CJ[6][6];  // (J C_in)^T rows: CJ[k][j] = (J C_in)_jk = sum_l J_jl C_in_lk
#pragma unroll
  for (int j = 0; j < 6; ++j)
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      S a = S(0);
#pragma unroll
      for (int l = 0; l < 6; ++l) {
        if (JS(j, l) == 0) continue;
        a = JS(j, l) == 1 ? a + C_in[S6(l, k)] : kfma(J[j][l], C_in[S6(l, k)], a);
      }
      CJ[j][k] = a;  // (J C_in)_jk
    }
  S pin[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    S a = S(0);
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      if (JS(i, k) == 0) continue;
      a = JS(i, k) == 1 ? a + pbp[i] : kfma(J[i][k], pbp[i], a);
    }
    pin[k] = a;
  }
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int l = 0; l < 6; ++l) {
      if (JS(i, l) != 2) continue;
      // Jbar_il = 2 sum_j Cbp_ij (J C_in)_jl
      S jb = S(0);
#pragma unroll
      for (int j = 0; j < 6; ++j) jb = kfma(Cbp[i][j], CJ[j][l], jb);
      jb *= S(2);
#pragma unroll
      for (int d = 0; d < NDIR; ++d) pin[dir_param(d)] = kfma(jb, dJ[i][l][d], pin[dir_param(d)]);
    }
  // Cbar_in = J^T Cbar' J
  S T1[6][6];  // Cbp J
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      S a = S(0);
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        if (JS(j, k) == 0) continue;
        a = JS(j, k) == 1 ? a + Cbp[i][j] : kfma(Cbp[i][j], J[j][k], a);
      }
      T1[i][k] = a;
    }
#pragma unroll
  for (int k = 0; k < 6; ++k)
#pragma unroll
    for (int m = k; m < 6; ++m) {
      S a = S(0);
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        if (JS(i, k) == 0) continue;
        a = JS(i, k) == 1 ? a + T1[i][m] : kfma(J[i][k], T1[i][m], a);
      }
      Cb[k][m] = a;
      Cb[m][k] = a;
    }
#pragma unroll
  for (int i = 0; i < 6; ++i) pb[i] = pin[i];
}

// Whether step k of a track (from the state before it) crosses its layer
// close to tangentially; the careful pass runs such steps in double.
__device__ __forceinline__ bool near_tangent(const DevGeom& g, const float (&p)[6], float R) {
  float zc, cosa;
  if (!crossing(p, R, g.kb, zc, cosa)) return false;
  return cosa < ADJ_CAREFUL_COS;
}

// Forward step in precision S on float storage.
template <class S>
__device__ __noinline__ void fwd_step_store(const DevGeom& g, float* st, const Hit<S>& h, bool first, bool last) {
  S p[6], C[21];
  for (int q = 0; q < 6; ++q) p[q] = (S)st[q];
  for (int q = 0; q < 21; ++q) C[q] = (S)st[6 + q];
  fwd_step<S>(g, p, C, h, first, last);
  for (int q = 0; q < 6; ++q) st[27 + q] = (float)p[q];
  for (int q = 0; q < 21; ++q) st[27 + 6 + q] = (float)C[q];
}

// Reverse step in precision S with the adjoints kept in A (double in the
// careful pass, float otherwise).
template <class S, class A>
__device__ __noinline__ void rev_step_store(const DevGeom& g, const float* st, const Hit<S>& h, bool first,
                                            bool last, A (&pbA)[6], A (&CbA)[6][6], A (&hbA)[3], A (&abA)[2]) {
  S p[6], C[21], pb[6], Cb[6][6], hb[3], ab[2];
  for (int q = 0; q < 6; ++q) p[q] = (S)st[q];
  for (int q = 0; q < 21; ++q) C[q] = (S)st[6 + q];
  for (int i = 0; i < 6; ++i) {
    pb[i] = (S)pbA[i];
    for (int j = 0; j < 6; ++j) Cb[i][j] = (S)CbA[i][j];
  }
  rev_step<S>(g, p, C, h, first, last, pb, Cb, hb, ab);
  for (int i = 0; i < 6; ++i) {
    pbA[i] = (A)pb[i];
    for (int j = 0; j < 6; ++j) CbA[i][j] = (A)Cb[i][j];
  }
  for (int i = 0; i < 3; ++i) hbA[i] = (A)hb[i];
  for (int i = 0; i < 2; ++i) abA[i] = (A)ab[i];
}

// Reverse sweep of one fitted track from the fit's checkpoints.  CAREFUL:
// the track the fit flagged as near-tangent; its near-tangent steps run in
// double precision and its adjoints are kept in double.
template <bool CAREFUL>
__device__ void adjoint_track(const AdjParams& P, int t, double* sh_align) {
  using A = typename std::conditional<CAREFUL, double, float>::type;
  const DevGeom& g = P.g;
  if (!CAREFUL) {
    if ((P.keep && !P.keep[t]) || P.fit_status[t] != KF_FIT_OK) {
      if (P.g_seed)  // not fitted: no contribution
        for (int k = 0; k < 6; ++k) P.g_seed[(size_t)k * P.ns + t] = 0.f;
      return;
    }
    if (P.careful_flag[t]) return;  // left to the careful pass
  } else if (P.fit_status[t] != KF_FIT_OK) {
    if (P.g_seed)
      for (int k = 0; k < 6; ++k) P.g_seed[(size_t)k * P.ns + t] = 0.f;
    return;
  }
  const int n = P.n_list[t];
  const int* lst = P.lists + (size_t)t * P.max_len;
  const int hoff = P.hit_off[P.seed_event[t]];
  const int stride = P.stride;
  A pb[6], Cb[6][6];
  for (int i = 0; i < 6; ++i) {
    pb[i] = A(0);
    for (int j = 0; j < 6; ++j) Cb[i][j] = A(0);
  }
  float seg[(MAX_CKPT_STRIDE + 1) * 27];  // states before each step of a segment
  for (int c = (n - 1) / stride; c >= 0; --c) {
    const int k0 = c * stride, k1 = min(n, k0 + stride);
    const float* ck = P.ckpt + (size_t)c * 27 * P.ns + t;
    for (int q = 0; q < 27; ++q) seg[q] = ck[(size_t)q * P.ns];
    for (int k = k0; k + 1 < k1; ++k) {
      float* st = seg + (k - k0) * 27;
      const int hi = hoff + lst[k];
      if (CAREFUL && k > 0) {
        float pf[6];
        for (int q = 0; q < 6; ++q) pf[q] = st[q];
        if (near_tangent(g, pf, g.radius[P.hlayer[hi]])) {
          fwd_step_store<double>(g, st, load_hit<double>(P, hi), k == 0, k + 1 == n);
          continue;
        }
      }
      fwd_step_store<float>(g, st, load_hit<float>(P, hi), k == 0, k + 1 == n);
    }
    for (int k = k1 - 1; k >= k0; --k) {
      const float* st = seg + (k - k0) * 27;
      const int hl = lst[k];
      const int hi = hoff + hl;
      A hb[3], ab[2];
      bool dbl = false;
      if (CAREFUL && k > 0) {
        float pf[6];
        for (int q = 0; q < 6; ++q) pf[q] = st[q];
        dbl = near_tangent(g, pf, g.radius[P.hlayer[hi]]);
      }
      if (dbl) rev_step_store<double, A>(g, st, load_hit<double>(P, hi), k == 0, k + 1 == n, pb, Cb, hb, ab);
      else rev_step_store<float, A>(g, st, load_hit<float>(P, hi), k == 0, k + 1 == n, pb, Cb, hb, ab);
      if (P.g_hits) {
        float* gh = P.g_hits + 3 * (size_t)hi;
        atomicAdd(gh + 0, (float)hb[0]);
        atomicAdd(gh + 1, (float)hb[1]);
        atomicAdd(gh + 2, (float)hb[2]);
      }
      const int L = P.hlayer[hi];
      atomicAdd(sh_align + 2 * L, (double)ab[0]);
      atomicAdd(sh_align + 2 * L + 1, (double)ab[1]);
    }
  }
  if (P.g_seed) {
    for (int k = 0; k < 6; ++k) P.g_seed[(size_t)k * P.ns + t] = (float)pb[k];
  }
}

template <bool CAREFUL>
__global__ void __launch_bounds__(128) k_adjoint(const AdjParams P) {
  __shared__ double sh_align[2 * KF_MAX_LAYERS];
  for (int i = threadIdx.x; i < 2 * KF_MAX_LAYERS; i += blockDim.x) sh_align[i] = 0.0;
  __syncthreads();
  if (!CAREFUL) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < P.ns) adjoint_track<false>(P, t, sh_align);
  } else {
    const unsigned n = *P.careful_count;
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
      adjoint_track<true>(P, P.careful_list[i], sh_align);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 2 * P.g.n_layers; i += blockDim.x)
    if (sh_align[i] != 0.0) atomicAdd(P.g_align_acc + i, sh_align[i]);
}

__global__ void k_adjoint_finish(const AdjParams P) {
  const int i = threadIdx.x;
  if (i < 2 * P.g.n_layers) P.g_align[i] = (float)P.g_align_acc[i];
}

}  // namespace

bool adjoint_stride_ok(int stride, int max_len) {
  return stride >= 1 && stride <= MAX_CKPT_STRIDE && max_len <= MAX_CKPT * stride;
}

cudaError_t launch_adjoint(const AdjParams& P, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(P.g_align_acc, 0, sizeof(double) * 2 * KF_MAX_LAYERS, st);
  if (e == cudaSuccess && P.g_hits) e = cudaMemsetAsync(P.g_hits, 0, sizeof(float) * 3 * (size_t)P.n_hits, st);
  if (e != cudaSuccess) return e;
  const int threads = 128;
  if (P.ns > 0) {
    k_adjoint<false><<<(P.ns + threads - 1) / threads, threads, 0, st>>>(P);
    k_adjoint<true><<<(P.ns / 20 + threads - 1) / threads + 1, threads, 0, st>>>(P);
  }
  k_adjoint_finish<<<1, 2 * KF_MAX_LAYERS, 0, st>>>(P);
  return cudaGetLastError();
}

}  // namespace kfg
