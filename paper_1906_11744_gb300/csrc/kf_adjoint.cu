// Adjoint of the Kalman re-fit: d(sum of chi2)/d(layer alignment offsets, hit
// positions, seed parameters), one thread per track.
//
// Forward: the fit of kf_fit.cu (prior at the first hit; per hit: propagate,
// tangent-frame measurement, chi2, update, scattering except after the last)
// writes the state (p, C) before every `stride`-th hit as a checkpoint.
// Reverse: for each segment from the last, the states before each step are
// recomputed from the segment's checkpoint, then the steps are reversed one
// by one:
//   * scattering C += Q(p): the Highland variances differentiated by hand
//     through log(theta0) (q/pT, theta, and phi relative to the position angle);
//   * update and chi2 with U = C H^T, S = H U + V, K = U S^-1,
//       p' = p + U S^-1 r,  C' = C - U S^-1 U^T,  chi2 = r^T S^-1 r,
//     reversed with the matrix identities dS^-1 = -S^-1 dS S^-1 (adjoints of
//     U, S^-1, r, H and C by hand);
//   * the measurement frame H(p) and residual r(p, m), m = R(-a_rphi/R_L) h - a_z e_z;
//   * propagation q = F(p), C' = J C J^T: Cbar <- J^T Cbar' J,
//     pbar <- J^T pbar' + sum_ij Jbar_ij dJ_ij/dp with Jbar = 2 Cbar' J C; the
//     contraction is one reverse sweep through the Jacobian's intermediates,
//     with the path length's dependence on p from the implicit function
//     theorem (ds/dp = -(dg/dp)/(dg/ds) for g = x(s)^2 + y(s)^2 - R^2) and
//     d sinc/dpsi = f1, d cosc/dpsi = f2.
// The adjoint of the final state is zero: the objective is the chi2 sum.
// Alignment: the corrected position depends on the layer's offsets only, and
// a rotation keeps cross products, so the alignment gradient of layer L is
// the sum over its hits of (-(x g_y - y g_x)/R_L, -g_z), g the gradient with
// respect to the raw position (x, y, z) of the hit; each reverse step adds
// its hit's share to its layer's sums (per block in shared memory, then in
// double precision across blocks).
// The tracks of the fit's careful list (a crossing with cos(alpha) < 0.5, a
// plane step along more than half a radian, or a loose prior) are reversed
// by separate passes, which can run beside the FP32 pass after the fit's own
// careful pass: those with a crossing below cos(alpha) = 0.2 or such a plane
// step keep their adjoints in double and run those steps in double; the
// others run the FP32 code.  The rest are reversed in FP32 from the
// checkpoints.
#include <type_traits>

#include "kf_common.cuh"
#include "kf_internal.h"

namespace kfg {

// Forward-mode derivatives in six directions (the state's parameters): the
// value v and d[k] = dv/dp_k.  The reverse of the energy-loss step takes the
// derivatives of its Jacobian row through eloss_row on this scalar.
template <class S>
struct Dir6 {
  S v, d[6];
  __device__ Dir6() : v(S(0)) {
#pragma unroll
    for (int k = 0; k < 6; ++k) d[k] = S(0);
  }
  __device__ Dir6(S x) : v(x) {  // NOLINT implicit: a constant
#pragma unroll
    for (int k = 0; k < 6; ++k) d[k] = S(0);
  }
};
template <class S>
__device__ __forceinline__ Dir6<S> operator+(const Dir6<S>& a, const Dir6<S>& b) {
  Dir6<S> r(a.v + b.v);
#pragma unroll
  for (int k = 0; k < 6; ++k) r.d[k] = a.d[k] + b.d[k];
  return r;
}
template <class S>
__device__ __forceinline__ Dir6<S> operator-(const Dir6<S>& a, const Dir6<S>& b) {
  Dir6<S> r(a.v - b.v);
#pragma unroll
  for (int k = 0; k < 6; ++k) r.d[k] = a.d[k] - b.d[k];
  return r;
}
template <class S>
__device__ __forceinline__ Dir6<S> operator-(const Dir6<S>& a) {
  Dir6<S> r(-a.v);
#pragma unroll
  for (int k = 0; k < 6; ++k) r.d[k] = -a.d[k];
  return r;
}
template <class S>
__device__ __forceinline__ Dir6<S> operator*(const Dir6<S>& a, const Dir6<S>& b) {
  Dir6<S> r(a.v * b.v);
#pragma unroll
  for (int k = 0; k < 6; ++k) r.d[k] = kfma(a.d[k], b.v, a.v * b.d[k]);
  return r;
}
template <class S>
__device__ __forceinline__ Dir6<S> kfma(const Dir6<S>& a, const Dir6<S>& b, const Dir6<S>& c) {
  Dir6<S> r(kfma(a.v, b.v, c.v));
#pragma unroll
  for (int k = 0; k < 6; ++k) r.d[k] = kfma(a.d[k], b.v, kfma(a.v, b.d[k], c.d[k]));
  return r;
}
template <class S>
__device__ __forceinline__ Dir6<S> kdiv(const Dir6<S>& a, const Dir6<S>& b) {
  Dir6<S> r(kdiv(a.v, b.v));
  const S ib = kdiv(S(1), b.v);
#pragma unroll
  for (int k = 0; k < 6; ++k) r.d[k] = (a.d[k] - r.v * b.d[k]) * ib;
  return r;
}
template <class S>
__device__ __forceinline__ Dir6<S> ksqrt(const Dir6<S>& a) {
  Dir6<S> r(ksqrt(a.v));
  const S h = kdiv(S(0.5), r.v);
#pragma unroll
  for (int k = 0; k < 6; ++k) r.d[k] = a.d[k] * h;
  return r;
}
template <class S>
__device__ __forceinline__ Dir6<S> krsqrt(const Dir6<S>& a) {
  Dir6<S> r(krsqrt(a.v));
  const S h = S(-0.5) * r.v * r.v * r.v;
#pragma unroll
  for (int k = 0; k < 6; ++k) r.d[k] = a.d[k] * h;
  return r;
}
template <class S>
__device__ __forceinline__ Dir6<S> kabs(const Dir6<S>& a) { return a.v < S(0) ? -a : a; }
template <class S>
__device__ __forceinline__ void ksincos(const Dir6<S>& a, Dir6<S>* s, Dir6<S>* c) {
  S sv, cv;
  ksincos(a.v, &sv, &cv);
  s->v = sv;
  c->v = cv;
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    s->d[k] = cv * a.d[k];
    c->d[k] = -sv * a.d[k];
  }
}
template <class S>
__device__ __forceinline__ S kval(const Dir6<S>& a) { return a.v; }
template <class S>
__device__ __forceinline__ void ksincos_acc(const Dir6<S>& a, Dir6<S>* s, Dir6<S>* c) {
  S sv, cv;
  ksincos_acc(a.v, &sv, &cv);
  *s = Dir6<S>(sv);
  *c = Dir6<S>(cv);
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    s->d[k] = cv * a.d[k];
    c->d[k] = -sv * a.d[k];
  }
}


namespace {

constexpr float ADJ_CAREFUL_COS = ADJOINT_CAREFUL_COS;
// Threads per block of the adjoint kernels; also the row stride (in floats)
// of the segment buffer in shared memory.
constexpr int ADJ_THREADS = 128;
constexpr int LD = ADJ_THREADS;
static_assert((LD & (LD - 1)) == 0, "column rotation by a mask");

// Derivatives of f1 and f2 (the helix functions of kf_common.cuh) in psi:
// f1' = -(sin psi + 2 f1)/psi, f2' = (cos psi - 2 f2)/psi, by the term-wise
// derivatives of the same power series below |psi| = 0.5.
template <class T>
__device__ __forceinline__ void helix_dfns(T psi, T f1, T f2, T& df1, T& df2) {
  if (kabs(psi) < T(0.5)) {
    const T q = psi * psi;
    df1 = kfma(q, kfma(q, kfma(q, kfma(q, T(-1.0 / 443520.0), T(1.0 / 6480.0)), T(-1.0 / 168.0)), T(0.1)),
               T(-1.0 / 3.0));
    df2 = psi * kfma(q, kfma(q, kfma(q, T(1.0 / 50400.0), T(-1.0 / 960.0)), T(1.0 / 36.0)), T(-0.25));
    if (sizeof(T) == 8) {  // the extra term of the double series
      const T q4 = q * q * q * q;
      df1 += q4 * q * T(1.0 / 47174400.0);
      df2 += psi * q4 * T(-1.0 / 4354560.0);
    }
  } else {
    T sn, cs;
    ksincos(psi, &sn, &cs);
    const T ip = T(1) / psi;
    df1 = -(sn + T(2) * f1) * ip;
    df2 = (cs - T(2) * f2) * ip;
  }
}

// Sine and cosine of a + d from those of a (sa, ca), for the small change d
// that an update makes to an angle: sin d and cos d by their Taylor series
// (|d| <= 0.1: truncation below 1e-9), else from the angle a + d itself.
template <class T>
__device__ __forceinline__ void rotate_small(T sa, T ca, T d, T angle, T& so, T& co) {
  if (kabs(d) > T(0.1)) {
    ksincos_acc(angle, &so, &co);
    return;
  }
  const T d2 = d * d;
  const T sd = d * kfma(d2, kfma(d2, T(1.0 / 120.0), T(-1.0 / 6.0)), T(1));
  const T cd = kfma(d2, kfma(d2, kfma(d2, T(-1.0 / 720.0), T(1.0 / 24.0)), T(-0.5)), T(1));
  so = kfma(sa, cd, ca * sd);
  co = kfma(ca, cd, -(sa * sd));
}

// v += sum_il Jb_il dJ_il/dp for the propagation Jacobian J(p) of
// prop_jacobian (to the layer it crossed at transverse path length s).  Jb
// is read at the structural non-zeros (JS == 2) only.  Reverse sweep through
// the Jacobian's intermediates in the opposite order of their computation.
// trig: sin, cos of phi and of theta at the start (as prop_jacobian gives them).
template <class T>
__device__ __forceinline__ void jac_vjp(const T (&p)[6], T s, T kb, const T (&Jb)[6][6], T (&v)[6],
                                        const T* trig) {
  const T x = p[0], y = p[1], h = kb * p[3];
  const T sf = trig[0], cf = trig[1], sth = trig[2], cth = trig[3];
  const T ist = T(1) / sth;
  const T cot = cth * ist;
  const T psi = h * s;
  T sc, cc, f1, f2, df1, df2;
  helix_fns<T>(psi, sc, cc, f1, f2);
  helix_dfns<T>(psi, f1, f2, df1, df2);
  const T Sx = s * sc, Cx = s * cc;
  const T dx = kfma(cf, Sx, -sf * Cx), dy = kfma(sf, Sx, cf * Cx);
  const T xn = x + dx, yn = y + dy;
  const T cpsi = kfma(-psi, cc, T(1)), spsi = psi * sc;
  const T cp = kfma(cf, cpsi, -sf * spsi), sp = kfma(sf, cpsi, cf * spsi);
  const T s2 = s * s, dSdh = s2 * f1, dCdh = s2 * f2;
  const T Fx3 = kb * kfma(cf, dSdh, -sf * dCdh), Fy3 = kb * kfma(sf, dSdh, cf * dCdh);
  const T Fx4 = -dy, Fy4 = dx;
  const T inv = T(-1) / kfma(xn, cp, yn * sp);
  const T g3 = kfma(xn, Fx3, yn * Fy3), g4 = kfma(xn, Fx4, yn * Fy4);
  const T ds[4] = {xn * inv, yn * inv, g3 * inv, g4 * inv};  // ds/d(x, y, q/pT, phi)
  // J rows 0, 1, 2, 4 over columns (x, y, q/pT, phi) are (cp, sp, cot, h) ds_c
  // plus terms free of ds; row 2 column theta is -s / sin^2 theta.
  T cpb = T(0), spb = T(0), cotb = T(0), hb = T(0), dsb[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int col = c < 2 ? c : c + 1;
    cpb = kfma(Jb[0][col], ds[c], cpb);
    spb = kfma(Jb[1][col], ds[c], spb);
    cotb = kfma(Jb[2][col], ds[c], cotb);
    hb = kfma(Jb[4][col], ds[c], hb);
    dsb[c] = kfma(Jb[0][col], cp, kfma(Jb[1][col], sp, kfma(Jb[2][col], cot, Jb[4][col] * h)));
  }
  T sb = kfma(Jb[4][3], kb, -Jb[2][5] * ist * ist);
  T sthb = T(2) * Jb[2][5] * s * ist * ist * ist;
  // ds_c = g_c inv with g = (xn, yn, g3, g4), inv = -1/(xn cp + yn sp)
  const T invb = kfma(dsb[0], xn, kfma(dsb[1], yn, kfma(dsb[2], g3, dsb[3] * g4)));
  T xnb = kfma(dsb[2], Fx3, kfma(dsb[3], Fx4, dsb[0])) * inv;
  T ynb = kfma(dsb[2], Fy3, kfma(dsb[3], Fy4, dsb[1])) * inv;
  const T Fx3b = kfma(dsb[2] * xn, inv, Jb[0][3]), Fy3b = kfma(dsb[2] * yn, inv, Jb[1][3]);
  const T Fx4b = kfma(dsb[3] * xn, inv, Jb[0][4]), Fy4b = kfma(dsb[3] * yn, inv, Jb[1][4]);
  const T dgdsb = invb * inv * inv;
  xnb = kfma(dgdsb, cp, xnb);
  ynb = kfma(dgdsb, sp, ynb);
  cpb = kfma(dgdsb, xn, cpb);
  spb = kfma(dgdsb, yn, spb);
  // F4 = (-dy, dx); F3 = kb R(phi) (dS/dh, dC/dh)
  T dxb = Fy4b + xnb, dyb = ynb - Fx4b;
  const T dSdhb = kb * kfma(Fx3b, cf, Fy3b * sf), dCdhb = kb * kfma(-Fx3b, sf, Fy3b * cf);
  T cfb = kb * kfma(Fx3b, dSdh, Fy3b * dCdh), sfb = kb * kfma(-Fx3b, dCdh, Fy3b * dSdh);
  sb = kfma(T(2) * s, kfma(dSdhb, f1, dCdhb * f2), sb);
  const T f1b = dSdhb * s2, f2b = dCdhb * s2;
  // (cp, sp) = R(phi) (cos psi, sin psi)
  cfb = kfma(cpb, cpsi, kfma(spb, spsi, cfb));
  sfb = kfma(-cpb, spsi, kfma(spb, cpsi, sfb));
  const T cpsib = kfma(cpb, cf, spb * sf), spsib = kfma(-cpb, sf, spb * cf);
  T psib = kfma(-cpsib, cc, spsib * sc);
  T ccb = -cpsib * psi, scb = spsib * psi;
  // (dx, dy) = R(phi) (S, C) with S = s sinc, C = s cosc
  cfb = kfma(dxb, Sx, kfma(dyb, Cx, cfb));
  sfb = kfma(-dxb, Cx, kfma(dyb, Sx, sfb));
  const T Sxb = kfma(dxb, cf, dyb * sf), Cxb = kfma(-dxb, sf, dyb * cf);
  sb = kfma(Sxb, sc, kfma(Cxb, cc, sb));
  scb = kfma(Sxb, s, scb);
  ccb = kfma(Cxb, s, ccb);
  psib = kfma(scb, f1, kfma(ccb, f2, kfma(f1b, df1, kfma(f2b, df2, psib))));
  hb = kfma(psib, s, hb);
  sb = kfma(psib, h, sb);
  // cot = cos theta / sin theta
  sthb = kfma(-cotb * cot, ist, sthb);
  v[0] += kfma(sb, ds[0], xnb);
  v[1] += kfma(sb, ds[1], ynb);
  v[3] += kfma(kb, hb, sb * ds[2]);
  v[4] += kfma(sfb, cf, kfma(-cfb, sf, sb * ds[3]));
  v[5] += kfma(sthb, cth, -cotb);
}

// v += b44 dq44/dp + b55 dq55/dp for the scattering variances of add_ms:
// with L = log theta0, dL = (beta^2 - 2)(d|q/pT|/|q/pT| + dsin/sin)
//   + (1/2 + 0.038/(1 + 0.038 log t)) dlog t,  t = x0/|sin theta cos(phi - phi_p)|,
// phi_p the position angle; dq55 = 2 q55 dL, dq44 = q44 (2 dL - 2 dsin/sin).
// The thickness x0 may depend on z (material map): dlog t gains
// (dx0/dz)/x0 dz.
// sth, cth, sph, cph: sin, cos of theta and phi of p.
template <class T>
__device__ __forceinline__ void ms_vjp(const T (&p)[6], T x0, T dx0dz, T b44, T b55, T (&v)[6], T sth, T cth,
                                       T sph, T cph) {
  if (p[3] == T(0) || x0 <= T(0)) return;
  const T ir = krsqrt(kfma(p[0], p[0], p[1] * p[1]));
  const T cdiff = kfma(cph, p[0], sph * p[1]) * ir;   // cos(phi - phi_p)
  const T sdiff = kfma(sph, p[0], -cph * p[1]) * ir;  // sin(phi - phi_p)
  const T pm = T(1) / (kabs(p[3]) * sth);
  const T e2 = kfma(pm, pm, T(MPION * MPION));
  const T beta = pm / ksqrt(e2);
  const T t = x0 / kabs(sth * cdiff);
  const T lt = klog(t);
  const T th0 = T(0.0136) / (beta * pm) * ksqrt(t) * kfma(T(0.038), lt, T(1));
  const T q55 = th0 * th0;
  const T q44 = q55 / (sth * sth);
  const T W = T(2) * kfma(b55, q55, b44 * q44);
  const T a = pm * pm / e2 - T(2);
  const T bt = T(0.5) + T(0.038) / kfma(T(0.038), lt, T(1));
  v[3] += -W * a / p[3];
  v[5] += kfma(-W, a + bt, T(-2) * b44 * q44) * cth / sth;
  const T wc = W * bt * sdiff / cdiff;  // adjoint of phi - phi_p
  v[4] += wc;
  v[0] = kfma(wc * p[1], ir * ir, v[0]);
  v[1] = kfma(-wc * p[0], ir * ir, v[1]);
  // a material map: the thickness depends on z, d(log t)/dz = (dx0/dz)/x0
  v[2] = kfma(W * bt, dx0dz / x0, v[2]);
}

// v += sum_il Jb_il dJ_il/dp for the Jacobian of the plane step
// (prop_plane_jacobian, to z = zd): rows x, y, phi over columns z and theta
// are (cos phi', sin phi', h) (ds/dz, ds/dtheta) with ds/dz = -tan(theta),
// ds/dtheta = s/(sin theta cos theta); column q/pT is kb R(phi) (dS/dh,
// dC/dh) and kb s; column phi is (-dy, dx).  s = (zd - z) tan(theta) depends
// on z and theta only.  Reverse sweep in the opposite order of the forward
// computation.
template <class T>
__device__ __forceinline__ void jac_vjp_plane(const T (&p)[6], T zd, T kb, const T (&Jb)[6][6], T (&v)[6]) {
  T sf, cf, sth, cth;
  ksincos_acc(p[4], &sf, &cf);
  ksincos_polar(p[5], &sth, &cth);
  const T tn = sth / cth;
  const T dzp = zd - p[2];
  const T s = dzp * tn;
  const T h = kb * p[3];
  const T psi = h * s;
  T sc, cc, f1, f2, df1, df2;
  helix_fns<T>(psi, sc, cc, f1, f2);
  helix_dfns<T>(psi, f1, f2, df1, df2);
  const T Sx = s * sc, Cx = s * cc;
  const T cpsi = kfma(-psi, cc, T(1)), spsi = psi * sc;
  const T cp = kfma(cf, cpsi, -sf * spsi), sp = kfma(sf, cpsi, cf * spsi);
  const T s2 = s * s, dSdh = s2 * f1, dCdh = s2 * f2;
  const T isc = T(1) / (sth * cth);
  const T ds2 = -tn, ds5 = s * isc;
  T cpb = kfma(Jb[0][2], ds2, Jb[0][5] * ds5);
  T spb = kfma(Jb[1][2], ds2, Jb[1][5] * ds5);
  T hb = kfma(Jb[4][2], ds2, Jb[4][5] * ds5);
  const T ds2b = kfma(Jb[0][2], cp, kfma(Jb[1][2], sp, Jb[4][2] * h));
  const T ds5b = kfma(Jb[0][5], cp, kfma(Jb[1][5], sp, Jb[4][5] * h));
  const T dSdhb = kb * kfma(Jb[0][3], cf, Jb[1][3] * sf);
  const T dCdhb = kb * kfma(-Jb[0][3], sf, Jb[1][3] * cf);
  T cfb = kb * kfma(Jb[0][3], dSdh, Jb[1][3] * dCdh);
  T sfb = kb * kfma(-Jb[0][3], dCdh, Jb[1][3] * dSdh);
  T sb = Jb[4][3] * kb;
  const T dxb = Jb[1][4], dyb = -Jb[0][4];
  // ds5 = s / (sin cos), ds2 = -sin / cos
  sb = kfma(ds5b, isc, sb);
  T sthb = -(ds5b * ds5 / sth) - ds2b / cth;
  T cthb = -(ds5b * ds5 / cth) + ds2b * tn / cth;
  // dS/dh = s^2 f1, dC/dh = s^2 f2
  sb = kfma(T(2) * s, kfma(dSdhb, f1, dCdhb * f2), sb);
  const T f1b = dSdhb * s2, f2b = dCdhb * s2;
  // (cp, sp) = R(phi) (cos psi, sin psi)
  cfb = kfma(cpb, cpsi, kfma(spb, spsi, cfb));
  sfb = kfma(-cpb, spsi, kfma(spb, cpsi, sfb));
  const T cpsib = kfma(cpb, cf, spb * sf), spsib = kfma(-cpb, sf, spb * cf);
  T psib = kfma(-cpsib, cc, spsib * sc);
  T ccb = -cpsib * psi, scb = spsib * psi;
  // (dx, dy) = R(phi) (S, C) with S = s sinc, C = s cosc
  cfb = kfma(dxb, Sx, kfma(dyb, Cx, cfb));
  sfb = kfma(-dxb, Cx, kfma(dyb, Sx, sfb));
  const T Sxb = kfma(dxb, cf, dyb * sf), Cxb = kfma(-dxb, sf, dyb * cf);
  sb = kfma(Sxb, sc, kfma(Cxb, cc, sb));
  scb = kfma(Sxb, s, scb);
  ccb = kfma(Cxb, s, ccb);
  psib = kfma(scb, f1, kfma(ccb, f2, kfma(f1b, df1, kfma(f2b, df2, psib))));
  hb = kfma(psib, s, hb);
  sb = kfma(psib, h, sb);
  // s = (zd - z) tan(theta), tan = sin / cos
  const T tnb = sb * dzp;
  sthb = kfma(tnb, T(1) / cth, sthb);
  cthb = kfma(-tnb, tn / cth, cthb);
  v[2] -= sb * tn;
  v[3] = kfma(kb, hb, v[3]);
  v[4] += kfma(sfb, cf, -cfb * sf);
  v[5] += kfma(sthb, cth, -cthb * sth);
}

// v += b44 dq44/dp + b55 dq55/dp for the scattering of a disk (add_ms_disk):
// as ms_vjp with t = x0/|cos(theta)|, so that d log t = tan(theta) dtheta and
// the variances depend on q/pT and theta only.
template <class T>
__device__ __forceinline__ void ms_vjp_disk(const T (&p)[6], T x0, T b44, T b55, T (&v)[6]) {
  if (p[3] == T(0) || x0 <= T(0)) return;
  T sth, cth;
  ksincos_polar(p[5], &sth, &cth);
  const T pm = T(1) / (kabs(p[3]) * sth);
  const T e2 = kfma(pm, pm, T(MPION * MPION));
  const T beta = pm / ksqrt(e2);
  const T t = x0 / kabs(cth);
  const T lt = klog(t);
  const T th0 = T(0.0136) / (beta * pm) * ksqrt(t) * kfma(T(0.038), lt, T(1));
  const T q55 = th0 * th0;
  const T q44 = q55 / (sth * sth);
  const T W = T(2) * kfma(b55, q55, b44 * q44);
  const T a = pm * pm / e2 - T(2);
  const T bt = T(0.5) + T(0.038) / kfma(T(0.038), lt, T(1));
  const T cot = cth / sth;
  v[3] += -W * a / p[3];
  v[5] += kfma(W, kfma(bt, sth / cth, -a * cot), T(-2) * b44 * q44 * cot);
}

// Reverse of add_eloss, out of line and through a record in local memory, so
// that the reverse step keeps its registers for the path without loss.  In:
// the step's prediction (p = the updated state, Cp the predicted covariance,
// U = Cp H^T, S^-1), the layer's thickness x0 and loss e, and the adjoints pb,
// Cb (upper triangle) of the state after the loss.  The state the loss acted
// on is the update's covariance plus the scattering; with F the identity but
// for row 3 = u(p) (eloss_row) and L = pb . p' + <Cb, F C F^T>:
//   Cbar = F^T Cb F;
//   pbar_k = pb_k (k != 3) + pb_3 u_k + sum_j ubar_j du_j/dp_k,
//   ubar_j = 2 sum_(b != 3) Cb_3b C_jb + 2 Cb_33 (C u)_j,
// du/dp in forward mode (Dir6).  pb, Cb are replaced by the adjoints before
// the loss.
template <class S>
struct ElossRev {
  S p[6], Cp[21], U[6][2], si00, si01, si11, x0, e;
  S pb[6], Cb[21];
};
template <class S, bool DISK = false>
__device__ __noinline__ void eloss_vjp(ElossRev<S>* io) {
  S C[21];
  for (int i = 0; i < 6; ++i) {
    const S k0 = kfma(io->U[i][0], io->si00, io->U[i][1] * io->si01);
    const S k1 = kfma(io->U[i][0], io->si01, io->U[i][1] * io->si11);
    for (int j = i; j < 6; ++j) C[S6(i, j)] = io->Cp[S6(i, j)] - kfma(k0, io->U[j][0], k1 * io->U[j][1]);
  }
  S p[6];
  for (int k = 0; k < 6; ++k) p[k] = io->p[k];
  if (DISK) add_ms_disk<S>(p, C, io->x0);
  else add_ms<S, true>(p, C, io->x0);
  Dir6<S> pd[6];
  for (int k = 0; k < 6; ++k) {
    pd[k] = Dir6<S>(p[k]);
    pd[k].d[k] = S(1);
  }
  Dir6<S> k1, u[6];
  eloss_row<Dir6<S>, DISK, true>(pd, Dir6<S>(io->e), k1, u);
  S uv[6], Cu[6], ub[6], pn[6];
  for (int j = 0; j < 6; ++j) uv[j] = u[j].v;
  for (int j = 0; j < 6; ++j) {
    S a = S(0);
    for (int b = 0; b < 6; ++b) a = kfma(C[S6(j, b)], uv[b], a);
    Cu[j] = a;
  }
  for (int j = 0; j < 6; ++j) {
    S a = io->Cb[S6(3, 3)] * Cu[j];
    for (int b = 0; b < 6; ++b)
      if (b != 3) a = kfma(io->Cb[S6(3, b)], C[S6(j, b)], a);
    ub[j] = S(2) * a;
  }
  for (int k = 0; k < 6; ++k) {
    S a = kfma(io->pb[3], uv[k], k == 3 ? S(0) : io->pb[k]);
    for (int j = 0; j < 6; ++j) a = kfma(ub[j], u[j].d[k], a);
    pn[k] = a;
  }
  // Cbar = F^T Cb F: X = Cb F (column k: Cb_:k for k != 3, plus Cb_:3 u_k),
  // then F^T X (row k: X_k: for k != 3, plus u_k X_3:)
  S X[6][6];
  for (int i = 0; i < 6; ++i)
    for (int k = 0; k < 6; ++k) X[i][k] = kfma(io->Cb[S6(i, 3)], uv[k], k == 3 ? S(0) : io->Cb[S6(i, k)]);
  for (int k = 0; k < 6; ++k)
    for (int m = k; m < 6; ++m) io->Cb[S6(k, m)] = kfma(uv[k], X[3][m], k == 3 ? S(0) : X[k][m]);
  for (int k = 0; k < 6; ++k) io->pb[k] = pn[k];
}

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
  if (is_disk(P.g, h.L)) {  // an endcap disk: the raw position, no alignment
    h.ca = S(1);
    h.sa = S(0);
    h.R = S(0);
    h.mx = (S)P.hx[hi];
    h.my = (S)P.hy[hi];
    h.mz = (S)P.hz[hi];
    return h;
  }
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
// EL: the detector has energy loss (kernels without it carry none of its code).
template <class S, bool EL, bool DISK = false>
__device__ __forceinline__ int fwd_step(const DevGeom& g, S (&p)[6], S (&C)[21], const Hit<S>& h, bool first,
                                        bool last) {
  if (DISK && is_disk(g, h.L)) {  // the plane step and the (r-phi, r) measurement
    if (!first && !propagate_plane<S, true>(p, C, (S)plane_z(g, h.L), field_kb<S>(g, p))) return KF_FIT_NO_CROSS;
    DiskFrameT<S> d;
    make_frame_disk<S>(p, C, (S)g.vr, (S)g.vrr, d);
    S r0, r1;
    if (!residual_disk<S>(p, d.f, h.mx, h.my, r0, r1)) return KF_FIT_FAR_SIDE;
    kf_update_disk<S>(p, C, d, r0, r1);
    if (!last) {
      add_ms_disk<S>(p, C, (S)g.disk_x0);
      if constexpr (EL) add_eloss_ool<S, true, true>(p, C, (S)g.disk_eloss);
    }
    return KF_FIT_OK;
  }
  if (!first) {
    S cosa = S(1);
    if (propagate<S, true>(p, C, h.R, field_kb<S>(g, p), S(INFINITY), &cosa) != 1) return KF_FIT_NO_CROSS;
    if (sizeof(S) == 4 && cosa < S(ADJ_CAREFUL_COS)) return 99;
  }
  FrameT<S> f;
  make_frame<S>(p, C, (S)g.vr, (S)g.vz, f);
  S r0, r1;
  if (!residual<S>(p, f, h.mx, h.my, h.mz, r0, r1)) return KF_FIT_FAR_SIDE;
  kf_update<S>(p, C, f, r0, r1);
  if (!last) {
    add_ms<S, true>(p, C, x0_at<S>(g, h.L, p[2]));
    if constexpr (EL) add_eloss_ool<S, false, true>(p, C, (S)g.eloss[h.L]);
  }
  return KF_FIT_OK;
}

// Reverse of one step onto an endcap disk (as rev_step below, out of line):
// the plane step (jac_vjp_plane), the measurement H = ((-su, cu, 0..), (cu,
// su, 0..)) whose rows and residual r = H (m - q) turn with the position
// angle phi_p of the prediction (dH0/dphi_p = -H1, dH1/dphi_p = H0, dr0/dphi_p
// = -r1, dr1/dphi_p = r0, dphi_p = (x dy - y dx)/rho^2), the disk's
// scattering and energy loss.  The hit gradient is with respect to its raw
// position (disks carry no alignment); its z component is zero.
template <class S, bool EL>
__device__ __forceinline__ void rev_step_disk(const DevGeom& g, const S (&p_in)[6], const S (&C_in)[21],
                                              const Hit<S>& h, bool first, bool last, S (&pb)[6], S (&Cb)[6][6],
                                              S (&hb)[3]) {
  // ---- forward recompute of the step
  S q[6], J[6][6], Cp[21];
  const S kb = field_kb<S>(g, p_in);
  const S zd = (S)plane_z(g, h.L);
  for (int k = 0; k < 21; ++k) Cp[k] = C_in[k];
  if (!first) {
    prop_plane_jacobian<S, true>(p_in, zd, kb, q, J);
    transport_plane<S>(J, Cp);
  } else {
    for (int k = 0; k < 6; ++k) q[k] = p_in[k];
  }
  const S rho2 = kfma(q[0], q[0], q[1] * q[1]);
  const S irho = krsqrt(rho2);
  const S cu = q[0] * irho, su = q[1] * irho;
  S U[6][2];
  for (int i = 0; i < 6; ++i) {
    U[i][0] = kfma(-su, Cp[S6(i, 0)], cu * Cp[S6(i, 1)]);
    U[i][1] = kfma(cu, Cp[S6(i, 0)], su * Cp[S6(i, 1)]);
  }
  const S s00 = kfma(-su, U[0][0], kfma(cu, U[1][0], (S)g.vr));
  const S s01 = kfma(-su, U[0][1], cu * U[1][1]);
  const S s11 = kfma(cu, U[0][1], kfma(su, U[1][1], (S)g.vrr));
  const S idet = S(1) / kfma(s00, s11, -s01 * s01);
  const S si00 = s11 * idet, si01 = -s01 * idet, si11 = s00 * idet;
  const S dx = h.mx - q[0], dy = h.my - q[1];
  const S r0 = kfma(-su, dx, cu * dy);
  const S r1 = kfma(cu, dx, su * dy);
  const S sir0 = kfma(si00, r0, si01 * r1), sir1 = kfma(si01, r0, si11 * r1);
  S pu[6];
  for (int i = 0; i < 6; ++i) pu[i] = q[i] + kfma(U[i][0], sir0, U[i][1] * sir1);

  // ---- reverse: energy loss and scattering
  S pbu[6];
  for (int i = 0; i < 6; ++i) pbu[i] = pb[i];
  if (!last) {
    const S e = (S)g.disk_eloss;
    if (EL && e > S(0) && pu[3] != S(0)) {
      ElossRev<S> io;
      for (int i = 0; i < 6; ++i) {
        io.p[i] = pu[i];
        io.pb[i] = pbu[i];
        io.U[i][0] = U[i][0];
        io.U[i][1] = U[i][1];
      }
      for (int k = 0; k < 21; ++k) io.Cp[k] = Cp[k];
      for (int i = 0; i < 6; ++i)
        for (int j = i; j < 6; ++j) io.Cb[S6(i, j)] = Cb[i][j];
      io.si00 = si00;
      io.si01 = si01;
      io.si11 = si11;
      io.x0 = (S)g.disk_x0;
      io.e = e;
      eloss_vjp<S, true>(&io);
      for (int i = 0; i < 6; ++i) pbu[i] = io.pb[i];
      for (int i = 0; i < 6; ++i)
        for (int j = i; j < 6; ++j) Cb[i][j] = Cb[j][i] = io.Cb[S6(i, j)];
    }
    ms_vjp_disk<S>(pu, (S)g.disk_x0, Cb[4][4], Cb[5][5], pbu);
  }
  // ---- reverse: update and chi2 (chi2 adjoint 1); the algebra of rev_step
  S w0 = S(0), w1 = S(0);
  for (int i = 0; i < 6; ++i) {
    w0 = kfma(U[i][0], pbu[i], w0);
    w1 = kfma(U[i][1], pbu[i], w1);
  }
  const S rb0 = kfma(si00, w0, si01 * w1) + S(2) * sir0;
  const S rb1 = kfma(si01, w0, si11 * w1) + S(2) * sir1;
  S CbU[6][2];
  for (int i = 0; i < 6; ++i) {
    S a0 = S(0), a1 = S(0);
    for (int j = 0; j < 6; ++j) {
      a0 = kfma(Cb[i][j], U[j][0], a0);
      a1 = kfma(Cb[i][j], U[j][1], a1);
    }
    CbU[i][0] = a0;
    CbU[i][1] = a1;
  }
  S UCU00 = S(0), UCU01 = S(0), UCU10 = S(0), UCU11 = S(0);
  for (int i = 0; i < 6; ++i) {
    UCU00 = kfma(U[i][0], CbU[i][0], UCU00);
    UCU01 = kfma(U[i][0], CbU[i][1], UCU01);
    UCU10 = kfma(U[i][1], CbU[i][0], UCU10);
    UCU11 = kfma(U[i][1], CbU[i][1], UCU11);
  }
  const S Sib00 = w0 * r0 - UCU00 + r0 * r0, Sib01 = w0 * r1 - UCU01 + r0 * r1;
  const S Sib10 = w1 * r0 - UCU10 + r1 * r0, Sib11 = w1 * r1 - UCU11 + r1 * r1;
  const S t00 = kfma(si00, Sib00, si01 * Sib10), t01 = kfma(si00, Sib01, si01 * Sib11);
  const S t10 = kfma(si01, Sib00, si11 * Sib10), t11 = kfma(si01, Sib01, si11 * Sib11);
  const S Sb00 = -kfma(t00, si00, t01 * si01), Sb01 = -kfma(t00, si01, t01 * si11);
  const S Sb10 = -kfma(t10, si00, t11 * si01), Sb11 = -kfma(t10, si01, t11 * si11);
  S Ub[6][2];
  for (int i = 0; i < 6; ++i) {
    Ub[i][0] = pbu[i] * sir0 - S(2) * kfma(CbU[i][0], si00, CbU[i][1] * si01);
    Ub[i][1] = pbu[i] * sir1 - S(2) * kfma(CbU[i][0], si01, CbU[i][1] * si11);
  }
  // + H^T Sbar (H rows (-su, cu) and (cu, su) on x, y)
  Ub[0][0] += kfma(-su, Sb00, cu * Sb10);
  Ub[0][1] += kfma(-su, Sb01, cu * Sb11);
  Ub[1][0] += kfma(cu, Sb00, su * Sb10);
  Ub[1][1] += kfma(cu, Sb01, su * Sb11);
  // Hbar (columns x, y) = Sbar U^T + Ubar^T C_pred
  S Hb00 = kfma(Sb00, U[0][0], Sb01 * U[0][1]);
  S Hb01 = kfma(Sb00, U[1][0], Sb01 * U[1][1]);
  S Hb10 = kfma(Sb10, U[0][0], Sb11 * U[0][1]);
  S Hb11 = kfma(Sb10, U[1][0], Sb11 * U[1][1]);
  for (int i = 0; i < 6; ++i) {
    Hb00 = kfma(Ub[i][0], Cp[S6(i, 0)], Hb00);
    Hb01 = kfma(Ub[i][0], Cp[S6(i, 1)], Hb01);
    Hb10 = kfma(Ub[i][1], Cp[S6(i, 0)], Hb10);
    Hb11 = kfma(Ub[i][1], Cp[S6(i, 1)], Hb11);
  }
  // Cbar_pred = Cb + sym(Ubar H)
  S Cbp[6][6];
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) Cbp[i][j] = Cb[i][j];
  for (int i = 0; i < 6; ++i) {
    const S v0 = S(0.5) * kfma(-su, Ub[i][0], cu * Ub[i][1]);
    const S v1 = S(0.5) * kfma(cu, Ub[i][0], su * Ub[i][1]);
    Cbp[i][0] += v0; Cbp[0][i] += v0;
    Cbp[i][1] += v1; Cbp[1][i] += v1;
  }
  // pbar of the prediction: pass-through, the residual's direct terms, and
  // the position angle through the residual and the rows of H
  S pbp[6];
  for (int i = 0; i < 6; ++i) pbp[i] = pbu[i];
  const S phib = kfma(-rb0, r1, rb1 * r0) + kfma(-Hb00, cu, -Hb01 * su) + kfma(-Hb10, su, Hb11 * cu);
  const S irho2 = irho * irho;
  pbp[0] += kfma(su, rb0, -cu * rb1) - phib * q[1] * irho2;
  pbp[1] += kfma(-cu, rb0, -su * rb1) + phib * q[0] * irho2;
  hb[0] = kfma(-su, rb0, cu * rb1);
  hb[1] = kfma(cu, rb0, su * rb1);
  hb[2] = S(0);
  // ---- reverse: the plane step
  if (first) {
    for (int i = 0; i < 6; ++i) pb[i] = pbp[i];
    return;
  }
  S CJ[6][6];  // (J C_in)_jk
  for (int j = 0; j < 6; ++j)
    for (int k = 0; k < 6; ++k) {
      S a = S(0);
      for (int l = 0; l < 6; ++l) {
        if (JSP(j, l) == 0) continue;
        a = JSP(j, l) == 1 ? a + C_in[S6(l, k)] : kfma(J[j][l], C_in[S6(l, k)], a);
      }
      CJ[j][k] = a;
    }
  S pin[6];
  for (int k = 0; k < 6; ++k) {
    S a = S(0);
    for (int i = 0; i < 6; ++i) {
      if (JSP(i, k) == 0) continue;
      a = JSP(i, k) == 1 ? a + pbp[i] : kfma(J[i][k], pbp[i], a);
    }
    pin[k] = a;
  }
  S Jb[6][6];
  for (int i = 0; i < 6; ++i)
    for (int l = 0; l < 6; ++l) {
      Jb[i][l] = S(0);
      if (JSP(i, l) != 2) continue;
      S jb = S(0);
      for (int j = 0; j < 6; ++j) jb = kfma(Cbp[i][j], CJ[j][l], jb);
      Jb[i][l] = S(2) * jb;
    }
  jac_vjp_plane<S>(p_in, zd, kb, Jb, pin);
  if (g.fcz != 0.f || g.fcr != 0.f) {  // the field moves with the starting point (as in rev_step)
    S jj = S(0);
    for (int i = 0; i < 6; ++i)
      if (JSP(i, 3) == 2) jj = kfma(Jb[i][3], J[i][3], jj);
    const S kbar = kdiv(kfma(p_in[3], pin[3] - pbp[3], jj), kb) * S(2) * (S)g.kb;
    pin[0] = kfma(kbar * (S)g.fcr, p_in[0], pin[0]);
    pin[1] = kfma(kbar * (S)g.fcr, p_in[1], pin[1]);
    pin[2] = kfma(kbar * (S)g.fcz, p_in[2], pin[2]);
  }
  // Cbar_in = J^T Cbar' J
  S T1[6][6];
  for (int i = 0; i < 6; ++i)
    for (int k = 0; k < 6; ++k) {
      S a = S(0);
      for (int j = 0; j < 6; ++j) {
        if (JSP(j, k) == 0) continue;
        a = JSP(j, k) == 1 ? a + Cbp[i][j] : kfma(Cbp[i][j], J[j][k], a);
      }
      T1[i][k] = a;
    }
  for (int k = 0; k < 6; ++k)
    for (int m = k; m < 6; ++m) {
      S a = S(0);
      for (int i = 0; i < 6; ++i) {
        if (JSP(i, k) == 0) continue;
        a = JSP(i, k) == 1 ? a + T1[i][m] : kfma(J[i][k], T1[i][m], a);
      }
      Cb[k][m] = a;
      Cb[m][k] = a;
    }
  for (int i = 0; i < 6; ++i) pb[i] = pin[i];
}

// The disk step's reverse out of line, through a record in local memory, so
// that the caller's adjoints stay in registers on its barrel steps.
template <class S>
struct DiskRev {
  S p[6], C[21], pb[6], Cb[6][6], hb[3];
  Hit<S> h;
};
template <class S, bool EL>
__device__ __noinline__ void rev_step_disk_rec(const DevGeom& g, DiskRev<S>* r, bool first, bool last) {
  rev_step_disk<S, EL>(g, r->p, r->C, r->h, first, last, r->pb, r->Cb, r->hb);
}

// Reverse of one step.  In: the state before the step (p_in, C_in), the
// adjoints of the state after it (pb, Cb: Cb a full symmetric 6x6).  Out: pb,
// Cb replaced by the adjoints of the state before it; the gradient of this
// step with respect to the raw hit position in hb[3].  DISK: the detector has
// endcap disks (a disk hit's step goes to rev_step_disk).
template <class S, bool EL, bool DISK = false>
__device__ __forceinline__ void rev_step(const DevGeom& g, const S (&p_in)[6], const S (&C_in)[21],
                                         const Hit<S>& h, bool first, bool last, S (&pb)[6], S (&Cb)[6][6],
                                         S (&hb)[3]) {
  if (DISK && is_disk(g, h.L)) {
    DiskRev<S> r;
#pragma unroll
    for (int k = 0; k < 6; ++k) r.p[k] = p_in[k];
#pragma unroll
    for (int k = 0; k < 21; ++k) r.C[k] = C_in[k];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      r.pb[i] = pb[i];
#pragma unroll
      for (int j = 0; j < 6; ++j) r.Cb[i][j] = Cb[i][j];
    }
    r.h = h;
    rev_step_disk_rec<S, EL>(g, &r, first, last);
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      pb[i] = r.pb[i];
#pragma unroll
      for (int j = 0; j < 6; ++j) Cb[i][j] = r.Cb[i][j];
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) hb[i] = r.hb[i];
    return;
  }
  // ---- forward recompute of the step
  S q[6], J[6][6], Cp[21], s_len = S(0);
  S trig[6];  // sin, cos of phi and theta at the start, of phi after the propagation
  const S kb = field_kb<S>(g, p_in);  // the field at the step's starting point
#pragma unroll
  for (int k = 0; k < 21; ++k) Cp[k] = C_in[k];
  if (!first) {
    prop_jacobian<S, true>(p_in, h.R, kb, S(INFINITY), q, J, nullptr, &s_len, trig);
    transport<S>(J, Cp);
  } else {
#pragma unroll
    for (int k = 0; k < 6; ++k) q[k] = p_in[k];
    ksincos_acc(p_in[4], &trig[4], &trig[5]);
    ksincos_acc(p_in[5], &trig[2], &trig[3]);
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

  // ---- reverse: energy loss and scattering, C_out = F (C_upd + Q(p_upd)) F^T
  S pbu[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) pbu[i] = pb[i];
  if (!last) {
    const S e = (S)g.eloss[h.L];
    if (EL && e > S(0) && pu[3] != S(0)) {
      ElossRev<S> io;
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        io.p[i] = pu[i];
        io.pb[i] = pbu[i];
        io.U[i][0] = U[i][0];
        io.U[i][1] = U[i][1];
      }
#pragma unroll
      for (int k = 0; k < 21; ++k) io.Cp[k] = Cp[k];
#pragma unroll
      for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int j = i; j < 6; ++j) io.Cb[S6(i, j)] = Cb[i][j];
      io.si00 = si00;
      io.si01 = si01;
      io.si11 = si11;
      io.x0 = x0_at<S>(g, h.L, pu[2]);
      io.e = e;
      eloss_vjp<S>(&io);
#pragma unroll
      for (int i = 0; i < 6; ++i) pbu[i] = io.pb[i];
#pragma unroll
      for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int j = i; j < 6; ++j) Cb[i][j] = Cb[j][i] = io.Cb[S6(i, j)];
    }
    S dx0dz;
    const S x0 = x0_at<S>(g, h.L, pu[2], &dx0dz);
    // the angles after the update, from those of the prediction
    S sph, cph, sth, cth;
    rotate_small<S>(trig[4], trig[5], pu[4] - q[4], pu[4], sph, cph);
    rotate_small<S>(trig[2], trig[3], pu[5] - q[5], pu[5], sth, cth);
    ms_vjp<S>(pu, x0, dx0dz, Cb[4][4], Cb[5][5], pbu, sth, cth, sph, cph);
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
  // hit: mbar = (-su, cu) rb0 + e_z rb1, rotated back to the raw position
  const S mbx = -su * rb0, mby = cu * rb0;
  hb[0] = kfma(h.ca, mbx, h.sa * mby);
  hb[1] = kfma(-h.sa, mbx, h.ca * mby);
  hb[2] = rb1;
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
  S Jb[6][6];  // Jbar_il = 2 sum_j Cbp_ij (J C_in)_jl at the structural non-zeros
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int l = 0; l < 6; ++l) {
      if (JS(i, l) != 2) continue;
      S jb = S(0);
#pragma unroll
      for (int j = 0; j < 6; ++j) jb = kfma(Cbp[i][j], CJ[j][l], jb);
      Jb[i][l] = S(2) * jb;
    }
  jac_vjp<S>(p_in, s_len, kb, Jb, pin, trig);
  if (g.fcz != 0.f || g.fcr != 0.f) {
    // The field at the starting point moves with it.  q and J depend on kb
    // and q/pT only through their product (J's q/pT column carries one more
    // factor kb), so the adjoint of kb is
    //   (p3 (pin_3 - pbar_3) + sum_i Jbar_i3 J_i3) / kb
    // with pin_3 the q/pT component of J^T pbar + Jbar . dJ/dp; kb = kb0 (1 +
    // fcz z^2 + fcr r^2) then passes it to x, y, z.
    S jj = S(0);
#pragma unroll
    for (int i = 0; i < 5; ++i)
      if (i != 3) jj = kfma(Jb[i][3], J[i][3], jj);
    const S kbar = kdiv(kfma(p_in[3], pin[3] - pbp[3], jj), kb) * S(2) * (S)g.kb;
    pin[0] = kfma(kbar * (S)g.fcr, p_in[0], pin[0]);
    pin[1] = kfma(kbar * (S)g.fcr, p_in[1], pin[1]);
    pin[2] = kfma(kbar * (S)g.fcz, p_in[2], pin[2]);
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
  if (!crossing(p, R, field_kb<float>(g, p), zc, cosa)) return false;
  return cosa < ADJ_CAREFUL_COS;
}

// Forward step in precision S on float storage: the state before the step at
// st[q * LD], q < 27; the state after it goes to st[(27 + q) * LD].
template <class S, bool EL, bool DISK>
__device__ __noinline__ void fwd_step_store(const DevGeom& g, float* st, const Hit<S>& h, bool first, bool last) {
  S p[6], C[21];
  for (int q = 0; q < 6; ++q) p[q] = (S)st[q * LD];
  for (int q = 0; q < 21; ++q) C[q] = (S)st[(6 + q) * LD];
  fwd_step<S, EL, DISK>(g, p, C, h, first, last);
  for (int q = 0; q < 6; ++q) st[(27 + q) * LD] = (float)p[q];
  for (int q = 0; q < 21; ++q) st[(27 + 6 + q) * LD] = (float)C[q];
}

// Reverse step in precision S with the adjoints kept in A (double in the
// careful pass, float otherwise); the state before the step at st[q * LD].
template <class S, class A, bool EL, bool DISK>
__device__ __noinline__ void rev_step_store(const DevGeom& g, const float* st, const Hit<S>& h, bool first,
                                            bool last, A (&pbA)[6], A (&CbA)[6][6], A (&hbA)[3]) {
  S p[6], C[21], pb[6], Cb[6][6], hb[3];
  for (int q = 0; q < 6; ++q) p[q] = (S)st[q * LD];
  for (int q = 0; q < 21; ++q) C[q] = (S)st[(6 + q) * LD];
  for (int i = 0; i < 6; ++i) {
    pb[i] = (S)pbA[i];
    for (int j = 0; j < 6; ++j) Cb[i][j] = (S)CbA[i][j];
  }
  rev_step<S, EL, DISK>(g, p, C, h, first, last, pb, Cb, hb);
  for (int i = 0; i < 6; ++i) {
    pbA[i] = (A)pb[i];
    for (int j = 0; j < 6; ++j) CbA[i][j] = (A)Cb[i][j];
  }
  for (int i = 0; i < 3; ++i) hbA[i] = (A)hb[i];
}

// Forward step of the FP32 pass, inlined (as rev_step_regs): the state
// before it at in[q * LD], the state after it to out[q * LD].
template <bool EL, bool DISK>
__device__ __forceinline__ void fwd_step_regs(const DevGeom& g, const float* in, float* out, const Hit<float>& h,
                                              bool first, bool last) {
  float p[6], C[21];
#pragma unroll
  for (int q = 0; q < 6; ++q) p[q] = in[q * LD];
#pragma unroll
  for (int q = 0; q < 21; ++q) C[q] = in[(6 + q) * LD];
  fwd_step<float, EL, DISK>(g, p, C, h, first, last);
#pragma unroll
  for (int q = 0; q < 6; ++q) out[q * LD] = p[q];
#pragma unroll
  for (int q = 0; q < 21; ++q) out[(6 + q) * LD] = C[q];
}

// The same reverse step inlined into the FP32 pass, so that the adjoints stay
// in registers (an out-of-line call takes them by reference, through local
// memory).
template <bool EL, bool DISK>
__device__ __forceinline__ void rev_step_regs(const DevGeom& g, const float* st, const Hit<float>& h, bool first,
                                              bool last, float (&pb)[6], float (&Cb)[6][6], float (&hb)[3]) {
  float p[6], C[21];
#pragma unroll
  for (int q = 0; q < 6; ++q) p[q] = st[q * LD];
#pragma unroll
  for (int q = 0; q < 21; ++q) C[q] = st[(6 + q) * LD];
  rev_step<float, EL, DISK>(g, p, C, h, first, last, pb, Cb, hb);
}

// Reverse sweep of the track at position i of the fit's order, from the
// fit's checkpoints (column i).  CAREFUL:
// the track the fit flagged as near-tangent; its near-tangent steps run in
// double precision and its adjoints are kept in double.  seg: this thread's
// column of the block's segment buffer in shared memory (states before each
// step of a segment, [slot][27][LD]).
template <bool CAREFUL, bool EL, bool DISK>
__device__ void adjoint_track(const AdjParams& P, int i, float* seg) {
  using A = typename std::conditional<CAREFUL, double, float>::type;
  const DevGeom& g = P.g;
  const int t = P.order[i];  // the track at position i of the fit's order (checkpoint column i)
  static_assert(CAREFUL, "the FP32 pass is adjoint_track_fp32");
  if (P.fit_status[t] != KF_FIT_OK) {
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
  for (int c = (n - 1) / stride; c >= 0; --c) {
    const int k0 = c * stride, k1 = min(n, k0 + stride);
    const float* ck = P.ckpt + (size_t)c * 27 * P.ns + i;
    for (int q = 0; q < 27; ++q) seg[q * LD] = ck[(size_t)q * P.ns];
    for (int k = k0; k + 1 < k1; ++k) {
      float* st = seg + (k - k0) * 27 * LD;
      const int hi = hoff + lst[k];
      if (CAREFUL && k > 0) {
        float pf[6];
        for (int q = 0; q < 6; ++q) pf[q] = st[q * LD];
        const int Lh = P.hlayer[hi];
        if (is_disk(g, Lh) ? plane_careful(g, pf, plane_z(g, Lh)) : near_tangent(g, pf, g.radius[Lh])) {
          fwd_step_store<double, EL, DISK>(g, st, load_hit<double>(P, hi), k == 0, k + 1 == n);
          continue;
        }
      }
      fwd_step_store<float, EL, DISK>(g, st, load_hit<float>(P, hi), k == 0, k + 1 == n);
    }
    for (int k = k1 - 1; k >= k0; --k) {
      const float* st = seg + (k - k0) * 27 * LD;
      const int hl = lst[k];
      const int hi = hoff + hl;
      A hb[3];
      bool dbl = false;
      if (CAREFUL && k > 0) {
        float pf[6];
        for (int q = 0; q < 6; ++q) pf[q] = st[q * LD];
        const int Lh = P.hlayer[hi];
        dbl = is_disk(g, Lh) ? plane_careful(g, pf, plane_z(g, Lh)) : near_tangent(g, pf, g.radius[Lh]);
      }
      if (dbl)
        rev_step_store<double, A, EL, DISK>(g, st, load_hit<double>(P, hi), k == 0, k + 1 == n, pb, Cb, hb);
      else
        rev_step_store<float, A, EL, DISK>(g, st, load_hit<float>(P, hi), k == 0, k + 1 == n, pb, Cb, hb);
      float* gh = P.g_hits + 3 * (size_t)hi;  // a hit can be on several tracks
      atomicAdd(gh + 0, (float)hb[0]);
      atomicAdd(gh + 1, (float)hb[1]);
      atomicAdd(gh + 2, (float)hb[2]);
      // the layer's alignment gradient (linear in the hit gradient; few
      // tracks); disks carry no alignment
      const int L = P.hlayer[hi];
      if (!is_disk(g, L)) {
        atomicAdd(P.g_align_acc + 2 * L, -((double)P.hx[hi] * hb[1] - (double)P.hy[hi] * hb[0]) / g.radius[L]);
        atomicAdd(P.g_align_acc + 2 * L + 1, -(double)hb[2]);
      }
    }
  }
  if (P.g_seed) {
    for (int k = 0; k < 6; ++k) P.g_seed[(size_t)k * P.ns + t] = (float)pb[k];
  }
}

// Asynchronous copy of one 4-byte word from global memory to this thread's
// shared memory (cp.async: no register holds it in flight), and the waits.
__device__ __forceinline__ void cp_async4(float* sdst, const void* gsrc) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Shared memory of the FP32 pass, in floats per thread column (LD apart):
//   seg [stride - 1][27]  states before a segment's steps after its first
//   ckb [2][27]           the segment's checkpoint (two buffers, by parity)
//   hbf [2][stride][5]    its hits: x, y, z, layer and event-global index (int bits)
//   lbf [2][stride]       event-local hit indices of a later segment
__host__ __device__ constexpr int fp32_col_floats(int stride) { return 27 * (stride - 1) + 54 + 12 * stride; }

// Reverse sweep of the track at position i of the fit's order in FP32 (the
// tracks the fit left without a crossing below ADJ_CAREFUL_COS).  Segment c-1's
// checkpoint and hits are copied into shared memory while segment c is
// reversed, and segment c-2's hit indices with them, so that a segment's
// steps wait on no global load.  col: this thread's column; s_al, s_R: the
// layers' alignment and radii in shared memory; ga: this thread's column of
// alignment-gradient sums (rows 2L and 2L + 1: layer L's rotation and z).
// listed: the track comes from the fit's careful list (else careful tracks
// are skipped: the careful passes take them).
template <bool EL, bool DISK>
__device__ void adjoint_track_fp32(const AdjParams& P, int i, float* col, const float4* s_al, const float* s_R,
                                   float* ga, bool listed) {
  const DevGeom& g = P.g;
  const int t = P.order[i];
  if (!listed && P.careful_flag[t]) return;  // the careful passes', which run beside this one
  if ((P.keep && !P.keep[t]) || P.fit_status[t] != KF_FIT_OK) {
    if (P.g_seed)  // not fitted: no contribution
      for (int k = 0; k < 6; ++k) P.g_seed[(size_t)k * P.ns + t] = 0.f;
    return;
  }
  const int n = P.n_list[t];
  const int* lst = P.lists + (size_t)t * P.max_len;
  const int hoff = P.hit_off[P.seed_event[t]];
  const int stride = P.stride;
  float* const seg = col;
  float* const ckb = col + 27 * (stride - 1) * LD;
  float* const hbf = ckb + 54 * LD;
  float* const lbf = hbf + 10 * stride * LD;
  auto seg_lists = [&](int c) {  // hit indices of segment c -> lbf[c & 1]
    const int k0 = c * stride, k1 = min(n, k0 + stride);
    float* d = lbf + (c & 1) * stride * LD;
    for (int k = k0; k < k1; ++k) cp_async4(d + (k - k0) * LD, lst + k);
  };
  auto seg_data = [&](int c) {  // checkpoint and hits of segment c (its indices in lbf[c & 1])
    const int k0 = c * stride, k1 = min(n, k0 + stride);
    const float* ck = P.ckpt + (size_t)c * 27 * P.ns + i;
    float* cd = ckb + (c & 1) * 27 * LD;
    for (int q = 0; q < 27; ++q) cp_async4(cd + q * LD, ck + (size_t)q * P.ns);
    const float* ls = lbf + (c & 1) * stride * LD;
    float* hd = hbf + (c & 1) * 5 * stride * LD;
    for (int k = k0; k < k1; ++k) {
      const int hi = hoff + __float_as_int(ls[(k - k0) * LD]);
      float* d = hd + (k - k0) * 5 * LD;
      cp_async4(d, P.hx + hi);
      cp_async4(d + LD, P.hy + hi);
      cp_async4(d + 2 * LD, P.hz + hi);
      cp_async4(d + 3 * LD, P.hlayer + hi);
      d[4 * LD] = __int_as_float(hi);
    }
  };
  float pb[6], Cb[6][6];
#pragma unroll
  for (int a = 0; a < 6; ++a) {
    pb[a] = 0.f;
#pragma unroll
    for (int b = 0; b < 6; ++b) Cb[a][b] = 0.f;
  }
  const int last = (n - 1) / stride;
  seg_lists(last);
  cp_async_commit();
  cp_async_wait_all();
  seg_data(last);
  if (last > 0) seg_lists(last - 1);
  cp_async_commit();
  for (int c = last; c >= 0; --c) {
    cp_async_wait_all();  // segment c's checkpoint and hits, segment c-1's indices
    if (c > 0) {
      seg_data(c - 1);
      if (c > 1) seg_lists(c - 2);
      cp_async_commit();
    }
    const int k0 = c * stride, k1 = min(n, k0 + stride);
    const float* ck = ckb + (c & 1) * 27 * LD;
    const float* hs = hbf + (c & 1) * 5 * stride * LD;
    auto hit_of = [&](int k) {
      const float* d = hs + (k - k0) * 5 * LD;
      Hit<float> h;
      h.L = __float_as_int(d[3 * LD]);
      const float x = d[0], y = d[LD], z = d[2 * LD];
      if (DISK && is_disk(g, h.L)) {  // raw position: disks carry no alignment
        h.ca = 1.f;
        h.sa = 0.f;
        h.R = 0.f;
        h.mx = x;
        h.my = y;
        h.mz = z;
        return h;
      }
      const float4 a = s_al[h.L];  // (cos, sin, dphi, az)
      h.ca = a.x;
      h.sa = a.y;
      h.R = s_R[h.L];
      h.mx = kfma(h.ca, x, -h.sa * y);
      h.my = kfma(h.sa, x, h.ca * y);
      h.mz = z - a.w;
      return h;
    };
    // state before step k: the checkpoint for k0, else seg slot k - k0 - 1
    for (int k = k0; k + 1 < k1; ++k)
      fwd_step_regs<EL, DISK>(g, k == k0 ? ck : seg + (k - k0 - 1) * 27 * LD, seg + (k - k0) * 27 * LD,
                              hit_of(k), k == 0, k + 1 == n);
    for (int k = k1 - 1; k >= k0; --k) {
      float hb[3];
      rev_step_regs<EL, DISK>(g, k == k0 ? ck : seg + (k - k0 - 1) * 27 * LD, hit_of(k), k == 0, k + 1 == n, pb, Cb,
                              hb);
      const float* hd = hs + (k - k0) * 5 * LD;
      const int hi = __float_as_int(hd[4 * LD]);
      float* gh = P.g_hits + 3 * (size_t)hi;  // a hit can be on several tracks
      atomicAdd(gh + 0, hb[0]);
      atomicAdd(gh + 1, hb[1]);
      atomicAdd(gh + 2, hb[2]);
      // the layer's alignment gradient (linear in the hit gradient), summed
      // in this thread's column
      const int L = __float_as_int(hd[3 * LD]);
      if (!DISK || !is_disk(g, L)) {
        ga[2 * L * LD] -= kfma(hd[0], hb[1], -hd[LD] * hb[0]) / s_R[L];
        ga[(2 * L + 1) * LD] -= hb[2];
      }
    }
  }
  if (P.g_seed) {
    for (int k = 0; k < 6; ++k) P.g_seed[(size_t)k * P.ns + t] = pb[k];
  }
}

// Passes of the adjoint: the FP32 pass over every position (the tracks of
// the fit's careful list skipped), and over the careful list the entries
// without CAREFUL_DBL_BIT in FP32 and those with it in double.
enum { ADJ_ALL = 0, ADJ_LIST_FP32 = 1, ADJ_LIST_DBL = 2 };

template <int MODE, bool EL, bool DISK = false>
__global__ void __launch_bounds__(ADJ_THREADS) k_adjoint(const AdjParams P) {
  // double pass: [stride][27][LD]; FP32 passes: columns of fp32_col_floats,
  // then 2 x layers rows of alignment-gradient sums
  extern __shared__ float seg_all[];
  float* seg = seg_all + threadIdx.x;
  if constexpr (MODE != ADJ_LIST_DBL) {
    __shared__ float4 s_al[KF_MAX_LAYERS];
    __shared__ float s_R[KF_MAX_LAYERS];
    const int nga = 2 * P.g.n_layers;
    float* const ga_all = seg_all + (size_t)fp32_col_floats(P.stride) * LD;  // [nga][LD]
    float* const ga = ga_all + threadIdx.x;
    for (int q = 0; q < nga; ++q) ga[q * LD] = 0.f;
    for (int l = threadIdx.x; l < P.g.n_layers; l += blockDim.x) {
      const Align4 a = P.align[l];
      s_al[l] = make_float4(a.ca, a.sa, a.dphi, a.az);
      s_R[l] = P.g.radius[l];
    }
    __syncthreads();
    if constexpr (MODE == ADJ_ALL) {
      const int i = blockIdx.x * blockDim.x + threadIdx.x;
      if (i < P.ns) adjoint_track_fp32<EL, DISK>(P, i, seg, s_al, s_R, ga, false);
    } else {
      const unsigned n = *P.careful_count;
      for (unsigned j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        const unsigned v = (unsigned)P.careful_list[j];
        if (!(v & CAREFUL_DBL_BIT)) adjoint_track_fp32<EL, DISK>(P, (int)v, seg, s_al, s_R, ga, true);
      }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < nga; q += blockDim.x) {  // row q over the columns, rotated by q (banks)
      float a = 0.f;
      for (int c = 0; c < LD; ++c) a += ga_all[q * LD + ((c + q) & (LD - 1))];
      if (a != 0.f) atomicAdd(P.g_align_acc + q, (double)a);
    }
  } else {  // packed list: the first blocks take all of them and the others end at once
    const unsigned n = *P.dbl_count;
    for (unsigned j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
      adjoint_track<true, EL, DISK>(P, P.dbl_list[j], seg);
  }
}

__global__ void k_adjoint_finish(const AdjParams P) {
  const int i = threadIdx.x;
  if (i < 2 * P.g.n_layers) P.g_align[i] = (float)P.g_align_acc[i];
}

}  // namespace

bool adjoint_stride_ok(int stride, int max_len) {
  return stride >= 1 && stride <= MAX_CKPT_STRIDE && max_len <= MAX_CKPT * stride;
}

cudaError_t launch_adjoint_begin(const AdjParams& P, cudaStream_t st) {
  if (!P.g_hits) return cudaErrorInvalidValue;  // the alignment gradient is formed from it
  cudaError_t e = cudaMemsetAsync(P.g_align_acc, 0, sizeof(double) * 2 * KF_MAX_LAYERS, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(P.g_hits, 0, sizeof(float) * 3 * (size_t)P.n_hits, st);
  if (e != cudaSuccess) return e;
  const int smem_c = (int)(sizeof(float) * 27 * (size_t)P.stride * ADJ_THREADS);
  const int smem_f = (int)(sizeof(float) * (fp32_col_floats(P.stride) + 2 * P.g.n_layers) * (size_t)ADJ_THREADS);
  const void* fns[12] = {(const void*)k_adjoint<ADJ_ALL, false>,        (const void*)k_adjoint<ADJ_LIST_FP32, false>,
                         (const void*)k_adjoint<ADJ_LIST_DBL, false>,   (const void*)k_adjoint<ADJ_ALL, true>,
                         (const void*)k_adjoint<ADJ_LIST_FP32, true>,   (const void*)k_adjoint<ADJ_LIST_DBL, true>,
                         (const void*)k_adjoint<ADJ_ALL, false, true>,  (const void*)k_adjoint<ADJ_LIST_FP32, false, true>,
                         (const void*)k_adjoint<ADJ_LIST_DBL, false, true>, (const void*)k_adjoint<ADJ_ALL, true, true>,
                         (const void*)k_adjoint<ADJ_LIST_FP32, true, true>, (const void*)k_adjoint<ADJ_LIST_DBL, true, true>};
  for (int k = 0; k < 12 && e == cudaSuccess; ++k)
    e = cudaFuncSetAttribute(fns[k], cudaFuncAttributeMaxDynamicSharedMemorySize, k % 3 == 2 ? smem_c : smem_f);
  return e;
}

cudaError_t launch_adjoint_pass(const AdjParams& P, bool careful, cudaStream_t st) {
  if (P.ns <= 0) return cudaSuccess;
  const size_t smem_c = sizeof(float) * 27 * (size_t)P.stride * ADJ_THREADS;
  const size_t smem_f = sizeof(float) * (fp32_col_floats(P.stride) + 2 * P.g.n_layers) * (size_t)ADJ_THREADS;
  bool el = false;  // energy loss on any layer: the variant with its code
  for (int l = 0; l < P.g.n_layers; ++l) el = el || P.g.eloss[l] > 0.f;
  const int grid_all = (P.ns + ADJ_THREADS - 1) / ADJ_THREADS;
  // flagged tracks are a few percent: a grid for a twentieth of all, striding
  // over however many there are
  const int grid_careful = (P.ns / 20 + ADJ_THREADS - 1) / ADJ_THREADS + 1;
  // the double pass: blocks of 32 threads (its tracks' double-precision
  // steps are bound by the SM's FP64 rate, so they spread over many SMs)
  constexpr int DBL_THREADS = 32;
  const int grid_dbl = (P.ns / 20 + DBL_THREADS - 1) / DBL_THREADS + 1;
  if (P.g.n_disks > 0) {  // the disk variants; energy loss on a layer or on the disks
    if (P.g.disk_eloss > 0.f) el = true;
    if (!careful) {
      if (el) k_adjoint<ADJ_ALL, true, true><<<grid_all, ADJ_THREADS, smem_f, st>>>(P);
      else k_adjoint<ADJ_ALL, false, true><<<grid_all, ADJ_THREADS, smem_f, st>>>(P);
    } else {
      if (el) k_adjoint<ADJ_LIST_DBL, true, true><<<grid_dbl, DBL_THREADS, smem_c, st>>>(P);
      else k_adjoint<ADJ_LIST_DBL, false, true><<<grid_dbl, DBL_THREADS, smem_c, st>>>(P);
      if (el) k_adjoint<ADJ_LIST_FP32, true, true><<<grid_careful, ADJ_THREADS, smem_f, st>>>(P);
      else k_adjoint<ADJ_LIST_FP32, false, true><<<grid_careful, ADJ_THREADS, smem_f, st>>>(P);
    }
  } else if (!careful) {
    if (el) k_adjoint<ADJ_ALL, true><<<grid_all, ADJ_THREADS, smem_f, st>>>(P);
    else k_adjoint<ADJ_ALL, false><<<grid_all, ADJ_THREADS, smem_f, st>>>(P);
  } else {  // the careful list: its tracks with double steps, then the others
    if (el) k_adjoint<ADJ_LIST_DBL, true><<<grid_dbl, DBL_THREADS, smem_c, st>>>(P);
    else k_adjoint<ADJ_LIST_DBL, false><<<grid_dbl, DBL_THREADS, smem_c, st>>>(P);
    if (el) k_adjoint<ADJ_LIST_FP32, true><<<grid_careful, ADJ_THREADS, smem_f, st>>>(P);
    else k_adjoint<ADJ_LIST_FP32, false><<<grid_careful, ADJ_THREADS, smem_f, st>>>(P);
  }
  return cudaGetLastError();
}

cudaError_t launch_adjoint_end(const AdjParams& P, cudaStream_t st) {
  k_adjoint_finish<<<1, 2 * KF_MAX_LAYERS, 0, st>>>(P);
  return cudaGetLastError();
}

}  // namespace kfg
