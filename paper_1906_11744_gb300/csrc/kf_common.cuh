// Device-side Kalman-filter arithmetic shared by the finding, fitting and
// adjoint kernels (registers only; templated on the scalar type so that the
// fit can redo an ill-conditioned step in double precision).
//
// Track state p = (x, y, z, q/pT, phi, theta); covariance C as the 21-float
// upper triangle.  The method follows the paper's Kalman-filter building and
// fitting (Sec. 2) with the largest matrices being the symmetric 6x6
// covariance (Sec. 2, Matriplex paragraph): every product below skips the
// structural zeros and ones of the propagation Jacobian, the GPU counterpart of
// the paper's known-element elimination.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "kf.h"

namespace kfg {

constexpr float KCURV = 0.00299792458f;  // 1/rho [1/cm] = KCURV * B[T] / pT[GeV]
constexpr double MPION = 0.13957;
constexpr float PI_F = 3.14159265358979323846f;
constexpr float TWO_PI_F = 6.28318530717958647692f;
constexpr int MAX_ETA_BINS = 256;
constexpr int ETA_LUT = 4096;  // uniform z cells per layer of the eta-bin first guess

// Geometry and settings, passed by value as a kernel parameter.
struct DevGeom {
  int n_layers;
  int max_cands;
  int max_holes;
  int n_eta;
  int n_phi;
  float z_max;
  float kb;  // -KCURV * bz: signed curvature h = kb * (q/pT) in the nominal field
  float fcz, fcr;  // field factor 1 + fcz z^2 + fcr r^2 at a point (0, 0: uniform)
  float vr;  // sigma_rphi^2
  float vz;  // sigma_z^2
  float chi2_cut;
  float phi_scale;      // n_phi / 2 pi
  float eta_lut_scale;  // ETA_LUT / (2 z_max)
  float radius[KF_MAX_LAYERS];
  float x0[KF_MAX_LAYERS];
  float eta_max[KF_MAX_LAYERS];  // asinh(z_max / R): half-range of the eta grid
  float eloss[KF_MAX_LAYERS];  // mean ionization loss per layer (GeV, 0: none)
  float eta_scale[KF_MAX_LAYERS];  // n_eta / (2 eta_max): eta bins per unit of eta
  float r_inv[KF_MAX_LAYERS];      // 1 / R
  // Material map (null: the per-layer x0): thickness [n_layers][n_z] at z
  // nodes spread evenly over [-z_max, z_max]; z_node_inv = (n_z - 1)/(2 z_max).
  const float* x0map;
  int n_z;
  float z_node_inv;
  // Endcap disks (n_disks = 0: a barrel detector): surfaces n_layers .. are
  // the +z disks at disk_z[k], then the -z disks at -disk_z[k].
  int n_surf;  // n_layers + 2 n_disks
  int n_plan;  // the longest search plan: n_layers + n_disks
  int n_disks;
  float disk_z[KF_MAX_DISKS];
  float disk_rmin, disk_rmax, disk_x0, disk_eloss;
  float vrr;          // sigma_r^2
  float disk_rscale;  // n_eta / (disk_rmax - disk_rmin): rows of a disk's hit grid, in r
  float eta_barrel;   // seeds with |eta| >= eta_barrel search their side's disks after the barrel
};

// Per-layer alignment: (cos a, sin a) of the correction rotation a = -a_rphi/R,
// the raw-angle offset a_rphi/R and a_z.
struct Align4 {
  float ca, sa, dphi, az;
};

__host__ __device__ constexpr int S6(int i, int j) {
  return i <= j ? i * 6 - i * (i - 1) / 2 + (j - i) : j * 6 - j * (j - 1) / 2 + (i - j);
}

// Structure of the propagation Jacobian: 0 = structural zero, 1 = one, 2 = value.
// Rows q/pT and theta are identity; x', y', phi' depend on (x, y, q/pT, phi);
// z' depends on all six with dz'/dz = 1.
__host__ __device__ constexpr int JS(int i, int j) {
  return (i == 3) ? (j == 3 ? 1 : 0)
         : (i == 5) ? (j == 5 ? 1 : 0)
         : (i == 2) ? (j == 2 ? 1 : 2)
         : ((j == 2 || j == 5) ? 0 : 2);
}
__host__ __device__ constexpr int JNNZ(int i) {
  return (i == 3 || i == 5) ? 1 : (i == 2 ? 6 : 4);
}

// Scalar-generic math (float -> single-precision intrinsics, double -> double).
__device__ __forceinline__ float kfma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double kfma(double a, double b, double c) { return fma(a, b, c); }
// FP32 sine and cosine by the hardware approximation (absolute error about
// 4e-7 on [-pi, pi], far below what the state's FP32 rounding already costs
// a track), after reducing the argument into [-pi, pi]; angles here are
// directions and polar angles, within a few turns.
__device__ __forceinline__ void ksincos(float x, float* s, float* c) {
  const float k = rintf(x * (1.f / TWO_PI_F));
  __sincosf(fmaf(-k, TWO_PI_F, x), s, c);
}
__device__ __forceinline__ void ksincos(double x, double* s, double* c) { sincos(x, s, c); }
// The library's sine and cosine (a relative error of a few ulp at every
// angle).  The hardware approximation's absolute error (about 4e-7) is a
// large relative error where the sine or cosine is small: a direction near
// an axis then moves a step's position across the axis by the step length
// times 4e-7, which single precision would resolve 30 times more finely.
// The fit and its adjoint take these (ACC); the finding, whose hit lists and
// parameters do not see the difference, the hardware approximation.
__device__ __forceinline__ void ksincos_acc(float x, float* s, float* c) { sincosf(x, s, c); }
__device__ __forceinline__ void ksincos_acc(double x, double* s, double* c) { sincos(x, s, c); }
template <bool ACC, class T>
__device__ __forceinline__ void ksc(T x, T* s, T* c) {
  if constexpr (ACC) ksincos_acc(x, s, c);
  else ksincos(x, s, c);
}
__device__ __forceinline__ float ksqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double ksqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float krsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double krsqrt(double x) { return 1.0 / sqrt(x); }
__device__ __forceinline__ float katan(float x) { return atanf(x); }
__device__ __forceinline__ double katan(double x) { return atan(x); }
__device__ __forceinline__ float ksin(float x) { return sinf(x); }
__device__ __forceinline__ double ksin(double x) { return sin(x); }
__device__ __forceinline__ float klog(float x) { return __logf(x); }  // hardware approximation
__device__ __forceinline__ double klog(double x) { return log(x); }
__device__ __forceinline__ float kabs(float x) { return fabsf(x); }
__device__ __forceinline__ double kabs(double x) { return fabs(x); }
__device__ __forceinline__ float kmin(float a, float b) { return fminf(a, b); }
// Quotient and reciprocal: FP32 by the hardware reciprocal (about 2 ulp, far
// below what the state's FP32 rounding already costs a track), double exact.
__device__ __forceinline__ float kdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double kdiv(double a, double b) { return a / b; }
__device__ __forceinline__ double kmin(double a, double b) { return fmin(a, b); }

// sinc(psi) = sin(psi)/psi, cosc(psi) = (1 - cos psi)/psi,
// f1 = (psi cos psi - sin psi)/psi^2, f2 = (psi sin psi - 1 + cos psi)/psi^2.
// Power series (derived from the Taylor series of sin and cos) below |psi| =
// 0.5, which covers every layer-to-layer step above pT = 0.5 GeV; direct forms
// without cancellation above.
template <class T>
__device__ __forceinline__ void helix_fns(T psi, T& sc, T& cc, T& f1, T& f2) {
  if (kabs(psi) < T(0.5)) {
    const T q = psi * psi;
    sc = kfma(q, kfma(q, kfma(q, kfma(q, T(1.0 / 362880.0), T(-1.0 / 5040.0)), T(1.0 / 120.0)), T(-1.0 / 6.0)), T(1));
    cc = psi * kfma(q, kfma(q, kfma(q, kfma(q, T(1.0 / 3628800.0), T(-1.0 / 40320.0)), T(1.0 / 720.0)),
                            T(-1.0 / 24.0)), T(0.5));
    f1 = psi * kfma(q, kfma(q, kfma(q, kfma(q, T(-1.0 / 3991680.0), T(1.0 / 45360.0)), T(-1.0 / 840.0)),
                            T(1.0 / 30.0)), T(-1.0 / 3.0));
    f2 = kfma(q, kfma(q, kfma(q, kfma(q, T(1.0 / 403200.0), T(-1.0 / 5760.0)), T(1.0 / 144.0)), T(-1.0 / 8.0)),
              T(0.5));
    if (sizeof(T) == 8) {  // double: extend each series by its next term
      const T q5 = q * q * q * q * q;
      sc += q5 * T(-1.0 / 39916800.0);
      cc += psi * q5 * T(-1.0 / 479001600.0);
      f1 += psi * q5 * T(12.0 / 6227020800.0);
      f2 += q5 * T(-11.0 / 479001600.0);
    }
  } else {
    T sn, cs;
    ksincos(psi, &sn, &cs);
    const T hs = ksin(T(0.5) * psi);
    const T ip = T(1) / psi;
    sc = sn * ip;
    cc = T(2) * hs * hs * ip;
    f1 = (cs - sc) * ip;
    f2 = (sn - cc) * ip;
  }
}

// Smallest s > 0 (transverse arc length) with x(s)^2 + y(s)^2 = R^2.
// psi = h s solves A sin psi + B (1 - cos psi) = E with A = b h, B = a h + 1,
// E = h^2 (R^2 - r0^2)/2; tau = tan(psi/2) solves (2B - E) tau^2 + 2A tau - E = 0,
// each root taken in its cancellation-free form.
template <class T>
__device__ __forceinline__ bool path_length(T x, T y, T h, T cf, T sf, T R, T& s) {
  const T b = kfma(x, cf, y * sf);
  const T a = kfma(y, cf, -x * sf);
  const T r0 = ksqrt(kfma(x, x, y * y));
  const T dR2 = (R - r0) * (R + r0);
  if (h == T(0)) {
    const T disc = kfma(b, b, dR2);
    if (disc < T(0)) return false;
    const T sq = ksqrt(disc);
    T lo, hi;
    if (b > T(0)) {
      lo = -(b + sq);
      hi = dR2 / (b + sq);
    } else {
      hi = sq - b;
      lo = (hi == T(0)) ? T(0) : -dR2 / hi;
    }
    if (lo > T(0)) { s = lo; return true; }
    if (hi > T(0)) { s = hi; return true; }
    return false;
  }
  const T A = b * h;
  const T B = kfma(a, h, T(1));
  const T E = T(0.5) * h * h * dR2;
  const T den = T(2) * B - E;
  const T D = kfma(A, A, E * den);
  if (D < T(0)) return false;
  const T sq = ksqrt(D);
  // Outward crossing (the usual step to the next layer): inside the cylinder
  // (E > 0), moving outward (b > 0, A = b h not zero) with den > 0, the root of
  // the sign of h is
  // tau = E / (A + sq) for h > 0 and E / (A - sq) for h < 0, and the other
  // root has the opposite sign, so the general selection below would take
  // exactly this one; its quotient, arctangent and arc length are the same
  // operations as there.
  if (E > T(0) && b > T(0) && den > T(0) && A != T(0)) {
    const T psi = T(2) * katan(kdiv(E, h > T(0) ? A + sq : A - sq));
    s = psi * kdiv(T(1), h);
    return true;
  }
  T n0, d0, n1, d1;
  if (A >= T(0)) {
    n0 = E; d0 = A + sq; n1 = -(A + sq); d1 = den;
  } else {
    n0 = sq - A; d0 = den; n1 = E; d1 = A - sq;
  }
  // s_k = psi_k / h with psi_k = 2 atan(tau_k), tau_k = n_k / d_k (psi = pi for
  // d_k = 0), plus a full turn when not positive; the smaller s is taken.
  // psi is increasing in tau, so the root is chosen on tau and one atan is
  // evaluated: for h > 0 positive tau (smallest first) before negative (most
  // negative first); for h < 0 negative tau (closest to 0 first) before
  // positive (largest first, d = 0 first of all); tau = 0 (s = a full turn)
  // and n = d = 0 (no root) last.
  const T turn = kdiv(T(2.0 * 3.14159265358979323846), kabs(h));
  const T ih = kdiv(T(1), h);
  const bool pos_h = h > T(0);
  // rank: 0 preferred class, 1 other sign, 2 tau = 0, 3 no root
  auto rank_of = [&](T nn, T dd, T& tau) {
    if (dd == T(0)) {
      tau = T(INFINITY);
      return nn == T(0) ? 3 : (pos_h ? 0 : 1);
    }
    tau = kdiv(nn, dd);
    if (tau == T(0)) return 2;
    return (tau > T(0)) == pos_h ? 0 : 1;
  };
  T t0, t1;
  const int k0 = rank_of(n0, d0, t0), k1 = rank_of(n1, d1, t1);
  if (k0 == 3 && k1 == 3) return false;
  // same rank: ascending tau for h > 0, descending for h < 0
  const bool first = k0 != k1 ? k0 < k1 : (pos_h ? t0 <= t1 : t0 >= t1);
  const T dd = first ? d0 : d1, tc = first ? t0 : t1;
  const T psi = dd == T(0) ? T(3.14159265358979323846) : T(2) * katan(tc);
  T best = psi * ih;
  if (best <= T(0)) best += turn;
  if (!(best < T(INFINITY))) return false;
  s = best;
  return true;
}

// C <- J C J^T using only the structural non-zeros of J (JS).  J entries with
// JS == 2 must be set; others are ignored.  Rows 3 and 5 of J are unit rows,
// so (J C) has C's rows there and C' keeps C's (3,3), (3,5), (5,5).  The
// other rows i are taken one at a time in the order 2, 0, 1, 4: T_i = J_i C,
// then C'_ik = T_i . J_k for the rows k not yet done (k = i included) and
// C'_i3 = T_i[3], C'_i5 = T_i[5] (the unit rows of J).  Only one row of J C is
// live at a time, which keeps the register demand of the step low.
template <class T>
__device__ __forceinline__ void transport(const T (&J)[6][6], T (&C)[21]) {
  constexpr int ORD[4] = {2, 0, 1, 4};
  T out[21];
  out[S6(3, 3)] = C[S6(3, 3)];
  out[S6(3, 5)] = C[S6(3, 5)];
  out[S6(5, 5)] = C[S6(5, 5)];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int i = ORD[a];
    T t[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      T acc = T(0);
      bool first = true;
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        if (JS(i, j) == 0) continue;
        const T c = C[S6(j, k)];
        if (JS(i, j) == 1) acc = first ? c : acc + c;
        else acc = first ? J[i][j] * c : kfma(J[i][j], c, acc);
        first = false;
      }
      t[k] = acc;
    }
    out[S6(i, 3)] = t[3];
    out[S6(i, 5)] = t[5];
#pragma unroll
    for (int b = a; b < 4; ++b) {
      const int kr = ORD[b];
      T acc = T(0);
      bool first = true;
#pragma unroll
      for (int m = 0; m < 6; ++m) {
        if (JS(kr, m) == 0) continue;
        if (JS(kr, m) == 1) acc = first ? t[m] : acc + t[m];
        else acc = first ? t[m] * J[kr][m] : kfma(t[m], J[kr][m], acc);
        first = false;
      }
      out[S6(i, kr)] = acc;
    }
  }
#pragma unroll
  for (int k = 0; k < 21; ++k) C[k] = out[k];
}

// kb of the field at the point (p[0], p[1], p[2]) (Sec. 3, parameterized
// field): kb (1 + fcz z^2 + fcr r^2); exactly kb in a uniform field.  Each
// propagation takes it at its starting point.
template <class T>
__device__ __forceinline__ T field_kb(const DevGeom& g, const T (&p)[6]) {
  return (T)g.kb * kfma((T)g.fcz, p[2] * p[2], kfma((T)g.fcr, kfma(p[0], p[0], p[1] * p[1]), T(1)));
}

// Path length and crossing geometry only: returns false without a crossing;
// z_out is z at the crossing and cos_out = |cos| of the angle between the
// direction and the radial direction there (1 = radial, 0 = tangent).
__device__ __forceinline__ bool crossing(const float (&p)[6], float R, float kb, float& z_out,
                                         float& cos_out) {
  float sf, cf;
  sincosf(p[4], &sf, &cf);
  const float h = kb * p[3];
  float s;
  if (!path_length<float>(p[0], p[1], h, cf, sf, R, s)) return false;
  float sth, cth;
  sincosf(p[5], &sth, &cth);
  z_out = fmaf(s, cth / sth, p[2]);
  const float psi = h * s;
  float sc, cc, f1, f2;
  helix_fns<float>(psi, sc, cc, f1, f2);
  const float Sx = s * sc, Cx = s * cc;
  const float xn = p[0] + fmaf(cf, Sx, -sf * Cx);
  const float yn = p[1] + fmaf(sf, Sx, cf * Cx);
  const float cpsi = fmaf(-psi, cc, 1.f), spsi = psi * sc;
  const float cp = fmaf(cf, cpsi, -sf * spsi), sp = fmaf(sf, cpsi, cf * spsi);
  cos_out = fabsf(fmaf(xn, cp, yn * sp)) * rsqrtf(fmaf(xn, xn, yn * yn));
  return true;
}

// Propagation to the cylinder of radius R (closed-form helix, exact
// Jacobian, covariance transport).  Returns 1 on success (p, C updated),
// 0 without a crossing, 2 when |z| at the crossing exceeds z_lim; p and C are
// untouched unless 1 is returned.  cos_out (optional) receives |cos| of the
// angle between the direction and the radial direction at the crossing,
// s_out (optional) the transverse path length, trig (optional, 6 values) the
// sine and cosine of phi and theta at the start and of phi at the crossing.
// ACC: the library's sine and cosine (ksincos_acc).
template <class T, bool ACC = false>
__device__ __forceinline__ int prop_jacobian(const T (&p)[6], T R, T kb, T z_lim, T (&q)[6], T (&J)[6][6],
                                             T* cos_out = nullptr, T* s_out = nullptr, T* trig = nullptr) {
  const T x = p[0], y = p[1], kap = p[3], phi = p[4], th = p[5];
  T sf, cf;
  ksc<ACC>(phi, &sf, &cf);
  const T h = kb * kap;
  T s;
  if (!path_length<T>(x, y, h, cf, sf, R, s)) return 0;
  T sth, cth;
  ksc<ACC>(th, &sth, &cth);
  const T cot = kdiv(cth, sth);
  const T zn = kfma(s, cot, p[2]);
  if (kabs(zn) > z_lim) return 2;
  const T psi = h * s;
  T sc, cc, f1, f2;
  helix_fns<T>(psi, sc, cc, f1, f2);
  const T Sx = s * sc, Cx = s * cc;
  const T dx = kfma(cf, Sx, -sf * Cx);
  const T dy = kfma(sf, Sx, cf * Cx);
  const T xn = x + dx, yn = y + dy;
  // direction at the crossing: cos psi = 1 - psi*cc, sin psi = psi*sc
  const T cpsi = kfma(-psi, cc, T(1)), spsi = psi * sc;
  const T cp = kfma(cf, cpsi, -sf * spsi);
  const T sp = kfma(sf, cpsi, cf * spsi);
  const T s2 = s * s;
  const T dSdh = s2 * f1, dCdh = s2 * f2;
  const T Fx3 = kb * kfma(cf, dSdh, -sf * dCdh);
  const T Fy3 = kb * kfma(sf, dSdh, cf * dCdh);
  const T Fx4 = -dy, Fy4 = dx;
  const T dgds = kfma(xn, cp, yn * sp);
  if (cos_out) *cos_out = kabs(dgds) / R;
  if (s_out) *s_out = s;
  if (trig) {
    trig[0] = sf;
    trig[1] = cf;
    trig[2] = sth;
    trig[3] = cth;
    trig[4] = sp;
    trig[5] = cp;
  }
  const T inv = kdiv(T(-1), dgds);
  const T ds0 = xn * inv, ds1 = yn * inv;
  const T ds3 = kfma(xn, Fx3, yn * Fy3) * inv;
  const T ds4 = kfma(xn, Fx4, yn * Fy4) * inv;
  J[0][0] = kfma(cp, ds0, T(1)); J[0][1] = cp * ds1; J[0][3] = kfma(cp, ds3, Fx3); J[0][4] = kfma(cp, ds4, Fx4);
  J[1][0] = sp * ds0; J[1][1] = kfma(sp, ds1, T(1)); J[1][3] = kfma(sp, ds3, Fy3); J[1][4] = kfma(sp, ds4, Fy4);
  J[2][0] = cot * ds0; J[2][1] = cot * ds1; J[2][3] = cot * ds3; J[2][4] = cot * ds4;
  J[2][5] = -kdiv(s, sth * sth);
  J[4][0] = h * ds0; J[4][1] = h * ds1; J[4][3] = kfma(h, ds3, kb * s); J[4][4] = kfma(h, ds4, T(1));
  q[0] = xn;
  q[1] = yn;
  q[2] = zn;
  q[3] = kap;
  q[4] = phi + psi;
  q[5] = th;
  return 1;
}

template <class T, bool ACC = false>
__device__ __forceinline__ int propagate(T (&p)[6], T (&C)[21], T R, T kb, T z_lim, T* cos_out = nullptr) {
  T q[6], J[6][6];
  const int rc = prop_jacobian<T, ACC>(p, R, kb, z_lim, q, J, cos_out);
  if (rc != 1) return rc;
  transport<T>(J, C);
#pragma unroll
  for (int k = 0; k < 6; ++k) p[k] = q[k];
  return 1;
}

// Tangent-frame measurement at the prediction: u = (-sin phi_p, cos phi_p)
// with (cos, sin) phi_p = (x, y)/r; a0 = C H0^T, S = H C H^T + V, S^-1.
template <class T>
struct FrameT {
  T su, cu;
  T a0[6];
  T s00, s11;
  T si00, si01, si11;
};
using Frame = FrameT<float>;

template <class T>
__device__ __forceinline__ void make_frame(const T (&p)[6], const T (&C)[21], T vr, T vz, FrameT<T>& f) {
  const T ir = krsqrt(kfma(p[0], p[0], p[1] * p[1]));
  f.cu = p[0] * ir;
  f.su = p[1] * ir;
#pragma unroll
  for (int i = 0; i < 6; ++i) f.a0[i] = kfma(-f.su, C[S6(i, 0)], f.cu * C[S6(i, 1)]);
  const T s00 = kfma(-f.su, f.a0[0], kfma(f.cu, f.a0[1], vr));
  const T s01 = f.a0[2];
  const T s11 = C[S6(2, 2)] + vz;
  const T idet = kdiv(T(1), kfma(s00, s11, -s01 * s01));
  f.s00 = s00;
  f.s11 = s11;
  f.si00 = s11 * idet;
  f.si01 = -s01 * idet;
  f.si11 = s00 * idet;
}

// Residual of a corrected hit m against the prediction; false on the far half.
template <class T>
__device__ __forceinline__ bool residual(const T (&p)[6], const FrameT<T>& f, T mx, T my, T mz, T& r0,
                                         T& r1) {
  if (kfma(mx, p[0], my * p[1]) <= T(0)) return false;
  r0 = kfma(-f.su, mx - p[0], f.cu * (my - p[1]));
  r1 = mz - p[2];
  return true;
}

template <class T>
__device__ __forceinline__ T chi2_of(const FrameT<T>& f, T r0, T r1) {
  return kfma(f.si00 * r0, r0, kfma(T(2) * f.si01 * r0, r1, f.si11 * r1 * r1));
}

// Gain K = C H^T S^-1, p += K r, C -= K H C (upper triangle).
template <class T>
__device__ __forceinline__ void kf_update(T (&p)[6], T (&C)[21], const FrameT<T>& f, T r0, T r1) {
  T a1[6], k0[6], k1[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) a1[i] = C[S6(i, 2)];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    k0[i] = kfma(f.a0[i], f.si00, a1[i] * f.si01);
    k1[i] = kfma(f.a0[i], f.si01, a1[i] * f.si11);
  }
#pragma unroll
  for (int i = 0; i < 6; ++i) p[i] = kfma(k0[i], r0, kfma(k1[i], r1, p[i]));
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int j = i; j < 6; ++j) C[S6(i, j)] -= kfma(k0[i], f.a0[j], k1[i] * a1[j]);
}

// Thin-scatterer multiple scattering (Highland width, pion mass for beta):
// Var(phi) += theta0^2 / sin^2(theta), Var(theta) += theta0^2.
// The two variance terms (phi-phi, theta-theta) the scattering adds.
template <class T, bool ACC = false>
__device__ __forceinline__ void ms_terms(const T (&p)[6], T x0, T& q44, T& q55) {
  if (p[3] == T(0) || x0 <= T(0)) {
    q44 = T(0);
    q55 = T(0);
    return;
  }
  T sth, cth, sph, cph;
  ksc<ACC>(p[5], &sth, &cth);
  ksc<ACC>(p[4], &sph, &cph);
  const T ir = krsqrt(kfma(p[0], p[0], p[1] * p[1]));
  const T cdiff = kfma(cph, p[0], sph * p[1]) * ir;  // cos(phi - phi_p)
  const T pm = kdiv(T(1), kabs(p[3]) * sth);
  const T beta = kdiv(pm, ksqrt(kfma(pm, pm, T(MPION * MPION))));
  const T t = kdiv(x0, kabs(sth * cdiff));
  const T th0 = kdiv(T(0.0136), beta * pm) * ksqrt(t) * kfma(T(0.038), klog(t), T(1));
  q55 = th0 * th0;
  q44 = kdiv(q55, sth * sth);
}

// Thickness of layer l (radiation lengths at normal incidence) at z: the
// per-layer value, or linear between the material-map nodes and constant
// beyond the ends (the detector's r-z material description, Sec. 3).  slope,
// if given, receives d(thickness)/dz.
template <class T>
__device__ __forceinline__ T x0_at(const DevGeom& g, int l, T z, T* slope = nullptr) {
  if (!g.x0map) {
    if (slope) *slope = T(0);
    return (T)g.x0[l];
  }
  const float* m = g.x0map + (size_t)l * g.n_z;
  const T u = (z + (T)g.z_max) * (T)g.z_node_inv;
  if (!(u > T(0)) || u >= T(g.n_z - 1)) {  // beyond an end (or not a number): the end node
    if (slope) *slope = T(0);
    return (T)m[u >= T(g.n_z - 1) ? g.n_z - 1 : 0];
  }
  const int k = min((int)u, g.n_z - 2);
  const T d = (T)m[k + 1] - (T)m[k];
  if (slope) *slope = d * (T)g.z_node_inv;
  return kfma(u - T(k), d, (T)m[k]);
}

// ---------------------------------------------------------------- energy loss
// Mean ionization loss of a thin layer, applied after its scattering (Sec. 3:
// the material description also serves energy loss), for outward motion:
//   dE = e f / beta^2,  f = 1/|sin(theta) cos(D)|,  D = phi - phi_p (phi_p the
//   position angle: f is the scattering's path factor),  beta = p/E for the
//   pion mass m;  E' = E - min(dE, (E - m)/2),  p' = sqrt(E'^2 - m^2),
//   k' = k p/p' for k = q/pT.
// The covariance follows the map: C' = F C F^T with F the identity but for
// its q/pT row u = dk'/d(x, y, z, k, phi, theta).  From log p = -log|k| -
// log sin(theta), log f = -log sin(theta) - log|cos D| and
//   d log p' = (E'/p'^2) dE' = A d log p + B d log f,
//   A = (E'/p'^2)(E beta^2 + 2 dE (1 - beta^2)),  B = -(E'/p'^2) dE,
// d log k' = A dk/k + (A + B - 1) cot(theta) dtheta - B tan(D) dD with
// dD = dphi - (x dy - y dx)/r^2, so
//   u = k' (-B tan(D) y/r^2, B tan(D) x/r^2, 0, A/k, -B tan(D), (A + B - 1) cot(theta)).
// kval gives the value of a scalar (the cap is a branch on values); the
// function is written for any scalar with the k* functions, so that the
// adjoint can take its derivatives in forward mode (Dir6 below).
__device__ __forceinline__ float kval(float x) { return x; }
__device__ __forceinline__ double kval(double x) { return x; }
// DISK: an endcap disk, whose path factor is f = 1/|cos(theta)| (normal along
// z): d log f = tan(theta) dtheta, so u = k' (0, 0, 0, A/k, 0, (A - 1)
// cot(theta) - B tan(theta)).
template <class T, bool DISK = false, bool ACC = false>
__device__ __forceinline__ void eloss_row(const T (&p)[6], T e, T& k1, T (&u)[6]) {
  T sth, cth, sph, cph;
  ksc<ACC>(p[5], &sth, &cth);
  ksc<ACC>(p[4], &sph, &cph);
  const T r2 = kfma(p[0], p[0], p[1] * p[1]);
  const T ir = krsqrt(r2);
  const T cd = kfma(cph, p[0], sph * p[1]) * ir;     // cos(phi - phi_p)
  const T sd = kfma(sph, p[0], -(cph * p[1])) * ir;  // sin(phi - phi_p)
  const T pm = kdiv(T(1), kabs(p[3]) * sth);
  const T m2 = T(MPION * MPION);
  const T p2 = pm * pm;
  const T E2 = p2 + m2;
  const T E = ksqrt(E2);
  T dE = kdiv(e * E2, p2 * (DISK ? kabs(cth) : kabs(sth * cd)));  // e f / beta^2
  const T cap = T(0.5) * (E - T(MPION));
  if (kval(dE) > kval(cap)) dE = cap;
  // The terms near 1 and 0 are formed without cancellation (at high momentum
  // dE/E is tiny): with x = dE (2E - dE)/p^2, p'^2 = p^2 (1 - x) and
  //   p/p' = (1 - x)^(-1/2),
  //   A - 1 = dE ((p^2 + 4 m^2)/E - dE (1 + 2 m^2/E^2)) / p'^2,
  //   A + B - 1 = dE m^2 (3E - 2 dE) / (E^2 p'^2),
  //   B = -(E - dE) dE / p'^2
  // (identities of the definitions above).
  const T x = kdiv(dE * (T(2) * E - dE), p2);
  const T ratio = krsqrt(T(1) - x);  // p/p'
  k1 = p[3] * ratio;
  const T p1sq = p2 * (T(1) - x);
  const T Am1 = kdiv(dE * (kdiv(p2 + T(4) * m2, E) - dE * (T(1) + kdiv(T(2) * m2, E2))), p1sq);
  const T ApBm1 = kdiv(dE * m2 * (T(3) * E - T(2) * dE), E2 * p1sq);
  const T B = -kdiv((E - dE) * dE, p1sq);
  if constexpr (DISK) {
    u[0] = T(0);
    u[1] = T(0);
    u[2] = T(0);
    u[3] = (T(1) + Am1) * ratio;
    u[4] = T(0);
    u[5] = k1 * (kdiv(cth, sth) * Am1 - B * kdiv(sth, cth));
    (void)ApBm1;
    (void)sd;
    return;
  }
  const T kbt = k1 * B * kdiv(sd, cd);
  const T ir2 = ir * ir;
  u[0] = -(kbt * p[1]) * ir2;
  u[1] = kbt * p[0] * ir2;
  u[2] = T(0);
  u[3] = (T(1) + Am1) * ratio;  // k' A / k
  u[4] = -kbt;
  u[5] = k1 * kdiv(cth, sth) * ApBm1;
}

// Energy loss of a layer with loss e (GeV; 0: none) on the state (p, C).
template <class T, bool DISK = false, bool ACC = false>
__device__ __forceinline__ void add_eloss(T (&p)[6], T (&C)[21], T e) {
  if (!(e > T(0)) || p[3] == T(0)) return;
  T k1, u[6];
  eloss_row<T, DISK, ACC>(p, e, k1, u);
  T cu[6];  // (F C) row 3 = u^T C
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    T a = T(0);
#pragma unroll
    for (int k = 0; k < 6; ++k)
      if (k != 2) a = kfma(u[k], C[S6(k, j)], a);
    cu[j] = a;
  }
  T c33 = T(0);
#pragma unroll
  for (int k = 0; k < 6; ++k)
    if (k != 2) c33 = kfma(cu[k], u[k], c33);
#pragma unroll
  for (int j = 0; j < 6; ++j)
    if (j != 3) C[S6(3, j)] = cu[j];
  C[S6(3, 3)] = c33;
  p[3] = k1;
}

// The same, out of line: a layer without loss costs a comparison; with a loss
// the state goes through a record in local memory, so that the register
// allocation of the caller's usual path does not carry the loss's code.
template <class T>
struct State27 {
  T p[6], C[21];
};
template <class T, bool DISK, bool ACC>
static __device__ __noinline__ void eloss_record(State27<T>* s, T e) { add_eloss<T, DISK, ACC>(s->p, s->C, e); }
template <class T, bool DISK = false, bool ACC = false>
__device__ __forceinline__ void add_eloss_ool(T (&p)[6], T (&C)[21], T e) {
  if (!(e > T(0))) return;
  State27<T> s;
#pragma unroll
  for (int k = 0; k < 6; ++k) s.p[k] = p[k];
#pragma unroll
  for (int k = 0; k < 21; ++k) s.C[k] = C[k];
  eloss_record<T, DISK, ACC>(&s, e);
#pragma unroll
  for (int k = 0; k < 6; ++k) p[k] = s.p[k];
#pragma unroll
  for (int k = 0; k < 21; ++k) C[k] = s.C[k];
}

template <class T, bool ACC = false>
__device__ __forceinline__ void add_ms(const T (&p)[6], T (&C)[21], T x0) {
  if (p[3] == T(0) || x0 <= T(0)) return;
  T sth, cth, sph, cph;
  ksc<ACC>(p[5], &sth, &cth);
  ksc<ACC>(p[4], &sph, &cph);
  const T ir = krsqrt(kfma(p[0], p[0], p[1] * p[1]));
  const T cdiff = kfma(cph, p[0], sph * p[1]) * ir;  // cos(phi - phi_p)
  const T pm = kdiv(T(1), kabs(p[3]) * sth);
  const T beta = kdiv(pm, ksqrt(kfma(pm, pm, T(MPION * MPION))));
  const T t = kdiv(x0, kabs(sth * cdiff));
  const T th0 = kdiv(T(0.0136), beta * pm) * ksqrt(t) * kfma(T(0.038), klog(t), T(1));
  const T v = th0 * th0;
  C[S6(4, 4)] += kdiv(v, sth * sth);
  C[S6(5, 5)] += v;
}

// ---------------------------------------------------------------- endcap disks
// (Sec. 2: the detector's barrel layers and endcap disks.)
__device__ __forceinline__ bool is_disk(const DevGeom& g, int s) { return s >= g.n_layers; }
// z of the plane of disk surface s (+z disks first, then -z).
__device__ __forceinline__ float plane_z(const DevGeom& g, int s) {
  const int k = s - g.n_layers;
  return k < g.n_disks ? g.disk_z[k] : -g.disk_z[k - g.n_disks];
}
// Surface searched at position pos of a seed's plan: barrel layers
// 0..n_layers-1, then disk pos - n_layers of the seed's side.
__device__ __forceinline__ int plan_surface(const DevGeom& g, int pos, bool neg) {
  return pos < g.n_layers ? pos : pos + (neg ? g.n_disks : 0);
}
// Region of a seed (Sec. 2: the event is split into eta regions): a prior
// with |eta| >= eta_barrel (transition and endcap regions) searches its
// side's disks after the barrel layers.  eta in double, as -log tan(theta/2).
__device__ __forceinline__ bool seed_forward(const DevGeom& g, float theta) {
  if (g.n_disks == 0) return false;
  const double eta = -log(tan(0.5 * (double)theta));
  return fabs(eta) >= (double)g.eta_barrel;
}
// The seed's side: eta < 0 (the -z disks).
__device__ __forceinline__ bool seed_eta_negative(float theta) { return -log(tan(0.5 * (double)theta)) < 0.0; }

// Sine and cosine of the polar angle in the disk computations: the plane
// step's length s = (z_d - z) tan(theta) carries the relative error of
// sin(theta), which the hardware approximation (absolute error about 4e-7)
// makes about 2e-6 for the forward tracks that reach the disks (theta of
// 0.1-0.4 rad); the library's sincosf keeps it at a few ulp.
__device__ __forceinline__ void ksincos_polar(float x, float* s, float* c) { sincosf(x, s, c); }
__device__ __forceinline__ void ksincos_polar(double x, double* s, double* c) { sincos(x, s, c); }

// Structure of the Jacobian of the step to a plane z = z_d: rows q/pT and
// theta unit; row z zero (z' = z_d whatever the start); x' has a unit entry
// in x and values in (z, q/pT, phi, theta), y' likewise in y, phi' a unit
// entry in phi and values in (z, q/pT, theta).
__host__ __device__ constexpr int JSP(int i, int j) {
  return (i == 3) ? (j == 3 ? 1 : 0)
         : (i == 5) ? (j == 5 ? 1 : 0)
         : (i == 2) ? 0
         : (i == 0) ? (j == 0 ? 1 : (j == 1 ? 0 : 2))
         : (i == 1) ? (j == 1 ? 1 : (j == 0 ? 0 : 2))
         : (j == 4 ? 1 : ((j == 0 || j == 1) ? 0 : 2));
}

// Propagation to the plane z = zd (an endcap disk): transverse arc s = (zd -
// z) tan(theta), which must be positive (the track moves towards the plane)
// and reach the plane within half a turn (|h s| < pi); the helix in the field
// of curvature factor kb.  J = dq/dp at that field: the partials at fixed s
// plus (dq/ds)(ds/dp) with ds/dz = -tan(theta), ds/dtheta = (zd - z)/cos^2
// theta = s/(sin theta cos theta) and dq/ds = (cos phi', sin phi', cot theta,
// 0, h, 0); the z row vanishes.  Returns false (p untouched) without such a
// crossing.
template <class T, bool ACC = false>
__device__ __forceinline__ bool prop_plane_jacobian(const T (&p)[6], T zd, T kb, T (&q)[6], T (&J)[6][6]) {
  T sth, cth;
  ksincos_polar(p[5], &sth, &cth);
  if (!(kabs(cth) > T(1e-12) * sth)) return false;
  const T s = kdiv((zd - p[2]) * sth, cth);
  if (!(s > T(0))) return false;
  const T h = kb * p[3];
  const T psi = h * s;
  if (!(kabs(psi) < T(3.14159265358979323846))) return false;
  T sf, cf;
  ksc<ACC>(p[4], &sf, &cf);
  T sc, cc, f1, f2;
  helix_fns<T>(psi, sc, cc, f1, f2);
  const T Sx = s * sc, Cx = s * cc;
  const T dx = kfma(cf, Sx, -sf * Cx);
  const T dy = kfma(sf, Sx, cf * Cx);
  const T cpsi = kfma(-psi, cc, T(1)), spsi = psi * sc;
  const T cp = kfma(cf, cpsi, -sf * spsi);
  const T sp = kfma(sf, cpsi, cf * spsi);
  const T s2 = s * s;
  const T dSdh = s2 * f1, dCdh = s2 * f2;
  const T ds2 = -kdiv(sth, cth);
  const T ds5 = kdiv(s, sth * cth);
  J[0][2] = cp * ds2; J[0][3] = kb * kfma(cf, dSdh, -sf * dCdh); J[0][4] = -dy; J[0][5] = cp * ds5;
  J[1][2] = sp * ds2; J[1][3] = kb * kfma(sf, dSdh, cf * dCdh); J[1][4] = dx; J[1][5] = sp * ds5;
  J[4][2] = h * ds2; J[4][3] = kb * s; J[4][5] = h * ds5;
  q[0] = p[0] + dx;
  q[1] = p[1] + dy;
  q[2] = zd;
  q[3] = p[3];
  q[4] = p[4] + psi;
  q[5] = p[5];
  return true;
}

// C <- J C J^T for a plane step's Jacobian (structure JSP): rows 0, 1, 4 one
// at a time as in transport; the z row and column of the result are zero.
template <class T>
__device__ __forceinline__ void transport_plane(const T (&J)[6][6], T (&C)[21]) {
  constexpr int ORD[3] = {0, 1, 4};
  T out[21];
#pragma unroll
  for (int k = 0; k < 6; ++k) out[S6(2, k)] = T(0);
  out[S6(3, 3)] = C[S6(3, 3)];
  out[S6(3, 5)] = C[S6(3, 5)];
  out[S6(5, 5)] = C[S6(5, 5)];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int i = ORD[a];
    T t[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      T acc = T(0);
      bool first = true;
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        if (JSP(i, j) == 0) continue;
        const T c = C[S6(j, k)];
        if (JSP(i, j) == 1) acc = first ? c : acc + c;
        else acc = first ? J[i][j] * c : kfma(J[i][j], c, acc);
        first = false;
      }
      t[k] = acc;
    }
    out[S6(i, 3)] = t[3];
    out[S6(i, 5)] = t[5];
#pragma unroll
    for (int b = a; b < 3; ++b) {
      const int kr = ORD[b];
      T acc = T(0);
      bool first = true;
#pragma unroll
      for (int m = 0; m < 6; ++m) {
        if (JSP(kr, m) == 0) continue;
        if (JSP(kr, m) == 1) acc = first ? t[m] : acc + t[m];
        else acc = first ? t[m] * J[kr][m] : kfma(t[m], J[kr][m], acc);
        first = false;
      }
      out[S6(i, kr)] = acc;
    }
  }
#pragma unroll
  for (int k = 0; k < 21; ++k) C[k] = out[k];
}

// Plane steps along more than PLANE_CAREFUL_PSI rad of the helix (loopers
// that reach a disk after much of a half-turn): the predicted (r-phi, r)
// variance then exceeds the hit's by 10^3-10^4, and the update C - K H C
// cancels as many digits, which FP32 cannot spare; the fit's careful pass
// runs such steps (and the adjoint their reverse) in double.  |psi| below
// 0.5 rad covers 99% of the steps onto disks of the barrel-plus-endcap event.
constexpr float PLANE_CAREFUL_PSI = 0.5f;
__device__ __forceinline__ bool plane_careful(const DevGeom& g, const float (&p)[6], float zd) {
  float sth, cth;
  ksincos_polar(p[5], &sth, &cth);
  const float psi = field_kb<float>(g, p) * p[3] * ((zd - p[2]) * sth / cth);
  return fabsf(psi) > PLANE_CAREFUL_PSI;
}

template <class T, bool ACC = false>
__device__ __forceinline__ bool propagate_plane(T (&p)[6], T (&C)[21], T zd, T kb) {
  T q[6], J[6][6];
  if (!prop_plane_jacobian<T, ACC>(p, zd, kb, q, J)) return false;
  transport_plane<T>(J, C);
#pragma unroll
  for (int k = 0; k < 6; ++k) p[k] = q[k];
  return true;
}

// Measurement on a disk: (r-phi, r) at the prediction, H0 = (-su, cu, 0, ..),
// H1 = (cu, su, 0, ..) with (cu, su) = (x, y)/r; a0 = C H0^T, a1 = C H1^T,
// S = H C H^T + diag(vr, vrr).  The frame's f carries S^-1 (and the window's
// S00, S11) as for a layer.
template <class T>
struct DiskFrameT {
  FrameT<T> f;
  T a1[6];
};
template <class T>
__device__ __forceinline__ void make_frame_disk(const T (&p)[6], const T (&C)[21], T vr, T vrr, DiskFrameT<T>& d) {
  FrameT<T>& f = d.f;
  const T ir = krsqrt(kfma(p[0], p[0], p[1] * p[1]));
  f.cu = p[0] * ir;
  f.su = p[1] * ir;
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    f.a0[i] = kfma(-f.su, C[S6(i, 0)], f.cu * C[S6(i, 1)]);
    d.a1[i] = kfma(f.cu, C[S6(i, 0)], f.su * C[S6(i, 1)]);
  }
  const T s00 = kfma(-f.su, f.a0[0], kfma(f.cu, f.a0[1], vr));
  const T s01 = kfma(f.cu, f.a0[0], f.su * f.a0[1]);
  const T s11 = kfma(f.cu, d.a1[0], kfma(f.su, d.a1[1], vrr));
  const T idet = kdiv(T(1), kfma(s00, s11, -s01 * s01));
  f.s00 = s00;
  f.s11 = s11;
  f.si00 = s11 * idet;
  f.si01 = -s01 * idet;
  f.si11 = s00 * idet;
}
// Residual (r-phi, r) of hit (mx, my) on a disk; false on the far half.
template <class T>
__device__ __forceinline__ bool residual_disk(const T (&p)[6], const FrameT<T>& f, T mx, T my, T& r0, T& r1) {
  if (kfma(mx, p[0], my * p[1]) <= T(0)) return false;
  const T dx = mx - p[0], dy = my - p[1];
  r0 = kfma(-f.su, dx, f.cu * dy);
  r1 = kfma(f.cu, dx, f.su * dy);
  return true;
}
template <class T>
__device__ __forceinline__ void kf_update_disk(T (&p)[6], T (&C)[21], const DiskFrameT<T>& d, T r0, T r1) {
  const FrameT<T>& f = d.f;
  T k0[6], k1[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    k0[i] = kfma(f.a0[i], f.si00, d.a1[i] * f.si01);
    k1[i] = kfma(f.a0[i], f.si01, d.a1[i] * f.si11);
  }
#pragma unroll
  for (int i = 0; i < 6; ++i) p[i] = kfma(k0[i], r0, kfma(k1[i], r1, p[i]));
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int j = i; j < 6; ++j) C[S6(i, j)] -= kfma(k0[i], f.a0[j], k1[i] * d.a1[j]);
}
// Scattering in a disk of x0 radiation lengths: the Highland width with the
// path factor 1/|cos(theta)|.
template <class T>
__device__ __forceinline__ void add_ms_disk(const T (&p)[6], T (&C)[21], T x0) {
  if (p[3] == T(0) || x0 <= T(0)) return;
  T sth, cth;
  ksincos_polar(p[5], &sth, &cth);
  const T pm = kdiv(T(1), kabs(p[3]) * sth);
  const T beta = kdiv(pm, ksqrt(kfma(pm, pm, T(MPION * MPION))));
  const T t = kdiv(x0, kabs(cth));
  const T th0 = kdiv(T(0.0136), beta * pm) * ksqrt(t) * kfma(T(0.038), klog(t), T(1));
  const T v = th0 * th0;
  C[S6(4, 4)] += kdiv(v, sth * sth);
  C[S6(5, 5)] += v;
}

// A seed prior much looser than the hit resolution (a position variance above
// LOOSE_PRIOR times the measurement variance, in r-phi or in z): the first
// updates then shrink the variances by more than the factor (position at the
// first hit, direction and curvature at the next two), and C - K H C cancels
// as many leading digits, which FP32 cannot spare.  The steps over the first
// LOOSE_STEPS hits of such a track run in double (the careful passes of the
// finding and the fit); the first update, at the prior point, through
// first_update_double.
constexpr int LOOSE_STEPS = 3;
constexpr float LOOSE_PRIOR = 1000.f;
__device__ __forceinline__ bool loose_prior(const float (&C)[21], const DevGeom& g) {
  return C[S6(0, 0)] + C[S6(1, 1)] > LOOSE_PRIOR * g.vr || C[S6(2, 2)] > LOOSE_PRIOR * g.vz;
}
// The first update in double: frame, residual, chi2 (added to chi2), update,
// then (if ms) the scattering and energy loss of layer l.  Returns false for a
// hit on the far half (nothing changed).
static __device__ __noinline__ bool first_update_double(float (&pf)[6], float (&Cf)[21], const DevGeom& g, int l,
                                                        float mx, float my, float mz, bool ms, float& chi2) {
  double p[6], C[21];
  for (int k = 0; k < 6; ++k) p[k] = pf[k];
  for (int k = 0; k < 21; ++k) C[k] = Cf[k];
  FrameT<double> f;
  make_frame<double>(p, C, (double)g.vr, (double)g.vz, f);
  double r0, r1;
  if (!residual<double>(p, f, (double)mx, (double)my, (double)mz, r0, r1)) return false;
  chi2 += (float)chi2_of<double>(f, r0, r1);
  kf_update<double>(p, C, f, r0, r1);
  if (ms) {
    add_ms<double>(p, C, x0_at<double>(g, l, p[2]));
    add_eloss<double>(p, C, (double)g.eloss[l]);
  }
  for (int k = 0; k < 6; ++k) pf[k] = (float)p[k];
  for (int k = 0; k < 21; ++k) Cf[k] = (float)C[k];
  return true;
}

// ---------------------------------------------------------------- hit grid
// phi bins: floor((phi + pi) * n_phi / 2pi) (monotone in phi; wrapped mod
// n_phi for hits).  eta bins: 64 equal steps of eta = asinh(z/R) over
// [-asinh(z_max/R), asinh(z_max/R)], realised as a step function of z through
// a per-layer table of bin edges in z (edge[k] = R sinh(eta_k)), so that the
// map is monotone in z and identical for hits and search windows.
__device__ __forceinline__ int phi_bin_raw(float phi, float phi_scale) {
  return (int)floorf((phi + PI_F) * phi_scale);
}
__device__ __forceinline__ int wrap_bin(int b, int n) {
  if (b >= 0 && b < n) return b;
  if (b < 0 && b >= -n) return b + n;
  if (b >= n && b < 2 * n) return b - n;
  b %= n;
  return b < 0 ? b + n : b;
}
__device__ __forceinline__ int eta_bin(float z, int n_eta, float z_max, float lut_scale, const unsigned char* lut,
                                       const float* edges) {
  // First guess: the bin of the lower end of z's cell in a uniform z grid;
  // the edge comparisons below make the result exact whatever the guess.
  const int c = min(max((int)floorf((z + z_max) * lut_scale), 0), ETA_LUT - 1);
  int b = lut[c];
  while (b > 0 && z < __ldg(edges + b)) --b;
  while (b < n_eta - 1 && z >= __ldg(edges + b + 1)) ++b;
  return b;
}

// Row of a disk hit at radius r in its disk's grid: n_eta equal steps of r
// over [disk_rmin, disk_rmax], clamped (monotone in r, identical for hits and
// search windows); r = sqrt(x^2 + y^2) as disk_r computes it.
__device__ __forceinline__ int r_bin(const DevGeom& g, float r) {
  return min(max((int)floorf((r - g.disk_rmin) * g.disk_rscale), 0), g.n_eta - 1);
}
__device__ __forceinline__ float disk_r(float x, float y) { return sqrtf(fmaf(x, x, y * y)); }

// Square root of a non-negative x through the hardware reciprocal square
// root (a few ulp; 0 for x <= 0): for window bounds, which are padded.
__device__ __forceinline__ float sqrt_bound(float x) { return x > 0.f ? x * rsqrtf(x) : 0.f; }

// atan2(y, x) for the centre of a search window: the quotient of the smaller
// by the larger of |x|, |y| through the hardware reciprocal, atan(t) = t P(t^2)
// on [0, 1] with a degree-6 polynomial in t^2 fitted to atan (weighted least
// squares on Chebyshev nodes), then the octant.  Largest error about 1e-6 rad
// (3.3e-7 from the polynomial in FP32, the rest from the quotient and the
// octant offsets); window bounds carry an absolute padding well above it.
__device__ __forceinline__ float atan2_window(float y, float x) {
  const float ax = fabsf(x), ay = fabsf(y);
  const float mx = fmaxf(ax, ay), mn = fminf(ax, ay);
  const float t = mx > 0.f ? __fdividef(mn, mx) : 0.f;
  const float q = t * t;
  float r = fmaf(q, 0.006811764f, -0.03360415f);
  r = fmaf(q, r, 0.07962362f);
  r = fmaf(q, r, -0.13233341f);
  r = fmaf(q, r, 0.19807817f);
  r = fmaf(q, r, -0.3331737f);
  r = fmaf(q, r, 0.99999613f);
  r *= t;
  if (ay > ax) r = 1.57079633f - r;
  if (x < 0.f) r = 3.14159265f - r;
  return copysignf(r, y);
}

// The same eta bin with the layer's edges in shared memory and an arithmetic
// first guess (eta = asinh(z/R) through the hardware logarithm; only a guess:
// the edge comparisons make the result exact), so that a window costs no
// global-memory lookup.
__device__ __forceinline__ int eta_bin_smem(float z, float r_inv, float eta_max, float eta_scale, int n_eta,
                                            const float* edges) {
  const float x = z * r_inv, ax = fabsf(x);
  const float eta = copysignf(__logf(ax + sqrt_bound(fmaf(ax, ax, 1.f))), x);
  int b = (int)floorf((eta + eta_max) * eta_scale);
  b = min(max(b, 0), n_eta - 1);
  while (b > 0 && z < edges[b]) --b;
  while (b < n_eta - 1 && z >= edges[b + 1]) ++b;
  return b;
}

// Ranking key of a candidate child (lower is better): 6 bits 63 - n_found,
// 32 bits chi2 sum (non-negative float bits are monotone), 4 bits parent
// slot, 1 bit non-hit, 21 bits hit index.
constexpr unsigned long long KEY_EMPTY = ~0ull;
__device__ __forceinline__ unsigned long long make_key(int n_found, float chi2, int parent,
                                                       int nonhit, int hit) {
  return ((unsigned long long)(63 - n_found) << 58) |
         ((unsigned long long)__float_as_uint(fmaxf(chi2, 0.f)) << 26) |
         ((unsigned long long)(parent & 15) << 22) | ((unsigned long long)(nonhit & 1) << 21) |
         (unsigned long long)(hit & 0x1FFFFF);
}
__device__ __forceinline__ int key_nfound(unsigned long long k) { return 63 - (int)(k >> 58); }
__device__ __forceinline__ float key_chi2(unsigned long long k) {
  return __uint_as_float((unsigned)((k >> 26) & 0xFFFFFFFFull));
}
__device__ __forceinline__ int key_parent(unsigned long long k) { return (int)((k >> 22) & 15); }
__device__ __forceinline__ int key_nonhit(unsigned long long k) { return (int)((k >> 21) & 1); }
__device__ __forceinline__ int key_hit(unsigned long long k) { return (int)(k & 0x1FFFFF); }

__device__ __forceinline__ void corrected_hit(const Align4& a, float x, float y, float z, float& mx,
                                              float& my, float& mz) {
  mx = fmaf(a.ca, x, -a.sa * y);
  my = fmaf(a.sa, x, a.ca * y);
  mz = z - a.az;
}

}  // namespace kfg
