// Forward-mode dual numbers with N directions, for the few places where the
// adjoint of the fit needs derivatives of a nonlinear function of the state:
// the propagation Jacobian J(p) (its derivative dJ/dp) and the scattering
// variances Q(p).  Branches compare values only.  Plugs into the scalar-generic
// math of kf_common.cuh through overloads of kfma, ksincos, ksqrt, ...
#pragma once

#include "kf_common.cuh"

namespace kfg {

template <class S, int N>
struct Dual {
  S v;
  S d[N];
  __device__ __forceinline__ Dual() {}
  __device__ __forceinline__ Dual(double c) : v((S)c) {  // NOLINT: implicit from constants
#pragma unroll
    for (int i = 0; i < N; ++i) d[i] = S(0);
  }
  // From a value already in S (no round trip through double for S = float).
  __device__ __forceinline__ static Dual of(S c) {
    Dual r;
    r.v = c;
#pragma unroll
    for (int i = 0; i < N; ++i) r.d[i] = S(0);
    return r;
  }
};

template <class S, int N>
__device__ __forceinline__ Dual<S, N> dvar(S x, int k) {
  Dual<S, N> r(0.0);
  r.v = x;
  r.d[k] = S(1);
  return r;
}

#define KF_DUAL_T template <class S, int N> __device__ __forceinline__
KF_DUAL_T Dual<S, N> operator+(const Dual<S, N>& a, const Dual<S, N>& b) {
  Dual<S, N> r; r.v = a.v + b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] + b.d[i];
  return r;
}
KF_DUAL_T Dual<S, N> operator-(const Dual<S, N>& a, const Dual<S, N>& b) {
  Dual<S, N> r; r.v = a.v - b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] - b.d[i];
  return r;
}
KF_DUAL_T Dual<S, N> operator-(const Dual<S, N>& a) {
  Dual<S, N> r; r.v = -a.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = -a.d[i];
  return r;
}
KF_DUAL_T Dual<S, N> operator*(const Dual<S, N>& a, const Dual<S, N>& b) {
  Dual<S, N> r; r.v = a.v * b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = kfma(a.d[i], b.v, a.v * b.d[i]);
  return r;
}
KF_DUAL_T Dual<S, N> operator/(const Dual<S, N>& a, const Dual<S, N>& b) {
  Dual<S, N> r; r.v = a.v / b.v;
  const S ib = S(1) / b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = (a.d[i] - r.v * b.d[i]) * ib;
  return r;
}
KF_DUAL_T Dual<S, N>& operator+=(Dual<S, N>& a, const Dual<S, N>& b) { a = a + b; return a; }
KF_DUAL_T Dual<S, N>& operator-=(Dual<S, N>& a, const Dual<S, N>& b) { a = a - b; return a; }
KF_DUAL_T bool operator<(const Dual<S, N>& a, const Dual<S, N>& b) { return a.v < b.v; }
KF_DUAL_T bool operator>(const Dual<S, N>& a, const Dual<S, N>& b) { return a.v > b.v; }
KF_DUAL_T bool operator<=(const Dual<S, N>& a, const Dual<S, N>& b) { return a.v <= b.v; }
KF_DUAL_T bool operator>=(const Dual<S, N>& a, const Dual<S, N>& b) { return a.v >= b.v; }
KF_DUAL_T bool operator==(const Dual<S, N>& a, const Dual<S, N>& b) { return a.v == b.v; }

KF_DUAL_T Dual<S, N> dchain(const Dual<S, N>& a, S f, S df) {
  Dual<S, N> r; r.v = f;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = df * a.d[i];
  return r;
}
KF_DUAL_T Dual<S, N> kfma(const Dual<S, N>& a, const Dual<S, N>& b, const Dual<S, N>& c) { return a * b + c; }
KF_DUAL_T void ksincos(const Dual<S, N>& x, Dual<S, N>* s, Dual<S, N>* c) {
  S sv, cv;
  ksincos(x.v, &sv, &cv);
  *s = dchain(x, sv, cv);
  *c = dchain(x, cv, -sv);
}
KF_DUAL_T Dual<S, N> ksin(const Dual<S, N>& x) {
  S sv, cv;
  ksincos(x.v, &sv, &cv);
  return dchain(x, sv, cv);
}
KF_DUAL_T Dual<S, N> ksqrt(const Dual<S, N>& x) {
  const S r = ksqrt(x.v);
  return dchain(x, r, S(0.5) / r);
}
KF_DUAL_T Dual<S, N> krsqrt(const Dual<S, N>& x) {
  const S r = S(1) / ksqrt(x.v);
  return dchain(x, r, S(-0.5) * r * r * r);
}
KF_DUAL_T Dual<S, N> katan(const Dual<S, N>& x) { return dchain(x, katan(x.v), S(1) / (S(1) + x.v * x.v)); }
KF_DUAL_T Dual<S, N> klog(const Dual<S, N>& x) { return dchain(x, klog(x.v), S(1) / x.v); }
KF_DUAL_T Dual<S, N> kabs(const Dual<S, N>& x) { return x.v < S(0) ? -x : x; }
KF_DUAL_T Dual<S, N> kmin(const Dual<S, N>& a, const Dual<S, N>& b) { return b.v < a.v ? b : a; }
#undef KF_DUAL_T

}  // namespace kfg
