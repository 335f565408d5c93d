// FP64 CPU oracle of the batched Kalman-filter track finder and fitter.
//
// TEST INFRASTRUCTURE ONLY.  The parity tests, the smoke check and the
// benchmark's CPU-baseline leg call this code; the library's product path
// never does.  It shares no code with the CUDA kernels.
//
// What it computes (the paper gives the method in outline only: Sec. 2 for the
// Kalman filter building, Sec. 3 for the geometry, Sec. 4.2 for duplicate
// removal, Sec. 4.3 for candidate scores; every formula below is the standard
// Kalman-filter reading recorded in the design notes):
//   * state p = (x, y, z, q/pT, phi, theta), symmetric 6x6 covariance C;
//   * barrel layers and endcap disks (Sec. 3), the event's seeds split into
//     eta regions (Sec. 2): barrel seeds search the barrel layers, transition
//     and endcap seeds the barrel layers and then their side's disks; a
//     candidate passes a surface it does not cross within its bounds;
//   * helix propagation to a cylinder of radius R in an axial field Bz, uniform
//     or parameterized (Sec. 3) as Bz(r, z) = bz (1 + cz z^2 + cr r^2) taken at
//     the starting point of each propagation, with the exact Jacobian of the
//     helix J = dF/dp + dF/ds ds/dp at that field;
//   * covariance transport C <- J C J^T;
//   * 2D tangent-frame measurement (r-phi, z) of a 3D hit on the cylinder, chi2;
//     on a disk: propagation to the plane z = z_k, measurement (r-phi, r);
//   * gain K = C H^T S^-1, p <- p + K r, C <- C - K H C;
//   * thin-scatterer multiple scattering after each layer (Highland width);
//   * combinatorial finding with per-seed top-N candidates (Sec. 2);
//   * greedy duplicate removal on shared-hit fraction with optional pT, eta
//     and phi pre-cuts, and seed cleaning before building (both Sec. 4.2);
//   * the full re-fit and the summed chi2, with forward-mode dual numbers for
//     d(chi2)/d(alignment, hits, seed parameters).
// Matrices are full 6x6 arrays and products are plain triple loops: no
// sparsity, blocking or fusion.
//
// Parity status: every function here is pinned by tests under tests/ (closed
// forms, Runge-Kutta integration, finite differences, brute force, least
// squares, pull widths; the parameterized field by tests/test_oracle_field.py,
// the endcap disks and eta regions by tests/test_oracle_endcap.py).  The finding's candidate selection (ranking key,
// truncation to N, hole limit, stop and carry rules, chi2 cut) is pinned by
// hand-made child lists and by a brute-force beam on tiny events that
// recomputes every path through orc_replay.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <numeric>
#include <map>
#include <tuple>
#include <vector>

namespace {

constexpr double KCURV = 0.00299792458;  // 1/rho[1/cm] = KCURV * B[T] / pT[GeV]
constexpr double MPION = 0.13957;        // mass hypothesis for beta (GeV)
constexpr double PI = 3.14159265358979323846;

// ---------------------------------------------------------------- dual numbers
// Forward-mode derivatives: value v plus derivatives d[0..g_nd) with respect to
// g_nd independent inputs.  Branches compare values only.  g_nd is per host
// thread, so that calls on different threads do not interfere.
// DualB<false> (Dual) is double precision.  DualB<true> (Dual32) rounds the
// value and every derivative to single precision after each operation: the
// same computation as single-precision arithmetic would do it (library
// functions rounded from their double values), which measures how far FP32
// rounding alone moves a result.
constexpr int DMAX = 112;
thread_local int g_nd = 0;

template <bool R32>
inline double rnd(double x) { return R32 ? (double)(float)x : x; }

template <bool R32>
struct DualB {
  double v;
  double d[DMAX];
  DualB() : v(0.0) { for (int i = 0; i < g_nd; ++i) d[i] = 0.0; }
  DualB(double x) : v(rnd<R32>(x)) { for (int i = 0; i < g_nd; ++i) d[i] = 0.0; }  // NOLINT implicit
};
using Dual = DualB<false>;
using Dual32 = DualB<true>;
template <bool R = false>
inline DualB<R> make_var(double x, int k) {
  DualB<R> r(x);
  r.d[k] = 1.0;
  return r;
}
inline double val(double x) { return x; }
template <bool R>
inline double val(const DualB<R>& x) { return x.v; }

template <bool R>
inline DualB<R> operator+(const DualB<R>& a, const DualB<R>& b) {
  DualB<R> r; r.v = rnd<R>(a.v + b.v);
  for (int i = 0; i < g_nd; ++i) r.d[i] = rnd<R>(a.d[i] + b.d[i]);
  return r;
}
template <bool R>
inline DualB<R> operator-(const DualB<R>& a, const DualB<R>& b) {
  DualB<R> r; r.v = rnd<R>(a.v - b.v);
  for (int i = 0; i < g_nd; ++i) r.d[i] = rnd<R>(a.d[i] - b.d[i]);
  return r;
}
template <bool R>
inline DualB<R> operator-(const DualB<R>& a) {
  DualB<R> r; r.v = -a.v;
  for (int i = 0; i < g_nd; ++i) r.d[i] = -a.d[i];
  return r;
}
template <bool R>
inline DualB<R> operator*(const DualB<R>& a, const DualB<R>& b) {
  DualB<R> r; r.v = rnd<R>(a.v * b.v);
  for (int i = 0; i < g_nd; ++i) r.d[i] = rnd<R>(rnd<R>(a.d[i] * b.v) + rnd<R>(a.v * b.d[i]));
  return r;
}
template <bool R>
inline DualB<R> operator/(const DualB<R>& a, const DualB<R>& b) {
  DualB<R> r; r.v = rnd<R>(a.v / b.v);
  const double ib = rnd<R>(1.0 / b.v);
  for (int i = 0; i < g_nd; ++i) r.d[i] = rnd<R>(rnd<R>(a.d[i] - rnd<R>(r.v * b.d[i])) * ib);
  return r;
}
template <bool R>
inline DualB<R> operator+(const DualB<R>& a, double b) { DualB<R> r = a; r.v = rnd<R>(r.v + b); return r; }
template <bool R>
inline DualB<R> operator+(double a, const DualB<R>& b) { return b + a; }
template <bool R>
inline DualB<R> operator-(const DualB<R>& a, double b) { DualB<R> r = a; r.v = rnd<R>(r.v - b); return r; }
template <bool R>
inline DualB<R> operator-(double a, const DualB<R>& b) { return (-b) + a; }
template <bool R>
inline DualB<R> operator*(const DualB<R>& a, double b) {
  DualB<R> r; r.v = rnd<R>(a.v * b);
  for (int i = 0; i < g_nd; ++i) r.d[i] = rnd<R>(a.d[i] * b);
  return r;
}
template <bool R>
inline DualB<R> operator*(double a, const DualB<R>& b) { return b * a; }
template <bool R>
inline DualB<R> operator/(const DualB<R>& a, double b) { return a * rnd<R>(1.0 / b); }
template <bool R>
inline DualB<R> operator/(double a, const DualB<R>& b) { return DualB<R>(a) / b; }
template <bool R>
inline DualB<R>& operator+=(DualB<R>& a, const DualB<R>& b) { a = a + b; return a; }
template <bool R>
inline DualB<R>& operator-=(DualB<R>& a, const DualB<R>& b) { a = a - b; return a; }
template <bool R>
inline DualB<R>& operator+=(DualB<R>& a, double b) { a = a + b; return a; }
template <bool R>
inline DualB<R>& operator-=(DualB<R>& a, double b) { a = a - b; return a; }

template <bool R>
inline DualB<R> chain(const DualB<R>& a, double f, double df) {
  DualB<R> r; r.v = rnd<R>(f);
  const double dr = rnd<R>(df);
  for (int i = 0; i < g_nd; ++i) r.d[i] = rnd<R>(dr * a.d[i]);
  return r;
}
template <bool R>
inline DualB<R> sin(const DualB<R>& a) { return chain(a, std::sin(a.v), std::cos(a.v)); }
template <bool R>
inline DualB<R> cos(const DualB<R>& a) { return chain(a, std::cos(a.v), -std::sin(a.v)); }
template <bool R>
inline DualB<R> atan(const DualB<R>& a) { return chain(a, std::atan(a.v), 1.0 / (1.0 + a.v * a.v)); }
template <bool R>
inline DualB<R> sqrt(const DualB<R>& a) { double s = std::sqrt(a.v); return chain(a, s, 0.5 / s); }
template <bool R>
inline DualB<R> log(const DualB<R>& a) { return chain(a, std::log(a.v), 1.0 / a.v); }
template <bool R>
inline DualB<R> fabs(const DualB<R>& a) { return a.v < 0 ? -a : a; }
template <bool R>
inline DualB<R> atan2(const DualB<R>& y, const DualB<R>& x) {
  const double r2 = x.v * x.v + y.v * y.v;
  DualB<R> r; r.v = rnd<R>(std::atan2(y.v, x.v));
  for (int i = 0; i < g_nd; ++i) r.d[i] = rnd<R>((x.v * y.d[i] - y.v * x.d[i]) / r2);
  return r;
}

// ---------------------------------------------------------------- operation census
// A counting scalar: each operation on Cn values is recorded as a node of a
// computation graph.  Trivial operations are not recorded: a product with a
// constant 0 is the constant 0, with a constant 1 (or -1) the other operand
// (or its negation); a sum with a constant 0 the other operand; operations on
// constants fold.  Identical operations on the same operands are one node.
// The operations a set of results needs are the nodes that reach them; sign
// changes and absolute values cost nothing, every other node one operation
// (an add, multiply, divide or special function).  The finding and fitting
// steps run unchanged on Cn through their templates; a symmetric matrix
// result is taken from its upper triangle (see symmetrize).
struct CnNode {
  char op;
  int a, b;
};
thread_local std::vector<CnNode> g_tape;
thread_local std::map<std::tuple<char, int, int>, int> g_cse;

struct Cn {
  double v;
  int id;  // a node of g_tape, or -1 for a constant (exactly v)
  Cn() : v(0.0), id(-1) {}
  Cn(double x) : v(x), id(-1) {}  // NOLINT implicit: a constant
};
inline double val(const Cn& x) { return x.v; }
inline Cn cn_input(double x) {
  g_tape.push_back({'i', -1, -1});
  Cn r(x);
  r.id = (int)g_tape.size() - 1;
  return r;
}
inline Cn cn_node(char op, const Cn& a, const Cn& b, double v, bool commutes) {
  int x = a.id, y = b.id;
  if (commutes && x > y) std::swap(x, y);
  const auto key = std::make_tuple(op, x, y);
  const auto it = g_cse.find(key);
  Cn r(v);
  if (it != g_cse.end()) {
    r.id = it->second;
  } else {
    g_tape.push_back({op, x, y});
    r.id = (int)g_tape.size() - 1;
    g_cse.emplace(key, r.id);
  }
  return r;
}
inline bool cn_is(const Cn& a, double c) { return a.id < 0 && a.v == c; }
inline Cn operator-(const Cn& a) {
  if (a.id < 0) return Cn(-a.v);
  return cn_node('n', a, Cn(), -a.v, false);
}
inline Cn operator+(const Cn& a, const Cn& b) {
  if (a.id < 0 && b.id < 0) return Cn(a.v + b.v);
  if (cn_is(a, 0.0)) return b;
  if (cn_is(b, 0.0)) return a;
  return cn_node('+', a, b, a.v + b.v, true);
}
inline Cn operator-(const Cn& a, const Cn& b) {
  if (a.id < 0 && b.id < 0) return Cn(a.v - b.v);
  if (cn_is(b, 0.0)) return a;
  if (cn_is(a, 0.0)) return -b;
  return cn_node('-', a, b, a.v - b.v, false);
}
inline Cn operator*(const Cn& a, const Cn& b) {
  if (a.id < 0 && b.id < 0) return Cn(a.v * b.v);
  if (cn_is(a, 0.0) || cn_is(b, 0.0)) return Cn(0.0);
  if (cn_is(a, 1.0)) return b;
  if (cn_is(b, 1.0)) return a;
  if (cn_is(a, -1.0)) return -b;
  if (cn_is(b, -1.0)) return -a;
  return cn_node('*', a, b, a.v * b.v, true);
}
inline Cn operator/(const Cn& a, const Cn& b) {
  if (a.id < 0 && b.id < 0) return Cn(a.v / b.v);
  if (cn_is(a, 0.0)) return Cn(0.0);
  if (cn_is(b, 1.0)) return a;
  return cn_node('/', a, b, a.v / b.v, false);
}
inline Cn& operator+=(Cn& a, const Cn& b) { a = a + b; return a; }
inline Cn& operator-=(Cn& a, const Cn& b) { a = a - b; return a; }
inline Cn cn_fn(char op, const Cn& a, double v) { return a.id < 0 ? Cn(v) : cn_node(op, a, Cn(), v, false); }
inline Cn sin(const Cn& a) { return cn_fn('s', a, std::sin(a.v)); }
inline Cn cos(const Cn& a) { return cn_fn('c', a, std::cos(a.v)); }
inline Cn atan(const Cn& a) { return cn_fn('t', a, std::atan(a.v)); }
inline Cn sqrt(const Cn& a) { return cn_fn('q', a, std::sqrt(a.v)); }
inline Cn log(const Cn& a) { return cn_fn('l', a, std::log(a.v)); }
inline Cn fabs(const Cn& a) { return cn_fn('a', a, std::fabs(a.v)); }
inline Cn atan2(const Cn& y, const Cn& x) {
  if (y.id < 0 && x.id < 0) return Cn(std::atan2(y.v, x.v));
  return cn_node('2', y, x, std::atan2(y.v, x.v), false);
}

// Operations needed for the results `outs` (node ids; constants need none):
// counts[0] adds and subtracts, [1] multiplies, [2] divides, [3] special
// functions (sine, cosine, arctangent, square root, logarithm).
void cn_count(const std::vector<int>& outs, long long counts[4]) {
  std::vector<char> seen(g_tape.size(), 0);
  std::vector<int> stack;
  for (int o : outs)
    if (o >= 0) stack.push_back(o);
  for (int k = 0; k < 4; ++k) counts[k] = 0;
  while (!stack.empty()) {
    const int n = stack.back();
    stack.pop_back();
    if (seen[n]) continue;
    seen[n] = 1;
    const CnNode& nd = g_tape[n];
    switch (nd.op) {
      case '+': case '-': counts[0]++; break;
      case '*': counts[1]++; break;
      case '/': counts[2]++; break;
      case 's': case 'c': case 't': case 'q': case 'l': case '2': counts[3]++; break;
      default: break;  // inputs, sign changes, absolute values
    }
    if (nd.a >= 0) stack.push_back(nd.a);
    if (nd.b >= 0) stack.push_back(nd.b);
  }
}

using std::atan;
using std::atan2;
using std::cos;
using std::fabs;
using std::log;
using std::sin;
using std::sqrt;

// ---------------------------------------------------------------- detector
// Axial field (Sec. 3: the field may be constant or parameterized).
// Reading: Bz(r, z) = bz (1 + cz z^2 + cr r^2), r^2 = x^2 + y^2 (cm); each
// propagation is a helix in the field at its starting point.
struct Field {
  double bz, cz, cr;
};

struct Det {
  int n_layers;
  double radius[64];
  double x0[64];
  double z_max;
  double bz;
  double sigma_rphi;
  double sigma_z;
  int n_z;               // material map nodes per layer (0: the per-layer x0)
  const double* x0_map;  // [n_layers][n_z] thickness at z_k = -z_max + k 2 z_max/(n_z - 1)
  double eloss[64];      // mean ionization loss per layer at normal incidence, beta -> 1 (GeV; 0: none)
  double field_cz, field_cr;  // Bz(r, z) = bz (1 + field_cz z^2 + field_cr r^2) (0, 0: uniform)
  // Endcap disks: planes at z = +-disk_z[k], disk_rmin <= r <= disk_rmax.
  // Surfaces: barrel layers 0..L-1, +z disks L..L+D-1, -z disks L+D..L+2D-1.
  int n_disks;
  double disk_z[32];
  double disk_rmin, disk_rmax, disk_x0, disk_eloss, sigma_r;
  double eta_barrel;  // seeds with |eta| >= eta_barrel search their side's disks after the barrel
  Field field() const { return Field{bz, field_cz, field_cr}; }
  int n_surfaces() const { return n_layers + 2 * n_disks; }
  bool is_disk(int s) const { return s >= n_layers; }
  double plane_z(int s) const {
    const int k = s - n_layers;
    return k < n_disks ? disk_z[k] : -disk_z[k - n_disks];
  }
};

struct Cfg {
  int max_cands;
  int max_holes;
  double chi2_cut;
};

inline int sym_index(int i, int j) {  // upper triangle, row-major
  if (i > j) std::swap(i, j);
  return i * 6 - i * (i - 1) / 2 + (j - i);
}

// ---------------------------------------------------------------- helix
// Series-safe helpers of psi = h*s:
//   sinc(psi) = sin(psi)/psi, cosc(psi) = (1-cos psi)/psi,
//   f1(psi) = (psi cos psi - sin psi)/psi^2 = d(sin(hs)/h)/dh / s^2,
//   f2(psi) = (psi sin psi - 1 + cos psi)/psi^2 = d((1-cos hs)/h)/dh / s^2.
template <class T>
void helix_functions(const T& psi, T& sc, T& cc, T& f1, T& f2) {
  if (std::fabs(val(psi)) < 0.1) {
    T p2 = psi * psi;
    sc = 1.0 - p2 / 6.0 + p2 * p2 / 120.0 - p2 * p2 * p2 / 5040.0 + p2 * p2 * p2 * p2 / 362880.0;
    cc = psi * (0.5 - p2 / 24.0 + p2 * p2 / 720.0 - p2 * p2 * p2 / 40320.0 +
                p2 * p2 * p2 * p2 / 3628800.0);
    f1 = psi * (-1.0 / 3.0 + p2 / 30.0 - p2 * p2 / 840.0 + p2 * p2 * p2 / 45360.0);
    f2 = 0.5 - p2 / 8.0 + p2 * p2 / 144.0 - p2 * p2 * p2 / 5760.0 + p2 * p2 * p2 * p2 / 403200.0;
  } else {
    T sn = sin(psi), cs = cos(psi);
    sc = sn / psi;
    cc = (1.0 - cs) / psi;
    f1 = (psi * cs - sn) / (psi * psi);
    f2 = (psi * sn - 1.0 + cs) / (psi * psi);
  }
}

// Path length s > 0 (transverse arc length) to the first crossing of the
// cylinder x^2 + y^2 = R^2.  With psi = h s, b = p_xy . t, a = p_xy . n
// (t the direction, n its left normal) the crossing condition is
//   A sin(psi) + B (1 - cos psi) = E,  A = b h, B = a h + 1, E = h^2 (R^2 - r0^2)/2,
// solved with tau = tan(psi/2):  (2B - E) tau^2 + 2 A tau - E = 0.
// h = 0 is the straight line s^2 + 2 b s - (R^2 - r0^2) = 0.
template <class T>
bool path_to_cylinder(const T& x, const T& y, const T& h, const T& phi, double R, T& s) {
  T cf = cos(phi), sf = sin(phi);
  T b = x * cf + y * sf;
  T a = -x * sf + y * cf;
  T r0 = sqrt(x * x + y * y);
  T dR2 = (R - r0) * (R + r0);
  if (val(h) == 0.0) {
    T disc = b * b + dR2;
    if (val(disc) < 0.0) return false;
    T sq = sqrt(disc);
    // Roots lo = -b - sq <= hi = -b + sq, each in its cancellation-free form.
    T lo, hi;
    if (val(b) > 0.0) {
      lo = -(b + sq);
      hi = dR2 / (b + sq);
    } else {
      hi = sq - b;
      lo = (val(hi) == 0.0) ? T(0.0) : -dR2 / hi;
    }
    if (val(lo) > 0.0) { s = lo; return true; }
    if (val(hi) > 0.0) { s = hi; return true; }
    return false;
  }
  T A = b * h, B = a * h + 1.0, E = 0.5 * h * h * dR2;
  T D = A * A + E * (2.0 * B - E);
  if (val(D) < 0.0) return false;
  T sq = sqrt(D);
  T den = 2.0 * B - E;
  T num[2], dnm[2];
  if (val(A) >= 0.0) {
    num[0] = E; dnm[0] = A + sq;
    num[1] = -(A + sq); dnm[1] = den;
  } else {
    num[0] = sq - A; dnm[0] = den;
    num[1] = E; dnm[1] = A - sq;
  }
  const double turn = 2.0 * PI / std::fabs(val(h));
  bool found = false;
  T best(0.0);
  for (int k = 0; k < 2; ++k) {
    T psi;
    if (val(dnm[k]) == 0.0) {
      if (val(num[k]) == 0.0) continue;
      psi = T(PI);
    } else {
      psi = 2.0 * atan(num[k] / dnm[k]);
    }
    T sk = psi / h;
    if (val(sk) <= 0.0) sk = sk + turn;
    if (!found || val(sk) < val(best)) { best = sk; found = true; }
  }
  if (!found) return false;
  s = best;
  return true;
}

// kb = -KCURV Bz at the point (x, y, z): the curvature per unit q/pT.
template <class T>
T field_kb(const Field& f, const T& x, const T& y, const T& z) {
  const double kb0 = -KCURV * f.bz;
  if (f.cz == 0.0 && f.cr == 0.0) return T(kb0);
  return kb0 * (1.0 + f.cz * (z * z) + f.cr * (x * x + y * y));
}

// Propagate p to the cylinder of radius R; q = F(p).  J = dq/dp with the
// field held at its value (the exact Jacobian of a helix; with a uniform
// field that of F itself).  The field's dependence on the starting point
// enters q (and so every derivative taken through the fit) but not J.
template <class T>
bool propagate(const Field& fld, const T p[6], double R, T q[6], T J[6][6]) {
  const T& x = p[0];
  const T& y = p[1];
  const T& z = p[2];
  const T& kap = p[3];
  const T& phi = p[4];
  const T& th = p[5];
  const T kb = field_kb(fld, x, y, z);
  T h = kb * kap;
  T s;
  if (!path_to_cylinder(x, y, h, phi, R, s)) return false;
  T psi = h * s;
  T sc, cc, f1, f2;
  helix_functions(psi, sc, cc, f1, f2);
  T cf = cos(phi), sf = sin(phi);
  T Sx = s * sc, Cx = s * cc;
  T cot = cos(th) / sin(th);
  q[0] = x + cf * Sx - sf * Cx;
  q[1] = y + sf * Sx + cf * Cx;
  q[2] = z + s * cot;
  q[3] = kap;
  q[4] = phi + psi;
  q[5] = th;
  // Partial derivatives at fixed s.
  T F[6][6];
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) F[i][j] = T(i == j ? 1.0 : 0.0);
  T dSdh = s * s * f1, dCdh = s * s * f2;
  F[0][3] = kb * (cf * dSdh - sf * dCdh);
  F[0][4] = -(q[1] - y);
  F[1][3] = kb * (sf * dSdh + cf * dCdh);
  F[1][4] = q[0] - x;
  T sth = sin(th);
  F[2][5] = -s / (sth * sth);
  F[4][3] = kb * s;
  // Implicit path length: g(p, s) = x'^2 + y'^2 - R^2 = 0.
  T cp = cos(q[4]), sp = sin(q[4]);
  T dgds = q[0] * cp + q[1] * sp;
  T dsdp[6];
  for (int j = 0; j < 6; ++j) dsdp[j] = -(q[0] * F[0][j] + q[1] * F[1][j]) / dgds;
  T dqds[6] = {cp, sp, cot, T(0.0), h, T(0.0)};
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) J[i][j] = F[i][j] + dqds[i] * dsdp[j];
  return true;
}

// Propagate p to the plane z = zd (an endcap disk): the transverse arc
// s = (zd - z) tan(theta) > 0 (the track must move towards the plane, and
// reach it within half a turn, |h s| < pi), the helix there in the field at
// the starting point; q[2] = zd.  J = dq/dp at
// that field: the partials at fixed s plus dq/ds ds/dp with ds/dz = -tan(theta),
// ds/dtheta = (zd - z)/cos^2(theta) (so the z row of J vanishes).
template <class T>
bool propagate_plane(const Field& fld, const T p[6], double zd, T q[6], T J[6][6]) {
  const T& x = p[0];
  const T& y = p[1];
  const T& z = p[2];
  const T& kap = p[3];
  const T& phi = p[4];
  const T& th = p[5];
  const T cot = cos(th) / sin(th);
  if (std::fabs(val(cot)) < 1e-12) return false;
  const T s = (zd - z) / cot;
  if (!(val(s) > 0.0)) return false;
  const T kb = field_kb(fld, x, y, z);
  const T h = kb * kap;
  const T psi = h * s;
  // within half a turn: a looper that would reach the plane after more turns
  // would meet the barrel layers again first, which the finding does not follow
  if (!(std::fabs(val(psi)) < M_PI)) return false;
  T sc, cc, f1, f2;
  helix_functions(psi, sc, cc, f1, f2);
  const T cf = cos(phi), sf = sin(phi);
  const T Sx = s * sc, Cx = s * cc;
  q[0] = x + cf * Sx - sf * Cx;
  q[1] = y + sf * Sx + cf * Cx;
  q[2] = z + s * cot;  // zd (its derivatives vanish)
  q[3] = kap;
  q[4] = phi + psi;
  q[5] = th;
  T F[6][6];
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) F[i][j] = T(i == j ? 1.0 : 0.0);
  const T dSdh = s * s * f1, dCdh = s * s * f2;
  F[0][3] = kb * (cf * dSdh - sf * dCdh);
  F[0][4] = -(q[1] - y);
  F[1][3] = kb * (sf * dSdh + cf * dCdh);
  F[1][4] = q[0] - x;
  const T sth = sin(th), cth = cos(th);
  F[2][5] = -s / (sth * sth);
  F[4][3] = kb * s;
  T dsdp[6] = {T(0.0), T(0.0), -1.0 / cot, T(0.0), T(0.0), (zd - z) / (cth * cth)};
  const T cp = cos(q[4]), sp = sin(q[4]);
  T dqds[6] = {cp, sp, cot, T(0.0), h, T(0.0)};
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) J[i][j] = F[i][j] + dqds[i] * dsdp[j];
  return true;
}

// C <- (out + out^T) / 2.  For the operation census a symmetric result is
// computed once: C takes the upper triangle of out (no operation).
template <class T>
void symmetrize(const T out[6][6], T C[6][6]) {
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) C[i][j] = 0.5 * (out[i][j] + out[j][i]);
}
inline void symmetrize(const Cn out[6][6], Cn C[6][6]) {
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) C[i][j] = i <= j ? out[i][j] : out[j][i];
}

template <class T>
void transport(const T J[6][6], T C[6][6]) {  // C <- J C J^T
  T JC[6][6], out[6][6];
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) {
      T acc(0.0);
      for (int k = 0; k < 6; ++k) acc += J[i][k] * C[k][j];
      JC[i][j] = acc;
    }
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) {
      T acc(0.0);
      for (int k = 0; k < 6; ++k) acc += JC[i][k] * J[j][k];
      out[i][j] = acc;
    }
  symmetrize(out, C);
}

// ---------------------------------------------------------------- measurement
// Hit m (alignment-corrected) against prediction p: r = (u.(m_xy - p_xy), m_z - z)
// with u = (-sin phi_p, cos phi_p), phi_p = atan2(y, x).  Hits on the far half
// of the cylinder (m_xy . p_xy <= 0) are incompatible.
template <class T>
struct Meas {
  T r[2];
  T H[2][6];
  T S[2][2];
  T Sinv[2][2];
  T chi2;
};

// On an endcap disk (disk = true) the second coordinate is radial:
// r = (u.(m_xy - p_xy), w.(m_xy - p_xy)) with w = (cos phi_p, sin phi_p), and
// vz is the radial variance.
template <class T>
bool measure(const T p[6], const T C[6][6], const T m[3], double vr, double vz, Meas<T>& o,
             bool disk = false) {
  if (val(m[0]) * val(p[0]) + val(m[1]) * val(p[1]) <= 0.0) return false;
  T phip = atan2(p[1], p[0]);
  T su = sin(phip), cu = cos(phip);
  o.r[0] = -su * (m[0] - p[0]) + cu * (m[1] - p[1]);
  o.r[1] = disk ? cu * (m[0] - p[0]) + su * (m[1] - p[1]) : m[2] - p[2];
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 6; ++j) o.H[i][j] = T(0.0);
  o.H[0][0] = -su;
  o.H[0][1] = cu;
  if (disk) {
    o.H[1][0] = cu;
    o.H[1][1] = su;
  } else {
    o.H[1][2] = T(1.0);
  }
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) {
      T acc(0.0);
      for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) acc += o.H[a][i] * C[i][j] * o.H[b][j];
      o.S[a][b] = acc;
    }
  o.S[0][0] += vr;
  o.S[1][1] += vz;
  T det = o.S[0][0] * o.S[1][1] - o.S[0][1] * o.S[1][0];
  o.Sinv[0][0] = o.S[1][1] / det;
  o.Sinv[1][1] = o.S[0][0] / det;
  o.Sinv[0][1] = -o.S[0][1] / det;
  o.Sinv[1][0] = -o.S[1][0] / det;
  o.chi2 = T(0.0);
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) o.chi2 += o.r[a] * o.Sinv[a][b] * o.r[b];
  return true;
}

template <class T>
void kf_update(T p[6], T C[6][6], const Meas<T>& m) {
  T CHt[6][2], K[6][2], HC[2][6];
  for (int i = 0; i < 6; ++i)
    for (int a = 0; a < 2; ++a) {
      T acc(0.0);
      for (int j = 0; j < 6; ++j) acc += C[i][j] * m.H[a][j];
      CHt[i][a] = acc;
    }
  for (int i = 0; i < 6; ++i)
    for (int a = 0; a < 2; ++a) K[i][a] = CHt[i][0] * m.Sinv[0][a] + CHt[i][1] * m.Sinv[1][a];
  for (int a = 0; a < 2; ++a)
    for (int j = 0; j < 6; ++j) {
      T acc(0.0);
      for (int i = 0; i < 6; ++i) acc += m.H[a][i] * C[i][j];
      HC[a][j] = acc;
    }
  for (int i = 0; i < 6; ++i) p[i] += K[i][0] * m.r[0] + K[i][1] * m.r[1];
  T out[6][6];
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) out[i][j] = C[i][j] - (K[i][0] * HC[0][j] + K[i][1] * HC[1][j]);
  symmetrize(out, C);
}

// Multiple scattering in a thin layer of x0 radiation lengths at the current
// position: Highland width theta0 = 0.0136/(beta p) sqrt(t) (1 + 0.038 ln t),
// t = x0 / |sin(theta) cos(phi - phi_p)|, p = pT/sin(theta), pion mass for beta.
// On an endcap disk (normal along z) t = x0 / |cos(theta)|.
template <class T>
T highland(const T p[6], T x0, bool disk = false) {
  T st = sin(p[5]);
  T pm = 1.0 / (fabs(p[3]) * st);
  T beta = pm / sqrt(pm * pm + MPION * MPION);
  T t;
  if (disk) {
    t = x0 / fabs(cos(p[5]));
  } else {
    T phip = atan2(p[1], p[0]);
    t = x0 / fabs(st * cos(p[4] - phip));
  }
  return 0.0136 / (beta * pm) * sqrt(t) * (1.0 + 0.038 * log(t));
}

template <class T>
void add_ms(const T p[6], T C[6][6], T x0, bool disk = false) {
  if (val(p[3]) == 0.0 || val(x0) <= 0.0) return;
  T th0 = highland(p, x0, disk);
  T st = sin(p[5]);
  T v = th0 * th0;
  C[4][4] += v / (st * st);
  C[5][5] += v;
}

// Thickness of layer L (radiation lengths at normal incidence) at z: the
// per-layer value, or with a material map (the detector's two-dimensional
// material description, Sec. 3: radiation lengths indexed in r and z, here
// per barrel layer and z node) linear between the nodes and constant beyond
// the ends.  The node is chosen from the value of z; the interpolation
// weight carries its derivative.
template <class T>
T x0_at(const Det& det, int L, const T& z) {
  if (det.n_z < 2) return T(det.x0[L]);
  const double h = 2.0 * det.z_max / (det.n_z - 1);
  const double* m = det.x0_map + (size_t)L * det.n_z;
  const double u = (val(z) + det.z_max) / h;
  if (u <= 0.0) return T(m[0]);
  if (u >= det.n_z - 1) return T(m[det.n_z - 1]);
  int k = (int)std::floor(u);
  if (k > det.n_z - 2) k = det.n_z - 2;
  const T f = (z + det.z_max) / h - (double)k;
  return m[k] + f * (m[k + 1] - m[k]);
}

// Mean ionization energy loss in a thin layer (the paper's material arrays
// serve scattering and energy loss, Sec. 3), outward motion:
//   dE = e f / beta^2,  f = 1/|sin(theta) cos(phi - phi_p)| (the scattering's path
//   factor), e = the layer's loss at normal incidence for beta -> 1 (leading
//   Bethe-Bloch dependence; logarithmic rise and density effect left out);
//   E' = E - dE (dE at most (E - m)/2),  p' = sqrt(E'^2 - m^2),  q/pT' = q/pT p/p'.
// The covariance follows the map: C' = F C F^T, F the identity but for the
// q/pT row dk'/dp (written out below; pinned against finite differences).
// Straggling is not modelled.
// On an endcap disk the path factor is f = 1/|cos(theta)|, so that
// d log f = tan(theta) d theta and q/pT' depends on neither position nor phi.
template <class T>
void add_eloss(T p[6], T C[6][6], double e, bool disk = false) {
  if (e <= 0.0 || val(p[3]) == 0.0) return;
  const T st = sin(p[5]), ct = cos(p[5]);
  const T pm = 1.0 / (fabs(p[3]) * st);
  const T E = sqrt(pm * pm + MPION * MPION);
  const T b2 = pm * pm / (E * E);
  const T phip = atan2(p[1], p[0]);
  const T cd = cos(p[4] - phip), sd = sin(p[4] - phip);
  const T f = disk ? 1.0 / fabs(ct) : 1.0 / fabs(st * cd);
  T dE = e * f / b2;
  if (val(dE) > 0.5 * (val(E) - MPION)) dE = 0.5 * (E - MPION);
  const T E1 = E - dE;
  const T pm1 = sqrt(E1 * E1 - MPION * MPION);
  const T k1 = p[3] * pm / pm1;
  // d log p' = A d log p + B d log f (dE from the formula; a capped dE is
  // treated the same way, a limit no test reaches)
  const T A = E1 / (pm1 * pm1) * (E * b2 - 2.0 * dE * (b2 - 1.0));
  const T B = -(E1 / (pm1 * pm1)) * dE;
  const T r2 = p[0] * p[0] + p[1] * p[1];
  const T tn = sd / cd;
  T F3[6];
  F3[0] = k1 * B * tn * (-p[1] / r2);
  F3[1] = k1 * B * tn * (p[0] / r2);
  F3[2] = T(0.0);
  F3[3] = k1 * A / p[3];
  F3[4] = -k1 * B * tn;
  F3[5] = k1 * (ct / st) * (A + B - 1.0);
  if (disk) {
    F3[0] = F3[1] = F3[4] = T(0.0);
    F3[5] = k1 * ((ct / st) * (A - 1.0) - B * (st / ct));
  }
  // C' = F C F^T with F = I except row 3
  T c3[6];  // row 3 of F C
  for (int j = 0; j < 6; ++j) {
    T a = T(0.0);
    for (int k = 0; k < 6; ++k) a = a + F3[k] * C[k][j];
    c3[j] = a;
  }
  T c33 = T(0.0);
  for (int k = 0; k < 6; ++k) c33 = c33 + c3[k] * F3[k];
  for (int j = 0; j < 6; ++j) {
    C[3][j] = c3[j];
    C[j][3] = c3[j];
  }
  C[3][3] = c33;
  p[3] = k1;
}

// Alignment correction of a raw hit on layer L: rotate by -a_rphi/R_L about z,
// then z -= a_z.
template <class T>
void correct_hit(const T raw[3], const T& a_rphi, const T& a_z, double R, T m[3]) {
  T ang = -a_rphi / R;
  T ca = cos(ang), sa = sin(ang);
  m[0] = ca * raw[0] - sa * raw[1];
  m[1] = sa * raw[0] + ca * raw[1];
  m[2] = raw[2] - a_z;
}

// Kalman fit over hits (raw positions, per-hit layer), from prior (p0, C0)
// placed at the first hit: no propagation before the first update, MS after
// each update except (optionally) the last.  Returns 0 or a negative status.
template <class T, class TC>
int fit_track(const Det& det, const T p0[6], const TC C0[6][6], int n, const T (*raw)[3],
              const int* layers, const T (*align)[2], bool ms_after_last, T p[6], T C[6][6],
              T& chi2, T* chi2_each = nullptr) {
  for (int i = 0; i < 6; ++i) {
    p[i] = p0[i];
    for (int j = 0; j < 6; ++j) C[i][j] = T(C0[i][j]);
  }
  chi2 = T(0.0);
  const double vr = det.sigma_rphi * det.sigma_rphi, vz = det.sigma_z * det.sigma_z;
  const double vrr = det.sigma_r * det.sigma_r;
  for (int k = 0; k < n; ++k) {
    const int L = layers[k];
    const bool disk = det.is_disk(L);  // an endcap disk: plane, radial coordinate, no alignment
    const double R = disk ? 0.0 : det.radius[L];
    if (k > 0) {
      T q[6], J[6][6];
      if (disk ? !propagate_plane(det.field(), p, det.plane_z(L), q, J) : !propagate(det.field(), p, R, q, J))
        return -1;
      for (int i = 0; i < 6; ++i) p[i] = q[i];
      transport(J, C);
    }
    T m[3];
    if (disk) {
      for (int i = 0; i < 3; ++i) m[i] = raw[k][i];
    } else {
      correct_hit(raw[k], align[L][0], align[L][1], R, m);
    }
    Meas<T> ms;
    if (!measure(p, C, m, vr, disk ? vrr : vz, ms, disk)) return -2;
    chi2 += ms.chi2;
    if (chi2_each) chi2_each[k] = ms.chi2;
    kf_update(p, C, ms);
    if (k + 1 < n || ms_after_last) {
      if (disk) {
        add_ms(p, C, T(det.disk_x0), true);
        add_eloss(p, C, det.disk_eloss, true);
      } else {
        add_ms(p, C, x0_at(det, L, p[2]));
        add_eloss(p, C, det.eloss[L]);
      }
    }
  }
  return 0;
}

// ---------------------------------------------------------------- finding
struct Cand {
  double p[6];
  double C[6][6];
  int n_found;
  int n_holes;
  double chi2;
  bool finished;
  std::vector<int> hits;
};

enum Kind { KIND_HIT = 0, KIND_HOLE = 1, KIND_CARRIED = 2 };

struct Child {
  int n_found;
  double chi2;
  int parent;
  int kind;
  int hit;
  int tag;  // not part of the key: carried through the selection unchanged
};

// Ranking key of the candidate score: more hits first, then lower chi2 sum,
// then parent rank, then hit before hole, then lower hit index.
bool child_less(const Child& a, const Child& b) {
  if (a.n_found != b.n_found) return a.n_found > b.n_found;
  if (a.chi2 != b.chi2) return a.chi2 < b.chi2;
  if (a.parent != b.parent) return a.parent < b.parent;
  if (a.kind != b.kind) return a.kind < b.kind;
  return a.hit < b.hit;
}

// The selection step of the finding: the children of all candidates of a
// seed on one layer ranked by child_less, the best max_cands kept in rank
// order (the new candidate slots).  Keys are unique: children of one parent
// differ in kind or hit, children of different parents in parent rank.
std::vector<Child> select_children(std::vector<Child> children, int max_cands) {
  std::sort(children.begin(), children.end(), child_less);
  if (children.size() > (size_t)max_cands) children.resize((size_t)max_cands);
  return children;
}

struct LayerIndex {  // hits of one layer sorted by z (exact chi2 pre-selection)
  std::vector<int> idx;
  std::vector<double> z;
};

struct Counters {
  long long steps;        // candidate propagated, transported and tested on a layer
  long long prop_calls;   // propagations attempted
  long long updates;      // kept hit-children updated
  long long ms;           // multiple-scattering applications
  long long chi2_evals;   // hits whose chi2 was evaluated
  long long seeds;
  long long children;     // children ranked
  long long holes;        // kept hole children (scattering without an update)
  long long window_hits;  // hits inside the bounding box of the chi2 < cut ellipse of the
                          // prediction (|r_rphi| and |r_z| within sqrt(cut S) each): the
                          // method's search window, implementation-independent
  long long disk_steps;   // the steps among `steps` onto endcap disks
  long long disk_updates;  // the updates among `updates` on endcap disks
  long long disk_holes;    // the holes among `holes` on endcap disks
  long long disk_window_hits;  // the window hits among `window_hits` on endcap disks
};

void seed_state(const double* params, const double* cov, long stride, long i, double p[6],
                double C[6][6]) {
  for (int k = 0; k < 6; ++k) p[k] = params[k * stride + i];
  for (int a = 0; a < 6; ++a)
    for (int b = 0; b < 6; ++b) C[a][b] = cov[sym_index(a, b) * stride + i];
}

void find_seed(const Det& det, const Cfg& cfg, const double* hx, const double* hy, const double* hz,
               const int* hlayer, const std::vector<LayerIndex>& lidx, bool brute, int n_hits,
               const double p0[6], const double C0[6][6], const int sh[3], const double (*align)[2],
               int* out_hits, int* out_n, double* out_chi2, double* out_p, double* out_C,
               Counters& cnt) {
  const int L = det.n_layers;
  const double vr = det.sigma_rphi * det.sigma_rphi, vz = det.sigma_z * det.sigma_z;
  Cand c0;
  {
    double raw[3][3];
    int lays[3];
    for (int k = 0; k < 3; ++k) {
      raw[k][0] = hx[sh[k]]; raw[k][1] = hy[sh[k]]; raw[k][2] = hz[sh[k]];
      lays[k] = hlayer[sh[k]];
    }
    double chi2;
    int st = fit_track<double, double>(det, p0, C0, 3, raw, lays, align, true, c0.p, c0.C, chi2);
    c0.n_found = 3;
    c0.n_holes = 0;
    c0.chi2 = chi2;
    c0.finished = st != 0;
    c0.hits = {sh[0], sh[1], sh[2]};
    if (st == 0) cnt.ms += 3;
  }
  std::vector<Cand> cands{c0};
  const int start = hlayer[sh[2]] + 1;
  // The surfaces the seed's candidates search (Sec. 2: the event is split into
  // eta regions, each with its layers): the barrel layers after the seed, and
  // for a seed in a forward region (|eta| >= eta_barrel; transition and endcap
  // regions alike) then the endcap disks of its side in order of |z|.
  std::vector<int> plan;
  for (int l = start; l < L; ++l) plan.push_back(l);
  const double eta0 = -std::log(std::tan(0.5 * p0[5]));
  const bool fwd = det.n_disks > 0 && std::fabs(eta0) >= det.eta_barrel;
  if (fwd)
    for (int k = 0; k < det.n_disks; ++k) plan.push_back(L + k + (eta0 < 0.0 ? det.n_disks : 0));
  const double vrr = det.sigma_r * det.sigma_r;
  for (const int Lyr : plan) {
    const bool disk = det.is_disk(Lyr);
    const double R = disk ? 0.0 : det.radius[Lyr];
    const double v2 = disk ? vrr : vz;
    std::vector<Child> children;
    std::vector<Cand> predicted(cands.size());
    for (size_t r = 0; r < cands.size(); ++r) {
      const Cand& c = cands[r];
      if (c.finished) {
        children.push_back({c.n_found, c.chi2, (int)r, KIND_CARRIED, -1, 0});
        continue;
      }
      Cand& pc = predicted[r];
      pc = c;
      double J[6][6];
      ++cnt.prop_calls;
      bool crossed;
      if (!disk) {
        crossed = propagate(det.field(), c.p, R, pc.p, J) && std::fabs(pc.p[2]) <= det.z_max;
      } else {
        crossed = propagate_plane(det.field(), c.p, det.plane_z(Lyr), pc.p, J);
        const double rr = crossed ? std::hypot(pc.p[0], pc.p[1]) : 0.0;
        crossed = crossed && rr >= det.disk_rmin && rr <= det.disk_rmax;
      }
      if (!crossed) {
        // a barrel-only plan: the candidate has left the detector (it is
        // carried, finished); a forward plan: it passes this surface unchanged
        // (tag 1: carried, not finished, no hole) and meets the next
        children.push_back({c.n_found, c.chi2, (int)r, KIND_CARRIED, -1, fwd ? 1 : 0});
        continue;
      }
      transport(J, pc.C);
      ++cnt.steps;
      if (disk) ++cnt.disk_steps;
      int n_children = 0;
      // Window on z: chi2 >= r_z^2 / S_zz for a 2x2 positive-definite S, so
      // hits with |m_z - z| > sqrt(cut * S_zz) cannot pass the cut.  A disk's
      // hits are all tested.
      const double szz = pc.C[2][2] + vz;
      double lo_z = -1e300, hi_z = 1e300;
      if (!brute && !disk) {
        // corrected z = raw z - a_z, so the raw-z interval is shifted by a_z
        const double w = std::sqrt(cfg.chi2_cut * szz) + 1e-9;
        lo_z = pc.p[2] + align[Lyr][1] - w;
        hi_z = pc.p[2] + align[Lyr][1] + w;
      }
      const LayerIndex& li = lidx[Lyr];
      size_t b = disk ? 0 : std::lower_bound(li.z.begin(), li.z.end(), lo_z) - li.z.begin();
      for (size_t k = b; k < li.idx.size() && (disk || li.z[k] <= hi_z); ++k) {
        const int hidx = li.idx[k];
        double raw[3] = {hx[hidx], hy[hidx], hz[hidx]}, m[3];
        if (disk) {
          for (int i = 0; i < 3; ++i) m[i] = raw[i];
        } else {
          correct_hit(raw, align[Lyr][0], align[Lyr][1], R, m);
        }
        Meas<double> ms;
        ++cnt.chi2_evals;
        if (!measure(pc.p, pc.C, m, vr, v2, ms, disk)) continue;
        if (std::fabs(ms.r[0]) < std::sqrt(cfg.chi2_cut * ms.S[0][0]) &&
            std::fabs(ms.r[1]) < std::sqrt(cfg.chi2_cut * ms.S[1][1])) {
          ++cnt.window_hits;
          if (disk) ++cnt.disk_window_hits;
        }
        if (ms.chi2 < cfg.chi2_cut) {
          children.push_back({c.n_found + 1, c.chi2 + ms.chi2, (int)r, KIND_HIT, hidx, 0});
          ++n_children;
        }
      }
      if (c.n_holes < cfg.max_holes) {
        children.push_back({c.n_found, c.chi2, (int)r, KIND_HOLE, -1, 0});
        ++n_children;
      }
      if (n_children == 0) {  // no compatible hit and no hole left: the candidate stops
        children.push_back({c.n_found, c.chi2, (int)r, KIND_CARRIED, -1, 0});
      }
    }
    cnt.children += (long long)children.size();
    children = select_children(std::move(children), cfg.max_cands);
    const size_t keep = children.size();
    std::vector<Cand> next;
    next.reserve(keep);
    for (size_t k = 0; k < keep; ++k) {
      const Child& ch = children[k];
      if (ch.kind == KIND_CARRIED) {
        Cand c = cands[ch.parent];
        if (ch.tag == 0) c.finished = true;  // tag 1: passed a surface, still searching
        next.push_back(c);
        continue;
      }
      Cand c = predicted[ch.parent];
      if (ch.kind == KIND_HIT) {
        double raw[3] = {hx[ch.hit], hy[ch.hit], hz[ch.hit]}, m[3];
        if (disk) {
          for (int i = 0; i < 3; ++i) m[i] = raw[i];
        } else {
          correct_hit(raw, align[Lyr][0], align[Lyr][1], R, m);
        }
        Meas<double> ms;
        measure(c.p, c.C, m, vr, v2, ms, disk);
        kf_update(c.p, c.C, ms);
        c.n_found += 1;
        c.chi2 = ch.chi2;
        c.hits.push_back(ch.hit);
        ++cnt.updates;
        if (disk) ++cnt.disk_updates;
      } else {
        c.n_holes += 1;
        ++cnt.holes;
        if (disk) ++cnt.disk_holes;
      }
      if (disk) {
        add_ms(c.p, c.C, det.disk_x0, true);
        add_eloss(c.p, c.C, det.disk_eloss, true);
      } else {
        add_ms(c.p, c.C, x0_at(det, Lyr, c.p[2]));
        add_eloss(c.p, c.C, det.eloss[Lyr]);
      }
      ++cnt.ms;
      next.push_back(c);
    }
    cands.swap(next);
  }
  const Cand& best = cands[0];
  const int S = det.n_surfaces();
  for (int k = 0; k < S; ++k) out_hits[k] = k < (int)best.hits.size() ? best.hits[k] : -1;
  *out_n = (int)best.hits.size();
  *out_chi2 = best.chi2;
  for (int k = 0; k < 6; ++k) out_p[k] = best.p[k];
  for (int a = 0; a < 6; ++a)
    for (int b = a; b < 6; ++b) out_C[sym_index(a, b)] = best.C[a][b];
  ++cnt.seeds;
  (void)n_hits;
}

}  // namespace

// ====================================================================== C API
// Kinematic quantities of a track state (Sec. 4.2 names pT, eta and phi as
// the criteria of seed cleaning and duplicate removal):
//   k[0] = eta = -ln tan(theta/2);
//   k[1] = |q/pT|;
//   k[2] = phi0, the transverse direction of motion at the point of the helix
//          closest to the z axis.  The track circle has centre
//          c = (x - sin(phi)/h, y + cos(phi)/h) and radius 1/|h|; its point
//          closest to the axis is c - c/(|c| |h|), where the direction of
//          motion is perpendicular to c: sign(h) (c_y, -c_x)/|c|.  A straight
//          track (h = 0) keeps its direction.
void kinematics_of(double bz, const double* p, double* k) {
  const double h = -KCURV * bz * p[3];
  k[0] = -std::log(std::tan(0.5 * p[5]));
  k[1] = std::fabs(p[3]);
  if (h == 0.0) {
    k[2] = std::atan2(std::sin(p[4]), std::cos(p[4]));
    return;
  }
  const double cx = p[0] - std::sin(p[4]) / h;
  const double cy = p[1] + std::cos(p[4]) / h;
  const double n = std::sqrt(cx * cx + cy * cy);
  const double sg = h > 0.0 ? 1.0 : -1.0;
  k[2] = std::atan2(-sg * cx / n, sg * cy / n);
}

// Kinematic closeness of two tracks: |d eta| < deta, |d phi0| < dphi (the
// difference taken on the circle) and ||k_a| - |k_b|| <= dpt max(|k_a|, |k_b|)
// (the relative pT difference); a cut <= 0 is not applied.
bool kin_close(const double* a, const double* b, double deta, double dphi, double dpt) {
  if (deta > 0.0 && !(std::fabs(a[0] - b[0]) < deta)) return false;
  if (dphi > 0.0) {
    double d = std::fabs(a[2] - b[2]);
    if (d > PI) d = 2.0 * PI - d;
    if (!(d < dphi)) return false;
  }
  if (dpt > 0.0 && !(std::fabs(a[1] - b[1]) <= dpt * std::max(a[1], b[1]))) return false;
  return true;
}

extern "C" {

struct orc_detector {
  int n_layers;
  double radius[64];
  double x0[64];
  double z_max;
  double bz;
  double sigma_rphi;
  double sigma_z;
  int n_z;               // material map nodes per layer (0: none)
  const double* x0_map;  // [n_layers][n_z]
  double eloss[64];      // mean ionization loss per layer (GeV; 0: none)
  double field_cz, field_cr;  // Bz(r, z) = bz (1 + field_cz z^2 + field_cr r^2)
  int n_disks;                // endcap disks per side (see Det)
  double disk_z[32];
  double disk_rmin, disk_rmax, disk_x0, disk_eloss, sigma_r, eta_barrel;
};

struct orc_config {
  int max_cands;
  int max_holes;
  double chi2_cut;
};

static Det to_det(const orc_detector* d) {
  Det o;
  o.n_layers = d->n_layers;
  for (int i = 0; i < 64; ++i) { o.radius[i] = d->radius[i]; o.x0[i] = d->x0[i]; }
  o.z_max = d->z_max;
  o.bz = d->bz;
  o.sigma_rphi = d->sigma_rphi;
  o.sigma_z = d->sigma_z;
  o.n_z = d->x0_map ? d->n_z : 0;
  o.x0_map = d->x0_map;
  for (int i = 0; i < 64; ++i) o.eloss[i] = d->eloss[i];
  o.field_cz = d->field_cz;
  o.field_cr = d->field_cr;
  o.n_disks = d->n_disks;
  for (int i = 0; i < 32; ++i) o.disk_z[i] = d->disk_z[i];
  o.disk_rmin = d->disk_rmin;
  o.disk_rmax = d->disk_rmax;
  o.disk_x0 = d->disk_x0;
  o.disk_eloss = d->disk_eloss;
  o.sigma_r = d->sigma_r;
  o.eta_barrel = d->eta_barrel;
  return o;
}

// Propagation of one state to radius R.  J is row-major 6x6.  Returns 1 if a
// crossing exists, 0 otherwise.
int orc_propagate(double bz, double cz, double cr, const double* p, double R, double* q, double* J) {
  double Jm[6][6];
  if (!propagate<double>(Field{bz, cz, cr}, p, R, q, Jm)) return 0;
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) J[i * 6 + j] = Jm[i][j];
  return 1;
}

// Path length to the crossing (pins of the closed form).
int orc_path_length(double bz, const double* p, double R, double* s) {
  return path_to_cylinder<double>(p[0], p[1], -KCURV * bz * p[3], p[4], R, *s) ? 1 : 0;
}

// Jacobian of the propagated state by forward-mode differentiation of the
// propagation itself (independent of the hand-derived J; with a field that
// varies, it includes the field's dependence on the starting point).
int orc_propagate_ad(double bz, double cz, double cr, const double* p, double R, double* Jad) {
  g_nd = 6;
  Dual pd[6], qd[6], Jd[6][6];
  for (int k = 0; k < 6; ++k) pd[k] = make_var(p[k], k);
  const bool ok = propagate<Dual>(Field{bz, cz, cr}, pd, R, qd, Jd);
  if (ok)
    for (int i = 0; i < 6; ++i)
      for (int j = 0; j < 6; ++j) Jad[i * 6 + j] = qd[i].d[j];
  g_nd = 0;
  return ok ? 1 : 0;
}

// C_out = J C J^T for full row-major 6x6 matrices.
void orc_transport(const double* J, const double* C, double* C_out) {
  double Jm[6][6], Cm[6][6];
  for (int i = 0; i < 36; ++i) { Jm[i / 6][i % 6] = J[i]; Cm[i / 6][i % 6] = C[i]; }
  transport(Jm, Cm);
  for (int i = 0; i < 36; ++i) C_out[i] = Cm[i / 6][i % 6];
}

// One measurement + update at the current state.  Returns 0 if the hit is on
// the far side, 1 otherwise.
// Propagation to the plane z = zd (an endcap disk), J row-major 6x6; and its
// Jacobian by forward-mode differentiation of the whole map.
int orc_propagate_plane(double bz, double cz, double cr, const double* p, double zd, double* q, double* J) {
  double Jm[6][6];
  if (!propagate_plane<double>(Field{bz, cz, cr}, p, zd, q, Jm)) return 0;
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) J[i * 6 + j] = Jm[i][j];
  return 1;
}

int orc_propagate_plane_ad(double bz, double cz, double cr, const double* p, double zd, double* Jad) {
  g_nd = 6;
  Dual pd[6], qd[6], Jd[6][6];
  for (int k = 0; k < 6; ++k) pd[k] = make_var(p[k], k);
  const bool ok = propagate_plane<Dual>(Field{bz, cz, cr}, pd, zd, qd, Jd);
  if (ok)
    for (int i = 0; i < 6; ++i)
      for (int j = 0; j < 6; ++j) Jad[i * 6 + j] = qd[i].d[j];
  g_nd = 0;
  return ok ? 1 : 0;
}

// One Kalman update on an endcap disk (radial second coordinate, variance vrr).
int orc_update_disk(const double* p, const double* C, const double* m, double vr, double vrr,
                    double* p_out, double* C_out, double* chi2, double* resid) {
  double pp[6], Cm[6][6];
  for (int i = 0; i < 6; ++i) pp[i] = p[i];
  for (int i = 0; i < 36; ++i) Cm[i / 6][i % 6] = C[i];
  Meas<double> ms;
  if (!measure(pp, Cm, m, vr, vrr, ms, true)) return 0;
  kf_update(pp, Cm, ms);
  for (int i = 0; i < 6; ++i) p_out[i] = pp[i];
  for (int i = 0; i < 36; ++i) C_out[i] = Cm[i / 6][i % 6];
  *chi2 = ms.chi2;
  if (resid) { resid[0] = ms.r[0]; resid[1] = ms.r[1]; }
  return 1;
}

// Energy loss step on a disk (path factor 1/|cos theta|): p [6], C [36] in place.
void orc_eloss_disk(double* p, double* C, double e) {
  double Cm[6][6];
  for (int i = 0; i < 36; ++i) Cm[i / 6][i % 6] = C[i];
  add_eloss(p, Cm, e, true);
  for (int i = 0; i < 36; ++i) C[i] = Cm[i / 6][i % 6];
}

double orc_highland_disk(const double* p, double x0) { return highland<double>(p, x0, true); }

int orc_update(const double* p, const double* C, const double* m, double vr, double vz,
               double* p_out, double* C_out, double* chi2, double* resid) {
  double pp[6], Cm[6][6];
  for (int i = 0; i < 6; ++i) pp[i] = p[i];
  for (int i = 0; i < 36; ++i) Cm[i / 6][i % 6] = C[i];
  Meas<double> ms;
  if (!measure(pp, Cm, m, vr, vz, ms)) return 0;
  kf_update(pp, Cm, ms);
  for (int i = 0; i < 6; ++i) p_out[i] = pp[i];
  for (int i = 0; i < 36; ++i) C_out[i] = Cm[i / 6][i % 6];
  *chi2 = ms.chi2;
  if (resid) { resid[0] = ms.r[0]; resid[1] = ms.r[1]; }
  return 1;
}

double orc_highland(const double* p, double x0) { return highland<double>(p, x0); }

// Energy loss step on one state (see add_eloss): p [6] and C [36] in place.
void orc_eloss(double* p, double* C, double e) {
  double Cm[6][6];
  for (int i = 0; i < 36; ++i) Cm[i / 6][i % 6] = C[i];
  add_eloss(p, Cm, e);
  for (int i = 0; i < 36; ++i) C[i] = Cm[i / 6][i % 6];
}

// Thickness of layer L at z (see x0_at).
double orc_x0_at(const orc_detector* dptr, int L, double z) { return x0_at(to_det(dptr), L, z); }

void orc_add_ms(const double* p, double* C, double x0) {
  double Cm[6][6];
  for (int i = 0; i < 36; ++i) Cm[i / 6][i % 6] = C[i];
  add_ms(p, Cm, x0);
  for (int i = 0; i < 36; ++i) C[i] = Cm[i / 6][i % 6];
}

// Kalman fit of n_tracks tracks.  prior_p [6][stride], prior_C [21][stride]
// (structure of arrays, seeds index t), hit_lists [n_tracks][max_len] of
// indices into hx/hy/hz/hlayer, n_hits [n_tracks], align [n_layers][2].
// Outputs: p_out [n][6], C_out [n][21], chi2 [n], chi2_each [n][max_len]
// (optional), status [n].
int orc_fit(const orc_detector* dptr, int n_tracks, const double* prior_p, const double* prior_C,
            long stride, const int* hit_lists, const int* n_hits, int max_len, const double* hx,
            const double* hy, const double* hz, const int* hlayer, const double* align,
            int ms_after_last, double* p_out, double* C_out, double* chi2, double* chi2_each,
            int* status) {
  const Det det = to_det(dptr);
  double al[64][2];
  for (int i = 0; i < det.n_layers; ++i) { al[i][0] = align[2 * i]; al[i][1] = align[2 * i + 1]; }
  std::vector<double> raw(3 * (size_t)max_len);
  std::vector<int> lays(max_len);
  for (int t = 0; t < n_tracks; ++t) {
    double p0[6], C0[6][6], p[6], C[6][6], c2;
    seed_state(prior_p, prior_C, stride, t, p0, C0);
    const int n = n_hits[t];
    for (int k = 0; k < n; ++k) {
      const int hidx = hit_lists[(size_t)t * max_len + k];
      raw[3 * k] = hx[hidx]; raw[3 * k + 1] = hy[hidx]; raw[3 * k + 2] = hz[hidx];
      lays[k] = hlayer[hidx];
    }
    status[t] = fit_track<double, double>(det, p0, C0, n, reinterpret_cast<const double(*)[3]>(raw.data()),
                                  lays.data(), al, ms_after_last != 0, p, C, c2,
                                  chi2_each ? chi2_each + (size_t)t * max_len : nullptr);
    for (int k = 0; k < 6; ++k) p_out[6 * t + k] = p[k];
    for (int a = 0; a < 6; ++a)
      for (int b = a; b < 6; ++b) C_out[21 * (size_t)t + sym_index(a, b)] = C[a][b];
    chi2[t] = c2;
  }
  return 0;
}

// Summed chi2 of the fits and its gradient by forward-mode dual numbers:
// g_align [n_layers][2], g_hits [n_hit_arrays][3] (accumulated over tracks
// sharing a hit), g_seed [n_tracks][6].
}  // extern "C"

// The summed fit chi2 and its gradient, forward mode (D = Dual, or Dual32 for
// the same computation with single-precision rounding after every operation).
template <class D>
int fit_grad_impl(const orc_detector* dptr, int n_tracks, const double* prior_p,
                 const double* prior_C, long stride, const int* hit_lists, const int* n_hits,
                 int max_len, const double* hx, const double* hy, const double* hz,
                 const int* hlayer, const double* align, double* chi2_total, double* g_align,
                 double* g_hits, double* g_seed, double* chi2_each) {
  const Det det = to_det(dptr);
  const int L = det.n_layers;
  double total = 0.0;
  for (int t = 0; t < n_tracks; ++t) {
    const int n = n_hits[t];
    g_nd = 6 + 3 * n + 2 * L;
    if (g_nd > DMAX) { g_nd = 0; return -1; }
    D p0[6];
    double C0[6][6], p0v[6];
    seed_state(prior_p, prior_C, stride, t, p0v, C0);
    for (int k = 0; k < 6; ++k) p0[k] = D(p0v[k]), p0[k].d[k] = 1.0;
    std::vector<D> rawv(3 * (size_t)n);
    std::vector<int> lays(n);
    for (int k = 0; k < n; ++k) {
      const int hidx = hit_lists[(size_t)t * max_len + k];
      rawv[3 * k] = D(hx[hidx]), rawv[3 * k].d[6 + 3 * k] = 1.0;
      rawv[3 * k + 1] = D(hy[hidx]), rawv[3 * k + 1].d[6 + 3 * k + 1] = 1.0;
      rawv[3 * k + 2] = D(hz[hidx]), rawv[3 * k + 2].d[6 + 3 * k + 2] = 1.0;
      lays[k] = hlayer[hidx];
    }
    std::vector<D> alv(2 * (size_t)L);
    for (int i = 0; i < L; ++i) {
      alv[2 * i] = D(align[2 * i]), alv[2 * i].d[6 + 3 * n + 2 * i] = 1.0;
      alv[2 * i + 1] = D(align[2 * i + 1]), alv[2 * i + 1].d[6 + 3 * n + 2 * i + 1] = 1.0;
    }
    D p[6], C[6][6], c2;
    const int st = fit_track<D, double>(det, p0, C0, n, reinterpret_cast<const D(*)[3]>(rawv.data()),
                                lays.data(), reinterpret_cast<const D(*)[2]>(alv.data()),
                                false, p, C, c2);
    if (st != 0) { g_nd = 0; return -2 - t; }
    total += c2.v;
    if (chi2_each) chi2_each[t] = c2.v;
    for (int k = 0; k < 6; ++k) g_seed[6 * (size_t)t + k] = c2.d[k];
    for (int k = 0; k < n; ++k) {
      const int hidx = hit_lists[(size_t)t * max_len + k];
      for (int c = 0; c < 3; ++c) g_hits[3 * (size_t)hidx + c] += c2.d[6 + 3 * k + c];
    }
    for (int i = 0; i < 2 * L; ++i) g_align[i] += c2.d[6 + 3 * n + i];
  }
  *chi2_total = total;
  g_nd = 0;
  return 0;
}

extern "C" {

int orc_fit_grad(const orc_detector* dptr, int n_tracks, const double* prior_p,
                 const double* prior_C, long stride, const int* hit_lists, const int* n_hits,
                 int max_len, const double* hx, const double* hy, const double* hz,
                 const int* hlayer, const double* align, double* chi2_total, double* g_align,
                 double* g_hits, double* g_seed, double* chi2_each) {
  return fit_grad_impl<Dual>(dptr, n_tracks, prior_p, prior_C, stride, hit_lists, n_hits, max_len, hx, hy, hz,
                             hlayer, align, chi2_total, g_align, g_hits, g_seed, chi2_each);
}

// The same gradient with every operation rounded to single precision (the
// inputs too): the FP32 rounding scale of each gradient component.
int orc_fit_grad32(const orc_detector* dptr, int n_tracks, const double* prior_p,
                   const double* prior_C, long stride, const int* hit_lists, const int* n_hits,
                   int max_len, const double* hx, const double* hy, const double* hz,
                   const int* hlayer, const double* align, double* chi2_total, double* g_align,
                   double* g_hits, double* g_seed, double* chi2_each) {
  return fit_grad_impl<Dual32>(dptr, n_tracks, prior_p, prior_C, stride, hit_lists, n_hits, max_len, hx, hy,
                               hz, hlayer, align, chi2_total, g_align, g_hits, g_seed, chi2_each);
}

// Combinatorial finding for seeds [s_begin, s_end) of one event.  Hits are
// the event's arrays (event-local indices); seeds are structure-of-arrays with
// the given stride; seed_hits [3][stride].  out_hits [n][surfaces] (padded -1),
// out_p [n][6], out_C [n][21].  counters [13]: see Counters.  brute != 0 tests every
// hit of the layer instead of the exact z pre-selection.
int orc_find_event(const orc_detector* dptr, const orc_config* cfgp, int n_hits, const double* hx,
                   const double* hy, const double* hz, const int* hlayer, const double* params,
                   const double* cov, const int* seed_hits, long stride, int s_begin, int s_end,
                   const double* align, int brute, int* out_hits, int* out_n, double* out_chi2,
                   double* out_p, double* out_C, long long* counters) {
  const Det det = to_det(dptr);
  Cfg cfg{cfgp->max_cands, cfgp->max_holes, cfgp->chi2_cut};
  const int L = det.n_layers, S = det.n_surfaces();
  double al[64][2];
  for (int i = 0; i < L; ++i) { al[i][0] = align[2 * i]; al[i][1] = align[2 * i + 1]; }
  std::vector<LayerIndex> lidx(S);
  for (int h = 0; h < n_hits; ++h)
    if (hlayer[h] >= 0 && hlayer[h] < S) lidx[hlayer[h]].idx.push_back(h);
  for (int l = 0; l < S; ++l) {
    LayerIndex& li = lidx[l];
    if (!brute)
      std::stable_sort(li.idx.begin(), li.idx.end(), [&](int a, int b) { return hz[a] < hz[b]; });
    for (int h : li.idx) li.z.push_back(brute ? 0.0 : (double)hz[h]);
  }
  Counters cnt{};
  for (int s = s_begin; s < s_end; ++s) {
    double p0[6], C0[6][6];
    seed_state(params, cov, stride, s, p0, C0);
    const int sh[3] = {seed_hits[0 * stride + s], seed_hits[1 * stride + s],
                       seed_hits[2 * stride + s]};
    const int o = s - s_begin;
    find_seed(det, cfg, hx, hy, hz, hlayer, lidx, brute != 0, n_hits, p0, C0, sh, al,
              out_hits + (size_t)o * S, out_n + o, out_chi2 + o, out_p + 6 * (size_t)o,
              out_C + 21 * (size_t)o, cnt);
  }
  if (counters) {
    counters[0] += cnt.steps; counters[1] += cnt.prop_calls; counters[2] += cnt.updates;
    counters[3] += cnt.ms; counters[4] += cnt.chi2_evals; counters[5] += cnt.seeds;
    counters[6] += cnt.children; counters[7] += cnt.holes; counters[8] += cnt.window_hits;
    counters[9] += cnt.disk_steps; counters[10] += cnt.disk_updates; counters[11] += cnt.disk_holes;
    counters[12] += cnt.disk_window_hits;
  }
  return 0;
}

// Operation census of one finding step (see Cn): a candidate (p [6], C [21])
// propagated to layer L, two hits m1, m2 [3] (raw positions, corrected by the
// alignment align [2] of L as in the finding) tested, the first kept and
// updated, then the layer's scattering (and energy loss).  out[4 k + c] holds
// (adds, multiplies, divides, special functions) for
//   k = 0: propagation and covariance transport (results: the predicted state
//          and the upper triangle of its covariance);
//   k = 1: the measurement frame and the z window of the pre-selection (the
//          hit-independent part of a chi2 test);
//   k = 2: one hit's chi2 (alignment correction, residual, quadratic form);
//   k = 3: the Kalman update of a kept hit-child;
//   k = 4: the scattering applied to a kept child.
// Alignment, state and hits are inputs of the count.  Returns 0, -1 without a
// crossing of L, -2 for a far-side hit.
int orc_census_step(const orc_detector* dptr, double chi2_cut, const double* p, const double* C21, int L,
                    const double* m1, const double* m2, const double* align, long long* out) {
  const Det det = to_det(dptr);
  g_tape.clear();
  g_cse.clear();
  Cn pc[6], Cc[6][6], q[6], J[6][6];
  for (int k = 0; k < 6; ++k) pc[k] = cn_input(p[k]);
  for (int a = 0; a < 6; ++a)
    for (int b = a; b < 6; ++b) Cc[a][b] = Cc[b][a] = cn_input(C21[sym_index(a, b)]);
  const Cn al0 = cn_input(align[0]), al1 = cn_input(align[1]);
  const double R = det.radius[L];
  if (!propagate(det.field(), pc, R, q, J)) return -1;
  transport(J, Cc);
  std::vector<int> outs;
  for (int k = 0; k < 6; ++k) outs.push_back(q[k].id);
  for (int a = 0; a < 6; ++a)
    for (int b = a; b < 6; ++b) outs.push_back(Cc[a][b].id);
  long long c0[4], c1[4], c2[4], c3[4], c4[4];
  cn_count(outs, c0);
  // the z window of the chi2 pre-selection, as the finding forms it
  const double vr = det.sigma_rphi * det.sigma_rphi, vz = det.sigma_z * det.sigma_z;
  const Cn w = sqrt(chi2_cut * (Cc[2][2] + vz)) + 1e-9;
  const Cn lo = q[2] + al1 - w, hi = q[2] + al1 + w;
  outs.push_back(lo.id);
  outs.push_back(hi.id);
  Cn r1[3], r2[3], mm1[3], mm2[3];
  for (int k = 0; k < 3; ++k) r1[k] = cn_input(m1[k]), r2[k] = cn_input(m2[k]);
  correct_hit(r1, al0, al1, R, mm1);
  correct_hit(r2, al0, al1, R, mm2);
  Meas<Cn> ms1, ms2;
  if (!measure(q, Cc, mm1, vr, vz, ms1) || !measure(q, Cc, mm2, vr, vz, ms2)) return -2;
  outs.push_back(ms1.chi2.id);
  cn_count(outs, c1);
  outs.push_back(ms2.chi2.id);
  cn_count(outs, c2);
  Cn pu[6], Cu[6][6];
  for (int k = 0; k < 6; ++k) pu[k] = q[k];
  for (int a = 0; a < 6; ++a)
    for (int b = 0; b < 6; ++b) Cu[a][b] = Cc[a][b];
  kf_update(pu, Cu, ms1);
  const size_t n_before = outs.size();
  for (int k = 0; k < 6; ++k) outs.push_back(pu[k].id);
  for (int a = 0; a < 6; ++a)
    for (int b = a; b < 6; ++b) outs.push_back(Cu[a][b].id);
  cn_count(outs, c3);
  add_ms(pu, Cu, x0_at(det, L, pu[2]));
  add_eloss(pu, Cu, det.eloss[L]);
  outs.resize(n_before);
  for (int k = 0; k < 6; ++k) outs.push_back(pu[k].id);
  for (int a = 0; a < 6; ++a)
    for (int b = a; b < 6; ++b) outs.push_back(Cu[a][b].id);
  cn_count(outs, c4);
  for (int c = 0; c < 4; ++c) {
    const long long hit = c2[c] - c1[c];
    out[0 + c] = c0[c];
    out[4 + c] = c1[c] - c0[c] - hit;
    out[8 + c] = hit;
    out[12 + c] = c3[c] - c2[c];
    out[16 + c] = c4[c] - c3[c];
  }
  g_tape.clear();
  g_cse.clear();
  return 0;
}

// Operation census of one finding step onto endcap disk surface S (as
// orc_census_step): the plane step and transport; the frame and the bounds
// of the r window of the chi2 < cut ellipse (r_p -+ sqrt(cut S_rr), the
// disk's analogue of the z window) with the first hit's chi2; one more hit's
// chi2; the update; the disk's scattering and energy loss.  out [5][4].
int orc_census_disk_step(const orc_detector* dptr, double chi2_cut, const double* p, const double* C21, int S,
                         const double* m1, const double* m2, long long* out) {
  const Det det = to_det(dptr);
  if (!det.is_disk(S)) return -3;
  g_tape.clear();
  g_cse.clear();
  Cn pc[6], Cc[6][6], q[6], J[6][6];
  for (int k = 0; k < 6; ++k) pc[k] = cn_input(p[k]);
  for (int a = 0; a < 6; ++a)
    for (int b = a; b < 6; ++b) Cc[a][b] = Cc[b][a] = cn_input(C21[sym_index(a, b)]);
  if (!propagate_plane(det.field(), pc, det.plane_z(S), q, J)) return -1;
  transport(J, Cc);
  std::vector<int> outs;
  for (int k = 0; k < 6; ++k) outs.push_back(q[k].id);
  for (int a = 0; a < 6; ++a)
    for (int b = a; b < 6; ++b) outs.push_back(Cc[a][b].id);
  long long c0[4], c1[4], c2[4], c3[4], c4[4];
  cn_count(outs, c0);
  const double vr = det.sigma_rphi * det.sigma_rphi, vrr = det.sigma_r * det.sigma_r;
  Cn mm1[3], mm2[3];
  for (int k = 0; k < 3; ++k) mm1[k] = cn_input(m1[k]), mm2[k] = cn_input(m2[k]);
  Meas<Cn> ms1, ms2;
  if (!measure(q, Cc, mm1, vr, vrr, ms1, true) || !measure(q, Cc, mm2, vr, vrr, ms2, true)) return -2;
  const Cn rp = sqrt(q[0] * q[0] + q[1] * q[1]);
  const Cn w = sqrt(chi2_cut * ms1.S[1][1]);
  const Cn lo = rp - w, hi = rp + w;
  outs.push_back(lo.id);
  outs.push_back(hi.id);
  outs.push_back(ms1.chi2.id);
  cn_count(outs, c1);
  outs.push_back(ms2.chi2.id);
  cn_count(outs, c2);
  Cn pu[6], Cu[6][6];
  for (int k = 0; k < 6; ++k) pu[k] = q[k];
  for (int a = 0; a < 6; ++a)
    for (int b = 0; b < 6; ++b) Cu[a][b] = Cc[a][b];
  kf_update(pu, Cu, ms1);
  const size_t n_before = outs.size();
  for (int k = 0; k < 6; ++k) outs.push_back(pu[k].id);
  for (int a = 0; a < 6; ++a)
    for (int b = a; b < 6; ++b) outs.push_back(Cu[a][b].id);
  cn_count(outs, c3);
  add_ms(pu, Cu, Cn(det.disk_x0), true);
  add_eloss(pu, Cu, det.disk_eloss, true);
  outs.resize(n_before);
  for (int k = 0; k < 6; ++k) outs.push_back(pu[k].id);
  for (int a = 0; a < 6; ++a)
    for (int b = a; b < 6; ++b) outs.push_back(Cu[a][b].id);
  cn_count(outs, c4);
  for (int c = 0; c < 4; ++c) {
    const long long hit = c2[c] - c1[c];
    out[0 + c] = c0[c];
    out[4 + c] = c1[c] - c0[c] - hit;
    out[8 + c] = hit;
    out[12 + c] = c3[c] - c2[c];
    out[16 + c] = c4[c] - c3[c];
  }
  g_tape.clear();
  g_cse.clear();
  return 0;
}

// Operation census of one covariance transport C <- J C J^T (the upper
// triangle of the result): entries of J equal to exactly 0 or 1 are constants,
// the others and C [21] inputs.  out4 as for orc_census_step.
int orc_census_transport(const double* J36, const double* C21, long long* out4) {
  g_tape.clear();
  g_cse.clear();
  Cn J[6][6], C[6][6];
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) {
      const double v = J36[6 * i + j];
      J[i][j] = (v == 0.0 || v == 1.0) ? Cn(v) : cn_input(v);
    }
  for (int a = 0; a < 6; ++a)
    for (int b = a; b < 6; ++b) C[a][b] = C[b][a] = cn_input(C21[sym_index(a, b)]);
  transport(J, C);
  std::vector<int> outs;
  for (int a = 0; a < 6; ++a)
    for (int b = a; b < 6; ++b) outs.push_back(C[a][b].id);
  cn_count(outs, out4);
  g_tape.clear();
  g_cse.clear();
  return 0;
}

// Operation census of a Kalman fit (as orc_fit, scattering after the last hit
// if ms_after_last) over n hits raw [n][3] on layers [n], from the prior (p0
// [6], C0 [21]) with the layers' alignment align [n_layers][2]; prior, hits and
// alignment are inputs of the count.  out4: (adds, multiplies, divides,
// special functions) of the final state, its covariance (upper triangle) and
// the chi2 sum.  Returns the fit's status.
int orc_census_fit(const orc_detector* dptr, const double* p0, const double* C21, int n, const double* raw,
                   const int* layers, const double* align, int ms_after_last, long long* out4) {
  const Det det = to_det(dptr);
  g_tape.clear();
  g_cse.clear();
  Cn pc[6], C0[6][6], p[6], C[6][6], chi2;
  for (int k = 0; k < 6; ++k) pc[k] = cn_input(p0[k]);
  for (int a = 0; a < 6; ++a)
    for (int b = a; b < 6; ++b) C0[a][b] = C0[b][a] = cn_input(C21[sym_index(a, b)]);
  std::vector<Cn> rv(3 * (size_t)n), av(2 * (size_t)det.n_layers);
  for (int k = 0; k < 3 * n; ++k) rv[k] = cn_input(raw[k]);
  for (int k = 0; k < 2 * det.n_layers; ++k) av[k] = cn_input(align[k]);
  const int st = fit_track<Cn, Cn>(det, pc, C0, n, reinterpret_cast<const Cn(*)[3]>(rv.data()), layers,
                                   reinterpret_cast<const Cn(*)[2]>(av.data()), ms_after_last != 0, p, C, chi2);
  std::vector<int> outs;
  for (int k = 0; k < 6; ++k) outs.push_back(p[k].id);
  for (int a = 0; a < 6; ++a)
    for (int b = a; b < 6; ++b) outs.push_back(C[a][b].id);
  outs.push_back(chi2.id);
  cn_count(outs, out4);
  g_tape.clear();
  g_cse.clear();
  return st;
}

// The selection step alone, for hand-made children (n of them, fields as in
// Child; kind 0 hit, 1 hole, 2 carried): writes the indices of the kept
// children in rank order to out_idx and returns how many were kept.
int orc_select_children(int n, const int* n_found, const double* chi2, const int* parent, const int* kind,
                        const int* hit, int max_cands, int* out_idx) {
  std::vector<Child> ch(n);
  for (int i = 0; i < n; ++i) {
    ch[i] = Child{n_found[i], chi2[i], parent[i], kind[i], hit[i], i};
  }
  const std::vector<Child> kept = select_children(ch, max_cands);
  for (size_t k = 0; k < kept.size(); ++k) out_idx[k] = kept[k].tag;
  return (int)kept.size();
}

// Replay one candidate path of the finding: seed fit over the three seed
// hits (scattering after the last), then for each layer from the one after
// the third seed hit: decisions[l] = hit index (update), -1 (hole) or -2
// (stop).  Scattering follows every update and every hole, as in finding.
// chi2_layer[l] receives each hit's chi2; p_out [6] and C_out [21] (may be
// NULL) the state at the end of the path.  Returns 0, or -1 when the
// propagation finds no crossing, -2 for a far-side hit.
int orc_replay(const orc_detector* dptr, const double* hx, const double* hy, const double* hz,
               const int* hlayer, const double* p0v, const double* C0v, const int* sh,
               const int* decisions, const double* align, double* chi2_layer, double* chi2sum,
               int* n_found, double* p_out, double* C_out) {
  const Det det = to_det(dptr);
  const int L = det.n_layers;
  double al[64][2];
  for (int i = 0; i < L; ++i) { al[i][0] = align[2 * i]; al[i][1] = align[2 * i + 1]; }
  double p0[6], C0[6][6], p[6], C[6][6], chi2;
  for (int k = 0; k < 6; ++k) p0[k] = p0v[k];
  for (int a = 0; a < 6; ++a)
    for (int b = 0; b < 6; ++b) C0[a][b] = C0v[sym_index(a, b)];
  double raw[3][3];
  int lays[3];
  for (int k = 0; k < 3; ++k) {
    raw[k][0] = hx[sh[k]]; raw[k][1] = hy[sh[k]]; raw[k][2] = hz[sh[k]];
    lays[k] = hlayer[sh[k]];
  }
  int st = fit_track<double, double>(det, p0, C0, 3, raw, lays, al, true, p, C, chi2);
  *n_found = 3;
  for (int l = 0; l < L; ++l) chi2_layer[l] = 0.0;
  if (st != 0) { *chi2sum = chi2; return st; }
  const double vr = det.sigma_rphi * det.sigma_rphi, vz = det.sigma_z * det.sigma_z;
  for (int l = lays[2] + 1; l < L; ++l) {
    if (decisions[l] == -2) break;
    double q[6], J[6][6];
    if (!propagate(det.field(), p, det.radius[l], q, J)) { *chi2sum = chi2; return -1; }
    for (int i = 0; i < 6; ++i) p[i] = q[i];
    transport(J, C);
    if (decisions[l] >= 0) {
      const int h = decisions[l];
      double rw[3] = {hx[h], hy[h], hz[h]}, m[3];
      correct_hit(rw, al[l][0], al[l][1], det.radius[l], m);
      Meas<double> ms;
      if (!measure(p, C, m, vr, vz, ms)) { *chi2sum = chi2; return -2; }
      chi2_layer[l] = ms.chi2;
      chi2 += ms.chi2;
      kf_update(p, C, ms);
      *n_found += 1;
    }
    add_ms(p, C, x0_at(det, l, p[2]));
    add_eloss(p, C, det.eloss[l]);
  }
  *chi2sum = chi2;
  if (p_out)
    for (int k = 0; k < 6; ++k) p_out[k] = p[k];
  if (C_out)
    for (int a = 0; a < 6; ++a)
      for (int b = a; b < 6; ++b) C_out[sym_index(a, b)] = C[a][b];
  return 0;
}

// Duplicate removal for one event's tracks: walk tracks by (more hits, lower
// chi2, lower index); keep a track unless it shares more than frac*min(nA, nB)
// hits with a track already kept and, when params is given, is also
// kinematically close to it (kin_close with deta, dphi, dpt; pT, eta and phi
// of the track states params [n][6]).  A track without hits is never kept.
// hits [n][max_len] event-local indices.  brute != 0 compares against every
// kept track directly.
int orc_dedup(int n_tracks, const int* hits, const int* n_hits, const double* chi2, int max_len,
              double frac, int brute, unsigned char* keep, const double* params, double bz, double deta,
              double dphi, double dpt) {
  std::vector<double> kin(params ? 3 * (size_t)n_tracks : 0);
  for (int t = 0; params && t < n_tracks; ++t) kinematics_of(bz, params + 6 * (size_t)t, &kin[3 * (size_t)t]);
  auto close = [&](int a, int b) {
    return !params || kin_close(&kin[3 * (size_t)a], &kin[3 * (size_t)b], deta, dphi, dpt);
  };
  std::vector<int> order(n_tracks);
  std::iota(order.begin(), order.end(), 0);
  std::sort(order.begin(), order.end(), [&](int a, int b) {
    if (n_hits[a] != n_hits[b]) return n_hits[a] > n_hits[b];
    if (chi2[a] != chi2[b]) return chi2[a] < chi2[b];
    return a < b;
  });
  std::vector<int> kept;
  // hit -> kept tracks holding it (index form of the same comparison)
  std::vector<std::pair<int, int>> owner;  // (hit, track), kept sorted by hit
  for (int t = 0; t < n_tracks; ++t) keep[t] = 0;
  std::vector<int> shared(n_tracks, 0);
  for (int t : order) {
    bool dup = false;
    const int* ht = hits + (size_t)t * max_len;
    if (brute) {
      for (int k : kept) {
        const int* hk = hits + (size_t)k * max_len;
        int nsh = 0;
        for (int a = 0; a < n_hits[t]; ++a)
          for (int b = 0; b < n_hits[k]; ++b) nsh += ht[a] == hk[b];
        if (nsh > frac * std::min(n_hits[t], n_hits[k]) && close(t, k)) { dup = true; break; }
      }
    } else {
      std::vector<int> touched;
      for (int a = 0; a < n_hits[t]; ++a) {
        auto it = std::lower_bound(owner.begin(), owner.end(), std::make_pair(ht[a], -1));
        for (; it != owner.end() && it->first == ht[a]; ++it) {
          if (shared[it->second]++ == 0) touched.push_back(it->second);
        }
      }
      for (int k : touched) {
        if (shared[k] > frac * std::min(n_hits[t], n_hits[k]) && close(t, k)) dup = true;
        shared[k] = 0;
      }
    }
    if (!dup && n_hits[t] > 0) {
      keep[t] = 1;
      kept.push_back(t);
      if (!brute) {
        for (int a = 0; a < n_hits[t]; ++a) {
          auto pr = std::make_pair(ht[a], t);
          owner.insert(std::upper_bound(owner.begin(), owner.end(), pr), pr);
        }
      }
    }
  }
  return 0;
}

// Kinematic quantities of n states params [n][6] into out [n][3]
// (eta, |q/pT|, phi0; see kinematics_of).
void orc_kinematics(int n, double bz, const double* params, double* out) {
  for (int i = 0; i < n; ++i) kinematics_of(bz, params + 6 * (size_t)i, out + 3 * (size_t)i);
}

// Seed cleaning before building (Sec. 4.2, first step), one event: visit the
// seeds by index and drop a seed when a seed already kept is kinematically
// close to it (kin_close with deta, dphi, dpt on the seed states params
// [n][6]) and shares at least min_shared of its three hits (hits [n][3]).
int orc_seed_clean(int n, const double* params, const int* hits, double bz, double deta, double dphi,
                   double dpt, int min_shared, unsigned char* keep) {
  std::vector<double> kin(3 * (size_t)n);
  for (int i = 0; i < n; ++i) kinematics_of(bz, params + 6 * (size_t)i, &kin[3 * (size_t)i]);
  std::vector<int> kept;
  for (int j = 0; j < n; ++j) {
    bool dup = false;
    for (int i : kept) {
      int shared = 0;
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) shared += hits[3 * (size_t)j + a] == hits[3 * (size_t)i + b];
      if (shared >= min_shared && kin_close(&kin[3 * (size_t)j], &kin[3 * (size_t)i], deta, dphi, dpt)) {
        dup = true;
        break;
      }
    }
    keep[j] = dup ? 0 : 1;
    if (!dup) kept.push_back(j);
  }
  return 0;
}

}  // extern "C"
