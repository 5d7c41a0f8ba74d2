// Plain FP64 CPU oracle of the multi-environment IPC step (GRIP, arXiv 2503.05020).
//
// TEST INFRASTRUCTURE ONLY. This file is the slow, obviously-correct reference that the CUDA
// path is checked against. Only the tests, the smoke check and the CPU-baseline leg of the
// benchmark may load it. It shares no code, header or table with the CUDA path.
//
// It follows the paper's description of the solver (Sec. II-C: barrier augmentation, CCD and
// projected Newton with a step-size filter; Sec. III-A: per-environment isolation of collision
// detection and step size, per-environment stopping and failure; Sec. III-D: dt, kappa, dhat,
// eps_v, at most 100 Newton iterations, FP64). The terms the paper names but does not restate
// follow their published definitions: the IPC log barrier, edge-edge mollifier and lagged
// smoothed friction (Li et al. 2020), Neo-Hookean tets, affine body dynamics (Lan et al. 2022)
// and additive CCD (Li, Kaufman & Jiang 2021).
//
// Derivatives: every energy's gradient and Hessian comes from second-order forward-mode
// automatic differentiation of the energy written out plainly, except friction whose lagged
// form has an explicit closed-form derivative. Negative eigenvalues are clamped with a cyclic
// Jacobi eigensolver. The linear solve is conjugate gradients to 1e-12 relative residual.
// Broad phase is all pairs. Built with -ffp-contract=off so that every expression rounds as
// written.
//
// Every function here is pinned by a test against closed forms, invariants, brute force or a
// library routine (tests/test_oracle_*.py). The adapted barrier stiffness (an option; the paper
// fixes kappa) is set once per step by a least-squares force balance that a resting body pins
// in closed form; it is not changed inside a step.
#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <thread>
#include <vector>

namespace orc {

// ============================================================== forward-mode AD (2nd order)
template <int N>
struct Dual {
  double v = 0.0;
  std::array<double, N> g{};
  std::array<double, N * N> h{};
  Dual() {}
  Dual(double c) : v(c) {}
  static Dual var(int i, double val) {
    Dual d(val);
    d.g[i] = 1.0;
    return d;
  }
};
template <int N> Dual<N> operator+(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r(a.v + b.v);
  for (int i = 0; i < N; ++i) r.g[i] = a.g[i] + b.g[i];
  for (int i = 0; i < N * N; ++i) r.h[i] = a.h[i] + b.h[i];
  return r;
}
template <int N> Dual<N> operator-(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r(a.v - b.v);
  for (int i = 0; i < N; ++i) r.g[i] = a.g[i] - b.g[i];
  for (int i = 0; i < N * N; ++i) r.h[i] = a.h[i] - b.h[i];
  return r;
}
template <int N> Dual<N> operator-(const Dual<N>& a) { return Dual<N>(0.0) - a; }
template <int N> Dual<N> operator*(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r(a.v * b.v);
  for (int i = 0; i < N; ++i) r.g[i] = a.v * b.g[i] + b.v * a.g[i];
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j)
      r.h[i * N + j] = a.v * b.h[i * N + j] + b.v * a.h[i * N + j] + a.g[i] * b.g[j] + b.g[i] * a.g[j];
  return r;
}
// f(a) for a scalar function with derivatives f1 = f'(a.v), f2 = f''(a.v)
template <int N> Dual<N> chain(const Dual<N>& a, double f0, double f1, double f2) {
  Dual<N> r(f0);
  for (int i = 0; i < N; ++i) r.g[i] = f1 * a.g[i];
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j) r.h[i * N + j] = f1 * a.h[i * N + j] + f2 * a.g[i] * a.g[j];
  return r;
}
template <int N> Dual<N> operator/(const Dual<N>& a, const Dual<N>& b) {
  double iv = 1.0 / b.v;
  return a * chain(b, iv, -iv * iv, 2.0 * iv * iv * iv);
}
template <int N> Dual<N> log(const Dual<N>& a) { return chain(a, std::log(a.v), 1.0 / a.v, -1.0 / (a.v * a.v)); }
template <int N> Dual<N> sqrt(const Dual<N>& a) {
  double s = std::sqrt(a.v);
  return chain(a, s, 0.5 / s, -0.25 / (s * a.v));
}
inline double value(double a) { return a; }
template <int N> double value(const Dual<N>& a) { return a.v; }
using std::log;
using std::sqrt;

template <class S> struct V3 { S x, y, z; };
template <class S> V3<S> sub(const V3<S>& a, const V3<S>& b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
template <class S> S dot(const V3<S>& a, const V3<S>& b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <class S> V3<S> cross(const V3<S>& a, const V3<S>& b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}

// ============================================================== symmetric eigen / PSD projection
// Cyclic Jacobi on a symmetric n x n matrix (row-major), run until the off-diagonal norm is
// below 1e-14 * ||A||_F; then A is rebuilt from the eigenpairs with negative eigenvalues set to 0.
static void jacobi_eigen(int n, const double* A, double* evals, double* evecs /* column k = vec k */) {
  std::vector<double> a(A, A + n * n), v(n * n, 0.0);
  for (int i = 0; i < n; ++i) v[i * n + i] = 1.0;
  double fro = 0.0;
  for (int i = 0; i < n * n; ++i) fro += a[i] * a[i];
  fro = std::sqrt(fro);
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j)
        if (i != j) off += a[i * n + j] * a[i * n + j];
    if (std::sqrt(off) <= 1e-14 * fro || off == 0.0) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        double apq = a[p * n + q];
        if (apq == 0.0) continue;
        double app = a[p * n + p], aqq = a[q * n + q];
        double theta = (aqq - app) / (2.0 * apq);
        double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {  // A <- A J
          double akp = a[k * n + p], akq = a[k * n + q];
          a[k * n + p] = c * akp - s * akq;
          a[k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {  // A <- J^T A
          double apk = a[p * n + k], aqk = a[q * n + k];
          a[p * n + k] = c * apk - s * aqk;
          a[q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          double vkp = v[k * n + p], vkq = v[k * n + q];
          v[k * n + p] = c * vkp - s * vkq;
          v[k * n + q] = s * vkp + c * vkq;
        }
      }
  }
  for (int i = 0; i < n; ++i) evals[i] = a[i * n + i];
  std::memcpy(evecs, v.data(), sizeof(double) * n * n);
}

static void project_psd(int n, double* A) {
  std::vector<double> ev(n), V(n * n);
  jacobi_eigen(n, A, ev.data(), V.data());
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      for (int k = 0; k < n; ++k)
        if (ev[k] > 0.0) s += V[i * n + k] * ev[k] * V[j * n + k];
      A[i * n + j] = s;
    }
}

// ============================================================== energies (templated on scalar)
// Neo-Hookean density (IPC 2020 form): mu/2 (tr F^T F - 3) - mu ln J + lam/2 (ln J)^2.
template <class S> S neo_hookean(const S F[9], double mu, double lam) {
  S J = F[0] * (F[4] * F[8] - F[5] * F[7]) - F[1] * (F[3] * F[8] - F[5] * F[6]) + F[2] * (F[3] * F[7] - F[4] * F[6]);
  S tr = F[0] * F[0];
  for (int i = 1; i < 9; ++i) tr = tr + F[i] * F[i];
  S lnJ = log(J);
  return S(0.5 * mu) * (tr - S(3.0)) - S(mu) * lnJ + S(0.5 * lam) * lnJ * lnJ;
}

// Log barrier b(d) = -(d - dhat)^2 ln(d / dhat) for 0 < d < dhat, else 0 (IPC 2020).
template <class S> S barrier(const S& d, double dhat) {
  if (value(d) >= dhat) return S(0.0);
  S t = d - S(dhat);
  return -(t * t) * log(d / S(dhat));
}
static void barrier_derivs(double d, double dhat, double* b, double* b1, double* b2) {
  Dual<1> x = Dual<1>::var(0, d);
  Dual<1> r = barrier(x, dhat);
  *b = r.v;
  *b1 = r.g[0];
  *b2 = r.h[0];
}

// ----- squared distances of the four base configurations
template <class S> S dist2_pp(const V3<S>& a, const V3<S>& b) {
  V3<S> d = sub(a, b);
  return dot(d, d);
}
template <class S> S dist2_pe(const V3<S>& p, const V3<S>& e0, const V3<S>& e1) {
  V3<S> c = cross(sub(e0, p), sub(e1, p));
  V3<S> e = sub(e1, e0);
  return dot(c, c) / dot(e, e);
}
template <class S> S dist2_pt_plane(const V3<S>& p, const V3<S>& t0, const V3<S>& t1, const V3<S>& t2) {
  V3<S> n = cross(sub(t1, t0), sub(t2, t0));
  S e = dot(sub(p, t0), n);
  return e * e / dot(n, n);
}
template <class S> S dist2_ee_line(const V3<S>& a0, const V3<S>& a1, const V3<S>& b0, const V3<S>& b1) {
  V3<S> n = cross(sub(a1, a0), sub(b1, b0));
  S e = dot(sub(b0, a0), n);
  return e * e / dot(n, n);
}

// Distance types. PT: closest feature of the triangle; EE: closest features of both edges.
enum PTType { PT_P0 = 0, PT_P1, PT_P2, PT_E01, PT_E12, PT_E20, PT_FACE };
enum EEType { EE_A0B0 = 0, EE_A0B1, EE_A1B0, EE_A1B1, EE_A_B0, EE_A_B1, EE_A0_B, EE_A1_B, EE_LINES };

static double d3dot(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

// Region of the closest point of triangle (a, b, c) to p, by the barycentric region tests of
// Ericson, "Real-Time Collision Detection" (2005), Sec. 5.1.5. w[] gets the closest-point weights.
static int pt_type(const double* p, const double* a, const double* b, const double* c, double w[3]) {
  double ab[3], ac[3], ap[3], bp[3], cp[3];
  for (int i = 0; i < 3; ++i) {
    ab[i] = b[i] - a[i];
    ac[i] = c[i] - a[i];
    ap[i] = p[i] - a[i];
    bp[i] = p[i] - b[i];
    cp[i] = p[i] - c[i];
  }
  double d1 = d3dot(ab, ap), d2 = d3dot(ac, ap);
  if (d1 <= 0 && d2 <= 0) { w[0] = 1; w[1] = 0; w[2] = 0; return PT_P0; }
  double d3 = d3dot(ab, bp), d4 = d3dot(ac, bp);
  if (d3 >= 0 && d4 <= d3) { w[0] = 0; w[1] = 1; w[2] = 0; return PT_P1; }
  double vc = d1 * d4 - d3 * d2;
  if (vc <= 0 && d1 >= 0 && d3 <= 0) {
    double t = d1 / (d1 - d3);
    w[0] = 1 - t; w[1] = t; w[2] = 0;
    return PT_E01;
  }
  double d5 = d3dot(ab, cp), d6 = d3dot(ac, cp);
  if (d6 >= 0 && d5 <= d6) { w[0] = 0; w[1] = 0; w[2] = 1; return PT_P2; }
  double vb = d5 * d2 - d1 * d6;
  if (vb <= 0 && d2 >= 0 && d6 <= 0) {
    double t = d2 / (d2 - d6);
    w[0] = 1 - t; w[1] = 0; w[2] = t;
    return PT_E20;
  }
  double va = d3 * d6 - d5 * d4;
  if (va <= 0 && (d4 - d3) >= 0 && (d5 - d6) >= 0) {
    double t = (d4 - d3) / ((d4 - d3) + (d5 - d6));
    w[0] = 0; w[1] = 1 - t; w[2] = t;
    return PT_E12;
  }
  double den = 1.0 / (va + vb + vc);
  double v = vb * den, ww = vc * den;
  w[0] = 1 - v - ww; w[1] = v; w[2] = ww;
  return PT_FACE;
}

// Closest points of segments a0a1 and b0b1 (Ericson 2005, Sec. 5.1.9), returning the type
// and the parameters s (on a) and t (on b).
static int ee_type(const double* a0, const double* a1, const double* b0, const double* b1, double* s_out, double* t_out) {
  double d1[3], d2[3], r[3];
  for (int i = 0; i < 3; ++i) {
    d1[i] = a1[i] - a0[i];
    d2[i] = b1[i] - b0[i];
    r[i] = a0[i] - b0[i];
  }
  double a = d3dot(d1, d1), e = d3dot(d2, d2), f = d3dot(d2, r), c = d3dot(d1, r), b = d3dot(d1, d2);
  double den = a * e - b * b;
  double s, t;
  if (den > 1e-10 * a * e) s = std::min(std::max((b * f - c * e) / den, 0.0), 1.0);  // sin^2 > 1e-10
  else s = 0.0;
  t = (b * s + f) / e;
  if (t < 0) { t = 0; s = std::min(std::max(-c / a, 0.0), 1.0); }
  else if (t > 1) { t = 1; s = std::min(std::max((b - c) / a, 0.0), 1.0); }
  *s_out = s;
  *t_out = t;
  bool s0 = s <= 0.0, s1 = s >= 1.0, t0 = t <= 0.0, t1 = t >= 1.0;
  bool sa = !(s0 || s1), tb = !(t0 || t1);
  if (sa && tb) return EE_LINES;
  if (sa) return t0 ? EE_A_B0 : EE_A_B1;
  if (tb) return s0 ? EE_A0_B : EE_A1_B;
  if (s0) return t0 ? EE_A0B0 : EE_A0B1;
  return t0 ? EE_A1B0 : EE_A1B1;
}

template <class S> S pt_dist2_typed(int type, const V3<S>& p, const V3<S>& a, const V3<S>& b, const V3<S>& c) {
  switch (type) {
    case PT_P0: return dist2_pp(p, a);
    case PT_P1: return dist2_pp(p, b);
    case PT_P2: return dist2_pp(p, c);
    case PT_E01: return dist2_pe(p, a, b);
    case PT_E12: return dist2_pe(p, b, c);
    case PT_E20: return dist2_pe(p, c, a);
    default: return dist2_pt_plane(p, a, b, c);
  }
}
template <class S> S ee_dist2_typed(int type, const V3<S>& a0, const V3<S>& a1, const V3<S>& b0, const V3<S>& b1) {
  switch (type) {
    case EE_A0B0: return dist2_pp(a0, b0);
    case EE_A0B1: return dist2_pp(a0, b1);
    case EE_A1B0: return dist2_pp(a1, b0);
    case EE_A1B1: return dist2_pp(a1, b1);
    case EE_A_B0: return dist2_pe(b0, a0, a1);
    case EE_A_B1: return dist2_pe(b1, a0, a1);
    case EE_A0_B: return dist2_pe(a0, b0, b1);
    case EE_A1_B: return dist2_pe(a1, b0, b1);
    default: return dist2_ee_line(a0, a1, b0, b1);
  }
}

// Unsigned squared distance of a PT (kind 0) or EE (kind 1) pair of 4 points.
static double pair_dist2(int kind, const double* x /*12*/, int* type_out = nullptr) {
  V3<double> P[4];
  for (int i = 0; i < 4; ++i) P[i] = {x[3 * i], x[3 * i + 1], x[3 * i + 2]};
  int type;
  double w[3], s, t;
  if (kind == 0) {
    type = pt_type(x, x + 3, x + 6, x + 9, w);
    if (type_out) *type_out = type;
    return pt_dist2_typed(type, P[0], P[1], P[2], P[3]);
  }
  type = ee_type(x, x + 3, x + 6, x + 9, &s, &t);
  if (type_out) *type_out = type;
  return ee_dist2_typed(type, P[0], P[1], P[2], P[3]);
}

// Closest-point coefficients c[4] (relative displacement = sum_i c_i dx_i) and unit normal n
// from the B side to the A side of the pair at configuration x.
static void pair_closest(int kind, const double* x, double c[4], double n[3]) {
  double ca[3], cb[3];
  if (kind == 0) {
    double w[3];
    int type = pt_type(x, x + 3, x + 6, x + 9, w);
    const double* a = x + 3; const double* b = x + 6; const double* cc = x + 9;
    double wb[3] = {w[0], w[1], w[2]};
    if (type == PT_E01 || type == PT_E12 || type == PT_E20) {  // projection onto the edge line
      const double* e0 = type == PT_E01 ? a : (type == PT_E12 ? b : cc);
      const double* e1 = type == PT_E01 ? b : (type == PT_E12 ? cc : a);
      double e[3] = {e1[0] - e0[0], e1[1] - e0[1], e1[2] - e0[2]};
      double q[3] = {x[0] - e0[0], x[1] - e0[1], x[2] - e0[2]};
      double t = d3dot(q, e) / d3dot(e, e);
      int i0 = type == PT_E01 ? 0 : (type == PT_E12 ? 1 : 2);
      int i1 = type == PT_E01 ? 1 : (type == PT_E12 ? 2 : 0);
      wb[0] = wb[1] = wb[2] = 0;
      wb[i0] = 1 - t;
      wb[i1] = t;
    } else if (type == PT_FACE) {  // projection onto the plane, barycentric weights
      double e1[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]}, e2[3] = {cc[0] - a[0], cc[1] - a[1], cc[2] - a[2]};
      double q[3] = {x[0] - a[0], x[1] - a[1], x[2] - a[2]};
      double A11 = d3dot(e1, e1), A12 = d3dot(e1, e2), A22 = d3dot(e2, e2);
      double r1 = d3dot(e1, q), r2 = d3dot(e2, q);
      double det = A11 * A22 - A12 * A12;
      double u = (r1 * A22 - r2 * A12) / det, v = (A11 * r2 - A12 * r1) / det;
      wb[0] = 1 - u - v; wb[1] = u; wb[2] = v;
    }
    c[0] = 1.0; c[1] = -wb[0]; c[2] = -wb[1]; c[3] = -wb[2];
    for (int i = 0; i < 3; ++i) {
      ca[i] = x[i];
      cb[i] = wb[0] * a[i] + wb[1] * b[i] + wb[2] * cc[i];
    }
  } else {
    double s, t;
    int type = ee_type(x, x + 3, x + 6, x + 9, &s, &t);
    const double* a0 = x; const double* a1 = x + 3; const double* b0 = x + 6; const double* b1 = x + 9;
    auto proj = [](const double* p, const double* e0, const double* e1) {
      double e[3] = {e1[0] - e0[0], e1[1] - e0[1], e1[2] - e0[2]};
      double q[3] = {p[0] - e0[0], p[1] - e0[1], p[2] - e0[2]};
      return d3dot(q, e) / d3dot(e, e);
    };
    switch (type) {
      case EE_A0B0: s = 0; t = 0; break;
      case EE_A0B1: s = 0; t = 1; break;
      case EE_A1B0: s = 1; t = 0; break;
      case EE_A1B1: s = 1; t = 1; break;
      case EE_A_B0: t = 0; s = proj(b0, a0, a1); break;
      case EE_A_B1: t = 1; s = proj(b1, a0, a1); break;
      case EE_A0_B: s = 0; t = proj(a0, b0, b1); break;
      case EE_A1_B: s = 1; t = proj(a1, b0, b1); break;
      default: {  // closest points of the two infinite lines
        double d1[3], d2[3], r[3];
        for (int i = 0; i < 3; ++i) { d1[i] = a1[i] - a0[i]; d2[i] = b1[i] - b0[i]; r[i] = a0[i] - b0[i]; }
        double a = d3dot(d1, d1), e = d3dot(d2, d2), f = d3dot(d2, r), cc = d3dot(d1, r), b = d3dot(d1, d2);
        double den = a * e - b * b;
        s = (b * f - cc * e) / den;
        t = (a * f - b * cc) / den;
      }
    }
    c[0] = 1 - s; c[1] = s; c[2] = -(1 - t); c[3] = -t;
    for (int i = 0; i < 3; ++i) {
      ca[i] = (1 - s) * a0[i] + s * a1[i];
      cb[i] = (1 - t) * b0[i] + t * b1[i];
    }
  }
  double d[3] = {ca[0] - cb[0], ca[1] - cb[1], ca[2] - cb[2]};
  double L = std::sqrt(d3dot(d, d));
  for (int i = 0; i < 3; ++i) n[i] = L > 0 ? d[i] / L : 0.0;
}

// EE mollifier (IPC 2020): e(c) = -(c/eps)^2 + 2 c/eps for c < eps, else 1, where
// c = |(a1 - a0) x (b1 - b0)|^2 and eps = 1e-3 |rest a|^2 |rest b|^2.
template <class S> S mollifier(const V3<S>& a0, const V3<S>& a1, const V3<S>& b0, const V3<S>& b1, double eps) {
  V3<S> cr = cross(sub(a1, a0), sub(b1, b0));
  S c = dot(cr, cr);
  if (value(c) >= eps) return S(1.0);
  S r = c / S(eps);
  return -(r * r) + S(2.0) * r;
}

// Barrier energy kappa * e * b(d) of one contact (without the h^2 factor).
template <class S> S contact_barrier_energy(int kind, const S* x12, double dhat, double kappa, double eps_x,
                                            int type) {
  V3<S> P[4];
  for (int i = 0; i < 4; ++i) P[i] = {x12[3 * i], x12[3 * i + 1], x12[3 * i + 2]};
  if (kind == 0) {
    S d2 = pt_dist2_typed(type, P[0], P[1], P[2], P[3]);
    return S(kappa) * barrier(sqrt(d2), dhat);
  }
  S d2 = ee_dist2_typed(type, P[0], P[1], P[2], P[3]);
  return S(kappa) * mollifier(P[0], P[1], P[2], P[3], eps_x) * barrier(sqrt(d2), dhat);
}

// Lagged smoothed friction f0 (IPC 2020): y < eps_v h: -y^3/(3 eps^2) + y^2/eps + eps/3, else y,
// with eps = eps_v * h. f1 = f0', f1' = f0''.
static void friction_f(double y, double eh, double* f0, double* f1, double* f2) {
  if (y < eh) {
    *f0 = -y * y * y / (3.0 * eh * eh) + y * y / eh + eh / 3.0;
    *f1 = -y * y / (eh * eh) + 2.0 * y / eh;
    *f2 = -2.0 * y / (eh * eh) + 2.0 / eh;
  } else {
    *f0 = y;
    *f1 = 1.0;
    *f2 = 0.0;
  }
}

// ACCD (Li, Kaufman & Jiang 2021): conservative time of impact of a PT (kind 0) or EE (kind 1)
// pair moving linearly by p over [0, 1], thickness 0, gap fraction s; returns t_c when no
// contact happens before t_c. iters gets the number of advancement iterations taken.
static double accd(int kind, const double* x0, const double* p0, double s, double t_c, long max_iter, long* iters) {
  double x[12], p[12];
  std::memcpy(x, x0, sizeof(x));
  std::memcpy(p, p0, sizeof(p));
  double mean[3] = {0, 0, 0};
  for (int i = 0; i < 4; ++i)
    for (int k = 0; k < 3; ++k) mean[k] += p[3 * i + k];
  for (int k = 0; k < 3; ++k) mean[k] = mean[k] / 4.0;
  for (int i = 0; i < 4; ++i)
    for (int k = 0; k < 3; ++k) p[3 * i + k] -= mean[k];
  double n[4];
  for (int i = 0; i < 4; ++i) n[i] = std::sqrt(d3dot(p + 3 * i, p + 3 * i));
  double lp = kind == 0 ? n[0] + std::max(n[1], std::max(n[2], n[3])) : std::max(n[0], n[1]) + std::max(n[2], n[3]);
  if (iters) *iters = 0;
  if (lp == 0.0) return t_c;
  double d = std::sqrt(pair_dist2(kind, x));
  double g = s * d;
  double t = 0.0;
  double tl = (1.0 - s) * d / lp;
  long it = 0;
  while (true) {
    if (it >= max_iter) break;
    ++it;
    for (int i = 0; i < 12; ++i) x[i] = x[i] + tl * p[i];
    d = std::sqrt(pair_dist2(kind, x));
    if (t > 0.0 && d < g) break;
    t = t + tl;
    if (t > t_c) { t = t_c; break; }
    tl = 0.9 * d / lp;
  }
  if (iters) *iters = it;
  return t;
}

// ============================================================== environment
struct Params {
  double dt, dhat, kappa, eps_v, newton_tol, pcg_rel_tol, kappa_affine, gravity[3];
  int32_t max_newton, max_ls, max_pcg, kappa_adapt;  // kappa_adapt: 1 = adapted barrier stiffness
};

struct SoftDesc {
  int32_t n_verts, n_tets, n_tris, pad;
  const double* verts;
  const int32_t* tets;
  const int32_t* tris;
  const uint8_t* kin;
  double E, nu, rho;
};
struct AffineDesc {
  int32_t n_verts, n_tris, kinematic, pad;
  const double* verts;
  const int32_t* tris;
  double rho;
  double q0[12];
  double qdot0[12];
  double pd_stiffness;  // k_pd (1/s^2); 0: no PD target potential
};
// A point joint between two affine bodies: the anchor of body a (its rest-frame coordinates) and
// the anchor of body b are held together by the potential 1/2 k |x_a - x_b|^2 (k in N/m). Two
// such joints on one axis make a hinge.
struct JointDesc {
  int32_t body_a, body_b;  // affine body indices of the env
  double anchor_a[3], anchor_b[3];
  double stiffness;
};
struct EnvDesc {
  int32_t n_soft, n_affine, n_steps, pad;
  const SoftDesc* soft;
  const AffineDesc* affine;
  double mu;
  const uint8_t* gravity;
  const double* targets;
  int32_t n_joints, pad2;
  const JointDesc* joints;
};

enum { ST_ACTIVE = 0, ST_DONE = 1, ST_FAILED = 2 };
enum { FAIL_NONE = 0, FAIL_NEWTON = 1, FAIL_LINESEARCH = 2, FAIL_NAN = 3 };

struct Point {
  int body;        // env-local body id (soft bodies first, then affine)
  int affine;      // 1 if on an affine body
  int index;       // soft: DOF node (vertex) index; affine: body index among affine bodies
  int kin;         // driven by the schedule
  double xb[3];    // affine: rest-frame coordinates
  double rest[3];  // rest position (mollifier reference)
};
struct Body {
  int dof;   // first DOF of q
  int kin;
  int handle;  // index into the per-step target table
  double kpd;  // PD target stiffness k_pd (1/s^2), free bodies only
  double M4[16];
  double vol;
  double lo[3], hi[3];
};
struct Joint {
  int a, b;  // affine body indices
  double xa[3], xb[3];
  double k;
};
struct Contact {
  int kind;
  int pts[4];
  int type;
  double eps_x;
};
struct FrictionContact {
  int pts[4];
  double c[4];
  double n[3];
  double lambda;
};

struct Env {
  Params P;
  double mu;
  int n_soft_verts = 0, n_bodies = 0, ndof = 0, n_soft_bodies = 0;
  std::vector<double> x, xt, v, xtilde;
  std::vector<double> mass;  // per soft vertex
  std::vector<int> vkin, vhandle;
  std::vector<double> X0;  // initial soft vertex positions
  std::vector<std::array<int, 4>> tets;
  std::vector<std::array<double, 9>> Dminv;
  std::vector<double> tvol, tmu, tlam;
  std::vector<Body> bodies;
  std::vector<Joint> joints;
  std::vector<Point> pts;
  std::vector<int> sv;
  std::vector<std::array<int, 2>> edges;
  std::vector<std::array<int, 3>> tris;
  int n_steps = 0, step = 0, n_handles = 0;
  std::vector<uint8_t> gravity;
  std::vector<double> targets;
  int status = ST_ACTIVE, reason = FAIL_NONE;
  long newton_iters = 0, ls_halvings = 0, cg_iters = 0, accd_iters = 0, steps_done = 0;
  double last_alpha = 1.0;
  std::vector<FrictionContact> fric;
  std::vector<double> ptx_t;  // point positions at step start
  double kappa = 0.0;            // barrier stiffness of the current step (P.kappa unless adapted)
  // per-iteration trace (optional)
  int trace = 0;
  std::vector<double> trace_E;
};

// point positions from a DOF vector: soft = node; affine = ((p + xb0 a1) + xb1 a2) + xb2 a3
static void point_positions(const Env& e, const double* q, std::vector<double>& out) {
  out.resize(3 * e.pts.size());
  for (size_t i = 0; i < e.pts.size(); ++i) {
    const Point& pt = e.pts[i];
    if (!pt.affine) {
      for (int k = 0; k < 3; ++k) out[3 * i + k] = q[3 * pt.index + k];
    } else {
      const double* b = q + e.bodies[pt.index].dof;
      for (int k = 0; k < 3; ++k) {
        double r = b[k] + pt.xb[0] * b[3 + k];
        r = r + pt.xb[1] * b[6 + k];
        r = r + pt.xb[2] * b[9 + k];
        out[3 * i + k] = r;
      }
    }
  }
}
// same linear map applied to a displacement (no translation special case: it is linear in q)
static void point_displacements(const Env& e, const double* p, std::vector<double>& out) { point_positions(e, p, out); }

// DOF weights of a point: soft -> (node dof, 1); affine -> 4 blocks (p, a1, a2, a3) with (1, xb)
struct PointMap {
  int n;
  int dof[4];
  double w[4];
};
static PointMap point_map(const Env& e, int pi) {
  PointMap m;
  const Point& pt = e.pts[pi];
  if (!pt.affine) {
    m.n = 1;
    m.dof[0] = 3 * pt.index;
    m.w[0] = 1.0;
  } else {
    m.n = 4;
    int d = e.bodies[pt.index].dof;
    for (int k = 0; k < 4; ++k) m.dof[k] = d + 3 * k;
    m.w[0] = 1.0; m.w[1] = pt.xb[0]; m.w[2] = pt.xb[1]; m.w[3] = pt.xb[2];
  }
  return m;
}

// Mass properties of a closed outward triangle mesh by the divergence theorem: each triangle
// with the origin spans a signed tet; M4 = rho * integral of [1, x^T; x, x x^T].
static void mass_properties(int nv, const double* v, int nt, const int32_t* t, double rho, double M4[16], double* vol) {
  double I0 = 0, I1[3] = {0, 0, 0}, I2[9] = {0};
  for (int f = 0; f < nt; ++f) {
    const double* a = v + 3 * t[3 * f];
    const double* b = v + 3 * t[3 * f + 1];
    const double* c = v + 3 * t[3 * f + 2];
    double bc[3] = {b[1] * c[2] - b[2] * c[1], b[2] * c[0] - b[0] * c[2], b[0] * c[1] - b[1] * c[0]};
    double det = d3dot(a, bc);
    I0 += det / 6.0;
    double s[3] = {a[0] + b[0] + c[0], a[1] + b[1] + c[1], a[2] + b[2] + c[2]};
    for (int i = 0; i < 3; ++i) I1[i] += det / 24.0 * s[i];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) I2[3 * i + j] += det / 120.0 * (a[i] * a[j] + b[i] * b[j] + c[i] * c[j] + s[i] * s[j]);
  }
  (void)nv;
  M4[0] = rho * I0;
  for (int i = 0; i < 3; ++i) { M4[1 + i] = rho * I1[i]; M4[4 * (1 + i)] = rho * I1[i]; }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) M4[4 * (1 + i) + 1 + j] = rho * I2[3 * i + j];
  *vol = I0;
}

// --------------------------------------------------------------- building an environment
static Env* build_env(const Params& P, const EnvDesc& D) {
  Env* e = new Env();
  e->P = P;
  e->kappa = P.kappa;
  e->mu = D.mu;
  e->n_soft_bodies = D.n_soft;
  e->n_handles = D.n_soft + D.n_affine;
  int nsv = 0;
  for (int b = 0; b < D.n_soft; ++b) nsv += D.soft[b].n_verts;
  e->n_soft_verts = nsv;
  e->n_bodies = D.n_affine;
  e->ndof = 3 * nsv + 12 * D.n_affine;
  e->x.assign(e->ndof, 0.0);
  e->v.assign(e->ndof, 0.0);
  e->mass.assign(nsv, 0.0);
  e->vkin.assign(nsv, 0);
  e->vhandle.assign(nsv, 0);
  e->X0.assign(3 * nsv, 0.0);
  // soft bodies: vertices, tets, lumped masses
  int voff = 0;
  for (int b = 0; b < D.n_soft; ++b) {
    const SoftDesc& S = D.soft[b];
    double mu = S.E / (2.0 * (1.0 + S.nu));
    double lam = S.E * S.nu / ((1.0 + S.nu) * (1.0 - 2.0 * S.nu));
    for (int i = 0; i < S.n_verts; ++i) {
      for (int k = 0; k < 3; ++k) {
        e->x[3 * (voff + i) + k] = S.verts[3 * i + k];
        e->X0[3 * (voff + i) + k] = S.verts[3 * i + k];
      }
      e->vkin[voff + i] = S.kin ? S.kin[i] : 0;
      e->vhandle[voff + i] = b;
    }
    for (int t = 0; t < S.n_tets; ++t) {
      std::array<int, 4> tt;
      for (int k = 0; k < 4; ++k) tt[k] = voff + S.tets[4 * t + k];
      const double* X[4];
      for (int k = 0; k < 4; ++k) X[k] = S.verts + 3 * S.tets[4 * t + k];
      double Dm[9];  // columns X1-X0, X2-X0, X3-X0
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) Dm[3 * r + c] = X[c + 1][r] - X[0][r];
      double det = Dm[0] * (Dm[4] * Dm[8] - Dm[5] * Dm[7]) - Dm[1] * (Dm[3] * Dm[8] - Dm[5] * Dm[6]) +
                   Dm[2] * (Dm[3] * Dm[7] - Dm[4] * Dm[6]);
      std::array<double, 9> inv;
      inv[0] = (Dm[4] * Dm[8] - Dm[5] * Dm[7]) / det;
      inv[1] = (Dm[2] * Dm[7] - Dm[1] * Dm[8]) / det;
      inv[2] = (Dm[1] * Dm[5] - Dm[2] * Dm[4]) / det;
      inv[3] = (Dm[5] * Dm[6] - Dm[3] * Dm[8]) / det;
      inv[4] = (Dm[0] * Dm[8] - Dm[2] * Dm[6]) / det;
      inv[5] = (Dm[2] * Dm[3] - Dm[0] * Dm[5]) / det;
      inv[6] = (Dm[3] * Dm[7] - Dm[4] * Dm[6]) / det;
      inv[7] = (Dm[1] * Dm[6] - Dm[0] * Dm[7]) / det;
      inv[8] = (Dm[0] * Dm[4] - Dm[1] * Dm[3]) / det;
      double vol = det / 6.0;
      e->tets.push_back(tt);
      e->Dminv.push_back(inv);
      e->tvol.push_back(vol);
      e->tmu.push_back(mu);
      e->tlam.push_back(lam);
      for (int k = 0; k < 4; ++k) e->mass[tt[k]] += S.rho * vol / 4.0;
    }
    voff += S.n_verts;
  }
  // affine bodies
  for (int b = 0; b < D.n_affine; ++b) {
    const AffineDesc& A = D.affine[b];
    Body B;
    B.dof = 3 * nsv + 12 * b;
    B.kin = A.kinematic;
    B.handle = D.n_soft + b;
    B.kpd = A.kinematic ? 0.0 : A.pd_stiffness;
    mass_properties(A.n_verts, A.verts, A.n_tris, A.tris, A.rho, B.M4, &B.vol);
    for (int k = 0; k < 3; ++k) { B.lo[k] = 1e300; B.hi[k] = -1e300; }
    for (int i = 0; i < A.n_verts; ++i)
      for (int k = 0; k < 3; ++k) {
        B.lo[k] = std::min(B.lo[k], A.verts[3 * i + k]);
        B.hi[k] = std::max(B.hi[k], A.verts[3 * i + k]);
      }
    for (int k = 0; k < 12; ++k) {
      e->x[B.dof + k] = A.q0[k];
      e->v[B.dof + k] = A.qdot0[k];
    }
    e->bodies.push_back(B);
  }
  for (int j = 0; j < D.n_joints; ++j) {
    const JointDesc& J = D.joints[j];
    Joint jt;
    jt.a = J.body_a;
    jt.b = J.body_b;
    for (int k = 0; k < 3; ++k) { jt.xa[k] = J.anchor_a[k]; jt.xb[k] = J.anchor_b[k]; }
    jt.k = J.stiffness;
    e->joints.push_back(jt);
  }
  // points: all soft vertices, then every affine rest vertex
  voff = 0;
  std::vector<int> soft_pt_off(D.n_soft), aff_pt_off(D.n_affine);
  for (int b = 0; b < D.n_soft; ++b) {
    soft_pt_off[b] = (int)e->pts.size();
    for (int i = 0; i < D.soft[b].n_verts; ++i) {
      Point pt;
      pt.body = b;
      pt.affine = 0;
      pt.index = voff + i;
      pt.kin = e->vkin[voff + i];
      for (int k = 0; k < 3; ++k) { pt.xb[k] = 0; pt.rest[k] = D.soft[b].verts[3 * i + k]; }
      e->pts.push_back(pt);
    }
    voff += D.soft[b].n_verts;
  }
  for (int b = 0; b < D.n_affine; ++b) {
    aff_pt_off[b] = (int)e->pts.size();
    for (int i = 0; i < D.affine[b].n_verts; ++i) {
      Point pt;
      pt.body = D.n_soft + b;
      pt.affine = 1;
      pt.index = b;
      pt.kin = D.affine[b].kinematic;
      for (int k = 0; k < 3; ++k) { pt.xb[k] = D.affine[b].verts[3 * i + k]; pt.rest[k] = pt.xb[k]; }
      e->pts.push_back(pt);
    }
  }
  // surface triangles (bodies in order), surface vertices (sorted unique), edges (sorted unique)
  for (int b = 0; b < D.n_soft; ++b)
    for (int f = 0; f < D.soft[b].n_tris; ++f)
      e->tris.push_back({soft_pt_off[b] + D.soft[b].tris[3 * f], soft_pt_off[b] + D.soft[b].tris[3 * f + 1],
                         soft_pt_off[b] + D.soft[b].tris[3 * f + 2]});
  for (int b = 0; b < D.n_affine; ++b)
    for (int f = 0; f < D.affine[b].n_tris; ++f)
      e->tris.push_back({aff_pt_off[b] + D.affine[b].tris[3 * f], aff_pt_off[b] + D.affine[b].tris[3 * f + 1],
                         aff_pt_off[b] + D.affine[b].tris[3 * f + 2]});
  std::vector<int> svs;
  std::vector<std::array<int, 2>> eds;
  for (auto& t : e->tris) {
    for (int k = 0; k < 3; ++k) {
      svs.push_back(t[k]);
      int a = t[k], b = t[(k + 1) % 3];
      eds.push_back({std::min(a, b), std::max(a, b)});
    }
  }
  std::sort(svs.begin(), svs.end());
  svs.erase(std::unique(svs.begin(), svs.end()), svs.end());
  std::sort(eds.begin(), eds.end());
  eds.erase(std::unique(eds.begin(), eds.end()), eds.end());
  e->sv = svs;
  e->edges = eds;
  // schedule
  e->n_steps = D.n_steps;
  e->gravity.assign(D.gravity, D.gravity + D.n_steps);
  e->targets.assign(D.targets, D.targets + (size_t)D.n_steps * e->n_handles * 12);
  e->xt = e->x;
  return e;
}

// ---------------------------------------------------------------- constraint sets (all pairs)
static void prim_box(const double* px, const int* ids, int n, double r, double lo[3], double hi[3]) {
  for (int k = 0; k < 3; ++k) {
    double mn = px[3 * ids[0] + k], mx = mn;
    for (int i = 1; i < n; ++i) {
      mn = std::min(mn, px[3 * ids[i] + k]);
      mx = std::max(mx, px[3 * ids[i] + k]);
    }
    lo[k] = mn - r;
    hi[k] = mx + r;
  }
}
static void prim_box_swept(const double* px, const double* pe, const int* ids, int n, double lo[3], double hi[3]) {
  for (int k = 0; k < 3; ++k) {
    double mn = px[3 * ids[0] + k], mx = mn;
    for (int i = 0; i < n; ++i) {
      double a = px[3 * ids[i] + k], b = pe[3 * ids[i] + k];
      mn = std::min(mn, std::min(a, b));
      mx = std::max(mx, std::max(a, b));
    }
    lo[k] = mn;
    hi[k] = mx;
  }
}
static bool boxes_overlap(const double* alo, const double* ahi, const double* blo, const double* bhi) {
  for (int k = 0; k < 3; ++k)
    if (!(alo[k] <= bhi[k] && blo[k] <= ahi[k])) return false;
  return true;
}
static bool pair_excluded(const Env& e, const int p[4]) {
  bool all_kin = e.pts[p[0]].kin && e.pts[p[1]].kin && e.pts[p[2]].kin && e.pts[p[3]].kin;
  if (all_kin) return true;
  int b = e.pts[p[0]].body;
  bool same = e.pts[p[1]].body == b && e.pts[p[2]].body == b && e.pts[p[3]].body == b;
  return same && e.pts[p[0]].affine;
}

// Candidate pairs: kind 0 = (surface vertex i, triangle j), kind 1 = (edge i, edge j), i < j.
// Boxes are inflated by r (dhat/2 for the constraint set); pe != nullptr gives swept boxes.
static void candidates(const Env& e, const std::vector<double>& px, const std::vector<double>* pe, double r,
                       std::vector<std::array<int, 3>>& out) {
  out.clear();
  size_t ns = e.sv.size(), nt = e.tris.size(), ne = e.edges.size();
  std::vector<double> tlo(3 * nt), thi(3 * nt), elo(3 * ne), ehi(3 * ne);
  for (size_t j = 0; j < nt; ++j) {
    if (pe) prim_box_swept(px.data(), pe->data(), e.tris[j].data(), 3, &tlo[3 * j], &thi[3 * j]);
    else prim_box(px.data(), e.tris[j].data(), 3, r, &tlo[3 * j], &thi[3 * j]);
  }
  for (size_t j = 0; j < ne; ++j) {
    if (pe) prim_box_swept(px.data(), pe->data(), e.edges[j].data(), 2, &elo[3 * j], &ehi[3 * j]);
    else prim_box(px.data(), e.edges[j].data(), 2, r, &elo[3 * j], &ehi[3 * j]);
  }
  for (size_t i = 0; i < ns; ++i) {
    double lo[3], hi[3];
    int v = e.sv[i];
    if (pe) prim_box_swept(px.data(), pe->data(), &v, 1, lo, hi);
    else prim_box(px.data(), &v, 1, r, lo, hi);
    for (size_t j = 0; j < nt; ++j) {
      const auto& t = e.tris[j];
      if (t[0] == v || t[1] == v || t[2] == v) continue;
      int p[4] = {v, t[0], t[1], t[2]};
      if (pair_excluded(e, p)) continue;
      if (boxes_overlap(lo, hi, &tlo[3 * j], &thi[3 * j])) out.push_back({0, (int)i, (int)j});
    }
  }
  for (size_t i = 0; i < ne; ++i)
    for (size_t j = i + 1; j < ne; ++j) {
      const auto& a = e.edges[i];
      const auto& b = e.edges[j];
      if (a[0] == b[0] || a[0] == b[1] || a[1] == b[0] || a[1] == b[1]) continue;
      int p[4] = {a[0], a[1], b[0], b[1]};
      if (pair_excluded(e, p)) continue;
      if (boxes_overlap(&elo[3 * i], &ehi[3 * i], &elo[3 * j], &ehi[3 * j])) out.push_back({1, (int)i, (int)j});
    }
}
static void cand_points(const Env& e, const std::array<int, 3>& c, int p[4]) {
  if (c[0] == 0) {
    p[0] = e.sv[c[1]];
    for (int k = 0; k < 3; ++k) p[1 + k] = e.tris[c[2]][k];
  } else {
    p[0] = e.edges[c[1]][0]; p[1] = e.edges[c[1]][1];
    p[2] = e.edges[c[2]][0]; p[3] = e.edges[c[2]][1];
  }
}
static void gather12(const std::vector<double>& px, const int p[4], double* x12) {
  for (int i = 0; i < 4; ++i)
    for (int k = 0; k < 3; ++k) x12[3 * i + k] = px[3 * p[i] + k];
}
static double rest_len2(const Env& e, int a, int b) {
  double s = 0;
  for (int k = 0; k < 3; ++k) {
    double d = e.pts[a].rest[k] - e.pts[b].rest[k];
    s += d * d;
  }
  return s;
}

// active constraint set: candidates with d < dhat
static void constraint_set(const Env& e, const std::vector<double>& px, std::vector<Contact>& out) {
  std::vector<std::array<int, 3>> cands;
  candidates(e, px, nullptr, 0.5 * e.P.dhat, cands);
  out.clear();
  double dh2 = e.P.dhat * e.P.dhat;
  for (auto& c : cands) {
    Contact k;
    k.kind = c[0];
    cand_points(e, c, k.pts);
    double x12[12];
    gather12(px, k.pts, x12);
    double d2 = pair_dist2(k.kind, x12, &k.type);
    if (!(d2 < dh2)) continue;
    k.eps_x = k.kind == 1 ? 1e-3 * rest_len2(e, k.pts[0], k.pts[1]) * rest_len2(e, k.pts[2], k.pts[3]) : 0.0;
    out.push_back(k);
  }
}

// ---------------------------------------------------------------- energy, gradient, Hessian
struct Triplets {
  std::vector<int> r, c;
  std::vector<double> v;
  void add(int i, int j, double x) {
    if (x == 0.0) return;
    r.push_back(i); c.push_back(j); v.push_back(x);
  }
};

static bool is_kin_dof(const Env& e, int d) {
  if (d < 3 * e.n_soft_verts) return e.vkin[d / 3];
  return e.bodies[(d - 3 * e.n_soft_verts) / 12].kin;
}

// Total incremental potential at DOFs q (with the constraint set already computed at q).
// want: 0 energy only, 1 + gradient, 2 + Hessian (PSD-projected per element).
// Returns +inf if some tet is inverted (J <= 0).
static double evaluate(Env& e, const std::vector<double>& q, const std::vector<Contact>& C, int want,
                       std::vector<double>* grad, Triplets* H) {
  const double h = e.P.dt, h2 = h * h;
  double Einert = 0, Eelas = 0, Ebar = 0, Efric = 0, Eorth = 0, Epd = 0, Ejoint = 0;
  if (grad) grad->assign(e.ndof, 0.0);
  // inertia of free soft vertices
  for (int i = 0; i < e.n_soft_verts; ++i) {
    if (e.vkin[i]) continue;
    for (int k = 0; k < 3; ++k) {
      double d = q[3 * i + k] - e.xtilde[3 * i + k];
      Einert += 0.5 * e.mass[i] * d * d;
      if (want >= 1) (*grad)[3 * i + k] += e.mass[i] * d;
      if (want >= 2) H->add(3 * i + k, 3 * i + k, e.mass[i]);
    }
  }
  // elastic tets: F = Ds Dm^-1, derivatives of psi over F by AD, projected 9x9, mapped to x
  for (size_t t = 0; t < e.tets.size(); ++t) {
    const auto& T = e.tets[t];
    const auto& Bi = e.Dminv[t];
    double Ds[9];
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) Ds[3 * r + c] = q[3 * T[c + 1] + r] - q[3 * T[0] + r];
    double F[9];
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) F[3 * r + c] = Ds[3 * r] * Bi[c] + Ds[3 * r + 1] * Bi[3 + c] + Ds[3 * r + 2] * Bi[6 + c];
    double J = F[0] * (F[4] * F[8] - F[5] * F[7]) - F[1] * (F[3] * F[8] - F[5] * F[6]) + F[2] * (F[3] * F[7] - F[4] * F[6]);
    if (!(J > 0.0)) return std::numeric_limits<double>::infinity();
    double w = h2 * e.tvol[t];
    if (want == 0) {
      Eelas += w * neo_hookean(F, e.tmu[t], e.tlam[t]);
      continue;
    }
    Dual<9> Fd[9];
    for (int i = 0; i < 9; ++i) Fd[i] = Dual<9>::var(i, F[i]);
    Dual<9> psi = neo_hookean(Fd, e.tmu[t], e.tlam[t]);
    Eelas += w * psi.v;
    // shape-function gradients B[i][c]: F_rc = sum_i x_{i,r} B[i][c]
    double B[4][3];
    for (int c = 0; c < 3; ++c) {
      B[1][c] = Bi[c]; B[2][c] = Bi[3 + c]; B[3][c] = Bi[6 + c];
      B[0][c] = -(B[1][c] + B[2][c] + B[3][c]);
    }
    for (int i = 0; i < 4; ++i)
      for (int s = 0; s < 3; ++s) {
        double g = 0;
        for (int c = 0; c < 3; ++c) g += psi.g[3 * s + c] * B[i][c];
        (*grad)[3 * T[i] + s] += w * g;
      }
    if (want >= 2) {
      double HF[81];
      for (int i = 0; i < 81; ++i) HF[i] = psi.h[i];
      project_psd(9, HF);
      for (int i = 0; i < 4; ++i)
        for (int s = 0; s < 3; ++s)
          for (int j = 0; j < 4; ++j)
            for (int u = 0; u < 3; ++u) {
              double acc = 0;
              for (int c = 0; c < 3; ++c)
                for (int d = 0; d < 3; ++d) acc += B[i][c] * HF[(3 * s + c) * 9 + 3 * u + d] * B[j][d];
              H->add(3 * T[i] + s, 3 * T[j] + u, w * acc);
            }
    }
  }
  // affine bodies: inertia 1/2 (q - qt)^T (M4 x I3) (q - qt) and h^2 kappa_A V |A A^T - I|^2
  for (const Body& B : e.bodies) {
    if (B.kin) continue;
    const double* qb = q.data() + B.dof;
    const double* qt = e.xtilde.data() + B.dof;
    for (int I = 0; I < 4; ++I)
      for (int Jn = 0; Jn < 4; ++Jn)
        for (int k = 0; k < 3; ++k) {
          double m = B.M4[4 * I + Jn];
          Einert += 0.5 * (qb[3 * I + k] - qt[3 * I + k]) * m * (qb[3 * Jn + k] - qt[3 * Jn + k]);
          if (want >= 1) (*grad)[B.dof + 3 * I + k] += m * (qb[3 * Jn + k] - qt[3 * Jn + k]);
          if (want >= 2) H->add(B.dof + 3 * I + k, B.dof + 3 * Jn + k, m);
        }
    // PD target potential 1/2 h^2 k_pd (q - q^)^T (M4 x I3) (q - q^) = 1/2 h^2 k_pd int rho |x - x^|^2,
    // q^ the body's scheduled coordinates for this step
    if (B.kpd > 0.0) {
      const int st = std::min(e.step, e.n_steps - 1);
      const double* qh = e.targets.data() + ((size_t)st * e.n_handles + B.handle) * 12;
      const double w = h2 * B.kpd;
      for (int I = 0; I < 4; ++I)
        for (int Jn = 0; Jn < 4; ++Jn)
          for (int k = 0; k < 3; ++k) {
            double m = B.M4[4 * I + Jn];
            Epd += 0.5 * w * (qb[3 * I + k] - qh[3 * I + k]) * m * (qb[3 * Jn + k] - qh[3 * Jn + k]);
            if (want >= 1) (*grad)[B.dof + 3 * I + k] += w * m * (qb[3 * Jn + k] - qh[3 * Jn + k]);
            if (want >= 2) H->add(B.dof + 3 * I + k, B.dof + 3 * Jn + k, w * m);
          }
    }
    // A[r][c] = a_c[r] = q[3 + 3c + r]
    Dual<9> A[9];
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) A[3 * r + c] = Dual<9>::var(3 * r + c, qb[3 + 3 * c + r]);
    Dual<9> E(0.0);
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        Dual<9> s = A[3 * i] * A[3 * j] + A[3 * i + 1] * A[3 * j + 1] + A[3 * i + 2] * A[3 * j + 2];
        if (i == j) s = s - Dual<9>(1.0);
        E = E + s * s;
      }
    double w = h2 * e.P.kappa_affine * B.vol;
    Eorth += w * E.v;
    auto qidx = [&](int a) { int r = a / 3, c = a % 3; return B.dof + 3 + 3 * c + r; };
    if (want >= 1)
      for (int a = 0; a < 9; ++a) (*grad)[qidx(a)] += w * E.g[a];
    if (want >= 2) {
      double HA[81];
      for (int i = 0; i < 81; ++i) HA[i] = E.h[i];
      project_psd(9, HA);
      for (int a = 0; a < 9; ++a)
        for (int b = 0; b < 9; ++b) H->add(qidx(a), qidx(b), w * HA[9 * a + b]);
    }
  }
  // joints: 1/2 h^2 k |x_a - x_b|^2 with x = p + A xbar for each anchor. With the weights
  // w = (1, xbar) of the blocks (p, a1, a2, a3) of q, x = sum_r w_r q_r, so the gradient on block
  // r of body a is h^2 k w_r (x_a - x_b) and the Hessian block (r, s) is h^2 k w_r w_s I3 (with a
  // minus sign between the two bodies): PSD as it stands, not projected.
  for (const Joint& J : e.joints) {
    const Body& Ba = e.bodies[J.a];
    const Body& Bb = e.bodies[J.b];
    const double wa[4] = {1.0, J.xa[0], J.xa[1], J.xa[2]}, wb[4] = {1.0, J.xb[0], J.xb[1], J.xb[2]};
    double r[3];
    for (int k = 0; k < 3; ++k) {
      double xa = 0.0, xb = 0.0;
      for (int m = 0; m < 4; ++m) {
        xa += wa[m] * q[Ba.dof + 3 * m + k];
        xb += wb[m] * q[Bb.dof + 3 * m + k];
      }
      r[k] = xa - xb;
    }
    const double c = h2 * J.k;
    Ejoint += 0.5 * c * (r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    const int dofs[2] = {Ba.dof, Bb.dof};
    const double* ws[2] = {wa, wb};
    const double sg[2] = {1.0, -1.0};
    if (want >= 1)
      for (int side = 0; side < 2; ++side)
        for (int m = 0; m < 4; ++m)
          for (int k = 0; k < 3; ++k) (*grad)[dofs[side] + 3 * m + k] += sg[side] * c * ws[side][m] * r[k];
    if (want >= 2)
      for (int s1 = 0; s1 < 2; ++s1)
        for (int s2 = 0; s2 < 2; ++s2)
          for (int m = 0; m < 4; ++m)
            for (int n = 0; n < 4; ++n)
              for (int k = 0; k < 3; ++k)
                H->add(dofs[s1] + 3 * m + k, dofs[s2] + 3 * n + k, sg[s1] * sg[s2] * c * ws[s1][m] * ws[s2][n]);
  }
  // contacts: barrier
  std::vector<double> px;
  point_positions(e, q.data(), px);
  auto scatter = [&](const int pts[4], const double* g12, const double* H12, double scale) {
    PointMap m[4];
    for (int a = 0; a < 4; ++a) m[a] = point_map(e, pts[a]);
    if (want >= 1)
      for (int a = 0; a < 4; ++a)
        for (int r = 0; r < m[a].n; ++r)
          for (int k = 0; k < 3; ++k) (*grad)[m[a].dof[r] + k] += scale * m[a].w[r] * g12[3 * a + k];
    if (want >= 2)
      for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b)
          for (int r = 0; r < m[a].n; ++r)
            for (int s = 0; s < m[b].n; ++s)
              for (int k = 0; k < 3; ++k)
                for (int l = 0; l < 3; ++l)
                  H->add(m[a].dof[r] + k, m[b].dof[s] + l,
                         scale * m[a].w[r] * m[b].w[s] * H12[(3 * a + k) * 12 + 3 * b + l]);
  };
  for (const Contact& c : C) {
    double x12[12];
    gather12(px, c.pts, x12);
    if (want == 0) {
      Ebar += h2 * contact_barrier_energy(c.kind, x12, e.P.dhat, e.kappa, c.eps_x, c.type);
      continue;
    }
    Dual<12> X[12];
    for (int i = 0; i < 12; ++i) X[i] = Dual<12>::var(i, x12[i]);
    Dual<12> E = contact_barrier_energy(c.kind, X, e.P.dhat, e.kappa, c.eps_x, c.type);
    Ebar += h2 * E.v;
    double H12[144];
    for (int i = 0; i < 144; ++i) H12[i] = E.h[i];
    if (want >= 2) project_psd(12, H12);
    scatter(c.pts, E.g.data(), H12, h2);
  }
  // lagged friction: h^2 mu lambda f0(|P rel|), rel = sum_i c_i (x_i - x_i^t), P = I - n n^T
  const double eh = e.P.eps_v * h;
  for (const FrictionContact& f : e.fric) {
    double rel[3] = {0, 0, 0};
    for (int a = 0; a < 4; ++a)
      for (int k = 0; k < 3; ++k) rel[k] += f.c[a] * (px[3 * f.pts[a] + k] - e.ptx_t[3 * f.pts[a] + k]);
    double nr = d3dot(f.n, rel);
    double u[3] = {rel[0] - nr * f.n[0], rel[1] - nr * f.n[1], rel[2] - nr * f.n[2]};
    double y = std::sqrt(d3dot(u, u));
    double f0, f1, f2;
    friction_f(y, eh, &f0, &f1, &f2);
    double s = h2 * e.mu * f.lambda;
    Efric += s * f0;
    if (want == 0) continue;
    double a = y > 0 ? f1 / y : 2.0 / eh;  // f1(y)/y, with its limit 2/eh at y = 0
    double bcoef = y > 0 ? (f2 * y - f1) / (y * y * y) : 0.0;
    double g12[12], H12[144];
    for (int i = 0; i < 4; ++i)
      for (int k = 0; k < 3; ++k) g12[3 * i + k] = f.c[i] * a * u[k];
    double M[9];
    for (int k = 0; k < 3; ++k)
      for (int l = 0; l < 3; ++l) M[3 * k + l] = a * ((k == l ? 1.0 : 0.0) - f.n[k] * f.n[l]) + bcoef * u[k] * u[l];
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j)
        for (int k = 0; k < 3; ++k)
          for (int l = 0; l < 3; ++l) H12[(3 * i + k) * 12 + 3 * j + l] = f.c[i] * f.c[j] * M[3 * k + l];
    scatter(f.pts, g12, H12, s);
  }
  return Einert + Eelas + Eorth + Epd + Ejoint + Ebar + Efric;
}

// ---------------------------------------------------------------- step pieces
static void target_dofs(const Env& e, std::vector<double>& tgt) {
  // kinematic DOF targets for the current step (non-kinematic entries are untouched copies of x)
  tgt = e.x;
  const int s = std::min(e.step, e.n_steps - 1);  // a finished env keeps its last schedule entry
  const double* T = e.targets.data() + (size_t)s * e.n_handles * 12;
  for (int i = 0; i < e.n_soft_verts; ++i) {
    if (!e.vkin[i]) continue;
    const double* qb = T + 12 * e.vhandle[i];
    for (int k = 0; k < 3; ++k) {
      double r = qb[k] + e.X0[3 * i] * qb[3 + k];
      r = r + e.X0[3 * i + 1] * qb[6 + k];
      r = r + e.X0[3 * i + 2] * qb[9 + k];
      tgt[3 * i + k] = r;
    }
  }
  for (const Body& B : e.bodies)
    if (B.kin)
      for (int k = 0; k < 12; ++k) tgt[B.dof + k] = T[12 * B.handle + k];
}

// Barrier stiffness at the start of a step (reading of the adapted-stiffness rule): with g_E the
// gradient of every other term of the incremental potential at x^t and G the gradient of the
// barrier term per unit stiffness, the kappa that minimises |g_E + kappa G| over the free DOFs,
// -(g_E . G) / (G . G), clamped to [kappa, 1000 kappa] of the scene; the scene's kappa when no
// pair is within dhat. Also records the smallest contact distance at x^t.
static void kappa_start(Env& e, const std::vector<Contact>& C) {
  if (C.empty()) return;
  std::vector<double> g0(e.ndof, 0.0), g1(e.ndof, 0.0);
  e.kappa = 0.0;
  evaluate(e, e.x, C, 1, &g0, nullptr);
  e.kappa = 1.0;
  evaluate(e, e.x, C, 1, &g1, nullptr);
  double eg = 0.0, gg = 0.0;
  for (int d = 0; d < e.ndof; ++d) {
    if (is_kin_dof(e, d)) continue;
    const double G = g1[d] - g0[d];
    eg += g0[d] * G;
    gg += G * G;
  }
  e.kappa = e.P.kappa;
  if (gg > 0.0) {
    const double k = -eg / gg;
    if (std::isfinite(k)) e.kappa = std::min(std::max(k, e.P.kappa), 1000.0 * e.P.kappa);
  }
}

static void step_setup(Env& e) {
  const double h = e.P.dt;
  e.xt = e.x;
  e.xtilde.assign(e.ndof, 0.0);
  // gravity of the step: 0 none, 1 the scene's vector, 2..7 its magnitude along +x, -x, +y, -y,
  // +z, -z (the axis-aligned phases of the grasp evaluation protocol, Sec. III-D)
  const int code = e.gravity[std::min(e.step, e.n_steps - 1)];
  double hh = code ? h * h : 0.0;
  double g[3] = {e.P.gravity[0], e.P.gravity[1], e.P.gravity[2]};
  if (code >= 2) {
    const double gm = std::sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
    g[0] = g[1] = g[2] = 0.0;
    g[(code - 2) / 2] = code % 2 == 0 ? gm : -gm;
  }
  for (int i = 0; i < e.n_soft_verts; ++i)
    for (int k = 0; k < 3; ++k) e.xtilde[3 * i + k] = (e.x[3 * i + k] + h * e.v[3 * i + k]) + hh * g[k];
  for (const Body& B : e.bodies)
    for (int k = 0; k < 12; ++k) {
      double r = e.x[B.dof + k] + h * e.v[B.dof + k];
      if (k < 3) r = r + hh * g[k];
      e.xtilde[B.dof + k] = r;
    }
  // friction lagged at x^t: normal force lambda = kappa e |b'(d)|, closest-point data
  point_positions(e, e.x.data(), e.ptx_t);
  std::vector<Contact> C;
  constraint_set(e, e.ptx_t, C);
  e.fric.clear();
  e.kappa = e.P.kappa;
  if (e.P.kappa_adapt) kappa_start(e, C);
  for (const Contact& c : C) {
    double x12[12];
    gather12(e.ptx_t, c.pts, x12);
    double d = std::sqrt(pair_dist2(c.kind, x12));
    double b, b1, b2;
    barrier_derivs(d, e.P.dhat, &b, &b1, &b2);
    double moll = 1.0;
    if (c.kind == 1) {
      V3<double> P[4];
      for (int i = 0; i < 4; ++i) P[i] = {x12[3 * i], x12[3 * i + 1], x12[3 * i + 2]};
      moll = mollifier(P[0], P[1], P[2], P[3], c.eps_x);
    }
    FrictionContact f;
    for (int i = 0; i < 4; ++i) f.pts[i] = c.pts[i];
    pair_closest(c.kind, x12, f.c, f.n);
    f.lambda = e.kappa * moll * std::fabs(b1);
    e.fric.push_back(f);
  }
}

// CSR from triplets restricted to all DOFs
struct CSR {
  int n;
  std::vector<int> rp, ci;
  std::vector<double> val;
};
static CSR to_csr(int n, const Triplets& T) {
  std::vector<size_t> idx(T.r.size());
  for (size_t i = 0; i < idx.size(); ++i) idx[i] = i;
  std::sort(idx.begin(), idx.end(), [&](size_t a, size_t b) {
    return T.r[a] != T.r[b] ? T.r[a] < T.r[b] : (T.c[a] != T.c[b] ? T.c[a] < T.c[b] : a < b);
  });
  CSR M;
  M.n = n;
  M.rp.assign(n + 1, 0);
  int lr = -1, lc = -1;
  for (size_t k : idx) {
    if (T.r[k] == lr && T.c[k] == lc) {
      M.val.back() += T.v[k];
      continue;
    }
    lr = T.r[k];
    lc = T.c[k];
    M.ci.push_back(lc);
    M.val.push_back(T.v[k]);
    M.rp[lr + 1]++;
  }
  for (int i = 0; i < n; ++i) M.rp[i + 1] += M.rp[i];
  return M;
}
static void csr_mv(const CSR& M, const std::vector<double>& x, std::vector<double>& y) {
  y.assign(M.n, 0.0);
  for (int i = 0; i < M.n; ++i) {
    double s = 0;
    for (int k = M.rp[i]; k < M.rp[i + 1]; ++k) s += M.val[k] * x[M.ci[k]];
    y[i] = s;
  }
}

// Conjugate gradients on the free DOFs (mask=1), Jacobi preconditioner, x0 = 0.
static long cg_solve(const CSR& M, const std::vector<int>& free_mask, const std::vector<double>& b, std::vector<double>& x,
                     double rel_tol, long max_it) {
  int n = M.n;
  x.assign(n, 0.0);
  std::vector<double> r(n), z(n), p(n), Ap(n), dinv(n, 0.0);
  for (int i = 0; i < n; ++i) {
    r[i] = free_mask[i] ? b[i] : 0.0;
    double d = 0;
    for (int k = M.rp[i]; k < M.rp[i + 1]; ++k)
      if (M.ci[k] == i) d = M.val[k];
    dinv[i] = (free_mask[i] && d > 0) ? 1.0 / d : 0.0;
  }
  double bn = 0;
  for (int i = 0; i < n; ++i) bn += r[i] * r[i];
  bn = std::sqrt(bn);
  if (bn == 0.0) return 0;
  for (int i = 0; i < n; ++i) { z[i] = dinv[i] * r[i]; p[i] = z[i]; }
  double rz = 0;
  for (int i = 0; i < n; ++i) rz += r[i] * z[i];
  long it = 0;
  for (; it < max_it; ++it) {
    csr_mv(M, p, Ap);
    for (int i = 0; i < n; ++i)
      if (!free_mask[i]) Ap[i] = 0.0;
    double pAp = 0;
    for (int i = 0; i < n; ++i) pAp += p[i] * Ap[i];
    if (!(pAp > 0)) break;
    double alpha = rz / pAp;
    double rn = 0;
    for (int i = 0; i < n; ++i) {
      x[i] += alpha * p[i];
      r[i] -= alpha * Ap[i];
      rn += r[i] * r[i];
    }
    if (std::sqrt(rn) <= rel_tol * bn) { ++it; break; }
    double rz2 = 0;
    for (int i = 0; i < n; ++i) { z[i] = dinv[i] * r[i]; rz2 += r[i] * z[i]; }
    double beta = rz2 / rz;
    rz = rz2;
    for (int i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
  }
  return it;
}

static bool all_tets_positive(const Env& e, const std::vector<double>& q) {
  for (size_t t = 0; t < e.tets.size(); ++t) {
    const auto& T = e.tets[t];
    double d[3][3];
    for (int c = 0; c < 3; ++c)
      for (int r = 0; r < 3; ++r) d[c][r] = q[3 * T[c + 1] + r] - q[3 * T[0] + r];
    double J = d[0][0] * (d[1][1] * d[2][2] - d[1][2] * d[2][1]) - d[0][1] * (d[1][0] * d[2][2] - d[1][2] * d[2][0]) +
               d[0][2] * (d[1][0] * d[2][1] - d[1][1] * d[2][0]);
    if (!(J > 0)) return false;
  }
  return true;
}

// largest collision-free step fraction over the swept candidates (ACCD), at most 1
static double ccd_alpha(Env& e, const std::vector<double>& q, const std::vector<double>& p) {
  std::vector<double> px, pp, pe;
  point_positions(e, q.data(), px);
  point_displacements(e, p.data(), pp);
  pe.resize(px.size());
  for (size_t i = 0; i < px.size(); ++i) pe[i] = px[i] + pp[i];
  std::vector<std::array<int, 3>> cands;
  candidates(e, px, &pe, 0.0, cands);
  double amax = 1.0;
  for (auto& c : cands) {
    int pts[4];
    cand_points(e, c, pts);
    double x12[12], p12[12];
    gather12(px, pts, x12);
    gather12(pp, pts, p12);
    long it = 0;
    double t = accd(c[0], x12, p12, 0.1, 1.0, 1000000, &it);
    e.accd_iters += it;
    amax = std::min(amax, t);
  }
  return amax;
}

// infinity norm of the Newton step in world space over the free DOFs
static double step_norm(const Env& e, const std::vector<double>& p) {
  double m = 0;
  for (int i = 0; i < e.n_soft_verts; ++i)
    if (!e.vkin[i])
      for (int k = 0; k < 3; ++k) m = std::max(m, std::fabs(p[3 * i + k]));
  for (const Body& B : e.bodies) {
    if (B.kin) continue;
    const double* pb = p.data() + B.dof;
    for (int c = 0; c < 8; ++c) {
      double xb[3] = {(c & 1) ? B.hi[0] : B.lo[0], (c & 2) ? B.hi[1] : B.lo[1], (c & 4) ? B.hi[2] : B.lo[2]};
      for (int k = 0; k < 3; ++k) {
        double r = pb[k] + xb[0] * pb[3 + k];
        r = r + xb[1] * pb[6 + k];
        r = r + xb[2] * pb[9 + k];
        m = std::max(m, std::fabs(r));
      }
    }
  }
  return m;
}

// one time step of one environment (Newton loop with CCD-filtered backtracking line search)
static void step_once(Env& e) {
  if (e.status != ST_ACTIVE) return;
  const double h = e.P.dt;
  step_setup(e);
  std::vector<double> tgt;
  target_dofs(e, tgt);
  std::vector<int> free_mask(e.ndof);
  for (int d = 0; d < e.ndof; ++d) free_mask[d] = !is_kin_dof(e, d);
  std::vector<double> px, grad, p(e.ndof), qtrial(e.ndof), Hpbar, rhs(e.ndof), delta;
  std::vector<Contact> C;
  bool converged = false;
  for (int it = 0; it < e.P.max_newton; ++it) {
    point_positions(e, e.x.data(), px);
    constraint_set(e, px, C);
    Triplets T;
    double E0 = evaluate(e, e.x, C, 2, &grad, &T);
    if (!std::isfinite(E0)) { e.status = ST_FAILED; e.reason = FAIL_NAN; return; }
    CSR M = to_csr(e.ndof, T);
    // kinematic part of the step and the reduced right-hand side -g_F - H_FD p_D
    std::vector<double> pbar(e.ndof, 0.0);
    bool constrained = false;
    for (int d = 0; d < e.ndof; ++d)
      if (!free_mask[d]) {
        pbar[d] = tgt[d] - e.x[d];
        if (pbar[d] != 0.0) constrained = true;
      }
    if (e.trace) {
      e.trace_E.push_back((double)e.step);
      e.trace_E.push_back((double)it);
      e.trace_E.push_back(constrained ? 1.0 : 0.0);
      e.trace_E.push_back(E0);
    }
    csr_mv(M, pbar, Hpbar);
    for (int d = 0; d < e.ndof; ++d) rhs[d] = free_mask[d] ? -grad[d] - Hpbar[d] : 0.0;
    e.cg_iters += cg_solve(M, free_mask, rhs, delta, 1e-12, 20L * e.ndof + 1000);
    for (int d = 0; d < e.ndof; ++d) p[d] = free_mask[d] ? delta[d] : pbar[d];
    e.newton_iters++;
    for (double v : p)
      if (!std::isfinite(v)) { e.status = ST_FAILED; e.reason = FAIL_NAN; return; }
    if (!constrained && step_norm(e, p) / h < e.P.newton_tol) { converged = true; break; }
    double alpha = ccd_alpha(e, e.x, p);
    int halvings = 0;
    while (true) {
      for (int d = 0; d < e.ndof; ++d) qtrial[d] = e.x[d] + alpha * p[d];
      bool ok = all_tets_positive(e, qtrial);
      if (ok && !constrained) {
        std::vector<double> pxt;
        point_positions(e, qtrial.data(), pxt);
        std::vector<Contact> Ct;
        constraint_set(e, pxt, Ct);
        double E1 = evaluate(e, qtrial, Ct, 0, nullptr, nullptr);
        ok = E1 <= E0;
      }
      if (ok) break;
      if (++halvings > e.P.max_ls) { e.status = ST_FAILED; e.reason = FAIL_LINESEARCH; return; }
      e.ls_halvings++;
      alpha = alpha / 2.0;
    }
    e.last_alpha = alpha;
    e.x = qtrial;
    if (constrained && alpha == 1.0)
      for (int d = 0; d < e.ndof; ++d)
        if (!free_mask[d]) e.x[d] = tgt[d];
  }
  if (!converged) { e.status = ST_FAILED; e.reason = FAIL_NEWTON; return; }
  for (int d = 0; d < e.ndof; ++d) e.v[d] = (e.x[d] - e.xt[d]) / h;
  e.step++;
  e.steps_done++;
  if (e.step >= e.n_steps) e.status = ST_DONE;
}

// proper segment-triangle crossing (Moller-Trumbore on the segment). Near-parallel segments
// and hits within a relative 1e-9 of the triangle boundary or the segment ends are not
// counted (coplanar or touching configurations); touching is covered by the distance invariant.
static bool seg_tri(const double* s0, const double* s1, const double* a, const double* b, const double* c) {
  double e1[3], e2[3], d[3], pv[3], tv[3], qv[3], n[3];
  for (int k = 0; k < 3; ++k) { e1[k] = b[k] - a[k]; e2[k] = c[k] - a[k]; d[k] = s1[k] - s0[k]; }
  n[0] = e1[1] * e2[2] - e1[2] * e2[1]; n[1] = e1[2] * e2[0] - e1[0] * e2[2]; n[2] = e1[0] * e2[1] - e1[1] * e2[0];
  pv[0] = d[1] * e2[2] - d[2] * e2[1]; pv[1] = d[2] * e2[0] - d[0] * e2[2]; pv[2] = d[0] * e2[1] - d[1] * e2[0];
  double det = d3dot(e1, pv);
  if (std::fabs(det) <= 1e-9 * std::sqrt(d3dot(n, n) * d3dot(d, d))) return false;
  double inv = 1.0 / det;
  for (int k = 0; k < 3; ++k) tv[k] = s0[k] - a[k];
  const double eps = 1e-9;
  double u = d3dot(tv, pv) * inv;
  if (u <= eps || u >= 1 - eps) return false;
  qv[0] = tv[1] * e1[2] - tv[2] * e1[1]; qv[1] = tv[2] * e1[0] - tv[0] * e1[2]; qv[2] = tv[0] * e1[1] - tv[1] * e1[0];
  double v = d3dot(d, qv) * inv;
  if (v <= eps || u + v >= 1 - eps) return false;
  double t = d3dot(e2, qv) * inv;
  return t > eps && t < 1 - eps;
}

}  // namespace orc

using namespace orc;

// ================================================================= C interface (ctypes)
extern "C" {

void* or_env_create(const Params* P, const EnvDesc* D) { return build_env(*P, *D); }
void or_env_destroy(void* h) { delete (Env*)h; }
double or_env_kappa(void* h) { return ((Env*)h)->kappa; }
// Von Mises stress of every tet at DOFs q: the Cauchy stress of the Neo-Hookean energy is
// sigma = P F^T / J with P = mu (F - F^-T) + lam ln J F^-T, i.e. (mu (F F^T - I) + lam ln J I) / J,
// and von Mises = sqrt(3/2 s:s) of its deviator s.
void or_env_tet_stress(void* h, const double* q, double* out) {
  const Env& e = *(const Env*)h;
  for (size_t t = 0; t < e.tets.size(); ++t) {
    const auto& T = e.tets[t];
    const auto& Bi = e.Dminv[t];
    double Ds[9], F[9];
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) Ds[3 * r + c] = q[3 * T[c + 1] + r] - q[3 * T[0] + r];
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) F[3 * r + c] = Ds[3 * r] * Bi[c] + Ds[3 * r + 1] * Bi[3 + c] + Ds[3 * r + 2] * Bi[6 + c];
    const double J = F[0] * (F[4] * F[8] - F[5] * F[7]) - F[1] * (F[3] * F[8] - F[5] * F[6]) + F[2] * (F[3] * F[7] - F[4] * F[6]);
    double sig[9];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        double b = 0.0;
        for (int k = 0; k < 3; ++k) b += F[3 * i + k] * F[3 * j + k];
        sig[3 * i + j] = (e.tmu[t] * (b - (i == j ? 1.0 : 0.0)) + (i == j ? e.tlam[t] * std::log(J) : 0.0)) / J;
      }
    const double p = (sig[0] + sig[4] + sig[8]) / 3.0;
    double ss = 0.0;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        const double d = sig[3 * i + j] - (i == j ? p : 0.0);
        ss += d * d;
      }
    out[t] = std::sqrt(1.5 * ss);
  }
}
int or_env_ndof(void* h) { return ((Env*)h)->ndof; }
int or_env_npoints(void* h) { return (int)((Env*)h)->pts.size(); }

// advance n steps; returns the status
int or_env_step(void* h, int n) {
  Env* e = (Env*)h;
  for (int i = 0; i < n && e->status == ST_ACTIVE; ++i) step_once(*e);
  return e->status;
}

// advance several environments on n_threads host threads (one env at a time per thread)
void or_run_batch(void** hs, int n_env, int n_steps, int n_threads) {
  std::atomic<int> next(0);
  auto work = [&]() {
    for (int i = next++; i < n_env; i = next++) or_env_step(hs[i], n_steps);
  };
  std::vector<std::thread> th;
  for (int t = 0; t < std::max(1, n_threads); ++t) th.emplace_back(work);
  for (auto& t : th) t.join();
}

void or_env_get_state(void* h, double* x, double* v) {
  Env* e = (Env*)h;
  if (x) std::memcpy(x, e->x.data(), sizeof(double) * e->ndof);
  if (v) std::memcpy(v, e->v.data(), sizeof(double) * e->ndof);
}
void or_env_set_state(void* h, const double* x, const double* v, int step) {
  Env* e = (Env*)h;
  std::memcpy(e->x.data(), x, sizeof(double) * e->ndof);
  std::memcpy(e->v.data(), v, sizeof(double) * e->ndof);
  e->step = step;
  e->status = step >= e->n_steps ? ST_DONE : ST_ACTIVE;
  e->reason = FAIL_NONE;
}
// status[0..2] = status, reason, steps_done; stats = newton, ls halvings, cg iters, accd iters
void or_env_status(void* h, int* st, long* stats, double* last_alpha) {
  Env* e = (Env*)h;
  st[0] = e->status; st[1] = e->reason; st[2] = (int)e->steps_done; st[3] = e->step;
  stats[0] = e->newton_iters; stats[1] = e->ls_halvings; stats[2] = e->cg_iters; stats[3] = e->accd_iters;
  *last_alpha = e->last_alpha;
}

// Energy and gradient at DOFs q, with x^t, v^t = the current state (step setup done here:
// predicted positions and friction lagged at x^t). Returns the energy.
double or_env_eval(void* h, const double* q, double* grad) {
  Env* e = (Env*)h;
  step_setup(*e);
  std::vector<double> qq(q, q + e->ndof), px, g;
  point_positions(*e, qq.data(), px);
  std::vector<Contact> C;
  constraint_set(*e, px, C);
  double E = evaluate(*e, qq, C, grad ? 1 : 0, grad ? &g : nullptr, nullptr);
  if (grad) std::memcpy(grad, g.data(), sizeof(double) * e->ndof);
  return E;
}

// Newton direction of the first iteration of the env's next step, taken at its current state
// (kinematic part target - x, free part from the CG solve of the projected Hessian system).
void or_env_newton_dir(void* h, double* out) {
  Env* e = (Env*)h;
  step_setup(*e);
  std::vector<double> tgt, px, grad, Hpbar, rhs(e->ndof), delta;
  target_dofs(*e, tgt);
  std::vector<int> free_mask(e->ndof);
  for (int d = 0; d < e->ndof; ++d) free_mask[d] = !is_kin_dof(*e, d);
  point_positions(*e, e->x.data(), px);
  std::vector<Contact> C;
  constraint_set(*e, px, C);
  Triplets T;
  evaluate(*e, e->x, C, 2, &grad, &T);
  CSR M = to_csr(e->ndof, T);
  std::vector<double> pbar(e->ndof, 0.0);
  for (int d = 0; d < e->ndof; ++d)
    if (!free_mask[d]) pbar[d] = tgt[d] - e->x[d];
  csr_mv(M, pbar, Hpbar);
  for (int d = 0; d < e->ndof; ++d) rhs[d] = free_mask[d] ? -grad[d] - Hpbar[d] : 0.0;
  cg_solve(M, free_mask, rhs, delta, 1e-12, 20L * e->ndof + 1000);
  for (int d = 0; d < e->ndof; ++d) out[d] = free_mask[d] ? delta[d] : pbar[d];
}

// Dense Hessian (PSD-projected) at q; for small systems in tests. out is ndof*ndof.
void or_env_hessian(void* h, const double* q, double* out) {
  Env* e = (Env*)h;
  step_setup(*e);
  std::vector<double> qq(q, q + e->ndof), px, g;
  point_positions(*e, qq.data(), px);
  std::vector<Contact> C;
  constraint_set(*e, px, C);
  Triplets T;
  evaluate(*e, qq, C, 2, &g, &T);
  std::memset(out, 0, sizeof(double) * e->ndof * e->ndof);
  for (size_t k = 0; k < T.r.size(); ++k) out[(size_t)T.r[k] * e->ndof + T.c[k]] += T.v[k];
}

// Candidate list at q (r = dhat/2) or swept over [q, q + p] (p != null, r = 0).
// out rows: kind, i, j (sorted); returns the count (writes at most cap rows).
int or_env_candidates(void* h, const double* q, const double* p, int32_t* out, int cap) {
  Env* e = (Env*)h;
  std::vector<double> px, pp, pe;
  point_positions(*e, q, px);
  std::vector<std::array<int, 3>> c;
  if (p) {
    point_displacements(*e, p, pp);
    pe.resize(px.size());
    for (size_t i = 0; i < px.size(); ++i) pe[i] = px[i] + pp[i];
    candidates(*e, px, &pe, 0.0, c);
  } else {
    candidates(*e, px, nullptr, 0.5 * e->P.dhat, c);
  }
  std::sort(c.begin(), c.end());
  for (int i = 0; i < (int)c.size() && i < cap; ++i)
    for (int k = 0; k < 3; ++k) out[3 * i + k] = c[i][k];
  return (int)c.size();
}
// active constraints at q: rows kind, i, j (of the candidate), type; returns count
int or_env_contacts(void* h, const double* q, int32_t* out, double* d2out, int cap) {
  Env* e = (Env*)h;
  std::vector<double> px;
  point_positions(*e, q, px);
  std::vector<std::array<int, 3>> cands;
  candidates(*e, px, nullptr, 0.5 * e->P.dhat, cands);
  std::sort(cands.begin(), cands.end());
  int n = 0;
  for (auto& c : cands) {
    int pts[4];
    cand_points(*e, c, pts);
    double x12[12];
    gather12(px, pts, x12);
    int type;
    double d2 = pair_dist2(c[0], x12, &type);
    if (!(d2 < e->P.dhat * e->P.dhat)) continue;
    if (n < cap) {
      out[4 * n] = c[0]; out[4 * n + 1] = c[1]; out[4 * n + 2] = c[2]; out[4 * n + 3] = type;
      if (d2out) d2out[n] = d2;
    }
    ++n;
  }
  return n;
}
// Normal force of every contact at q, in or_env_contacts' order: kappa e |b'(d)| (N), with e the
// edge-edge mollifier (1 for point-triangle pairs) and kappa the env's current stiffness.
int or_env_contact_forces(void* h, const double* q, double* out, int cap) {
  Env* e = (Env*)h;
  std::vector<double> px;
  point_positions(*e, q, px);
  std::vector<std::array<int, 3>> cands;
  candidates(*e, px, nullptr, 0.5 * e->P.dhat, cands);
  std::sort(cands.begin(), cands.end());
  int n = 0;
  for (auto& c : cands) {
    int pts[4];
    cand_points(*e, c, pts);
    double x12[12];
    gather12(px, pts, x12);
    double d2 = pair_dist2(c[0], x12);
    if (!(d2 < e->P.dhat * e->P.dhat)) continue;
    double b, b1, b2;
    barrier_derivs(std::sqrt(d2), e->P.dhat, &b, &b1, &b2);
    double moll = 1.0;
    if (c[0] == 1) {
      V3<double> P[4];
      for (int i = 0; i < 4; ++i) P[i] = {x12[3 * i], x12[3 * i + 1], x12[3 * i + 2]};
      moll = mollifier(P[0], P[1], P[2], P[3], 1e-3 * rest_len2(*e, pts[0], pts[1]) * rest_len2(*e, pts[2], pts[3]));
    }
    if (n < cap) out[n] = e->kappa * moll * std::fabs(b1);
    ++n;
  }
  return n;
}
// Bodies of the two sides of every contact at q, in or_env_contacts' order (env-local handles:
// soft bodies first, then affine bodies): the point's and the triangle's, or the two edges'.
int or_env_contact_bodies(void* h, const double* q, int32_t* out, int cap) {
  Env* e = (Env*)h;
  std::vector<double> px;
  point_positions(*e, q, px);
  std::vector<std::array<int, 3>> cands;
  candidates(*e, px, nullptr, 0.5 * e->P.dhat, cands);
  std::sort(cands.begin(), cands.end());
  int n = 0;
  for (auto& c : cands) {
    int pts[4];
    cand_points(*e, c, pts);
    double x12[12];
    gather12(px, pts, x12);
    if (!(pair_dist2(c[0], x12) < e->P.dhat * e->P.dhat)) continue;
    if (n < cap) {
      out[2 * n] = e->pts[pts[0]].body;
      out[2 * n + 1] = e->pts[pts[c[0] == 0 ? 1 : 2]].body;
    }
    ++n;
  }
  return n;
}
// Rewrite rows first .. first + n - 1 of the env's schedule of kinematic targets (n rows of
// (soft + affine bodies) x 12 values); rows outside the schedule are ignored.
void or_env_set_targets(void* h, int first, int n, const double* targets) {
  Env* e = (Env*)h;
  const size_t row = (size_t)e->n_handles * 12;
  for (int r = 0; r < n; ++r) {
    const int s = first + r;
    if (s < 0 || s >= e->n_steps) continue;
    std::copy(targets + r * row, targets + (r + 1) * row, e->targets.begin() + s * row);
  }
}
// Tangential force of every lagged friction stencil of the current (or last) step at DOFs q:
// mu lambda f1(|u|), u the tangential relative displacement since the step start (N).
int or_env_friction_forces(void* h, const double* q, double* out, int cap) {
  Env* e = (Env*)h;
  std::vector<double> px;
  point_positions(*e, q, px);
  const double eh = e->P.eps_v * e->P.dt;
  int n = 0;
  for (const FrictionContact& f : e->fric) {
    double rel[3] = {0, 0, 0};
    for (int a = 0; a < 4; ++a)
      for (int k = 0; k < 3; ++k) rel[k] += f.c[a] * (px[3 * f.pts[a] + k] - e->ptx_t[3 * f.pts[a] + k]);
    double nr = d3dot(f.n, rel);
    double u[3] = {rel[0] - nr * f.n[0], rel[1] - nr * f.n[1], rel[2] - nr * f.n[2]};
    double f0, f1, f2;
    friction_f(std::sqrt(d3dot(u, u)), eh, &f0, &f1, &f2);
    if (n < cap) out[n] = e->mu * f.lambda * f1;
    ++n;
  }
  return n;
}
// world positions of all points at q (npoints x 3)
void or_env_points(void* h, const double* q, double* out) {
  Env* e = (Env*)h;
  std::vector<double> px;
  point_positions(*e, q, px);
  std::memcpy(out, px.data(), sizeof(double) * px.size());
}
// invariants at q: [0] segment-triangle intersections, [1] inverted tets, [2] min PT/EE distance
void or_env_invariants(void* h, const double* q, double* out) {
  Env* e = (Env*)h;
  std::vector<double> px;
  point_positions(*e, q, px);
  std::vector<double> qq(q, q + e->ndof);
  long inter = 0;
  for (auto& ed : e->edges)
    for (auto& t : e->tris) {
      if (ed[0] == t[0] || ed[0] == t[1] || ed[0] == t[2] || ed[1] == t[0] || ed[1] == t[1] || ed[1] == t[2]) continue;
      bool same_aff = e->pts[ed[0]].affine && e->pts[ed[0]].body == e->pts[t[0]].body &&
                      e->pts[ed[1]].body == e->pts[t[0]].body;
      if (same_aff) continue;
      if (seg_tri(&px[3 * ed[0]], &px[3 * ed[1]], &px[3 * t[0]], &px[3 * t[1]], &px[3 * t[2]])) ++inter;
    }
  long inv = 0;
  for (size_t t = 0; t < e->tets.size(); ++t) {
    const auto& T = e->tets[t];
    double d[3][3];
    for (int c = 0; c < 3; ++c)
      for (int r = 0; r < 3; ++r) d[c][r] = qq[3 * T[c + 1] + r] - qq[3 * T[0] + r];
    double J = d[0][0] * (d[1][1] * d[2][2] - d[1][2] * d[2][1]) - d[0][1] * (d[1][0] * d[2][2] - d[1][2] * d[2][0]) +
               d[0][2] * (d[1][0] * d[2][1] - d[1][1] * d[2][0]);
    if (!(J > 0)) ++inv;
  }
  // minimum distance over all non-excluded PT and EE pairs
  double mind = 1e300;
  for (size_t i = 0; i < e->sv.size(); ++i)
    for (auto& t : e->tris) {
      int v = e->sv[i];
      if (t[0] == v || t[1] == v || t[2] == v) continue;
      int p[4] = {v, t[0], t[1], t[2]};
      if (pair_excluded(*e, p)) continue;
      double x12[12];
      gather12(px, p, x12);
      mind = std::min(mind, pair_dist2(0, x12));
    }
  for (size_t i = 0; i < e->edges.size(); ++i)
    for (size_t j = i + 1; j < e->edges.size(); ++j) {
      auto& a = e->edges[i];
      auto& b = e->edges[j];
      if (a[0] == b[0] || a[0] == b[1] || a[1] == b[0] || a[1] == b[1]) continue;
      int p[4] = {a[0], a[1], b[0], b[1]};
      if (pair_excluded(*e, p)) continue;
      double x12[12];
      gather12(px, p, x12);
      mind = std::min(mind, pair_dist2(1, x12));
    }
  out[0] = (double)inter;
  out[1] = (double)inv;
  out[2] = std::sqrt(mind);
}
void or_env_trace(void* h, int on) { ((Env*)h)->trace = on; ((Env*)h)->trace_E.clear(); }
int or_env_trace_get(void* h, double* out, int cap) {
  Env* e = (Env*)h;
  int n = (int)e->trace_E.size();
  for (int i = 0; i < n && i < cap; ++i) out[i] = e->trace_E[i];
  return n;
}
// total mass-matrix data of affine body b: M4 (16) and volume
void or_env_body_mass(void* h, int b, double* M4, double* vol) {
  Env* e = (Env*)h;
  std::memcpy(M4, e->bodies[b].M4, sizeof(double) * 16);
  *vol = e->bodies[b].vol;
}
void or_env_soft_mass(void* h, double* out) {
  Env* e = (Env*)h;
  std::memcpy(out, e->mass.data(), sizeof(double) * e->mass.size());
}

// ---- element-level entry points for the oracle's own pins
void or_neo_hookean(const double* F, double mu, double lam, double* psi, double* P9, double* H81, int project) {
  Dual<9> Fd[9];
  for (int i = 0; i < 9; ++i) Fd[i] = Dual<9>::var(i, F[i]);
  Dual<9> r = neo_hookean(Fd, mu, lam);
  *psi = r.v;
  for (int i = 0; i < 9; ++i) P9[i] = r.g[i];
  for (int i = 0; i < 81; ++i) H81[i] = r.h[i];
  if (project) project_psd(9, H81);
}
void or_project_psd(int n, double* A) { project_psd(n, A); }
void or_eigh(int n, const double* A, double* evals, double* evecs) { jacobi_eigen(n, A, evals, evecs); }
void or_barrier(double d, double dhat, double* out3) { barrier_derivs(d, dhat, &out3[0], &out3[1], &out3[2]); }
// squared distance, its type, gradient and Hessian over the 12 coordinates
double or_pair_dist2(int kind, const double* x12, int* type, double* g12, double* H144) {
  int t;
  double d2 = pair_dist2(kind, x12, &t);
  if (type) *type = t;
  Dual<12> X[12];
  for (int i = 0; i < 12; ++i) X[i] = Dual<12>::var(i, x12[i]);
  V3<Dual<12>> P[4];
  for (int i = 0; i < 4; ++i) P[i] = {X[3 * i], X[3 * i + 1], X[3 * i + 2]};
  Dual<12> r = kind == 0 ? pt_dist2_typed(t, P[0], P[1], P[2], P[3]) : ee_dist2_typed(t, P[0], P[1], P[2], P[3]);
  if (g12) for (int i = 0; i < 12; ++i) g12[i] = r.g[i];
  if (H144) for (int i = 0; i < 144; ++i) H144[i] = r.h[i];
  return d2;
}
// squared distance of a given type (for checking continuity across region boundaries)
double or_pair_dist2_typed(int kind, int type, const double* x12) {
  V3<double> P[4];
  for (int i = 0; i < 4; ++i) P[i] = {x12[3 * i], x12[3 * i + 1], x12[3 * i + 2]};
  return kind == 0 ? pt_dist2_typed(type, P[0], P[1], P[2], P[3]) : ee_dist2_typed(type, P[0], P[1], P[2], P[3]);
}
void or_pair_closest(int kind, const double* x12, double* c4, double* n3) { pair_closest(kind, x12, c4, n3); }
// barrier energy (kappa e b) of one contact, gradient and unprojected Hessian
double or_contact_barrier(int kind, const double* x12, double dhat, double kappa, double eps_x, double* g12, double* H144) {
  int type;
  pair_dist2(kind, x12, &type);
  Dual<12> X[12];
  for (int i = 0; i < 12; ++i) X[i] = Dual<12>::var(i, x12[i]);
  Dual<12> r = contact_barrier_energy(kind, X, dhat, kappa, eps_x, type);
  if (g12) for (int i = 0; i < 12; ++i) g12[i] = r.g[i];
  if (H144) for (int i = 0; i < 144; ++i) H144[i] = r.h[i];
  return r.v;
}
double or_mollifier(const double* x12, double eps) {
  V3<double> P[4];
  for (int i = 0; i < 4; ++i) P[i] = {x12[3 * i], x12[3 * i + 1], x12[3 * i + 2]};
  return mollifier(P[0], P[1], P[2], P[3], eps);
}
void or_friction_f(double y, double eh, double* out3) { friction_f(y, eh, &out3[0], &out3[1], &out3[2]); }
double or_accd(int kind, const double* x12, const double* p12, double s, double t_c, long max_iter, long* iters) {
  return accd(kind, x12, p12, s, t_c, max_iter, iters);
}
void or_mass_properties(int nv, const double* v, int nt, const int32_t* t, double rho, double* M4, double* vol) {
  mass_properties(nv, v, nt, t, rho, M4, vol);
}

}  // extern "C"
