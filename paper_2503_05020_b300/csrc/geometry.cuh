// Contact geometry on the device: point-triangle / edge-edge distance classification, squared
// distances and their derivatives, the log barrier with the edge-edge mollifier, lagged
// friction, and additive CCD.
//
// Distance types follow the closest features: PT 0..2 point-vertex, 3..5 point-edge (t0t1,
// t1t2, t2t0), 6 point-face; EE 0..3 vertex-vertex (a0b0, a0b1, a1b0, a1b1), 4..5 edge a to
// vertex b0/b1, 6..7 vertex a0/a1 to edge b, 8 line-line.
#pragma once
#include "common.cuh"
#include "dist_poly.cuh"

enum { PT_FACE = 6, EE_LINES = 8 };

// ------------------------------------------------------------------ classification
// Point-triangle: project p on the plane; inside -> face. Otherwise the closest point lies on
// the boundary: take the nearest of the three clamped edge projections.
DEV int pt_classify(d3 p, d3 t0, d3 t1, d3 t2, double w[3]) {
  d3 e1 = t1 - t0, e2 = t2 - t0, q = p - t0;
  double A11 = dot(e1, e1), A12 = dot(e1, e2), A22 = dot(e2, e2);
  double r1 = dot(e1, q), r2 = dot(e2, q);
  double det = A11 * A22 - A12 * A12;
  double u = (r1 * A22 - r2 * A12) / det, v = (A11 * r2 - A12 * r1) / det;
  if (u >= 0.0 && v >= 0.0 && u + v <= 1.0) {
    w[0] = 1.0 - u - v;
    w[1] = u;
    w[2] = v;
    return PT_FACE;
  }
  const d3 V[3] = {t0, t1, t2};
  double best = INFINITY;
  int type = 0;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    d3 a = V[k], b = V[(k + 1) % 3];
    d3 e = b - a;
    double s = dot(p - a, e) / dot(e, e);
    s = fmin(fmax(s, 0.0), 1.0);
    d3 c = a + s * e;
    d3 dd = p - c;
    double d2 = dot(dd, dd);
    if (d2 < best) {
      best = d2;
      double wk[3] = {0.0, 0.0, 0.0};
      int t;
      if (s <= 0.0) {
        wk[k] = 1.0;
        t = k;
      } else if (s >= 1.0) {
        wk[(k + 1) % 3] = 1.0;
        t = (k + 1) % 3;
      } else {
        wk[k] = 1.0 - s;
        wk[(k + 1) % 3] = s;
        t = 3 + k;
      }
      w[0] = wk[0];
      w[1] = wk[1];
      w[2] = wk[2];
      type = t;
    }
  }
  return type;
}

// Edge-edge: interior of both segments for the line-line closest points -> lines; otherwise
// the nearest of the four endpoint-to-segment projections. s on a, t on b.
DEV int ee_classify(d3 a0, d3 a1, d3 b0, d3 b1, double* s_out, double* t_out) {
  d3 ea = a1 - a0, eb = b1 - b0, r = a0 - b0;
  double A = dot(ea, ea), B = dot(ea, eb), C = dot(eb, eb), D = dot(ea, r), E = dot(eb, r);
  double den = A * C - B * B;
  // sin^2 of the angle <= 1e-10: treated as parallel (the closest pair then has an endpoint)
  if (den > 1e-10 * A * C) {
    double s = (B * E - C * D) / den, t = (A * E - B * D) / den;
    if (s > 0.0 && s < 1.0 && t > 0.0 && t < 1.0) {
      *s_out = s;
      *t_out = t;
      return EE_LINES;
    }
  }
  double best = INFINITY;
  int type = 0;
  double bs = 0, bt = 0;
  // endpoints of a against segment b
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    d3 pa = k == 0 ? a0 : a1;
    double t = fmin(fmax(dot(pa - b0, eb) / C, 0.0), 1.0);
    d3 dd = pa - (b0 + t * eb);
    double d2 = dot(dd, dd);
    if (d2 < best) {
      best = d2;
      bs = k;
      bt = t;
      type = t <= 0.0 ? (k == 0 ? 0 : 2) : (t >= 1.0 ? (k == 0 ? 1 : 3) : 6 + k);
    }
  }
  // endpoints of b against segment a
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    d3 pb = k == 0 ? b0 : b1;
    double s = fmin(fmax(dot(pb - a0, ea) / A, 0.0), 1.0);
    d3 dd = pb - (a0 + s * ea);
    double d2 = dot(dd, dd);
    if (d2 < best) {
      best = d2;
      bs = s;
      bt = k;
      type = s <= 0.0 ? (k == 0 ? 0 : 1) : (s >= 1.0 ? (k == 0 ? 2 : 3) : 4 + k);
    }
  }
  *s_out = bs;
  *t_out = bt;
  return type;
}

DEV double d2_pp(d3 a, d3 b) {
  d3 d = a - b;
  return dot(d, d);
}
DEV double d2_pe(d3 p, d3 e0, d3 e1) {
  d3 c = cross(e0 - p, e1 - p);
  d3 e = e1 - e0;
  return dot(c, c) / dot(e, e);
}
DEV double d2_plane(d3 p, d3 t0, d3 t1, d3 t2) {
  d3 n = cross(t1 - t0, t2 - t0);
  double e = dot(p - t0, n);
  return e * e / dot(n, n);
}
DEV double d2_lines(d3 a0, d3 a1, d3 b0, d3 b1) {
  d3 n = cross(a1 - a0, b1 - b0);
  double e = dot(b0 - a0, n);
  return e * e / dot(n, n);
}

// Points involved in each typed formula, as slots of the 4-point contact.
// PT slots: 0 = p, 1..3 = t0..t2. EE slots: 0 = a0, 1 = a1, 2 = b0, 3 = b1.
struct TypeSlots {
  int form;  // 0 PP, 1 PE, 2 plane / lines
  int s[4];
};
DEV TypeSlots type_slots(int kind, int type) {
  TypeSlots r;
  if (kind == 0) {
    if (type <= 2) { r.form = 0; r.s[0] = 0; r.s[1] = 1 + type; }
    else if (type <= 5) { int k = type - 3; r.form = 1; r.s[0] = 0; r.s[1] = 1 + k; r.s[2] = 1 + (k + 1) % 3; }
    else { r.form = 2; r.s[0] = 0; r.s[1] = 1; r.s[2] = 2; r.s[3] = 3; }
  } else {
    switch (type) {
      case 0: r.form = 0; r.s[0] = 0; r.s[1] = 2; break;
      case 1: r.form = 0; r.s[0] = 0; r.s[1] = 3; break;
      case 2: r.form = 0; r.s[0] = 1; r.s[1] = 2; break;
      case 3: r.form = 0; r.s[0] = 1; r.s[1] = 3; break;
      case 4: r.form = 1; r.s[0] = 2; r.s[1] = 0; r.s[2] = 1; break;
      case 5: r.form = 1; r.s[0] = 3; r.s[1] = 0; r.s[2] = 1; break;
      case 6: r.form = 1; r.s[0] = 0; r.s[1] = 2; r.s[2] = 3; break;
      case 7: r.form = 1; r.s[0] = 1; r.s[1] = 2; r.s[2] = 3; break;
      default: r.form = 2; r.s[0] = 0; r.s[1] = 1; r.s[2] = 2; r.s[3] = 3;
    }
  }
  return r;
}

DEV double typed_d2(int kind, int type, const d3 X[4]) {
  TypeSlots t = type_slots(kind, type);
  if (t.form == 0) return d2_pp(X[t.s[0]], X[t.s[1]]);
  if (t.form == 1) return d2_pe(X[t.s[0]], X[t.s[1]], X[t.s[2]]);
  return kind == 0 ? d2_plane(X[0], X[1], X[2], X[3]) : d2_lines(X[0], X[1], X[2], X[3]);
}

// Unsigned squared distance of a contact (classification + typed formula).
DEV double pair_d2(int kind, const d3 X[4], int* type_out) {
  int type;
  if (kind == 0) {
    double w[3];
    type = pt_classify(X[0], X[1], X[2], X[3], w);
  } else {
    double s, t;
    type = ee_classify(X[0], X[1], X[2], X[3], &s, &t);
  }
  if (type_out) *type_out = type;
  return typed_d2(kind, type, X);
}

// Gradient g[12] and packed upper Hessian H[78] of the squared distance of the given type.
// Kept out of line for the same reason as project_psd_jacobi.
__device__ __noinline__ void d2_derivs(int kind, int type, const d3 X[4], double* s_out, double g[12], double H[78]) {
#pragma unroll 1
  for (int i = 0; i < 12; ++i) g[i] = 0.0;
#pragma unroll 1
  for (int i = 0; i < 78; ++i) H[i] = 0.0;
  TypeSlots t = type_slots(kind, type);
  if (t.form == 0) {
    int a = t.s[0], b = t.s[1];
    d3 d = X[a] - X[b];
    *s_out = dot(d, d);
    for (int k = 0; k < 3; ++k) {
      g[3 * a + k] = 2.0 * comp(d, k);
      g[3 * b + k] = -2.0 * comp(d, k);
      H[sym_idx(3 * a + k, 3 * a + k, 12)] += 2.0;
      H[sym_idx(3 * b + k, 3 * b + k, 12)] += 2.0;
      H[sym_idx(3 * a + k, 3 * b + k, 12)] += -2.0;
    }
    return;
  }
  // local quotient d^2 = C / D over n local coordinates mapped to slots
  int n = t.form == 1 ? 9 : 12;
  double C, Cg[12], Ch[78], D, Dg[12], Dh[78];
  if (t.form == 1) {
    double pp[3] = {X[t.s[0]].x, X[t.s[0]].y, X[t.s[0]].z};
    double q0[3] = {X[t.s[1]].x, X[t.s[1]].y, X[t.s[1]].z};
    double q1[3] = {X[t.s[2]].x, X[t.s[2]].y, X[t.s[2]].z};
    pe_poly(pp, q0, q1, &C, Cg, Ch, &D, Dg, Dh);
  } else {
    double P[12];
    for (int i = 0; i < 4; ++i) {
      P[3 * i] = X[i].x;
      P[3 * i + 1] = X[i].y;
      P[3 * i + 2] = X[i].z;
    }
    double N, Ng[12], Nh[78];
    if (kind == 0) pt_poly(P, P + 3, P + 6, P + 9, &N, Ng, Nh, &D, Dg, Dh);
    else ee_poly(P, P + 3, P + 6, P + 9, &N, Ng, Nh, &D, Dg, Dh);
    C = N * N;
    for (int i = 0; i < 12; ++i) Cg[i] = 2.0 * N * Ng[i];
    for (int i = 0; i < 12; ++i)
      for (int j = i; j < 12; ++j) Ch[up_idx(i, j, 12)] = 2.0 * (Ng[i] * Ng[j] + N * Nh[up_idx(i, j, 12)]);
  }
  double iD = 1.0 / D, s = C * iD;
  *s_out = s;
  int slot[12];
  for (int i = 0; i < n; ++i) slot[i] = 3 * t.s[i / 3] + (i % 3);
  for (int i = 0; i < n; ++i) g[slot[i]] = (Cg[i] - s * Dg[i]) * iD;
  for (int i = 0; i < n; ++i)
    for (int j = i; j < n; ++j) {
      int u = up_idx(i, j, n);
      double h = (Ch[u] - (Cg[i] * Dg[j] + Dg[i] * Cg[j]) * iD - s * Dh[u] + 2.0 * s * Dg[i] * Dg[j] * iD) * iD;
      H[sym_idx(slot[i], slot[j], 12)] += h;
    }
}

// Barrier b(d) = -(d - dhat)^2 ln(d / dhat) and its first two derivatives, 0 < d < dhat.
DEV void barrier3(double d, double dhat, double* b, double* b1, double* b2) {
  if (d >= dhat) {
    *b = *b1 = *b2 = 0.0;
    return;
  }
  double t = d - dhat, L = log(d / dhat);
  *b = -t * t * L;
  *b1 = -2.0 * t * L - t * t / d;
  *b2 = -2.0 * L - 4.0 * t / d + t * t / (d * d);
}

// Closest-point coefficients c[4] and unit normal n (from side B to side A) of a contact.
DEV void pair_closest(int kind, const d3 X[4], double c[4], d3* n) {
  d3 ca, cb;
  if (kind == 0) {
    double w[3];
    pt_classify(X[0], X[1], X[2], X[3], w);
    c[0] = 1.0;
    c[1] = -w[0];
    c[2] = -w[1];
    c[3] = -w[2];
    ca = X[0];
    cb = w[0] * X[1] + w[1] * X[2] + w[2] * X[3];
  } else {
    double s, t;
    ee_classify(X[0], X[1], X[2], X[3], &s, &t);
    c[0] = 1.0 - s;
    c[1] = s;
    c[2] = -(1.0 - t);
    c[3] = -t;
    ca = (1.0 - s) * X[0] + s * X[1];
    cb = (1.0 - t) * X[2] + t * X[3];
  }
  d3 d = ca - cb;
  double L = sqrt(dot(d, d));
  *n = L > 0.0 ? (1.0 / L) * d : mk3(0, 0, 0);
}

// ACCD (Li, Kaufman & Jiang 2021): conservative time of impact in (0, t_c] of 4 points moving
// by P over [0, 1], thickness 0, gap fraction s; returns t_c if no contact happens before t_c.
DEV double accd(int kind, const d3 X0[4], const d3 P0[4], double s, double t_c, long max_iter, long* iters) {
  d3 X[4], P[4];
  d3 mean = mk3(0, 0, 0);
  for (int i = 0; i < 4; ++i) mean = mean + P0[i];
  mean = 0.25 * mean;
  double nrm[4];
  for (int i = 0; i < 4; ++i) {
    X[i] = X0[i];
    P[i] = P0[i] - mean;
    nrm[i] = sqrt(dot(P[i], P[i]));
  }
  double lp = kind == 0 ? nrm[0] + fmax(nrm[1], fmax(nrm[2], nrm[3])) : fmax(nrm[0], nrm[1]) + fmax(nrm[2], nrm[3]);
  *iters = 0;
  if (lp == 0.0) return t_c;
  double d = sqrt(pair_d2(kind, X, nullptr));
  double g = s * d;
  double t = 0.0;
  double tl = (1.0 - s) * d / lp;
  long it = 0;
  while (it < max_iter) {
    ++it;
    for (int i = 0; i < 4; ++i) X[i] = X[i] + tl * P[i];
    d = sqrt(pair_d2(kind, X, nullptr));
    if (t > 0.0 && d < g) break;
    t = t + tl;
    if (t > t_c) {
      t = t_c;
      break;
    }
    tl = 0.9 * d / lp;
  }
  *iters = it;
  return t;
}
