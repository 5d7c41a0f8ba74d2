// Energy stencils of the incremental potential
//   E(x) = 1/2 |x - x~|_M^2 + h^2 [ sum_tets V Psi(F) + sum_bodies kappa_A V |A A^T - I|^2
//                                  + kappa sum_k e_k b(d_k) + sum_k mu lambda_k f0(|P_k rel_k|) ]
// (IPC 2020 incremental potential with the affine-body orthogonality term of Lan et al. 2022),
// each written per element so that one thread owns one tet, body or contact. Outputs are
// per-element energies, gradients and PSD-projected Hessians; a later pass gathers them in a
// fixed order (deterministic, no atomics on values).
#pragma once
#include "common.cuh"
#include "geometry.cuh"

enum { MODE_ENERGY = 0, MODE_GRAD = 1, MODE_HESS = 2 };

struct StepConst {
  double h, dhat, kappa, eps_v, kappa_affine;
  double g[3];
};

// ----------------------------------------------------------------- point positions
// soft point: its node; affine point: ((p + xb0 a1) + xb1 a2) + xb2 a3, rounded as written.
__global__ void k_points(int n_pts, const int* __restrict__ pt_node, const double* __restrict__ pt_xb,
                         const int* __restrict__ body_node, const double* __restrict__ q, double* __restrict__ out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_pts) return;
  int nd = pt_node[i];
  if (nd >= 0) {
    out[3 * i] = q[3 * nd];
    out[3 * i + 1] = q[3 * nd + 1];
    out[3 * i + 2] = q[3 * nd + 2];
  } else {
    const double* b = q + 3 * (long)body_node[-1 - nd];
    double x0 = pt_xb[3 * i], x1 = pt_xb[3 * i + 1], x2 = pt_xb[3 * i + 2];
    for (int k = 0; k < 3; ++k) {
      double r = add_mul_rn(b[k], x0, b[3 + k]);
      r = add_mul_rn(r, x1, b[6 + k]);
      r = add_mul_rn(r, x2, b[9 + k]);
      out[3 * i + k] = r;
    }
  }
}

// ----------------------------------------------------------------- Neo-Hookean tets
// Analytic eigensystem of d2Psi/dF2 (Smith, de Goes & Kim 2019) for
// Psi = mu/2 (|F|^2 - 3) - mu ln J + lam/2 (ln J)^2 with F = U diag(s) V^T:
//   scaling modes: eigenpairs of A_ii = mu + (mu - lam lnJ + lam)/s_i^2, A_ij = lam/(s_i s_j),
//   twist (i,j):   mu + (lam lnJ - mu)/(s_i s_j),  U (e_i e_j^T - e_j e_i^T) V^T / sqrt 2,
//   flip (i,j):    mu + (mu - lam lnJ)/(s_i s_j),  U (e_i e_j^T + e_j e_i^T) V^T / sqrt 2.
// Negative eigenvalues are dropped (projected Newton); the 12x12 Hessian is
// h^2 V sum_m lam_m^+ w_m w_m^T with w_m[a] = Q_m b_a (b_a: shape-function gradients), formed
// blockwise in the frame of the SVD (tet_hessian).
// F = Ds Dm^-1, its cofactor, J and the weighted energy h^2 V Psi(F). Not inlined: every mode
// calls the same machine code, so Newton and line-search energies round identically.
__device__ __noinline__ double tet_energy(d3 x0, d3 x1, d3 x2, d3 x3, const double* __restrict__ Bm, double mu,
                                          double lam, double w, double* F, double* cof, double* Jout) {
  d3 c1 = x1 - x0, c2 = x2 - x0, c3 = x3 - x0;
  const d3 Cc[3] = {c1, c2, c3};
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c)
      F[3 * r + c] = comp(Cc[0], r) * Bm[c] + comp(Cc[1], r) * Bm[3 + c] + comp(Cc[2], r) * Bm[6 + c];
  cof[0] = F[4] * F[8] - F[5] * F[7];
  cof[1] = F[5] * F[6] - F[3] * F[8];
  cof[2] = F[3] * F[7] - F[4] * F[6];
  cof[3] = F[2] * F[7] - F[1] * F[8];
  cof[4] = F[0] * F[8] - F[2] * F[6];
  cof[5] = F[1] * F[6] - F[0] * F[7];
  cof[6] = F[1] * F[5] - F[2] * F[4];
  cof[7] = F[2] * F[3] - F[0] * F[5];
  cof[8] = F[0] * F[4] - F[1] * F[3];
  double J = F[0] * cof[0] + F[1] * cof[1] + F[2] * cof[2];
  *Jout = J;
  if (!(J > 0.0)) return 0.0;
  double lnJ = log(J);
  double tr = 0.0;
  for (int i = 0; i < 9; ++i) tr += F[i] * F[i];
  return w * (0.5 * mu * (tr - 3.0) - mu * lnJ + 0.5 * lam * lnJ * lnJ);
}

// Smallest squared singular value used when dividing by s_i (a degenerate tet).
template <class T>
struct TinyS2;
template <>
struct TinyS2<double> {
  static constexpr double v = 1e-300;
};
template <>
struct TinyS2<float> {
  static constexpr float v = 1e-30f;
};

// PSD-projected Hessian of the weighted Neo-Hookean energy w Psi(F), in the precision HT, as
// the 10 upper 3x3 blocks (a <= b, row-major) of the 12x12 tet Hessian (90 values). F, the
// Lame parameters, ln J, Dm^-1 (Bm) and w come in FP64 and are rounded to HT first.
template <class HT>
DEV void tet_hessian(const double* F64, double mu64, double lam64, double lnJ64, const double* Bm, double w64,
                     HT* __restrict__ out) {
  const HT mu = HT(mu64), lam = HT(lam64), lnJ = HT(lnJ64);
  HT F[9];
  for (int i = 0; i < 9; ++i) F[i] = HT(F64[i]);
  // shape-function gradients b_a: b1..b3 = rows of Dm^-1, b0 = -(b1 + b2 + b3)
  HT b[4][3];
  for (int c = 0; c < 3; ++c) {
    b[1][c] = HT(Bm[c]);
    b[2][c] = HT(Bm[3 + c]);
    b[3][c] = HT(Bm[6 + c]);
    b[0][c] = HT(-(Bm[c] + Bm[3 + c] + Bm[6 + c]));
  }
  // SVD through the eigen-decomposition of F^T F
  HT C[9];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) C[3 * r + c] = F[r] * F[c] + F[3 + r] * F[3 + c] + F[6 + r] * F[6 + c];
  HT s2[3], V[9];
  eig_sym3<HT>(C, s2, V);
  HT s[3];
  for (int i = 0; i < 3; ++i) s[i] = sqrt(fmax(s2[i], TinyS2<HT>::v));
  HT U[9];  // U = F V diag(1/s)
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c)
      U[3 * r + c] = (F[3 * r] * V[c] + F[3 * r + 1] * V[3 + c] + F[3 * r + 2] * V[6 + c]) / s[c];
  // c_a = V^T b_a
  HT cb[4][3];
  for (int a = 0; a < 4; ++a)
    for (int k = 0; k < 3; ++k) cb[a][k] = V[k] * b[a][0] + V[3 + k] * b[a][1] + V[6 + k] * b[a][2];
  // The projected d2Psi/dF2 in the frame of the SVD (F^ = U^T F V = diag(s)) is block-diagonal:
  // the scaling block on the (ii, kk) entries, projected to S+ (its eigenpairs with positive
  // eigenvalue; the block itself when it is positive definite, the common case, which needs no
  // eigen-decomposition), and for each pair i < j the 2x2 block of the twist and flip modes on
  // the (ij, ji) entries, (lt+ + lf+)/2 on its diagonal and (lf+ - lt+)/2 off it. With
  // dF^ = sum_a dx^_a c_a^T (x^ = U^T x, c_a = V^T b_a), the 3x3 block (a, b) of the tet Hessian
  // in that frame is
  //   H^_ab[i][i] = S+_ii ca_i cb_i + sum_{j != i} P_ij ca_j cb_j,
  //   H^_ab[i][k] = S+_ik ca_i cb_k + Q_ik ca_k cb_i   (i != k),
  // and H_ab = U H^_ab U^T: the same sum of the nine clamped modes as lam_m w_m w_m^T, without
  // forming each mode.
  HT A[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      A[3 * i + j] = (i == j) ? mu + (mu - lam * lnJ + lam) / (s[i] * s[i]) : lam / (s[i] * s[j]);
  HT Sp[9];
  const HT m2 = A[0] * A[4] - A[1] * A[1];
  const HT det = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
                 A[2] * (A[3] * A[7] - A[4] * A[6]);
  if (A[0] > HT(0) && m2 > HT(0) && det > HT(0)) {  // leading minors positive: A is its own projection
    for (int i = 0; i < 9; ++i) Sp[i] = A[i];
  } else {
    HT la[3], av[9];
    eig_sym3<HT>(A, la, av);
    for (int i = 0; i < 9; ++i) Sp[i] = HT(0);
    for (int k = 0; k < 3; ++k) {
      if (!(la[k] > HT(0))) continue;
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) Sp[3 * i + j] += la[k] * av[3 * i + k] * av[3 * j + k];
    }
  }
  // twist (lt) and flip (lf) eigenvalues of the pairs (0,1), (1,2), (0,2), clamped at zero
  HT Pp[3], Qp[3];
  for (int pr = 0; pr < 3; ++pr) {
    const int i = pr == 2 ? 0 : pr, j = pr == 2 ? 2 : pr + 1;
    const HT ss = s[i] * s[j];
    const HT lt = fmax(mu + (lam * lnJ - mu) / ss, HT(0)), lf = fmax(mu + (mu - lam * lnJ) / ss, HT(0));
    Pp[pr] = HT(0.5) * (lt + lf);
    Qp[pr] = HT(0.5) * (lf - lt);
  }
  const HT w = HT(w64);
  int blk = 0;
  for (int a = 0; a < 4; ++a)
    for (int bb = a; bb < 4; ++bb, ++blk) {
      const HT* ca = cb[a];
      const HT* cc = cb[bb];
      const HT p0 = ca[0] * cc[0], p1 = ca[1] * cc[1], p2 = ca[2] * cc[2];
      HT Hh[9];
      Hh[0] = Sp[0] * p0 + Pp[0] * p1 + Pp[2] * p2;
      Hh[4] = Sp[4] * p1 + Pp[0] * p0 + Pp[1] * p2;
      Hh[8] = Sp[8] * p2 + Pp[2] * p0 + Pp[1] * p1;
      Hh[1] = Sp[1] * ca[0] * cc[1] + Qp[0] * ca[1] * cc[0];
      Hh[3] = Sp[3] * ca[1] * cc[0] + Qp[0] * ca[0] * cc[1];
      Hh[5] = Sp[5] * ca[1] * cc[2] + Qp[1] * ca[2] * cc[1];
      Hh[7] = Sp[7] * ca[2] * cc[1] + Qp[1] * ca[1] * cc[2];
      Hh[2] = Sp[2] * ca[0] * cc[2] + Qp[2] * ca[2] * cc[0];
      Hh[6] = Sp[6] * ca[2] * cc[0] + Qp[2] * ca[0] * cc[2];
      HT T[9];  // U H^
      for (int r = 0; r < 3; ++r)
        for (int k = 0; k < 3; ++k) T[3 * r + k] = U[3 * r] * Hh[k] + U[3 * r + 1] * Hh[3 + k] + U[3 * r + 2] * Hh[6 + k];
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c)
          out[9 * blk + 3 * r + c] = w * (T[3 * r] * U[3 * c] + T[3 * r + 1] * U[3 * c + 1] + T[3 * r + 2] * U[3 * c + 2]);
    }
}

template <int MODE, class HT = double>
__global__ void k_elastic(int n_tets, const int4* __restrict__ tets, const double* __restrict__ prm,
                          const int* __restrict__ tenv, const uint8_t* __restrict__ act, const double* __restrict__ q,
                          double h2, double* __restrict__ tE, double* __restrict__ tg, HT* __restrict__ tH,
                          int* __restrict__ env_bad, unsigned long long* __restrict__ units) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_tets) return;
  int e = tenv[t];
  if (units) {  // count the tets this launch processes (one atomic per warp)
    unsigned m = __ballot_sync(__activemask(), act[e] != 0);
    if ((threadIdx.x & 31) == __ffs(__activemask()) - 1) atomicAdd(units, (unsigned long long)__popc(m));
  }
  if (!act[e]) return;
  int4 T = tets[t];
  const double* P = prm + 12 * (long)t;
  d3 x0 = ld3(q, T.x), x1 = ld3(q, T.y), x2 = ld3(q, T.z), x3 = ld3(q, T.w);
  double Bm[9];
  for (int i = 0; i < 9; ++i) Bm[i] = P[i];
  double vol = P[9], mu = P[10], lam = P[11];
  double w = h2 * vol;
  double F[9], cof[9], J;
  double En = tet_energy(x0, x1, x2, x3, Bm, mu, lam, w, F, cof, &J);
  if (!(J > 0.0)) {
    env_bad[e] = 1;
    tE[t] = 0.0;
    return;
  }
  tE[t] = En;
  double lnJ = log(J);
  if (MODE == MODE_ENERGY) return;
  // gradient (FP64): w P(F) b_a, first Piola-Kirchhoff stress P = mu F + (lam lnJ - mu) cof(F) / J,
  // b_a the shape-function gradients (b1..b3 = rows of Dm^-1, b0 = -(b1 + b2 + b3))
  d3 b[4];
  b[1] = mk3(Bm[0], Bm[1], Bm[2]);
  b[2] = mk3(Bm[3], Bm[4], Bm[5]);
  b[3] = mk3(Bm[6], Bm[7], Bm[8]);
  b[0] = mk3(-(Bm[0] + Bm[3] + Bm[6]), -(Bm[1] + Bm[4] + Bm[7]), -(Bm[2] + Bm[5] + Bm[8]));
  double kk = (lam * lnJ - mu) / J;
  double Pk[9];
  for (int i = 0; i < 9; ++i) Pk[i] = mu * F[i] + kk * cof[i];
  for (int a = 0; a < 4; ++a) {
    d3 ga = mk3(Pk[0] * b[a].x + Pk[1] * b[a].y + Pk[2] * b[a].z, Pk[3] * b[a].x + Pk[4] * b[a].y + Pk[5] * b[a].z,
                Pk[6] * b[a].x + Pk[7] * b[a].y + Pk[8] * b[a].z);
    tg[12 * (long)t + 3 * a] = w * ga.x;
    tg[12 * (long)t + 3 * a + 1] = w * ga.y;
    tg[12 * (long)t + 3 * a + 2] = w * ga.z;
  }
  if (MODE == MODE_GRAD) return;
  tet_hessian<HT>(F, mu, lam, lnJ, Bm, w, tH + 90 * (long)t);
}

// ----------------------------------------------------------------- affine bodies
// Inertia 1/2 (q - q~)^T (M4 x I3) (q - q~) and orthogonality h^2 kappa_A V |A A^T - I|_F^2,
// A[r][c] = q[3 + 3c + r]. d2/dA2 of |S|^2, S = A A^T - I, is
// 4 [d_km (A^T A)_nl + A_kn A_ml + S_km d_ln] at (kl, mn); it is projected to PSD.
// inertia + orthogonality (+ PD target) value of one free body, with A and S = A A^T - I (not
// inlined, see tet_energy). The PD target term is 1/2 wpd (q - q^)^T (M4 x I3) (q - q^) with
// wpd = h^2 k_pd, q^ = Qh.
__device__ __noinline__ double body_energy(const double* __restrict__ Q, const double* __restrict__ Qt,
                                           const double* __restrict__ M, double wk, double* dq, double* A, double* S,
                                           const double* __restrict__ Qh, double wpd) {
  for (int i = 0; i < 12; ++i) dq[i] = Q[i] - Qt[i];
  double Ein = 0.0;
  for (int I = 0; I < 4; ++I)
    for (int k = 0; k < 3; ++k) {
      double s = 0.0;
      for (int Jn = 0; Jn < 4; ++Jn) s += M[4 * I + Jn] * dq[3 * Jn + k];
      Ein += 0.5 * dq[3 * I + k] * s;
    }
  if (wpd > 0.0)
    for (int I = 0; I < 4; ++I)
      for (int k = 0; k < 3; ++k) {
        double s = 0.0;
        for (int Jn = 0; Jn < 4; ++Jn) s += M[4 * I + Jn] * (Q[3 * Jn + k] - Qh[3 * Jn + k]);
        Ein += 0.5 * wpd * (Q[3 * I + k] - Qh[3 * I + k]) * s;
      }
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) A[3 * r + c] = Q[3 + 3 * c + r];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      S[3 * i + j] = A[3 * i] * A[3 * j] + A[3 * i + 1] * A[3 * j + 1] + A[3 * i + 2] * A[3 * j + 2] - (i == j ? 1.0 : 0.0);
  double f = 0.0;
  for (int i = 0; i < 9; ++i) f += S[i] * S[i];
  return Ein + wk * f;
}

// Energy, gradient (MODE >= MODE_GRAD) and, for MODE_HESS, the unprojected 9x9 orthogonality
// Hessian d2|S|^2/dA2 in the precision HT (row-major, leading dimension ldo) of one free body.
template <int MODE, class HT>
DEV double body_eval(const double* __restrict__ Q, const double* __restrict__ Qt, const double* __restrict__ M,
                     double wk, const double* __restrict__ Qh, double wpd, double* g, HT* Ho, int ldo) {
  double dq[12], A[9], S[9];
  double E = body_energy(Q, Qt, M, wk, dq, A, S, Qh, wpd);
  if (MODE == MODE_ENERGY) return E;
  for (int I = 0; I < 4; ++I)
    for (int k = 0; k < 3; ++k) {
      double s = 0.0;
      for (int Jn = 0; Jn < 4; ++Jn) s += M[4 * I + Jn] * dq[3 * Jn + k];
      if (wpd > 0.0)
        for (int Jn = 0; Jn < 4; ++Jn) s += wpd * M[4 * I + Jn] * (Q[3 * Jn + k] - Qh[3 * Jn + k]);
      g[3 * I + k] = s;
    }
  // gradient of |S|^2 wrt A: 4 S A
  for (int k = 0; k < 3; ++k)
    for (int l = 0; l < 3; ++l) {
      double sa = S[3 * k] * A[l] + S[3 * k + 1] * A[3 + l] + S[3 * k + 2] * A[6 + l];
      g[3 + 3 * l + k] += wk * 4.0 * sa;
    }
  if (MODE == MODE_GRAD) return E;
  HT Ah[9], Sh[9];
  for (int i = 0; i < 9; ++i) {
    Ah[i] = HT(A[i]);
    Sh[i] = HT(S[i]);
  }
  HT AtA[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) AtA[3 * i + j] = Ah[i] * Ah[j] + Ah[3 + i] * Ah[3 + j] + Ah[6 + i] * Ah[6 + j];
  for (int k = 0; k < 3; ++k)
    for (int l = 0; l < 3; ++l)
      for (int m = 0; m < 3; ++m)
        for (int n = 0; n < 3; ++n) {
          HT v = Ah[3 * k + n] * Ah[3 * m + l];
          if (k == m) v += AtA[3 * n + l];
          if (l == n) v += Sh[3 * k + m];
          Ho[(3 * k + l) * ldo + 3 * m + n] = HT(4) * v;
        }
  return E;
}

// energy and gradient modes: one thread per body
template <int MODE>
__global__ void k_bodies(int n_bodies, const int* __restrict__ bnode, const int* __restrict__ benv,
                         const uint8_t* __restrict__ bkin, const double* __restrict__ M4, const double* __restrict__ bvol,
                         const uint8_t* __restrict__ act, const double* __restrict__ q, const double* __restrict__ qt,
                         const double* __restrict__ qh, const double* __restrict__ kpd, double h2, double h2kA,
                         double* __restrict__ bE, double* __restrict__ bg) {
  static_assert(MODE != MODE_HESS, "the Hessian mode is k_bodies_hess");
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n_bodies) return;
  int e = benv[b];
  if (!act[e]) return;
  if (bkin[b]) {
    bE[b] = 0.0;
    if (MODE >= MODE_GRAD)
      for (int i = 0; i < 12; ++i) bg[12 * (long)b + i] = 0.0;
    return;
  }
  double g[12];
  bE[b] = body_eval<MODE, double>(q + 3 * (long)bnode[b], qt + 3 * (long)bnode[b], M4 + 16 * (long)b,
                                  h2kA * bvol[b], qh + 3 * (long)bnode[b], h2 * kpd[b], g, (double*)nullptr, 0);
  if (MODE == MODE_GRAD)
    for (int i = 0; i < 12; ++i) bg[12 * (long)b + i] = g[i];
}

// Hessian mode: one half-warp per body. Lane 0 forms the energy, gradient and the 9x9
// orthogonality Hessian (padded to 10x10 with zeros) in shared memory, the half-warp projects it
// to PSD in the precision HT, and the 12x12 block ((1 + h^2 k_pd) times the mass blocks, plus
// h^2 kappa_A V times the projection) is written out.
constexpr int BODY_HESS_THREADS = 64;
template <class HT>
__global__ void __launch_bounds__(BODY_HESS_THREADS)
    k_bodies_hess(int n_bodies, const int* __restrict__ bnode, const int* __restrict__ benv,
                  const uint8_t* __restrict__ bkin, const double* __restrict__ M4, const double* __restrict__ bvol,
                  const uint8_t* __restrict__ act, const double* __restrict__ q, const double* __restrict__ qt,
                  const double* __restrict__ qh, const double* __restrict__ kpd, double h2, double h2kA,
                  double* __restrict__ bE, double* __restrict__ bg, HT* __restrict__ bH) {
  constexpr int HALVES = BODY_HESS_THREADS / 16;
  __shared__ HT shA[HALVES][100], shV[HALVES][100], shR[HALVES][30];
  const int half = threadIdx.x >> 4, hl = threadIdx.x & 15;
  const unsigned mask = 0xffffu << (threadIdx.x & 16);
  const int b = (blockIdx.x * BODY_HESS_THREADS + threadIdx.x) >> 4;
  if (b >= n_bodies) return;  // uniform over the half-warp
  if (!act[benv[b]]) return;
  HT* Hout = bH + 144 * (long)b;
  if (bkin[b]) {
    if (hl == 0) {
      bE[b] = 0.0;
      for (int i = 0; i < 12; ++i) bg[12 * (long)b + i] = 0.0;
    }
    for (int i = hl; i < 144; i += 16) Hout[i] = (i % 13 == 0) ? HT(1) : HT(0);
    return;
  }
  const double* M = M4 + 16 * (long)b;
  const double wk = h2kA * bvol[b], wpd = h2 * kpd[b];
  HT* A = shA[half];
  for (int i = hl; i < 100; i += 16) A[i] = HT(0);
  __syncwarp(mask);
  if (hl == 0) {
    double g[12];
    bE[b] = body_eval<MODE_HESS, HT>(q + 3 * (long)bnode[b], qt + 3 * (long)bnode[b], M, wk, qh + 3 * (long)bnode[b],
                                     wpd, g, A, 10);
    for (int i = 0; i < 12; ++i) bg[12 * (long)b + i] = g[i];
  }
  __syncwarp(mask);
  project_psd_hw<10, HT>(A, shV[half], shR[half], hl, mask);
  const HT wkh = HT(wk);
  for (int e = hl; e < 144; e += 16) {
    const int qi = e / 12, qj = e % 12;
    const int I = qi / 3, k = qi % 3, Jn = qj / 3, m = qj % 3;
    HT v = (k == m) ? HT(M[4 * I + Jn] + wpd * M[4 * I + Jn]) : HT(0);  // inertia + PD target
    if (qi >= 3 && qj >= 3) {  // q index 3 + 3 l + k  <->  orthogonality index 3 k + l
      const int l = (qi - 3) / 3, n = (qj - 3) / 3;
      v += wkh * A[(3 * k + l) * 10 + 3 * m + n];
    }
    Hout[e] = v;
  }
}

// ----------------------------------------------------------------- contacts (barrier)
struct ContactRec {
  int pts[4];
  int kind, type, env, cand;
  double eps_x;
};

// h^2 kappa e(c) b(d) with PSD-projected Hessian; d = sqrt(s), grad b = b'/(2d) grad s,
// hess b = (b''/(4 d^2) - b'/(4 d^3)) grad s grad s^T + b'/(2d) hess s.
// kappa h^2 e(c) b(d) value (not inlined, see tet_energy)
__device__ __noinline__ double barrier_energy(int kind, int type, const d3* X, double eps_x, double dhat, double scale,
                                              double* s_out, double* c_out) {
  double s = typed_d2(kind, type, X);
  *s_out = s;
  double d = sqrt(s);
  double b = 0.0;
  if (d < dhat) {
    double t = d - dhat;
    b = -t * t * log(d / dhat);
  }
  double m = 1.0;
  double cc = 0.0;
  if (kind == 1) {
    d3 n = cross(X[1] - X[0], X[3] - X[2]);
    cc = dot(n, n);
    if (cc < eps_x) {
      double r = cc / eps_x;
      m = -r * r + 2.0 * r;
    }
  }
  *c_out = cc;
  return scale * m * b;
}

// Energy (returned), gradient g (MODE >= MODE_GRAD) and the unprojected 12x12 Hessian H
// (MODE == MODE_HESS, row-major) of one contact, in FP64.
template <int MODE>
DEV double barrier_eval(const ContactRec& c, const double* __restrict__ ptx, double h2, double dhat, double kappa,
                        double* g, double* H) {
  d3 X[4];
  for (int i = 0; i < 4; ++i) X[i] = ld3(ptx, c.pts[i]);
  // the energy value comes from the same function in every mode, so that line-search energies
  // and Newton energies round identically; the generated code gives derivatives only
  double scale = h2 * kappa;
  double s, cc;
  double Eb = barrier_energy(c.kind, c.type, X, c.eps_x, dhat, scale, &s, &cc);
  if (MODE == MODE_ENERGY) return Eb;
  double gs[12], Hs[78];
  {
    double s_unused;
    d2_derivs(c.kind, c.type, X, &s_unused, gs, Hs);
  }
  double d = sqrt(s);
  double b, b1, b2;
  barrier3(d, dhat, &b, &b1, &b2);
  double m = 1.0, m1 = 0.0, m2 = 0.0, gc[12], Hc[78];
  if (c.kind == 1) {
    double P[12], N, Ng[12], Nh[78];
    for (int i = 0; i < 4; ++i) {
      P[3 * i] = X[i].x;
      P[3 * i + 1] = X[i].y;
      P[3 * i + 2] = X[i].z;
    }
    double cc_unused;
    ee_poly(P, P + 3, P + 6, P + 9, &N, Ng, Nh, &cc_unused, gc, Hc);
    if (cc < c.eps_x) {
      double r = cc / c.eps_x;
      m = -r * r + 2.0 * r;
      m1 = (-2.0 * r + 2.0) / c.eps_x;
      m2 = -2.0 / (c.eps_x * c.eps_x);
    }
  }
  double gb[12], kb = b1 / (2.0 * d);
  for (int i = 0; i < 12; ++i) gb[i] = kb * gs[i];
  double gm[12];
  for (int i = 0; i < 12; ++i) gm[i] = c.kind == 1 ? m1 * gc[i] : 0.0;
  for (int i = 0; i < 12; ++i) g[i] = scale * (m * gb[i] + b * gm[i]);
  if (MODE == MODE_GRAD) return Eb;
  double ka = b2 / (4.0 * d * d) - b1 / (4.0 * d * d * d);
  for (int i = 0; i < 12; ++i)
    for (int j = i; j < 12; ++j) {
      int u = up_idx(i, j, 12);
      double hb = ka * gs[i] * gs[j] + kb * Hs[u];
      double v = m * hb;
      if (c.kind == 1) v += b * (m2 * gc[i] * gc[j] + m1 * Hc[u]) + gm[i] * gb[j] + gb[i] * gm[j];
      H[12 * i + j] = scale * v;
      H[12 * j + i] = scale * v;
    }
  return Eb;
}

// Von Mises stress of every tet of the envs in act at DOFs q, one thread per tet: the
// Neo-Hookean Cauchy stress is (mu (F F^T - I) + lam ln J I) / J, so its deviator is
// (mu / J) dev(F F^T) and von Mises = (mu / J) sqrt(3/2 dev(F F^T) : dev(F F^T)).
__global__ void k_tet_von_mises(int n_tets, const int4* __restrict__ tets, const double* __restrict__ prm,
                                const int* __restrict__ tenv, const uint8_t* __restrict__ act,
                                const double* __restrict__ q, double* __restrict__ out) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_tets || !act[tenv[t]]) return;
  const int4 T = tets[t];
  const double* P = prm + 12 * (long)t;
  const d3 x0 = ld3(q, T.x), x1 = ld3(q, T.y), x2 = ld3(q, T.z), x3 = ld3(q, T.w);
  const double Ds[9] = {x1.x - x0.x, x2.x - x0.x, x3.x - x0.x, x1.y - x0.y, x2.y - x0.y,
                        x3.y - x0.y, x1.z - x0.z, x2.z - x0.z, x3.z - x0.z};
  double F[9];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) F[3 * r + c] = Ds[3 * r] * P[c] + Ds[3 * r + 1] * P[3 + c] + Ds[3 * r + 2] * P[6 + c];
  const double J = F[0] * (F[4] * F[8] - F[5] * F[7]) - F[1] * (F[3] * F[8] - F[5] * F[6]) +
                   F[2] * (F[3] * F[7] - F[4] * F[6]);
  double B[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) B[3 * i + j] = F[3 * i] * F[3 * j] + F[3 * i + 1] * F[3 * j + 1] + F[3 * i + 2] * F[3 * j + 2];
  const double m = (B[0] + B[4] + B[8]) / 3.0;
  double ss = 0.0;
  for (int i = 0; i < 9; ++i) {
    const double d = B[i] - ((i % 4 == 0) ? m : 0.0);
    ss += d * d;
  }
  out[t] = P[10] / J * sqrt(1.5 * ss);
}

// energy and gradient modes: one thread per contact
template <int MODE>
__global__ void k_barrier(int n_ct, const ContactRec* __restrict__ ct, const uint8_t* __restrict__ act,
                          const double* __restrict__ ptx, double h2, double dhat, const double* __restrict__ kappa,
                          double* __restrict__ sE, double* __restrict__ sg) {
  static_assert(MODE != MODE_HESS, "the Hessian mode is k_barrier_hess");
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_ct) return;
  ContactRec c = ct[k];
  if (!act[c.env]) return;
  double g[12];
  sE[k] = barrier_eval<MODE>(c, ptx, h2, dhat, kappa[c.env], g, nullptr);
  if (MODE == MODE_GRAD)
    for (int i = 0; i < 12; ++i) sg[12 * (long)k + i] = g[i];
}

// Hessian mode, in two launches. First one thread per contact forms the energy, gradient and
// unprojected 12x12 Hessian (FP64; row-major into the scratch Hl, 144 values per contact): a
// long dependent FP64 chain, so every contact of the batch gets its own thread and the chains
// overlap. Then one block of BARRIER_HESS_THREADS per contact projects its Hessian to PSD in
// FP64 (FP32-warm-started Jacobi, one or two matrix elements per thread per round) and stores
// the packed upper triangle in the precision HT. The split keeps the chain's registers out of
// the projection's blocks, so many contacts are projected per SM at once.
constexpr int BARRIER_LOCAL_THREADS = 64;
__global__ void __launch_bounds__(BARRIER_LOCAL_THREADS)
    k_barrier_local(int n_ct, const ContactRec* __restrict__ ct, const uint8_t* __restrict__ act,
                    const double* __restrict__ ptx, double h2, double dhat, const double* __restrict__ kappa,
                    double* __restrict__ sE, double* __restrict__ sg, double* __restrict__ Hl) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_ct) return;
  const ContactRec c = ct[k];
  if (!act[c.env]) return;
  double g[12];
  sE[k] = barrier_eval<MODE_HESS>(c, ptx, h2, dhat, kappa[c.env], g, Hl + 144 * (long)k);
  for (int i = 0; i < 12; ++i) sg[12 * (long)k + i] = g[i];
}

constexpr int BARRIER_HESS_THREADS = 128;
template <class HT>
__global__ void __launch_bounds__(BARRIER_HESS_THREADS, 12)
    k_barrier_hess(int n_ct, const ContactRec* __restrict__ ct, const uint8_t* __restrict__ act,
                   const double* __restrict__ Hl, HT* __restrict__ sH) {
  static_assert(144 <= 2 * BARRIER_HESS_THREADS, "two matrix elements per thread at most");
  __shared__ double A[144], V[144], W[144], R[36];
  __shared__ float Af[144], Vf[144], Rf[36];
  const int k = blockIdx.x, t = threadIdx.x;
  if (k >= n_ct) return;  // uniform over the block
  if (!act[ct[k].env]) return;
  for (int e = t; e < 144; e += BARRIER_HESS_THREADS) A[e] = Hl[144 * (long)k + e];
  __syncthreads();
  project_psd_block_warm<12>(A, V, W, R, Af, Vf, Rf);
  for (int e = t; e < 144; e += BARRIER_HESS_THREADS) {
    const int i = e / 12, j = e % 12;
    if (j >= i) sH[78 * (long)k + up_idx(i, j, 12)] = HT(A[e]);
  }
}

// ----------------------------------------------------------------- lagged friction
struct FrictionRec {
  int pts[4];
  int env, pad;
  double c[4];
  double n[3];
  double mu_lambda;
};

// h^2 mu lambda f0(|u|), u = P rel, rel = sum_i c_i (x_i - x_i^t), P = I - n n^T; gradient
// c_i a u and Hessian c_i c_j (a P + b u u^T) with a = f1/y, b = (f1' y - f1)/y^3 (PSD for the
// IPC smoothing f0; at y = 0, a = 2/(eps_v h) and the u u^T term vanishes).
// h^2 mu lambda f0(|u|) value with u and |u| (not inlined, see tet_energy)
__device__ __noinline__ double friction_energy(const FrictionRec& f, const double* __restrict__ ptx,
                                               const double* __restrict__ ptx_t, double h2, double eh, d3* u_out,
                                               double* y_out) {
  d3 rel = mk3(0, 0, 0);
  for (int i = 0; i < 4; ++i) rel = rel + f.c[i] * (ld3(ptx, f.pts[i]) - ld3(ptx_t, f.pts[i]));
  d3 n = mk3(f.n[0], f.n[1], f.n[2]);
  d3 u = rel - dot(n, rel) * n;
  double y = sqrt(dot(u, u));
  *u_out = u;
  *y_out = y;
  double f0 = y < eh ? -y * y * y / (3.0 * eh * eh) + y * y / eh + eh / 3.0 : y;
  return h2 * f.mu_lambda * f0;
}

// tangential force mu lambda f1(|u|) of every lagged friction stencil at positions ptx (N)
__global__ void k_friction_force(int n_fr, const FrictionRec* __restrict__ fr, const double* __restrict__ ptx,
                                 const double* __restrict__ ptx_t, double eh, double* __restrict__ out) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_fr) return;
  const FrictionRec f = fr[k];
  d3 u;
  double y;
  friction_energy(f, ptx, ptx_t, 0.0, eh, &u, &y);
  out[k] = f.mu_lambda * (y < eh ? -y * y / (eh * eh) + 2.0 * y / eh : 1.0);
}

template <int MODE, class HT = double>
__global__ void k_friction(int n_fr, const FrictionRec* __restrict__ fr, const uint8_t* __restrict__ act,
                           const double* __restrict__ ptx, const double* __restrict__ ptx_t, double h2, double eh,
                           double* __restrict__ sE, double* __restrict__ sg, HT* __restrict__ sH) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_fr) return;
  FrictionRec f = fr[k];
  if (!act[f.env]) return;
  d3 u;
  double y;
  sE[k] = friction_energy(f, ptx, ptx_t, h2, eh, &u, &y);
  if (MODE == MODE_ENERGY) return;
  double s = h2 * f.mu_lambda;
  double f1, f2;
  if (y < eh) {
    f1 = -y * y / (eh * eh) + 2.0 * y / eh;
    f2 = -2.0 * y / (eh * eh) + 2.0 / eh;
  } else {
    f1 = 1.0;
    f2 = 0.0;
  }
  double a = y > 0.0 ? f1 / y : 2.0 / eh;
  double bc = y > 0.0 ? (f2 * y - f1) / (y * y * y) : 0.0;
  for (int i = 0; i < 4; ++i) {
    sg[12 * (long)k + 3 * i] = s * f.c[i] * a * u.x;
    sg[12 * (long)k + 3 * i + 1] = s * f.c[i] * a * u.y;
    sg[12 * (long)k + 3 * i + 2] = s * f.c[i] * a * u.z;
  }
  if (MODE == MODE_GRAD) return;
  double M[9];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) M[3 * r + c] = a * ((r == c ? 1.0 : 0.0) - f.n[r] * f.n[c]) + bc * comp(u, r) * comp(u, c);
  for (int i = 0; i < 12; ++i)
    for (int j = i; j < 12; ++j)
      sH[78 * (long)k + up_idx(i, j, 12)] = HT(s * f.c[i / 3] * f.c[j / 3] * M[3 * (i % 3) + (j % 3)]);
}

// ----------------------------------------------------------------- joints
// A point joint between two affine bodies: its two anchors are points of the point table (on
// their bodies, not on any surface). As a stencil its points are (a, b, a, b) with the last two
// carrying nothing.
struct JointRec {
  int pts[2];
  int env, pad;
  double k;  // stiffness (N/m)
};
// 1/2 h^2 k |x_a - x_b|^2: gradient h^2 k (r, -r) on the two anchors, Hessian h^2 k [I, -I; -I, I]
// (PSD as it stands).
template <int MODE, class HT = double>
__global__ void k_joint(int n_jt, const JointRec* __restrict__ jt, const uint8_t* __restrict__ act,
                        const double* __restrict__ ptx, double h2, double* __restrict__ sE, double* __restrict__ sg,
                        HT* __restrict__ sH) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_jt) return;
  const JointRec J = jt[k];
  if (!act[J.env]) return;
  const d3 xa = ld3(ptx, J.pts[0]), xb = ld3(ptx, J.pts[1]);
  const double r[3] = {xa.x - xb.x, xa.y - xb.y, xa.z - xb.z};
  const double c = h2 * J.k;
  sE[k] = 0.5 * c * (r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
  if (MODE == MODE_ENERGY) return;
  for (int i = 0; i < 3; ++i) {
    sg[12 * (long)k + i] = c * r[i];
    sg[12 * (long)k + 3 + i] = -c * r[i];
    sg[12 * (long)k + 6 + i] = 0.0;
    sg[12 * (long)k + 9 + i] = 0.0;
  }
  if (MODE == MODE_GRAD) return;
  for (int i = 0; i < 12; ++i)
    for (int j = i; j < 12; ++j) {
      double v = 0.0;
      if (i < 6 && j < 6 && (i % 3) == (j % 3)) v = (i / 3 == j / 3) ? c : -c;
      sH[78 * (long)k + up_idx(i, j, 12)] = HT(v);
    }
}

// ----------------------------------------------------------------- per-env energy sums
// One block per env; every sub-range is summed by a fixed-order tree. Dynamic lists (contacts,
// friction) are env-sorted; their env ranges are found by binary search.
DEV int lower_env(const int* envs, int lo, int hi, int e) {
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (envs[mid] < e) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}
struct EnergyLists {
  const double* nodeE; const int* node_off;     // soft-node inertia per node
  const double* tetE; const int* tet_off;
  const double* bodyE; const int* body_off;
  const double* stE; const int* st_env; int n_pt, n_ee, n_frpt, n_fr, n_jt;  // stencils: [pt|ee|frpt|free|joints]
};
__global__ void k_env_energy(int n_env, EnergyLists L, const uint8_t* __restrict__ act, double* __restrict__ out) {
  __shared__ double sh[256];
  int e = blockIdx.x;
  if (!act[e]) return;
  double acc = 0.0;
  auto range_sum = [&](const double* v, int b, int en) {
    double s = 0.0;
    for (int i = b + threadIdx.x; i < en; i += blockDim.x) s += v[i];
    return block_sum(s, sh);
  };
  acc += range_sum(L.nodeE, L.node_off[e], L.node_off[e + 1]);
  acc += range_sum(L.tetE, L.tet_off[e], L.tet_off[e + 1]);
  acc += range_sum(L.bodyE, L.body_off[e], L.body_off[e + 1]);
  const int nc = L.n_pt + L.n_ee;
  int bounds[6] = {0, L.n_pt, nc, nc + L.n_frpt, nc + L.n_fr, nc + L.n_fr + L.n_jt};
  for (int r = 0; r < 5; ++r) {
    int b = lower_env(L.st_env, bounds[r], bounds[r + 1], e);
    int en = lower_env(L.st_env, bounds[r], bounds[r + 1], e + 1);
    acc += range_sum(L.stE, b, en);
  }
  if (threadIdx.x == 0) out[e] = acc;
}
