// Assembly and the per-environment block-Jacobi PCG (the "parallel computing in linear solves"
// of Sec. III-A). Soft vertices are 3-DOF nodes in a 3x3-block BSR matrix whose pattern is
// fixed by the tet mesh; each affine body is 4 nodes with a dense 12x12 block; contacts and
// friction are 4-point stencils applied matrix-free. Everything is gathered in fixed order.
//
// Work is cut into tiles that never straddle environments: a soft tile holds up to TILE nodes
// of one env (one thread per node), a body tile up to TILE bodies of one env (one thread per
// body). Per-tile partial dot products are reduced per env in tile order, so each env's PCG
// scalars are exact functions of its own data and every env stops on its own.
#pragma once
#include "common.cuh"
#include "energy.cuh"

constexpr int TILE = 256;

struct Tiles {
  const int* env;
  const int* kind;  // 0 soft nodes, 1 bodies
  const int* begin;
  const int* end;
  const int* env_off;  // per env tile range
};

struct Layout {
  const int* node_env;
  const int* node_body;   // body index for body nodes, -1 for soft nodes
  const uint8_t* node_kin;
  const double* node_mass;
  const int* body_node;
  const uint8_t* body_kin;
  const int* pt_node;
  const double* pt_xb;
};

// weight of DOF node i in the position of point pt (1 for soft points; 1, xb0, xb1, xb2 for
// the p, a1, a2, a3 nodes of an affine point)
DEV double point_weight(const Layout& L, int pt, int node) {
  int nd = L.pt_node[pt];
  if (nd >= 0) return 1.0;
  int blk = node - L.body_node[-1 - nd];
  return blk == 0 ? 1.0 : L.pt_xb[3 * pt + blk - 1];
}

DEV d3 point_gather(const Layout& L, int pt, const double* __restrict__ v) {
  int nd = L.pt_node[pt];
  if (nd >= 0) return ld3(v, nd);
  long base = L.body_node[-1 - nd];
  return ld3(v, base) + L.pt_xb[3 * pt] * ld3(v, base + 1) + L.pt_xb[3 * pt + 1] * ld3(v, base + 2) +
         L.pt_xb[3 * pt + 2] * ld3(v, base + 3);
}

// ---------------------------------------------------------------- gradient / BSR / precond
__global__ void k_assemble_grad(int n_nodes, Layout L, const uint8_t* __restrict__ act, const double* __restrict__ x,
                                const double* __restrict__ xtilde, const int* __restrict__ nt_ptr,
                                const int* __restrict__ nt_src, const double* __restrict__ tg,
                                const double* __restrict__ bg, const int* __restrict__ ns_ptr,
                                const int* __restrict__ ns_src, const int* __restrict__ st_pts,
                                const double* __restrict__ sg, double* __restrict__ grad, double* __restrict__ nodeE) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_nodes) return;
  if (!act[L.node_env[i]]) return;
  d3 g = mk3(0, 0, 0);
  int b = L.node_body[i];
  if (b < 0) {
    if (!L.node_kin[i]) {
      d3 dx = ld3(x, i) - ld3(xtilde, i);
      g = L.node_mass[i] * dx;
    }
    for (int k = nt_ptr[i]; k < nt_ptr[i + 1]; ++k) {
      int src = nt_src[k];
      g = g + ld3(tg, src);  // tg rows are (tet*4 + local) triples
    }
  } else {
    int blk = i - L.body_node[b];
    g = ld3(bg, 4L * b + blk);
  }
  for (int k = ns_ptr[i]; k < ns_ptr[i + 1]; ++k) {
    int e = ns_src[k], s = e >> 2, slot = e & 3;
    double w = point_weight(L, st_pts[4 * s + slot], i);
    g = g + w * ld3(sg, 4L * s + slot);
  }
  st3(grad, i, g);
}

// inertia energy of soft free nodes, 1/2 m |x - x~|^2 (per node, summed later in env order)
__global__ void k_inertia_energy(int n_nodes, Layout L, const uint8_t* __restrict__ act, const double* __restrict__ x,
                                 const double* __restrict__ xtilde, double* __restrict__ nodeE) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_nodes) return;
  if (!act[L.node_env[i]]) return;
  double e = 0.0;
  if (L.node_body[i] < 0 && !L.node_kin[i]) {
    d3 dx = ld3(x, i) - ld3(xtilde, i);
    e = 0.5 * L.node_mass[i] * dot(dx, dx);
  }
  nodeE[i] = e;
}

// BSR block k = sum of the tet Hessian blocks that land on it (+ lumped mass on the diagonal)
__global__ void k_assemble_bsr(int nnzb, const int* __restrict__ blk_row, const int* __restrict__ bsr_col, Layout L,
                               const uint8_t* __restrict__ act, const int* __restrict__ bptr,
                               const int* __restrict__ bsrc, const double* __restrict__ tH, double* __restrict__ val) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nnzb) return;
  int row = blk_row[k];
  if (!act[L.node_env[row]]) return;
  double v[9];
  double m = (bsr_col[k] == row) ? L.node_mass[row] : 0.0;
  for (int i = 0; i < 9; ++i) v[i] = (i % 4 == 0) ? m : 0.0;
  for (int c = bptr[k]; c < bptr[k + 1]; ++c) {
    int src = bsrc[c];
    int t = src >> 4, a = (src >> 2) & 3, b = src & 3;
    const double* H = tH + 90L * t + 9 * up_idx(min(a, b), max(a, b), 4);
    if (a <= b)
      for (int i = 0; i < 9; ++i) v[i] += H[i];
    else
      for (int r = 0; r < 3; ++r)
        for (int cc = 0; cc < 3; ++cc) v[3 * r + cc] += H[3 * cc + r];
  }
  for (int i = 0; i < 9; ++i) val[9L * k + i] = v[i];
}

// 3x3 block of a packed 12x12 stencil Hessian between slots a and b
DEV void stencil_block(const double* __restrict__ H78, int a, int b, double* out) {
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) out[3 * r + c] = H78[sym_idx(3 * a + r, 3 * b + c, 12)];
}

__global__ void k_precond_soft(int n_nodes, Layout L, const uint8_t* __restrict__ act, const int* __restrict__ diag,
                               const double* __restrict__ bsr_val, const int* __restrict__ ns_ptr,
                               const int* __restrict__ ns_src, const double* __restrict__ sH, double* __restrict__ Pinv) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_nodes) return;
  if (L.node_body[i] >= 0 || !act[L.node_env[i]]) return;
  double D[9];
  if (L.node_kin[i]) {
    for (int k = 0; k < 9; ++k) Pinv[9L * i + k] = 0.0;
    return;
  }
  for (int k = 0; k < 9; ++k) D[k] = bsr_val[9L * diag[i] + k];
  for (int k = ns_ptr[i]; k < ns_ptr[i + 1]; ++k) {
    int e = ns_src[k], s = e >> 2, slot = e & 3;
    double B[9];
    stencil_block(sH + 78L * s, slot, slot, B);
    for (int q = 0; q < 9; ++q) D[q] += B[q];
  }
  inv_sym3(D, Pinv + 9L * i);
}

// one block of 144 threads per body: thread (row, col) of the 12x12 body block adds
// sum over the body's stencil slot pairs (a, c) of w_a[I] w_c[J] H_s[3a+k][3c+l].
__global__ void k_precond_body(int n_bodies, Layout L, const int* __restrict__ benv, const uint8_t* __restrict__ act,
                               const double* __restrict__ bH, const int* __restrict__ ns_ptr,
                               const int* __restrict__ ns_src, const int* __restrict__ st_pts,
                               const double* __restrict__ sH, double* __restrict__ Pinv) {
  __shared__ double P[144];
  int b = blockIdx.x;
  if (!act[benv[b]]) return;
  int t = threadIdx.x;
  int row = t / 12, col = t % 12;
  int I = row / 3, k = row % 3, J = col / 3, l = col % 3;
  double v = bH[144L * b + t];
  if (!L.body_kin[b]) {
    int pn = L.body_node[b];
    int beg = ns_ptr[pn], end = ns_ptr[pn + 1];
    int g = beg;
    while (g < end) {
      int s = ns_src[g] >> 2;
      int ge = g;
      while (ge < end && (ns_src[ge] >> 2) == s) ++ge;
      for (int x = g; x < ge; ++x) {
        int a = ns_src[x] & 3;
        int pa = st_pts[4 * s + a];
        double wa = I == 0 ? 1.0 : L.pt_xb[3 * pa + I - 1];
        for (int y = g; y < ge; ++y) {
          int c = ns_src[y] & 3;
          int pc = st_pts[4 * s + c];
          double wc = J == 0 ? 1.0 : L.pt_xb[3 * pc + J - 1];
          v += wa * wc * sH[78L * s + sym_idx(3 * a + k, 3 * c + l, 12)];
        }
      }
      g = ge;
    }
  }
  P[t] = v;
  __syncthreads();
  if (t == 0) {
    double A[144];
    for (int i = 0; i < 144; ++i) A[i] = P[i];
    if (L.body_kin[b]) {
      for (int i = 0; i < 144; ++i) A[i] = 0.0;
    } else {
      spd_inverse<12>(A);
    }
    for (int i = 0; i < 144; ++i) P[i] = A[i];
  }
  __syncthreads();
  Pinv[144L * b + t] = P[t];
}

// ---------------------------------------------------------------- matrix-free stencil product
// t_s = H_s (P_s d) for every stencil of an env whose solve is still running
__global__ void k_stencil_mv(int n_st, Layout L, const int* __restrict__ st_env, const int* __restrict__ st_pts,
                             const uint8_t* __restrict__ run, const double* __restrict__ sH, const double* __restrict__ d,
                             double* __restrict__ st_t) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_st) return;
  if (!run[st_env[s]]) return;
  double u[12];
  for (int a = 0; a < 4; ++a) {
    d3 v = point_gather(L, st_pts[4 * s + a], d);
    u[3 * a] = v.x;
    u[3 * a + 1] = v.y;
    u[3 * a + 2] = v.z;
  }
  const double* H = sH + 78L * s;
  for (int i = 0; i < 12; ++i) {
    double acc = 0.0;
    for (int j = 0; j < 12; ++j) acc += H[sym_idx(i, j, 12)] * u[j];
    st_t[12L * s + i] = acc;
  }
}

struct SpmvArgs {
  const int* bsr_ptr;
  const int* bsr_col;
  const double* bsr_val;
  const double* bH;
  const int* ns_ptr;
  const int* ns_src;
  const int* st_pts;
  const double* st_t;
};

DEV d3 stencil_gather(const Layout& L, const SpmvArgs& A, int i) {
  d3 acc = mk3(0, 0, 0);
  for (int k = A.ns_ptr[i]; k < A.ns_ptr[i + 1]; ++k) {
    int e = A.ns_src[k], s = e >> 2, slot = e & 3;
    double w = point_weight(L, A.st_pts[4 * s + slot], i);
    acc = acc + w * ld3(A.st_t, 4L * s + slot);
  }
  return acc;
}

// y = A d on one tile; returns this thread's d . y (kinematic rows give y = 0)
DEV double spmv_tile_item(const Layout& L, const SpmvArgs& A, int kind, int item, const double* __restrict__ d,
                          double* __restrict__ y) {
  if (kind == 0) {
    int i = item;
    d3 acc = mk3(0, 0, 0);
    if (!L.node_kin[i]) {
      for (int k = A.bsr_ptr[i]; k < A.bsr_ptr[i + 1]; ++k) {
        const double* B = A.bsr_val + 9L * k;
        d3 dv = ld3(d, A.bsr_col[k]);
        acc = acc + mk3(B[0] * dv.x + B[1] * dv.y + B[2] * dv.z, B[3] * dv.x + B[4] * dv.y + B[5] * dv.z,
                        B[6] * dv.x + B[7] * dv.y + B[8] * dv.z);
      }
      acc = acc + stencil_gather(L, A, i);
    }
    st3(y, i, acc);
    return dot(acc, ld3(d, i));
  }
  int b = item;
  long base = L.body_node[b];
  double r = 0.0;
  if (L.body_kin[b]) {
    for (int k = 0; k < 12; ++k) y[3 * base + k] = 0.0;
    return 0.0;
  }
  const double* H = A.bH + 144L * b;
  double dv[12];
  for (int k = 0; k < 12; ++k) dv[k] = d[3 * base + k];
  for (int I = 0; I < 4; ++I) {
    d3 sg = stencil_gather(L, A, base + I);
    for (int k = 0; k < 3; ++k) {
      double acc = comp(sg, k);
      for (int j = 0; j < 12; ++j) acc += H[12 * (3 * I + k) + j] * dv[j];
      y[3 * (base + I) + k] = acc;
      r += acc * dv[3 * I + k];
    }
  }
  return r;
}

// algorithmic bytes of one row item: BSR blocks (72 B values + 4 B index), the d read and y
// write (24 B each), row pointers (8 B), stencil entries (4 B index + 24 B stencil product);
// a body row item is its dense 12x12 block (1152 B) plus 96 B read and 96 B written.
DEV double spmv_item_bytes(const Layout& L, const SpmvArgs& A, int kind, int item) {
  if (kind == 0) {
    if (L.node_kin[item]) return 24.0;
    return 76.0 * (A.bsr_ptr[item + 1] - A.bsr_ptr[item]) + 56.0 + 8.0 +
           28.0 * (A.ns_ptr[item + 1] - A.ns_ptr[item]);
  }
  long base = L.body_node[item];
  return 1344.0 + 28.0 * (A.ns_ptr[base + 4] - A.ns_ptr[base]);
}

__global__ void k_spmv(Tiles T, Layout L, SpmvArgs A, const uint8_t* __restrict__ run, const double* __restrict__ d,
                       double* __restrict__ y, double* __restrict__ part, unsigned long long* __restrict__ bytes) {
  __shared__ double sh[TILE];
  int tile = blockIdx.x;
  int e = T.env[tile];
  if (!run[e]) return;
  int item = T.begin[tile] + threadIdx.x;
  double v = 0.0;
  bool ok = item < T.end[tile];
  if (ok) v = spmv_tile_item(L, A, T.kind[tile], item, d, y);
  v = block_sum(v, sh);
  if (threadIdx.x == 0) part[tile] = v;
  if (bytes) {
    double b = block_sum(ok ? spmv_item_bytes(L, A, T.kind[tile], item) : 0.0, sh);
    if (threadIdx.x == 0) atomicAdd(bytes, (unsigned long long)b);
  }
}

// sum of an env's per-tile partials in tile order (thread 0), broadcast to the block
DEV double env_total(const Tiles& T, int e, const double* __restrict__ part, double* sh1) {
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = T.env_off[e]; k < T.env_off[e + 1]; ++k) s += part[k];
    *sh1 = s;
  }
  __syncthreads();
  double r = *sh1;
  __syncthreads();
  return r;
}

// z = M^-1 r for one item, returns (r.z, r.r) contributions
DEV void precond_item(const Layout& L, int kind, int item, const double* __restrict__ Ps, const double* __restrict__ Pb,
                      const double* __restrict__ r, double* __restrict__ z, double* rz, double* rr) {
  if (kind == 0) {
    int i = item;
    d3 rv = ld3(r, i);
    const double* P = Ps + 9L * i;
    d3 zv = mk3(P[0] * rv.x + P[1] * rv.y + P[2] * rv.z, P[3] * rv.x + P[4] * rv.y + P[5] * rv.z,
                P[6] * rv.x + P[7] * rv.y + P[8] * rv.z);
    st3(z, i, zv);
    *rz = dot(rv, zv);
    *rr = dot(rv, rv);
    return;
  }
  int b = item;
  long base = 3L * L.body_node[b];
  const double* P = Pb + 144L * b;
  double rv[12];
  for (int k = 0; k < 12; ++k) rv[k] = r[base + k];
  double a = 0.0, c = 0.0;
  for (int i = 0; i < 12; ++i) {
    double s = 0.0;
    for (int j = 0; j < 12; ++j) s += P[12 * i + j] * rv[j];
    z[base + i] = s;
    a += rv[i] * s;
    c += rv[i] * rv[i];
  }
  *rz = a;
  *rr = c;
}

// PCG initialisation: z = M^-1 r, d = z, x = 0; partials of r.z and r.r
__global__ void k_pcg_init(Tiles T, Layout L, const uint8_t* __restrict__ act, const double* __restrict__ Ps,
                           const double* __restrict__ Pb, const double* __restrict__ r, double* __restrict__ z,
                           double* __restrict__ d, double* __restrict__ xs, double* __restrict__ prz,
                           double* __restrict__ prr) {
  __shared__ double sh[TILE];
  int tile = blockIdx.x;
  int e = T.env[tile];
  if (!act[e]) return;
  int item = T.begin[tile] + threadIdx.x;
  double a = 0.0, c = 0.0;
  if (item < T.end[tile]) {
    int kind = T.kind[tile];
    precond_item(L, kind, item, Ps, Pb, r, z, &a, &c);
    int n0 = kind == 0 ? item : L.body_node[item];
    int nn = kind == 0 ? 1 : 4;
    for (int k = 3 * n0; k < 3 * (n0 + nn); ++k) {
      d[k] = z[k];
      xs[k] = 0.0;
    }
  }
  a = block_sum(a, sh);
  c = block_sum(c, sh);
  if (threadIdx.x == 0) {
    prz[tile] = a;
    prr[tile] = c;
  }
}

struct PcgState {
  double* rz;      // [2][n_env]
  double* bb;      // |b|^2
  int* it;
  uint8_t* run;    // 1 while the env's solve is running
  int* active;     // number of running solves
  long long* total_iters;  // per env cumulative
};

__global__ void k_pcg_init_env(int n_env, Tiles T, const uint8_t* __restrict__ act, const double* __restrict__ prz,
                               const double* __restrict__ prr, PcgState S) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_env) return;
  if (!act[e]) {
    S.run[e] = 0;
    return;
  }
  double a = 0.0, c = 0.0;
  for (int k = T.env_off[e]; k < T.env_off[e + 1]; ++k) {
    a += prz[k];
    c += prr[k];
  }
  S.rz[e] = a;
  S.bb[e] = c;
  S.it[e] = 0;
  bool go = c > 0.0;
  S.run[e] = go ? 1 : 0;
  if (go) atomicAdd(S.active, 1);
}

// alpha = rz / d.y; x += alpha d; r -= alpha y; z = M^-1 r; partials of r.z and r.r
__global__ void k_pcg_update(Tiles T, Layout L, PcgState S, int parity, int n_env, const double* __restrict__ pdy,
                             const double* __restrict__ Ps, const double* __restrict__ Pb, const double* __restrict__ d,
                             const double* __restrict__ y, double* __restrict__ xs, double* __restrict__ r,
                             double* __restrict__ z, double* __restrict__ prz, double* __restrict__ prr) {
  __shared__ double sh[TILE];
  __shared__ double s1;
  int tile = blockIdx.x;
  int e = T.env[tile];
  if (!S.run[e]) return;
  double dy = env_total(T, e, pdy, &s1);
  double alpha = dy > 0.0 ? S.rz[parity * n_env + e] / dy : 0.0;
  int item = T.begin[tile] + threadIdx.x;
  double a = 0.0, c = 0.0;
  if (item < T.end[tile]) {
    int kind = T.kind[tile];
    int n0 = kind == 0 ? item : L.body_node[item];
    int nn = kind == 0 ? 1 : 4;
    for (int k = 3 * n0; k < 3 * (n0 + nn); ++k) {
      xs[k] += alpha * d[k];
      r[k] -= alpha * y[k];
    }
    precond_item(L, kind, item, Ps, Pb, r, z, &a, &c);
  }
  a = block_sum(a, sh);
  c = block_sum(c, sh);
  if (threadIdx.x == 0) {
    prz[tile] = a;
    prr[tile] = c;
  }
}

// beta = rz_new / rz; d = z + beta d; the env's first tile records rz_new and the stop test
__global__ void k_pcg_direction(Tiles T, Layout L, PcgState S, int parity, int n_env, double tol2, int max_it,
                                const double* __restrict__ prz, const double* __restrict__ prr,
                                const double* __restrict__ pdy, const double* __restrict__ z, double* __restrict__ d) {
  __shared__ double s1, s2, s3;
  int tile = blockIdx.x;
  int e = T.env[tile];
  if (!S.run[e]) return;
  if (threadIdx.x == 0) {
    double a = 0.0, c = 0.0, g = 0.0;
    for (int k = T.env_off[e]; k < T.env_off[e + 1]; ++k) {
      a += prz[k];
      c += prr[k];
      g += pdy[k];
    }
    s1 = a;
    s2 = c;
    s3 = g;
  }
  __syncthreads();
  double rz_new = s1, rr = s2, dy = s3;
  double rz_old = S.rz[parity * n_env + e];
  double beta = rz_old > 0.0 ? rz_new / rz_old : 0.0;
  int item = T.begin[tile] + threadIdx.x;
  if (item < T.end[tile]) {
    int kind = T.kind[tile];
    int n0 = kind == 0 ? item : L.body_node[item];
    int nn = kind == 0 ? 1 : 4;
    for (int k = 3 * n0; k < 3 * (n0 + nn); ++k) d[k] = z[k] + beta * d[k];
  }
  if (tile == T.env_off[e] && threadIdx.x == 0) {
    S.rz[(1 - parity) * n_env + e] = rz_new;
    int it = S.it[e] + 1;
    S.it[e] = it;
    S.total_iters[e] += 1;
    bool stop = rr <= tol2 * S.bb[e] || it >= max_it || !(dy > 0.0) || !isfinite(rr);
    if (stop) {
      S.run[e] = 0;
      atomicSub(S.active, 1);
    }
  }
}
