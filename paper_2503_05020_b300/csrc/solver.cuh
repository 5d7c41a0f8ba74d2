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

// Soft-node rows are stored as sliced ELL: 32 consecutive rows form a slice padded to its longest
// row; block kk of lane l, element e (row-major 3x3) sits at vbase + (kk*9 + e)*32 + l, so every
// warp-wide load of one element is one contiguous 256-byte access. Padding columns are -1.
// BSR block k (CSR order) = sum of the tet Hessian blocks that land on it (+ lumped mass on the
// diagonal), written to its sliced-ELL position pos[k].
// Values and sums are in the Hessian precision HT.
template <class HT>
__global__ void k_assemble_bsr(int nnzb, const int* __restrict__ blk_row, const int* __restrict__ bsr_col, Layout L,
                               const uint8_t* __restrict__ act, const int* __restrict__ bptr,
                               const int* __restrict__ bsrc, const HT* __restrict__ tH, const long* __restrict__ pos,
                               HT* __restrict__ val) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nnzb) return;
  int row = blk_row[k];
  if (!act[L.node_env[row]]) return;
  HT v[9];
  HT m = (bsr_col[k] == row) ? HT(L.node_mass[row]) : HT(0);
  for (int i = 0; i < 9; ++i) v[i] = (i % 4 == 0) ? m : HT(0);
  for (int c = bptr[k]; c < bptr[k + 1]; ++c) {
    int src = bsrc[c];
    int t = src >> 4, a = (src >> 2) & 3, b = src & 3;
    const HT* H = tH + 90L * t + 9 * up_idx(min(a, b), max(a, b), 4);
    if (a <= b)
      for (int i = 0; i < 9; ++i) v[i] += H[i];
    else
      for (int r = 0; r < 3; ++r)
        for (int cc = 0; cc < 3; ++cc) v[3 * r + cc] += H[3 * cc + r];
  }
  for (int i = 0; i < 9; ++i) val[pos[k] + 32L * i] = v[i];
}

// 3x3 block of a packed 12x12 stencil Hessian between slots a and b
template <class HT>
DEV void stencil_block(const HT* __restrict__ H78, int a, int b, HT* out) {
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) out[3 * r + c] = H78[sym_idx(3 * a + r, 3 * b + c, 12)];
}

template <class HT>
__global__ void k_precond_soft(int n_nodes, Layout L, const uint8_t* __restrict__ act, const long* __restrict__ diag_pos,
                               const HT* __restrict__ bsr_val, const int* __restrict__ ns_ptr,
                               const int* __restrict__ ns_src, const HT* __restrict__ sH, HT* __restrict__ Pinv) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_nodes) return;
  if (L.node_body[i] >= 0 || !act[L.node_env[i]]) return;
  HT D[9];
  if (L.node_kin[i]) {
    for (int k = 0; k < 9; ++k) Pinv[9L * i + k] = HT(0);
    return;
  }
  for (int k = 0; k < 9; ++k) D[k] = bsr_val[diag_pos[i] + 32L * k];
  for (int k = ns_ptr[i]; k < ns_ptr[i + 1]; ++k) {
    int e = ns_src[k], s = e >> 2, slot = e & 3;
    HT B[9];
    stencil_block(sH + 78L * s, slot, slot, B);
    for (int q = 0; q < 9; ++q) D[q] += B[q];
  }
  inv_sym3<HT>(D, Pinv + 9L * i);
}

// one block of 144 threads per body: thread (row, col) of the 12x12 body block adds
// sum over the body's stencil slot pairs (a, c) of w_a[I] w_c[J] H_s[3a+k][3c+l].
template <class HT>
__global__ void k_precond_body(int n_bodies, Layout L, const int* __restrict__ benv, const uint8_t* __restrict__ act,
                               const HT* __restrict__ bH, const int* __restrict__ ns_ptr,
                               const int* __restrict__ ns_src, const HT* __restrict__ ns_xb,
                               const HT* __restrict__ sH, HT* __restrict__ Pinv) {
  __shared__ double P[144];  // the block and its inverse in FP64 whatever HT is: the 12x12
  __shared__ double D[12];   // body block mixes mass, orthogonality and contact scales
  int b = blockIdx.x;
  if (!act[benv[b]]) return;
  int t = threadIdx.x;
  int row = t / 12, col = t % 12;
  int I = row / 3, k = row % 3, J = col / 3, l = col % 3;
  double v = double(bH[144L * b + t]);
  const bool kin = L.body_kin[b];
  if (!kin) {
    // every pair of slots (a, c) of one stencil on the body adds (1, xb_a)(1, xb_c)^T (x) H_ac;
    // a stencil's entries are consecutive (at most 4), so the partners of entry x lie within
    // x - 3 .. x + 3, and every load of an entry depends on its index alone
    int pn = L.body_node[b];
    int beg = ns_ptr[pn], end = ns_ptr[pn + 1];
    for (int x = beg; x < end; ++x) {
      const int ex = ns_src[x], s = ex >> 2, a = ex & 3;
      const double wa = I == 0 ? 1.0 : double(ns_xb[3L * x + I - 1]);
      for (int y = max(beg, x - 3); y <= min(end - 1, x + 3); ++y) {
        const int ey = ns_src[y];
        if ((ey >> 2) != s) continue;
        const int c = ey & 3;
        const double wc = J == 0 ? 1.0 : double(ns_xb[3L * y + J - 1]);
        v += wa * wc * double(sH[78L * s + sym_idx(3 * a + k, 3 * c + l, 12)]);
      }
    }
  }
  P[t] = v;
  if (row == col) D[row] = v;
  __syncthreads();
  // In-place Gauss-Jordan inverse, one entry per thread, no pivoting: for an SPD block the
  // pivots are the squared Cholesky pivots, all positive. A pivot that is not positive (a block
  // that is not SPD) falls back to the inverse of the diagonal, 0 where that is not > 0.
  bool ok = !kin;
  for (int q = 0; q < 12 && ok; ++q) {
    const double pqq = P[13 * q], piq = P[12 * row + q], pqj = P[12 * q + col], pij = P[t];
    __syncthreads();
    if (!(pqq > 0.0)) {  // uniform over the block
      ok = false;
      break;
    }
    const double inv = 1.0 / pqq;
    double nv;
    if (row == q && col == q) nv = inv;
    else if (row == q) nv = pqj * inv;
    else if (col == q) nv = -piq * inv;
    else nv = pij - piq * pqj * inv;
    P[t] = nv;
    __syncthreads();
  }
  double out = P[t];
  if (kin) out = 0.0;
  else if (!ok) out = (row == col && D[row] > 0.0) ? 1.0 / D[row] : 0.0;
  Pinv[144L * b + t] = HT(out);
}

// ---------------------------------------------------------------- matrix-free stencil product
// Vector loads: plain, or L2-coherent (for vectors that other CTAs write while a kernel runs).
template <bool CG, class VT>
DEV VT ldv(const VT* p, long i) {
  if (CG) return __ldcg(p + i);
  return p[i];
}
DEV d3 ldcg3(const double* p, long i) { return d3{__ldcg(p + 3 * i), __ldcg(p + 3 * i + 1), __ldcg(p + 3 * i + 2)}; }

// position-weighted gather of a 3-vector field at point pt: the node's value for a soft point,
// v_p + xb0 v_a1 + xb1 v_a2 + xb2 v_a3 for a point of an affine body
template <bool CG, class VT>
DEV void point_gather_t(const Layout& L, int pt, const VT* v, VT out[3]) {
  int nd = L.pt_node[pt];
  if (nd >= 0) {
    for (int c = 0; c < 3; ++c) out[c] = ldv<CG>(v, 3L * nd + c);
    return;
  }
  long base = L.body_node[-1 - nd];
  const double* xb = L.pt_xb + 3 * pt;
  const VT x0 = VT(xb[0]), x1 = VT(xb[1]), x2 = VT(xb[2]);
  for (int c = 0; c < 3; ++c)
    out[c] = ldv<CG>(v, 3 * base + c) + x0 * ldv<CG>(v, 3 * base + 3 + c) + x1 * ldv<CG>(v, 3 * base + 6 + c) +
             x2 * ldv<CG>(v, 3 * base + 9 + c);
}

// t_s = H_s (P_s d) for stencil s by the 16 lanes of a half-warp (H_s: packed upper triangle,
// 78 values in the Hessian precision HT; products and sums in the vector type VT). Every lane
// of the warp calls it (shuffles); ok = false idles a half. Lanes 0..3 gather the stencil's
// points, the 12 entries of P_s d reach every lane by shuffles, and lane i < 12 forms row i from
// 12 independent loads, summed in column order.
template <bool CG, class HT, class VT>
DEV void stencil_product_hw(const Layout& L, const int* __restrict__ st_pts, const HT* __restrict__ sH, const VT* d,
                            VT* st_t, int s, bool ok) {
  const int lane = threadIdx.x & 31, half = lane & 16, l = lane & 15;
  VT v[3] = {VT(0), VT(0), VT(0)};
  if (ok && l < 4) point_gather_t<CG>(L, st_pts[4 * s + l], d, v);
  VT u[12];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 3; ++c) u[3 * a + c] = __shfl_sync(0xffffffffu, v[c], half + a);
  if (ok && l < 12) {
    const HT* H = sH + 78L * s;
    VT acc = VT(0);
#pragma unroll
    for (int j = 0; j < 12; ++j) acc += VT(H[sym_idx(l, j, 12)]) * u[j];
    st_t[12L * s + l] = acc;
  }
}

// every stencil of an env whose solve is still running; one half-warp per stencil
template <class HT, class VT>
__global__ void k_stencil_mv(int n_st, Layout L, const int* __restrict__ st_env, const int* __restrict__ st_pts,
                             const uint8_t* __restrict__ run, const HT* __restrict__ sH, const VT* __restrict__ d,
                             VT* __restrict__ st_t) {
  int s = (blockIdx.x * blockDim.x + threadIdx.x) >> 4;
  bool ok = s < n_st && run[st_env[s]];
  stencil_product_hw<false>(L, st_pts, sH, d, st_t, s, ok);
}

template <class HT>
struct SellT {
  const int* tile_slice;  // first slice of each soft tile
  const int* width;       // blocks per row of each slice
  const long* vbase;      // value offset of each slice
  const long* cbase;      // column offset of each slice
  const int* col;         // block column (node); padding blocks point at the row itself
  const HT* val;
};

// Matrix in the Hessian precision HT, vectors (and stencil products) in VT.
template <class HT, class VT>
struct SpmvArgsT {
  SellT<HT> S;
  const int* bsr_ptr;  // CSR row pointers (for the algorithmic byte count only)
  const HT* bH;
  const int* ns_ptr;
  const int* ns_src;  // stencil*4 + slot of each incidence entry (row-sorted)
  const HT* ns_w;     // weight of the entry's node in the slot's point position
  const HT* ns_xb;    // body p-node entries: rest coordinates (xb) of the entry's point
  const int* st_pts;
  const VT* st_t;      // stencil products
  const HT* sH;        // stencil Hessians (packed)
  const int* sn;       // per stencil point: its node, or -1 - the p node of its affine body
  const HT* sxb;       // per stencil point: rest coordinates of an affine point (else 0)
};
using SpmvArgs = SpmvArgsT<double, double>;

// Point nodes of every stencil, once per Newton iteration, so that the PCG's stencil products
// need one dependent load (the node) before the vector loads. One thread per stencil point.
template <class HT>
__global__ void k_stencil_nodes(int n_st, Layout L, const int* __restrict__ st_pts, const int* __restrict__ st_env,
                                const uint8_t* __restrict__ act, int* __restrict__ sn, HT* __restrict__ sxb) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= 4 * n_st) return;
  if (!act[st_env[k >> 2]]) return;
  int pt = st_pts[k], nd = L.pt_node[pt];
  if (nd >= 0) {
    sn[k] = nd;
    for (int c = 0; c < 3; ++c) sxb[3L * k + c] = HT(0);
  } else {
    sn[k] = -1 - L.body_node[-1 - nd];
    for (int c = 0; c < 3; ++c) sxb[3L * k + c] = HT(L.pt_xb[3 * pt + c]);
  }
}

// t_s = H_s (P_s v) + beta t_s for stencil s by the 16 lanes of a half-warp, like
// stencil_product_hw but with the point nodes precomputed (k_stencil_nodes): lanes 0..3 load
// their point's node and then its vector entries. beta = 0 overwrites t_s without reading it.
// Every lane of the warp calls it; ok = false idles a half.
template <bool CG, class T>
DEV void stencil_product_nodes(const SpmvArgsT<T, T>& A, const T* d, T* st_t, int s, bool ok, T beta = T(0)) {
  const int lane = threadIdx.x & 31, half = lane & 16, l = lane & 15;
  T v[3] = {T(0), T(0), T(0)};
  if (ok && l < 4) {
    const int nd = A.sn[4 * s + l];
    if (nd >= 0) {
      for (int c = 0; c < 3; ++c) v[c] = ldv<CG>(d, 3L * nd + c);
    } else {
      const long base = -1 - nd;
      const T* xb = A.sxb + 3L * (4 * s + l);
      const T x0 = xb[0], x1 = xb[1], x2 = xb[2];
      for (int c = 0; c < 3; ++c)
        v[c] = ldv<CG>(d, 3 * base + c) + x0 * ldv<CG>(d, 3 * base + 3 + c) + x1 * ldv<CG>(d, 3 * base + 6 + c) +
               x2 * ldv<CG>(d, 3 * base + 9 + c);
    }
  }
  T u[12];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 3; ++c) u[3 * a + c] = __shfl_sync(0xffffffffu, v[c], half + a);
  if (ok && l < 12) {
    const T* H = A.sH + 78L * s;
    T acc = T(0);
#pragma unroll
    for (int j = 0; j < 12; ++j) acc += H[sym_idx(l, j, 12)] * u[j];
    if (beta != T(0)) acc = fma(beta, st_t[12L * s + l], acc);
    st_t[12L * s + l] = acc;
  }
}

// weight of every incidence entry, once per Newton iteration, one thread per entry (keys: the
// entry's node, from the sorted incidence keys); entries of a body's p node also get the rest
// coordinates of their point, so one pass over that list serves all 4 body nodes
template <class HT>
__global__ void k_entry_weights(int n_entries, Layout L, const uint8_t* __restrict__ act,
                                const unsigned long long* __restrict__ keys, const int* __restrict__ ns_src,
                                const int* __restrict__ st_pts, HT* __restrict__ ns_w, HT* __restrict__ ns_xb) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_entries) return;
  const int i = (int)keys[k];
  if (!act[L.node_env[i]]) return;
  int b = L.node_body[i];
  bool pnode = b >= 0 && L.body_node[b] == i;
  int pt = st_pts[ns_src[k]];
  ns_w[k] = HT(point_weight(L, pt, i));
  if (pnode)
    for (int c = 0; c < 3; ++c) ns_xb[3L * k + c] = HT(L.pt_xb[3 * pt + c]);
}

// deterministic warp sum (fixed butterfly)
template <class T>
DEV T warp_sum(T v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// y row of one soft node from its sliced-ELL blocks (slice, lane) and its stencil entries;
// returns d_row . y_row. Products in VT; the entries' stencil products are read from st_t.
template <bool CG, class HT, class VT>
DEV VT soft_row(const SpmvArgsT<HT, VT>& A, int slice, int lane, int row, const VT* d, VT* y) {
  VT acc[3] = {VT(0), VT(0), VT(0)};
  int w = A.S.width[slice];
  const int* col = A.S.col + A.S.cbase[slice] + lane;
  const HT* V = A.S.val + A.S.vbase[slice] + lane;
#pragma unroll 4
  for (int kk = 0; kk < w; ++kk) {
    long c = col[32 * kk];  // padding blocks: the row itself, zero values
    VT d0 = ldv<CG>(d, 3 * c), d1 = ldv<CG>(d, 3 * c + 1), d2 = ldv<CG>(d, 3 * c + 2);
    const HT* B = V + 288L * kk;
#pragma unroll
    for (int a = 0; a < 3; ++a) {  // one FMA per block entry
      acc[a] = fma(VT(B[96 * a]), d0, acc[a]);
      acc[a] = fma(VT(B[96 * a + 32]), d1, acc[a]);
      acc[a] = fma(VT(B[96 * a + 64]), d2, acc[a]);
    }
  }
  int k = A.ns_ptr[row], end = A.ns_ptr[row + 1];
#pragma unroll 4
  for (; k < end; ++k) {
    const VT wk = VT(A.ns_w[k]);
    const long src = A.ns_src[k];
    for (int c = 0; c < 3; ++c) acc[c] = acc[c] + wk * ldv<CG>(A.st_t, 3 * src + c);
  }
  for (int c = 0; c < 3; ++c) y[3L * row + c] = acc[c];
  return acc[0] * ldv<CG>(d, 3L * row) + acc[1] * ldv<CG>(d, 3L * row + 1) + acc[2] * ldv<CG>(d, 3L * row + 2);
}

// the same row for a tile thread: kinematic rows get y = 0
template <class HT, class VT>
DEV VT spmv_soft_row(const Layout& L, const SpmvArgsT<HT, VT>& A, int slice, int lane, int row, const VT* __restrict__ d,
                     VT* __restrict__ y) {
  if (L.node_kin[row]) {
    for (int c = 0; c < 3; ++c) y[3L * row + c] = VT(0);
    return VT(0);
  }
  return soft_row<false>(A, slice, lane, row, d, y);
}

// One rigid body per block: y = H_b d_b + sum over every stencil slot on the body of
// (1, xb) (x) t_s[slot], gathered once from the body's p-node list (every slot on the body
// appears there once). 12 partial sums are reduced by warp butterflies, then across warps in
// fixed order. Returns d.y on thread 0.
template <class HT, class VT>
DEV VT spmv_body(const Layout& L, const SpmvArgsT<HT, VT>& A, int b, const VT* __restrict__ d, VT* __restrict__ y) {
  __shared__ VT red[12][TILE / 32];
  __shared__ VT dv[12];
  __shared__ VT dy[12];
  const int t = threadIdx.x, lane = t & 31, wp = t >> 5;
  long base = L.body_node[b];
  bool kin = L.body_kin[b];
  if (t < 12) dv[t] = d[3 * base + t];
  __syncthreads();
  VT acc[12];
  for (int q = 0; q < 12; ++q) acc[q] = VT(0);
  if (!kin) {
    int kb = A.ns_ptr[base], ke = A.ns_ptr[base + 1];
#pragma unroll 2
    for (int k = kb + t; k < ke; k += blockDim.x) {
      const long src = A.ns_src[k];
      const VT tx = A.st_t[3 * src], ty = A.st_t[3 * src + 1], tz = A.st_t[3 * src + 2];
      const HT* xb = A.ns_xb + 3L * k;
      const VT w1 = VT(xb[0]), w2 = VT(xb[1]), w3 = VT(xb[2]);
      acc[0] += tx;
      acc[1] += ty;
      acc[2] += tz;
      acc[3] += w1 * tx;
      acc[4] += w1 * ty;
      acc[5] += w1 * tz;
      acc[6] += w2 * tx;
      acc[7] += w2 * ty;
      acc[8] += w2 * tz;
      acc[9] += w3 * tx;
      acc[10] += w3 * ty;
      acc[11] += w3 * tz;
    }
  }
  for (int q = 0; q < 12; ++q) {
    VT v = warp_sum(acc[q]);
    if (lane == 0) red[q][wp] = v;
  }
  __syncthreads();
  if (t < 12) {
    VT v = VT(0);
    if (!kin) {
      const HT* H = A.bH + 144L * b + 12 * t;
      for (int j = 0; j < 12; ++j) v += VT(H[j]) * dv[j];
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[t][w];
    }
    y[3 * base + t] = v;
    dy[t] = v * dv[t];
  }
  __syncthreads();
  VT r = VT(0);
  if (t == 0)
    for (int q = 0; q < 12; ++q) r += dy[q];
  __syncthreads();
  return r;
}

// algorithmic bytes of one row item with H values of hb bytes: sliced-ELL blocks (9 hb values
// + 4 B column), the d read and y write (3 vb each), row pointers (8 B), stencil entries (4 B
// index + hb weight + 3 vb stencil product); a body is its dense 12x12 block (144 hb) plus its
// d read and y written (12 vb each), and per p-node entry 4 B index + 3 hb rest coordinates +
// 3 vb stencil product.
template <class HT, class VT>
DEV double spmv_item_bytes(const Layout& L, const SpmvArgsT<HT, VT>& A, int kind, int item) {
  const double hb = sizeof(HT), vb = sizeof(VT);
  if (kind == 0) {
    if (L.node_kin[item]) return 3 * vb;
    return (9 * hb + 4) * (A.bsr_ptr[item + 1] - A.bsr_ptr[item]) + 6 * vb + 8.0 +
           (4 + hb + 3 * vb) * (A.ns_ptr[item + 1] - A.ns_ptr[item]);
  }
  long base = L.body_node[item];
  return 144 * hb + 24 * vb + (4 + 3 * hb + 3 * vb) * (A.ns_ptr[base + 1] - A.ns_ptr[base]);
}

template <class HT, class VT>
__global__ void __launch_bounds__(TILE) k_spmv(Tiles T, Layout L, SpmvArgsT<HT, VT> A, const uint8_t* __restrict__ run,
                                               const VT* __restrict__ d, VT* __restrict__ y, double* __restrict__ part,
                                               unsigned long long* __restrict__ bytes) {
  __shared__ double sh[TILE];
  int tile = blockIdx.x;
  int e = T.env[tile];
  if (!run[e]) return;
  int kind = T.kind[tile];
  double v = 0.0, nb = 0.0;
  if (kind == 0) {
    int row = T.begin[tile] + threadIdx.x;
    int slice = A.S.tile_slice[tile] + (threadIdx.x >> 5);
    bool ok = row < T.end[tile];
    if (ok) v = double(spmv_soft_row(L, A, slice, threadIdx.x & 31, row, d, y));
    if (bytes && ok) nb = spmv_item_bytes(L, A, 0, row);
  } else {
    v = double(spmv_body(L, A, T.begin[tile], d, y));
    if (bytes && threadIdx.x == 0) nb = spmv_item_bytes(L, A, 1, T.begin[tile]);
  }
  v = block_sum(v, sh);
  if (threadIdx.x == 0) part[tile] = v;
  if (bytes) {
    double b = block_sum(nb, sh);
    if (threadIdx.x == 0) atomicAdd(bytes, (unsigned long long)b);
  }
}

// sum of an env's per-tile partials by warp 0 (lane-strided, fixed butterfly: deterministic and
// the same in every tile of the env), broadcast to the block
DEV double partial_sum_warp(const Tiles& T, int e, const double* __restrict__ part) {
  int lane = threadIdx.x & 31;
  double s = 0.0;
  for (int k = T.env_off[e] + lane; k < T.env_off[e + 1]; k += 32) s += part[k];
  return warp_sum(s);
}
DEV double env_total(const Tiles& T, int e, const double* __restrict__ part, double* sh1) {
  if (threadIdx.x < 32) {
    double s = partial_sum_warp(T, e, part);
    if (threadIdx.x == 0) *sh1 = s;
  }
  __syncthreads();
  double r = *sh1;
  __syncthreads();
  return r;
}

// z = M^-1 r for one soft node, returns (r.z, r.r)
template <class T>
DEV void precond_soft(int i, const T* __restrict__ Ps, const T* __restrict__ r, T* __restrict__ z, T* rz, T* rr) {
  const T r0 = r[3L * i], r1 = r[3L * i + 1], r2 = r[3L * i + 2];
  const T* P = Ps + 9L * i;
  const T z0 = P[0] * r0 + P[1] * r1 + P[2] * r2, z1 = P[3] * r0 + P[4] * r1 + P[5] * r2,
          z2 = P[6] * r0 + P[7] * r1 + P[8] * r2;
  z[3L * i] = z0;
  z[3L * i + 1] = z1;
  z[3L * i + 2] = z2;
  *rz = r0 * z0 + r1 * z1 + r2 * z2;
  *rr = r0 * r0 + r1 * r1 + r2 * r2;
}

// body preconditioner on one block: threads 0..11 hold one DOF each; rs must be in shared memory
template <class T>
DEV void precond_body(const T* __restrict__ Pb, int b, const T* rs, long base3, T* __restrict__ z, T* rz, T* rr) {
  int t = threadIdx.x;
  *rz = T(0);
  *rr = T(0);
  if (t < 12) {
    const T* P = Pb + 144L * b + 12 * t;
    T s = T(0);
    for (int j = 0; j < 12; ++j) s += P[j] * rs[j];
    z[base3 + t] = s;
    *rz = rs[t] * s;
    *rr = rs[t] * rs[t];
  }
}

// PCG initialisation: z = M^-1 r, d = z, x = 0; partials of r.z and r.r
__global__ void __launch_bounds__(TILE) k_pcg_init(Tiles T, Layout L, const uint8_t* __restrict__ act,
                                                   const double* __restrict__ Ps, const double* __restrict__ Pb,
                                                   const double* __restrict__ r, double* __restrict__ z,
                                                   double* __restrict__ d, double* __restrict__ xs,
                                                   double* __restrict__ prz, double* __restrict__ prr) {
  __shared__ double sh[TILE];
  __shared__ double rs[12];
  int tile = blockIdx.x;
  int e = T.env[tile];
  if (!act[e]) return;
  double a = 0.0, c = 0.0;
  if (T.kind[tile] == 0) {
    int i = T.begin[tile] + threadIdx.x;
    if (i < T.end[tile]) {
      precond_soft(i, Ps, r, z, &a, &c);
      for (int k = 3 * i; k < 3 * i + 3; ++k) {
        d[k] = z[k];
        xs[k] = 0.0;
      }
    }
  } else {
    int b = T.begin[tile];
    long base3 = 3L * L.body_node[b];
    if (threadIdx.x < 12) rs[threadIdx.x] = r[base3 + threadIdx.x];
    __syncthreads();
    precond_body(Pb, b, rs, base3, z, &a, &c);
    if (threadIdx.x < 12) {
      d[base3 + threadIdx.x] = z[base3 + threadIdx.x];
      xs[base3 + threadIdx.x] = 0.0;
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

// one warp per env (launch with 32 threads per block, one block per env)
__global__ void k_pcg_init_env(int n_env, Tiles T, const uint8_t* __restrict__ act, const double* __restrict__ prz,
                               const double* __restrict__ prr, PcgState S) {
  int e = blockIdx.x;
  if (e >= n_env) return;
  if (!act[e]) {
    if (threadIdx.x == 0) S.run[e] = 0;
    return;
  }
  double a = partial_sum_warp(T, e, prz), c = partial_sum_warp(T, e, prr);
  if (threadIdx.x != 0) return;
  S.rz[e] = a;
  S.bb[e] = c;
  S.it[e] = 0;
  bool go = c > 0.0;
  S.run[e] = go ? 1 : 0;
  if (go) atomicAdd(S.active, 1);
}

// alpha = rz / d.y; x += alpha d; r -= alpha y; z = M^-1 r; partials of r.z and r.r
__global__ void __launch_bounds__(TILE) k_pcg_update(Tiles T, Layout L, PcgState S, int parity, int n_env,
                                                     const double* __restrict__ pdy, const double* __restrict__ Ps,
                                                     const double* __restrict__ Pb, const double* __restrict__ d,
                                                     const double* __restrict__ y, double* __restrict__ xs,
                                                     double* __restrict__ r, double* __restrict__ z,
                                                     double* __restrict__ prz, double* __restrict__ prr) {
  __shared__ double sh[TILE];
  __shared__ double s1;
  __shared__ double rs[12];
  int tile = blockIdx.x;
  int e = T.env[tile];
  if (!S.run[e]) return;
  double dy = env_total(T, e, pdy, &s1);
  double alpha = dy > 0.0 ? S.rz[parity * n_env + e] / dy : 0.0;
  double a = 0.0, c = 0.0;
  if (T.kind[tile] == 0) {
    int i = T.begin[tile] + threadIdx.x;
    if (i < T.end[tile]) {
      for (int k = 3 * i; k < 3 * i + 3; ++k) {
        xs[k] += alpha * d[k];
        r[k] -= alpha * y[k];
      }
      precond_soft(i, Ps, r, z, &a, &c);
    }
  } else {
    int b = T.begin[tile];
    long base3 = 3L * L.body_node[b];
    if (threadIdx.x < 12) {
      long k = base3 + threadIdx.x;
      xs[k] += alpha * d[k];
      double rv = r[k] - alpha * y[k];
      r[k] = rv;
      rs[threadIdx.x] = rv;
    }
    __syncthreads();
    precond_body(Pb, b, rs, base3, z, &a, &c);
  }
  a = block_sum(a, sh);
  c = block_sum(c, sh);
  if (threadIdx.x == 0) {
    prz[tile] = a;
    prr[tile] = c;
  }
}

// beta = rz_new / rz; d = z + beta d; the env's first tile records rz_new and the stop test
__global__ void __launch_bounds__(TILE) k_pcg_direction(Tiles T, Layout L, PcgState S, int parity, int n_env,
                                                        double tol2, int max_it, const double* __restrict__ prz,
                                                        const double* __restrict__ prr, const double* __restrict__ pdy,
                                                        const double* __restrict__ z, double* __restrict__ d) {
  __shared__ double s1, s2, s3;
  int tile = blockIdx.x;
  int e = T.env[tile];
  if (!S.run[e]) return;
  if (threadIdx.x < 32) {
    double a = partial_sum_warp(T, e, prz), c = partial_sum_warp(T, e, prr), g = partial_sum_warp(T, e, pdy);
    if (threadIdx.x == 0) {
      s1 = a;
      s2 = c;
      s3 = g;
    }
  }
  __syncthreads();
  double rz_new = s1, rr = s2, dy = s3;
  double rz_old = S.rz[parity * n_env + e];
  double beta = rz_old > 0.0 ? rz_new / rz_old : 0.0;
  if (T.kind[tile] == 0) {
    int i = T.begin[tile] + threadIdx.x;
    if (i < T.end[tile])
      for (int k = 3 * i; k < 3 * i + 3; ++k) d[k] = z[k] + beta * d[k];
  } else if (threadIdx.x < 12) {
    long k = 3L * L.body_node[T.begin[tile]] + threadIdx.x;
    d[k] = z[k] + beta * d[k];
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
