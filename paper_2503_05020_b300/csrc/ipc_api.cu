// Host side of the B300 multi-environment IPC stepper: environment records, the flattened
// device layout of a batch, and the batched Newton loop (Sec. III-A: per-env collision
// isolation, step size, stopping and failure). Every numerical stage runs in the kernels of
// the included headers; the host sequences launches, sizes buffers and polls small counters.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <map>
#include <mutex>
#include <memory>
#include <numeric>
#include <stdexcept>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/ipc.h"
#include "common.cuh"
#include "geometry.cuh"
#include "lbvh.cuh"
#include "energy.cuh"
#include "solver.cuh"
#include "kernels_misc.cuh"
#include "pcg_cluster.cuh"

namespace {

thread_local std::string g_err;

struct IpcError {
  ipc_status st;
  std::string msg;
};
[[noreturn]] void fail_with(ipc_status st, const std::string& m) { throw IpcError{st, m}; }

#define CK(call)                                                                                   \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess) fail_with(IPC_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

template <class T>
struct DBuf {
  T* p = nullptr;
  size_t n = 0;
  DBuf() = default;
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  ~DBuf() { release(); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
  void alloc(size_t m) {  // at least m elements, contents undefined; reuses a capacity of m..2m+1024
    if (m == 0) m = 1;
    if (p && m <= n && n <= 2 * m + 1024) return;
    release();
    cudaError_t e = cudaMalloc(&p, m * sizeof(T));
    if (e != cudaSuccess) {
      p = nullptr;
      fail_with(IPC_ERR_OOM, std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
    }
    n = m;
  }
  void ensure(size_t m) {  // grow-only, contents not preserved
    if (m <= n && p) return;
    alloc(std::max(m, (size_t)(n * 3 / 2 + 64)));
  }
  void upload(const std::vector<T>& v, cudaStream_t s) {
    alloc(v.size());
    if (!v.empty()) CK(cudaMemcpyAsync(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s));
  }
  void zero(cudaStream_t s, size_t m = (size_t)-1) {
    if (p) CK(cudaMemsetAsync(p, 0, std::min(m, n) * sizeof(T), s));
  }
};

// ---------------------------------------------------------------- host environment record
struct HostEnv {
  int id = -1;
  // copies of the descriptor
  struct Soft {
    std::vector<double> verts;
    std::vector<int> tets, tris;
    std::vector<uint8_t> kin;
    double E, nu, rho;
  };
  struct Aff {
    std::vector<double> verts;
    std::vector<int> tris;
    double rho;
    double q0[12], qdot0[12];
    int kin;
    double kpd;  // PD target stiffness (free bodies)
  };
  std::vector<Soft> soft;
  std::vector<Aff> aff;
  double mu = 0;
  int n_steps = 0;
  std::vector<uint8_t> grav;
  std::vector<double> targets;
  // derived (env-local)
  int nsv_verts = 0, nbodies = 0, ntets = 0, ndof = 0;
  std::vector<int> tet_nodes;        // 4 per tet, env-local nodes
  std::vector<double> tet_prm;       // 12 per tet
  std::vector<double> mass;          // per soft node
  std::vector<uint8_t> node_kin;     // per soft node
  std::vector<int> node_handle;      // per node (soft + 4 per body)
  std::vector<double> X0;            // per soft node
  std::vector<double> M4, bvol, bbox;  // per body
  // points: env-local node (soft) or -1-body
  std::vector<int> pt_node;
  std::vector<double> pt_xb, pt_rest;
  std::vector<int> pt_body;  // affine body index (local) or -1 - soft body index
  std::vector<uint8_t> pt_kin;
  std::vector<int> sv, edges, tris;  // point ids
  std::vector<double> edge_rest2;
  // point joints: local anchor points (appended after the surface-capable points) and stiffness
  struct Joint {
    int pa, pb;
    double k;
  };
  std::vector<Joint> joints;
  int n_surf_pts = 0;  // points before the joint anchors
  // the grasped object named by the descriptor (-1: none): a soft body's node range, or an
  // affine body with the mean of its rest vertices; its centre of mass at the initial state
  int obj = -1, obj_affine = 0, obj_first = 0, obj_count = 0;
  double obj_xbar[3] = {0, 0, 0}, obj_com0[3] = {0, 0, 0};
  // state
  std::vector<double> x, v;
  int step = 0, status = ST_ACTIVE, reason = FAIL_NONE;
  long long stats[5] = {0, 0, 0, 0, 0};
  bool checked = false;  // initial intersection check done
  uint64_t est_bytes = 0;
  // Hessian pattern in env-local numbering, built once (an env's pattern never changes), so that
  // a relayout of the batch only concatenates: 3x3-block rows of every local node (body nodes
  // have none), the tet-block contributions of each block in tet order, and the tet corners of
  // each node.
  bool have_pattern = false;
  std::vector<int> bptr, bcol;      // CSR over local nodes (nsv_verts + 4 nbodies rows)
  std::vector<int> blkptr, blksrc;  // per block: contributions 16 t + 4 a + b (local t)
  std::vector<int> ntptr, ntsrc;    // per node: tet corners 4 t + a (local t)
};

// The env's Hessian pattern (see HostEnv): blocks of each row are the sorted distinct tet
// neighbours; an isolated soft vertex keeps a diagonal (mass) block.
void build_pattern(HostEnv& h) {
  if (h.have_pattern) return;
  const int nn = h.nsv_verts + 4 * h.nbodies, nt = h.ntets;
  std::vector<std::vector<int>> adj(nn);
  for (int t = 0; t < nt; ++t)
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) adj[h.tet_nodes[4 * t + a]].push_back(h.tet_nodes[4 * t + b]);
  h.bptr.assign(1, 0);
  h.bcol.clear();
  for (int i = 0; i < nn; ++i) {
    auto& a = adj[i];
    std::sort(a.begin(), a.end());
    a.erase(std::unique(a.begin(), a.end()), a.end());
    for (int j : a) h.bcol.push_back(j);
    if (i < h.nsv_verts && a.empty()) h.bcol.push_back(i);
    h.bptr.push_back((int)h.bcol.size());
  }
  const int nnzb = (int)h.bcol.size();
  auto find_blk = [&](int r, int c) {
    auto b = h.bcol.begin() + h.bptr[r], e = h.bcol.begin() + h.bptr[r + 1];
    return (int)(std::lower_bound(b, e, c) - h.bcol.begin());
  };
  // counting sort of the contributions by block, tet order kept within a block
  std::vector<int> blk(16 * (size_t)nt);
  h.blkptr.assign(nnzb + 1, 0);
  h.ntptr.assign(nn + 1, 0);
  for (int t = 0; t < nt; ++t)
    for (int a = 0; a < 4; ++a) {
      h.ntptr[h.tet_nodes[4 * t + a] + 1]++;
      for (int b = 0; b < 4; ++b) {
        int k = find_blk(h.tet_nodes[4 * t + a], h.tet_nodes[4 * t + b]);
        blk[16 * t + 4 * a + b] = k;
        h.blkptr[k + 1]++;
      }
    }
  for (int k = 0; k < nnzb; ++k) h.blkptr[k + 1] += h.blkptr[k];
  for (int i = 0; i < nn; ++i) h.ntptr[i + 1] += h.ntptr[i];
  h.blksrc.assign(16 * (size_t)nt, 0);
  std::vector<int> fill(h.blkptr.begin(), h.blkptr.end() - 1);
  for (int src = 0; src < 16 * nt; ++src) h.blksrc[fill[blk[src]]++] = src;
  h.ntsrc.assign(4 * (size_t)nt, 0);
  std::vector<int> fillp(h.ntptr.begin(), h.ntptr.end() - 1);
  for (int t = 0; t < nt; ++t)
    for (int a = 0; a < 4; ++a) h.ntsrc[fillp[h.tet_nodes[4 * t + a]]++] = 4 * t + a;
  h.have_pattern = true;
}

// partner slots per query of a collect traversal: edge-edge queries on fine surfaces find a few
// dozen non-adjacent neighbours within the step filter's grown boxes
constexpr int CAND_SLOTS = 128;

uint64_t estimate_bytes(const HostEnv& h, int precision) {
  uint64_t nn = h.nsv_verts + 4 * h.nbodies;
  uint64_t hb = precision == IPC_MIXED ? 4 : 8;
  uint64_t b = nn * (24 * 14 + 72) + (uint64_t)h.ntets * (96 + 16 + 96 + 90 * 8 + 64) + nn * 15 * (9 * hb + 8);
  uint64_t np = h.pt_node.size(), nprim = h.tris.size() / 3 + h.edges.size() / 2 + h.sv.size();
  // contact capacity estimate: collect slots, kept list boxes (6 doubles per primitive)
  b += np * 96 + nprim * (4 * CAND_SLOTS + 48) + 4096 * (78 * 8 + 200);
  b += (uint64_t)h.targets.size() * 8;
  return b;
}

void build_env(HostEnv& h, const ipc_env_desc* D) {
  if (!D || D->n_steps <= 0 || (D->n_soft + D->n_affine) <= 0) fail_with(IPC_ERR_ARG, "env: empty or no steps");
  if (!D->gravity_on || !D->targets) fail_with(IPC_ERR_ARG, "env: gravity_on and targets are required");
  h.mu = D->friction_mu;
  h.n_steps = D->n_steps;
  h.grav.assign(D->gravity_on, D->gravity_on + D->n_steps);
  for (uint8_t gcode : h.grav)
    if (gcode > 7) fail_with(IPC_ERR_ARG, "env: gravity codes are 0..7");
  int nh = D->n_soft + D->n_affine;
  h.targets.assign(D->targets, D->targets + (size_t)D->n_steps * nh * 12);
  int nsv = 0;
  for (int b = 0; b < D->n_soft; ++b) {
    const ipc_soft_body_desc& S = D->soft[b];
    if (S.n_verts <= 0 || S.n_tets <= 0 || !S.verts || !S.tets) fail_with(IPC_ERR_ARG, "soft body: empty");
    HostEnv::Soft s;
    s.verts.assign(S.verts, S.verts + 3 * S.n_verts);
    s.tets.assign(S.tets, S.tets + 4 * S.n_tets);
    if (S.n_tris > 0) s.tris.assign(S.tris, S.tris + 3 * S.n_tris);
    s.kin.assign(S.n_verts, 0);
    if (S.kinematic) s.kin.assign(S.kinematic, S.kinematic + S.n_verts);
    s.E = S.youngs;
    s.nu = S.poisson;
    s.rho = S.density;
    for (int i : s.tets)
      if (i < 0 || i >= S.n_verts) fail_with(IPC_ERR_ARG, "soft body: tet index out of range");
    for (int i : s.tris)
      if (i < 0 || i >= S.n_verts) fail_with(IPC_ERR_ARG, "soft body: triangle index out of range");
    nsv += S.n_verts;
    h.soft.push_back(std::move(s));
  }
  for (int b = 0; b < D->n_affine; ++b) {
    const ipc_affine_body_desc& A = D->affine[b];
    if (A.n_verts <= 0 || A.n_tris <= 0) fail_with(IPC_ERR_ARG, "affine body: empty surface");
    HostEnv::Aff a;
    a.verts.assign(A.verts, A.verts + 3 * A.n_verts);
    a.tris.assign(A.tris, A.tris + 3 * A.n_tris);
    for (int i : a.tris)
      if (i < 0 || i >= A.n_verts) fail_with(IPC_ERR_ARG, "affine body: triangle index out of range");
    a.rho = A.density;
    std::memcpy(a.q0, A.q0, sizeof(a.q0));
    std::memcpy(a.qdot0, A.qdot0, sizeof(a.qdot0));
    a.kin = A.kinematic;
    a.kpd = A.kinematic ? 0.0 : A.pd_stiffness;
    h.aff.push_back(std::move(a));
  }
  h.nsv_verts = nsv;
  h.nbodies = D->n_affine;
  h.ndof = 3 * nsv + 12 * D->n_affine;
  h.x.assign(h.ndof, 0.0);
  h.v.assign(h.ndof, 0.0);
  h.mass.assign(nsv, 0.0);
  h.node_kin.assign(nsv, 0);
  h.X0.assign(3 * nsv, 0.0);
  h.node_handle.assign(nsv + 4 * D->n_affine, 0);
  // soft: rest shape matrices, volumes, Lame parameters, lumped masses
  int off = 0;
  for (size_t b = 0; b < h.soft.size(); ++b) {
    auto& s = h.soft[b];
    double mu = s.E / (2.0 * (1.0 + s.nu)), lam = s.E * s.nu / ((1.0 + s.nu) * (1.0 - 2.0 * s.nu));
    int nv = (int)s.verts.size() / 3;
    for (int i = 0; i < nv; ++i) {
      for (int k = 0; k < 3; ++k) {
        h.x[3 * (off + i) + k] = s.verts[3 * i + k];
        h.X0[3 * (off + i) + k] = s.verts[3 * i + k];
      }
      h.node_kin[off + i] = s.kin[i] ? 1 : 0;
      h.node_handle[off + i] = (int)b;
    }
    int nt = (int)s.tets.size() / 4;
    for (int t = 0; t < nt; ++t) {
      const double* X[4];
      for (int k = 0; k < 4; ++k) X[k] = &s.verts[3 * s.tets[4 * t + k]];
      double Dm[9];
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) Dm[3 * r + c] = X[c + 1][r] - X[0][r];
      double det = Dm[0] * (Dm[4] * Dm[8] - Dm[5] * Dm[7]) - Dm[1] * (Dm[3] * Dm[8] - Dm[5] * Dm[6]) +
                   Dm[2] * (Dm[3] * Dm[7] - Dm[4] * Dm[6]);
      if (!(det > 0.0)) fail_with(IPC_ERR_INIT_INVERTED, "a tet has non-positive rest volume");
      double inv[9] = {(Dm[4] * Dm[8] - Dm[5] * Dm[7]) / det, (Dm[2] * Dm[7] - Dm[1] * Dm[8]) / det,
                       (Dm[1] * Dm[5] - Dm[2] * Dm[4]) / det, (Dm[5] * Dm[6] - Dm[3] * Dm[8]) / det,
                       (Dm[0] * Dm[8] - Dm[2] * Dm[6]) / det, (Dm[2] * Dm[3] - Dm[0] * Dm[5]) / det,
                       (Dm[3] * Dm[7] - Dm[4] * Dm[6]) / det, (Dm[1] * Dm[6] - Dm[0] * Dm[7]) / det,
                       (Dm[0] * Dm[4] - Dm[1] * Dm[3]) / det};
      double vol = det / 6.0;
      for (int k = 0; k < 4; ++k) h.tet_nodes.push_back(off + s.tets[4 * t + k]);
      for (int k = 0; k < 9; ++k) h.tet_prm.push_back(inv[k]);
      h.tet_prm.push_back(vol);
      h.tet_prm.push_back(mu);
      h.tet_prm.push_back(lam);
      for (int k = 0; k < 4; ++k) h.mass[off + s.tets[4 * t + k]] += s.rho * vol / 4.0;
    }
    off += nv;
  }
  h.ntets = (int)h.tet_nodes.size() / 4;
  // affine bodies: mass matrix from the closed surface (divergence theorem), rest bbox
  for (size_t b = 0; b < h.aff.size(); ++b) {
    auto& a = h.aff[b];
    double I0 = 0, I1[3] = {0, 0, 0}, I2[9] = {0};
    int nt = (int)a.tris.size() / 3;
    for (int f = 0; f < nt; ++f) {
      const double* A = &a.verts[3 * a.tris[3 * f]];
      const double* B = &a.verts[3 * a.tris[3 * f + 1]];
      const double* Cc = &a.verts[3 * a.tris[3 * f + 2]];
      double det = A[0] * (B[1] * Cc[2] - B[2] * Cc[1]) - A[1] * (B[0] * Cc[2] - B[2] * Cc[0]) +
                   A[2] * (B[0] * Cc[1] - B[1] * Cc[0]);
      double s[3] = {A[0] + B[0] + Cc[0], A[1] + B[1] + Cc[1], A[2] + B[2] + Cc[2]};
      I0 += det / 6.0;
      for (int i = 0; i < 3; ++i) I1[i] += det * s[i] / 24.0;
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) I2[3 * i + j] += det * (A[i] * A[j] + B[i] * B[j] + Cc[i] * Cc[j] + s[i] * s[j]) / 120.0;
    }
    double M[16];
    M[0] = a.rho * I0;
    for (int i = 0; i < 3; ++i) M[1 + i] = M[4 * (1 + i)] = a.rho * I1[i];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) M[4 * (1 + i) + 1 + j] = a.rho * I2[3 * i + j];
    if (!a.kin && !(I0 > 0.0)) fail_with(IPC_ERR_ARG, "affine body: surface encloses no volume (not closed / inward)");
    for (int i = 0; i < 16; ++i) h.M4.push_back(M[i]);
    h.bvol.push_back(I0);
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (size_t i = 0; i < a.verts.size() / 3; ++i)
      for (int k = 0; k < 3; ++k) {
        lo[k] = std::min(lo[k], a.verts[3 * i + k]);
        hi[k] = std::max(hi[k], a.verts[3 * i + k]);
      }
    for (int k = 0; k < 3; ++k) h.bbox.push_back(lo[k]);
    for (int k = 0; k < 3; ++k) h.bbox.push_back(hi[k]);
    int dof = 3 * nsv + 12 * (int)b;
    for (int k = 0; k < 12; ++k) {
      h.x[dof + k] = a.q0[k];
      h.v[dof + k] = a.qdot0[k];
    }
    for (int k = 0; k < 4; ++k) h.node_handle[nsv + 4 * b + k] = (int)h.soft.size() + (int)b;
  }
  // points, triangles, surface vertices, edges
  std::vector<int> soft_off, aff_off;
  off = 0;
  for (size_t b = 0; b < h.soft.size(); ++b) {
    soft_off.push_back((int)h.pt_node.size());
    int nv = (int)h.soft[b].verts.size() / 3;
    for (int i = 0; i < nv; ++i) {
      h.pt_node.push_back(off + i);
      for (int k = 0; k < 3; ++k) {
        h.pt_xb.push_back(0.0);
        h.pt_rest.push_back(h.soft[b].verts[3 * i + k]);
      }
      h.pt_body.push_back(-1 - (int)b);
      h.pt_kin.push_back(h.soft[b].kin[i] ? 1 : 0);
    }
    off += nv;
  }
  for (size_t b = 0; b < h.aff.size(); ++b) {
    aff_off.push_back((int)h.pt_node.size());
    int nv = (int)h.aff[b].verts.size() / 3;
    for (int i = 0; i < nv; ++i) {
      h.pt_node.push_back(-1 - (int)b);
      for (int k = 0; k < 3; ++k) {
        h.pt_xb.push_back(h.aff[b].verts[3 * i + k]);
        h.pt_rest.push_back(h.aff[b].verts[3 * i + k]);
      }
      h.pt_body.push_back((int)b);
      h.pt_kin.push_back(h.aff[b].kin ? 1 : 0);
    }
  }
  for (size_t b = 0; b < h.soft.size(); ++b)
    for (int v : h.soft[b].tris) h.tris.push_back(soft_off[b] + v);
  for (size_t b = 0; b < h.aff.size(); ++b)
    for (int v : h.aff[b].tris) h.tris.push_back(aff_off[b] + v);
  std::vector<int> sv(h.tris);
  std::sort(sv.begin(), sv.end());
  sv.erase(std::unique(sv.begin(), sv.end()), sv.end());
  h.sv = sv;
  std::vector<std::pair<int, int>> ed;
  for (size_t f = 0; f < h.tris.size() / 3; ++f)
    for (int k = 0; k < 3; ++k) {
      int a = h.tris[3 * f + k], b = h.tris[3 * f + (k + 1) % 3];
      ed.push_back({std::min(a, b), std::max(a, b)});
    }
  std::sort(ed.begin(), ed.end());
  ed.erase(std::unique(ed.begin(), ed.end()), ed.end());
  for (auto& e : ed) {
    h.edges.push_back(e.first);
    h.edges.push_back(e.second);
    double s = 0;
    for (int k = 0; k < 3; ++k) {
      double d = h.pt_rest[3 * e.first + k] - h.pt_rest[3 * e.second + k];
      s += d * d;
    }
    h.edge_rest2.push_back(s);
  }
  // joint anchors: points on their bodies that belong to no surface (no contact)
  h.n_surf_pts = (int)h.pt_node.size();
  if (D->n_joints < 0 || (D->n_joints > 0 && !D->joints)) fail_with(IPC_ERR_ARG, "env: bad joint list");
  for (int j = 0; j < D->n_joints; ++j) {
    const ipc_joint_desc& J = D->joints[j];
    if (J.body_a < 0 || J.body_a >= D->n_affine || J.body_b < 0 || J.body_b >= D->n_affine || J.body_a == J.body_b)
      fail_with(IPC_ERR_ARG, "joint: bodies must be two distinct affine bodies of the env");
    if (!(J.stiffness > 0.0) || !std::isfinite(J.stiffness)) fail_with(IPC_ERR_ARG, "joint: stiffness must be > 0");
    HostEnv::Joint hj;
    const int bodies[2] = {J.body_a, J.body_b};
    const double* anchors[2] = {J.anchor_a, J.anchor_b};
    for (int side = 0; side < 2; ++side) {
      const int b = bodies[side];
      (side == 0 ? hj.pa : hj.pb) = (int)h.pt_node.size();
      h.pt_node.push_back(-1 - b);
      for (int k = 0; k < 3; ++k) {
        if (!std::isfinite(anchors[side][k])) fail_with(IPC_ERR_ARG, "joint: anchor not finite");
        h.pt_xb.push_back(anchors[side][k]);
        h.pt_rest.push_back(anchors[side][k]);
      }
      h.pt_body.push_back(b);
      h.pt_kin.push_back(h.aff[b].kin ? 1 : 0);
    }
    hj.k = J.stiffness;
    h.joints.push_back(hj);
  }
  if (D->grasped_object < 0 || D->grasped_object > D->n_soft + D->n_affine)
    fail_with(IPC_ERR_ARG, "env: grasped_object out of range");
  h.obj = D->grasped_object - 1;
  if (h.obj >= 0) {
    if (h.obj < D->n_soft) {
      int first = 0;
      for (int b = 0; b < h.obj; ++b) first += D->soft[b].n_verts;
      h.obj_first = first;
      h.obj_count = D->soft[h.obj].n_verts;
      for (int i = 0; i < h.obj_count; ++i)
        for (int k = 0; k < 3; ++k) h.obj_com0[k] += h.x[3 * (first + i) + k] / h.obj_count;
    } else {
      const int a = h.obj - D->n_soft;
      h.obj_affine = 1;
      h.obj_first = a;
      const auto& av = h.aff[a].verts;
      const int nv = (int)av.size() / 3;
      for (int i = 0; i < nv; ++i)
        for (int k = 0; k < 3; ++k) h.obj_xbar[k] += av[3 * i + k] / nv;
      const double* q = h.aff[a].q0;
      for (int k = 0; k < 3; ++k)
        h.obj_com0[k] = q[k] + h.obj_xbar[0] * q[3 + k] + h.obj_xbar[1] * q[6 + k] + h.obj_xbar[2] * q[9 + k];
    }
  }
}

}  // namespace

// per-env PCG iteration counts into the statistics
__global__ void k_add_stats(int n_env, const long long* __restrict__ it, long long* __restrict__ stats) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n_env) stats[5 * e + STAT_PCG] += it[e];
}

// ==================================================================== the scene
struct ipc_scene {
  ipc_scene_desc desc;
  cudaStream_t stream = nullptr;
  // side stream for the latency-bound contact and body Hessians, which overlap the element
  // Hessians of the same evaluation (fork and join through the two events)
  cudaStream_t side = nullptr;
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
  bool own_stream = false;
  int device = 0;
  std::map<int, HostEnv> envs;
  int next_id = 0;
  bool dirty = true;
  uint64_t used_bytes = 0;
  long long launches = 0;

  // ---------------- layout sizes
  int E = 0, NN = 0, NB = 0, NT = 0, NP = 0, NSV = 0, NED = 0, NTR = 0, NTILE = 0, NNZB = 0;
  int max_env_slices = 0, max_env_bodies = 0, n_slices = 0;
  int pcg_C = 0;  // CTAs per env cluster of the last solve's first persistent-PCG launch (0: tiled PCG)
  int pcg_resident[5] = {0, 0, 0, 0, 0};  // clusters of 1, 2, 4, 8, 16 CTAs resident at once
  long sell_nval = 0;
  std::vector<int> ids;  // layout index -> env id
  std::vector<int> h_node_off, h_tet_off, h_pt_off, h_sv_off, h_ed_off, h_tri_off, h_body_off, h_tile_off;
  // ---------------- device arrays (static per layout)
  DBuf<int> node_off, tet_off, body_off, nsteps, grav_off, nh, tile_env, tile_kind, tile_begin, tile_end, tile_off;
  DBuf<long> sched_off;
  DBuf<double> env_mu, sched;
  DBuf<uint8_t> grav;
  DBuf<int> node_env, node_body, node_handle, body_node, body_env;
  DBuf<uint8_t> node_kin, body_kin;
  DBuf<double> node_mass, X0, M4, bvol, bbox, body_pd;
  DBuf<int4> tets;
  DBuf<double> tet_prm;
  DBuf<int> tet_env;
  DBuf<int> pt_node, pt_body, pt_env;
  DBuf<double> pt_xb;
  DBuf<uint8_t> pt_kin;
  DBuf<int> sv_pt, sv_env, ed_pt, ed_env, tri_pt, tri_env;
  DBuf<double> ed_rest2;
  DBuf<int> bsr_ptr, bsr_col, blk_row, blk_ptr, blk_src, nt_ptr, nt_src;
  DBuf<int> tile_slice, slice_w, sell_col, pslice_off, pslice_row, pslice_sel;
  DBuf<long> slice_vbase, slice_cbase, blk_pos, diag_pos;
  // ---------------- state
  DBuf<double> x, v, xt, xtilde, xtarget, xtrial, p, pbar, grad;
  DBuf<double> ptx, ptx_t, ptp, pte;
  // env control
  DBuf<int> e_status, e_reason, e_step, e_constrained, e_bad, e_nanp, e_halv, e_newton_it, e_count, e_rem;
  // barrier stiffness per env, its closest-contact tracking and the step-start sums
  DBuf<double> e_kappa, e_kdots, g0buf;
  DBuf<double> e_trace;  // per env: the incremental potential at each Newton iterate of its step
  DBuf<int> e_trace_n;
  int trace_cap() const { return std::max(desc.max_newton, 1); }
  DBuf<double> tet_vm;  // per-tet stress or per-contact force of a query
  DBuf<uint8_t> e_stepping, e_iter, e_ls, e_accept, e_sel, e_all, e_start, e_cover;
  DBuf<double> e_E0, e_Et, e_alpha;
  DBuf<unsigned long long> e_alpha_bits, e_pnorm_bits, e_inter, e_inv;
  DBuf<long long> e_stats;
  // energies / stencils
  DBuf<double> nodeE, tetE, tet_g, tet_H, bodyE, body_g, body_H;
  DBuf<double> bsr_val, Ps, Pb;
  // mixed precision: FP32 Hessians, sliced-ELL values, preconditioner blocks, stencil Hessians,
  // entry weights and every vector of the PCG (the FP64 twins above hold them otherwise)
  DBuf<float> f_tet_H, f_body_H, f_bsr_val, f_Ps, f_Pb, f_sH, f_ns_w, f_ns_xb, f_st_t, f_st_xb;
  DBuf<float> f_r, f_z, f_d, f_y, f_x;
  bool mixed() const { return desc.precision == IPC_MIXED; }
  template <class T>
  static T* hp(DBuf<double>& d, DBuf<float>& f) {
    if constexpr (std::is_same<T, double>::value) return d.p;
    else return f.p;
  }
  DBuf<double> pcg_r, pcg_z, pcg_d, pcg_y, pcg_x, part_a, part_b, part_c, pcg_rz, pcg_bb;
  DBuf<int> pcg_it, pcg_active;
  DBuf<double> pcg_rzs, pcg_bbs, pcg_iterb, pcg_iterf;  // per-env state of the persistent PCG
  DBuf<unsigned long long> pcg_tune_iters;                 // env-iterations of a timed launch
  cudaEvent_t tune_ev[2] = {nullptr, nullptr};
  DBuf<int> pcg_its, env_iota, env_list;
  DBuf<uint8_t> pcg_runs;
  DBuf<uint8_t> pcg_run;
  // trees
  struct TreeBufs {
    DBuf<double> pbox;
    DBuf<float4> nbox;  // outward-rounded FP32 node boxes, 2 float4 per node
    DBuf<unsigned long long> keys, keys2;
    DBuf<unsigned> vals, vals2;
    DBuf<int> child, parent, range, root, flags, hist;
    DBuf<unsigned long long> emin, emax;
    int n = 0;
    bool built = false;
  } ttri, tedge;
  // candidates / contacts
  DBuf<int> cnt_pt, off_pt, cnt_ee, off_ee, cand_j, cand_q, nflag, noff, scan_tmp, overflow;
  DBuf<int> ccd_cnt_pt, ccd_off_pt, ccd_cnt_ee, ccd_off_ee, ccd_j, ccd_q;  // swept-box candidates
  DBuf<int> slots_pt, slots_ee;  // partner slots of collect traversals (cand_cap() per query)
  DBuf<ContactRec> ct_tmp, ct, cand_rec, ccd_rec;  // contacts; pair records of the two lists
  DBuf<FrictionRec> fr, fr_new, fr_tmp;
  DBuf<unsigned long long> fr_keys, fr_keys2;
  DBuf<unsigned> fr_vals, fr_vals2;
  DBuf<int> fr_hist;
  int n_pt = 0, n_ee = 0, n_ct = 0, n_ct_pt = 0, n_fr = 0, n_fr_pt = 0, n_inc = 0;
  DBuf<JointRec> jt;  // point joints of the batch, env-sorted (static per layout)
  int n_jt = 0;
  int n_st() const { return n_ct + n_fr + n_jt; }  // stencils: contacts, friction, joints
  DBuf<int> st_pts, st_env, st_cnt, st_off, ns_ptr, ns_src, ns_cnt;
  DBuf<unsigned long long> st_keys, st_keys2;
  DBuf<unsigned> st_vals, st_vals2;
  DBuf<double> sE, sg, sH, st_t, ns_w, ns_xb, st_xb;
  DBuf<double> ct_Hl;  // unprojected 12x12 barrier Hessians of one evaluation (144 per contact)
  DBuf<int> st_node;  // per stencil point: its node, or -1 - the p node of its affine body
  DBuf<long long> pcg_iters;
  DBuf<int> st_hist, root_off_tri, root_off_ed;
  // profiling: event pairs per family, device work counters
  bool prof_on = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_ev[IPC_PROF_COUNT];
  std::vector<cudaEvent_t> ev_pool;
  long long prof_launches[IPC_PROF_COUNT] = {0};
  DBuf<unsigned long long> prof_units;
  cudaEvent_t take_event() {
    if (ev_pool.empty()) {
      cudaEvent_t e;
      CK(cudaEventCreate(&e));
      return e;
    }
    cudaEvent_t e = ev_pool.back();
    ev_pool.pop_back();
    return e;
  }
  int prof_cur = -1;
  cudaEvent_t prof_start{};
  // events recorded inside a captured graph (external record nodes), resolved after each replay
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> graph_ev;
  double prof_graph_ms[IPC_PROF_COUNT] = {0};
  void pbeg(int fam) {
    if (!prof_on) return;
    prof_cur = fam;
    prof_start = take_event();
    if (capturing) CK(cudaEventRecordWithFlags(prof_start, stream, cudaEventRecordExternal));
    else CK(cudaEventRecord(prof_start, stream));
  }
  void pend(int fam) {
    if (!prof_on || prof_cur != fam) return;
    cudaEvent_t e = take_event();
    if (capturing) {
      CK(cudaEventRecordWithFlags(e, stream, cudaEventRecordExternal));
      graph_ev.push_back({fam, {prof_start, e}});
    } else {
      CK(cudaEventRecord(e, stream));
      prof_ev[fam].push_back({prof_start, e});
      prof_launches[fam]++;
    }
    prof_cur = -1;
  }
  // after a graph replay has completed: add its kernel times
  void graph_prof_collect() {
    for (auto& g : graph_ev) {
      float m = 0.f;
      CK(cudaEventElapsedTime(&m, g.second.first, g.second.second));
      prof_graph_ms[g.first] += m;
      prof_launches[g.first]++;
    }
  }
  void graph_prof_release() {
    for (auto& g : graph_ev) {
      ev_pool.push_back(g.second.first);
      ev_pool.push_back(g.second.second);
    }
    graph_ev.clear();
  }
  unsigned long long* punits(int fam) { return prof_on ? prof_units.p + fam : nullptr; }
  // algorithmic bytes of a family's launches that the host can count from the sizes it launches
  // with (the launch's whole extent: records, gathered points and outputs, each once)
  double prof_host_work[IPC_PROF_COUNT] = {0};
  void pwork(int fam, double bytes) {
    if (prof_on && !capturing) prof_host_work[fam] += bytes;
  }
  // one pair of collect traversals (point-triangle, edge-edge) that listed np + ne candidates:
  // query records (surface vertex ids and point, edge ids and box), the leaf boxes and the FP32
  // node boxes with child links of both trees, the per-query counts and the listed partners
  double traversal_bytes(int np, int ne) const {
    return (double)NSV * (4 + 4 + 24) + (double)NED * (8 + 4 + 48) + (double)(NTR + NED) * 48 +
           2.0 * (NTR + NED) * 40 + (double)(NSV + NED) * 4 + (double)(np + ne) * 4;
  }
  // pinned host scratch
  int* hpin = nullptr;

  ~ipc_scene() {
    for (auto& v : prof_ev)
      for (auto& pr : v) {
        cudaEventDestroy(pr.first);
        cudaEventDestroy(pr.second);
      }
    for (auto e : ev_pool) cudaEventDestroy(e);
    for (auto e : tune_ev)
      if (e) cudaEventDestroy(e);
    if (hpin) cudaFreeHost(hpin);
    if (fork_ev) cudaEventDestroy(fork_ev);
    if (join_ev) cudaEventDestroy(join_ev);
    if (side) cudaStreamDestroy(side);
    if (own_stream && stream) cudaStreamDestroy(stream);
  }

  // ------------------------------------------------------------------ launch helpers
  bool capturing = false;
  long long captured_kernels = 0;
  template <class K, class... Args>
  void launch(K kern, long n_threads, int block, Args... args) {
    if (n_threads <= 0) return;
    mark_resume();
    long grid = (n_threads + block - 1) / block;
    kern<<<(unsigned)grid, block, 0, stream>>>(args...);
    if (capturing) ++captured_kernels;
    else ++launches;
    CK(cudaGetLastError());
  }
  template <class K, class... Args>
  void launch_grid(K kern, long grid, int block, Args... args) {
    if (grid <= 0) return;
    mark_resume();
    kern<<<(unsigned)grid, block, 0, stream>>>(args...);
    if (capturing) ++captured_kernels;
    else ++launches;
    CK(cudaGetLastError());
  }
  // A host round trip inside the stepping loop (a count or flag the host needs before its next
  // launch). With profiling on, an event recorded behind the work before the wait and one recorded
  // at the next kernel launch bound the time the GPU sat idle because of it (family
  // IPC_PROF_HOST_IDLE).
  cudaEvent_t idle_from = nullptr;
  void host_sync() {
    if (prof_on && !capturing) {
      if (idle_from) ev_pool.push_back(idle_from);
      idle_from = take_event();
      CK(cudaEventRecord(idle_from, stream));
    }
    CK(cudaStreamSynchronize(stream));
  }
  void mark_resume() {
    if (!idle_from) return;
    cudaEvent_t e = take_event();
    CK(cudaEventRecord(e, stream));
    prof_ev[IPC_PROF_HOST_IDLE].push_back({idle_from, e});
    prof_launches[IPC_PROF_HOST_IDLE]++;
    idle_from = nullptr;
  }
  void read_ints(const int* dptr, int* out, int n) {
    CK(cudaMemcpyAsync(hpin, dptr, n * sizeof(int), cudaMemcpyDeviceToHost, stream));
    host_sync();
    for (int i = 0; i < n; ++i) out[i] = hpin[i];
  }
  int read_int(const int* dptr) {
    CK(cudaMemcpyAsync(hpin, dptr, sizeof(int), cudaMemcpyDeviceToHost, stream));
    host_sync();
    return *hpin;
  }
  int count_flags(const uint8_t* f) {
    launch_grid(k_count_flags, 1, 256, E, f, e_count.p);
    return read_int(e_count.p);
  }
  // exclusive scan of n ints into out[0..n] (out[n] = total); returns total (sync)
  int scan(const int* in, int n, int* out, bool read_total = true) {
    if (n <= 0) {
      CK(cudaMemsetAsync(out, 0, sizeof(int), stream));
      return 0;
    }
    int nb = (n + SCAN_BLOCK - 1) / SCAN_BLOCK;
    scan_tmp.ensure(nb + 1);
    launch_grid(k_scan_block_sums, nb, SCAN_BLOCK, in, n, scan_tmp.p);
    launch_grid(k_scan_sums, 1, SCAN_BLOCK, scan_tmp.p, nb);
    launch_grid(k_scan_apply, nb, SCAN_BLOCK, in, n, (const int*)scan_tmp.p, out);
    return read_total ? read_int(out + n) : 0;
  }
  // stable sort of (key, value) pairs over key bits [0, bits)
  void radix_sort(DBuf<unsigned long long>& k, DBuf<unsigned>& v, DBuf<unsigned long long>& k2, DBuf<unsigned>& v2,
                  DBuf<int>& hist, int n, int bits) {
    if (n <= 1) return;
    int nblk = (n + RS_TILE - 1) / RS_TILE;
    hist.ensure(256 * nblk + 1);
    k2.ensure(n);
    v2.ensure(n);
    for (int shift = 0; shift < bits; shift += 8) {
      launch_grid(k_rs_hist, nblk, RS_THREADS, (const unsigned long long*)k.p, n, shift, nblk, hist.p);
      scan(hist.p, 256 * nblk, hist.p, false);  // in place is safe: apply reads 'in' block-locally first
      launch_grid(k_rs_scatter, nblk, RS_THREADS, (const unsigned long long*)k.p, (const unsigned*)v.p, k2.p, v2.p, n,
                  shift, nblk, (const int*)hist.p);
      std::swap(k.p, k2.p);
      std::swap(k.n, k2.n);
      std::swap(v.p, v2.p);
      std::swap(v.n, v2.n);
    }
  }

  Layout layout() const {
    return Layout{node_env.p, node_body.p, node_kin.p, node_mass.p, body_node.p, body_kin.p, pt_node.p, pt_xb.p};
  }
  Tiles tiles() const { return Tiles{tile_env.p, tile_kind.p, tile_begin.p, tile_end.p, tile_off.p}; }
  EnvCtl ctl() {
    return EnvCtl{e_status.p, e_reason.p, e_step.p, nsteps.p, e_stepping.p, e_iter.p, e_ls.p, e_accept.p,
                  e_constrained.p, e_bad.p, e_nanp.p, e_halv.p, e_newton_it.p, e_E0.p, e_Et.p, e_alpha.p,
                  e_alpha_bits.p, e_pnorm_bits.p, e_stats.p, e_count.p, e_rem.p};
  }
  Sched sched_view() const {
    return Sched{sched.p, grav.p, sched_off.p, grav_off.p, nh.p, node_handle.p, X0.p};
  }
  PtInfo ptinfo() const { return PtInfo{pt_body.p, pt_kin.p}; }
  Tree tree(TreeBufs& T) const { return Tree{T.n, T.vals.p, T.child.p, T.nbox.p, T.pbox.p, T.root.p}; }

  // ------------------------------------------------------------------ layout
  void pull_state() {
    // copy the device state of the current layout back into the env records
    if (ids.empty()) return;
    std::vector<double> hx(3 * (size_t)NN), hv(3 * (size_t)NN);
    std::vector<int> st(E), rs(E), sp(E);
    std::vector<long long> stats(5 * (size_t)E);
    CK(cudaMemcpyAsync(hx.data(), x.p, hx.size() * 8, cudaMemcpyDeviceToHost, stream));
    CK(cudaMemcpyAsync(hv.data(), v.p, hv.size() * 8, cudaMemcpyDeviceToHost, stream));
    CK(cudaMemcpyAsync(st.data(), e_status.p, E * 4, cudaMemcpyDeviceToHost, stream));
    CK(cudaMemcpyAsync(rs.data(), e_reason.p, E * 4, cudaMemcpyDeviceToHost, stream));
    CK(cudaMemcpyAsync(sp.data(), e_step.p, E * 4, cudaMemcpyDeviceToHost, stream));
    CK(cudaMemcpyAsync(stats.data(), e_stats.p, E * 40, cudaMemcpyDeviceToHost, stream));
    CK(cudaStreamSynchronize(stream));
    for (int li = 0; li < E; ++li) {
      auto it = envs.find(ids[li]);
      if (it == envs.end()) continue;
      HostEnv& h = it->second;
      size_t o = 3 * (size_t)h_node_off[li];
      std::copy(hx.begin() + o, hx.begin() + o + h.ndof, h.x.begin());
      std::copy(hv.begin() + o, hv.begin() + o + h.ndof, h.v.begin());
      h.status = st[li];
      h.reason = rs[li];
      h.step = sp[li];
      for (int k = 0; k < 5; ++k) h.stats[k] = stats[5 * li + k];
    }
  }

  void commit() {
    if (!dirty) return;
    if (envs.empty()) fail_with(IPC_ERR_NO_ENV, "scene holds no environment");
    CK(cudaSetDevice(device));
    pull_state();
    ids.clear();
    for (auto& kv : envs) ids.push_back(kv.first);
    E = (int)ids.size();
    std::vector<int> node_off_h{0}, tet_off_h{0}, pt_off_h{0}, sv_off_h{0}, ed_off_h{0}, tri_off_h{0}, body_off_h{0};
    std::vector<int> nsteps_h, grav_off_h, nh_h;
    std::vector<long> sched_off_h;
    std::vector<double> mu_h, sched_h;
    std::vector<uint8_t> grav_h;
    std::vector<int> node_env_h, node_body_h, node_handle_h, body_node_h, body_env_h;
    std::vector<uint8_t> node_kin_h, body_kin_h, pt_kin_h;
    std::vector<double> node_mass_h, X0_h, M4_h, bvol_h, bpd_h, bbox_h, tet_prm_h, pt_xb_h, ed_rest2_h, x_h, v_h;
    std::vector<int4> tets_h;
    std::vector<int> tet_env_h, pt_node_h, pt_body_h, pt_env_h, sv_pt_h, sv_env_h, ed_pt_h, ed_env_h, tri_pt_h, tri_env_h;
    std::vector<int> status_h, reason_h, step_h;
    std::vector<JointRec> jt_h;
    std::vector<long long> stats_h;
    int body_base = 0, soft_body_base = 0;
    for (int li = 0; li < E; ++li) {
      HostEnv& h = envs[ids[li]];
      int n0 = node_off_h.back(), p0 = pt_off_h.back(), t0 = tet_off_h.back(), b0 = body_off_h.back();
      int nsv = h.nsv_verts;
      // nodes: soft vertices, then 4 per body
      for (int i = 0; i < nsv; ++i) {
        node_env_h.push_back(li);
        node_body_h.push_back(-1);
        node_kin_h.push_back(h.node_kin[i]);
        node_mass_h.push_back(h.mass[i]);
        node_handle_h.push_back(h.node_handle[i]);
        for (int k = 0; k < 3; ++k) X0_h.push_back(h.X0[3 * i + k]);
      }
      for (int b = 0; b < h.nbodies; ++b) {
        body_node_h.push_back(n0 + nsv + 4 * b);
        body_env_h.push_back(li);
        body_kin_h.push_back(h.aff[b].kin ? 1 : 0);
        for (int k = 0; k < 16; ++k) M4_h.push_back(h.M4[16 * b + k]);
        bvol_h.push_back(h.bvol[b]);
        bpd_h.push_back(h.aff[b].kpd);
        for (int k = 0; k < 6; ++k) bbox_h.push_back(h.bbox[6 * b + k]);
        for (int k = 0; k < 4; ++k) {
          node_env_h.push_back(li);
          node_body_h.push_back(b0 + b);
          node_kin_h.push_back(0);
          node_mass_h.push_back(0.0);
          node_handle_h.push_back(h.node_handle[nsv + 4 * b + k]);
          for (int q = 0; q < 3; ++q) X0_h.push_back(0.0);
        }
      }
      for (double d : h.x) x_h.push_back(d);
      for (double d : h.v) v_h.push_back(d);
      for (int t = 0; t < h.ntets; ++t) {
        tets_h.push_back(make_int4(n0 + h.tet_nodes[4 * t], n0 + h.tet_nodes[4 * t + 1], n0 + h.tet_nodes[4 * t + 2],
                                   n0 + h.tet_nodes[4 * t + 3]));
        tet_env_h.push_back(li);
        for (int k = 0; k < 12; ++k) tet_prm_h.push_back(h.tet_prm[12 * t + k]);
      }
      for (size_t i = 0; i < h.pt_node.size(); ++i) {
        int nd = h.pt_node[i];
        pt_node_h.push_back(nd >= 0 ? n0 + nd : -1 - (b0 + (-1 - nd)));
        int pb = h.pt_body[i];
        pt_body_h.push_back(pb >= 0 ? b0 + pb : -1 - (soft_body_base + (-1 - pb)));
        pt_kin_h.push_back(h.pt_kin[i]);
        pt_env_h.push_back(li);
        for (int k = 0; k < 3; ++k) pt_xb_h.push_back(h.pt_xb[3 * i + k]);
      }
      for (int s : h.sv) {
        sv_pt_h.push_back(p0 + s);
        sv_env_h.push_back(li);
      }
      for (size_t e = 0; e < h.edges.size() / 2; ++e) {
        ed_pt_h.push_back(p0 + h.edges[2 * e]);
        ed_pt_h.push_back(p0 + h.edges[2 * e + 1]);
        ed_env_h.push_back(li);
        ed_rest2_h.push_back(h.edge_rest2[e]);
      }
      for (size_t f = 0; f < h.tris.size() / 3; ++f) {
        for (int k = 0; k < 3; ++k) tri_pt_h.push_back(p0 + h.tris[3 * f + k]);
        tri_env_h.push_back(li);
      }
      for (const HostEnv::Joint& j : h.joints) {
        JointRec r;
        r.pts[0] = p0 + j.pa;
        r.pts[1] = p0 + j.pb;
        r.env = li;
        r.pad = 0;
        r.k = j.k;
        jt_h.push_back(r);
      }
      nsteps_h.push_back(h.n_steps);
      grav_off_h.push_back((int)grav_h.size());
      grav_h.insert(grav_h.end(), h.grav.begin(), h.grav.end());
      nh_h.push_back((int)(h.soft.size() + h.aff.size()));
      sched_off_h.push_back((long)sched_h.size());
      sched_h.insert(sched_h.end(), h.targets.begin(), h.targets.end());
      mu_h.push_back(h.mu);
      status_h.push_back(h.status);
      reason_h.push_back(h.reason);
      step_h.push_back(h.step);
      for (int k = 0; k < 5; ++k) stats_h.push_back(h.stats[k]);
      node_off_h.push_back(n0 + nsv + 4 * h.nbodies);
      tet_off_h.push_back(t0 + h.ntets);
      pt_off_h.push_back(p0 + (int)h.pt_node.size());
      sv_off_h.push_back(sv_off_h.back() + (int)h.sv.size());
      ed_off_h.push_back(ed_off_h.back() + (int)h.edges.size() / 2);
      tri_off_h.push_back(tri_off_h.back() + (int)h.tris.size() / 3);
      body_off_h.push_back(b0 + h.nbodies);
      body_base += h.nbodies;
      soft_body_base += (int)h.soft.size();
    }
    NN = node_off_h.back();
    NT = tet_off_h.back();
    NP = pt_off_h.back();
    NSV = sv_off_h.back();
    NED = ed_off_h.back();
    NTR = tri_off_h.back();
    NB = body_off_h.back();
    h_node_off = node_off_h;
    h_tet_off = tet_off_h;
    h_pt_off = pt_off_h;
    h_sv_off = sv_off_h;
    h_ed_off = ed_off_h;
    h_tri_off = tri_off_h;
    h_body_off = body_off_h;
    // tiles: per env, soft-node tiles then body tiles
    std::vector<int> te, tk, tb, tn, toff{0};
    for (int li = 0; li < E; ++li) {
      int n0 = node_off_h[li];
      int nsv = envs[ids[li]].nsv_verts;
      for (int s = 0; s < nsv; s += TILE) {
        te.push_back(li);
        tk.push_back(0);
        tb.push_back(n0 + s);
        tn.push_back(n0 + std::min(nsv, s + TILE));
      }
      for (int s = body_off_h[li]; s < body_off_h[li + 1]; ++s) {  // one block per rigid body
        te.push_back(li);
        tk.push_back(1);
        tb.push_back(s);
        tn.push_back(s + 1);
      }
      toff.push_back((int)te.size());
    }
    NTILE = (int)te.size();
    h_tile_off = toff;
    // BSR pattern, block contributions and tet corners: each env's cached pattern, shifted
    std::vector<int> bptr{0}, bcol, brow, blkptr{0}, blksrc, ntcnt{0}, ntsrc;
    for (int li = 0; li < E; ++li) {
      HostEnv& h = envs[ids[li]];
      build_pattern(h);
      const int n0 = node_off_h[li], t0 = tet_off_h[li], nn = node_off_h[li + 1] - n0;
      const int b0 = (int)bcol.size(), c0 = blkptr.back(), q0 = ntcnt.back();
      for (int i = 0; i < nn; ++i) {
        for (int k = h.bptr[i]; k < h.bptr[i + 1]; ++k) {
          bcol.push_back(n0 + h.bcol[k]);
          brow.push_back(n0 + i);
        }
        bptr.push_back(b0 + h.bptr[i + 1]);
        ntcnt.push_back(q0 + h.ntptr[i + 1]);
      }
      for (size_t k = 1; k < h.blkptr.size(); ++k) blkptr.push_back(c0 + h.blkptr[k]);
      for (int src : h.blksrc) blksrc.push_back(16 * t0 + src);
      for (int src : h.ntsrc) ntsrc.push_back(4 * t0 + src);
    }
    NNZB = (int)bcol.size();
    // sliced ELL of the soft rows: 32-row slices inside each soft tile, padded to the slice's
    // longest row; block kk, element e of lane l at vbase + (kk*9 + e)*32 + l
    std::vector<int> tslice(te.size(), -1), sw, row_sel(NN, -1);
    std::vector<long> svb, scb, bpos(NNZB, -1), dpos(NN, -1);
    std::vector<int> scol;
    long vtot = 0, ctot = 0;
    for (size_t ti = 0; ti < te.size(); ++ti) {
      if (tk[ti] != 0) continue;
      tslice[ti] = (int)sw.size();
      for (int r0 = tb[ti]; r0 < tn[ti]; r0 += 32) {
        int r1 = std::min(tn[ti], r0 + 32);
        int w = 0;
        for (int r = r0; r < r1; ++r) w = std::max(w, bptr[r + 1] - bptr[r]);
        sw.push_back(w);
        svb.push_back(vtot);
        scb.push_back(ctot);
        scol.resize(ctot + 32L * w, -1);
        for (int r = r0; r < r1; ++r) {
          int lane = r - r0;
          row_sel[r] = 32 * ((int)sw.size() - 1) + lane;
          // padding blocks of a row point at the row itself with zero values, so the product
          // loop needs no branch (the values stay zero: assembly writes only real blocks)
          for (int kk = bptr[r + 1] - bptr[r]; kk < w; ++kk) scol[ctot + 32L * kk + lane] = r;
          for (int k = bptr[r]; k < bptr[r + 1]; ++k) {
            int kk = k - bptr[r];
            scol[ctot + 32L * kk + lane] = bcol[k];
            bpos[k] = vtot + 288L * kk + lane;
            if (bcol[k] == r) dpos[r] = bpos[k];
          }
        }
        vtot += 288L * w;
        ctot += 32L * w;
      }
    }
    // ---------- upload
    cudaStream_t s = stream;
    tile_slice.upload(tslice, s);
    // free soft rows of each env in node order, in chunks of 32 (the persistent PCG's slices):
    // kinematic rows have r = 0 and a zero preconditioner block, so their d, z stay 0 and the
    // solve never needs them
    {
      std::vector<int> prow, psel, poff(E + 1, 0);
      std::vector<std::vector<int>> free_rows(E);
      for (size_t ti = 0; ti < te.size(); ++ti)
        if (tk[ti] == 0)
          for (int r = tb[ti]; r < tn[ti]; ++r)
            if (!node_kin_h[r]) free_rows[te[ti]].push_back(r);
      for (int li = 0; li < E; ++li) {
        int nf = (int)free_rows[li].size(), nch = (nf + 31) / 32;
        for (int q = 0; q < 32 * nch; ++q) {
          int r = q < nf ? free_rows[li][q] : -1;
          prow.push_back(r);
          psel.push_back(r >= 0 ? row_sel[r] : -1);
        }
        poff[li + 1] = poff[li] + nch;
      }
      n_slices = poff[E];
      max_env_slices = 0;
      for (int li = 0; li < E; ++li) max_env_slices = std::max(max_env_slices, poff[li + 1] - poff[li]);
      pslice_off.upload(poff, s);
      pslice_row.upload(prow, s);
      pslice_sel.upload(psel, s);
      max_env_bodies = 0;
      for (int li = 0; li < E; ++li) max_env_bodies = std::max(max_env_bodies, body_off_h[li + 1] - body_off_h[li]);
    }
    slice_w.upload(sw, s);
    slice_vbase.upload(svb, s);
    slice_cbase.upload(scb, s);
    sell_col.upload(scol, s);
    blk_pos.upload(bpos, s);
    diag_pos.upload(dpos, s);
    sell_nval = vtot;
    node_off.upload(node_off_h, s);
    tet_off.upload(tet_off_h, s);
    body_off.upload(body_off_h, s);
    nsteps.upload(nsteps_h, s);
    grav_off.upload(grav_off_h, s);
    nh.upload(nh_h, s);
    sched_off.upload(sched_off_h, s);
    env_mu.upload(mu_h, s);
    sched.upload(sched_h, s);
    grav.upload(grav_h, s);
    node_env.upload(node_env_h, s);
    node_body.upload(node_body_h, s);
    node_handle.upload(node_handle_h, s);
    node_kin.upload(node_kin_h, s);
    node_mass.upload(node_mass_h, s);
    X0.upload(X0_h, s);
    body_node.upload(body_node_h, s);
    body_env.upload(body_env_h, s);
    body_kin.upload(body_kin_h, s);
    M4.upload(M4_h, s);
    bvol.upload(bvol_h, s);
    body_pd.upload(bpd_h, s);
    bbox.upload(bbox_h, s);
    tets.upload(tets_h, s);
    tet_prm.upload(tet_prm_h, s);
    tet_env.upload(tet_env_h, s);
    pt_node.upload(pt_node_h, s);
    pt_body.upload(pt_body_h, s);
    pt_env.upload(pt_env_h, s);
    pt_kin.upload(pt_kin_h, s);
    pt_xb.upload(pt_xb_h, s);
    sv_pt.upload(sv_pt_h, s);
    sv_env.upload(sv_env_h, s);
    ed_pt.upload(ed_pt_h, s);
    ed_env.upload(ed_env_h, s);
    ed_rest2.upload(ed_rest2_h, s);
    tri_pt.upload(tri_pt_h, s);
    tri_env.upload(tri_env_h, s);
    n_jt = (int)jt_h.size();
    jt.upload(jt_h, s);
    tile_env.upload(te, s);
    tile_kind.upload(tk, s);
    tile_begin.upload(tb, s);
    tile_end.upload(tn, s);
    tile_off.upload(toff, s);
    pcg_C = 0;
    tune_reset();  // a new batch composition is tuned afresh
    if (desc.pcg_cluster >= 0 || mixed()) {
      std::vector<int> iota(E);
      std::iota(iota.begin(), iota.end(), 0);
      env_iota.upload(iota, s);
      env_list.alloc(E + 1);
      pcg_rzs.alloc(E);
      pcg_bbs.alloc(E);
      pcg_iterb.alloc(E);
      pcg_iterf.alloc(E);
      pcg_its.alloc(E);
      pcg_runs.alloc(E);
      if (mixed()) pcg_shapes<float>();
      else pcg_shapes<double>();
    }
    root_off_tri.upload(tri_off_h, s);
    root_off_ed.upload(ed_off_h, s);
    bsr_ptr.upload(bptr, s);
    bsr_col.upload(bcol, s);
    blk_row.upload(brow, s);
    blk_ptr.upload(blkptr, s);
    blk_src.upload(blksrc, s);
    nt_ptr.upload(ntcnt, s);
    nt_src.upload(ntsrc, s);
    x.upload(x_h, s);
    v.upload(v_h, s);
    size_t n3 = 3 * (size_t)NN;
    for (DBuf<double>* b : {&xt, &xtilde, &xtarget, &xtrial, &p, &pbar, &grad, &pcg_r, &pcg_z, &pcg_d, &pcg_y, &pcg_x})
      b->alloc(n3);
    xtarget.zero(s);
    // trial points are written only for envs in a line search: start them at x
    CK(cudaMemcpyAsync(xtrial.p, x.p, n3 * sizeof(double), cudaMemcpyDeviceToDevice, s));
    // the persistent PCG never writes kinematic soft rows: their d (read by neighbours) stays 0
    for (DBuf<double>* b : {&pcg_r, &pcg_z, &pcg_d, &pcg_y, &pcg_x}) b->zero(s);
    for (DBuf<double>* b : {&ptx, &ptx_t, &ptp, &pte}) b->alloc(3 * (size_t)NP);
    e_status.upload(status_h, s);
    e_reason.upload(reason_h, s);
    e_step.upload(step_h, s);
    e_stats.upload(stats_h, s);
    for (DBuf<int>* b : {&e_constrained, &e_bad, &e_nanp, &e_halv, &e_newton_it, &e_rem}) b->alloc(E);
    e_count.alloc(4);
    for (DBuf<uint8_t>* b : {&e_stepping, &e_iter, &e_ls, &e_accept, &e_sel, &e_all, &e_start, &e_cover}) {
      b->alloc(E);
      b->zero(s);
    }
    launch(k_fill_u8, E, 256, E, e_all.p, (uint8_t)1);
    for (DBuf<double>* b : {&e_E0, &e_Et, &e_alpha}) b->alloc(E);
    e_kappa.alloc(E);
    e_trace.alloc((size_t)E * trace_cap());
    e_trace_n.alloc(E);
    e_trace_n.zero(s);
    e_kdots.alloc(2 * (size_t)E);
    launch(k_env_fill, E, 128, E, (const uint8_t*)nullptr, e_kappa.p, desc.kappa);
    for (DBuf<unsigned long long>* b : {&e_alpha_bits, &e_pnorm_bits, &e_inter, &e_inv}) b->alloc(E);
    nodeE.alloc(NN);
    tetE.alloc(NT);
    tet_g.alloc(12 * (size_t)NT);
    bodyE.alloc(NB);
    body_g.alloc(12 * (size_t)NB);
    if (mixed()) {
      f_tet_H.alloc(90 * (size_t)NT);
      f_body_H.alloc(144 * (size_t)NB);
      f_bsr_val.alloc(std::max(sell_nval, 1L));
      f_bsr_val.zero(s);  // padding blocks must read as zero
      f_Ps.alloc(9 * (size_t)NN);
      f_Pb.alloc(144 * (size_t)NB);
      for (DBuf<float>* b : {&f_r, &f_z, &f_d, &f_y, &f_x}) {
        b->alloc(n3);
        b->zero(s);  // kinematic soft rows are never written by the persistent PCG: d stays 0
      }
    } else {
      tet_H.alloc(90 * (size_t)NT);
      body_H.alloc(144 * (size_t)NB);
      bsr_val.alloc(std::max(sell_nval, 1L));
      bsr_val.zero(s);  // padding blocks must read as zero
      Ps.alloc(9 * (size_t)NN);
      Pb.alloc(144 * (size_t)NB);
    }
    for (DBuf<double>* b : {&part_a, &part_b, &part_c}) b->alloc(NTILE);
    pcg_rz.alloc(2 * (size_t)E);
    pcg_bb.alloc(E);
    pcg_it.alloc(E);
    pcg_run.alloc(E);
    pcg_active.alloc(1);
    cnt_pt.alloc(NSV + 1);
    off_pt.alloc(NSV + 1);
    cnt_ee.alloc(NED + 1);
    off_ee.alloc(NED + 1);
    overflow.alloc(2);
    overflow.zero(s);
    ns_ptr.alloc(NN + 1);
    ns_cnt.alloc(NN + 1);
    ttri.built = tedge.built = false;
    ttri.n = NTR;
    tedge.n = NED;
    n_ct = n_ct_pt = n_fr = n_fr_pt = n_pt = n_ee = 0;
    CK(cudaStreamSynchronize(s));
    dirty = false;
    initial_checks();
  }

  // ------------------------------------------------------------------ BVH
  void tree_build(TreeBufs& T, const int* prim_pt, int nv, const int* prim_env, const int* prim_off) {
    int n = T.n;
    T.pbox.ensure(6 * (size_t)std::max(n, 1));
    T.nbox.ensure(2 * (size_t)std::max(2 * n - 1, 1));
    T.keys.ensure(std::max(n, 1));
    T.vals.ensure(std::max(n, 1));
    T.child.ensure(2 * (size_t)std::max(n, 1));
    T.parent.ensure(std::max(2 * n - 1, 1));
    T.range.ensure(2 * (size_t)std::max(n, 1));
    T.root.ensure(E);
    T.flags.ensure(std::max(n, 1));
    T.emin.ensure(3 * (size_t)E);
    T.emax.ensure(3 * (size_t)E);
    if (n == 0) {
      CK(cudaMemsetAsync(T.root.p, 0xff, E * sizeof(int), stream));
      T.built = true;
      return;
    }
    if (nv == 3) launch(k_prim_boxes<3>, n, 256, n, prim_pt, (const double*)ptx.p, (const double*)nullptr, 0.0, T.pbox.p);
    else launch(k_prim_boxes<2>, n, 256, n, prim_pt, (const double*)ptx.p, (const double*)nullptr, 0.0, T.pbox.p);
    CK(cudaMemsetAsync(T.emin.p, 0xff, 3 * E * sizeof(unsigned long long), stream));
    CK(cudaMemsetAsync(T.emax.p, 0, 3 * E * sizeof(unsigned long long), stream));
    launch(k_env_bounds, n, 256, (const double*)T.pbox.p, prim_env, n, T.emin.p, T.emax.p);
    launch(k_morton, n, 256, (const double*)T.pbox.p, prim_env, n, (const unsigned long long*)T.emin.p,
           (const unsigned long long*)T.emax.p, T.keys.p, T.vals.p);
    int env_bits = 1;
    while ((1 << env_bits) < E) ++env_bits;
    radix_sort(T.keys, T.vals, T.keys2, T.vals2, T.hist, n, 32 + env_bits);
    CK(cudaMemsetAsync(T.root.p, 0xff, E * sizeof(int), stream));
    if (n == 1) {
      int m1 = -1;
      CK(cudaMemcpyAsync(T.parent.p, &m1, sizeof(int), cudaMemcpyHostToDevice, stream));
    }
    launch(k_karras, n - 1, 256, (const unsigned long long*)T.keys.p, n, T.child.p, T.parent.p, T.range.p);
    launch(k_env_roots, std::max(n - 1, E), 256, n, (const int*)T.range.p, prim_off, E, prim_env, T.root.p);
    T.built = true;
  }
  void tree_refit(TreeBufs& T) {
    if (T.n == 0) return;
    CK(cudaMemsetAsync(T.flags.p, 0, T.n * sizeof(int), stream));
    launch(k_refit, T.n, 256, T.n, (const unsigned*)T.vals.p, (const double*)T.pbox.p, (const int*)T.child.p,
           (const int*)T.parent.p, T.nbox.p, T.flags.p);
  }
  // build both trees at the current ptx
  void build_trees() {
    tree_build(ttri, tri_pt.p, 3, tri_env.p, root_off_tri.p);
    tree_build(tedge, ed_pt.p, 2, ed_env.p, root_off_ed.p);
  }
  // primitive boxes at ptx (r) or swept to pte (r = 0), then refit
  void boxes_and_refit(const double* end, double r) {
    launch(k_prim_boxes<3>, NTR, 256, NTR, (const int*)tri_pt.p, (const double*)ptx.p, end, r, ttri.pbox.p);
    launch(k_prim_boxes<2>, NED, 256, NED, (const int*)ed_pt.p, (const double*)ptx.p, end, r, tedge.pbox.p);
    tree_refit(ttri);
    tree_refit(tedge);
  }
  void check_overflow() { collect_spilled(); }
  // reads and clears the traversal flags; fails on a stack overflow, returns whether a collect
  // traversal had a query with more partners than its slots
  bool collect_spilled() {
    CK(cudaMemcpyAsync(hpin, overflow.p, 2 * sizeof(int), cudaMemcpyDeviceToHost, stream));
    host_sync();
    const int stack = hpin[0], spill = hpin[1];
    if (stack || spill) overflow.zero(stream);
    if (stack) fail_with(IPC_ERR_INTERNAL, "BVH traversal stack overflow");
    return spill != 0;
  }
  // partner slots per query of a collect traversal (a scene option; more partners send the pass
  // to a count-then-fill traversal)
  int cand_cap() const { return desc.collect_slots > 0 ? desc.collect_slots : CAND_SLOTS; }
  long long spills = 0;  // collect passes that spilled into a fill traversal
  // the candidate totals of a pair of collect traversals (the last entries of their offset
  // scans) and the traversal flags, in one read-back; fails on a stack overflow, returns
  // whether a query had more partners than its slots
  bool read_totals(const int* tot_pt, const int* tot_ee, int* np, int* ne) {
    CK(cudaMemcpyAsync(hpin, tot_pt, sizeof(int), cudaMemcpyDeviceToHost, stream));
    CK(cudaMemcpyAsync(hpin + 1, tot_ee, sizeof(int), cudaMemcpyDeviceToHost, stream));
    CK(cudaMemcpyAsync(hpin + 2, overflow.p, 2 * sizeof(int), cudaMemcpyDeviceToHost, stream));
    host_sync();
    *np = hpin[0];
    *ne = hpin[1];
    const int stack = hpin[2], spill = hpin[3];
    if (stack || spill) overflow.zero(stream);
    if (stack) fail_with(IPC_ERR_INTERNAL, "BVH traversal stack overflow");
    spills += spill != 0;
    return spill != 0;
  }

  // ------------------------------------------------------------------ constraint set
  // contacts (d < dhat) of the envs in act at positions ptx (already computed)
  void constraint_set(const uint8_t* act) {
    double r = 0.5 * desc.dhat;
    boxes_and_refit(nullptr, r);
    // one traversal per query kind keeps up to cand_cap() partners per query (edge-edge queries
    // on fine surfaces find a few dozen non-adjacent neighbours); a fill traversal
    // runs only if some query found more
    slots_pt.ensure((size_t)NSV * cand_cap() + 1);
    slots_ee.ensure((size_t)NED * cand_cap() + 1);
    CandOut o{cnt_pt.p, nullptr, slots_pt.p, overflow.p, cand_cap()};
    pbeg(IPC_PROF_BROAD);
    launch(k_trav_pt<TRAV_COLLECT>, NSV, 128, NSV, (const int*)sv_pt.p, (const int*)sv_env.p, act,
           (const double*)ptx.p, (const double*)nullptr, r, tree(ttri), (const int*)tri_pt.p, ptinfo(), o);
    CandOut oe{cnt_ee.p, nullptr, slots_ee.p, overflow.p, cand_cap()};
    launch(k_trav_ee<TRAV_COLLECT>, NED, 128, NED, (const int*)ed_pt.p, (const int*)ed_env.p, act,
           (const double*)tedge.pbox.p, tree(tedge), ptinfo(), oe);
    pend(IPC_PROF_BROAD);
    scan(cnt_pt.p, NSV, off_pt.p, false);
    scan(cnt_ee.p, NED, off_ee.p, false);
    const bool spilled = read_totals(off_pt.p + NSV, off_ee.p + NED, &n_pt, &n_ee);
    pwork(IPC_PROF_BROAD, traversal_bytes(n_pt, n_ee));
    int nc = n_pt + n_ee;
    cand_j.ensure(nc + 1);
    cand_q.ensure(nc + 1);
    if (spilled) {
      CandOut f{nullptr, off_pt.p, cand_j.p, overflow.p, 0, cand_q.p};
      launch(k_trav_pt<TRAV_FILL>, NSV, 128, NSV, (const int*)sv_pt.p, (const int*)sv_env.p, act, (const double*)ptx.p,
             (const double*)nullptr, r, tree(ttri), (const int*)tri_pt.p, ptinfo(), f);
      CandOut fe{nullptr, off_ee.p, cand_j.p + n_pt, overflow.p, 0, cand_q.p + n_pt};
      launch(k_trav_ee<TRAV_FILL>, NED, 128, NED, (const int*)ed_pt.p, (const int*)ed_env.p, act,
             (const double*)tedge.pbox.p, tree(tedge), ptinfo(), fe);
    } else {
      launch(k_gather_cands, NSV, 256, NSV, cand_cap(), (const int*)cnt_pt.p, (const int*)slots_pt.p,
             (const int*)off_pt.p, cand_j.p, cand_q.p, 1);
      launch(k_gather_cands, NED, 256, NED, cand_cap(), (const int*)cnt_ee.p, (const int*)slots_ee.p,
             (const int*)off_ee.p, cand_j.p + n_pt, cand_q.p + n_pt, 1);
    }
    cand_rec.ensure(nc + 1);
    launch(k_cand_records, nc, 256, n_pt, n_ee, (const int*)cand_q.p, (const int*)cand_j.p, (const int*)sv_pt.p,
           (const int*)sv_env.p, (const int*)tri_pt.p, (const int*)ed_pt.p, (const int*)ed_env.p,
           (const double*)ed_rest2.p, cand_rec.p);
    contacts_from_list(nullptr, n_pt, n_ee, cand_rec.p);
  }
  // Narrow phase over a candidate list (point-triangle per surface vertex, then edge-edge per
  // edge, partners ascending): contacts d < dhat at positions ptx, in list order. act (or null)
  // keeps only the envs of this evaluation when the list holds more.
  void contacts_from_list(const uint8_t* act, int np, int ne, const ContactRec* rec) {
    const int nc = np + ne;
    nflag.ensure(nc + 1);
    noff.ensure(nc + 1);
    ct_tmp.ensure(nc + 1);
    double dh2 = desc.dhat * desc.dhat;
    launch(k_narrow, nc, 128, nc, rec, act, (const double*)ptx.p, dh2, nflag.p, ct_tmp.p);
    scan(nflag.p, nc, noff.p, false);
    // the contacts' count and the point-triangle part of it, in one read-back
    CK(cudaMemcpyAsync(hpin, noff.p + np, sizeof(int), cudaMemcpyDeviceToHost, stream));
    CK(cudaMemcpyAsync(hpin + 1, noff.p + nc, sizeof(int), cudaMemcpyDeviceToHost, stream));
    host_sync();
    n_ct_pt = hpin[0];
    n_ct = hpin[1];
    ct.ensure(n_ct + 1);
    launch(k_compact_contacts, nc, 256, nc, (const int*)nflag.p, (const int*)noff.p, (const ContactRec*)ct_tmp.p, ct.p);
  }
  // Where the contact set of the next evaluation inside a time step comes from. STATIC: the
  // step start's list at x^t, while the DOFs are still x^t. SWEPT: the step filter's list of
  // boxes swept over [x, x + p] and grown by dhat/2 (plus a margin far above the rounding of
  // x + alpha p): a pair that comes within dhat anywhere on that segment has overlapping grown
  // boxes, so the list holds every contact of every line-search trial and of the accepted
  // point. Either way the narrow phase keeps exactly the pairs with d < dhat, in the order a
  // fresh traversal gives (per query, partners ascending): the contacts, and every result, are
  // the same as with a traversal at each evaluation.
  enum { CAND_FRESH = 0, CAND_STATIC = 1, CAND_SWEPT = 2 };
  int cand_src = CAND_FRESH;
  int ccd_np = 0, ccd_ne = 0;
  bool reuse_lists() const { return desc.fresh_broad_phase == 0; }
  double swept_growth() const { return reuse_lists() ? 0.5 * desc.dhat * (1.0 + 1e-6) : 0.0; }
  void contacts_at(const uint8_t* act) {
    if (cand_src == CAND_SWEPT) contacts_from_list(act, ccd_np, ccd_ne, ccd_rec.p);
    else if (cand_src == CAND_STATIC) contacts_from_list(act, n_pt, n_ee, cand_rec.p);
    else constraint_set(act);
  }
  void stencil_table() {
    int ns = n_st();
    st_pts.ensure(4 * (size_t)ns + 4);
    st_env.ensure(ns + 1);
    sE.ensure(ns + 1);
    sg.ensure(12 * (size_t)ns + 12);
    st_t.ensure(12 * (size_t)ns + 12);
    st_node.ensure(4 * (size_t)ns + 4);
    ct_Hl.ensure(144 * (size_t)n_ct + 144);
    if (mixed()) {
      f_sH.ensure(78 * (size_t)ns + 78);
      f_st_t.ensure(12 * (size_t)ns + 12);
      f_st_xb.ensure(12 * (size_t)ns + 12);
    } else {
      sH.ensure(78 * (size_t)ns + 78);
      st_xb.ensure(12 * (size_t)ns + 12);
    }
    launch(k_stencil_table, ns, 256, n_ct, n_fr, n_jt, (const ContactRec*)ct.p, (const FrictionRec*)fr.p,
           (const JointRec*)jt.p, st_pts.p, st_env.p);
  }
  // ------------------------------------------------------------------ energy
  // energies (and derivatives) of the envs in act at DOFs q; positions/contacts at q are
  // computed here. Result per env in out.
  template <int MODE>
  void evaluate(const double* q, const uint8_t* act, double* out) {
    if (MODE == MODE_HESS && mixed()) evaluate_t<MODE, float>(q, act, out);
    else evaluate_t<MODE, double>(q, act, out);
  }
  // HT: precision of the Hessians (energies and gradients are FP64 in every mode)
  template <int MODE, class HT>
  void evaluate_t(const double* q, const uint8_t* act, double* out) {
    launch(k_points, NP, 256, NP, (const int*)pt_node.p, (const double*)pt_xb.p, (const int*)body_node.p, q, ptx.p);
    contacts_at(act);
    stencil_table();
    // Hessian outputs (taken after stencil_table, which may grow the stencil buffers)
    HT* tH = MODE == MODE_HESS ? hp<HT>(tet_H, f_tet_H) : nullptr;
    HT* bH = MODE == MODE_HESS ? hp<HT>(body_H, f_body_H) : nullptr;
    HT* sHp = MODE == MODE_HESS ? hp<HT>(sH, f_sH) : nullptr;
    double h = desc.dt, h2 = h * h;
    // Hessian evaluations: the body and contact kernels (few blocks, long serial FP64 chains)
    // run on the side stream beside the element kernels; they write disjoint outputs
    const bool fork = MODE == MODE_HESS && !capturing;
    if (fork) {
      CK(cudaEventRecord(fork_ev, stream));
      CK(cudaStreamWaitEvent(side, fork_ev, 0));
      std::swap(stream, side);  // the launches below go to the side stream
      launch_contacts<MODE, HT>(act, q, h2, bH, sHp);
      CK(cudaEventRecord(join_ev, stream));
      std::swap(stream, side);
    }
    launch(k_inertia_energy, NN, 256, NN, layout(), act, q, (const double*)xtilde.p, nodeE.p);
    int efam = MODE == MODE_ENERGY ? IPC_PROF_LS_ENERGY : IPC_PROF_ELASTIC;
    pbeg(efam);
    launch(k_elastic<MODE, HT>, NT, 128, NT, (const int4*)tets.p, (const double*)tet_prm.p, (const int*)tet_env.p, act,
           q, h2, tetE.p, tet_g.p, tH, e_bad.p, MODE == MODE_ENERGY ? (unsigned long long*)nullptr : punits(IPC_PROF_ELASTIC));
    pend(efam);
    if (fork) CK(cudaStreamWaitEvent(stream, join_ev, 0));
    else launch_contacts<MODE, HT>(act, q, h2, bH, sHp);
    EnergyLists L{nodeE.p, node_off.p, tetE.p, tet_off.p, bodyE.p, body_off.p, sE.p, st_env.p,
                  n_ct_pt, n_ct - n_ct_pt, n_fr_pt, n_fr, n_jt};
    launch_grid(k_env_energy, E, 256, E, L, act, out);
  }
  // affine bodies, barrier and friction stencils of one evaluation
  template <int MODE, class HT>
  void launch_contacts(const uint8_t* act, const double* q, double h2, HT* bH, HT* sHp) {
    const double h = desc.dt;
    if constexpr (MODE == MODE_HESS)
      launch(k_bodies_hess<HT>, 16L * NB, BODY_HESS_THREADS, NB, (const int*)body_node.p, (const int*)body_env.p,
             (const uint8_t*)body_kin.p, (const double*)M4.p, (const double*)bvol.p, act, q, (const double*)xtilde.p,
             (const double*)xtarget.p, (const double*)body_pd.p, h2, h2 * desc.kappa_affine, bodyE.p, body_g.p, bH);
    else
      launch(k_bodies<MODE>, NB, 64, NB, (const int*)body_node.p, (const int*)body_env.p, (const uint8_t*)body_kin.p,
             (const double*)M4.p, (const double*)bvol.p, act, q, (const double*)xtilde.p, (const double*)xtarget.p,
             (const double*)body_pd.p, h2, h2 * desc.kappa_affine, bodyE.p, body_g.p);
    int cfam = MODE == MODE_ENERGY ? IPC_PROF_LS_ENERGY : IPC_PROF_CONTACT;
    pbeg(cfam);
    if constexpr (MODE != MODE_ENERGY) {
      // per stencil: record, gathered points (friction: at x and x^t), barrier stiffness; energy,
      // 12 gradient and (Hessian evaluations) 78 packed Hessian entries out
      const double hb = MODE == MODE_HESS ? 78.0 * sizeof(HT) : 0.0;
      pwork(IPC_PROF_CONTACT, (double)n_ct * (40 + 96 + 8 + 8 + 96 + hb) + (double)n_fr * (88 + 192 + 8 + 96 + hb) +
                                  (double)n_jt * (24 + 48 + 8 + 96 + hb));
    }
    if constexpr (MODE == MODE_HESS)
    {
      launch(k_barrier_local, n_ct, BARRIER_LOCAL_THREADS, n_ct, (const ContactRec*)ct.p, act, (const double*)ptx.p,
             h2, desc.dhat, (const double*)e_kappa.p, sE.p, sg.p, ct_Hl.p);
      launch(k_barrier_hess<HT>, (long)BARRIER_HESS_THREADS * n_ct, BARRIER_HESS_THREADS, n_ct, (const ContactRec*)ct.p,
             act, (const double*)ct_Hl.p, sHp);
    }
    else
      launch(k_barrier<MODE>, n_ct, 64, n_ct, (const ContactRec*)ct.p, act, (const double*)ptx.p, h2, desc.dhat,
             (const double*)e_kappa.p, sE.p, sg.p);
    launch(k_friction<MODE, HT>, n_fr, 128, n_fr, (const FrictionRec*)fr.p, act, (const double*)ptx.p,
           (const double*)ptx_t.p, h2, desc.eps_v * h, sE.p + n_ct, sg.p + 12 * (size_t)n_ct,
           sHp ? sHp + 78 * (size_t)n_ct : sHp);
    const size_t j0 = (size_t)n_ct + n_fr;
    launch(k_joint<MODE, HT>, n_jt, 128, n_jt, (const JointRec*)jt.p, act, (const double*)ptx.p, h2, sE.p + j0,
           sg.p + 12 * j0, sHp ? sHp + 78 * j0 : sHp);
    pend(cfam);
  }

  // ------------------------------------------------------------------ adapted stiffness
  // gradient of the incremental potential at the DOFs x for the envs in act, into grad
  void gradient_at_x(const uint8_t* act) {
    evaluate<MODE_GRAD>(x.p, act, e_Et.p);
    stencil_incidence(act);
    launch(k_assemble_grad, NN, 256, NN, layout(), act, (const double*)x.p, (const double*)xtilde.p,
           (const int*)nt_ptr.p, (const int*)nt_src.p, (const double*)tet_g.p, (const double*)body_g.p,
           (const int*)ns_ptr.p, (const int*)ns_src.p, (const int*)st_pts.p, (const double*)sg.p, grad.p, nodeE.p);
  }
  // stiffness of the envs in act at their step start (x = x^t; their friction lag not yet made,
  // or made at x^t, where it has no gradient)
  void kappa_start(const uint8_t* act) {
    g0buf.ensure(3 * (size_t)NN);
    launch(k_env_fill, E, 128, E, act, e_kappa.p, 0.0);
    gradient_at_x(act);
    CK(cudaMemcpyAsync(g0buf.p, grad.p, 3 * (size_t)NN * sizeof(double), cudaMemcpyDeviceToDevice, stream));
    launch(k_env_fill, E, 128, E, act, e_kappa.p, 1.0);
    gradient_at_x(act);
    launch_grid(k_env_kappa_dots, E, 256, E, layout(), act, (const int*)node_off.p, (const double*)g0buf.p,
                (const double*)grad.p, e_kdots.p);
    launch(k_env_kappa_start, E, 128, E, act, (const double*)e_kdots.p, desc.kappa, 1000.0 * desc.kappa, e_kappa.p);
  }

  // stencil -> node incidence (stable by stencil order within each node)
  void stencil_incidence(const uint8_t* act) {
    int ns = n_st();
    st_cnt.ensure(ns + 1);
    st_off.ensure(ns + 1);
    launch(k_stencil_nent, ns, 256, ns, (const int*)st_pts.p, (const int*)st_env.p, act, (const int*)pt_node.p, st_cnt.p);
    int ne = scan(st_cnt.p, ns, st_off.p);
    n_inc = ne;
    st_keys.ensure(ne + 1);
    st_vals.ensure(ne + 1);
    launch(k_stencil_emit, ns, 256, ns, (const int*)st_pts.p, (const int*)st_env.p, act, (const int*)pt_node.p,
           (const int*)body_node.p, (const int*)st_off.p, st_keys.p, st_vals.p);
    int bits = 1;
    while ((1 << bits) < NN) ++bits;
    radix_sort(st_keys, st_vals, st_keys2, st_vals2, st_hist, ne, bits);
    CK(cudaMemsetAsync(ns_cnt.p, 0, (NN + 1) * sizeof(int), stream));
    launch(k_count_keys, ne, 256, ne, (const unsigned long long*)st_keys.p, ns_cnt.p);
    scan(ns_cnt.p, NN, ns_ptr.p, false);
    ns_src.ensure(ne + 1);
    if (ne > 0) CK(cudaMemcpyAsync(ns_src.p, st_vals.p, ne * sizeof(unsigned), cudaMemcpyDeviceToDevice, stream));
    if (mixed()) {
      f_ns_w.ensure(ne + 1);
      f_ns_xb.ensure(3 * (size_t)ne + 3);
      launch(k_entry_weights<float>, ne, 256, ne, layout(), act, (const unsigned long long*)st_keys.p,
             (const int*)ns_src.p, (const int*)st_pts.p, f_ns_w.p, f_ns_xb.p);
      launch(k_stencil_nodes<float>, 4L * ns, 256, ns, layout(), (const int*)st_pts.p, (const int*)st_env.p, act,
             st_node.p, f_st_xb.p);
    } else {
      ns_w.ensure(ne + 1);
      ns_xb.ensure(3 * (size_t)ne + 3);
      launch(k_entry_weights<double>, ne, 256, ne, layout(), act, (const unsigned long long*)st_keys.p,
             (const int*)ns_src.p, (const int*)st_pts.p, ns_w.p, ns_xb.p);
      launch(k_stencil_nodes<double>, 4L * ns, 256, ns, layout(), (const int*)st_pts.p, (const int*)st_env.p, act,
             st_node.p, st_xb.p);
    }
  }

  // matrix in HT, vectors and stencil products (st) in VT
  template <class HT, class VT>
  SpmvArgsT<HT, VT> spmv_args(const VT* st) {
    SellT<HT> S{tile_slice.p, slice_w.p, slice_vbase.p, slice_cbase.p, sell_col.p, hp<HT>(bsr_val, f_bsr_val)};
    return SpmvArgsT<HT, VT>{S,      bsr_ptr.p,  hp<HT>(body_H, f_body_H), ns_ptr.p,
                             ns_src.p, hp<HT>(ns_w, f_ns_w), hp<HT>(ns_xb, f_ns_xb), st_pts.p,
                             st,     hp<HT>(sH, f_sH), st_node.p, hp<HT>(st_xb, f_st_xb)};
  }
  SpmvArgs spmv_args() { return spmv_args<double, double>(st_t.p); }
  // y = H d over the envs in run (stencil product, then BSR/body rows); partial d.y per tile.
  // FP64 vectors; the matrix is in the scene's Hessian precision.
  void matvec(const uint8_t* run, const double* d, double* y, double* part) {
    if (mixed()) matvec_t<float>(run, d, y, part);
    else matvec_t<double>(run, d, y, part);
  }
  template <class HT>
  void matvec_t(const uint8_t* run, const double* d, double* y, double* part) {
    int ns = n_st();
    launch(k_stencil_mv<HT, double>, 16L * ns, 128, ns, layout(), (const int*)st_env.p, (const int*)st_pts.p, run,
           (const HT*)hp<HT>(sH, f_sH), d, st_t.p);
    pbeg(IPC_PROF_SPMV);
    launch_grid(k_spmv<HT, double>, NTILE, TILE, tiles(), layout(), spmv_args<HT, double>(st_t.p), run, d, y, part,
                punits(IPC_PROF_SPMV));
    pend(IPC_PROF_SPMV);
  }

  // ------------------------------------------------------------------ PCG
  // Clusters that can be resident at once for a cluster size C (occupancy of k_pcg_cluster<C>).
  template <int C>
  static cudaLaunchAttribute cluster_attr() {
    cudaLaunchAttribute at;
    at.id = cudaLaunchAttributeClusterDimension;
    at.val.clusterDim.x = C;
    at.val.clusterDim.y = 1;
    at.val.clusterDim.z = 1;
    return at;
  }
  // Slot partials of the persistent PCG live in the CTAs' shared memory: slots one CTA of a
  // C-cluster owns, and the dynamic shared memory that takes.
  int ns_loc(int C) const { return (std::max(max_env_slices, 1) + C - 1) / C; }
  int nb_loc(int C) const { return (std::max(max_env_bodies, 1) + C - 1) / C; }
  template <class T>
  size_t pcg_smem(int C) const { return pcg_smem_bytes<T>(ns_loc(C), nb_loc(C)); }
  static constexpr size_t PCG_SMEM_CAP = 160 * 1024;  // leaves room for the static arrays
  int pcg_c_min = 1;  // smallest cluster size whose slot partials fit PCG_SMEM_CAP
  template <int C, class T>
  int resident_clusters() {
    if (C > 8) CK(cudaFuncSetAttribute(k_pcg_cluster<C, T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    const size_t smem = pcg_smem<T>(C);
    if (smem > PCG_SMEM_CAP) return 0;  // never chosen
    CK(cudaFuncSetAttribute(k_pcg_cluster<C, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    cudaLaunchAttribute at = cluster_attr<C>();
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(C * std::max(E, 1)));
    cfg.blockDim = dim3(PCG_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cfg.attrs = &at;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k_pcg_cluster<C, T>, &cfg) != cudaSuccess) {
      cudaGetLastError();  // a size the device cannot schedule: never chosen
      n = 0;
    }
    return n;
  }
  template <class T>
  void pcg_shapes() {
    pcg_resident[0] = resident_clusters<1, T>();
    pcg_resident[1] = resident_clusters<2, T>();
    pcg_resident[2] = resident_clusters<4, T>();
    pcg_resident[3] = resident_clusters<8, T>();
    pcg_resident[4] = resident_clusters<16, T>();
    pcg_c_min = 0;
    for (int k = 0; k <= 4 && !pcg_c_min; ++k)
      if (pcg_smem<T>(1 << k) <= PCG_SMEM_CAP) pcg_c_min = 1 << k;
    if (!pcg_c_min)
      fail_with(IPC_ERR_INTERNAL, "an environment has too many free soft rows for the persistent PCG (" +
                                      std::to_string(32L * max_env_slices) + ")");
  }
  // Cluster size for n running solves: the caller's choice, else the largest C <= 16 whose n
  // clusters are all resident at once and that still leaves each CTA two 32-row slices of the
  // largest env; never below the smallest size whose slot partials fit in shared memory. Fewer
  // running solves get more SMs each; the bits do not depend on C.
  int pick_cluster(int n) {
    if (desc.pcg_cluster > 0) return std::max(desc.pcg_cluster, pcg_c_min);
    for (int k = 4; k > 0; --k) {
      int C = 1 << k;
      if (2 * C <= std::max(max_env_slices, 2) && n <= pcg_resident[k]) return std::max(C, pcg_c_min);
    }
    return pcg_c_min;
  }
  // Launch-shape autotuner of the persistent PCG. The running-env count of a launch falls in one
  // of three buckets (more than fit resident with 8-CTA clusters; more than fit with 16; fewer).
  // A bucket's candidates are the largest all-resident cluster size h (pick_cluster) and 2h,
  // which oversubscribes the GPU but gives each env more SMs; they are tried alternately on the
  // bucket's first launches, timed with CUDA events per env-iteration, and the faster is kept.
  // The cluster size changes no bit of any result, so tuning never changes a trajectory.
  struct TuneBucket {
    int cand[2] = {0, 0};
    double ms[2] = {0.0, 0.0};
    unsigned long long its[2] = {0, 0};
    int tries[2] = {0, 0};
    int best = -1;
  };
  static constexpr int TUNE_TRIES = 2;
  TuneBucket tune[3];
  void tune_reset() {
    for (auto& b : tune) b = TuneBucket();
  }
  int bucket_of(int n) const { return n > pcg_resident[3] ? 0 : (n > pcg_resident[4] ? 1 : 2); }
  // cluster size for the next launch over n running envs, and the candidate slot being timed (-1)
  int tuned_cluster(int n, int* slot) {
    *slot = -1;
    int h = pick_cluster(n);
    if (desc.pcg_cluster > 0) return h;
    TuneBucket& b = tune[bucket_of(n)];
    if (b.cand[0] == 0) {
      b.cand[0] = h;
      int h2 = 2 * h, k2 = h2 == 2 ? 1 : h2 == 4 ? 2 : h2 == 8 ? 3 : h2 == 16 ? 4 : -1;
      b.cand[1] = (k2 > 0 && pcg_resident[k2] > 0 && 2 * h2 <= std::max(max_env_slices, 2)) ? h2 : 0;
      if (b.cand[1] == 0) b.best = 0;
    }
    if (b.best >= 0) return b.cand[b.best];
    *slot = b.tries[0] <= b.tries[1] ? 0 : 1;
    return b.cand[*slot];
  }
  void tune_record(int n, int slot, float ms, unsigned long long its) {
    TuneBucket& b = tune[bucket_of(n)];
    if (slot < 0 || b.best >= 0 || its == 0) return;
    b.ms[slot] += ms;
    b.its[slot] += its;
    b.tries[slot]++;
    if (b.tries[0] >= TUNE_TRIES && b.tries[1] >= TUNE_TRIES)
      b.best = (b.ms[1] / (double)b.its[1] < b.ms[0] / (double)b.its[0]) ? 1 : 0;
  }
  template <int C, class T>
  void launch_pcg_cluster(const PcgClusterArgs<T>& a0, int n) {
    PcgClusterArgs<T> a = a0;
    a.ns_loc = ns_loc(C);
    a.nb_loc = nb_loc(C);
    const size_t smem = pcg_smem_bytes<T>(a.ns_loc, a.nb_loc);
    if (smem > PCG_SMEM_CAP) fail_with(IPC_ERR_INTERNAL, "PCG slot partials exceed shared memory");
    if (C > 8) CK(cudaFuncSetAttribute(k_pcg_cluster<C, T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    CK(cudaFuncSetAttribute(k_pcg_cluster<C, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    cudaLaunchAttribute at = cluster_attr<C>();
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(C * n));
    cfg.blockDim = dim3(PCG_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cfg.attrs = &at;
    cfg.numAttrs = 1;
    mark_resume();
    CK(cudaLaunchKernelEx(&cfg, k_pcg_cluster<C, T>, a));
    ++launches;
  }
  template <class T>
  void launch_pcg_any(int C, const PcgClusterArgs<T>& a, int n) {
    switch (C) {
      case 1: launch_pcg_cluster<1>(a, n); break;
      case 2: launch_pcg_cluster<2>(a, n); break;
      case 4: launch_pcg_cluster<4>(a, n); break;
      case 8: launch_pcg_cluster<8>(a, n); break;
      case 16: launch_pcg_cluster<16>(a, n); break;
      default: fail_with(IPC_ERR_ARG, "pcg_cluster must be -1, 0, 1, 2, 4, 8 or 16");
    }
  }
  // The solves of the envs in act, pcg_chunk() iterations per launch at most: after each launch the
  // envs still running are listed on the device and relaunched, with a cluster size chosen for
  // their number. The first launch starts every solve.
  // iterations per launch: the FP64 solve (arithmetic-bound) gains from compacting the running
  // envs more often, the FP32 solve (latency-bound) from fewer host round trips (measured)
  template <class T>
  static constexpr int pcg_chunk() {
    return sizeof(T) == 8 ? 16 : 64;
  }
  // T: precision of the solve (FP64, or FP32 in mixed precision)
  template <class T>
  void pcg_persistent(const uint8_t* act) {
    PcgClusterArgs<T> a;
    a.L = layout();
    T* st = hp<T>(st_t, f_st_t);
    a.A = spmv_args<T, T>(st);
    a.pslice_off = pslice_off.p;
    a.pslice_row = pslice_row.p;
    a.pslice_sel = pslice_sel.p;
    a.body_off = body_off.p;
    a.st_env = st_env.p;
    a.sH = hp<T>(sH, f_sH);
    int b[6] = {0, n_ct_pt, n_ct, n_ct + n_fr_pt, n_ct + n_fr, n_st()};
    for (int i = 0; i < 6; ++i) a.st_bounds[i] = b[i];
    a.Ps = hp<T>(Ps, f_Ps);
    a.Pb = hp<T>(Pb, f_Pb);
    a.act = act;
    a.x = hp<T>(pcg_x, f_x);
    a.r = hp<T>(pcg_r, f_r);
    a.z = hp<T>(pcg_z, f_z);
    a.d = hp<T>(pcg_d, f_d);
    a.y = hp<T>(pcg_y, f_y);
    a.st_t = st;
    a.tol2 = desc.pcg_rel_tol * desc.pcg_rel_tol;
    a.max_it = desc.max_pcg_iters;
    a.env_list = env_iota.p;
    a.first = 1;
    a.chunk = pcg_chunk<T>();
    a.rz_state = pcg_rzs.p;
    a.bb_state = pcg_bbs.p;
    a.iterb_state = pcg_iterb.p;
    a.iterf_state = pcg_iterf.p;
    a.it_state = pcg_its.p;
    a.run = pcg_runs.p;
    a.stats = e_stats.p;
    a.bytes = punits(IPC_PROF_PCG_SOLVE);
    a.flops = punits(IPC_PROF_PCG_FLOPS);
    int n = E, slot = -1;
    int C = tuned_cluster(n, &slot);
    pcg_C = C;
    if (!tune_ev[0]) {
      CK(cudaEventCreate(&tune_ev[0]));
      CK(cudaEventCreate(&tune_ev[1]));
    }
    pcg_tune_iters.ensure(1);
    for (;;) {
      const int n_launch = n;
      a.iters = slot >= 0 ? pcg_tune_iters.p : nullptr;
      if (slot >= 0) {
        CK(cudaMemsetAsync(pcg_tune_iters.p, 0, sizeof(unsigned long long), stream));
        CK(cudaEventRecord(tune_ev[0], stream));
      }
      pbeg(IPC_PROF_PCG_SOLVE);
      launch_pcg_any(C, a, n);
      pend(IPC_PROF_PCG_SOLVE);
      if (slot >= 0) CK(cudaEventRecord(tune_ev[1], stream));
      launch_grid(k_list_running, 1, 32, E, (const uint8_t*)pcg_runs.p, env_list.p, pcg_active.p);
      n = read_int(pcg_active.p);  // synchronises the stream
      if (slot >= 0) {
        float ms = 0.f;
        unsigned long long its = 0;
        CK(cudaEventElapsedTime(&ms, tune_ev[0], tune_ev[1]));
        CK(cudaMemcpy(&its, pcg_tune_iters.p, sizeof(its), cudaMemcpyDeviceToHost));
        tune_record(n_launch, slot, ms, its);
      }
      if (n == 0) break;
      a.first = 0;
      a.env_list = env_list.p;
      C = tuned_cluster(n, &slot);
      // once every running solve fits in the largest clusters, a relaunch gives none of them more
      // CTAs: run them to the end in long chunks (fewer launches and host round trips)
      if (bucket_of(n) == 2) a.chunk = PCG_TAIL_CHUNK;
    }
  }
  static constexpr int PCG_TAIL_CHUNK = 128;
  void pcg(const uint8_t* act) {
    if (mixed()) {
      pcg_persistent<float>(act);
      return;
    }
    if (desc.pcg_cluster >= 0) {
      pcg_persistent<double>(act);
      return;
    }
    PcgState S{pcg_rz.p, pcg_bb.p, pcg_it.p, pcg_run.p, pcg_active.p, e_stats.p + 0};
    // per-env cumulative iterations live in e_stats[5e + 1]: pass a strided view via a kernel
    CK(cudaMemsetAsync(pcg_active.p, 0, sizeof(int), stream));
    launch_grid(k_pcg_init, NTILE, TILE, tiles(), layout(), act, (const double*)Ps.p, (const double*)Pb.p,
                (const double*)pcg_r.p, pcg_z.p, pcg_d.p, pcg_x.p, part_b.p, part_c.p);
    pcg_iters.ensure(E);
    pcg_iters.zero(stream, E);
    S.total_iters = pcg_iters.p;
    launch_grid(k_pcg_init_env, E, 32, E, tiles(), act, (const double*)part_b.p, (const double*)part_c.p, S);
    int active = read_int(pcg_active.p);
    int parity = 0;
    int done_iters = 0;
    double tol2 = desc.pcg_rel_tol * desc.pcg_rel_tol;
    const int chunk = 8;  // even, so every replay starts at parity 0
    cudaGraphExec_t exec = nullptr;
    long long graph_kernels = 0;
    while (active > 0 && done_iters < desc.max_pcg_iters) {
      if (!exec) {
        capturing = true;
        captured_kernels = 0;
        CK(cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal));
        for (int c = 0; c < chunk; ++c) {
          matvec(pcg_run.p, pcg_d.p, pcg_y.p, part_a.p);
          pbeg(IPC_PROF_PCG_VECTOR);
          launch_grid(k_pcg_update, NTILE, TILE, tiles(), layout(), S, parity, E, (const double*)part_a.p,
                      (const double*)Ps.p, (const double*)Pb.p, (const double*)pcg_d.p, (const double*)pcg_y.p,
                      pcg_x.p, pcg_r.p, pcg_z.p, part_b.p, part_c.p);
          launch_grid(k_pcg_direction, NTILE, TILE, tiles(), layout(), S, parity, E, tol2, desc.max_pcg_iters,
                      (const double*)part_b.p, (const double*)part_c.p, (const double*)part_a.p,
                      (const double*)pcg_z.p, pcg_d.p);
          pend(IPC_PROF_PCG_VECTOR);
          parity ^= 1;
        }
        cudaGraph_t g;
        cudaError_t ce = cudaStreamEndCapture(stream, &g);
        capturing = false;
        graph_kernels = captured_kernels;
        CK(ce);
        CK(cudaGraphInstantiate(&exec, g, 0));
        CK(cudaGraphDestroy(g));
      }
      CK(cudaGraphLaunch(exec, stream));
      launches += graph_kernels;
      done_iters += chunk;
      active = read_int(pcg_active.p);
      if (prof_on) graph_prof_collect();
    }
    if (exec) CK(cudaGraphExecDestroy(exec));
    graph_prof_release();
    launch(k_add_stats, E, 128, E, (const long long*)pcg_iters.p, e_stats.p);
    CK(cudaStreamSynchronize(stream));
  }

  // ------------------------------------------------------------------ one Newton iteration
  void assemble(const uint8_t* act) {
    pbeg(IPC_PROF_ASSEMBLY);
    stencil_incidence(act);
    launch(k_assemble_grad, NN, 256, NN, layout(), act, (const double*)x.p, (const double*)xtilde.p, (const int*)nt_ptr.p,
           (const int*)nt_src.p, (const double*)tet_g.p, (const double*)body_g.p, (const int*)ns_ptr.p,
           (const int*)ns_src.p, (const int*)st_pts.p, (const double*)sg.p, grad.p, nodeE.p);
    if (mixed()) assemble_h<float>(act);
    else assemble_h<double>(act);
    pend(IPC_PROF_ASSEMBLY);
    // gradient gather (per node: x, x~, mass, offsets, the gradient out; per tet corner and per
    // stencil entry: index and 3 gradient values), sliced-ELL gather (per block: row, column,
    // offsets, position and 9 values out; per tet-block contribution: index and 9 values), the
    // soft and body preconditioner blocks (read and written once); the incidence sort is not
    // counted
    const double b = mixed() ? 4.0 : 8.0;
    pwork(IPC_PROF_ASSEMBLY, (double)NN * 88 + 4.0 * NT * 28 + (double)n_inc * 32 + (double)NNZB * (24 + 9 * b) +
                                 16.0 * NT * (4 + 9 * b) + (double)NN * (8 + 18 * b) + (double)n_inc * (4 + 9 * b) +
                                 (double)NB * 288 * b);
  }
  // sliced-ELL values and block-Jacobi blocks in the Hessian precision HT
  template <class HT>
  void assemble_h(const uint8_t* act) {
    HT* val = hp<HT>(bsr_val, f_bsr_val);
    const HT* sHp = hp<HT>(sH, f_sH);
    launch(k_assemble_bsr<HT>, NNZB, 128, NNZB, (const int*)blk_row.p, (const int*)bsr_col.p, layout(), act,
           (const int*)blk_ptr.p, (const int*)blk_src.p, (const HT*)hp<HT>(tet_H, f_tet_H), (const long*)blk_pos.p,
           val);
    launch(k_precond_soft<HT>, NN, 256, NN, layout(), act, (const long*)diag_pos.p, (const HT*)val,
           (const int*)ns_ptr.p, (const int*)ns_src.p, sHp, hp<HT>(Ps, f_Ps));
    launch_grid(k_precond_body<HT>, NB, 144, NB, layout(), (const int*)body_env.p, act,
                (const HT*)hp<HT>(body_H, f_body_H), (const int*)ns_ptr.p, (const int*)ns_src.p,
                (const HT*)hp<HT>(ns_xb, f_ns_xb), sHp, hp<HT>(Pb, f_Pb));
  }
  // r = -g - H pbar in the solve's precision, for the envs in act
  void rhs(const uint8_t* act) {
    if (mixed())
      launch(k_rhs<float>, NN, 256, NN, layout(), act, (const double*)grad.p, (const double*)pcg_y.p, f_r.p);
    else
      launch(k_rhs<double>, NN, 256, NN, layout(), act, (const double*)grad.p, (const double*)pcg_y.p, pcg_r.p);
  }
  void direction(EnvCtl C) {
    if (mixed())
      launch(k_direction<float>, NN, 256, NN, layout(), C, (const float*)f_x.p, (const double*)pbar.p,
             (const double*)bbox.p, p.p);
    else
      launch(k_direction<double>, NN, 256, NN, layout(), C, (const double*)pcg_x.p, (const double*)pbar.p,
             (const double*)bbox.p, p.p);
  }

  // step set-up for the envs in act: x^t, x~, targets, positions at x^t, trees, friction lag
  void step_setup(const uint8_t* act) {
    launch(k_step_setup_nodes, NN, 256, NN, layout(), ctl(), act, sched_view(), desc.dt, desc.gravity[0],
           desc.gravity[1], desc.gravity[2], (const double*)x.p, (const double*)v.p, xt.p, xtilde.p, xtarget.p);
    launch(k_points, NP, 256, NP, (const int*)pt_node.p, (const double*)pt_xb.p, (const int*)body_node.p,
           (const double*)x.p, ptx.p);
    build_trees();
    n_fr = n_fr_pt = 0;
    cand_src = CAND_FRESH;
    list_ok = false;
    constraint_set(act);
    CK(cudaMemcpyAsync(ptx_t.p, ptx.p, 3 * (size_t)NP * sizeof(double), cudaMemcpyDeviceToDevice, stream));
    if (desc.kappa_adapt) {
      CK(cudaMemsetAsync(e_newton_it.p, 0, E * sizeof(int), stream));  // the evaluations here are iterate 0
      kappa_start(act);  // its evaluations leave the contacts of act at x^t in ct
    }
    fr.ensure(n_ct + 1);
    launch(k_friction_setup, n_ct, 128, n_ct, (const ContactRec*)ct.p, (const double*)ptx.p, (const double*)env_mu.p,
           desc.dhat, (const double*)e_kappa.p, fr.p);
    n_fr = n_ct;
    n_fr_pt = n_ct_pt;
  }

  // CCD step filter on the envs still iterating: swept-box candidates at [x, x + p] (boxes
  // already refit), then additive CCD per candidate pair; each env's alpha_max is the minimum
  // The step filter's candidate list is kept across Newton rounds of a call while it covers the
  // new segments: it is made with boxes grown by an extra slack, and remade only when some
  // primitive's swept box (grown by the plain growth) leaves the box it was listed with.
  DBuf<double> keep_tri, keep_ed, keep_sv;  // boxes the kept list was made with
  bool list_ok = false;
  double swept_slack() const { return reuse_lists() ? 0.25 * desc.dhat : 0.0; }
  bool list_covers(const uint8_t* act) {
    if (!list_ok) return false;
    CK(cudaMemsetAsync(e_count.p + 2, 0, sizeof(int), stream));
    const double r = swept_growth();
    launch(k_swept_inside<3>, NTR, 256, NTR, (const int*)tri_pt.p, (const int*)tri_env.p, act, (const double*)ptx.p,
           (const double*)pte.p, r, (const double*)keep_tri.p, e_count.p + 2);
    launch(k_swept_inside<2>, NED, 256, NED, (const int*)ed_pt.p, (const int*)ed_env.p, act, (const double*)ptx.p,
           (const double*)pte.p, r, (const double*)keep_ed.p, e_count.p + 2);
    launch(k_swept_inside<1>, NSV, 256, NSV, (const int*)sv_pt.p, (const int*)sv_env.p, act, (const double*)ptx.p,
           (const double*)pte.p, r, (const double*)keep_sv.p, e_count.p + 2);
    pwork(IPC_PROF_CCD, (double)NTR * (3 * 48 + 48) + (double)NED * (2 * 48 + 48) + (double)NSV * (48 + 48));
    return read_int(e_count.p + 2) == 0;
  }
  // CCD step filter on the envs in act: swept-box candidates at [x, x + p] (ptx, pte current),
  // then additive CCD per candidate pair of the iterating envs; each env's alpha_max is the
  // minimum
  void ccd_filter(EnvCtl C, const uint8_t* act) {
    const bool keep = reuse_lists();  // the list also serves the narrow phases: sorted per query
    if (keep && list_covers(act)) {
      accd_all(C, keep);
      return;
    }
    if (since_build >= TREE_REBUILD_ROUNDS) {  // refits keep the trees valid; a rebuild keeps them tight
      build_trees();
      since_build = 0;
    }
    const double r = swept_growth() + swept_slack();
    boxes_and_refit(pte.p, r);
    ccd_cnt_pt.ensure(NSV + 1);
    ccd_off_pt.ensure(NSV + 1);
    ccd_cnt_ee.ensure(NED + 1);
    ccd_off_ee.ensure(NED + 1);
    slots_pt.ensure((size_t)NSV * cand_cap() + 1);
    slots_ee.ensure((size_t)NED * cand_cap() + 1);
    ccd_np = ccd_ne = 0;
    list_ok = false;
    CandOut cp{ccd_cnt_pt.p, nullptr, slots_pt.p, overflow.p, cand_cap()};
    launch(k_trav_pt<TRAV_COLLECT>, NSV, 128, NSV, (const int*)sv_pt.p, (const int*)sv_env.p, act,
           (const double*)ptx.p, (const double*)pte.p, r, tree(ttri), (const int*)tri_pt.p, ptinfo(), cp);
    CandOut ce{ccd_cnt_ee.p, nullptr, slots_ee.p, overflow.p, cand_cap()};
    launch(k_trav_ee<TRAV_COLLECT>, NED, 128, NED, (const int*)ed_pt.p, (const int*)ed_env.p, act,
           (const double*)tedge.pbox.p, tree(tedge), ptinfo(), ce);
    scan(ccd_cnt_pt.p, NSV, ccd_off_pt.p, false);
    scan(ccd_cnt_ee.p, NED, ccd_off_ee.p, false);
    int np = 0, ne = 0;
    const bool spilled = read_totals(ccd_off_pt.p + NSV, ccd_off_ee.p + NED, &np, &ne);
    pwork(IPC_PROF_CCD, traversal_bytes(np, ne));
    ccd_np = np;
    ccd_ne = ne;
    ccd_j.ensure(np + ne + 1);
    ccd_q.ensure(np + ne + 1);
    if (np + ne > 0) {
      if (spilled) {
        CandOut fp{nullptr, ccd_off_pt.p, ccd_j.p, overflow.p, 0, ccd_q.p};
        CandOut fe{nullptr, ccd_off_ee.p, ccd_j.p + np, overflow.p, 0, ccd_q.p + np};
        if (keep) {
          launch(k_trav_pt<TRAV_FILL>, NSV, 128, NSV, (const int*)sv_pt.p, (const int*)sv_env.p, act,
                 (const double*)ptx.p, (const double*)pte.p, r, tree(ttri), (const int*)tri_pt.p, ptinfo(), fp);
          launch(k_trav_ee<TRAV_FILL>, NED, 128, NED, (const int*)ed_pt.p, (const int*)ed_env.p, act,
                 (const double*)tedge.pbox.p, tree(tedge), ptinfo(), fe);
        } else {
          launch(k_trav_pt<TRAV_FILLU>, NSV, 128, NSV, (const int*)sv_pt.p, (const int*)sv_env.p, act,
                 (const double*)ptx.p, (const double*)pte.p, r, tree(ttri), (const int*)tri_pt.p, ptinfo(), fp);
          launch(k_trav_ee<TRAV_FILLU>, NED, 128, NED, (const int*)ed_pt.p, (const int*)ed_env.p, act,
                 (const double*)tedge.pbox.p, tree(tedge), ptinfo(), fe);
        }
      } else {
        launch(k_gather_cands, NSV, 256, NSV, cand_cap(), (const int*)ccd_cnt_pt.p, (const int*)slots_pt.p,
               (const int*)ccd_off_pt.p, ccd_j.p, ccd_q.p, keep ? 1 : 0);
        launch(k_gather_cands, NED, 256, NED, cand_cap(), (const int*)ccd_cnt_ee.p, (const int*)slots_ee.p,
               (const int*)ccd_off_ee.p, ccd_j.p + np, ccd_q.p + np, keep ? 1 : 0);
      }
    }
    ccd_rec.ensure(np + ne + 1);
    launch(k_cand_records, np + ne, 256, np, ne, (const int*)ccd_q.p, (const int*)ccd_j.p, (const int*)sv_pt.p,
           (const int*)sv_env.p, (const int*)tri_pt.p, (const int*)ed_pt.p, (const int*)ed_env.p,
           (const double*)ed_rest2.p, ccd_rec.p);
    if (keep) {  // the boxes this list was made with: triangles, edges (the trees' boxes), vertices
      keep_tri.ensure(6 * (size_t)std::max(NTR, 1));
      keep_ed.ensure(6 * (size_t)std::max(NED, 1));
      keep_sv.ensure(6 * (size_t)std::max(NSV, 1));
      if (NTR) CK(cudaMemcpyAsync(keep_tri.p, ttri.pbox.p, 6 * (size_t)NTR * 8, cudaMemcpyDeviceToDevice, stream));
      if (NED) CK(cudaMemcpyAsync(keep_ed.p, tedge.pbox.p, 6 * (size_t)NED * 8, cudaMemcpyDeviceToDevice, stream));
      launch(k_prim_boxes<1>, NSV, 256, NSV, (const int*)sv_pt.p, (const double*)ptx.p, (const double*)pte.p, r,
             keep_sv.p);
      list_ok = true;
    }
    accd_all(C, keep);
  }
  // ACCD of the listed pairs; with a grown list (keep) only the pairs whose plain swept boxes
  // overlap are tested
  void accd_all(EnvCtl C, bool keep) {
    if (ccd_np + ccd_ne == 0) return;
    pwork(IPC_PROF_CCD, (double)(ccd_np + ccd_ne) * (40 + 4 * 48));  // pair record, x and p of 4 points
    launch(k_accd_pairs, ccd_np + ccd_ne, 128, ccd_np + ccd_ne, (const ContactRec*)ccd_rec.p, (const double*)ptx.p,
           (const double*)ptp.p, keep ? (const double*)pte.p : nullptr, C);
  }

  // ------------------------------------------------------------------ time stepping
  // Every env of the scene advances n time steps (fewer where its schedule ends or it fails),
  // each at its own pace (Sec. III-A: every environment keeps its own Newton loop and stopping
  // test). A round runs one Newton iteration of every env inside a step; an env whose Newton
  // loop stopped ends its step in that round and starts its next step in the following round,
  // so the batch stays full while slow envs iterate. Each env goes through exactly the
  // operations of stepping it alone, in the same order: its results do not depend on the batch.
  void run_steps(int n) {
    if (n <= 0) return;
    EnvCtl C = ctl();
    launch(k_env_call_begin, E, 128, E, C, n);
    cand_src = CAND_FRESH;
    list_ok = false;
    const long max_rounds = (long)n * (desc.max_newton + 1) + 1;
    for (long round = 0;; ++round) {
      launch_grid(k_env_round_begin, 1, 256, E, C, e_start.p);
      int cnt[2];
      read_ints(e_count.p, cnt, 2);  // [starting, iterating]
      if (cnt[1] == 0) break;
      if (round > max_rounds) fail_with(IPC_ERR_INTERNAL, "time stepping did not finish");
      if (cnt[0] > 0) step_start(e_start.p);
      newton_round(C);
      // the envs whose Newton loop stopped this round end their step
      launch(k_end_step_nodes, NN, 256, NN, layout(), C, desc.dt, (const double*)x.p, (const double*)xt.p, v.p);
      launch(k_env_end_step, E, 128, E, C);
    }
    cand_src = CAND_FRESH;
    CK(cudaStreamSynchronize(stream));
  }
  // Step set-up of the envs in start: x^t, x~, targets, positions and contacts at x^t, the
  // friction lag. Their contacts come from the previous round's swept candidates, which cover
  // x^t (an env done with a step stays at its last point); in a call's first round, from a
  // traversal (then every iterating env is a starting one).
  int since_build = 0;  // rounds since the trees' topology was last built
  void step_start(const uint8_t* start) {
    launch(k_step_setup_nodes, NN, 256, NN, layout(), ctl(), start, sched_view(), desc.dt, desc.gravity[0],
           desc.gravity[1], desc.gravity[2], (const double*)x.p, (const double*)v.p, xt.p, xtilde.p, xtarget.p);
    launch(k_points, NP, 256, NP, (const int*)pt_node.p, (const double*)pt_xb.p, (const int*)body_node.p,
           (const double*)x.p, ptx.p);
    if (cand_src == CAND_SWEPT) {
      contacts_from_list(start, ccd_np, ccd_ne, ccd_rec.p);
    } else {
      build_trees();
      since_build = 0;
      constraint_set(start);
      if (reuse_lists()) cand_src = CAND_STATIC;  // this round's evaluations are at x^t
    }
    launch(k_copy_points_env, NP, 256, NP, layout(), start, (const double*)ptx.p, ptx_t.p);
    if (desc.kappa_adapt) kappa_start(start);
    friction_merge(start);
  }
  // lagged friction records of the starting envs from their contacts at x^t (ct), merged with
  // the records of the envs that stay inside their step; every sublist stays env-sorted
  void friction_merge(const uint8_t* start) {
    const int n_new = n_ct, n_new_pt = n_ct_pt, n_old = n_fr, n_old_pt = n_fr_pt, tot = n_old + n_new;
    fr_new.ensure(n_new + 1);
    launch(k_friction_setup, n_new, 128, n_new, (const ContactRec*)ct.p, (const double*)ptx.p,
           (const double*)env_mu.p, desc.dhat, (const double*)e_kappa.p, fr_new.p);
    if (tot == 0) {
      n_fr = n_fr_pt = 0;
      return;
    }
    fr_keys.ensure(tot);
    fr_vals.ensure(tot);
    CK(cudaMemsetAsync(e_count.p + 2, 0, 2 * sizeof(int), stream));
    launch(k_fr_keys, tot, 256, n_old, n_old_pt, (const FrictionRec*)fr.p, n_new, n_new_pt,
           (const FrictionRec*)fr_new.p, (const uint8_t*)e_stepping.p, start, fr_keys.p, fr_vals.p, e_count.p + 2);
    radix_sort(fr_keys, fr_vals, fr_keys2, fr_vals2, fr_hist, tot, 34);
    int c[2];
    read_ints(e_count.p + 2, c, 2);  // [kept point-triangle, kept]
    fr_tmp.ensure(c[1] + 1);
    launch(k_fr_gather, c[1], 256, c[1], (const unsigned*)fr_vals.p, n_old, (const FrictionRec*)fr.p,
           (const FrictionRec*)fr_new.p, fr_tmp.p);
    std::swap(fr.p, fr_tmp.p);
    std::swap(fr.n, fr_tmp.n);
    n_fr = c[1];
    n_fr_pt = c[0];
  }
  // one Newton iteration of every iterating env
  void newton_round(EnvCtl C) {
    launch(k_env_iter_begin, E, 128, E, C);
    evaluate<MODE_HESS>(x.p, e_iter.p, e_E0.p);
    launch(k_trace_record, E, 128, E, C, (const double*)e_E0.p, e_trace.p, e_trace_n.p, trace_cap());
    assemble(e_iter.p);
    // kinematic step and the reduced right-hand side -g - H pbar
    launch(k_pbar, NN, 256, NN, layout(), C, (const double*)x.p, (const double*)xtarget.p, pbar.p);
    matvec(e_iter.p, pbar.p, pcg_y.p, part_a.p);
    rhs(e_iter.p);
    pcg(e_iter.p);
    direction(C);
    launch(k_env_converge, E, 128, E, C, desc.dt, desc.newton_tol);
    launch_grid(k_env_cover, 1, 256, E, C, e_cover.p);
    int cnt[2];
    read_ints(e_count.p, cnt, 2);  // [iterating, covered]
    if (cnt[1] > 0) {
      // CCD step filter: swept candidates at [x, x + p] (also for the envs that start their next
      // step next round: the segment starts at their point), ACCD and per-env minimum
      launch(k_points, NP, 256, NP, (const int*)pt_node.p, (const double*)pt_xb.p, (const int*)body_node.p,
             (const double*)x.p, ptx.p);
      launch(k_points, NP, 256, NP, (const int*)pt_node.p, (const double*)pt_xb.p, (const int*)body_node.p,
             (const double*)p.p, ptp.p);
      launch(k_add_vec, 3L * NP, 256, 3L * NP, (const double*)ptx.p, (const double*)ptp.p, pte.p);
      pbeg(IPC_PROF_CCD);
      ccd_filter(C, e_cover.p);
      pend(IPC_PROF_CCD);
      if (reuse_lists()) cand_src = CAND_SWEPT;  // the trials and the next round's points
    }
    if (cnt[0] > 0) {
      // backtracking line search on the envs still iterating
      launch(k_env_ls_begin, E, 128, E, C);
      for (int ls = 0; ls <= desc.max_ls_halvings + 1; ++ls) {
        launch(k_trial, NN, 256, NN, layout(), C, (const double*)x.p, (const double*)p.p, xtrial.p);
        evaluate<MODE_ENERGY>(xtrial.p, e_ls.p, e_Et.p);
        launch(k_env_ls_decide, E, 128, E, C, desc.max_ls_halvings);
        if (count_flags(e_ls.p) == 0) break;
      }
      launch(k_accept, NN, 256, NN, layout(), C, (const double*)xtrial.p, (const double*)xtarget.p, x.p);
    }
    launch(k_env_newton_end, E, 128, E, C, desc.max_newton);
    ++since_build;
  }
  static constexpr int TREE_REBUILD_ROUNDS = 16;

  // ------------------------------------------------------------------ validation / queries
  void invariants(const uint8_t* act, const double* q) {
    CK(cudaMemsetAsync(e_inter.p, 0, E * 8, stream));
    CK(cudaMemsetAsync(e_inv.p, 0, E * 8, stream));
    launch(k_points, NP, 256, NP, (const int*)pt_node.p, (const double*)pt_xb.p, (const int*)body_node.p, q, ptx.p);
    if (!ttri.built || !tedge.built) build_trees();
    boxes_and_refit(nullptr, 0.0);
    launch(k_intersections, NED, 128, NED, (const int*)ed_pt.p, (const int*)ed_env.p, act, (const double*)tedge.pbox.p,
           tree(ttri), (const int*)tri_pt.p, ptinfo(), (const double*)ptx.p, e_inter.p, overflow.p);
    launch(k_inverted, NT, 256, NT, (const int4*)tets.p, (const int*)tet_env.p, act, q, e_inv.p);
    check_overflow();
  }
  void initial_checks() {
    // newly laid-out envs that were never checked: an intersecting start fails the env
    std::vector<uint8_t> sel(E, 0);
    bool any = false;
    for (int li = 0; li < E; ++li)
      if (!envs[ids[li]].checked) {
        sel[li] = 1;
        any = true;
      }
    if (!any) return;
    CK(cudaMemcpyAsync(e_sel.p, sel.data(), E, cudaMemcpyHostToDevice, stream));
    invariants(e_sel.p, x.p);
    std::vector<unsigned long long> inter(E);
    CK(cudaMemcpyAsync(inter.data(), e_inter.p, E * 8, cudaMemcpyDeviceToHost, stream));
    CK(cudaStreamSynchronize(stream));
    std::vector<int> st(E), rs(E);
    CK(cudaMemcpy(st.data(), e_status.p, E * 4, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(rs.data(), e_reason.p, E * 4, cudaMemcpyDeviceToHost));
    for (int li = 0; li < E; ++li) {
      if (!sel[li]) continue;
      envs[ids[li]].checked = true;
      if (inter[li] > 0) {
        st[li] = ST_FAILED;
        rs[li] = FAIL_INIT_INTERSECT;
      }
    }
    CK(cudaMemcpy(e_status.p, st.data(), E * 4, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(e_reason.p, rs.data(), E * 4, cudaMemcpyHostToDevice));
    ttri.built = tedge.built = false;
  }
  int layout_index(int id) {
    for (int li = 0; li < E; ++li)
      if (ids[li] == id) return li;
    fail_with(IPC_ERR_ARG, "unknown env id " + std::to_string(id));
  }
  void select(int li) { launch(k_set_single, E, 128, E, e_sel.p, li); }
  // the bodies of the two sides of each contact of env li at its current DOFs (env-local handles)
  std::vector<int> contact_handles(int li) {
    select(li);
    launch(k_points, NP, 256, NP, (const int*)pt_node.p, (const double*)pt_xb.p, (const int*)body_node.p,
           (const double*)x.p, ptx.p);
    build_trees();
    constraint_set(e_sel.p);
    const int n = n_ct;
    nflag.ensure(2 * (size_t)n + 2);
    launch(k_contact_handles, n, 128, n, (const ContactRec*)ct.p, (const int*)pt_node.p, (const int*)body_node.p,
           (const int*)node_handle.p, nflag.p);
    std::vector<int> v(2 * (size_t)n);
    if (n) CK(cudaMemcpyAsync(v.data(), nflag.p, 2 * n * sizeof(int), cudaMemcpyDeviceToHost, stream));
    CK(cudaStreamSynchronize(stream));
    ttri.built = tedge.built = false;
    return v;
  }
};


// ==================================================================== C ABI
#define API_BEGIN try {
#define API_END                              \
  }                                          \
  catch (const IpcError& err) {              \
    g_err = err.msg;                         \
    return err.st;                           \
  }                                          \
  catch (const std::bad_alloc&) {            \
    g_err = "host allocation failed";        \
    return IPC_ERR_OOM;                      \
  }                                          \
  catch (const std::exception& ex) {         \
    g_err = ex.what();                       \
    return IPC_ERR_INTERNAL;                 \
  }                                          \
  return IPC_OK;

extern "C" {

const char* ipc_last_error(void) { return g_err.c_str(); }
const char* ipc_version(void) { return "b300-ipc 0.1 (sm_103a, FP64)"; }

ipc_status ipc_scene_create(const ipc_scene_desc* desc, ipc_scene** out) {
  API_BEGIN
  if (!desc || !out) fail_with(IPC_ERR_ARG, "null argument");
  if (!(desc->dt > 0) || !(desc->dhat > 0) || !(desc->kappa > 0)) fail_with(IPC_ERR_ARG, "dt, dhat and kappa must be > 0");
  if (desc->precision != IPC_FP64 && desc->precision != IPC_MIXED) fail_with(IPC_ERR_ARG, "unknown precision");
  if (desc->collect_slots < 0 || desc->collect_slots > 4096) fail_with(IPC_ERR_ARG, "collect_slots must be 0..4096");
  {
    int c = desc->pcg_cluster;
    if (c != -1 && c != 0 && c != 1 && c != 2 && c != 4 && c != 8 && c != 16)
      fail_with(IPC_ERR_ARG, "pcg_cluster must be -1, 0, 1, 2, 4, 8 or 16");
  }
  std::unique_ptr<ipc_scene> s(new ipc_scene());
  s->desc = *desc;
  if (s->desc.max_newton <= 0) s->desc.max_newton = 100;
  if (s->desc.max_ls_halvings <= 0) s->desc.max_ls_halvings = 40;
  if (s->desc.max_pcg_iters <= 0) s->desc.max_pcg_iters = 1000;
  s->device = desc->device;
  CK(cudaSetDevice(s->device));
  if (desc->cuda_stream) {
    s->stream = (cudaStream_t)desc->cuda_stream;
  } else {
    CK(cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking));
    s->own_stream = true;
  }
  CK(cudaMallocHost(&s->hpin, 64));
  CK(cudaStreamCreateWithFlags(&s->side, cudaStreamNonBlocking));
  CK(cudaEventCreateWithFlags(&s->fork_ev, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&s->join_ev, cudaEventDisableTiming));
  *out = s.release();
  API_END
}

ipc_status ipc_scene_destroy(ipc_scene* s) {
  API_BEGIN
  if (!s) fail_with(IPC_ERR_ARG, "null scene");
  cudaSetDevice(s->device);
  if (s->stream) cudaStreamSynchronize(s->stream);
  delete s;
  API_END
}

ipc_status ipc_env_estimate_bytes(const ipc_env_desc* env, int32_t precision, uint64_t* bytes) {
  API_BEGIN
  if (!bytes) fail_with(IPC_ERR_ARG, "null output");
  HostEnv h;
  build_env(h, env);
  *bytes = estimate_bytes(h, precision);
  API_END
}

ipc_status ipc_env_add(ipc_scene* s, const ipc_env_desc* env, int32_t* env_id) {
  API_BEGIN
  if (!s || !env) fail_with(IPC_ERR_ARG, "null argument");
  HostEnv h;
  build_env(h, env);
  h.est_bytes = estimate_bytes(h, s->desc.precision);
  if (s->desc.hbm_budget_bytes && s->used_bytes + h.est_bytes > s->desc.hbm_budget_bytes)
    fail_with(IPC_ERR_BUDGET, "env does not fit the HBM budget");
  if (!s->dirty && !s->ids.empty()) {
    CK(cudaSetDevice(s->device));
    s->pull_state();
  }
  h.id = s->next_id++;
  s->used_bytes += h.est_bytes;
  int id = h.id;
  s->envs.emplace(id, std::move(h));
  s->dirty = true;
  if (env_id) *env_id = id;
  API_END
}

ipc_status ipc_env_remove(ipc_scene* s, int32_t env_id) {
  API_BEGIN
  if (!s) fail_with(IPC_ERR_ARG, "null scene");
  auto it = s->envs.find(env_id);
  if (it == s->envs.end()) fail_with(IPC_ERR_ARG, "unknown env id");
  if (!s->dirty && !s->ids.empty()) {
    CK(cudaSetDevice(s->device));
    s->pull_state();
  }
  s->used_bytes -= it->second.est_bytes;
  s->envs.erase(it);
  s->dirty = true;
  API_END
}

ipc_status ipc_step(ipc_scene* s, int32_t n_steps) {
  API_BEGIN
  if (!s || n_steps < 0) fail_with(IPC_ERR_ARG, "bad argument");
  CK(cudaSetDevice(s->device));
  s->commit();
  s->run_steps(n_steps);
  API_END
}

ipc_status ipc_env_set_state(ipc_scene* s, int32_t env_id, const double* x, const double* v, int32_t step) {
  API_BEGIN
  if (!s || !x || !v) fail_with(IPC_ERR_ARG, "null argument");
  CK(cudaSetDevice(s->device));
  s->commit();
  int li = s->layout_index(env_id);
  HostEnv& h = s->envs[env_id];
  if (step < 0 || step > h.n_steps) fail_with(IPC_ERR_ARG, "step out of range");
  size_t o = 3 * (size_t)s->h_node_off[li];
  CK(cudaMemcpyAsync(s->x.p + o, x, h.ndof * 8, cudaMemcpyHostToDevice, s->stream));
  CK(cudaMemcpyAsync(s->v.p + o, v, h.ndof * 8, cudaMemcpyHostToDevice, s->stream));
  int st = step >= h.n_steps ? ST_DONE : ST_ACTIVE, rs = FAIL_NONE;
  CK(cudaMemcpyAsync(s->e_step.p + li, &step, 4, cudaMemcpyHostToDevice, s->stream));
  CK(cudaMemcpyAsync(s->e_status.p + li, &st, 4, cudaMemcpyHostToDevice, s->stream));
  CK(cudaMemcpyAsync(s->e_reason.p + li, &rs, 4, cudaMemcpyHostToDevice, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  API_END
}

ipc_status ipc_eval(ipc_scene* s, int32_t env_id, const double* q, double* energy, double* grad) {
  API_BEGIN
  if (!s || !q || !energy) fail_with(IPC_ERR_ARG, "null argument");
  CK(cudaSetDevice(s->device));
  s->commit();
  int li = s->layout_index(env_id);
  HostEnv& h = s->envs[env_id];
  s->select(li);
  s->step_setup(s->e_sel.p);
  size_t o = 3 * (size_t)s->h_node_off[li];
  CK(cudaMemcpyAsync(s->xtrial.p, s->x.p, 3 * (size_t)s->NN * 8, cudaMemcpyDeviceToDevice, s->stream));
  CK(cudaMemcpyAsync(s->xtrial.p + o, q, h.ndof * 8, cudaMemcpyHostToDevice, s->stream));
  s->evaluate<MODE_GRAD>(s->xtrial.p, s->e_sel.p, s->e_E0.p);
  // gradient: gather with the stencil incidence of this evaluation, at q
  s->stencil_incidence(s->e_sel.p);
  s->launch(k_assemble_grad, s->NN, 256, s->NN, s->layout(), (const uint8_t*)s->e_sel.p, (const double*)s->xtrial.p,
            (const double*)s->xtilde.p, (const int*)s->nt_ptr.p, (const int*)s->nt_src.p, (const double*)s->tet_g.p,
            (const double*)s->body_g.p, (const int*)s->ns_ptr.p, (const int*)s->ns_src.p, (const int*)s->st_pts.p,
            (const double*)s->sg.p, s->grad.p, s->nodeE.p);
  CK(cudaMemcpyAsync(energy, s->e_E0.p + li, 8, cudaMemcpyDeviceToHost, s->stream));
  if (grad) CK(cudaMemcpyAsync(grad, s->grad.p + o, h.ndof * 8, cudaMemcpyDeviceToHost, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  s->ttri.built = s->tedge.built = false;
  API_END
}

ipc_status ipc_newton_direction(ipc_scene* s, int32_t env_id, double* pout) {
  API_BEGIN
  if (!s || !pout) fail_with(IPC_ERR_ARG, "null argument");
  CK(cudaSetDevice(s->device));
  s->commit();
  int li = s->layout_index(env_id);
  HostEnv& h = s->envs[env_id];
  s->select(li);
  s->step_setup(s->e_sel.p);
  CK(cudaMemcpyAsync(s->e_iter.p, s->e_sel.p, s->E, cudaMemcpyDeviceToDevice, s->stream));
  EnvCtl C = s->ctl();
  s->launch(k_env_iter_begin, s->E, 128, s->E, C);
  s->evaluate<MODE_HESS>(s->x.p, s->e_iter.p, s->e_E0.p);
  s->assemble(s->e_iter.p);
  s->launch(k_pbar, s->NN, 256, s->NN, s->layout(), C, (const double*)s->x.p, (const double*)s->xtarget.p, s->pbar.p);
  s->matvec(s->e_iter.p, s->pbar.p, s->pcg_y.p, s->part_a.p);
  s->rhs(s->e_iter.p);
  s->pcg(s->e_iter.p);
  s->direction(C);
  CK(cudaMemcpyAsync(pout, s->p.p + 3 * (size_t)s->h_node_off[li], h.ndof * 8, cudaMemcpyDeviceToHost, s->stream));
  CK(cudaMemsetAsync(s->e_iter.p, 0, s->E, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  s->ttri.built = s->tedge.built = false;
  API_END
}

ipc_status ipc_hessian_apply(ipc_scene* s, int32_t env_id, const double* d, double* y) {
  API_BEGIN
  if (!s || !d || !y) fail_with(IPC_ERR_ARG, "null argument");
  CK(cudaSetDevice(s->device));
  s->commit();
  int li = s->layout_index(env_id);
  HostEnv& h = s->envs[env_id];
  s->select(li);
  s->step_setup(s->e_sel.p);
  EnvCtl C = s->ctl();
  s->launch(k_env_iter_begin, s->E, 128, s->E, C);
  s->evaluate<MODE_HESS>(s->x.p, s->e_sel.p, s->e_E0.p);
  s->assemble(s->e_sel.p);
  size_t o = 3 * (size_t)s->h_node_off[li];
  CK(cudaMemsetAsync(s->pbar.p, 0, 3 * (size_t)s->NN * 8, s->stream));
  CK(cudaMemcpyAsync(s->pbar.p + o, d, h.ndof * 8, cudaMemcpyHostToDevice, s->stream));
  s->matvec(s->e_sel.p, s->pbar.p, s->pcg_y.p, s->part_a.p);
  CK(cudaMemcpyAsync(y, s->pcg_y.p + o, h.ndof * 8, cudaMemcpyDeviceToHost, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  s->ttri.built = s->tedge.built = false;
  API_END
}

static ipc_status copy_out(const void* src, size_t bytes, void* out, size_t out_bytes, size_t* written) {
  if (written) *written = bytes;
  if (out_bytes < bytes || (!out && bytes)) {
    g_err = "output buffer too small";
    return IPC_ERR_ARG;
  }
  if (bytes) std::memcpy(out, src, bytes);
  return IPC_OK;
}

ipc_status ipc_query(ipc_scene* s, int32_t env_id, int32_t kind, void* out, size_t out_bytes, size_t* written) {
  API_BEGIN
  if (!s) fail_with(IPC_ERR_ARG, "null scene");
  CK(cudaSetDevice(s->device));
  s->commit();
  if (kind == IPC_Q_ALL_STATUS) {
    const int E = s->E;
    std::vector<int> st(E), rs(E), sp(E), v(4 * (size_t)E);
    CK(cudaMemcpyAsync(st.data(), s->e_status.p, E * 4, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaMemcpyAsync(rs.data(), s->e_reason.p, E * 4, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaMemcpyAsync(sp.data(), s->e_step.p, E * 4, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    for (int li = 0; li < E; ++li) {
      v[4 * li] = s->ids[li];
      v[4 * li + 1] = st[li];
      v[4 * li + 2] = rs[li];
      v[4 * li + 3] = sp[li];
    }
    return copy_out(v.data(), v.size() * 4, out, out_bytes, written);
  }
  int li = s->layout_index(env_id);
  HostEnv& h = s->envs[env_id];
  size_t o = 3 * (size_t)s->h_node_off[li];
  switch (kind) {
    case IPC_Q_DOFS:
    case IPC_Q_VELOCITIES: {
      std::vector<double> buf(h.ndof);
      CK(cudaMemcpyAsync(buf.data(), (kind == IPC_Q_DOFS ? s->x.p : s->v.p) + o, h.ndof * 8, cudaMemcpyDeviceToHost,
                         s->stream));
      CK(cudaStreamSynchronize(s->stream));
      return copy_out(buf.data(), buf.size() * 8, out, out_bytes, written);
    }
    case IPC_Q_STATUS: {
      int v[4];
      CK(cudaMemcpyAsync(&v[0], s->e_status.p + li, 4, cudaMemcpyDeviceToHost, s->stream));
      CK(cudaMemcpyAsync(&v[1], s->e_reason.p + li, 4, cudaMemcpyDeviceToHost, s->stream));
      CK(cudaMemcpyAsync(&v[3], s->e_step.p + li, 4, cudaMemcpyDeviceToHost, s->stream));
      CK(cudaStreamSynchronize(s->stream));
      v[2] = v[3];
      return copy_out(v, sizeof(v), out, out_bytes, written);
    }
    case IPC_Q_CONTACT_FORCES: {
      s->select(li);
      s->launch(k_points, s->NP, 256, s->NP, (const int*)s->pt_node.p, (const double*)s->pt_xb.p,
                (const int*)s->body_node.p, (const double*)s->x.p, s->ptx.p);
      s->build_trees();
      s->constraint_set(s->e_sel.p);
      const int n = s->n_ct;
      s->tet_vm.ensure((size_t)std::max(n, 1));
      s->launch(k_contact_force, n, 128, n, (const ContactRec*)s->ct.p, (const double*)s->ptx.p, s->desc.dhat,
                (const double*)s->e_kappa.p, s->tet_vm.p);
      std::vector<double> v(std::max(n, 1));
      if (n) CK(cudaMemcpyAsync(v.data(), s->tet_vm.p, n * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
      CK(cudaStreamSynchronize(s->stream));
      s->ttri.built = s->tedge.built = false;
      return copy_out(v.data(), n * sizeof(double), out, out_bytes, written);
    }
    case IPC_Q_CONTACT_HANDLES: {
      std::vector<int> v = s->contact_handles(li);
      return copy_out(v.data(), v.size() * sizeof(int), out, out_bytes, written);
    }
    case IPC_Q_GRASP_RESULT: {
      if (h.obj < 0) fail_with(IPC_ERR_ARG, "the env names no grasped object");
      std::vector<double> xs(h.ndof), vs(h.ndof);
      CK(cudaMemcpyAsync(xs.data(), s->x.p + o, h.ndof * 8, cudaMemcpyDeviceToHost, s->stream));
      CK(cudaMemcpyAsync(vs.data(), s->v.p + o, h.ndof * 8, cudaMemcpyDeviceToHost, s->stream));
      CK(cudaStreamSynchronize(s->stream));
      double com[3] = {0, 0, 0}, vel[3] = {0, 0, 0};
      if (!h.obj_affine) {
        for (int i = 0; i < h.obj_count; ++i)
          for (int k = 0; k < 3; ++k) {
            com[k] += xs[3 * (h.obj_first + i) + k] / h.obj_count;
            vel[k] += vs[3 * (h.obj_first + i) + k] / h.obj_count;
          }
      } else {
        const size_t d = 3 * (size_t)h.nsv_verts + 12 * (size_t)h.obj_first;
        for (int k = 0; k < 3; ++k) {
          com[k] = xs[d + k] + h.obj_xbar[0] * xs[d + 3 + k] + h.obj_xbar[1] * xs[d + 6 + k] + h.obj_xbar[2] * xs[d + 9 + k];
          vel[k] = vs[d + k] + h.obj_xbar[0] * vs[d + 3 + k] + h.obj_xbar[1] * vs[d + 6 + k] + h.obj_xbar[2] * vs[d + 9 + k];
        }
      }
      std::vector<int> hd = s->contact_handles(li);
      bool touch = false;
      for (size_t c = 0; c + 1 < hd.size(); c += 2) touch |= (hd[c] == h.obj) != (hd[c + 1] == h.obj);
      const double step = s->desc.dt * std::sqrt(vel[0] * vel[0] + vel[1] * vel[1] + vel[2] * vel[2]);
      double r[4] = {touch ? 1.0 : 0.0, step, (touch && step < s->desc.eps_v * s->desc.dt) ? 1.0 : 0.0,
                     com[2] - h.obj_com0[2]};
      return copy_out(r, sizeof(r), out, out_bytes, written);
    }
    case IPC_Q_FRICTION_FORCES: {
      const int n = s->n_fr;
      s->launch(k_points, s->NP, 256, s->NP, (const int*)s->pt_node.p, (const double*)s->pt_xb.p,
                (const int*)s->body_node.p, (const double*)s->x.p, s->ptx.p);
      s->tet_vm.ensure((size_t)std::max(n, 1));
      s->launch(k_friction_force, n, 128, n, (const FrictionRec*)s->fr.p, (const double*)s->ptx.p,
                (const double*)s->ptx_t.p, s->desc.eps_v * s->desc.dt, s->tet_vm.p);
      std::vector<double> v(std::max(n, 1));
      std::vector<FrictionRec> recs(std::max(n, 1));
      if (n) {
        CK(cudaMemcpyAsync(v.data(), s->tet_vm.p, n * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
        CK(cudaMemcpyAsync(recs.data(), s->fr.p, n * sizeof(FrictionRec), cudaMemcpyDeviceToHost, s->stream));
      }
      CK(cudaStreamSynchronize(s->stream));
      std::vector<double> mine;  // this env's records, in list order (point-triangle, then edge-edge)
      for (int k = 0; k < n; ++k)
        if (recs[k].env == li) mine.push_back(v[k]);
      return copy_out(mine.data(), mine.size() * sizeof(double), out, out_bytes, written);
    }
    case IPC_Q_TET_STRESS: {
      const int t0 = s->h_tet_off[li], nt = s->h_tet_off[li + 1] - t0;
      s->select(li);
      s->tet_vm.ensure((size_t)std::max(s->NT, 1));
      s->launch(k_tet_von_mises, s->NT, 256, s->NT, (const int4*)s->tets.p, (const double*)s->tet_prm.p,
                (const int*)s->tet_env.p, (const uint8_t*)s->e_sel.p, (const double*)s->x.p, s->tet_vm.p);
      std::vector<double> v(std::max(nt, 1));
      if (nt) CK(cudaMemcpyAsync(v.data(), s->tet_vm.p + t0, nt * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
      CK(cudaStreamSynchronize(s->stream));
      return copy_out(v.data(), nt * sizeof(double), out, out_bytes, written);
    }
    case IPC_Q_KAPPA: {
      double v = 0.0;
      CK(cudaMemcpyAsync(&v, s->e_kappa.p + li, 8, cudaMemcpyDeviceToHost, s->stream));
      CK(cudaStreamSynchronize(s->stream));
      return copy_out(&v, sizeof(v), out, out_bytes, written);
    }
    case IPC_Q_STATS: {
      long long v[5];
      CK(cudaMemcpyAsync(v, s->e_stats.p + 5 * li, 40, cudaMemcpyDeviceToHost, s->stream));
      CK(cudaStreamSynchronize(s->stream));
      return copy_out(v, sizeof(v), out, out_bytes, written);
    }
    case IPC_Q_SCENE_COUNTERS: {
      std::vector<int> ptr(s->NN + 1);
      CK(cudaMemcpy(ptr.data(), s->ns_ptr.p, (s->NN + 1) * 4, cudaMemcpyDeviceToHost));
      long long mx = 0;
      for (int i = 0; i < s->NN; ++i) mx = std::max(mx, (long long)(ptr[i + 1] - ptr[i]));
      long long v[12] = {s->n_ct, s->n_ct_pt, s->n_fr, s->n_inc, mx, (long long)s->n_pt + s->n_ee, s->NNZB,
                         s->sell_nval / 288, s->pcg_C, s->max_env_slices, s->n_jt, s->spills};
      return copy_out(v, sizeof(v), out, out_bytes, written);
    }
    case IPC_Q_ENERGY_TRACE: {
      int n = 0;
      CK(cudaMemcpyAsync(&n, s->e_trace_n.p + li, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
      CK(cudaStreamSynchronize(s->stream));
      std::vector<double> buf(std::max(n, 0));
      if (n > 0)
        CK(cudaMemcpyAsync(buf.data(), s->e_trace.p + (size_t)li * s->trace_cap(), n * sizeof(double),
                           cudaMemcpyDeviceToHost, s->stream));
      CK(cudaStreamSynchronize(s->stream));
      return copy_out(buf.data(), buf.size() * 8, out, out_bytes, written);
    }
    case IPC_Q_SIZES: {
      long long v[8] = {h.ndof, (long long)h.n_surf_pts, (long long)h.sv.size(), (long long)h.edges.size() / 2,
                        (long long)h.tris.size() / 3, h.ntets, h.nbodies, h.n_steps};
      return copy_out(v, sizeof(v), out, out_bytes, written);
    }
    case IPC_Q_POINTS: {
      s->launch(k_points, s->NP, 256, s->NP, (const int*)s->pt_node.p, (const double*)s->pt_xb.p,
                (const int*)s->body_node.p, (const double*)s->x.p, s->ptx.p);
      int np = h.n_surf_pts;
      std::vector<double> buf(3 * (size_t)np);
      CK(cudaMemcpyAsync(buf.data(), s->ptx.p + 3 * (size_t)s->h_pt_off[li], buf.size() * 8, cudaMemcpyDeviceToHost,
                         s->stream));
      CK(cudaStreamSynchronize(s->stream));
      return copy_out(buf.data(), buf.size() * 8, out, out_bytes, written);
    }
    case IPC_Q_INTERSECTIONS: {
      s->select(li);
      s->invariants(s->e_sel.p, s->x.p);
      long long v[2];
      CK(cudaMemcpyAsync(&v[0], s->e_inter.p + li, 8, cudaMemcpyDeviceToHost, s->stream));
      CK(cudaMemcpyAsync(&v[1], s->e_inv.p + li, 8, cudaMemcpyDeviceToHost, s->stream));
      CK(cudaStreamSynchronize(s->stream));
      s->ttri.built = s->tedge.built = false;
      return copy_out(v, sizeof(v), out, out_bytes, written);
    }
    case IPC_Q_CANDIDATES:
    case IPC_Q_CONTACTS: {
      s->select(li);
      s->launch(k_points, s->NP, 256, s->NP, (const int*)s->pt_node.p, (const double*)s->pt_xb.p,
                (const int*)s->body_node.p, (const double*)s->x.p, s->ptx.p);
      s->build_trees();
      s->constraint_set(s->e_sel.p);
      int nc = s->n_pt + s->n_ee;
      std::vector<int> cj(nc), offp(s->NSV + 1), offe(s->NED + 1);
      std::vector<ContactRec> ct(s->n_ct);
      if (nc) CK(cudaMemcpyAsync(cj.data(), s->cand_j.p, nc * 4, cudaMemcpyDeviceToHost, s->stream));
      CK(cudaMemcpyAsync(offp.data(), s->off_pt.p, (s->NSV + 1) * 4, cudaMemcpyDeviceToHost, s->stream));
      CK(cudaMemcpyAsync(offe.data(), s->off_ee.p, (s->NED + 1) * 4, cudaMemcpyDeviceToHost, s->stream));
      if (s->n_ct) CK(cudaMemcpyAsync(ct.data(), s->ct.p, s->n_ct * sizeof(ContactRec), cudaMemcpyDeviceToHost, s->stream));
      CK(cudaStreamSynchronize(s->stream));
      s->ttri.built = s->tedge.built = false;
      int sv0 = s->h_sv_off[li], ed0 = s->h_ed_off[li], tr0 = s->h_tri_off[li];
      std::vector<int> rows;
      if (kind == IPC_Q_CANDIDATES) {
        for (int q = s->h_sv_off[li]; q < s->h_sv_off[li + 1]; ++q)
          for (int k = offp[q]; k < offp[q + 1]; ++k) rows.insert(rows.end(), {0, q - sv0, cj[k] - tr0});
        for (int q = s->h_ed_off[li]; q < s->h_ed_off[li + 1]; ++q)
          for (int k = offe[q]; k < offe[q + 1]; ++k) rows.insert(rows.end(), {1, q - ed0, cj[s->n_pt + k] - ed0});
      } else {
        for (auto& c : ct) {
          int i = c.cand;
          if (c.kind == 0) {
            int q = (int)(std::upper_bound(offp.begin(), offp.end(), i) - offp.begin()) - 1;
            while (q + 1 <= s->NSV && offp[q + 1] <= i) ++q;
            rows.insert(rows.end(), {0, q - sv0, cj[i] - tr0, c.type});
          } else {
            int k = i - s->n_pt;
            int q = (int)(std::upper_bound(offe.begin(), offe.end(), k) - offe.begin()) - 1;
            rows.insert(rows.end(), {1, q - ed0, cj[i] - ed0, c.type});
          }
        }
      }
      return copy_out(rows.data(), rows.size() * 4, out, out_bytes, written);
    }
    default:
      fail_with(IPC_ERR_ARG, "unknown query kind");
  }
  API_END
}

ipc_status ipc_set_next_targets(ipc_scene* s, const double* targets, size_t bytes) {
  API_BEGIN
  if (!s || !targets) fail_with(IPC_ERR_ARG, "null argument");
  CK(cudaSetDevice(s->device));
  s->commit();
  std::vector<int> st(s->E), sp(s->E);
  CK(cudaMemcpyAsync(st.data(), s->e_status.p, s->E * 4, cudaMemcpyDeviceToHost, s->stream));
  CK(cudaMemcpyAsync(sp.data(), s->e_step.p, s->E * 4, cudaMemcpyDeviceToHost, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  size_t need = 0;
  for (int li = 0; li < s->E; ++li)
    if (st[li] == ST_ACTIVE) need += 12 * 8 * (s->envs[s->ids[li]].soft.size() + s->envs[s->ids[li]].aff.size());
  if (bytes != need) fail_with(IPC_ERR_ARG, "targets: expected " + std::to_string(need) + " bytes");
  size_t src = 0;
  long so = 0;
  for (int li = 0; li < s->E; ++li) {
    HostEnv& h = s->envs[s->ids[li]];
    int nhb = (int)(h.soft.size() + h.aff.size());
    if (st[li] == ST_ACTIVE) {
      size_t dst = so + (size_t)sp[li] * nhb * 12;
      CK(cudaMemcpyAsync(s->sched.p + dst, targets + src, nhb * 12 * 8, cudaMemcpyHostToDevice, s->stream));
      src += nhb * 12;
    }
    so += (long)h.targets.size();
  }
  API_END
}

ipc_status ipc_env_set_targets(ipc_scene* s, int32_t env_id, int32_t first_step, int32_t n_steps,
                               const double* targets) {
  API_BEGIN
  if (!s || !targets || n_steps < 0) fail_with(IPC_ERR_ARG, "bad argument");
  auto it = s->envs.find(env_id);
  if (it == s->envs.end()) fail_with(IPC_ERR_ARG, "unknown env id " + std::to_string(env_id));
  HostEnv& h = it->second;
  if (first_step < 0 || first_step + n_steps > h.n_steps) fail_with(IPC_ERR_ARG, "steps out of the schedule");
  const size_t nh = h.soft.size() + h.aff.size(), row = nh * 12;
  std::copy(targets, targets + (size_t)n_steps * row, h.targets.begin() + (size_t)first_step * row);
  if (!s->dirty) {  // the laid-out schedule too (a relayout re-uploads the host copy)
    CK(cudaSetDevice(s->device));
    long so = 0;
    for (int li = 0; li < s->E; ++li) {
      HostEnv& o = s->envs[s->ids[li]];
      if (s->ids[li] == env_id) {
        if (n_steps)
          CK(cudaMemcpyAsync(s->sched.p + so + (size_t)first_step * row, targets, (size_t)n_steps * row * 8,
                             cudaMemcpyHostToDevice, s->stream));
        CK(cudaStreamSynchronize(s->stream));
        break;
      }
      so += (long)o.targets.size();
    }
  }
  API_END
}

ipc_status ipc_get_all_dofs(ipc_scene* s, double* out, size_t out_bytes, size_t* written) {
  API_BEGIN
  if (!s) fail_with(IPC_ERR_ARG, "null scene");
  CK(cudaSetDevice(s->device));
  s->commit();
  size_t bytes = 3 * (size_t)s->NN * 8;
  if (written) *written = bytes;
  if (out_bytes < bytes || !out) fail_with(IPC_ERR_ARG, "output buffer too small");
  CK(cudaMemcpyAsync(out, s->x.p, bytes, cudaMemcpyDeviceToHost, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  API_END
}

ipc_status ipc_profile_enable(ipc_scene* s, int32_t on) {
  API_BEGIN
  if (!s) fail_with(IPC_ERR_ARG, "null scene");
  CK(cudaSetDevice(s->device));
  CK(cudaStreamSynchronize(s->stream));
  for (int f = 0; f < IPC_PROF_COUNT; ++f) {
    for (auto& pr : s->prof_ev[f]) {
      s->ev_pool.push_back(pr.first);
      s->ev_pool.push_back(pr.second);
    }
    s->prof_ev[f].clear();
    s->prof_launches[f] = 0;
    s->prof_graph_ms[f] = 0.0;
    s->prof_host_work[f] = 0.0;
  }
  s->prof_units.ensure(IPC_PROF_COUNT);
  s->prof_units.zero(s->stream, IPC_PROF_COUNT);
  CK(cudaStreamSynchronize(s->stream));
  if (s->idle_from) s->ev_pool.push_back(s->idle_from);
  s->idle_from = nullptr;  // a wait before profiling started is not counted
  s->prof_on = on != 0;
  API_END
}

ipc_status ipc_profile_read(ipc_scene* s, int32_t fam, int64_t* launches, double* ms, double* work) {
  API_BEGIN
  if (!s || fam < 0 || fam >= IPC_PROF_COUNT) fail_with(IPC_ERR_ARG, "bad argument");
  CK(cudaSetDevice(s->device));
  CK(cudaStreamSynchronize(s->stream));
  const int tf = fam == IPC_PROF_PCG_FLOPS ? IPC_PROF_PCG_SOLVE : fam;  // a work-only family
  double t = s->prof_graph_ms[tf];
  for (auto& pr : s->prof_ev[tf]) {
    float m = 0.f;
    CK(cudaEventElapsedTime(&m, pr.first, pr.second));
    t += m;
  }
  unsigned long long u[IPC_PROF_COUNT] = {0};
  if (s->prof_units.p) CK(cudaMemcpy(u, s->prof_units.p, sizeof(u), cudaMemcpyDeviceToHost));
  if (launches) *launches = s->prof_launches[tf];
  if (ms) *ms = t;
  if (work) *work = (double)u[fam] + s->prof_host_work[fam];
  API_END
}

// ---- allocation-free Neo-Hookean energy: scratch in a file-scope device array
static __device__ __align__(256) double g_noalloc_tet_energy[IPC_NOALLOC_MAX_TETS];
static double* g_noalloc_ptr[256] = {nullptr};
static std::mutex g_noalloc_mutex;

// The group bound g as the kernels use it: the caller's offset clamped to [0, n_tets], so that
// every access stays inside the tets and the scratch array whatever the offsets hold, and the
// energy kernel and the group sum agree on which tets belong to which group.
__device__ __forceinline__ int noalloc_bound(const int* __restrict__ goff, int g, int n_tets) {
  return min(max(goff[g], 0), n_tets);
}
// per-tet energy into the scratch array (same tet_energy as the scene path); the group of a tet
// is found by binary search in the clamped offsets; an inverted tet flags its group. Tets outside
// [goff[0], goff[n_groups]) belong to no group: neither flagged nor summed. The tet's four node
// indices are read as scalars (the caller's pointer need only be int-aligned).
__global__ void k_noalloc_tet_energy(int n_tets, const int* __restrict__ tets, const double* __restrict__ prm,
                                     const double* __restrict__ x, int n_groups, const int* __restrict__ goff, double h2,
                                     double* __restrict__ tE, int* __restrict__ inverted) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_tets) return;
  tE[t] = 0.0;
  if (t < noalloc_bound(goff, 0, n_tets) || t >= noalloc_bound(goff, n_groups, n_tets)) return;
  int lo = 0, hi = n_groups - 1;  // last group g with bound(g) <= t
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (noalloc_bound(goff, mid, n_tets) <= t) lo = mid;
    else hi = mid - 1;
  }
  const int* T = tets + 4L * t;
  const double* P = prm + 12L * t;
  double F[9], cof[9], J;
  double En = tet_energy(ld3(x, T[0]), ld3(x, T[1]), ld3(x, T[2]), ld3(x, T[3]), P, P[10], P[11], h2 * P[9], F, cof, &J);
  if (!(J > 0.0)) {
    inverted[lo] = 1;
    En = 0.0;
  }
  tE[t] = En;
}
__global__ void k_noalloc_clear(int n, int* __restrict__ a) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] = 0;
}
// one block per group over its clamped range, the same strided fixed-order block reduction as
// the scene path
__global__ void k_noalloc_group_sum(int n_groups, int n_tets, const int* __restrict__ goff,
                                    const double* __restrict__ tE, double* __restrict__ out) {
  __shared__ double sh[256];
  int g = blockIdx.x;
  if (g >= n_groups) return;
  const int b0 = noalloc_bound(goff, g, n_tets), b1 = noalloc_bound(goff, g + 1, n_tets);
  double s = 0.0;
  for (int i = b0 + threadIdx.x; i < b1; i += blockDim.x) s += tE[i];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) out[g] = s;
}

ipc_status ipc_elastic_energy_noalloc(int32_t n_tets, const int32_t* tets, const double* tet_params, const double* x,
                                      int32_t n_groups, const int32_t* group_offsets, double h2, double* energy,
                                      int32_t* inverted, void* stream) {
  API_BEGIN
  if (n_tets < 0 || n_groups <= 0 || !group_offsets || !energy || !inverted || (n_tets > 0 && (!tets || !tet_params || !x)))
    fail_with(IPC_ERR_ARG, "ipc_elastic_energy_noalloc: null pointer or bad count");
  if (n_tets > IPC_NOALLOC_MAX_TETS)
    fail_with(IPC_ERR_ARG, "ipc_elastic_energy_noalloc: " + std::to_string(n_tets) + " tets exceed the maximum of " +
                               std::to_string(IPC_NOALLOC_MAX_TETS));
  if (n_groups > IPC_NOALLOC_MAX_GROUPS)
    fail_with(IPC_ERR_ARG, "ipc_elastic_energy_noalloc: more than " + std::to_string(IPC_NOALLOC_MAX_GROUPS) + " groups");
  auto misaligned = [](const void* ptr, size_t a) { return ((uintptr_t)ptr) % a != 0; };
  if (misaligned(tets, 4) || misaligned(group_offsets, 4) || misaligned(inverted, 4) || misaligned(tet_params, 8) ||
      misaligned(x, 8) || misaligned(energy, 8))
    fail_with(IPC_ERR_ARG, "ipc_elastic_energy_noalloc: a pointer is not aligned to its element type");
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 256) fail_with(IPC_ERR_ARG, "ipc_elastic_energy_noalloc: device ordinal out of range");
  double* scratch;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {  // once per device, with that device current
      void* p = nullptr;
      CK(cudaGetSymbolAddress(&p, g_noalloc_tet_energy));
      g_noalloc_ptr[dev] = (double*)p;
    }
    scratch = g_noalloc_ptr[dev];
  }
  cudaStream_t st = (cudaStream_t)stream;
  k_noalloc_clear<<<(n_groups + 255) / 256, 256, 0, st>>>(n_groups, inverted);
  CK(cudaGetLastError());
  if (n_tets > 0) {
    k_noalloc_tet_energy<<<(n_tets + 127) / 128, 128, 0, st>>>(n_tets, tets, tet_params, x, n_groups, group_offsets,
                                                               h2, scratch, inverted);
    CK(cudaGetLastError());
  }
  k_noalloc_group_sum<<<n_groups, 256, 0, st>>>(n_groups, n_tets, group_offsets, scratch, energy);
  CK(cudaGetLastError());
  API_END
}

ipc_status ipc_launch_count(ipc_scene* s, int64_t* count) {
  API_BEGIN
  if (!s || !count) fail_with(IPC_ERR_ARG, "null argument");
  *count = s->launches;
  API_END
}

}  // extern "C"
