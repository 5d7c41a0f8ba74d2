// Per-node, per-env and per-candidate control kernels of the batched Newton loop: step
// set-up, kinematic targets, Newton direction bookkeeping, convergence, line search, candidate
// generation, narrow phase, CCD step filter, friction lagging and stencil incidence.
#pragma once
#include "common.cuh"
#include "geometry.cuh"
#include "lbvh.cuh"
#include "energy.cuh"
#include "solver.cuh"

enum { ST_ACTIVE = 0, ST_DONE = 1, ST_FAILED = 2 };
enum { FAIL_NONE = 0, FAIL_NEWTON = 1, FAIL_LINESEARCH = 2, FAIL_NAN = 3, FAIL_INIT_INTERSECT = 4, FAIL_INTERNAL = 5 };
enum { STAT_NEWTON = 0, STAT_PCG = 1, STAT_LS = 2, STAT_STEPS = 3, STAT_ACCD = 4 };

struct EnvCtl {
  int* status;
  int* reason;
  int* step;
  int* nsteps;
  uint8_t* stepping;   // stepping in the current time step
  uint8_t* iter;       // Newton still iterating
  uint8_t* ls;         // line search pending
  uint8_t* accept;     // accepted a trial this iteration
  int* constrained;    // kinematic DOFs not at target
  int* bad;            // some tet inverted at the trial
  int* nanp;           // non-finite Newton direction
  int* halv;
  int* newton_it;
  double* E0;
  double* Et;
  double* alpha;
  unsigned long long* alpha_bits;
  unsigned long long* pnorm_bits;
  long long* stats;    // 5 per env
  int* flag_count;
  int* rem;            // time steps left in the current ipc_step call
};

struct Sched {
  const double* targets;
  const uint8_t* gravity;
  const long* sched_off;  // doubles
  const int* grav_off;
  const int* nh;          // handles per env
  const int* node_handle; // env-local handle of each node (soft: its body; body nodes: n_soft + b)
  const double* X0;
};

// x^t = x; predicted x~ = (x^t + h v) + h^2 g (gravity only on soft nodes and body translations);
// kinematic targets of this step.
__global__ void k_step_setup_nodes(int n_nodes, Layout L, EnvCtl C, const uint8_t* __restrict__ act, Sched S, double h,
                                   double gx, double gy, double gz, const double* __restrict__ x,
                                   const double* __restrict__ v, double* __restrict__ xt, double* __restrict__ xtilde,
                                   double* __restrict__ xtarget) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_nodes) return;
  int e = L.node_env[i];
  if (!act[e]) return;
  int step = C.step[e];
  if (step >= C.nsteps[e]) step = C.nsteps[e] - 1;
  // gravity of this step: 0 none, 1 the scene's vector, 2..7 its magnitude along +x, -x, +y,
  // -y, +z, -z (the axis-aligned phases of the grasp evaluation protocol)
  const int code = S.gravity[S.grav_off[e] + step];
  double hh = code ? h * h : 0.0;
  int b = L.node_body[i];
  bool grav_node = b < 0 || (i - L.body_node[b]) == 0;
  double g[3] = {gx, gy, gz};
  if (code >= 2) {
    const double gm = sqrt(gx * gx + gy * gy + gz * gz);
    g[0] = g[1] = g[2] = 0.0;
    g[(code - 2) / 2] = (code % 2 == 0) ? gm : -gm;
  }
  for (int k = 0; k < 3; ++k) {
    double xv = x[3L * i + k];
    xt[3L * i + k] = xv;
    double r = xv + h * v[3L * i + k];
    if (grav_node) r = r + hh * g[k];
    xtilde[3L * i + k] = r;
  }
  const double* T = S.targets + S.sched_off[e] + ((long)step * S.nh[e] + S.node_handle[i]) * 12;
  if (b < 0) {
    if (L.node_kin[i]) {
      const double* X0 = S.X0 + 3L * i;
      for (int k = 0; k < 3; ++k) {
        double r = add_mul_rn(T[k], X0[0], T[3 + k]);
        r = add_mul_rn(r, X0[1], T[6 + k]);
        r = add_mul_rn(r, X0[2], T[9 + k]);
        xtarget[3L * i + k] = r;
      }
    }
  } else {  // every body: kinematic bodies follow it, PD-driven bodies are pulled toward it
    int blk = i - L.body_node[b];
    for (int k = 0; k < 3; ++k) xtarget[3L * i + k] = T[3 * blk + k];
  }
}

// kinematic part of the Newton step: pbar = target - x on kinematic nodes, 0 elsewhere
__global__ void k_pbar(int n_nodes, Layout L, EnvCtl C, const double* __restrict__ x, const double* __restrict__ xtarget,
                       double* __restrict__ pbar) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_nodes) return;
  int e = L.node_env[i];
  if (!C.iter[e]) return;
  int b = L.node_body[i];
  bool kin = b < 0 ? L.node_kin[i] : L.body_kin[b];
  d3 p = mk3(0, 0, 0);
  if (kin) {
    p = ld3(xtarget, i) - ld3(x, i);
    if (p.x != 0.0 || p.y != 0.0 || p.z != 0.0) atomicOr(&C.constrained[e], 1);
  }
  st3(pbar, i, p);
}

// r = -g - y on free DOFs, 0 on kinematic ones (formed in FP64, stored in the solve's type VT)
template <class VT>
__global__ void k_rhs(int n_nodes, Layout L, const uint8_t* __restrict__ act, const double* __restrict__ g,
                      const double* __restrict__ y, VT* __restrict__ r) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_nodes) return;
  if (!act[L.node_env[i]]) return;
  int b = L.node_body[i];
  bool kin = b < 0 ? L.node_kin[i] : L.body_kin[b];
  for (int k = 0; k < 3; ++k) r[3L * i + k] = kin ? VT(0) : VT(-g[3L * i + k] - y[3L * i + k]);
}

// p = delta (free) or pbar (kinematic); infinity norm in world space of the free part
template <class VT>
__global__ void k_direction(int n_nodes, Layout L, EnvCtl C, const VT* __restrict__ delta,
                            const double* __restrict__ pbar, const double* __restrict__ bbox, double* __restrict__ p) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_nodes) return;
  int e = L.node_env[i];
  if (!C.iter[e]) return;
  int b = L.node_body[i];
  bool kin = b < 0 ? L.node_kin[i] : L.body_kin[b];
  d3 v = kin ? ld3(pbar, i) : mk3(double(delta[3L * i]), double(delta[3L * i + 1]), double(delta[3L * i + 2]));
  st3(p, i, v);
  if (!(isfinite(v.x) && isfinite(v.y) && isfinite(v.z))) atomicOr(&C.nanp[e], 1);
  if (kin) return;
  double m = 0.0;
  if (b < 0) {
    m = fmax(fabs(v.x), fmax(fabs(v.y), fabs(v.z)));
  } else if (i == L.body_node[b]) {
    // max over the 8 rest bounding-box corners of |J(corner) p_q|_inf
    long base = i;
    d3 pq[4];
    for (int k = 0; k < 4; ++k)
      pq[k] = mk3(double(delta[3 * (base + k)]), double(delta[3 * (base + k) + 1]), double(delta[3 * (base + k) + 2]));
    const double* B = bbox + 6L * b;
    for (int c = 0; c < 8; ++c) {
      double xb0 = (c & 1) ? B[3] : B[0], xb1 = (c & 2) ? B[4] : B[1], xb2 = (c & 4) ? B[5] : B[2];
      for (int k = 0; k < 3; ++k) {
        double r = add_mul_rn(comp(pq[0], k), xb0, comp(pq[1], k));
        r = add_mul_rn(r, xb1, comp(pq[2], k));
        r = add_mul_rn(r, xb2, comp(pq[3], k));
        m = fmax(m, fabs(r));
      }
    }
  } else {
    return;
  }
  if (isfinite(m)) atomic_max_pos(&C.pnorm_bits[e], m);
}

// trial point x + alpha p of the envs still searching; an env that has accepted keeps its
// accepted trial point while the others go on halving
__global__ void k_trial(int n_nodes, Layout L, EnvCtl C, const double* __restrict__ x, const double* __restrict__ p,
                        double* __restrict__ xtr) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_nodes) return;
  int e = L.node_env[i];
  if (!C.ls[e]) return;
  const double a = C.alpha[e];
  for (int k = 0; k < 3; ++k) xtr[3L * i + k] = x[3L * i + k] + a * p[3L * i + k];
}

__global__ void k_accept(int n_nodes, Layout L, EnvCtl C, const double* __restrict__ xtr,
                         const double* __restrict__ xtarget, double* __restrict__ x) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_nodes) return;
  int e = L.node_env[i];
  if (!C.accept[e]) return;
  int b = L.node_body[i];
  bool kin = b < 0 ? L.node_kin[i] : L.body_kin[b];
  bool snap = kin && C.constrained[e] && C.alpha[e] == 1.0;
  for (int k = 0; k < 3; ++k) x[3L * i + k] = snap ? xtarget[3L * i + k] : xtr[3L * i + k];
}

__global__ void k_end_step_nodes(int n_nodes, Layout L, EnvCtl C, double h, const double* __restrict__ x,
                                 const double* __restrict__ xt, double* __restrict__ v) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_nodes) return;
  int e = L.node_env[i];
  if (!C.stepping[e] || C.iter[e] || C.status[e] != ST_ACTIVE) return;
  for (int k = 0; k < 3; ++k) v[3L * i + k] = (x[3L * i + k] - xt[3L * i + k]) / h;
}

// ---------------------------------------------------------------- per-env control
// Continuous stepping: within one ipc_step call every env runs its time steps at its own pace.
// A round is one Newton iteration of every env inside a step; an env whose Newton loop stopped
// ends its step in that round and starts the next one in the following round.
__global__ void k_env_call_begin(int n_env, EnvCtl C, int n_steps) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_env) return;
  C.rem[e] = n_steps;
  C.stepping[e] = 0;
  C.iter[e] = 0;
}
// envs that start a time step this round (not inside one, active, schedule and call budget
// left); counts of [starting, iterating] envs go to C.flag_count[0..1]
__global__ void k_env_round_begin(int n_env, EnvCtl C, uint8_t* __restrict__ start) {
  __shared__ int cnt[2];
  if (threadIdx.x < 2) cnt[threadIdx.x] = 0;
  __syncthreads();
  for (int e = threadIdx.x; e < n_env; e += blockDim.x) {
    bool go = !C.stepping[e] && C.status[e] == ST_ACTIVE && C.step[e] < C.nsteps[e] && C.rem[e] > 0;
    start[e] = go;
    if (go) {
      C.stepping[e] = 1;
      C.iter[e] = 1;
      C.newton_it[e] = 0;
      atomicAdd(&cnt[0], 1);
    }
    if (C.iter[e]) atomicAdd(&cnt[1], 1);
  }
  __syncthreads();
  if (threadIdx.x < 2) C.flag_count[threadIdx.x] = cnt[threadIdx.x];
}
// after the convergence test: envs whose contacts the next round takes from this round's
// swept candidates (still iterating, or done with this step and starting another in this call);
// counts of [iterating, covered] envs go to C.flag_count[0..1]
__global__ void k_env_cover(int n_env, EnvCtl C, uint8_t* __restrict__ cover) {
  __shared__ int cnt[2];
  if (threadIdx.x < 2) cnt[threadIdx.x] = 0;
  __syncthreads();
  for (int e = threadIdx.x; e < n_env; e += blockDim.x) {
    bool next = C.stepping[e] && !C.iter[e] && C.status[e] == ST_ACTIVE && C.rem[e] > 1 && C.step[e] + 1 < C.nsteps[e];
    bool c = C.iter[e] || next;
    cover[e] = c;
    if (C.iter[e]) atomicAdd(&cnt[0], 1);
    if (c) atomicAdd(&cnt[1], 1);
  }
  __syncthreads();
  if (threadIdx.x < 2) C.flag_count[threadIdx.x] = cnt[threadIdx.x];
}
__global__ void k_env_iter_begin(int n_env, EnvCtl C) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_env) return;
  C.constrained[e] = 0;
  C.nanp[e] = 0;
  C.bad[e] = 0;
  C.pnorm_bits[e] = 0ull;
  C.accept[e] = 0;
}
// after the Newton solve: failure on non-finite values, convergence test, CCD start value
__global__ void k_env_converge(int n_env, EnvCtl C, double h, double tol) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_env) return;
  if (!C.iter[e]) return;
  C.stats[5 * e + STAT_NEWTON] += 1;
  if (C.nanp[e] || !isfinite(C.E0[e]) || C.bad[e]) {
    C.iter[e] = 0;
    C.status[e] = ST_FAILED;
    C.reason[e] = FAIL_NAN;
    return;
  }
  double pn = bits_to_double(C.pnorm_bits[e]);
  if (!C.constrained[e] && pn / h < tol) {
    C.iter[e] = 0;  // converged: frozen for the rest of this step
    return;
  }
  C.alpha_bits[e] = (unsigned long long)__double_as_longlong(1.0);
}
__global__ void k_env_ls_begin(int n_env, EnvCtl C) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_env) return;
  C.ls[e] = C.iter[e];
  C.halv[e] = 0;
  if (C.iter[e]) C.alpha[e] = bits_to_double(C.alpha_bits[e]);
  C.bad[e] = 0;
}
__global__ void k_env_ls_decide(int n_env, EnvCtl C, int max_ls) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_env) return;
  if (!C.ls[e]) return;
  bool ok = !C.bad[e] && (C.constrained[e] || C.Et[e] <= C.E0[e]);
  C.bad[e] = 0;
  if (ok) {
    C.ls[e] = 0;
    C.accept[e] = 1;
    return;
  }
  int hv = C.halv[e] + 1;
  C.halv[e] = hv;
  if (hv > max_ls) {
    C.ls[e] = 0;
    C.iter[e] = 0;
    C.status[e] = ST_FAILED;
    C.reason[e] = FAIL_LINESEARCH;
    return;
  }
  C.stats[5 * e + STAT_LS] += 1;
  C.alpha[e] = C.alpha[e] / 2.0;
}
// the incremental potential at the iterate of each env still iterating, at its place in the env's
// trace of the current step (index = Newton iterations already done in the step)
__global__ void k_trace_record(int n_env, EnvCtl C, const double* __restrict__ E0, double* __restrict__ trace,
                               int* __restrict__ trace_n, int cap) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_env || !C.iter[e]) return;
  const int k = C.newton_it[e];
  if (k < 0 || k >= cap) return;
  trace[(long)e * cap + k] = E0[e];
  trace_n[e] = k + 1;
}
__global__ void k_env_newton_end(int n_env, EnvCtl C, int max_newton) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_env) return;
  if (!C.iter[e]) return;
  int it = C.newton_it[e] + 1;
  C.newton_it[e] = it;
  if (it >= max_newton) {
    C.iter[e] = 0;
    C.status[e] = ST_FAILED;
    C.reason[e] = FAIL_NEWTON;
  }
}
// the envs inside a step whose Newton loop stopped leave the step; the active ones count it
__global__ void k_env_end_step(int n_env, EnvCtl C) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_env) return;
  if (!C.stepping[e] || C.iter[e]) return;
  C.stepping[e] = 0;
  if (C.status[e] != ST_ACTIVE) return;
  int s = C.step[e] + 1;
  C.step[e] = s;
  C.rem[e] -= 1;
  C.stats[5 * e + STAT_STEPS] += 1;
  if (s >= C.nsteps[e]) C.status[e] = ST_DONE;
}
__global__ void k_count_flags(int n, const uint8_t* __restrict__ f, int* __restrict__ out) {
  __shared__ int sh[256];
  int acc = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += f[i] ? 1 : 0;
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}
__global__ void k_fill_u8(int n, uint8_t* a, uint8_t v) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] = v;
}
__global__ void k_set_single(int n, uint8_t* a, int which) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] = (i == which) ? 1 : 0;
}
__global__ void k_add_vec(long n, const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ c) {
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i < n) c[i] = __dadd_rn(a[i], b[i]);
}

// ---------------------------------------------------------------- primitive boxes
// box = [min - r, max + r] per axis (r = dhat/2), or swept [min(x, x_end), max(x, x_end)].
template <int NV>
__global__ void k_prim_boxes(int n, const int* __restrict__ prim_pt, const double* __restrict__ ptx,
                             const double* __restrict__ pte, double r, double* __restrict__ box) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int k = 0; k < 3; ++k) {
    double lo = INFINITY, hi = -INFINITY;
    for (int v = 0; v < NV; ++v) {
      int pt = prim_pt[NV * i + v];
      double a = ptx[3L * pt + k];
      lo = fmin(lo, a);
      hi = fmax(hi, a);
      if (pte) {
        double b = pte[3L * pt + k];
        lo = fmin(lo, b);
        hi = fmax(hi, b);
      }
    }
    box[6L * i + k] = __dsub_rn(lo, r);
    box[6L * i + 3 + k] = __dadd_rn(hi, r);
  }
}

// Whether the swept boxes [min(x, x_end) - r, max(x, x_end) + r] of the primitives of the envs in
// act (computed as k_prim_boxes computes them) lie inside the boxes a stored candidate list was
// made with; a primitive outside sets *out. Inside, every pair whose new boxes overlap had
// overlapping stored boxes, so the stored list still holds it.
template <int NV>
__global__ void k_swept_inside(int n, const int* __restrict__ prim_pt, const int* __restrict__ prim_env,
                               const uint8_t* __restrict__ act, const double* __restrict__ ptx,
                               const double* __restrict__ pte, double r, const double* __restrict__ stored,
                               int* __restrict__ out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || !act[prim_env[i]]) return;
  for (int k = 0; k < 3; ++k) {
    double lo = INFINITY, hi = -INFINITY;
    for (int v = 0; v < NV; ++v) {
      int pt = prim_pt[NV * i + v];
      double a = ptx[3L * pt + k], b = pte[3L * pt + k];
      lo = fmin(fmin(lo, a), b);
      hi = fmax(fmax(hi, a), b);
    }
    if (__dsub_rn(lo, r) < stored[6L * i + k] || __dadd_rn(hi, r) > stored[6L * i + 3 + k]) {
      atomicOr(out, 1);
      return;
    }
  }
}

// ---------------------------------------------------------------- candidates
struct PtInfo {
  const int* body;     // affine body index (>= 0) or -1 - soft body id
  const uint8_t* kin;
};
DEV bool excluded(const PtInfo& P, int a, int b, int c, int d) {
  if (P.kin[a] && P.kin[b] && P.kin[c] && P.kin[d]) return true;
  int ba = P.body[a];
  return ba >= 0 && P.body[b] == ba && P.body[c] == ba && P.body[d] == ba;
}

// fill (partners sorted per query, at offsets from a previous count), fill unsorted, and
// collect: count while keeping the first `cap` partners of each query in its own slots (one
// traversal instead of count + fill when no query finds more than cap)
enum { TRAV_FILL = 1, TRAV_FILLU = 3, TRAV_COLLECT = 4 };

struct CandOut {
  int* cnt;        // per query (count and collect modes)
  const int* off;  // per query (fill mode)
  int* cj;         // candidate partner (fill mode), or cap slots per query (collect mode)
  int* overflow;   // [0]: traversal stack overflow, [1]: a query found more than cap (collect)
  int cap = 0;
  int* cq = nullptr;  // fill modes: the query of each candidate (beside cj), or null
};

// point-triangle candidates: surface vertex q against the triangle tree of its env
template <int MODE>
__global__ void k_trav_pt(int n_sv, const int* __restrict__ sv_pt, const int* __restrict__ sv_env,
                          const uint8_t* __restrict__ act, const double* __restrict__ ptx, const double* __restrict__ pte,
                          double r, Tree T, const int* __restrict__ tri_pt, PtInfo P, CandOut O) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n_sv) return;
  int e = sv_env[q];
  if (!act[e]) {
    if (MODE == TRAV_COLLECT) O.cnt[q] = 0;
    return;
  }
  int v = sv_pt[q];
  double qb[6];
  for (int k = 0; k < 3; ++k) {
    double a = ptx[3L * v + k];
    double lo = a, hi = a;
    if (pte) {
      lo = fmin(lo, pte[3L * v + k]);
      hi = fmax(hi, pte[3L * v + k]);
    }
    qb[k] = __dsub_rn(lo, r);
    qb[3 + k] = __dadd_rn(hi, r);
  }
  int count = 0;
  int base = (MODE == TRAV_FILL || MODE == TRAV_FILLU) ? O.off[q] : 0;
  bool ok = bvh_visit(T, e, qb, [&](int j) {
    int a = tri_pt[3 * j], b = tri_pt[3 * j + 1], c = tri_pt[3 * j + 2];
    if (a == v || b == v || c == v) return;
    if (excluded(P, v, a, b, c)) return;
    if (MODE == TRAV_FILL || MODE == TRAV_FILLU) {
      O.cj[base + count] = j;
      if (O.cq) O.cq[base + count] = q;
    }
    if (MODE == TRAV_COLLECT && count < O.cap) O.cj[(long)q * O.cap + count] = j;
    ++count;
  });
  if (!ok) atomicOr(O.overflow, 1);
  if (MODE == TRAV_COLLECT) O.cnt[q] = count;
  if (MODE == TRAV_COLLECT && count > O.cap) atomicOr(O.overflow + 1, 1);
  if (MODE == TRAV_FILL) {
    // sort this query's partners ascending (insertion sort; short lists)
    int* s = O.cj + base;
    for (int i = 1; i < count; ++i) {
      int key = s[i], k = i - 1;
      while (k >= 0 && s[k] > key) {
        s[k + 1] = s[k];
        --k;
      }
      s[k + 1] = key;
    }
  }
}

// edge-edge candidates: edge q against the edge tree of its env, partners j > q
template <int MODE>
__global__ void k_trav_ee(int n_ed, const int* __restrict__ ed_pt, const int* __restrict__ ed_env,
                          const uint8_t* __restrict__ act, const double* __restrict__ edge_box, Tree T, PtInfo P,
                          CandOut O) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n_ed) return;
  int e = ed_env[q];
  if (!act[e]) {
    if (MODE == TRAV_COLLECT) O.cnt[q] = 0;
    return;
  }
  int a0 = ed_pt[2 * q], a1 = ed_pt[2 * q + 1];
  const double* qb = edge_box + 6L * q;
  int count = 0;
  int base = (MODE == TRAV_FILL || MODE == TRAV_FILLU) ? O.off[q] : 0;
  bool ok = bvh_visit(T, e, qb, [&](int j) { return j > q; }, [&](int j) {
    int b0 = ed_pt[2 * j], b1 = ed_pt[2 * j + 1];
    if (a0 == b0 || a0 == b1 || a1 == b0 || a1 == b1) return;
    if (excluded(P, a0, a1, b0, b1)) return;
    if (MODE == TRAV_FILL || MODE == TRAV_FILLU) {
      O.cj[base + count] = j;
      if (O.cq) O.cq[base + count] = q;
    }
    if (MODE == TRAV_COLLECT && count < O.cap) O.cj[(long)q * O.cap + count] = j;
    ++count;
  });
  if (!ok) atomicOr(O.overflow, 1);
  if (MODE == TRAV_COLLECT) O.cnt[q] = count;
  if (MODE == TRAV_COLLECT && count > O.cap) atomicOr(O.overflow + 1, 1);
  if (MODE == TRAV_FILL) {
    int* s = O.cj + base;
    for (int i = 1; i < count; ++i) {
      int key = s[i], k = i - 1;
      while (k >= 0 && s[k] > key) {
        s[k + 1] = s[k];
        --k;
      }
      s[k + 1] = key;
    }
  }
}

// The pair record of every listed candidate (kind, points, env, EE mollifier threshold, list
// index), made once per candidate list, so that each narrow phase and ACCD read one record per
// pair. cq[i] is the query of candidate i, cj[i] its partner.
__global__ void k_cand_records(int n_pt, int n_ee, const int* __restrict__ cq, const int* __restrict__ cj,
                               const int* __restrict__ sv_pt, const int* __restrict__ sv_env,
                               const int* __restrict__ tri_pt, const int* __restrict__ ed_pt,
                               const int* __restrict__ ed_env, const double* __restrict__ ed_rest2,
                               ContactRec* __restrict__ rec) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_pt + n_ee) return;
  ContactRec c;
  const int q = cq[i], j = cj[i];
  if (i < n_pt) {
    c.kind = 0;
    c.pts[0] = sv_pt[q];
    c.pts[1] = tri_pt[3 * j];
    c.pts[2] = tri_pt[3 * j + 1];
    c.pts[3] = tri_pt[3 * j + 2];
    c.env = sv_env[q];
    c.eps_x = 0.0;
  } else {
    c.kind = 1;
    c.pts[0] = ed_pt[2 * q];
    c.pts[1] = ed_pt[2 * q + 1];
    c.pts[2] = ed_pt[2 * j];
    c.pts[3] = ed_pt[2 * j + 1];
    c.env = ed_env[q];
    c.eps_x = 1e-3 * ed_rest2[q] * ed_rest2[j];
  }
  c.type = 0;
  c.cand = i;
  rec[i] = c;
}

// narrow phase: keep the listed pairs with d^2 < dhat^2 (flag), typed for the stencils; the
// record of a kept pair goes to tmp[i]. act (or null) keeps only the envs of this evaluation.
__global__ void k_narrow(int n, const ContactRec* __restrict__ rec, const uint8_t* __restrict__ act,
                         const double* __restrict__ ptx, double dhat2, int* __restrict__ flag,
                         ContactRec* __restrict__ tmp) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  ContactRec c = rec[i];
  if (act && !act[c.env]) {  // a list that holds envs outside this evaluation
    flag[i] = 0;
    return;
  }
  d3 X[4];
  for (int k = 0; k < 4; ++k) X[k] = ld3(ptx, c.pts[k]);
  // a pair whose boxes are more than dhat apart along an axis is no contact: tested before
  // the distance, with a margin far above the rounding of the box differences
  const double gap = sqrt(dhat2) * (1.0 + 1e-9);
  const int na = c.kind == 0 ? 1 : 2;
  double ga[3] = {X[0].x, X[0].y, X[0].z}, gb[3] = {X[na].x, X[na].y, X[na].z};
  double ha[3] = {ga[0], ga[1], ga[2]}, hb[3] = {gb[0], gb[1], gb[2]};
  for (int k = 1; k < 4; ++k) {
    const double u[3] = {X[k].x, X[k].y, X[k].z};
    double* lo = k < na ? ga : gb;
    double* hi = k < na ? ha : hb;
    for (int a = 0; a < 3; ++a) {
      lo[a] = fmin(lo[a], u[a]);
      hi[a] = fmax(hi[a], u[a]);
    }
  }
  for (int a = 0; a < 3; ++a)
    if (gb[a] - ha[a] > gap || ga[a] - hb[a] > gap) {
      flag[i] = 0;
      return;
    }
  int type;
  double d2 = pair_d2(c.kind, X, &type);
  c.type = type;
  const bool keep = d2 < dhat2;
  if (keep) tmp[i] = c;
  flag[i] = keep ? 1 : 0;
}

// Candidates of a collect traversal to their final places: query q's partners (at most cap,
// in its slots) go to out[off[q] ...], sorted ascending when `sorted` (the fill mode's order).
__global__ void k_gather_cands(int nq, int cap, const int* __restrict__ cnt, const int* __restrict__ slots,
                               const int* __restrict__ off, int* __restrict__ out, int* __restrict__ out_q, int sorted) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nq) return;
  const int n = cnt[q];
  if (n == 0) return;
  int* o = out + off[q];
  const int* sl = slots + (long)q * cap;
  for (int i = 0; i < n; ++i) {
    o[i] = sl[i];
    out_q[off[q] + i] = q;
  }
  if (!sorted) return;
  for (int i = 1; i < n; ++i) {
    int key = o[i], k = i - 1;
    while (k >= 0 && o[k] > key) {
      o[k + 1] = o[k];
      --k;
    }
    o[k + 1] = key;
  }
}

// Swept box [min(x, x_end), max(x, x_end)] of n points: the box k_prim_boxes and the
// point-triangle query build with no growth.
DEV void swept_box(const double* __restrict__ ptx, const double* __restrict__ pte, const int* pts, int n,
                   double* box) {
  for (int k = 0; k < 3; ++k) {
    double lo = INFINITY, hi = -INFINITY;
    for (int v = 0; v < n; ++v) {
      const double a = ptx[3L * pts[v] + k], b = pte[3L * pts[v] + k];
      lo = fmin(lo, fmin(a, b));
      hi = fmax(hi, fmax(a, b));
    }
    box[k] = lo;
    box[3 + k] = hi;
  }
}

// Additive CCD of every swept candidate pair (point-triangle pairs first, then edge-edge), one
// thread per pair: the time of impact along [x, x + p] lowers the env's step bound alpha_max
// (an atomic minimum on non-negative doubles: exact and independent of order). When the
// candidates were gathered with grown boxes (pte given), a pair whose plain swept boxes do
// not overlap is skipped, so the set of tested pairs is the plain swept-box set.
__global__ void k_accd_pairs(int n, const ContactRec* __restrict__ rec, const double* __restrict__ ptx,
                             const double* __restrict__ ptp, const double* __restrict__ pte, EnvCtl C) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const ContactRec& c = rec[i];
  const int kind = c.kind, e = c.env;
  int pts[4] = {c.pts[0], c.pts[1], c.pts[2], c.pts[3]};
  if (!C.iter[e]) return;  // an env covered for its next step only needs the candidates
  if (pte) {
    const int na = kind == 0 ? 1 : 2;
    double ba[6], bb[6];
    swept_box(ptx, pte, pts, na, ba);
    swept_box(ptx, pte, pts + na, 4 - na, bb);
    if (!box_overlap(ba, bb)) return;
  }
  d3 X[4], Pd[4];
  for (int a = 0; a < 4; ++a) {
    X[a] = ld3(ptx, pts[a]);
    Pd[a] = ld3(ptp, pts[a]);
  }
  long it;
  double t = accd(kind, X, Pd, 0.1, 1.0, 1000000L, &it);
  atomic_min_pos(&C.alpha_bits[e], t);
  atomicAdd((unsigned long long*)&C.stats[5 * e + STAT_ACCD], (unsigned long long)it);
}
__global__ void k_compact_contacts(int n, const int* __restrict__ flag, const int* __restrict__ off,
                                   const ContactRec* __restrict__ tmp, ContactRec* __restrict__ out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (flag[i]) out[off[i]] = tmp[i];
}

// the bodies (env-local handles: soft bodies first, then affine bodies) of the two sides of
// every contact: the point and the triangle of a point-triangle pair, the two edges of an
// edge-edge pair
__global__ void k_contact_handles(int n_ct, const ContactRec* __restrict__ ct, const int* __restrict__ pt_node,
                                  const int* __restrict__ body_node, const int* __restrict__ node_handle,
                                  int* __restrict__ out) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_ct) return;
  const ContactRec c = ct[k];
  auto handle = [&](int p) {
    const int nd = pt_node[p];
    return node_handle[nd >= 0 ? nd : body_node[-1 - nd]];
  };
  out[2 * k] = handle(c.pts[0]);
  out[2 * k + 1] = handle(c.pts[c.kind == 0 ? 1 : 2]);
}

// normal force of every contact: kappa e |b'(d)| (the friction lag's lambda), per env kappa
__global__ void k_contact_force(int n_ct, const ContactRec* __restrict__ ct, const double* __restrict__ ptx,
                                double dhat, const double* __restrict__ kappa_env, double* __restrict__ out) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_ct) return;
  ContactRec c = ct[k];
  d3 X[4];
  for (int i = 0; i < 4; ++i) X[i] = ld3(ptx, c.pts[i]);
  double d = sqrt(typed_d2(c.kind, c.type, X));
  double b, b1, b2;
  barrier3(d, dhat, &b, &b1, &b2);
  double m = 1.0;
  if (c.kind == 1) {
    d3 n = cross(X[1] - X[0], X[3] - X[2]);
    double cc = dot(n, n);
    if (cc < c.eps_x) {
      double r = cc / c.eps_x;
      m = -r * r + 2.0 * r;
    }
  }
  out[k] = kappa_env[c.env] * m * fabs(b1);
}

// lagged friction at x^t: lambda = kappa e |b'(d)|, closest-point coefficients and normal
__global__ void k_friction_setup(int n_ct, const ContactRec* __restrict__ ct, const double* __restrict__ ptx,
                                 const double* __restrict__ env_mu, double dhat, const double* __restrict__ kappa_env,
                                 FrictionRec* __restrict__ fr) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_ct) return;
  ContactRec c = ct[k];
  d3 X[4];
  for (int i = 0; i < 4; ++i) X[i] = ld3(ptx, c.pts[i]);
  double d = sqrt(typed_d2(c.kind, c.type, X));
  double b, b1, b2;
  barrier3(d, dhat, &b, &b1, &b2);
  double m = 1.0;
  if (c.kind == 1) {
    d3 n = cross(X[1] - X[0], X[3] - X[2]);
    double cc = dot(n, n);
    if (cc < c.eps_x) {
      double r = cc / c.eps_x;
      m = -r * r + 2.0 * r;
    }
  }
  FrictionRec f;
  for (int i = 0; i < 4; ++i) f.pts[i] = c.pts[i];
  f.env = c.env;
  f.pad = 0;
  d3 n;
  pair_closest(c.kind, X, f.c, &n);
  f.n[0] = n.x;
  f.n[1] = n.y;
  f.n[2] = n.z;
  f.mu_lambda = env_mu[c.env] * kappa_env[c.env] * m * fabs(b1);
  fr[k] = f;
}

// stencil table [contacts | friction]: points and env of every 4-point stencil
__global__ void k_stencil_table(int n_ct, int n_fr, int n_jt, const ContactRec* __restrict__ ct,
                                const FrictionRec* __restrict__ fr, const JointRec* __restrict__ jt,
                                int* __restrict__ st_pts, int* __restrict__ st_env) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_ct + n_fr + n_jt) return;
  if (s >= n_ct + n_fr) {  // a joint: points (a, b, a, b), the last two carry nothing
    const JointRec& J = jt[s - n_ct - n_fr];
    for (int k = 0; k < 4; ++k) st_pts[4 * s + k] = J.pts[k & 1];
    st_env[s] = J.env;
    return;
  }
  const int* p;
  int e;
  if (s < n_ct) {
    p = ct[s].pts;
    e = ct[s].env;
  } else {
    p = fr[s - n_ct].pts;
    e = fr[s - n_ct].env;
  }
  for (int k = 0; k < 4; ++k) st_pts[4 * s + k] = p[k];
  st_env[s] = e;
}

// stencil -> node incidence entries: number per stencil, then (node key, stencil*4 + slot)
__global__ void k_stencil_nent(int n_st, const int* __restrict__ st_pts, const int* __restrict__ st_env,
                               const uint8_t* __restrict__ act, const int* __restrict__ pt_node, int* __restrict__ cnt) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_st) return;
  int c = 0;
  if (act[st_env[s]])
    for (int a = 0; a < 4; ++a) c += pt_node[st_pts[4 * s + a]] >= 0 ? 1 : 4;
  cnt[s] = c;
}
__global__ void k_stencil_emit(int n_st, const int* __restrict__ st_pts, const int* __restrict__ st_env,
                               const uint8_t* __restrict__ act, const int* __restrict__ pt_node,
                               const int* __restrict__ body_node, const int* __restrict__ off,
                               unsigned long long* __restrict__ keys, unsigned* __restrict__ vals) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_st) return;
  if (!act[st_env[s]]) return;
  int o = off[s];
  for (int a = 0; a < 4; ++a) {
    int nd = pt_node[st_pts[4 * s + a]];
    if (nd >= 0) {
      keys[o] = (unsigned long long)nd;
      vals[o++] = (unsigned)(4 * s + a);
    } else {
      int base = body_node[-1 - nd];
      for (int k = 0; k < 4; ++k) {
        keys[o] = (unsigned long long)(base + k);
        vals[o++] = (unsigned)(4 * s + a);
      }
    }
  }
}
__global__ void k_count_keys(int n, const unsigned long long* __restrict__ keys, int* __restrict__ cnt) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) atomicAdd(&cnt[keys[i]], 1);
}

// ---------------------------------------------------------------- adapted barrier stiffness
// Start of a step: per env, over its free DOFs, g0 . G and G . G with g0 the gradient without the
// barrier (stiffness 0) and G = g1 - g0 the barrier's gradient per unit stiffness; one block per
// env, fixed-order block sums (the result does not depend on the batch).
__global__ void k_env_kappa_dots(int n_env, Layout L, const uint8_t* __restrict__ act, const int* __restrict__ node_off,
                                 const double* __restrict__ g0, const double* __restrict__ g1, double* __restrict__ dots) {
  __shared__ double sh[256];
  const int e = blockIdx.x;
  if (e >= n_env || !act[e]) return;
  double a = 0.0, b = 0.0;
  for (long i = 3L * node_off[e] + threadIdx.x; i < 3L * node_off[e + 1]; i += blockDim.x) {
    const int nd = (int)(i / 3), bd = L.node_body[nd];
    const bool kin = bd < 0 ? L.node_kin[nd] : L.body_kin[bd];
    if (kin) continue;
    const double G = g1[i] - g0[i];
    a += g0[i] * G;
    b += G * G;
  }
  a = block_sum(a, sh);
  b = block_sum(b, sh);
  if (threadIdx.x == 0) {
    dots[2 * e] = a;
    dots[2 * e + 1] = b;
  }
}
// kappa = -(g0 . G) / (G . G) clamped to [kmin, kmax]; kmin where no contact pulls (G = 0)
__global__ void k_env_kappa_start(int n_env, const uint8_t* __restrict__ act, const double* __restrict__ dots,
                                  double kmin, double kmax, double* __restrict__ kappa) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_env || !act[e]) return;
  double k = kmin;
  const double gg = dots[2 * e + 1];
  if (gg > 0.0) {
    const double r = -dots[2 * e] / gg;
    if (isfinite(r)) k = fmin(fmax(r, kmin), kmax);
  }
  kappa[e] = k;
}
__global__ void k_env_fill(int n_env, const uint8_t* __restrict__ act, double* __restrict__ a, double v) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n_env && (!act || act[e])) a[e] = v;
}

// ---------------------------------------------------------------- per-env step start
// positions of the points of the envs in act, src -> dst
__global__ void k_copy_points_env(int n_pts, Layout L, const uint8_t* __restrict__ act, const double* __restrict__ src,
                                  double* __restrict__ dst) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n_pts) return;
  int nd = L.pt_node[q];
  int e = L.node_env[nd >= 0 ? nd : L.body_node[-1 - nd]];
  if (!act[e]) return;
  for (int k = 0; k < 3; ++k) dst[3L * q + k] = src[3L * q + k];
}
// Friction records after some envs started a step: the old records of the envs that stay
// inside their step, and the new records of the starting envs, keyed (kind, env) for a stable
// sort that keeps each env's records in their order; dropped records sort last.
__global__ void k_fr_keys(int n_old, int n_old_pt, const FrictionRec* __restrict__ old_fr, int n_new, int n_new_pt,
                          const FrictionRec* __restrict__ new_fr, const uint8_t* __restrict__ stepping,
                          const uint8_t* __restrict__ start, unsigned long long* __restrict__ keys,
                          unsigned* __restrict__ vals, int* __restrict__ cnt) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_old + n_new) return;
  unsigned long long key;
  if (i < n_old) {
    int e = old_fr[i].env;
    bool keep = stepping[e] && !start[e];
    key = keep ? ((unsigned long long)(i >= n_old_pt) << 32) | (unsigned)e : (2ull << 32);
  } else {
    int j = i - n_old;
    key = ((unsigned long long)(j >= n_new_pt) << 32) | (unsigned)new_fr[j].env;
  }
  keys[i] = key;
  vals[i] = (unsigned)i;
  if (key < (1ull << 32)) atomicAdd(&cnt[0], 1);  // kept point-triangle records
  if (key < (2ull << 32)) atomicAdd(&cnt[1], 1);  // kept records
}
__global__ void k_fr_gather(int n, const unsigned* __restrict__ vals, int n_old, const FrictionRec* __restrict__ old_fr,
                            const FrictionRec* __restrict__ new_fr, FrictionRec* __restrict__ out) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  int v = (int)vals[k];
  out[k] = v < n_old ? old_fr[v] : new_fr[v - n_old];
}

// ---------------------------------------------------------------- invariants
DEV double orient3(d3 a, d3 b, d3 c, d3 d) { return dot(cross(b - a, c - a), d - a); }
// proper crossing of segment s0s1 through triangle abc by signed volumes; values within a
// relative 1e-9 of zero (coplanar or touching configurations) do not count as crossings,
// touching is covered by the positive-distance invariant instead
DEV bool seg_tri_cross(d3 s0, d3 s1, d3 a, d3 b, d3 c) {
  d3 ds = s1 - s0, e1 = b - a, e2 = c - a;
  double Ls = sqrt(dot(ds, ds)), Le = fmax(sqrt(dot(e1, e1)), sqrt(dot(e2, e2)));
  double eps_p = 1e-9 * sqrt(dot(cross(e1, e2), cross(e1, e2))) * Ls;
  double o0 = orient3(a, b, c, s0), o1 = orient3(a, b, c, s1);
  if (!((o0 > eps_p && o1 < -eps_p) || (o0 < -eps_p && o1 > eps_p))) return false;
  double eps_e = 1e-9 * Ls * Le * Le;
  double u = orient3(s0, s1, a, b), v = orient3(s0, s1, b, c), w = orient3(s0, s1, c, a);
  return (u > eps_e && v > eps_e && w > eps_e) || (u < -eps_e && v < -eps_e && w < -eps_e);
}
__global__ void k_intersections(int n_ed, const int* __restrict__ ed_pt, const int* __restrict__ ed_env,
                                const uint8_t* __restrict__ act, const double* __restrict__ edge_box, Tree T,
                                const int* __restrict__ tri_pt, PtInfo P, const double* __restrict__ ptx,
                                unsigned long long* __restrict__ count, int* __restrict__ overflow) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n_ed) return;
  int e = ed_env[q];
  if (!act[e]) return;
  int a0 = ed_pt[2 * q], a1 = ed_pt[2 * q + 1];
  unsigned long long n = 0;
  bool ok = bvh_visit(T, e, edge_box + 6L * q, [&](int j) {
    int a = tri_pt[3 * j], b = tri_pt[3 * j + 1], c = tri_pt[3 * j + 2];
    if (a0 == a || a0 == b || a0 == c || a1 == a || a1 == b || a1 == c) return;
    int ba = P.body[a0];
    if (ba >= 0 && P.body[a1] == ba && P.body[a] == ba) return;
    if (seg_tri_cross(ld3(ptx, a0), ld3(ptx, a1), ld3(ptx, a), ld3(ptx, b), ld3(ptx, c))) ++n;
  });
  if (!ok) atomicOr(overflow, 1);
  if (n) atomicAdd(&count[e], n);
}
__global__ void k_inverted(int n_tets, const int4* __restrict__ tets, const int* __restrict__ tenv,
                           const uint8_t* __restrict__ act, const double* __restrict__ q,
                           unsigned long long* __restrict__ count) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_tets) return;
  int e = tenv[t];
  if (!act[e]) return;
  int4 T = tets[t];
  d3 x0 = ld3(q, T.x);
  double J = dot(cross(ld3(q, T.y) - x0, ld3(q, T.z) - x0), ld3(q, T.w) - x0);
  if (!(J > 0.0)) atomicAdd(&count[e], 1ull);
}
