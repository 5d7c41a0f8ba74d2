// Persistent per-environment PCG: one thread-block cluster per environment runs the whole
// block-Jacobi conjugate-gradient solve of that environment (Sec. III-A: one linear solve per
// environment, each with its own scalars and its own stop). The cluster's CTAs synchronise with
// hardware cluster barriers; there is no host round trip and no launch per iteration.
//
// Work split inside a cluster: stencil products go to half-warps round-robin over the cluster; the
// env's free soft rows, in chunks of 32 (one row per lane), are dealt to CTAs round-robin and,
// inside a CTA, to warps on demand, so a row's x, r, y, z entries stay on one SM; a rigid body
// belongs to CTA (body index mod C), its 12 DOFs to that CTA's threads 0..11.
// Kinematic soft rows are never visited: their right-hand side and preconditioner block are
// zero, so their d and z stay zero (d is zeroed when the buffers are laid out).
//
// One iteration has three phases, each ended by a cluster barrier: y = A d with the slot
// partials of d.y; x, r, z updates with the partials of r.z and r.r; d = z + beta d together with
// the stencil products of the next iteration, t_s = H_s P_s d = H_s P_s z + beta t_s (by
// linearity, from z, which the previous barrier published, so no barrier sits between the
// direction update and the products).
//
// Determinism: every dot product is summed per slot (a slice: warp butterfly over its 32 rows; a
// body: fixed CTA tree), and the env's slots are added in a fixed order that depends on the env
// alone. So the results are the same bits for every cluster size and every batch the env is in.
// A slot's partial lives in the shared memory of the CTA that owns the slot; after the barrier
// that publishes the partials every CTA reads all of the env's slots over distributed shared
// memory (the SM-to-SM network of the cluster, no L2 round trip) in that fixed order. Vectors
// that other CTAs write inside the kernel (d, t) are read with L2-coherent loads after the
// cluster barrier that publishes them.
#pragma once
#include <cooperative_groups.h>

#include "kernels_misc.cuh"
#include "solver.cuh"

namespace cg = cooperative_groups;

constexpr int PCG_THREADS = 256;
constexpr int N_ST_LISTS = 5;  // stencil sublists: contacts pt, ee; friction pt, ee; joints
constexpr int PCG_WARPS = PCG_THREADS / 32;
// CTAs per SM the register budget must allow: the FP64 solve keeps 128 registers a thread (it
// is bound by the FP64 pipe, and fewer registers spill); the FP32 solve is bound by memory
// latency and gains from 4 resident CTAs (64 registers, a few spilled bytes on cold paths).
template <class T>
constexpr int pcg_min_ctas() {
  return sizeof(T) == 8 ? 2 : 4;
}

// T: precision of the matrix, the vectors and every sum (FP64, or FP32 in mixed precision).
template <class T>
struct PcgClusterArgs {
  Layout L;
  SpmvArgsT<T, T> A;
  const int* pslice_off;  // per env: first slice of its free soft rows (n_env + 1 entries)
  const int* pslice_row;  // 32 per slice: the row (node), -1 for padding
  const int* pslice_sel;  // 32 per slice: sliced-ELL slice * 32 + lane of that row
  const int* body_off;    // per env: first body (n_env + 1 entries)
  const int* st_env;
  const T* sH;
  int st_bounds[6];       // stencil sublists [pt | ee | friction pt | friction ee | joints], each env-sorted
  const T* Ps;
  const T* Pb;
  const uint8_t* act;
  T* x;                   // solution (delta), out
  T* r;                   // in: right-hand side; out: residual
  T* z;
  T* d;
  T* y;
  T* st_t;                // stencil products (the same buffer SpmvArgs reads)
  double tol2;             // (relative tolerance)^2
  int max_it;
  int ns_loc;                 // slice slots one CTA owns at most (ceil(most slices of an env / C))
  int nb_loc;                 // body slots one CTA owns at most (ceil(most bodies of an env / C))
  const int* env_list;        // env of each cluster
  int first;                  // 1: start the solves (z = M^-1 r, d = z, x = 0); 0: resume them
  int chunk;                  // iterations at most in this launch
  double* rz_state;           // per env: r.z after the last iteration
  double* bb_state;           // per env: |b|^2 (right-hand side)
  double* iterb_state;        // per env: algorithmic bytes of one iteration
  double* iterf_state;        // per env: floating-point operations of one iteration
  int* it_state;              // per env: iterations so far
  uint8_t* run;               // per env: 1 while the solve continues
  long long* stats;           // 5 per env; [STAT_PCG] += iterations of this solve
  unsigned long long* bytes;  // algorithmic bytes of all iterations (may be null)
  unsigned long long* flops;  // floating-point operations of all iterations (null when bytes is)
  unsigned long long* iters;  // env-iterations done by this launch (may be null)
};

// Dynamic shared memory of one CTA: per owned slot, one d.y partial, then four values (r.z, r.r
// and, at the start, the algorithmic bytes and flops of one iteration). Slice slot j of the env
// (j = slice - first slice) is owned by CTA j mod C at local index j / C; body slot j by CTA
// j mod C at local index ns_loc + j / C.
template <class T>
constexpr size_t pcg_smem_bytes(int ns_loc, int nb_loc) {
  return (size_t)5 * (ns_loc + nb_loc) * sizeof(T);
}

// Sum of an env's slot partials (its slices, then its bodies) in a fixed order that depends on
// the env alone: lane l of warp 0 adds slots l, l + 32, ... (each read from its owner CTA's
// shared memory) and the lanes are combined by a fixed butterfly. Every CTA of the cluster
// computes the same bits; the result is broadcast through shared memory. Call after a cluster
// barrier that publishes the partials. base: this CTA's copy of the array (stride values per
// slot, the first K summed).
template <int K, int C, class T>
DEV void env_sum(const cg::cluster_group& cl, T* base, int stride, int ns, int nb, int ns_loc, T* tot, T (&v)[K]) {
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x, n = ns + nb;
    T s[K];
#pragma unroll
    for (int q = 0; q < K; ++q) s[q] = T(0);
#pragma unroll 4
    for (int j = lane; j < n; j += 32) {  // unrolled: the loads of several slots in flight at once
      const int jj = j < ns ? j : j - ns;
      const int li = j < ns ? jj / C : ns_loc + jj / C;
      const T* src = C == 1 ? base : cl.map_shared_rank(base, (unsigned)(jj % C));
#pragma unroll
      for (int q = 0; q < K; ++q) s[q] += src[stride * li + q];
    }
#pragma unroll
    for (int q = 0; q < K; ++q) {
      s[q] = warp_sum(s[q]);
      if (lane == 0) tot[q] = s[q];
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < K; ++q) v[q] = tot[q];
}

// Algorithmic bytes of one PCG iteration, per item, with values of b = sizeof(T) bytes. A soft
// row: its sliced-ELL blocks (9b + 4 B column each), d read and y written (6b), 16 B of row
// pointers, its stencil entries (4 B index + b weight each), then the vector phase: x, r read
// and written (12b), d, y read (6b), the 3x3 preconditioner block (9b), z written (3b) and
// d = z + beta d (9b). A rigid body: dense block (144b), its d and y (24b), per p-node entry
// 4 B + 3b rest coordinates, the 12x12 preconditioner (144b) and 12 DOFs x 10b of vector
// traffic. A stencil: packed Hessian (78b), 4 point nodes (16 B), their rest coordinates (12b),
// 4 gathered z triples (12b), t read and written (24b); each entry then reads its slot of t (3b).
template <class T>
DEV double soft_iter_bytes(const SpmvArgsT<T, T>& A, int row) {
  const double b = sizeof(T);
  return (9 * b + 4) * (A.bsr_ptr[row + 1] - A.bsr_ptr[row]) + 6 * b + 16.0 +
         (4 + 4 * b) * (A.ns_ptr[row + 1] - A.ns_ptr[row]) + 39 * b;
}
template <class T>
DEV double body_iter_bytes(const Layout& L, const SpmvArgsT<T, T>& A, int bd) {
  const double b = sizeof(T);
  long base = L.body_node[bd];
  return 168 * b + (4 + 6 * b) * (A.ns_ptr[base + 1] - A.ns_ptr[base]) + 144 * b + 120 * b;
}
template <class T>
DEV double stencil_iter_bytes() {
  return 78.0 * sizeof(T) + 16.0 + 48.0 * sizeof(T);
}
// Floating-point operations of one iteration (an FMA counts 2). A soft row: 18 per sliced-ELL
// block, 6 per stencil entry, 6 for d.y; then x, r updates (12), z = M^-1 r (18), r.z and r.r
// (12), d = z + beta d (6). A rigid body: 21 per p-node entry, the dense block (288) and d.y
// (24), x, r updates (48), the 12x12 preconditioner (288), r.z and r.r (48), d update (24). A
// stencil: the 12x12 product (288).
template <class T>
DEV double soft_iter_flops(const SpmvArgsT<T, T>& A, int row) {
  return 18.0 * (A.bsr_ptr[row + 1] - A.bsr_ptr[row]) + 6.0 * (A.ns_ptr[row + 1] - A.ns_ptr[row]) + 6.0 + 48.0;
}
template <class T>
DEV double body_iter_flops(const Layout& L, const SpmvArgsT<T, T>& A, int bd) {
  long base = L.body_node[bd];
  return 21.0 * (A.ns_ptr[base + 1] - A.ns_ptr[base]) + 288.0 + 24.0 + 48.0 + 288.0 + 48.0 + 24.0;
}
constexpr double STENCIL_ITER_FLOPS = 288.0;

template <int C, class T>
__global__ void __launch_bounds__(PCG_THREADS, pcg_min_ctas<T>()) k_pcg_cluster(PcgClusterArgs<T> P) {
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const int e = P.env_list[blockIdx.x / C];
  if (P.first && !P.act[e]) {  // uniform over the cluster: every CTA leaves
    if (rank == 0 && threadIdx.x == 0) P.run[e] = 0;
    return;
  }
  extern __shared__ __align__(16) unsigned char pcg_dyn[];
  __shared__ T wred[PCG_WARPS][12];
  __shared__ T tot[4];
  __shared__ T sbody[12];
  __shared__ int srange[2 * N_ST_LISTS];
  __shared__ int grab[4];  // per phase: the next of this CTA's slices to hand to a warp
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // warps are interleaved over the cluster's CTAs, so consecutive slices land on different SMs
  const int gwarp = warp * C + rank, nwarps = C * PCG_WARPS;
  const Layout& L = P.L;
  const int S0 = P.pslice_off[e], S1 = P.pslice_off[e + 1];
  const int b0 = P.body_off[e], b1 = P.body_off[e + 1];
  const int NSL = P.ns_loc;
  T* part_dy = (T*)pcg_dyn;                      // 1 value per owned slot
  T* part_rz = part_dy + (P.ns_loc + P.nb_loc);  // (r.z, r.r, bytes, flops) per owned slot
  if (tid < N_ST_LISTS) {  // this env's range in each stencil sublist
    int lo = P.st_bounds[tid], hi = P.st_bounds[tid + 1];
    srange[2 * tid] = lower_env(P.st_env, lo, hi, e);
    srange[2 * tid + 1] = lower_env(P.st_env, lo, hi, e + 1);
  }
  if (tid < 4) grab[tid] = 0;
  __syncthreads();
  // Slices go to CTAs round-robin (slice S0 + rank + C j belongs to this CTA) and, inside the
  // CTA, to whichever warp asks next, so warps of uneven rows finish a phase together. A row
  // stays on its CTA's SM in every phase. Counters are reset in a later phase, after a barrier
  // that every warp passes only once it has stopped asking.
  const int n_mine = (S1 - S0 > rank) ? (S1 - S0 - rank + C - 1) / C : 0;
  auto next_slice = [&](int ph) -> int {
    int j = 0;
    if (lane == 0) j = atomicAdd(&grab[ph], 1);
    j = __shfl_sync(0xffffffffu, j, 0);
    return j < n_mine ? S0 + rank + C * j : -1;
  };
  int n_stencils = 0;
  for (int q = 0; q < N_ST_LISTS; ++q) n_stencils += srange[2 * q + 1] - srange[2 * q];

  T rz, bb;
  double iter_bytes, iter_flops;
  int it;
  bool go;
  if (P.first) {
    // ---- z = M^-1 r, d = z, x = 0; per-slot (r.z, r.r) and the bytes of one iteration
    for (int sl = next_slice(0); sl >= 0; sl = next_slice(0)) {  // warp-uniform
      T a = T(0), c = T(0), nb = T(0), nf = T(0);
      const int i = P.pslice_row[32 * sl + lane];
      if (i >= 0) {
        precond_soft(i, P.Ps, P.r, P.z, &a, &c);
        for (int k = 3 * i; k < 3 * i + 3; ++k) {
          P.d[k] = P.z[k];
          P.x[k] = T(0);
        }
        if (P.bytes) {
          nb = T(soft_iter_bytes(P.A, i));
          nf = T(soft_iter_flops(P.A, i));
        }
      }
      a = warp_sum(a);
      c = warp_sum(c);
      nb = warp_sum(nb);
      nf = warp_sum(nf);
      if (lane == 0) {
        T* o = part_rz + 4 * ((sl - S0) / C);
        o[0] = a;
        o[1] = c;
        o[2] = nb;
        o[3] = nf;
      }
    }
    for (int b = b0; b < b1; ++b) {
      if (rank != (b - b0) % C) continue;  // CTA-uniform
      long base3 = 3L * L.body_node[b];
      if (tid < 12) sbody[tid] = P.r[base3 + tid];
      __syncthreads();
      T a, c;
      precond_body(P.Pb, b, sbody, base3, P.z, &a, &c);
      if (tid < 12) {
        P.d[base3 + tid] = P.z[base3 + tid];
        P.x[base3 + tid] = T(0);
      }
      if (warp == 0) {
        a = warp_sum(a);
        c = warp_sum(c);
        if (lane == 0) {
          T* o = part_rz + 4 * (NSL + (b - b0) / C);
          o[0] = a;
          o[1] = c;
          o[2] = P.bytes ? T(body_iter_bytes(L, P.A, b)) : T(0);
          o[3] = P.bytes ? T(body_iter_flops(L, P.A, b)) : T(0);
        }
      }
      __syncthreads();
    }
    cl.sync();
    T v4[4];
    env_sum<4, C>(cl, part_rz, 4, S1 - S0, b1 - b0, NSL, tot, v4);
    rz = v4[0];
    bb = v4[1];
    iter_bytes = double(v4[2]) + (P.bytes ? stencil_iter_bytes<T>() * n_stencils : 0.0);
    iter_flops = double(v4[3]) + (P.bytes ? STENCIL_ITER_FLOPS * n_stencils : 0.0);
    it = 0;
    go = bb > T(0) && isfinite(bb);
    // ---- t_s = H_s (P_s d) for the env's stencils, one half-warp per stencil (d = z was
    // published by the barrier above)
    if (go)
      for (int q = 0; q < N_ST_LISTS; ++q)  // warp-uniform loop
        for (int s0 = srange[2 * q] + 2 * gwarp; s0 < srange[2 * q + 1]; s0 += 2 * nwarps) {
          int s = s0 + (lane >> 4);
          stencil_product_nodes<true>(P.A, (const T*)P.d, P.st_t, s, s < srange[2 * q + 1]);
        }
  } else {
    rz = T(P.rz_state[e]);
    bb = T(P.bb_state[e]);
    iter_bytes = P.iterb_state[e];
    iter_flops = P.iterf_state[e];
    it = P.it_state[e];
    go = true;
  }
  const T tol2 = T(P.tol2);
  const int it0 = it;
  bool more = go;  // the solve continues after this launch
  for (int k = 0; go && k < P.chunk; ++k) {
    // the barrier publishes every CTA's d and stencil products t = H_s (P_s d)
    cl.sync();
    if (tid == 0) grab[3] = 0;  // every warp is past the direction update (barrier above)
    // ---- y = A d: soft rows, one partial d.y per slice
    for (int sl = next_slice(1); sl >= 0; sl = next_slice(1)) {
      T dy = T(0);
      const int i = P.pslice_row[32 * sl + lane];
      if (i >= 0) {
        const int sel = P.pslice_sel[32 * sl + lane];
        dy = soft_row<true>(P.A, sel >> 5, sel & 31, i, (const T*)P.d, P.y);
      }
      dy = warp_sum(dy);
      if (lane == 0) part_dy[(sl - S0) / C] = dy;
    }
    // ---- rigid bodies on their owner CTA: stencil entries gathered by its threads in a fixed
    // partition, the dense 12x12 block, one partial d.y per body
    for (int b = b0; b < b1; ++b) {
      if (rank != (b - b0) % C) continue;  // CTA-uniform
      long base = L.body_node[b];
      bool kin = L.body_kin[b];
      T acc[12];
      for (int q = 0; q < 12; ++q) acc[q] = T(0);
      if (!kin) {
        int kb = P.A.ns_ptr[base], ke = P.A.ns_ptr[base + 1];
        for (int k2 = kb + tid; k2 < ke; k2 += PCG_THREADS) {
          const long src = P.A.ns_src[k2];
          const T tx = __ldcg(P.A.st_t + 3 * src), ty = __ldcg(P.A.st_t + 3 * src + 1),
                  tz = __ldcg(P.A.st_t + 3 * src + 2);
          const T* xb = P.A.ns_xb + 3L * k2;
          const T w1 = xb[0], w2 = xb[1], w3 = xb[2];
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
#pragma unroll
      for (int q = 0; q < 12; ++q) {
        T sq = warp_sum(acc[q]);
        if (lane == 0) wred[warp][q] = sq;
      }
      __syncthreads();
      if (warp == 0) {
        T dyb = T(0);
        if (lane < 12) {
          T v = T(0);
          if (!kin) {
            for (int w = 0; w < PCG_WARPS; ++w) v += wred[w][lane];
            const T* H = P.A.bH + 144L * b + 12 * lane;
            for (int j = 0; j < 12; ++j) v += H[j] * __ldcg(P.d + 3 * base + j);
          }
          P.y[3 * base + lane] = v;
          dyb = v * __ldcg(P.d + 3 * base + lane);
        }
        dyb = warp_sum(dyb);
        if (lane == 0) part_dy[NSL + (b - b0) / C] = dyb;
      }
      __syncthreads();
    }
    cl.sync();
    T dy[1];
    env_sum<1, C>(cl, part_dy, 1, S1 - S0, b1 - b0, NSL, tot, dy);
    const T alpha = dy[0] > T(0) ? rz / dy[0] : T(0);
    // ---- x += alpha d; r -= alpha y; z = M^-1 r (owner threads only)
    if (tid == 0) grab[1] = 0;  // every warp is past the product phase (barrier above)
    for (int sl = next_slice(2); sl >= 0; sl = next_slice(2)) {
      T a = T(0), c = T(0);
      const int i = P.pslice_row[32 * sl + lane];
      if (i >= 0) {
        for (int k2 = 3 * i; k2 < 3 * i + 3; ++k2) {
          P.x[k2] += alpha * P.d[k2];
          P.r[k2] -= alpha * P.y[k2];
        }
        precond_soft(i, P.Ps, P.r, P.z, &a, &c);
      }
      a = warp_sum(a);
      c = warp_sum(c);
      if (lane == 0) {
        part_rz[4 * ((sl - S0) / C)] = a;
        part_rz[4 * ((sl - S0) / C) + 1] = c;
      }
    }
    for (int b = b0; b < b1; ++b) {
      if (rank != (b - b0) % C) continue;  // CTA-uniform
      long base3 = 3L * L.body_node[b];
      if (tid < 12) {
        long k2 = base3 + tid;
        P.x[k2] += alpha * P.d[k2];
        T rv = P.r[k2] - alpha * P.y[k2];
        P.r[k2] = rv;
        sbody[tid] = rv;
      }
      __syncthreads();
      T a, c;
      precond_body(P.Pb, b, sbody, base3, P.z, &a, &c);
      if (warp == 0) {
        a = warp_sum(a);
        c = warp_sum(c);
        if (lane == 0) {
          part_rz[4 * (NSL + (b - b0) / C)] = a;
          part_rz[4 * (NSL + (b - b0) / C) + 1] = c;
        }
      }
      __syncthreads();
    }
    cl.sync();
    T u2[2];
    env_sum<2, C>(cl, part_rz, 4, S1 - S0, b1 - b0, NSL, tot, u2);
    const T rz_new = u2[0], rr = u2[1];
    ++it;
    if (rr <= tol2 * bb || it >= P.max_it || !(dy[0] > T(0)) || !isfinite(rr)) {
      more = false;
      break;
    }
    const T beta = rz > T(0) ? rz_new / rz : T(0);
    rz = rz_new;
    // ---- d = z + beta d (owner threads)
    if (tid == 0) grab[2] = 0;  // every warp is past the update phase (barrier above)
    for (int sl = next_slice(3); sl >= 0; sl = next_slice(3)) {
      const int i = P.pslice_row[32 * sl + lane];
      if (i >= 0)
        for (int k2 = 3 * i; k2 < 3 * i + 3; ++k2) P.d[k2] = P.z[k2] + beta * P.d[k2];
    }
    for (int b = b0; b < b1; ++b)
      if (rank == (b - b0) % C && tid < 12) {
        long k2 = 3L * L.body_node[b] + tid;
        P.d[k2] = P.z[k2] + beta * P.d[k2];
      }
    // ---- the stencil products follow d by linearity, H_s P_s d_new = H_s P_s z + beta t_s,
    // so they need z (published by the barrier above) and not the d being written: the next
    // product phase waits on one barrier instead of two
    for (int q = 0; q < N_ST_LISTS; ++q)  // warp-uniform loop
      for (int s0 = srange[2 * q] + 2 * gwarp; s0 < srange[2 * q + 1]; s0 += 2 * nwarps) {
        int s = s0 + (lane >> 4);
        stencil_product_nodes<true>(P.A, (const T*)P.z, P.st_t, s, s < srange[2 * q + 1], beta);
      }
  }
  // the CTAs of the cluster read each other's shared memory up to the last sum: none may leave
  // (and release its shared memory) before all are past it
  if (C > 1) cl.sync();
  // CTA 0 records the env's state
  if (rank == 0 && tid == 0) {
    P.rz_state[e] = double(rz);
    P.bb_state[e] = double(bb);
    P.iterb_state[e] = iter_bytes;
    P.iterf_state[e] = iter_flops;
    P.it_state[e] = it;
    P.run[e] = more ? 1 : 0;
    P.stats[5 * e + STAT_PCG] += it - it0;
    if (P.iters) atomicAdd(P.iters, (unsigned long long)(it - it0));
    if (P.bytes) {
      atomicAdd(P.bytes, (unsigned long long)(iter_bytes * (it - it0)));
      atomicAdd(P.flops, (unsigned long long)(iter_flops * (it - it0)));
    }
  }
}

// ids of the envs whose solve continues, in env order, and their count (one warp)
__global__ void k_list_running(int n_env, const uint8_t* __restrict__ run, int* __restrict__ list,
                               int* __restrict__ count) {
  const int lane = threadIdx.x & 31;
  int base = 0;
  for (int e0 = 0; e0 < n_env; e0 += 32) {
    int e = e0 + lane;
    bool f = e < n_env && run[e];
    unsigned m = __ballot_sync(0xffffffffu, f);
    if (f) list[base + __popc(m & ((1u << lane) - 1u))] = e;
    base += __popc(m);
  }
  if (lane == 0) *count = base;
}
