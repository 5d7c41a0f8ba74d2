// Broad phase: one linear BVH over the primitives of all environments, keyed by
// (environment, Morton code) so that every environment owns a separate subtree. Queries start
// at their environment's subtree root, which isolates the environments by construction
// (Sec. III-A). Karras (HPG 2012) binary radix tree, built from a stable LSD radix sort, refit
// bottom-up whenever the boxes move; traversal with a bounded per-thread stack.
#pragma once
#include "common.cuh"

constexpr int RS_THREADS = 256;
constexpr int RS_IPT = 8;
constexpr int RS_TILE = RS_THREADS * RS_IPT;
constexpr int SCAN_BLOCK = 1024;

// ------------------------------------------------------------------ device-wide scan (int32)
__global__ void k_scan_block_sums(const int* __restrict__ in, int n, int* __restrict__ sums) {
  __shared__ int sh[SCAN_BLOCK];
  int i = blockIdx.x * SCAN_BLOCK + threadIdx.x;
  int v = i < n ? in[i] : 0;
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int s = SCAN_BLOCK / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) sums[blockIdx.x] = sh[0];
}
// exclusive scan of m block sums by one block; total written to sums[m]
__global__ void k_scan_sums(int* __restrict__ sums, int m) {
  __shared__ int sh[SCAN_BLOCK];
  int per = (m + SCAN_BLOCK - 1) / SCAN_BLOCK;
  int b = threadIdx.x * per, e = min(b + per, m);
  int loc = 0;
  for (int i = b; i < e; ++i) loc += sums[i];
  sh[threadIdx.x] = loc;
  __syncthreads();
  // Hillis-Steele inclusive scan
  for (int off = 1; off < SCAN_BLOCK; off <<= 1) {
    int t = threadIdx.x >= off ? sh[threadIdx.x - off] : 0;
    __syncthreads();
    sh[threadIdx.x] += t;
    __syncthreads();
  }
  int run = sh[threadIdx.x] - loc;
  for (int i = b; i < e; ++i) {
    int v = sums[i];
    sums[i] = run;
    run += v;
  }
  if (threadIdx.x == SCAN_BLOCK - 1) sums[m] = sh[SCAN_BLOCK - 1];
}
__global__ void k_scan_apply(const int* __restrict__ in, int n, const int* __restrict__ sums, int* __restrict__ out) {
  __shared__ int sh[SCAN_BLOCK];
  int i = blockIdx.x * SCAN_BLOCK + threadIdx.x;
  int v = i < n ? in[i] : 0;
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int off = 1; off < SCAN_BLOCK; off <<= 1) {
    int t = threadIdx.x >= off ? sh[threadIdx.x - off] : 0;
    __syncthreads();
    sh[threadIdx.x] += t;
    __syncthreads();
  }
  if (i < n) out[i] = sums[blockIdx.x] + sh[threadIdx.x] - v;
  if (i == n - 1) out[n] = sums[blockIdx.x] + sh[threadIdx.x];
}

// ------------------------------------------------------------------ radix sort (stable LSD)
__global__ void k_rs_hist(const unsigned long long* __restrict__ keys, int n, int shift, int nblk, int* __restrict__ hist) {
  __shared__ int cnt[256];
  cnt[threadIdx.x] = 0;
  __syncthreads();
  int base = blockIdx.x * RS_TILE;
  for (int r = 0; r < RS_IPT; ++r) {
    int i = base + r * RS_THREADS + threadIdx.x;
    if (i < n) atomicAdd(&cnt[(keys[i] >> shift) & 255], 1);
  }
  __syncthreads();
  hist[threadIdx.x * nblk + blockIdx.x] = cnt[threadIdx.x];
}

__global__ void k_rs_scatter(const unsigned long long* __restrict__ kin, const unsigned* __restrict__ vin,
                             unsigned long long* __restrict__ kout, unsigned* __restrict__ vout, int n, int shift,
                             int nblk, const int* __restrict__ offs) {
  __shared__ int base[256], run[256], tot[256];
  __shared__ int wcnt[RS_THREADS / 32][257];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  base[t] = offs[t * nblk + blockIdx.x];
  run[t] = 0;
  for (int k = 0; k < RS_THREADS / 32; ++k) wcnt[k][t] = 0;
  __syncthreads();
  const unsigned lt = (1u << lane) - 1u;
  for (int r = 0; r < RS_IPT; ++r) {
    int i = blockIdx.x * RS_TILE + r * RS_THREADS + t;
    bool valid = i < n;
    unsigned long long key = valid ? kin[i] : 0ull;
    int dg = valid ? (int)((key >> shift) & 255) : 256;
    unsigned peers = __match_any_sync(0xffffffffu, dg);
    int rank = __popc(peers & lt);
    int leader = __ffs(peers) - 1;
    if (lane == leader && valid) wcnt[w][dg] = __popc(peers);
    __syncthreads();
    {
      int s = 0;
      for (int k = 0; k < RS_THREADS / 32; ++k) {
        int c = wcnt[k][t];
        wcnt[k][t] = s;
        s += c;
      }
      tot[t] = s;
    }
    __syncthreads();
    if (valid) {
      int pos = base[dg] + run[dg] + wcnt[w][dg] + rank;
      kout[pos] = key;
      vout[pos] = vin[i];
    }
    __syncthreads();
    run[t] += tot[t];
    for (int k = 0; k < RS_THREADS / 32; ++k) wcnt[k][t] = 0;
    __syncthreads();
  }
}

// ------------------------------------------------------------------ Morton codes
DEV unsigned expand_bits10(unsigned v) {
  v &= 1023u;
  v = (v | (v << 16)) & 0x030000FFu;
  v = (v | (v << 8)) & 0x0300F00Fu;
  v = (v | (v << 4)) & 0x030C30C3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}
DEV unsigned morton3(double x, double y, double z) {
  unsigned a = (unsigned)fmin(fmax(x * 1024.0, 0.0), 1023.0);
  unsigned b = (unsigned)fmin(fmax(y * 1024.0, 0.0), 1023.0);
  unsigned c = (unsigned)fmin(fmax(z * 1024.0, 0.0), 1023.0);
  return (expand_bits10(a) << 2) | (expand_bits10(b) << 1) | expand_bits10(c);
}

// per-env bounds of primitive box centres (ordered-bit atomics: exact, order independent)
__global__ void k_env_bounds(const double* __restrict__ box, const int* __restrict__ penv, int n,
                             unsigned long long* __restrict__ emin, unsigned long long* __restrict__ emax) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int e = penv[i];
  for (int k = 0; k < 3; ++k) {
    double c = 0.5 * (box[6 * i + k] + box[6 * i + 3 + k]);
    atomicMin(&emin[3 * e + k], ordered_bits(c));
    atomicMax(&emax[3 * e + k], ordered_bits(c));
  }
}
__global__ void k_morton(const double* __restrict__ box, const int* __restrict__ penv, int n,
                         const unsigned long long* __restrict__ emin, const unsigned long long* __restrict__ emax,
                         unsigned long long* __restrict__ keys, unsigned* __restrict__ vals) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int e = penv[i];
  double u[3];
  for (int k = 0; k < 3; ++k) {
    double lo = ordered_to_double(emin[3 * e + k]), hi = ordered_to_double(emax[3 * e + k]);
    double c = 0.5 * (box[6 * i + k] + box[6 * i + 3 + k]);
    u[k] = hi > lo ? (c - lo) / (hi - lo) : 0.5;
  }
  keys[i] = ((unsigned long long)e << 32) | morton3(u[0], u[1], u[2]);
  vals[i] = (unsigned)i;
}

// ------------------------------------------------------------------ Karras build
DEV int lcp_delta(const unsigned long long* __restrict__ k, int n, int i, int j) {
  if (j < 0 || j >= n) return -1;
  unsigned long long a = k[i], b = k[j];
  if (a == b) return 64 + __clz((unsigned)(i ^ j));
  return __clzll(a ^ b);
}
// Internal nodes 0..n-2; leaf j is node n-1+j. child[2i..2i+1], parent[], range[2i..2i+1].
__global__ void k_karras(const unsigned long long* __restrict__ k, int n, int* __restrict__ child,
                         int* __restrict__ parent, int* __restrict__ range) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n - 1) return;
  int d = (lcp_delta(k, n, i, i + 1) - lcp_delta(k, n, i, i - 1)) >= 0 ? 1 : -1;
  int dmin = lcp_delta(k, n, i, i - d);
  int lmax = 2;
  while (lcp_delta(k, n, i, i + lmax * d) > dmin && lmax < (1 << 30)) lmax <<= 1;
  int l = 0;
  for (int t = lmax >> 1; t >= 1; t >>= 1)
    if (lcp_delta(k, n, i, i + (l + t) * d) > dmin) l += t;
  int j = i + l * d;
  int dnode = lcp_delta(k, n, i, j);
  int s = 0, t = l;
  do {
    t = (t + 1) >> 1;
    if (lcp_delta(k, n, i, i + (s + t) * d) > dnode) s += t;
  } while (t > 1);
  int split = i + s * d + min(d, 0);
  int first = min(i, j), last = max(i, j);
  int left = (first == split) ? (n - 1 + split) : split;
  int right = (last == split + 1) ? (n - 1 + split + 1) : split + 1;
  child[2 * i] = left;
  child[2 * i + 1] = right;
  parent[left] = i;
  parent[right] = i;
  range[2 * i] = first;
  range[2 * i + 1] = last;
  if (i == 0) parent[0] = -1;
}
// Subtree root of every environment: the internal node whose leaf range is exactly the
// environment's primitive range, or the leaf itself for a single primitive.
__global__ void k_env_roots(int n, const int* __restrict__ range, const int* __restrict__ off, int n_env,
                            const int* __restrict__ penv, int* __restrict__ root) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n - 1) {
    int f = range[2 * i], l = range[2 * i + 1];
    int e = penv[f];
    if (off[e] == f && off[e + 1] - 1 == l) root[e] = i;
  }
  if (i < n_env) {
    if (off[i + 1] - off[i] == 1) root[i] = n - 1 + off[i];
  }
}

// Node boxes are FP32, rounded outward from the FP64 primitive boxes (min down, max up), as two
// float4 (lo, hi; w unused): a node box contains the exact box of everything below it, so a
// culling test on them never drops a pair whose FP64 boxes overlap. Leaves are decided by the
// exact FP64 test on the primitive boxes, so the candidate set is that of FP64 boxes.
DEV void round_box_out(const double* b, float4* out) {
  out[0] = make_float4(__double2float_rd(b[0]), __double2float_rd(b[1]), __double2float_rd(b[2]), 0.f);
  out[1] = make_float4(__double2float_ru(b[3]), __double2float_ru(b[4]), __double2float_ru(b[5]), 0.f);
}

// Refit: leaves take their primitive boxes (rounded outward); the second thread to reach an
// internal node writes the union of its children and continues upward. flags must be zero on
// entry.
__global__ void k_refit(int n, const unsigned* __restrict__ sorted, const double* __restrict__ pbox,
                        const int* __restrict__ child, const int* __restrict__ parent, float4* nbox,
                        int* __restrict__ flags) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  int leaf = n - 1 + j;
  round_box_out(pbox + 6 * (long)sorted[j], nbox + 2 * (long)leaf);
  int node = parent[leaf];
  while (node >= 0) {
    __threadfence();
    if (atomicAdd(&flags[node], 1) == 0) return;
    __threadfence();
    int a = child[2 * node], c = child[2 * node + 1];
    float4 alo = __ldcg(nbox + 2 * (long)a), ahi = __ldcg(nbox + 2 * (long)a + 1);
    float4 clo = __ldcg(nbox + 2 * (long)c), chi = __ldcg(nbox + 2 * (long)c + 1);
    nbox[2 * (long)node] = make_float4(fminf(alo.x, clo.x), fminf(alo.y, clo.y), fminf(alo.z, clo.z), 0.f);
    nbox[2 * (long)node + 1] = make_float4(fmaxf(ahi.x, chi.x), fmaxf(ahi.y, chi.y), fmaxf(ahi.z, chi.z), 0.f);
    node = parent[node];
  }
}

DEV bool box_overlap(const double* a, const double* b) {
  return a[0] <= b[3] && b[0] <= a[3] && a[1] <= b[4] && b[1] <= a[4] && a[2] <= b[5] && b[2] <= a[5];
}
DEV bool box_overlap_f(const float4& alo, const float4& ahi, const float4& blo, const float4& bhi) {
  return alo.x <= bhi.x && blo.x <= ahi.x && alo.y <= bhi.y && blo.y <= ahi.y && alo.z <= bhi.z && blo.z <= ahi.z;
}

constexpr int BVH_STACK = 64;

// Tree view passed to traversal kernels.
struct Tree {
  int n;                  // primitives
  const unsigned* sorted; // leaf j -> primitive
  const int* child;
  const float4* nbox;     // 2n-1 outward-rounded boxes (internal then leaves), 2 float4 each
  const double* pbox;     // exact primitive boxes (by primitive index)
  const int* root;        // per env
};

// Visit every primitive of env e whose box overlaps qbox; f(prim) is called in traversal order.
// Returns false if the stack overflowed (then the visit is incomplete).
// Visit every primitive j of env e with pre(j) true and an FP64 box overlapping qbox; f(j) is
// called once for each, in no particular order. Children are tested on their outward-rounded
// FP32 boxes before they are pushed; a leaf's exact FP64 test runs only after pre(j) and its FP32
// test pass. Returns false if the stack overflowed (then the visit is incomplete).
template <class P, class F>
DEV bool bvh_visit(const Tree& T, int e, const double* qbox, P&& pre, F&& f) {
  int r = T.root[e];
  if (r < 0) return true;
  float4 q[2];
  round_box_out(qbox, q);
  const int n1 = T.n - 1;
  auto leaf = [&](int node) {
    const int prim = (int)T.sorted[node - n1];
    if (pre(prim) && box_overlap(qbox, T.pbox + 6 * (long)prim)) f(prim);
  };
  if (!box_overlap_f(q[0], q[1], T.nbox[2 * (long)r], T.nbox[2 * (long)r + 1])) return true;
  if (r >= n1) {
    leaf(r);
    return true;
  }
  int stack[BVH_STACK];
  int sp = 0;
  stack[sp++] = r;
  while (sp > 0) {
    const int node = stack[--sp];
    const int c0 = T.child[2 * node], c1 = T.child[2 * node + 1];
    const bool o0 = box_overlap_f(q[0], q[1], T.nbox[2 * (long)c0], T.nbox[2 * (long)c0 + 1]);
    const bool o1 = box_overlap_f(q[0], q[1], T.nbox[2 * (long)c1], T.nbox[2 * (long)c1 + 1]);
    if (o1) {
      if (c1 >= n1) leaf(c1);
      else if (sp < BVH_STACK) stack[sp++] = c1;
      else return false;
    }
    if (o0) {
      if (c0 >= n1) leaf(c0);
      else if (sp < BVH_STACK) stack[sp++] = c0;
      else return false;
    }
  }
  return true;
}
template <class F>
DEV bool bvh_visit(const Tree& T, int e, const double* qbox, F&& f) {
  return bvh_visit(T, e, qbox, [](int) { return true; }, f);
}
