// Device helpers shared by the sm_103a kernels: 3-vector math, order-preserving atomics on
// non-negative doubles, small symmetric eigensolvers and inverses.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <math.h>

#define DEV __device__ __forceinline__
#define HD __host__ __device__ __forceinline__

struct d3 {
  double x, y, z;
};
HD d3 mk3(double a, double b, double c) { return d3{a, b, c}; }
HD d3 operator+(d3 a, d3 b) { return d3{a.x + b.x, a.y + b.y, a.z + b.z}; }
HD d3 operator-(d3 a, d3 b) { return d3{a.x - b.x, a.y - b.y, a.z - b.z}; }
HD d3 operator*(double s, d3 a) { return d3{s * a.x, s * a.y, s * a.z}; }
HD double dot(d3 a, d3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
HD d3 cross(d3 a, d3 b) { return d3{a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }
HD double comp(d3 a, int k) { return k == 0 ? a.x : (k == 1 ? a.y : a.z); }

DEV d3 ld3(const double* __restrict__ p, long i) { return d3{p[3 * i], p[3 * i + 1], p[3 * i + 2]}; }
DEV void st3(double* __restrict__ p, long i, d3 v) {
  p[3 * i] = v.x;
  p[3 * i + 1] = v.y;
  p[3 * i + 2] = v.z;
}

// Exactly rounded a + b*c without contraction into an FMA.
DEV double add_mul_rn(double a, double b, double c) { return __dadd_rn(a, __dmul_rn(b, c)); }

// Non-negative doubles order like their bit patterns: atomic min/max on the bits is exact and
// independent of arrival order.
DEV void atomic_min_pos(unsigned long long* a, double v) {
  atomicMin(a, (unsigned long long)__double_as_longlong(v));
}
DEV void atomic_max_pos(unsigned long long* a, double v) {
  atomicMax(a, (unsigned long long)__double_as_longlong(v));
}
HD double bits_to_double(unsigned long long b) {
  union {
    unsigned long long u;
    double d;
  } c;
  c.u = b;
  return c.d;
}
// Order-preserving map of any double to uint64 (for min/max of signed values).
DEV unsigned long long ordered_bits(double v) {
  unsigned long long b = (unsigned long long)__double_as_longlong(v);
  return (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
}
HD double ordered_to_double(unsigned long long b) {
  unsigned long long r = (b & 0x8000000000000000ull) ? (b & 0x7fffffffffffffffull) : ~b;
  return bits_to_double(r);
}

// Packed upper-triangle index of (i, j), i <= j, in an n x n symmetric matrix.
HD int up_idx(int i, int j, int n) { return i * n - i * (i - 1) / 2 + (j - i); }
HD int sym_idx(int i, int j, int n) { return i <= j ? up_idx(i, j, n) : up_idx(j, i, n); }

// Squared relative size of the off-diagonal part at which the Jacobi sweeps below stop.
template <class T>
struct JacobiTol;
template <>
struct JacobiTol<double> {
  static constexpr double psd = 1e-28, eig3 = 1e-30;
};
template <>
struct JacobiTol<float> {
  static constexpr float psd = 1e-13f, eig3 = 1e-13f;
};

// Cyclic Jacobi on a symmetric N x N matrix held in A (row-major, thread-local), in the
// precision T. On return A holds the PSD projection V max(Lambda, 0) V^T. At most 24 sweeps
// (a fixed bound).
// Kept out of line: inlined into kernels that hold other large local arrays, the device
// optimizer produced wrong results for this routine (measured on sm_103a with CUDA 13.0).
template <int N, class T = double>
__device__ __noinline__ void project_psd_jacobi(T* A) {
  T V[N * N];
#pragma unroll 1
  for (int i = 0; i < N * N; ++i) V[i] = T(0);
#pragma unroll 1
  for (int i = 0; i < N; ++i) V[i * N + i] = T(1);
  T fro = T(0);
#pragma unroll 1
  for (int i = 0; i < N * N; ++i) fro += A[i] * A[i];
  if (fro == T(0)) return;
  const T tol = JacobiTol<T>::psd * fro;
#pragma unroll 1
  for (int sweep = 0; sweep < 24; ++sweep) {
    T off = T(0);
#pragma unroll 1
    for (int i = 0; i < N; ++i)
#pragma unroll 1
      for (int j = i + 1; j < N; ++j) off += T(2) * A[i * N + j] * A[i * N + j];
    if (off <= tol) break;
#pragma unroll 1
    for (int p = 0; p < N - 1; ++p) {
#pragma unroll 1
      for (int q = p + 1; q < N; ++q) {
        T apq = A[p * N + q];
        if (apq == T(0)) continue;
        T app = A[p * N + p], aqq = A[q * N + q];
        T theta = (aqq - app) / (T(2) * apq);
        T t = (theta >= T(0) ? T(1) : T(-1)) / (fabs(theta) + sqrt(theta * theta + T(1)));
        T c = rsqrt(t * t + T(1)), s = t * c;
#pragma unroll 1
        for (int k = 0; k < N; ++k) {
          T akp = A[k * N + p], akq = A[k * N + q];
          A[k * N + p] = c * akp - s * akq;
          A[k * N + q] = s * akp + c * akq;
        }
#pragma unroll 1
        for (int k = 0; k < N; ++k) {
          T apk = A[p * N + k], aqk = A[q * N + k];
          A[p * N + k] = c * apk - s * aqk;
          A[q * N + k] = s * apk + c * aqk;
        }
#pragma unroll 1
        for (int k = 0; k < N; ++k) {
          T vkp = V[k * N + p], vkq = V[k * N + q];
          V[k * N + p] = c * vkp - s * vkq;
          V[k * N + q] = s * vkp + c * vkq;
        }
      }
    }
  }
  T lam[N];
#pragma unroll 1
  for (int i = 0; i < N; ++i) lam[i] = A[i * N + i];
  // rebuild only the clamped part: A_proj = sum_k max(lam_k, 0) v_k v_k^T
#pragma unroll 1
  for (int i = 0; i < N; ++i)
#pragma unroll 1
    for (int j = i; j < N; ++j) {
      T s = T(0);
#pragma unroll 1
      for (int k = 0; k < N; ++k)
        if (lam[k] > T(0)) s += V[i * N + k] * lam[k] * V[j * N + k];
      A[i * N + j] = s;
      A[j * N + i] = s;
    }
}

// Half-warp-parallel cyclic Jacobi with round-robin ordering (Brent & Luk 1985): each round
// applies N/2 disjoint plane rotations at once, computed from the same matrix, and N - 1 rounds
// make a sweep over all N (N - 1) / 2 pairs. A and V are N x N row-major arrays in shared memory
// owned by the calling half-warp (lanes hw_lane = 0..15, mask = its 16 lanes); rot holds 3N
// values of scratch. On return A holds the PSD projection V max(Lambda, 0) V^T (sweeps stop when
// the off-diagonal part is below JacobiTol<T>::psd of the Frobenius norm, 24 at most). N is even
// and at most 16; pad odd sizes with a zero row and column.
template <int N, class T>
DEV void project_psd_hw(T* A, T* V, T* rot, int hw_lane, unsigned mask) {
  static_assert(N % 2 == 0 && N <= 16, "N must be even and at most 16");
  constexpr int NE = (N * N + 15) / 16;  // elements per lane
  T* alpha = rot;          // coefficient of column i in the new column i
  T* beta = rot + N;       // coefficient of its partner column
  int* partner = (int*)(rot + 2 * N);
  for (int e = hw_lane; e < N * N; e += 16) V[e] = (e / N == e % N) ? T(1) : T(0);
  T fro = T(0);
  for (int e = hw_lane; e < N * N; e += 16) fro += A[e] * A[e];
  for (int o = 8; o > 0; o >>= 1) fro += __shfl_xor_sync(mask, fro, o);
  __syncwarp(mask);
  if (fro == T(0)) return;
  const T tol = JacobiTol<T>::psd * fro;
  for (int sweep = 0; sweep < 24; ++sweep) {
    T off = T(0);
    for (int e = hw_lane; e < N * N; e += 16)
      if (e / N < e % N) off += T(2) * A[e] * A[e];
    for (int o = 8; o > 0; o >>= 1) off += __shfl_xor_sync(mask, off, o);
    if (off <= tol) break;
    for (int r = 0; r < N - 1; ++r) {
      if (hw_lane < N / 2) {  // pair k = hw_lane of round r
        const int k = hw_lane;
        int a = k == 0 ? 0 : 1 + (r + k) % (N - 1);
        int b = k == 0 ? 1 + r % (N - 1) : 1 + (r - k + N - 1) % (N - 1);
        const int p = a < b ? a : b, q = a < b ? b : a;
        const T apq = A[p * N + q];
        T c = T(1), sn = T(0);
        if (apq != T(0)) {
          const T app = A[p * N + p], aqq = A[q * N + q];
          const T theta = (aqq - app) / (T(2) * apq);
          const T t = (theta >= T(0) ? T(1) : T(-1)) / (fabs(theta) + sqrt(theta * theta + T(1)));
          c = rsqrt(t * t + T(1));
          sn = t * c;
        }
        // new column p = c col_p - s col_q, new column q = s col_p + c col_q
        alpha[p] = c;
        beta[p] = -sn;
        partner[p] = q;
        alpha[q] = c;
        beta[q] = sn;
        partner[q] = p;
      }
      __syncwarp(mask);
      T na[NE], nv[NE];
#pragma unroll
      for (int u = 0; u < NE; ++u) {
        const int e = hw_lane + 16 * u;
        if (e < N * N) {
          const int i = e / N, j = e % N, i2 = partner[i], j2 = partner[j];
          const T ai = alpha[i], bi = beta[i], aj = alpha[j], bj = beta[j];
          na[u] = ai * (aj * A[i * N + j] + bj * A[i * N + j2]) + bi * (aj * A[i2 * N + j] + bj * A[i2 * N + j2]);
          nv[u] = aj * V[i * N + j] + bj * V[i * N + j2];
        }
      }
      __syncwarp(mask);
#pragma unroll
      for (int u = 0; u < NE; ++u) {
        const int e = hw_lane + 16 * u;
        if (e < N * N) {
          A[e] = na[u];
          V[e] = nv[u];
        }
      }
      __syncwarp(mask);
    }
  }
  // A_proj = sum_k max(lam_k, 0) v_k v_k^T, lam_k = A[k][k]
  T out[NE];
#pragma unroll
  for (int u = 0; u < NE; ++u) {
    const int e = hw_lane + 16 * u;
    out[u] = T(0);
    if (e < N * N) {
      const int i = e / N, j = e % N;
      for (int k = 0; k < N; ++k) {
        const T lk = A[k * N + k];
        if (lk > T(0)) out[u] += V[i * N + k] * lk * V[j * N + k];
      }
    }
  }
  __syncwarp(mask);
#pragma unroll
  for (int u = 0; u < NE; ++u) {
    const int e = hw_lane + 16 * u;
    if (e < N * N) A[e] = out[u];
  }
  __syncwarp(mask);
}

// The same round-robin Jacobi by a whole thread block: every thread updates the matrix
// elements e = threadIdx.x, threadIdx.x + blockDim.x (N * N <= 2 blockDim) of each round, three
// block barriers per round. For kernels with few matrices and latency to hide (a few hundred
// contacts per Newton iteration). A, V (N x N) and rot (3N) in shared memory; every thread of the
// block calls it. FROM_V: V already holds an orthonormal basis to continue from (else V = I).
// PROJECT: on return A = V max(Lambda, 0) V^T (else A is left diagonalised, V its eigenvectors).
// Sweeps stop when the off-diagonal part is below tol_rel of the Frobenius norm (squared), or
// after max_sweeps.
template <int N, class T, bool FROM_V, bool PROJECT>
DEV void jacobi_block(T* A, T* V, T* rot, T tol_rel = JacobiTol<T>::psd, int max_sweeps = 24) {
  static_assert(N % 2 == 0, "N must be even");
  const int t = threadIdx.x, nt = blockDim.x;
  T* alpha = rot;
  T* beta = rot + N;
  int* partner = (int*)(rot + 2 * N);
  __shared__ T red[32];
  if (!FROM_V)
    for (int e = t; e < N * N; e += nt) V[e] = (e / N == e % N) ? T(1) : T(0);
  // sums over the matrix: per-warp butterflies, warps added in order (same value in every thread)
  auto block_sum2 = [&](T v) -> T {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((t & 31) == 0) red[t >> 5] = v;
    __syncthreads();
    T s = T(0);
    for (int w = 0; w < (nt + 31) / 32; ++w) s += red[w];
    __syncthreads();
    return s;
  };
  T fro = T(0);
  for (int e = t; e < N * N; e += nt) fro += A[e] * A[e];
  fro = block_sum2(fro);
  if (fro == T(0)) return;
  const T tol = tol_rel * fro;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    T off = T(0);
    for (int e = t; e < N * N; e += nt)
      if (e / N < e % N) off += T(2) * A[e] * A[e];
    off = block_sum2(off);
    if (off <= tol) break;
    for (int r = 0; r < N - 1; ++r) {
      if (t < N / 2) {
        const int k = t;
        int a = k == 0 ? 0 : 1 + (r + k) % (N - 1);
        int b = k == 0 ? 1 + r % (N - 1) : 1 + (r - k + N - 1) % (N - 1);
        const int p = a < b ? a : b, q = a < b ? b : a;
        const T apq = A[p * N + q];
        T c = T(1), sn = T(0);
        if (apq != T(0)) {
          const T app = A[p * N + p], aqq = A[q * N + q];
          const T theta = (aqq - app) / (T(2) * apq);
          const T tt = (theta >= T(0) ? T(1) : T(-1)) / (fabs(theta) + sqrt(theta * theta + T(1)));
          c = rsqrt(tt * tt + T(1));
          sn = tt * c;
        }
        alpha[p] = c;
        beta[p] = -sn;
        partner[p] = q;
        alpha[q] = c;
        beta[q] = sn;
        partner[q] = p;
      }
      __syncthreads();
      T na[2], nv[2];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int e = t + u * nt;
        if (e < N * N) {
          const int i = e / N, j = e % N, i2 = partner[i], j2 = partner[j];
          const T ai = alpha[i], bi = beta[i], aj = alpha[j], bj = beta[j];
          na[u] = ai * (aj * A[i * N + j] + bj * A[i * N + j2]) + bi * (aj * A[i2 * N + j] + bj * A[i2 * N + j2]);
          nv[u] = aj * V[i * N + j] + bj * V[i * N + j2];
        }
      }
      __syncthreads();
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int e = t + u * nt;
        if (e < N * N) {
          A[e] = na[u];
          V[e] = nv[u];
        }
      }
      __syncthreads();
    }
  }
  if (!PROJECT) return;
  T out[2];
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const int e = t + u * nt;
    out[u] = T(0);
    if (e < N * N) {
      const int i = e / N, j = e % N;
      for (int k = 0; k < N; ++k) {
        const T lk = A[k * N + k];
        if (lk > T(0)) out[u] += V[i * N + k] * lk * V[j * N + k];
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const int e = t + u * nt;
    if (e < N * N) A[e] = out[u];
  }
  __syncthreads();
}

// FP64 PSD projection of the symmetric N x N matrix A by a thread block, warm-started in FP32:
// Jacobi sweeps in FP32 give an approximate eigenbasis; one Newton-Schulz step
// V <- V (3 I - V^T V) / 2 makes it orthonormal in FP64, A is rotated into it (V^T A V, nearly
// diagonal), and FP64 Jacobi sweeps from there (quadratic convergence: one or two) finish the
// eigen-decomposition to the FP64 tolerance. The result is the FP64 projection; the FP32 stage only
// saves FP64 rotations. Shared arrays: A, V, W (N x N doubles), rot (3N doubles), Af, Vf (N x N
// floats), rotf (3N floats).
template <int N>
DEV void project_psd_block_warm(double* A, double* V, double* W, double* rot, float* Af, float* Vf, float* rotf) {
  const int t = threadIdx.x, nt = blockDim.x;
  for (int e = t; e < N * N; e += nt) Af[e] = float(A[e]);
  __syncthreads();
  // FP32 stops where its rounding floor starts (off-diagonal ~3e-6 of the norm, at most 12 sweeps)
  jacobi_block<N, float, false, false>(Af, Vf, rotf, 1e-11f, 12);
  for (int e = t; e < N * N; e += nt) V[e] = double(Vf[e]);
  __syncthreads();
  // W = V^T V
  for (int e = t; e < N * N; e += nt) {
    const int i = e / N, j = e % N;
    double s = 0.0;
    for (int k = 0; k < N; ++k) s += V[k * N + i] * V[k * N + j];
    W[e] = s;
  }
  __syncthreads();
  double nv[2];
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const int e = t + u * nt;
    if (e < N * N) {
      const int i = e / N, j = e % N;
      double s = 0.0;
      for (int k = 0; k < N; ++k) s += V[i * N + k] * ((k == j ? 3.0 : 0.0) - W[k * N + j]);
      nv[u] = 0.5 * s;
    }
  }
  __syncthreads();
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const int e = t + u * nt;
    if (e < N * N) V[e] = nv[u];
  }
  __syncthreads();
  // A <- V^T A V (W = A V first), symmetrised
  for (int e = t; e < N * N; e += nt) {
    const int i = e / N, j = e % N;
    double s = 0.0;
    for (int k = 0; k < N; ++k) s += A[i * N + k] * V[k * N + j];
    W[e] = s;
  }
  __syncthreads();
  double nb[2];
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const int e = t + u * nt;
    if (e < N * N) {
      const int i = e / N, j = e % N;
      double s1 = 0.0, s2 = 0.0;
      for (int k = 0; k < N; ++k) {
        s1 += V[k * N + i] * W[k * N + j];
        s2 += V[k * N + j] * W[k * N + i];
      }
      nb[u] = 0.5 * (s1 + s2);
    }
  }
  __syncthreads();
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const int e = t + u * nt;
    if (e < N * N) A[e] = nb[u];
  }
  __syncthreads();
  jacobi_block<N, double, true, true>(A, V, rot);
}

// Symmetric 3x3 eigen-decomposition by cyclic Jacobi in the precision T: A (row-major) ->
// eigenvalues w and eigenvector columns of V (det V = +1).
template <class T>
DEV void eig_sym3(const T A_in[9], T w[3], T V[9]) {
  T A[9];
  for (int i = 0; i < 9; ++i) A[i] = A_in[i];
  for (int i = 0; i < 9; ++i) V[i] = (i % 4 == 0) ? T(1) : T(0);
  T fro = T(0);
  for (int i = 0; i < 9; ++i) fro += A[i] * A[i];
#pragma unroll 1
  for (int sweep = 0; sweep < 16; ++sweep) {
    T off = T(2) * (A[1] * A[1] + A[2] * A[2] + A[5] * A[5]);
    if (off <= JacobiTol<T>::eig3 * fro || off == T(0)) break;
#pragma unroll
    for (int pq = 0; pq < 3; ++pq) {
      const int p = pq == 2 ? 1 : 0;
      const int q = pq == 0 ? 1 : 2;
      T apq = A[p * 3 + q];
      if (apq == T(0)) continue;
      T app = A[p * 3 + p], aqq = A[q * 3 + q];
      T theta = (aqq - app) / (T(2) * apq);
      T t = (theta >= T(0) ? T(1) : T(-1)) / (fabs(theta) + sqrt(theta * theta + T(1)));
      T c = rsqrt(t * t + T(1)), s = t * c;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        T akp = A[k * 3 + p], akq = A[k * 3 + q];
        A[k * 3 + p] = c * akp - s * akq;
        A[k * 3 + q] = s * akp + c * akq;
      }
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        T apk = A[p * 3 + k], aqk = A[q * 3 + k];
        A[p * 3 + k] = c * apk - s * aqk;
        A[q * 3 + k] = s * apk + c * aqk;
      }
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        T vkp = V[k * 3 + p], vkq = V[k * 3 + q];
        V[k * 3 + p] = c * vkp - s * vkq;
        V[k * 3 + q] = s * vkp + c * vkq;
      }
    }
  }
  w[0] = A[0];
  w[1] = A[4];
  w[2] = A[8];
  T det = V[0] * (V[4] * V[8] - V[5] * V[7]) - V[1] * (V[3] * V[8] - V[5] * V[6]) + V[2] * (V[3] * V[7] - V[4] * V[6]);
  if (det < T(0)) {
    V[2] = -V[2];
    V[5] = -V[5];
    V[8] = -V[8];
  }
}

// 3x3 symmetric positive-definite inverse by the adjugate (row-major); zero if not invertible.
template <class T>
DEV void inv_sym3(const T* M, T* R) {
  T a = M[0], b = M[1], c = M[2], d = M[4], e = M[5], f = M[8];
  T A = d * f - e * e, B = c * e - b * f, C = b * e - c * d;
  T det = a * A + b * B + c * C;
  if (!(det > T(0)) || !isfinite(det)) {
    for (int i = 0; i < 9; ++i) R[i] = T(0);
    if (a > 0) R[0] = T(1) / a;
    if (d > 0) R[4] = T(1) / d;
    if (f > 0) R[8] = T(1) / f;
    return;
  }
  T id = T(1) / det;
  R[0] = A * id;
  R[1] = B * id;
  R[2] = C * id;
  R[3] = B * id;
  R[4] = (a * f - c * c) * id;
  R[5] = (b * c - a * e) * id;
  R[6] = C * id;
  R[7] = (b * c - a * e) * id;
  R[8] = (a * d - b * b) * id;
}

// Block-wide sum of one double per thread in fixed order (deterministic). blockDim <= 1024.
DEV double block_sum(double v, double* sh) {
  const int t = threadIdx.x;
  sh[t] = v;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (t < s) sh[t] += sh[t + s];
    __syncthreads();
  }
  double r = sh[0];
  __syncthreads();
  return r;
}
