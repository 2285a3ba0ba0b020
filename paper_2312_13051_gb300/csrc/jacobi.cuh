// Block-wide two-sided Jacobi eigensolver for a Hermitian matrix in shared memory.
//
// Parallel cyclic Jacobi with round-robin pairing: each round rotates n/2 disjoint
// index pairs at once (rows first, then columns), n-1 rounds make a sweep, and
// sweeps repeat until the off-diagonal Frobenius norm falls below 8 eps ||A||_F.
// A complex 2x2 rotation J = [[c, s e^{i phi}], [-s e^{-i phi}, c]] annihilates
// A[p][q] = |b| e^{i phi}: with tau = (A_qq - A_pp) / (2|b|) and
// t = sign(tau) / (|tau| + sqrt(1 + tau^2)), c = 1/sqrt(1+t^2), s = t c, and
// A_pp -> A_pp - t|b|, A_qq -> A_qq + t|b|.  A rotation is skipped when
// |A_pq| <= 4 eps sqrt(|A_pp| |A_qq|) (negligible against its diagonal pair); a sweep
// without any rotation also ends the iteration.  Without that test, clusters of
// equal eigenvalues keep off-diagonal entries at the rounding level that no
// rotation removes, and a pure norm test may never be met in FP32.
#pragma once

#include "common.cuh"

namespace bw {

template <typename T>
struct JacRot {
  int p, q;
  T c, app, aqq;
  cx<T> sc;  // s e^{i phi}
};

template <typename T>
__device__ __forceinline__ T eps_of();
template <>
__device__ __forceinline__ double eps_of<double>() { return 2.220446049250313e-16; }
template <>
__device__ __forceinline__ float eps_of<float>() { return 1.1920929e-7f; }

// Round-robin pair k of round r over np (even) players; indices >= n are dummies.
__device__ __forceinline__ void rr_pair(int r, int k, int np, int& p, int& q) {
  const int m = np - 1;
  if (k == 0) {
    p = m;
    q = r;
  } else {
    p = (r + k) % m;
    q = (r - k + m) % m;
  }
  if (p > q) { int t = p; p = q; q = t; }
}

// Diagonalises A (n x n, leading dimension ld) in place and accumulates V = prod J.
// On return A's diagonal holds the eigenvalues (unsorted).  rot: >= n/2+1 JacRot
// slots; red: >= 32 doubles.  Returns the number of sweeps, or -1 without
// convergence after max_sweeps.  Every thread of the block must call it.
template <typename T>
__device__ int jacobi_eigh(cx<T>* A, cx<T>* V, int n, int ld, int max_sweeps, JacRot<T>* rot,
                           double* red) {
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int e = tid; e < n * n; e += nt) {
    const int r = e / n, c = e - r * n;
    V[r * ld + c] = cx<T>(T(r == c), T(0));
  }
  if (n == 1) {
    __syncthreads();
    return 0;
  }
  const int np = (n + 1) & ~1, npairs = np >> 1;
  // ||A||_F (invariant under the rotations)
  double fro = 0.0;
  for (int e = tid; e < n * n; e += nt) {
    const int r = e / n, c = e - r * n;
    fro += double(abs2(A[r * ld + c]));
  }
  fro = block_sum(fro, red);
  const double tol = 8.0 * double(eps_of<T>()) * sqrt(fro);
  __shared__ int s_rotated;
  for (int sweep = 0; sweep <= max_sweeps; ++sweep) {
    double off = 0.0;
    for (int e = tid; e < n * n; e += nt) {
      const int r = e / n, c = e - r * n;
      if (r != c) off += double(abs2(A[r * ld + c]));
    }
    off = block_sum(off, red);
    if (sqrt(off) <= tol || fro == 0.0) return sweep;
    if (sweep == max_sweeps) break;
    if (tid == 0) s_rotated = 0;
    __syncthreads();
    for (int r = 0; r < np - 1; ++r) {
      for (int k = tid; k < npairs; k += nt) {
        int p, q;
        rr_pair(r, k, np, p, q);
        JacRot<T> R;
        R.p = p;
        R.q = q;
        R.c = T(1);
        R.sc = cx<T>(T(0), T(0));
        R.app = T(0);
        R.aqq = T(0);
        if (q < n) {
          const cx<T> b = A[p * ld + q];
          const T ab = sqrt(abs2(b));
          const T a = A[p * ld + p].re, d = A[q * ld + q].re;
          R.app = a;
          R.aqq = d;
          if (ab > T(4) * eps_of<T>() * sqrt(fabs(a) * fabs(d)) && ab > T(0)) {
            s_rotated = 1;
            const T tau = (d - a) / (T(2) * ab);
            const T t = (tau >= T(0) ? T(1) : T(-1)) / (fabs(tau) + sqrt(T(1) + tau * tau));
            const T c = T(1) / sqrt(T(1) + t * t);
            const T s = t * c;
            R.c = c;
            R.sc = cx<T>(s * b.re / ab, s * b.im / ab);
            R.app = a - t * ab;
            R.aqq = d + t * ab;
          }
        } else {
          R.q = -1;  // dummy pair
        }
        rot[k] = R;
      }
      __syncthreads();
      // rows: A <- J^dagger A
      for (int e = tid; e < npairs * n; e += nt) {
        const int k = e / n, col = e - k * n;
        const JacRot<T> R = rot[k];
        if (R.q < 0 || (R.sc.re == T(0) && R.sc.im == T(0))) continue;
        const cx<T> ap = A[R.p * ld + col], aq = A[R.q * ld + col];
        A[R.p * ld + col] = R.c * ap - R.sc * aq;
        A[R.q * ld + col] = conj(R.sc) * ap + R.c * aq;
      }
      __syncthreads();
      // columns: A <- A J, V <- V J
      for (int e = tid; e < npairs * n; e += nt) {
        const int k = e / n, row = e - k * n;
        const JacRot<T> R = rot[k];
        if (R.q < 0 || (R.sc.re == T(0) && R.sc.im == T(0))) continue;
        const cx<T> ap = A[row * ld + R.p], aq = A[row * ld + R.q];
        A[row * ld + R.p] = R.c * ap - aq * conj(R.sc);
        A[row * ld + R.q] = ap * R.sc + R.c * aq;
        const cx<T> vp = V[row * ld + R.p], vq = V[row * ld + R.q];
        V[row * ld + R.p] = R.c * vp - vq * conj(R.sc);
        V[row * ld + R.q] = vp * R.sc + R.c * vq;
      }
      __syncthreads();
      for (int k = tid; k < npairs; k += nt) {
        const JacRot<T> R = rot[k];
        if (R.q < 0 || (R.sc.re == T(0) && R.sc.im == T(0))) continue;
        A[R.p * ld + R.q] = cx<T>(T(0), T(0));
        A[R.q * ld + R.p] = cx<T>(T(0), T(0));
        A[R.p * ld + R.p] = cx<T>(R.app, T(0));
        A[R.q * ld + R.q] = cx<T>(R.aqq, T(0));
      }
      __syncthreads();
    }
    if (!s_rotated) return sweep + 1;
  }
  return -1;
}

// Sort key that puts NaN after every number, so that ranks always form a
// permutation (NaN only appears when the input was not finite).
template <typename T>
__device__ __forceinline__ T rank_key(T x) { return isnan(x) ? T(INFINITY) : x; }

// order[rank] = index of the rank-th smallest diagonal entry (stable, NaN last).
template <typename T>
__device__ void sort_diag(const cx<T>* A, int n, int ld, int* order) {
  for (int a = threadIdx.x; a < n; a += blockDim.x) {
    const T la = rank_key(A[a * ld + a].re);
    int rank = 0;
    for (int b = 0; b < n; ++b) {
      const T lb = rank_key(A[b * ld + b].re);
      rank += (lb < la) || (lb == la && b < a);
    }
    order[rank] = a;
  }
  __syncthreads();
}

}  // namespace bw
