// Device-side helpers shared by the Wilson-loop kernels: a small complex type,
// the sticky status word, and the device view of a hopping-list plan.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace bw {

template <typename T>
struct __align__(2 * sizeof(T)) cx {
  T re, im;
  cx() = default;
  __host__ __device__ constexpr cx(T r, T i = T(0)) : re(r), im(i) {}
};

template <typename T>
__host__ __device__ __forceinline__ cx<T> operator+(cx<T> a, cx<T> b) {
  return cx<T>(a.re + b.re, a.im + b.im);
}
template <typename T>
__host__ __device__ __forceinline__ cx<T> operator-(cx<T> a, cx<T> b) {
  return cx<T>(a.re - b.re, a.im - b.im);
}
template <typename T>
__host__ __device__ __forceinline__ cx<T> operator-(cx<T> a) {
  return cx<T>(-a.re, -a.im);
}
template <typename T>
__host__ __device__ __forceinline__ cx<T> operator*(cx<T> a, cx<T> b) {
  return cx<T>(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <typename T>
__host__ __device__ __forceinline__ cx<T> operator*(T s, cx<T> a) {
  return cx<T>(s * a.re, s * a.im);
}
template <typename T>
__host__ __device__ __forceinline__ cx<T> conj(cx<T> a) {
  return cx<T>(a.re, -a.im);
}
template <typename T>
__host__ __device__ __forceinline__ T abs2(cx<T> a) {
  return a.re * a.re + a.im * a.im;
}
// acc += conj(a) * b
template <typename T>
__host__ __device__ __forceinline__ void cfma_conj(cx<T>& acc, cx<T> a, cx<T> b) {
  acc.re += a.re * b.re + a.im * b.im;
  acc.im += a.re * b.im - a.im * b.re;
}
// acc += a * b
template <typename T>
__host__ __device__ __forceinline__ void cfma(cx<T>& acc, cx<T> a, cx<T> b) {
  acc.re += a.re * b.re - a.im * b.im;
  acc.im += a.re * b.im + a.im * b.re;
}
template <typename To, typename Ti>
__host__ __device__ __forceinline__ cx<To> ccast(cx<Ti> a) {
  return cx<To>(To(a.re), To(a.im));
}

typedef cx<double> z64;
typedef cx<float> c32;

// Status codes (mirror bw_status).
enum : int {
  ST_OK = 0, ST_EINVAL = 1, ST_ENOMEM = 2, ST_EGAP = 3, ST_EPSOGAP = 4, ST_EWANGAP = 5,
  ST_ENOCONV = 6, ST_ETIMEOUT = 7, ST_ECUDA = 8
};

// Sticky device status: the first error wins, its k index and a value are kept.
struct DevStatus {
  int code;
  int pad;
  long long k_index;
  double value;
};

__device__ __forceinline__ void report(DevStatus* st, int code, long long k, double v) {
  if (atomicCAS(&st->code, 0, code) == 0) {
    st->k_index = k;
    st->value = v;
  }
}

// Device view of a hopping-list plan: entries are the distinct (row, col) pairs of
// H, each owning a contiguous segment of hoppings (amplitude and translation id).
struct DevModel {
  int n;
  int n_R;            // distinct translations
  int n_ent;          // distinct (row, col) pairs
  int n_hop;          // grouped hoppings (ent_start[n_ent])
  const int* Rv;      // n_R x 3
  const int* ent_row;
  const int* ent_col;
  const int* ent_start;  // n_ent + 1
  const int* hop_r;      // translation id per hopping (sorted by entry)
  const z64* hop_t;
  const float* hop_tdf;  // hop_t as double-float pairs: (re hi, re lo, im hi, im lo)
};

// Sparse operator (spin operator): entries (row, col, value).
struct DevOp {
  int nnz;
  const int* row;
  const int* col;
  const z64* val;
};

// Plane parameters passed by value.
// A stack of N_s parallel planes: row i (0 <= i < N_t = N_s N_tp) is transverse point
// it = i mod N_tp of plane s = i / N_tp, whose origin is moved by (s / N_s) sweep
// (an integer reciprocal vector).  One plane: N_s = 1, N_tp = N_t, sweep = 0.
struct DevPlane {
  double origin[3];
  double loop_dir[3];
  double trans_dir[3];
  int N, N_t;
  int N_s, N_tp;
  int sweep[3];
};

__device__ __forceinline__ void plane_f(const DevPlane& pl, int i, int j, double f[3]) {
  const double a = double(j) / double(pl.N);
  if (pl.N_s > 1) {
    const int s = i / pl.N_tp, it = i - s * pl.N_tp;
    const double b = double(it) / double(pl.N_tp), c = double(s) / double(pl.N_s);
    for (int d = 0; d < 3; ++d)
      f[d] = pl.origin[d] + a * pl.loop_dir[d] + b * pl.trans_dir[d] + c * double(pl.sweep[d]);
    return;
  }
  const double b = double(i) / double(pl.N_t);
  for (int d = 0; d < 3; ++d) f[d] = pl.origin[d] + a * pl.loop_dir[d] + b * pl.trans_dir[d];
}

// Index m of exp(i 2pi m / N_t) for the transverse and sweep part of the Bloch phase of
// a translation at row i (integer trans_dir and sweep): tq = trans_dir . R, sq =
// sweep . R; (it tq / N_tp + s sq / N_s) = (it tq N_s + s sq N_tp) / N_t.
__host__ __device__ __forceinline__ long long plane_row_index(const DevPlane& pl, int i, int tq, int sq) {
  if (pl.N_s <= 1) return (long long)i * tq;
  const int s = i / pl.N_tp, it = i - s * pl.N_tp;
  return (long long)it * tq * pl.N_s + (long long)s * sq * pl.N_tp;
}

// exp(i 2 pi f . R), argument reduced exactly by sincospi.
__device__ __forceinline__ z64 bloch_phase(const double f[3], const int* R) {
  const double x = f[0] * double(R[0]) + f[1] * double(R[1]) + f[2] * double(R[2]);
  double s, c;
  sincospi(2.0 * x, &s, &c);
  return z64(c, s);
}

// Block-wide sum of one double per thread; `red` holds >= blockDim.x / 32 doubles.
__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  for (int k = 0; k < nw; ++k) s += red[k];
  __syncthreads();
  return s;
}

__device__ __forceinline__ double block_min(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[w] = v;
  __syncthreads();
  double s = red[0];
  for (int k = 1; k < nw; ++k) s = fmin(s, red[k]);
  __syncthreads();
  return s;
}

// In-place lower Cholesky factor of the Hermitian p x p matrix G (row-major, lower
// triangle read and overwritten: G = L L^dagger), by the first warp of the CTA,
// column by column with the lanes along the rows.  *flag = 0 when a pivot is not
// positive.  Every thread must call it; it ends with a block barrier.
__device__ inline void chol_lower_warp(z64* G, int p, int* flag) {
  const int tid = threadIdx.x, lane = tid & 31;
  if (tid == 0) *flag = 1;
  __syncthreads();
  if (tid < 32) {
    for (int j = 0; j < p; ++j) {
      double part = 0.0;
      for (int k = lane; k < j; k += 32) part += abs2(G[j * p + k]);
      for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
      const double d2 = G[j * p + j].re - part;
      if (!(d2 > 0.0) && lane == 0) *flag = 0;
      const double d = sqrt(fmax(d2, 1e-300));
      for (int i = j + 1 + lane; i < p; i += 32) {
        z64 v = G[i * p + j];
        for (int k = 0; k < j; ++k) v = v - G[i * p + k] * conj(G[j * p + k]);
        G[i * p + j] = (1.0 / d) * v;
      }
      __syncwarp();
      if (lane == 0) G[j * p + j] = z64(d, 0.0);
      __syncwarp();
    }
  }
  __syncthreads();
}

}  // namespace bw
