// Occupied states for large n (supercells, many-band models): Bloch Hamiltonian,
// Householder tridiagonalisation, bisection, inverse iteration, back-transform,
// and for the mixed path an FP64 Newton correction of the occupied block
// (Sec. I "exact diagonalization" at many k-points; Eq. 1 occupied bands).
//
// Each stage is its own kernel over a wave of W k-points, one CTA (or one thread
// per eigenpair) per k-point, with the wave's scratch in the context arena:
//   A[kw]   n x n complex, reduced in place; the unit Householder vectors u_c are
//           kept below the subdiagonal (column c, rows c+1..n-1)
//   dg, od  diagonal and |off-diagonal| of the real tridiagonal T' = D^dag T D
//   Dp      the unit phases D (x = Q D z maps eigenvectors z of T' to those of H)
//   lam, Z  eigenvalues (ascending) and eigenvectors of T' (Z[kw][row][col])
// T is the working precision of the reduction (double: FP64 path, float: mixed).
#include <float.h>

#include <algorithm>
#include <type_traits>

#include "ctagemm.cuh"
#include "df32.cuh"
#include "jacobi.cuh"
#include "launch.h"

namespace bw {

template <typename T>
__device__ __forceinline__ T lg_eps();
template <>
__device__ __forceinline__ double lg_eps<double>() { return 2.220446049250313e-16; }
template <>
__device__ __forceinline__ float lg_eps<float>() { return 1.1920929e-7f; }

// Warp-wide sum of a complex value.
template <typename T>
__device__ __forceinline__ cx<T> warp_csum(cx<T> v) {
  for (int o = 16; o > 0; o >>= 1) {
    v.re += __shfl_xor_sync(0xffffffffu, v.re, o);
    v.im += __shfl_xor_sync(0xffffffffu, v.im, o);
  }
  return v;
}


__device__ __forceinline__ void lg_kpoint(const LargeArgs& a, long long k, double f[3]) {
  if (a.f) {
    f[0] = a.f[3 * k]; f[1] = a.f[3 * k + 1]; f[2] = a.f[3 * k + 2];
  } else {
    const int i = int(k / a.plane.N), j = int(k - (long long)i * a.plane.N);
    plane_f(a.plane, i, j, f);
  }
}

__device__ __forceinline__ void split64(z64 x, c32& hi, c32& lo) {
  hi = c32(float(x.re), float(x.im));
  lo = c32(float(x.re - double(hi.re)), float(x.im - double(hi.im)));
}

// ---------------------------------------------------------------------------
// Stage 1: Bloch Hamiltonian of the wave's k-points (full Hermitian matrix).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_lg_build(LargeArgs a) {
  __shared__ __align__(16) unsigned char phs_raw[PHASE_CACHE * sizeof(z64)];
  z64* phs = reinterpret_cast<z64*>(phs_raw);
  const DevModel& md = a.model;
  const int n = a.n, tid = threadIdx.x, nt = blockDim.x;
  const int nRs = min(md.n_R, PHASE_CACHE);
  for (long long kw = blockIdx.x; kw < a.W; kw += gridDim.x) {
    if (a.Hin) {  // explicit matrix: lower triangle mirrored, FP64 entries kept for the refinement
      const z64* Hm = a.Hin + a.h_off[a.idx[a.k0 + kw]];
      cx<T>* A = reinterpret_cast<cx<T>*>(a.A) + kw * (long long)n * n;
      c32* He = a.Hent ? reinterpret_cast<c32*>(a.Hent + kw * (long long)n * n) : nullptr;
      for (int r = tid >> 5; r < n; r += nt >> 5)
        for (int q = tid & 31; q <= r; q += 32) {
          z64 h = Hm[(long long)r * n + q];
          if (q == r) h.im = 0.0;
          A[(long long)r * n + q] = ccast<T>(h);
          A[(long long)q * n + r] = ccast<T>(conj(h));
          if (He) {
            c32 hi, lo;
            split64(h, hi, lo);
            He[2 * ((long long)r * n + q)] = hi;
            He[2 * ((long long)r * n + q) + 1] = lo;
            split64(conj(h), hi, lo);
            He[2 * ((long long)q * n + r)] = hi;
            He[2 * ((long long)q * n + r) + 1] = lo;
          }
        }
      __syncthreads();
      continue;
    }
    const long long k = a.k0 + kw * (a.kstride > 0 ? a.kstride : 1);
    double f[3];
    lg_kpoint(a, k, f);
    cx<T>* A = reinterpret_cast<cx<T>*>(a.A) + kw * (long long)n * n;
    for (long long e = tid; e < (long long)n * n; e += nt) A[e] = cx<T>(T(0), T(0));
    if (a.Hent && md.hop_tdf) {
      // mixed path: entries in double-float on the FP32 pipe (FP64-grade for the
      // refinement's residual, the FP32 matrix is the high part)
      cdf* phd = reinterpret_cast<cdf*>(phs);
      for (int r = tid; r < nRs; r += nt) phd[r] = cdf_from(bloch_phase(f, md.Rv + 3 * r));
      __syncthreads();
      for (int e = tid; e < md.n_ent; e += nt) {
        cdf acc(df(0.f), df(0.f));
        for (int h = md.ent_start[e]; h < md.ent_start[e + 1]; ++h) {
          const int r = md.hop_r[h];
          const float* t4 = md.hop_tdf + 4 * h;
          acc = acc + cdf(df(t4[0], t4[1]), df(t4[2], t4[3])) *
                          (r < nRs ? phd[r] : cdf_from(bloch_phase(f, md.Rv + 3 * r)));
        }
        A[(long long)md.ent_row[e] * n + md.ent_col[e]] = cx<T>(T(acc.re.hi), T(acc.im.hi));
        c32* dst = reinterpret_cast<c32*>(a.Hent + kw * (long long)md.n_ent + e);
        dst[0] = c32(acc.re.hi, acc.im.hi);
        dst[1] = c32(acc.re.lo, acc.im.lo);
      }
      __syncthreads();
      continue;
    }
    for (int r = tid; r < nRs; r += nt) phs[r] = bloch_phase(f, md.Rv + 3 * r);
    __syncthreads();
    for (int e = tid; e < md.n_ent; e += nt) {
      z64 acc(0.0, 0.0);
      for (int h = md.ent_start[e]; h < md.ent_start[e + 1]; ++h) {
        const int r = md.hop_r[h];
        cfma(acc, md.hop_t[h], r < nRs ? phs[r] : bloch_phase(f, md.Rv + 3 * r));
      }
      A[(long long)md.ent_row[e] * n + md.ent_col[e]] = ccast<T>(acc);
      if (a.Hent) {  // FP64 entry as an unevaluated sum of two floats (hi, lo)
        c32 hi, lo;
        split64(acc, hi, lo);
        c32* dst = reinterpret_cast<c32*>(a.Hent + kw * (long long)md.n_ent + e);
        dst[0] = hi;
        dst[1] = lo;
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Stage 2: Householder reduction to tridiagonal form, one CTA per k-point.
// For column c, x = A[c+1:, c]; P = I - 2 u u^dagger with u ~ x - alpha e_1,
// alpha = -e^{i arg x_0} |x|, maps x to alpha e_1.  With p = A22 u, K = u^dag p
// and w = p - K u, the trailing block becomes A22 - 2 (u w^dag + w u^dag).
// The complex subdiagonal alpha_c is made real by D: D_0 = 1,
// D_{c+1} = D_c alpha_c / |alpha_c|, off-diagonal |alpha_c|.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_lg_tridiag(LargeArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int n = a.n, tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nwarp = nt >> 5;
  cx<T>* u = reinterpret_cast<cx<T>*>(smem);          // n
  cx<T>* w = u + n;                                   // n
  cx<T>* al = w + n;                                  // n   complex subdiagonal
  double* red = reinterpret_cast<double*>(al + n);    // 64
  __shared__ double s_nrm2, s_x0re, s_x0im;
  __shared__ int s_skip;
  for (long long kw = blockIdx.x; kw < a.W; kw += gridDim.x) {
    cx<T>* A = reinterpret_cast<cx<T>*>(a.A) + kw * (long long)n * n;
    T* dg = reinterpret_cast<T*>(a.dg) + kw * n;
    T* od = reinterpret_cast<T*>(a.od) + kw * n;
    cx<T>* Dp = reinterpret_cast<cx<T>*>(a.Dp) + kw * n;
    for (int c = 0; c + 2 < n; ++c) {
      const int m = n - c - 1;  // length of x
      double s = 0.0;
      for (int r = tid; r < m; r += nt) {
        const cx<T> x = A[(long long)(c + 1 + r) * n + c];
        u[r] = x;
        s += double(abs2(x));
      }
      s = block_sum(s, red);
      if (tid == 0) {
        s_nrm2 = s;
        s_x0re = double(u[0].re);
        s_x0im = double(u[0].im);
        s_skip = !(s - (s_x0re * s_x0re + s_x0im * s_x0im) > 0.0);
      }
      __syncthreads();
      const double nx = sqrt(s_nrm2), ax0 = hypot(s_x0re, s_x0im);
      if (s_skip) {  // already tridiagonal in this column: no reflection
        for (int r = tid; r < m; r += nt) A[(long long)(c + 1 + r) * n + c] = cx<T>(T(0), T(0));
        if (tid == 0) {
          al[c] = cx<T>(T(s_x0re), T(s_x0im));
          dg[c] = A[(long long)c * n + c].re;
        }
        __syncthreads();
        continue;
      }
      const double phr = ax0 > 0.0 ? s_x0re / ax0 : 1.0, phi = ax0 > 0.0 ? s_x0im / ax0 : 0.0;
      // v = x - alpha e1 with alpha = -ph |x|: v_0 = ph (|x0| + |x|); |v|^2 = (|x0|+|x|)^2 + tail
      const double tail = s_nrm2 - ax0 * ax0;
      const double v0m = ax0 + nx;
      const T inv = T(1.0 / sqrt(v0m * v0m + tail));
      __syncthreads();
      for (int r = tid; r < m; r += nt) {
        cx<T> v = u[r];
        if (r == 0) v = cx<T>(T(phr * v0m), T(phi * v0m));
        u[r] = inv * v;
      }
      __syncthreads();
      // p = A22 u: one warp per row, lanes along the row
      for (int r = warp; r < m; r += nwarp) {
        const cx<T>* row = A + (long long)(c + 1 + r) * n + (c + 1);
        cx<T> acc(T(0), T(0));
        for (int q = lane; q < m; q += 32) cfma(acc, row[q], u[q]);
        acc = warp_csum(acc);
        if (lane == 0) w[r] = acc;
      }
      __syncthreads();
      double kr = 0.0;
      for (int r = tid; r < m; r += nt) kr += double(u[r].re * w[r].re + u[r].im * w[r].im);
      kr = block_sum(kr, red);
      for (int r = tid; r < m; r += nt) w[r] = w[r] - T(kr) * u[r];
      __syncthreads();
      // A22 <- A22 - 2 (u w^dag + w u^dag)
      for (int r = warp; r < m; r += nwarp) {
        cx<T>* row = A + (long long)(c + 1 + r) * n + (c + 1);
        const cx<T> ur = u[r], wr = w[r];
        for (int q = lane; q < m; q += 32) row[q] = row[q] - T(2) * (ur * conj(w[q]) + wr * conj(u[q]));
      }
      if (tid == 0) {
        al[c] = cx<T>(T(-phr * nx), T(-phi * nx));
        dg[c] = A[(long long)c * n + c].re;
      }
      // keep u below the subdiagonal for the back-transform
      for (int r = tid; r < m; r += nt) A[(long long)(c + 1 + r) * n + c] = u[r];
      __syncthreads();
    }
    if (tid == 0) {
      if (n >= 2) {
        dg[n - 2] = A[(long long)(n - 2) * n + (n - 2)].re;
        al[n - 2] = A[(long long)(n - 1) * n + (n - 2)];
      }
      dg[n - 1] = A[(long long)(n - 1) * n + (n - 1)].re;
      // the last subdiagonal entry is not a reflector: clear it for the back-transform
      if (n >= 2) A[(long long)(n - 1) * n + (n - 2)] = cx<T>(T(0), T(0));
    }
    __syncthreads();
    // unit phases of the subdiagonal, then their prefix products (serial: cheap)
    for (int c = tid; c + 1 < n; c += nt) {
      const T aa = sqrt(abs2(al[c]));
      od[c] = aa;
      al[c] = aa > T(0) ? cx<T>(al[c].re / aa, al[c].im / aa) : cx<T>(T(1), T(0));
    }
    __syncthreads();
    if (tid == 0) {
      cx<T> dcur(T(1), T(0));
      Dp[0] = dcur;
      for (int c = 0; c + 1 < n; ++c) {
        dcur = dcur * al[c];
        Dp[c + 1] = dcur;
      }
      od[n - 1] = T(0);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Stage 2, lower-triangle form (used when its shared memory fits, see the launcher).
// Same reflectors and T' as k_lg_tridiag, one pass over the trailing lower triangle
// per column: the column c+1 of the updated matrix is formed first, its reflector
// u' built, and then the rank-2 update of step c and the product p' = A' u' of step
// c+1 run in the same sweep.  A' u' takes A'_rq u'_q from the stored lower triangle
// and conj(A'_rq) u'_r for the mirrored upper one; the mirrored terms go to one
// accumulator array per warp (lane-private entries: entry q of a warp's array is
// only touched by lane (q - lo) mod 32), summed over warps in a fixed order, so the
// result does not depend on scheduling.
// ---------------------------------------------------------------------------

// Turns xs[c+1..n) (column c below the diagonal) into the unit reflector u with
// (I - 2 u u^dag) x = alpha e_1 and returns alpha; u = 0 when nothing lies below the
// subdiagonal.  Block-wide.
// Block-wide sum in the working precision (FP32 for the mixed solve: GB300's FP64
// pipe is ~70x narrower, and these per-step reductions would otherwise cost as much
// as the sweep over the matrix).
template <typename T>
__device__ __forceinline__ T block_sum_t(T v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  T* r = reinterpret_cast<T*>(red);
  const int w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) r[w] = v;
  __syncthreads();
  T s = T(0);
  for (int k = 0; k < nw; ++k) s += r[k];
  __syncthreads();
  return s;
}

// Turns xs[c+1..n) (column c below the diagonal) into the unit reflector u with
// (I - 2 u u^dag) x = alpha e_1 and returns alpha; u = 0 when nothing lies below the
// subdiagonal.  Block-wide, in the working precision T.
template <typename T>
__device__ cx<T> lg_reflector(cx<T>* xs, int c, int n, double* red) {
  const int tid = threadIdx.x, nt = blockDim.x;
  T s = T(0);
  for (int r = c + 1 + tid; r < n; r += nt) s += abs2(xs[r]);
  s = block_sum_t(s, red);
  const cx<T> x0 = xs[c + 1];
  const T ax0 = sqrt(abs2(x0)), tail = s - ax0 * ax0;
  __syncthreads();
  if (!(tail > T(0))) {
    for (int r = c + 1 + tid; r < n; r += nt) xs[r] = cx<T>(T(0), T(0));
    __syncthreads();
    return x0;
  }
  const T nx = sqrt(s);
  const T phr = ax0 > T(0) ? x0.re / ax0 : T(1), phi = ax0 > T(0) ? x0.im / ax0 : T(0);
  const T v0m = ax0 + nx;
  const T inv = T(1) / sqrt(v0m * v0m + tail);
  for (int r = c + 1 + tid; r < n; r += nt) {
    const cx<T> v = r == c + 1 ? cx<T>(phr * v0m, phi * v0m) : xs[r];
    xs[r] = inv * v;
  }
  __syncthreads();
  return cx<T>(-phr * nx, -phi * nx);
}

// Rows and columns lo..n-1 of the lower triangle: with upd, A <- A - 2 (u w^dag + w u^dag);
// then pa = A u2 (pw: per-warp accumulators, stride n).  A warp takes RW rows at a
// time (r, r + nwarp, ...) and walks their columns together, so that RW loads per
// lane are in flight even when the rows are short.  Ends with pa complete.
template <typename T>
__device__ void lg_hpass(cx<T>* A, int n, int lo, bool upd, const cx<T>* u, const cx<T>* w,
                         const cx<T>* u2, cx<T>* pw, cx<T>* pa) {
  constexpr int RW = sizeof(T) == 4 ? 8 : 4;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  for (int e = threadIdx.x; e < nwarp * (n - lo); e += blockDim.x) {
    const int ww = e / (n - lo), q = lo + (e - ww * (n - lo));
    pw[ww * n + q] = cx<T>(T(0), T(0));
  }
  __syncthreads();
  cx<T>* acc_w = pw + warp * n;
  const cx<T> zero(T(0), T(0));
  for (int r0 = lo + warp; r0 < n; r0 += RW * nwarp) {
    int rr[RW];
    cx<T> ur[RW], wr[RW], u2r[RW], acc[RW];
    int rmax = r0;
#pragma unroll
    for (int i = 0; i < RW; ++i) {
      rr[i] = r0 + i * nwarp;
      const bool ok = rr[i] < n;
      if (ok) rmax = rr[i];
      ur[i] = ok && upd ? u[rr[i]] : zero;
      wr[i] = ok && upd ? w[rr[i]] : zero;
      u2r[i] = ok ? u2[rr[i]] : zero;
      acc[i] = zero;
      if (!ok) rr[i] = -1;
    }
    for (int q = lo + lane; q <= rmax; q += 32) {
      cx<T> v[RW];
#pragma unroll
      for (int i = 0; i < RW; ++i)
        v[i] = q <= rr[i] ? A[(long long)rr[i] * n + q] : zero;
      const cx<T> wq = upd ? w[q] : zero, uq = upd ? u[q] : zero, u2q = u2[q];
      cx<T> tq = zero;
#pragma unroll
      for (int i = 0; i < RW; ++i) {
        if (q > rr[i]) continue;
        cx<T> x = v[i];
        if (upd) {
          x = x - T(2) * (ur[i] * conj(wq) + wr[i] * conj(uq));
          if (q == rr[i]) x.im = T(0);
          A[(long long)rr[i] * n + q] = x;
        }
        cfma(acc[i], x, u2q);
        if (q < rr[i]) tq = tq + conj(x) * u2r[i];
      }
      acc_w[q] = acc_w[q] + tq;
    }
#pragma unroll
    for (int i = 0; i < RW; ++i) {
      const cx<T> t = warp_csum(acc[i]);
      // entry r belongs to lane (r - lo) mod 32 of this warp's array
      if (rr[i] >= 0 && lane == ((rr[i] - lo) & 31)) acc_w[rr[i]] = acc_w[rr[i]] + t;
    }
    __syncwarp();
  }
  __syncthreads();
  for (int q = lo + threadIdx.x; q < n; q += blockDim.x) {
    cx<T> t(T(0), T(0));
    for (int ww = 0; ww < nwarp; ++ww) t = t + pw[ww * n + q];
    pa[q] = t;
  }
  __syncthreads();
}

// w = p - (u^dag p) u on lo..n-1 (p in pa).
template <typename T>
__device__ void lg_make_w(const cx<T>* u, const cx<T>* pa, cx<T>* w, int lo, int n, double* red) {
  T kr = T(0);
  for (int r = lo + threadIdx.x; r < n; r += blockDim.x) kr += u[r].re * pa[r].re + u[r].im * pa[r].im;
  kr = block_sum_t(kr, red);
  for (int r = lo + threadIdx.x; r < n; r += blockDim.x) w[r] = pa[r] - kr * u[r];
  __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(512) k_lg_tridiag_h(LargeArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int n = a.n, tid = threadIdx.x, nt = blockDim.x;
  cx<T>* u = reinterpret_cast<cx<T>*>(smem);  // reflector of the current step
  cx<T>* w = u + n;
  cx<T>* u2 = w + n;                          // reflector of the next step
  cx<T>* pa = u2 + n;                         // A u2
  cx<T>* al = pa + n;                         // complex subdiagonal
  cx<T>* pw = al + n;                         // (blockDim / 32) x n per-warp accumulators
  double* red = reinterpret_cast<double*>(pw + (nt >> 5) * n);
  for (long long kw = blockIdx.x; kw < a.W; kw += gridDim.x) {
    cx<T>* A = reinterpret_cast<cx<T>*>(a.A) + kw * (long long)n * n;
    T* dg = reinterpret_cast<T*>(a.dg) + kw * n;
    T* od = reinterpret_cast<T*>(a.od) + kw * n;
    cx<T>* Dp = reinterpret_cast<cx<T>*>(a.Dp) + kw * n;
    // step 0: reflector of column 0 and p = A22 u
    for (int r = 1 + tid; r < n; r += nt) u[r] = A[(long long)r * n];
    __syncthreads();
    cx<T> alpha = lg_reflector(u, 0, n, red);
    if (tid == 0) {
      al[0] = alpha;
      dg[0] = A[0].re;
    }
    for (int r = 1 + tid; r < n; r += nt) A[(long long)r * n] = u[r];
    __syncthreads();
    lg_hpass<T>(A, n, 1, false, nullptr, nullptr, u, pw, pa);
    lg_make_w(u, pa, w, 1, n, red);
    for (int c = 0; c + 2 < n; ++c) {
      // column c+1 of A - 2 (u w^dag + w u^dag), rows c+1..n-1
      const cx<T> uc = u[c + 1], wc = w[c + 1];
      for (int r = c + 1 + tid; r < n; r += nt)
        u2[r] = A[(long long)r * n + c + 1] - T(2) * (u[r] * conj(wc) + w[r] * conj(uc));
      __syncthreads();
      if (tid == 0) dg[c + 1] = u2[c + 1].re;
      if (c + 3 == n) {  // last 2 x 2 block: its subdiagonal and diagonal, no reflector
        if (tid == 0) {
          al[n - 2] = u2[n - 1];
          const cx<T> un = u[n - 1], wn = w[n - 1];
          dg[n - 1] = A[(long long)(n - 1) * n + n - 1].re - T(4) * (un.re * wn.re + un.im * wn.im);
          A[(long long)(n - 1) * n + n - 2] = cx<T>(T(0), T(0));
        }
        __syncthreads();
        break;
      }
      alpha = lg_reflector(u2, c + 1, n, red);
      if (tid == 0) al[c + 1] = alpha;
      for (int r = c + 2 + tid; r < n; r += nt) A[(long long)r * n + c + 1] = u2[r];
      __syncthreads();
      lg_hpass<T>(A, n, c + 2, true, u, w, u2, pw, pa);
      lg_make_w(u2, pa, w, c + 2, n, red);
      for (int r = c + 2 + tid; r < n; r += nt) u[r] = u2[r];
      __syncthreads();
    }
    // unit phases of the subdiagonal, then their prefix products (serial: cheap)
    for (int c = tid; c + 1 < n; c += nt) {
      const T aa = sqrt(abs2(al[c]));
      od[c] = aa;
      al[c] = aa > T(0) ? cx<T>(al[c].re / aa, al[c].im / aa) : cx<T>(T(1), T(0));
    }
    __syncthreads();
    if (tid == 0) {
      cx<T> dcur(T(1), T(0));
      Dp[0] = dcur;
      for (int c = 0; c + 1 < n; ++c) {
        dcur = dcur * al[c];
        Dp[c + 1] = dcur;
      }
      od[n - 1] = T(0);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Stage 3: eigenvalues of T' by bisection on Sturm counts, one thread per
// (k-point, eigenvalue index), Gershgorin interval.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ int sturm_count(const T* dg, const T* od, int n, T x, T pivmin) {
  int cnt = 0;
  T q = dg[0] - x;
  if (fabs(q) < pivmin) q = -pivmin;
  cnt += q < T(0);
  for (int i = 1; i < n; ++i) {
    q = dg[i] - x - od[i - 1] * od[i - 1] / q;
    if (fabs(q) < pivmin) q = -pivmin;
    cnt += q < T(0);
  }
  return cnt;
}

template <typename T>
__device__ __forceinline__ void gershgorin(const T* dg, const T* od, int n, T& lo, T& hi, T& tn) {
  lo = T(INFINITY);
  hi = -T(INFINITY);
  tn = T(0);
  for (int i = 0; i < n; ++i) {
    const T r = (i > 0 ? od[i - 1] : T(0)) + (i + 1 < n ? od[i] : T(0));
    lo = fmin(lo, dg[i] - r);
    hi = fmax(hi, dg[i] + r);
    tn = fmax(tn, fabs(dg[i]) + r);
  }
}

template <typename T>
__global__ void k_lg_bisect(LargeArgs a) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= a.W * a.nval) return;
  const long long kw = t / a.nval;
  const int idx = int(t - kw * a.nval), n = a.n;
  const T* dg = reinterpret_cast<const T*>(a.dg) + kw * n;
  const T* od = reinterpret_cast<const T*>(a.od) + kw * n;
  T lo, hi, tn;
  gershgorin(dg, od, n, lo, hi, tn);
  const T span = fmax(hi - lo, T(1e-30));
  lo -= T(4) * lg_eps<T>() * span + T(1e-30);
  hi += T(4) * lg_eps<T>() * span + T(1e-30);
  const T pivmin = T(1e-30) * fmax(T(1), tn * tn);
  for (int it = 0; it < 96; ++it) {
    const T mid = T(0.5) * (lo + hi);
    if (!(mid > lo && mid < hi)) break;
    if (hi - lo <= T(2) * lg_eps<T>() * fmax(fabs(lo), fabs(hi))) break;
    if (sturm_count(dg, od, n, mid, pivmin) > idx)
      hi = mid;
    else
      lo = mid;
  }
  reinterpret_cast<T*>(a.lam)[kw * a.nval + idx] = T(0.5) * (lo + hi);
}

// ---------------------------------------------------------------------------
// Stage 4: eigenvectors of T' by inverse iteration.  (T' - lambda) = P L U with
// partial pivoting (U has two superdiagonals); three solves from a fixed
// pseudo-random start.  Eigenvalues closer than 1e-3 ||T'|| form a cluster, whose
// vectors one thread computes in order, orthogonalising each against the earlier
// ones of its cluster at every iteration.  Above INVIT_WINDOW_N, where the spectrum
// of a supercell is so dense that the chained clusters span most of it, a vector is
// orthogonalised only against the earlier ones within 1e-3 ||T'|| of its eigenvalue:
// two vectors further apart are orthogonal to ~eps ||T'|| / (1e-3 ||T'||) already, the
// bound the cluster rule accepts between clusters, and the cost per vector is O(n)
// instead of O(n x cluster size).
// Where only the span of the computed vectors matters (subspace_only: the PSO
// sector), every vector iterates on its own thread at once instead, converging into
// its cluster's invariant subspace from a distinct start, and a second kernel
// orthonormalises each cluster's vectors by modified Gram-Schmidt applied twice,
// one warp per cluster: a cluster of p/2 exactly degenerate PSO eigenvalues no
// longer serialises on one thread.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double hash_unit(unsigned long long x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  x ^= x >> 31;
  return double(x >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
}

// Interleaved per-thread arrays: element r of thread t's array a lives at
// base[(a * n + r) * NT + t], so a warp's accesses to the same r are contiguous.
template <typename T>
struct Strided {
  T* base;
  long long NT;
  int n;
  __device__ __forceinline__ T& at(int a, int r, long long t) const { return base[((long long)a * n + r) * NT + t]; }
};

template <typename T>
__device__ void tri_factor(const T* dg, const T* od, int n, T lam, T tiny, const Strided<T>& W,
                           long long t) {
  T c0 = dg[0] - lam, c1 = n > 1 ? od[0] : T(0);
  for (int i = 0; i + 1 < n; ++i) {
    const T b = od[i];                          // subdiagonal entry of row i+1
    const T a1 = dg[i + 1] - lam;               // diagonal of row i+1
    const T e1 = i + 2 < n ? od[i + 1] : T(0);  // superdiagonal of row i+1
    if (fabs(b) > fabs(c0)) {                   // swap rows i and i+1
      const T m = c0 / b;
      W.at(0, i, t) = b; W.at(1, i, t) = a1; W.at(2, i, t) = e1;
      W.at(3, i, t) = m; W.at(4, i, t) = T(1);
      const T r1 = c1 - m * a1, r2 = -m * e1;   // remaining row: columns i+1, i+2
      c0 = r1; c1 = r2;
    } else {
      if (c0 == T(0)) c0 = tiny;
      const T m = b / c0;
      W.at(0, i, t) = c0; W.at(1, i, t) = c1; W.at(2, i, t) = T(0);
      W.at(3, i, t) = m; W.at(4, i, t) = T(0);
      c0 = a1 - m * c1;
      c1 = e1;
    }
  }
  W.at(0, n - 1, t) = c0 == T(0) ? tiny : c0;
  W.at(1, n - 1, t) = T(0);
  W.at(2, n - 1, t) = T(0);
}

// Solves (T' - lambda) x = b in place on array 5 of the thread's scratch.
template <typename T>
__device__ void tri_solve(int n, T tiny, const Strided<T>& W, long long t) {
  for (int i = 0; i + 1 < n; ++i) {
    T xi = W.at(5, i, t), xn = W.at(5, i + 1, t);
    if (W.at(4, i, t) != T(0)) { const T q = xi; xi = xn; xn = q; }
    W.at(5, i, t) = xi;
    W.at(5, i + 1, t) = xn - W.at(3, i, t) * xi;
  }
  T x1 = T(0), x2 = T(0);  // x_{i+1}, x_{i+2}
  for (int i = n - 1; i >= 0; --i) {
    T sv = W.at(5, i, t) - W.at(1, i, t) * x1 - W.at(2, i, t) * x2;
    T d = W.at(0, i, t);
    if (fabs(d) < tiny) d = d < T(0) ? -tiny : tiny;
    const T xi = sv / d;
    W.at(5, i, t) = xi;
    x2 = x1;
    x1 = xi;
  }
}

constexpr int INVIT_WINDOW_N = 512;

template <typename T>
__global__ void k_lg_invit(LargeArgs a) {
  const long long NT = a.W * a.nvec;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= NT) return;
  const long long kw = t / a.nvec;
  const int idx = int(t - kw * a.nvec), n = a.n, nv = a.nvec;
  const T* dg = reinterpret_cast<const T*>(a.dg) + kw * n;
  const T* od = reinterpret_cast<const T*>(a.od) + kw * n;
  const T* lam = reinterpret_cast<const T*>(a.lam) + kw * a.nval;
  T lo, hi, tn;
  gershgorin(dg, od, n, lo, hi, tn);
  const T tolc = T(1e-3) * tn;
  if (idx > 0 && lam[idx] - lam[idx - 1] <= tolc) return;  // not the first of its cluster
  int end = idx;
  while (end + 1 < nv && lam[end + 1] - lam[end] <= tolc) ++end;
  T* Z = reinterpret_cast<T*>(a.Z) + kw * (long long)nv * n;   // row-major n x nvec
  const Strided<T> W{reinterpret_cast<T*>(a.work), NT, n};
  const T tiny = fmax(lg_eps<T>() * tn, T(1e-30));
  const bool windowed = n > INVIT_WINDOW_N;
  int q0 = idx;  // first earlier vector of the cluster to orthogonalise against
  for (int j = idx; j <= end; ++j) {
    if (windowed)
      while (lam[j] - lam[q0] > tolc) ++q0;
    tri_factor(dg, od, n, lam[j], tiny, W, t);
    for (int r = 0; r < n; ++r) W.at(5, r, t) = T(hash_unit((unsigned long long)j * 1000003ull + r));
    for (int it = 0; it < 3; ++it) {
      tri_solve(n, tiny, W, t);
      for (int q = q0; q < j; ++q) {  // orthogonalise within the cluster (or its window)
        T d = T(0);
        for (int r = 0; r < n; ++r) d += Z[(long long)r * nv + q] * W.at(5, r, t);
        for (int r = 0; r < n; ++r) W.at(5, r, t) -= d * Z[(long long)r * nv + q];
      }
      T s2 = T(0);
      for (int r = 0; r < n; ++r) s2 += W.at(5, r, t) * W.at(5, r, t);
      s2 = T(1) / sqrt(s2);
      for (int r = 0; r < n; ++r) W.at(5, r, t) *= s2;
    }
    for (int r = 0; r < n; ++r) Z[(long long)r * nv + j] = W.at(5, r, t);
  }
}

template <typename T>
__global__ void k_lg_invit_par(LargeArgs a) {
  const long long NT = a.W * a.nvec;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= NT) return;
  const long long kw = t / a.nvec;
  const int j = int(t - kw * a.nvec), n = a.n, nv = a.nvec;
  const T* dg = reinterpret_cast<const T*>(a.dg) + kw * n;
  const T* od = reinterpret_cast<const T*>(a.od) + kw * n;
  const T* lam = reinterpret_cast<const T*>(a.lam) + kw * a.nval;
  T lo, hi, tn;
  gershgorin(dg, od, n, lo, hi, tn);
  T* Z = reinterpret_cast<T*>(a.Z) + kw * (long long)nv * n;   // row-major n x nvec
  const Strided<T> W{reinterpret_cast<T*>(a.work), NT, n};
  const T tiny = fmax(lg_eps<T>() * tn, T(1e-30));
  tri_factor(dg, od, n, lam[j], tiny, W, t);
  for (int r = 0; r < n; ++r) W.at(5, r, t) = T(hash_unit((unsigned long long)j * 1000003ull + r));
  for (int it = 0; it < 3; ++it) {
    tri_solve(n, tiny, W, t);
    T s2 = T(0);
    for (int r = 0; r < n; ++r) s2 += W.at(5, r, t) * W.at(5, r, t);
    s2 = T(1) / sqrt(s2);
    for (int r = 0; r < n; ++r) W.at(5, r, t) *= s2;
  }
  for (int r = 0; r < n; ++r) Z[(long long)r * nv + j] = W.at(5, r, t);
}

// Orthonormalises the vectors of each cluster in place: one warp per eigenvalue index,
// working only where the index starts a cluster of two or more.
template <typename T>
__global__ void k_lg_invit_orth(LargeArgs a) {
  const long long NT = a.W * a.nvec;
  const long long t = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (t >= NT) return;
  const long long kw = t / a.nvec;
  const int idx = int(t - kw * a.nvec), n = a.n, nv = a.nvec;
  const T* dg = reinterpret_cast<const T*>(a.dg) + kw * n;
  const T* od = reinterpret_cast<const T*>(a.od) + kw * n;
  const T* lam = reinterpret_cast<const T*>(a.lam) + kw * a.nval;
  T lo, hi, tn;
  gershgorin(dg, od, n, lo, hi, tn);
  const T tolc = T(1e-3) * tn;
  if (idx > 0 && lam[idx] - lam[idx - 1] <= tolc) return;  // not the first of its cluster
  int end = idx;
  while (end + 1 < nv && lam[end + 1] - lam[end] <= tolc) ++end;
  if (end == idx) return;
  T* Z = reinterpret_cast<T*>(a.Z) + kw * (long long)nv * n;
  for (int j = idx; j <= end; ++j) {
    for (int pass = 0; pass < 2; ++pass)
      for (int q = idx; q < j; ++q) {
        T d = T(0);
        for (int r = lane; r < n; r += 32) d += Z[(long long)r * nv + q] * Z[(long long)r * nv + j];
        for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
        for (int r = lane; r < n; r += 32) Z[(long long)r * nv + j] -= d * Z[(long long)r * nv + q];
      }
    T s2 = T(0);
    for (int r = lane; r < n; r += 32) s2 += Z[(long long)r * nv + j] * Z[(long long)r * nv + j];
    for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    s2 = T(1) / sqrt(s2);
    for (int r = lane; r < n; r += 32) Z[(long long)r * nv + j] *= s2;
  }
}

// ---------------------------------------------------------------------------
// Stage 5: back-transform x = Q D z for the first ncol eigenvectors, Q = P_0 ... P_{n-3}:
// X = D Z, then X <- P_c X for c = n-3 down to 0 (P_c = I - 2 u_c u_c^dagger): one
// reflector at a time in FP64, in blocks of 32 reflectors (compact WY form) in FP32.
// Output X[r][col] with leading dimension ncol, precision To.
// ---------------------------------------------------------------------------
template <typename T, typename To>
__global__ void __launch_bounds__(256, 2) k_lg_backtransform(LargeArgs a, cx<To>* out, long long out_stride,
                                                             int ncol, int pw) {
  static_assert(std::is_same<T, To>::value, "the back-transform keeps the solver's precision");
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr bool kTc = std::is_same<T, float>::value;  // FP32: compact WY on the tensor cores
  __shared__ uint32_t tmem_slot;
  __shared__ __align__(8) uint64_t tc_bar;
  tc::State ts{};
  if constexpr (kTc) ts = tc::setup(&tmem_slot, &tc_bar);
  const int n = a.n, tid = threadIdx.x, nt = blockDim.x;
  for (long long kw = blockIdx.x; kw < a.W; kw += gridDim.x) {
    const cx<T>* A = reinterpret_cast<const cx<T>*>(a.A) + kw * (long long)n * n;
    const cx<T>* Dp = reinterpret_cast<const cx<T>*>(a.Dp) + kw * n;
    const T* Z = reinterpret_cast<const T*>(a.Z) + kw * (long long)a.nvec * n;
    cx<To>* X = out + kw * out_stride;
    for (int r = tid >> 5; r < n; r += nt >> 5) {
      const cx<T> d = Dp[r];
      for (int col = tid & 31; col < ncol; col += 32) {
        const T z = Z[(long long)r * a.nvec + col];
        X[(long long)r * ncol + col] = cx<To>(To(d.re * z), To(d.im * z));
      }
    }
    __syncthreads();
    if constexpr (!kTc) {
      cta_reflect<T, To>(A, n, X, ncol, ncol, true, smem, pw);   // FP64-pipe bound: fewest flops
    } else if (!ts.failed) {                                     // blocked, tensor-core GEMMs
      if (!cta_reflect_wy(A, n, X, ncol, ncol, true, smem, ts) && tid == 0)
        report(a.status, ST_ETIMEOUT, a.k0 + kw, 0.0);
    }
  }
  if constexpr (kTc) tc::teardown(ts);
}

// FP64 back-transform for large n (a one-reflector panel would hold fewer than 16
// columns): X = D Z, then the reflectors in compact-WY blocks through FP64 GEMMs.
__global__ void __launch_bounds__(256, 2) k_lg_backtransform_wy64(LargeArgs a, z64* out, long long out_stride,
                                                                  int ncol) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int n = a.n, tid = threadIdx.x, nt = blockDim.x;
  for (long long kw = blockIdx.x; kw < a.W; kw += gridDim.x) {
    const z64* A = reinterpret_cast<const z64*>(a.A) + kw * (long long)n * n;
    const z64* Dp = reinterpret_cast<const z64*>(a.Dp) + kw * n;
    const double* Z = reinterpret_cast<const double*>(a.Z) + kw * (long long)a.nvec * n;
    z64* X = out + kw * out_stride;
    for (int r = tid >> 5; r < n; r += nt >> 5) {
      const z64 d = Dp[r];
      for (int col = tid & 31; col < ncol; col += 32) {
        const double z = Z[(long long)r * a.nvec + col];
        X[(long long)r * ncol + col] = z64(d.re * z, d.im * z);
      }
    }
    __syncthreads();
    cta_reflect_wy_simt<double>(A, n, X, ncol, ncol, true, smem);
  }
}

// FP64 path: direct gap from the bisection eigenvalues.
__global__ void k_lg_gap64(LargeArgs a) {
  const long long kw = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (kw >= a.W) return;
  const double* lam = reinterpret_cast<const double*>(a.lam) + kw * a.nval;
  const double g = a.p < a.n ? lam[a.p] - lam[a.p - 1] : INFINITY;
  const long long k = a.k0 + kw * (a.kstride > 0 ? a.kstride : 1);
  a.gap[k] = g;
  if (!(g > a.gap_tol)) report(a.status, ST_EGAP, k, g);
}

__host__ __device__ inline size_t refine_work_offset(int p) {
  return ((size_t(p) + 66) * sizeof(double) + 15) & ~size_t(15);
}

// ---------------------------------------------------------------------------
// Stage 6 (mixed): one Newton correction of the occupied block.
//   Q = X[:, :p] holds FP32 eigenvectors (exact FP32 numbers).  H Q from the hopping
//   plan's FP64 entries with compensated FP32 dot products; rho_c = q_c^dag H q_c and
//   R = H Q - Q rho in FP64; the complement's coefficients
//   C[a][c] = z_a^T D^dag Q_h^dag R_c / (rho_c - lam_a) and the update
//   Q_h D Z_u C in FP32 through the reflectors (R is small, FP32 keeps it to ~1e-7
//   relative); Q64 = Q + update.  Then one first-order Lowdin step,
//   Q <- Q - Q (Q^dag Q - I) / 2, with Q32^dag Q32 - I compensated and the small
//   terms in FP32.  The gap comes from FP64 Rayleigh quotients of the (p-1)-th
//   and p-th FP32 vectors.  The off-diagonal part of Q^dag H Q is of the order of
//   the FP32 error; its projection on the complement enters at second order.
// ---------------------------------------------------------------------------
// Two CTAs per SM: the compensated GEMM tiles hold 64 accumulator registers per
// thread, and without the bound the kernel takes 136 registers (one CTA per SM).
__global__ void __launch_bounds__(256, 2) k_lg_refine(LargeArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int n = a.n, p = a.p, nbt = a.nbt, tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nwarp = nt >> 5;
  const DevModel& md = a.model;
  double* rho = reinterpret_cast<double*>(smem);     // p + 2
  double* red = rho + p + 2;                         // 64
  unsigned char* work = smem + refine_work_offset(p);  // block reflectors / GEMM tiles
  __shared__ uint32_t tmem_slot;
  __shared__ __align__(8) uint64_t tc_bar;
  tc::State ts = tc::setup(&tmem_slot, &tc_bar);      // plain FP32 products: tensor cores
  for (long long kw = blockIdx.x; kw < a.W; kw += gridDim.x) {
    const long long k = a.k0 + kw * (a.kstride > 0 ? a.kstride : 1);
    const c32* A = reinterpret_cast<const c32*>(a.A) + kw * (long long)n * n;
    const c32* Dp = reinterpret_cast<const c32*>(a.Dp) + kw * n;
    const float* Z = reinterpret_cast<const float*>(a.Z) + kw * (long long)a.nvec * n;
    const float* lam = reinterpret_cast<const float*>(a.lam) + kw * a.nval;
    const c32* X = reinterpret_cast<const c32*>(a.X) + kw * (long long)n * nbt;
    const bool dense = a.Hin != nullptr;  // explicit matrix: entries r n + q, all columns
    const z64* He = a.Hent + kw * (long long)(dense ? n * n : md.n_ent);
    z64* Q = a.U + kw * (long long)n * p;
    z64* R = a.R64 + kw * (long long)n * p;          // H Q, later FP32 scratch
    c32* C = a.C32 + kw * (long long)n * p;
    c32* E = reinterpret_cast<c32*>(a.G64 + kw * (long long)p * p);  // Q^dag Q - I (p x p)
    // R = H Q32 (compensated): a tiled GEMM when H is dense, else one warp per row
    if (dense || md.n_ent == n * n) {
      cta_gemm<GemmSplitComp, true, true>(
          n, p, n,
          [&](int r, int q) {
            const c32* hp = reinterpret_cast<const c32*>(He + (long long)r * n + q);
            return SplitC{hp[0], hp[1]};
          },
          [&](int q, int c) { return X[(long long)q * nbt + c]; },
          [&](int r, int c, const CDF& acc) { R[(long long)r * p + c] = acc.value(); }, work);
    } else
    for (int r = warp; r < n; r += nwarp) {
      for (int c0 = 0; c0 < p; c0 += 32) {
        const int c = c0 + lane;
        CDF acc;
        const int q0 = dense ? r * n : a.row_ptr[r], q1 = dense ? (r + 1) * n : a.row_ptr[r + 1];
        for (int q = q0; q < q1; ++q) {
          const c32* hp = reinterpret_cast<const c32*>(He + q);
          const int col = dense ? q - q0 : md.ent_col[q];
          if (c < p) acc.add_prod(hp[0], hp[1], X[(long long)col * nbt + c]);
        }
        if (c < p) R[(long long)r * p + c] = acc.value();
      }
    }
    __syncthreads();
    for (int c = tid; c < p; c += nt) {
      double sum = 0.0;
      for (int r = 0; r < n; ++r) {
        const c32 q = X[(long long)r * nbt + c];
        const z64 h = R[(long long)r * p + c];
        sum += double(q.re) * h.re + double(q.im) * h.im;
      }
      rho[c] = sum;
    }
    __syncthreads();
    // residual to FP32
    for (int r = warp; r < n; r += nwarp)
      for (int c = lane; c < p; c += 32) {
        const z64 h = R[(long long)r * p + c];
        const c32 q = X[(long long)r * nbt + c];
        C[(long long)r * p + c] = c32(float(h.re - rho[c] * double(q.re)), float(h.im - rho[c] * double(q.im)));
      }
    __syncthreads();
    // C <- D^dag Q_h^dag C
    bool tc_ok = cta_reflect_wy(A, n, C, p, p, false, work, ts);
    for (int r = warp; r < n; r += nwarp) {
      const c32 d = conj(Dp[r]);
      for (int c = lane; c < p; c += 32) C[(long long)r * p + c] = d * C[(long long)r * p + c];
    }
    __syncthreads();
    // complement coefficients (FP32), kept in the R workspace
    c32* coef = reinterpret_cast<c32*>(R);
    const int nu = n - p;
    const int nvec = a.nvec;
    // coef[ua][c] = (Z_u^T C)[ua][c] / (rho_c - lam_{p+ua})
    tc_ok = tc_ok && cta_cgemm_tc<false, true>(
        nu, p, n, [&](int ua, int r) { return c32(Z[(long long)r * nvec + p + ua], 0.f); },
        [&](int r, int c) { return C[(long long)r * p + c]; },
        [&](int ua, int c, c32 v) {
          coef[(long long)ua * p + c] = float(1.0 / (rho[c] - double(lam[p + ua]))) * v;
        },
        work, ts);
    __syncthreads();
    // update = Q_h D Z_u coef
    tc_ok = tc_ok && cta_cgemm_tc<true, true>(
        n, p, nu, [&](int r, int ua) { return c32(Z[(long long)r * nvec + p + ua], 0.f); },
        [&](int ua, int c) { return coef[(long long)ua * p + c]; },
        [&](int r, int c, c32 v) { C[(long long)r * p + c] = Dp[r] * v; }, work, ts);
    __syncthreads();
    tc_ok = tc_ok && cta_reflect_wy(A, n, C, p, p, true, work, ts);
    // E = Q^dag Q - I with Q = Q32 + C: Q32^dag Q32 - I compensated (the FP32 basis is
    // orthonormal to ~1e-7, so the difference needs the extra precision), then the
    // small terms Q32^dag C + C^dag (Q32 + C) in FP32 as one GEMM over 2 n rows
    cta_gemm<GemmGramComp, false, true>(
        p, p, n, [&](int x, int r) { return X[(long long)r * nbt + x]; },
        [&](int r, int y) { return X[(long long)r * nbt + y]; },
        [&](int x, int y, const CDF& acc) {
          z64 v = acc.value();
          if (x == y) v.re -= 1.0;
          E[(long long)x * p + y] = c32(float(v.re), float(v.im));
        },
        work);
    __syncthreads();
    tc_ok = tc_ok && cta_cgemm_tc<false, true>(
        p, p, 2 * n,
        [&](int x, int k) {
          return conj(k < n ? X[(long long)k * nbt + x] : C[(long long)(k - n) * p + x]);
        },
        [&](int k, int y) {
          return k < n ? C[(long long)k * p + y] : X[(long long)(k - n) * nbt + y] + C[(long long)(k - n) * p + y];
        },
        [&](int x, int y, c32 v) { E[(long long)x * p + y] = E[(long long)x * p + y] + v; }, work, ts);
    __syncthreads();
    // Q = (Q32 + C) - (Q32 + C) E / 2, the correction in FP32
    tc_ok = tc_ok && cta_cgemm_tc<true, true>(
        n, p, p, [&](int r, int q) { return X[(long long)r * nbt + q] + C[(long long)r * p + q]; },
        [&](int q, int c) { return E[(long long)q * p + c]; },
        [&](int r, int c, c32 v) {
          const c32 x32 = X[(long long)r * nbt + c], dc = C[(long long)r * p + c];
          Q[(long long)r * p + c] = z64(double(x32.re) + double(dc.re) - 0.5 * double(v.re),
                                        double(x32.im) + double(dc.im) - 0.5 * double(v.im));
        },
        work, ts);
    __syncthreads();
    if (!tc_ok && tid == 0) report(a.status, ST_ETIMEOUT, k, 0.0);
    // gap from FP64 Rayleigh quotients of the FP32 vectors p-1 and p: rho[p-1] is
    // already q^dag H q of vector p-1; H x_p by one warp per row (lanes along the row,
    // coalesced), in FP64
    if (p < n) {
      double num = 0.0, den = 0.0, den1 = 0.0;
      for (int r = warp; r < n; r += nwarp) {
        z64 hv(0.0, 0.0);
        const int q0 = dense ? r * n : a.row_ptr[r], q1 = dense ? (r + 1) * n : a.row_ptr[r + 1];
        for (int q = q0 + lane; q < q1; q += 32) {
          const c32* hp = reinterpret_cast<const c32*>(He + q);
          const z64 h(double(hp[0].re) + double(hp[1].re), double(hp[0].im) + double(hp[1].im));
          cfma(hv, h, ccast<double>(X[(long long)(dense ? q - q0 : md.ent_col[q]) * nbt + p]));
        }
        for (int o = 16; o > 0; o >>= 1) {
          hv.re += __shfl_xor_sync(0xffffffffu, hv.re, o);
          hv.im += __shfl_xor_sync(0xffffffffu, hv.im, o);
        }
        if (lane == 0) {
          const z64 v = ccast<double>(X[(long long)r * nbt + p]);
          num += v.re * hv.re + v.im * hv.im;
          den += abs2(v);
          den1 += abs2(ccast<double>(X[(long long)r * nbt + p - 1]));
        }
      }
      num = block_sum(num, red);
      den = block_sum(den, red);
      den1 = block_sum(den1, red);
      if (tid == 0) {
        const double g = num / den - rho[p - 1] / den1;
        a.gap[k] = g;
        if (!(g > a.gap_tol)) report(a.status, ST_EGAP, k, g);
      }
    } else if (tid == 0) {
      a.gap[k] = INFINITY;
    }
    __syncthreads();
  }
  tc::teardown(ts);
}

// ---------------------------------------------------------------------------
// Launcher: every stage of one wave, in stream order.
// ---------------------------------------------------------------------------
namespace {
constexpr int LG_THREADS = 256;

int lg_grid(long long units) {
  const long long cap = 152LL * 4;
  return int(units < cap ? (units > 0 ? units : 1) : cap);
}

void lg_mark(const LargeArgs& a, const char* name) {
  if (a.mark) a.mark(a.mark_user, name);
}

template <typename T>
cudaError_t lg_common(const LargeArgs& a, cudaStream_t s) {
  k_lg_build<T><<<lg_grid(a.W), LG_THREADS, 0, s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  lg_mark(a, "lg_build");
  // lower-triangle kernel: 5 n + (warps) n complex values of shared memory, with up
  // to 16 warps and at least 4; one CTA per SM keeps the matrices being reduced
  // resident in L2 (n = 256: 152 x 512 KB in complex64)
  const size_t vec_b = size_t(a.n) * sizeof(cx<T>), lim = size_t(200) << 10;
  const size_t fixed = 5 * vec_b + 64 * sizeof(double);
  // Each step waits on a few dependent L2 round trips, so several k-points per SM
  // (more CTAs with fewer warps each) hide more latency than more warps on one
  // k-point; a small wave gives each of its CTAs more warps instead.
  const int fit = fixed < lim ? int(std::min<size_t>(16, (lim - fixed) / vec_b)) : 0;
  const int want = a.W >= 4 * 152 ? 4 : (a.W >= 2 * 152 ? 8 : 16);
  const int warps = std::min(fit, want);
  if (warps >= 4) {
    const size_t sm_h = fixed + size_t(warps) * vec_b;
    static size_t cached_h = 0;
    if ((e = set_smem_once(k_lg_tridiag_h<T>, sm_h, cached_h)) != cudaSuccess) return e;
    const long long ctas = std::min<long long>(a.W, 152LL * (16 / warps));
    k_lg_tridiag_h<T><<<int(ctas), 32 * warps, sm_h, s>>>(a);
  } else {
    const size_t sm_tri = 3 * size_t(a.n) * sizeof(cx<T>) + 64 * sizeof(double);
    static size_t cached = 0;
    if ((e = set_smem_once(k_lg_tridiag<T>, sm_tri, cached)) != cudaSuccess) return e;
    k_lg_tridiag<T><<<lg_grid(a.W), LG_THREADS, sm_tri, s>>>(a);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  lg_mark(a, "lg_tridiag");
  const long long nb = a.W * a.nval;
  k_lg_bisect<T><<<int((nb + 127) / 128), 128, 0, s>>>(a);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  lg_mark(a, "lg_bisect");
  const long long ni = a.W * a.nvec;
  if (ni > 0) {
    if (a.subspace_only) {
      k_lg_invit_par<T><<<int((ni + 63) / 64), 64, 0, s>>>(a);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      const long long nw = ni * 32;
      if (nw / 128 + 1 > 0x7fffffffLL) return cudaErrorInvalidValue;
      k_lg_invit_orth<T><<<int((nw + 127) / 128), 128, 0, s>>>(a);
    } else {
      k_lg_invit<T><<<int((ni + 63) / 64), 64, 0, s>>>(a);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    lg_mark(a, "lg_invit");
  }
  return cudaSuccess;
}
}  // namespace

cudaError_t launch_states_large(const LargeArgs& a, cudaStream_t s) {
  if (a.W <= 0) return cudaSuccess;
  cudaError_t e;
  if (!a.mixed) {
    if ((e = lg_common<double>(a, s)) != cudaSuccess) return e;
    if (a.p == 0) return cudaSuccess;  // values only
    // one-reflector panels while a panel holds at least 16 columns (n <= ~780); beyond,
    // a panel of a few columns would sweep every reflector once per few columns, so
    // the reflectors are applied in compact-WY blocks through FP64 GEMMs (pw = 0)
    const int pw = reflect_pw<double>(a.n, size_t(200) << 10);
    if (pw >= 16) {
      const size_t sm = reflect_smem<double>(a.n, pw);
      static size_t cached = 0;
      if ((e = set_smem_once(k_lg_backtransform<double, double>, sm, cached)) != cudaSuccess) return e;
      k_lg_backtransform<double, double><<<lg_grid(a.W), LG_THREADS, sm, s>>>(
          a, a.U, (long long)a.n * a.p, a.p, pw);
    } else {
      const size_t sm = reflect_wy_simt_smem<double>();
      static size_t cached_wy = 0;
      if ((e = set_smem_once(k_lg_backtransform_wy64, sm, cached_wy)) != cudaSuccess) return e;
      k_lg_backtransform_wy64<<<lg_grid(a.W), LG_THREADS, sm, s>>>(a, a.U, (long long)a.n * a.p, a.p);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    lg_mark(a, "lg_backtransform");
    if (a.Hin) return cudaSuccess;  // batched eigensolve: every eigenvalue is returned, no gap test
    k_lg_gap64<<<int((a.W + 127) / 128), 128, 0, s>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    lg_mark(a, "lg_gap");
    return cudaSuccess;
  }
  if ((e = lg_common<float>(a, s)) != cudaSuccess) return e;
  if (a.no_refine) return cudaSuccess;
  const size_t sm = reflect_wy_smem();
  static size_t cached = 0;
  if ((e = set_smem_once(k_lg_backtransform<float, float>, sm, cached)) != cudaSuccess) return e;
  k_lg_backtransform<float, float><<<lg_grid(a.W), LG_THREADS, sm, s>>>(
      a, reinterpret_cast<c32*>(a.X), (long long)a.n * a.nbt, a.nbt, 0);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  lg_mark(a, "lg_backtransform");
  const size_t smr = refine_work_offset(a.p) + std::max(std::max(reflect_wy_smem(), tc::SMEM), CG_SMEM);
  static size_t cached_r = 0;
  if ((e = set_smem_once(k_lg_refine, smr, cached_r)) != cudaSuccess) return e;
  k_lg_refine<<<lg_grid(a.W), LG_THREADS, smr, s>>>(a);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  lg_mark(a, "lg_refine");
  return cudaSuccess;
}

// ---------------------------------------------------------------------------
// Batched eigensolve of explicit matrices: FP64 Rayleigh-Ritz of the refined block
// (mixed path, p <= 64) and the scatter of eigenvalues / eigenvectors to the
// caller's packed layout.
// ---------------------------------------------------------------------------
__global__ void k_eigh_ritz(LargeArgs a, double* ritz) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int n = a.n, p = a.p, tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nwarp = nt >> 5;
  z64* G = reinterpret_cast<z64*>(smem);    // p x p
  z64* V = G + p * p;                       // p x p
  JacRot<double>* rot = reinterpret_cast<JacRot<double>*>(V + p * p);
  double* red = reinterpret_cast<double*>(rot + (p / 2 + 2));
  int* ord = reinterpret_cast<int*>(red + 64);
  for (long long kw = blockIdx.x; kw < a.W; kw += gridDim.x) {
    const c32* He = reinterpret_cast<const c32*>(a.Hent + kw * (long long)n * n);
    z64* Q = a.U + kw * (long long)n * p;
    z64* HQ = a.R64 + kw * (long long)n * p;
    for (int r = warp; r < n; r += nwarp)  // H Q in FP64 (H from its float-pair split)
      for (int c = lane; c < p; c += 32) {
        z64 acc(0.0, 0.0);
        for (int q = 0; q < n; ++q) {
          const c32 hi = He[2 * ((long long)r * n + q)], lo = He[2 * ((long long)r * n + q) + 1];
          cfma(acc, z64(double(hi.re) + double(lo.re), double(hi.im) + double(lo.im)), Q[(long long)q * p + c]);
        }
        HQ[(long long)r * p + c] = acc;
      }
    __syncthreads();
    for (int e = tid; e < p * p; e += nt) {
      const int x = e / p, y = e - x * p;
      z64 acc(0.0, 0.0);
      for (int r = 0; r < n; ++r) cfma_conj(acc, Q[(long long)r * p + x], HQ[(long long)r * p + y]);
      G[e] = acc;
    }
    __syncthreads();
    for (int e = tid; e < p * p; e += nt) {  // Hermitian part
      const int x = e / p, y = e - x * p;
      if (x < y) {
        const z64 h = 0.5 * (G[x * p + y] + conj(G[y * p + x]));
        G[x * p + y] = h;
        G[y * p + x] = conj(h);
      } else if (x == y) {
        G[e] = z64(G[e].re, 0.0);
      }
    }
    __syncthreads();
    const int sw = jacobi_eigh<double>(G, V, p, p, 40, rot, red);
    if (sw < 0 && tid == 0) report(a.status, ST_ENOCONV, a.k0 + kw, 0.0);
    sort_diag(G, p, p, ord);
    for (int c = tid; c < p; c += nt) ritz[kw * p + c] = G[ord[c] * p + ord[c]].re;
    // Q <- Q V (columns in ascending order), row by row through HQ as scratch
    for (int r = warp; r < n; r += nwarp)
      for (int c = lane; c < p; c += 32) {
        z64 acc(0.0, 0.0);
        for (int q = 0; q < p; ++q) cfma(acc, Q[(long long)r * p + q], V[q * p + ord[c]]);
        HQ[(long long)r * p + c] = acc;
      }
    __syncthreads();
    for (long long e = tid; e < (long long)n * p; e += nt) Q[e] = HQ[e];
    __syncthreads();
  }
}

cudaError_t launch_eigh_ritz(const LargeArgs& a, double* ritz, cudaStream_t s) {
  if (a.W <= 0 || a.p <= 0) return cudaSuccess;
  if (a.p > 64) return cudaErrorInvalidValue;
  const size_t sm = 2 * size_t(a.p) * a.p * sizeof(z64) + (a.p / 2 + 2) * sizeof(JacRot<double>) +
                    64 * sizeof(double) + size_t(a.p) * sizeof(int) + 16;
  static size_t cached = 0;
  cudaError_t e = set_smem_once(k_eigh_ritz, sm, cached);
  if (e != cudaSuccess) return e;
  k_eigh_ritz<<<lg_grid(a.W), LG_THREADS, sm, s>>>(a, ritz);
  return cudaGetLastError();
}

__global__ void k_eigh_scatter(EighScatterArgs e) {
  for (long long kw = blockIdx.x; kw < e.W; kw += gridDim.x) {
    const int b = e.idx[e.k0 + kw];
    double* ev = e.evals + e.e_off[b];
    for (int i = threadIdx.x; i < e.n; i += blockDim.x) {
      double v;
      if (e.ritz && i < e.p)
        v = e.ritz[kw * e.p + i];
      else if (e.mixed)
        v = double(reinterpret_cast<const float*>(e.lam)[kw * e.nval + i]);
      else
        v = reinterpret_cast<const double*>(e.lam)[kw * e.nval + i];
      ev[i] = v;
    }
    if (e.evecs && e.p > 0) {
      const z64* src = e.U + kw * (long long)e.n * e.p;
      z64* dst = e.evecs + e.v_off[b];
      for (long long x = threadIdx.x; x < (long long)e.n * e.p; x += blockDim.x) dst[x] = src[x];
    }
  }
}

cudaError_t launch_eigh_scatter(const EighScatterArgs& e, cudaStream_t s) {
  if (e.W <= 0) return cudaSuccess;
  k_eigh_scatter<<<lg_grid(e.W), 256, 0, s>>>(e);
  return cudaGetLastError();
}

}  // namespace bw
