// Loop kernels for many occupied bands (p > 64, supercells): the Wilson matrix of
// Eq. 2 no longer fits in shared memory, so the loop is streamed along its k-points.
//
//  - k_zgemm:    batched complex FP64 GEMM C_b = op(A_b) B_b, op in {identity,
//                conjugate transpose}.  It forms the overlaps
//                M_j = U(k_{j+1})^dagger U(k_j) (Eq. 2) and the running product
//                W <- M_j W (later k on the left) for every loop of a block at once.
//  - k_geig_big: one CTA per loop: general complex eigenvalues of W in global
//                memory (Householder-Hessenberg + shifted QR, the same solver as the
//                shared-memory path), theta = arg(lambda) sorted ascending, and the
//                loop's minimum direct gap.
//  - k_geig_cluster: the same eigenphases on a cluster of CTAs per loop, for larger p.
#include <float.h>

#include <cooperative_groups.h>

#include <algorithm>
#include <cstring>

#include "df32.cuh"
#include "geig.cuh"
#include "jacobi.cuh"
#include "launch.h"

namespace bw {

// ---------------------------------------------------------------------------
// Batched complex GEMM.  CTA tile 64 x 64 of C, 256 threads; thread (ty, tx)
// owns rows ty + 16 a and columns tx + 16 b (a, b < 4), so that the shared-memory
// reads of a warp are conflict-free broadcasts or consecutive words.  The k
// dimension advances in chunks of 16 staged in shared memory, zero-filled past the
// ragged edges.  FP64 FMA throughput bounds it (GB300: ~1.7 FP64 FMA per clock
// per SM), far below the shared-memory bandwidth the tile needs.
// ---------------------------------------------------------------------------
constexpr int GT = 64, GK = 16;

template <typename E>
__device__ __forceinline__ E gemm_zero();
template <>
__device__ __forceinline__ z64 gemm_zero<z64>() { return z64(0.0, 0.0); }
template <>
__device__ __forceinline__ cdf gemm_zero<cdf>() { return cdf_zero(); }

// E = z64: FP64.  E = cdf: complex double-float on the FP32 pipe (A, B and C hold
// complex double-float; the mixed request's many-band overlaps and loop products).
template <typename E>
__global__ void __launch_bounds__(256) k_zgemm(GemmArgs g) {
  __shared__ E As[GK][GT];
  __shared__ E Bs[GK][GT];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int tiles_n = (g.n + GT - 1) / GT;
  const long long bl = g.b0 + blockIdx.y, b = g.kfirst + bl;
  const long long ba = g.a_next_N > 0 ? (b / g.a_next_N) * g.a_next_N + (b % g.a_next_N + 1) % g.a_next_N
                       : g.a_mod > 0  ? (b + g.a_shift) % g.a_mod
                                      : b;
  const int r0 = (blockIdx.x / tiles_n) * GT, c0 = (blockIdx.x % tiles_n) * GT;
  const E* A = reinterpret_cast<const E*>(g.A) + ba * g.sA;
  const E* B = reinterpret_cast<const E*>(g.B) + b * g.sB;
  E* C = reinterpret_cast<E*>(g.C) + bl * g.sC;
  E acc[4][4];
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int y = 0; y < 4; ++y) acc[x][y] = gemm_zero<E>();
  for (int k0 = 0; k0 < g.k; k0 += GK) {
    // stage op(A)[r0 .. r0+64, k0 .. k0+16] as As[kk][r]
    for (int e = tid; e < GK * GT; e += 256) {
      int kk, r;
      if (g.opA) {  // A^dagger: row r of op(A) is column r of A (contiguous in r)
        kk = e / GT;
        r = e - kk * GT;
      } else {      // A: contiguous in kk
        r = e / GK;
        kk = e - r * GK;
      }
      const int gr = r0 + r, gk = k0 + kk;
      E v = gemm_zero<E>();
      if (gr < g.m && gk < g.k) {
        if (g.opA) {
          v = conj(A[(long long)gk * g.lda + gr]);
        } else {
          v = A[(long long)gr * g.lda + gk];
        }
      }
      As[kk][r] = v;
    }
    for (int e = tid; e < GK * GT; e += 256) {
      const int kk = e / GT, c = e - kk * GT;
      const int gc = c0 + c, gk = k0 + kk;
      Bs[kk][c] = (gc < g.n && gk < g.k) ? B[(long long)gk * g.ldb + gc] : gemm_zero<E>();
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < GK; ++kk) {
      E av[4], bv[4];
#pragma unroll
      for (int x = 0; x < 4; ++x) av[x] = As[kk][ty + 16 * x];
#pragma unroll
      for (int y = 0; y < 4; ++y) bv[y] = Bs[kk][tx + 16 * y];
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) cfma(acc[x][y], av[x], bv[y]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int x = 0; x < 4; ++x) {
    const int gr = r0 + ty + 16 * x;
    if (gr >= g.m) continue;
#pragma unroll
    for (int y = 0; y < 4; ++y) {
      const int gc = c0 + tx + 16 * y;
      if (gc < g.n) C[(long long)gr * g.ldc + gc] = acc[x][y];
    }
  }
}

cudaError_t launch_zgemm(const GemmArgs& g, cudaStream_t s, bool df) {
  if (g.batch <= 0 || g.m <= 0 || g.n <= 0) return cudaSuccess;
  const long long tiles = (long long)((g.m + GT - 1) / GT) * ((g.n + GT - 1) / GT);
  if (tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
  for (long long b0 = 0; b0 < g.batch; b0 += 65535) {  // grid.y holds at most 65535
    GemmArgs h = g;
    h.b0 = b0;
    dim3 grid(unsigned(tiles), unsigned(std::min<long long>(65535, g.batch - b0)));
    if (df)
      k_zgemm<cdf><<<grid, 256, 0, s>>>(h);
    else
      k_zgemm<z64><<<grid, 256, 0, s>>>(h);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// In place: complex FP64 <-> complex double-float (the same 16 bytes per element).
__global__ void k_z64_to_cdf(z64* x, long long count) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count;
       e += (long long)gridDim.x * blockDim.x) {
    const z64 v = x[e];
    reinterpret_cast<cdf*>(x)[e] = cdf_from(v);
  }
}

__global__ void k_cdf_to_z64(z64* x, long long count) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count;
       e += (long long)gridDim.x * blockDim.x) {
    const cdf v = reinterpret_cast<const cdf*>(x)[e];
    x[e] = cdf_to_z64(v);
  }
}

cudaError_t launch_convert_cdf(z64* x, long long count, bool to_cdf, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  const unsigned grid = unsigned(std::min<long long>((count + 255) / 256, 152LL * 16));
  if (to_cdf)
    k_z64_to_cdf<<<grid, 256, 0, s>>>(x, count);
  else
    k_cdf_to_z64<<<grid, 256, 0, s>>>(x, count);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Phase of a determinant (the link variables of the plaquette Berry flux for p > 64).
// Right-looking LU with partial pivoting of one p x p matrix per CTA in global memory:
// the row exchanges are kept in a permutation (rows are not moved), so
// det = sign(perm) prod_c A[perm[c]][c].  Only the phase is kept, as the product of the
// unit pivots (no overflow or underflow at any p); a zero pivot gives 0.  The pivot is
// the largest |A[perm[r]][c]| over r >= c, the smallest r on ties.  The trailing update
// gives each thread whole columns, so the warp's accesses to a row are contiguous.
// ---------------------------------------------------------------------------
constexpr int DET_THREADS = 256;

__global__ void __launch_bounds__(DET_THREADS) k_det_phase(z64* A, long long sA, int p, long long nb,
                                                          z64* out) {
  extern __shared__ __align__(16) unsigned char smem[];
  z64* mult = reinterpret_cast<z64*>(smem);
  int* perm = reinterpret_cast<int*>(mult + p);
  __shared__ double red_v[DET_THREADS / 32];
  __shared__ int red_i[DET_THREADS / 32];
  __shared__ z64 pv_sh;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  for (long long b = blockIdx.x; b < nb; b += gridDim.x) {
    z64* M = A + b * sA;
    for (int r = tid; r < p; r += DET_THREADS) perm[r] = r;
    z64 phase(1.0, 0.0);  // thread 0
    __syncthreads();
    for (int c = 0; c < p; ++c) {
      double best = -1.0;
      int bi = p;
      for (int r = c + tid; r < p; r += DET_THREADS) {
        const double v = abs2(M[(long long)perm[r] * p + c]);
        if (v > best) {
          best = v;
          bi = r;
        }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_down_sync(0xffffffffu, best, o);
        const int oi = __shfl_down_sync(0xffffffffu, bi, o);
        if (ov > best || (ov == best && oi < bi)) {
          best = ov;
          bi = oi;
        }
      }
      if (lane == 0) {
        red_v[wid] = best;
        red_i[wid] = bi;
      }
      __syncthreads();
      if (tid == 0) {
        for (int w = 1; w < DET_THREADS / 32; ++w)
          if (red_v[w] > best || (red_v[w] == best && red_i[w] < bi)) {
            best = red_v[w];
            bi = red_i[w];
          }
        if (bi >= p) bi = c;  // every candidate is NaN: keep the row order
        const int t = perm[c];
        perm[c] = perm[bi];
        perm[bi] = t;
        const z64 pv = M[(long long)perm[c] * p + c];
        const double a = sqrt(abs2(pv));
        if (a > 0.0) {
          phase = phase * z64(pv.re / a, pv.im / a);
          if (bi != c) phase = z64(-phase.re, -phase.im);
        } else {
          phase = z64(0.0, 0.0);
        }
        pv_sh = pv;
      }
      __syncthreads();
      const z64 pv = pv_sh;
      const double pa = abs2(pv);
      for (int r = c + 1 + tid; r < p; r += DET_THREADS) {
        const z64 v = M[(long long)perm[r] * p + c];
        mult[r] = pa > 0.0 ? z64((v.re * pv.re + v.im * pv.im) / pa, (v.im * pv.re - v.re * pv.im) / pa)
                           : z64(0.0, 0.0);
      }
      __syncthreads();
      const z64* prow = M + (long long)perm[c] * p;
      for (int cc = c + 1 + tid; cc < p; cc += DET_THREADS) {
        const z64 t = prow[cc];
        for (int r = c + 1; r < p; ++r) {
          z64* e = M + (long long)perm[r] * p + cc;
          *e = *e - mult[r] * t;
        }
      }
      __syncthreads();
    }
    if (tid == 0) out[b] = phase;
    __syncthreads();
  }
}

cudaError_t launch_det_phase(z64* A, long long sA, int p, long long nb, z64* out, cudaStream_t s) {
  if (nb <= 0 || p <= 0) return cudaSuccess;
  const size_t sm = size_t(p) * (sizeof(z64) + sizeof(int));
  static size_t cached = 0;
  cudaError_t e = set_smem_once(k_det_phase, sm, cached);
  if (e != cudaSuccess) return e;
  const long long cap = 152LL * 4;
  k_det_phase<<<int(nb < cap ? nb : cap), DET_THREADS, sm, s>>>(A, sA, p, nb, out);
  return cudaGetLastError();
}

cudaError_t launch_plaquettes_big(const LoopArgs& a, z64* Lmat, long long kb, z64* Lx, z64* Ly,
                                  double* flux, double* chern, cudaStream_t s) {
  const long long K = (long long)a.N * a.N_t;
  if (K <= 0) return cudaSuccess;
  const int p = a.p;
  const long long sU = (long long)a.n * p, sL = (long long)p * p;
  cudaError_t e;
  for (long long k0 = 0; k0 < K; k0 += kb) {
    const long long nb = std::min(kb, K - k0);
    for (int dir = 0; dir < 2; ++dir) {
      // Lx(j, i) = det U(j+1, i)^dag U(j, i);  Ly(j, i) = det U(j, i+1)^dag U(j, i)
      GemmArgs g;
      memset(&g, 0, sizeof(g));
      g.A = a.U; g.B = a.U; g.C = Lmat;
      g.m = p; g.n = p; g.k = a.n; g.opA = 1;
      g.lda = p; g.ldb = p; g.ldc = p;
      g.sA = sU; g.sB = sU; g.sC = sL;
      g.kfirst = k0;
      if (dir == 0) {
        g.a_next_N = a.N;
      } else {
        g.a_shift = a.N;
        g.a_mod = K;
      }
      g.batch = nb;
      if ((e = launch_zgemm(g, s)) != cudaSuccess) return e;
      if ((e = launch_det_phase(Lmat, sL, p, nb, (dir == 0 ? Lx : Ly) + k0, s)) != cudaSuccess) return e;
    }
  }
  return launch_plaquette_flux(a, Lx, Ly, flux, chern, s);
}

// ---------------------------------------------------------------------------
// Eigenphases of the Wilson matrices of a block of loops.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_geig_big(BigEigArgs a) {
  __shared__ GeigShared sh;
  __shared__ double red[64];
  const int p = a.p, tid = threadIdx.x, nt = blockDim.x;
  for (int l = blockIdx.x; l < a.nl; l += gridDim.x) {
    const int i = a.i0 + l;  // transverse index of the loop
    const long long k0 = (long long)i * a.N;
    if (a.min_gap) {
      double g = INFINITY;
      for (int j = tid; j < a.N; j += nt) g = fmin(g, a.gap[k0 + j]);
      g = block_min(g, red);
      if (tid == 0) a.min_gap[i] = g;
    }
    if (a.min_pso_gap && a.pso_gap) {
      double g = INFINITY;
      for (int j = tid; j < a.N; j += nt) g = fmin(g, a.pso_gap[k0 + j]);
      g = block_min(g, red);
      if (tid == 0) a.min_pso_gap[i] = g;
    }
    z64* W = a.W + (long long)l * a.sW;
    z64* lam = a.lam + (long long)l * p;
    z64* vec = a.vec + (long long)l * p;
    double* th = a.th + (long long)l * p;
    int* ord = a.ord + (long long)l * p;
    const int rc = geig(W, nullptr, p, p, false, lam, vec, &sh);
    if (rc != 0 && tid == 0) report(a.status, ST_ENOCONV, k0, 0.0);
    for (int c = tid; c < p; c += nt) th[c] = atan2(lam[c].im, lam[c].re);
    __syncthreads();
    for (int c = tid; c < p; c += nt) {
      const double x = rank_key(th[c]);
      int rank = 0;
      for (int d = 0; d < p; ++d) {
        const double y = rank_key(th[d]);
        rank += (y < x) || (y == x && d < c);
      }
      ord[rank] = c;
    }
    __syncthreads();
    for (int c = tid; c < p; c += nt) a.phases[(long long)i * p + c] = th[ord[c]];
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Spin-resolved loop with many occupied bands (Sec. IV).  The occupied-space spin
// operator S = U^dagger s U of a wave comes from one sparse application Y = sigma s U
// and one batched GEMM U^dagger Y; its eigen-decomposition runs on the tridiagonal
// path in FP64 (sigma = +1 for the sector s < 0, -1 for s > 0, so that the sector
// is always the lowest p/2 eigenvectors of sigma S); the sector states U V then go
// through the same batched-GEMM loop as the plain Wilson loop.
// ---------------------------------------------------------------------------
__global__ void k_spin_apply(const z64* U, z64* Y, long long W, int n, int p, const int* rowp,
                             const int* col, const z64* val, double sigma) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= W * n * p) return;
  const long long kw = e / ((long long)n * p);
  const int rc = int(e - kw * n * p), r = rc / p, c = rc - r * p;
  const z64* Uk = U + kw * (long long)n * p;
  z64 acc(0.0, 0.0);
  for (int q = rowp[r]; q < rowp[r + 1]; ++q) cfma(acc, val[q], Uk[(long long)col[q] * p + c]);
  Y[e] = sigma * acc;
}

cudaError_t launch_spin_apply(const z64* U, z64* Y, long long W, int n, int p, const int* rowp,
                              const int* col, const z64* val, double sigma, cudaStream_t s) {
  const long long tot = W * n * p;
  if (tot <= 0) return cudaSuccess;
  const long long blocks = (tot + 255) / 256;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
  k_spin_apply<<<unsigned(blocks), 256, 0, s>>>(U, Y, W, n, p, rowp, col, val, sigma);
  return cudaGetLastError();
}

__global__ void k_pso_post(const double* nu, int nval, long long W, long long k0, int p,
                           double sigma, double tol, int median, double* pso_evals, double* pso_gap,
                           DevStatus* status) {
  const long long kw = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (kw >= W) return;
  const double* v = nu + kw * nval;
  const int h = p / 2;
  const long long k = k0 + kw;
  const double lo = v[h - 1], hi = v[h];
  const double g = median ? hi - lo : fmin(fabs(lo), fabs(hi));
  if (pso_gap) pso_gap[k] = g;
  if (pso_evals)
    for (int c = 0; c < p; ++c) pso_evals[k * p + c] = sigma > 0.0 ? v[c] : -v[p - 1 - c];
  if (!((median || (lo < 0.0 && hi > 0.0)) && g > tol)) report(status, ST_EPSOGAP, k, g);
}

cudaError_t launch_pso_post(const double* nu, int nval, long long W, long long k0, int p,
                            double sigma, double tol, int median, double* pso_evals, double* pso_gap,
                            DevStatus* status, cudaStream_t s) {
  if (W <= 0) return cudaSuccess;
  k_pso_post<<<unsigned((W + 127) / 128), 128, 0, s>>>(nu, nval, W, k0, p, sigma, tol, median,
                                                       pso_evals, pso_gap, status);
  return cudaGetLastError();
}

__global__ void k_iota(long long* off, int* idx, long long W, long long stride) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= W) return;
  off[t] = t * stride;
  idx[t] = int(t);
}

cudaError_t launch_iota(long long* off, int* idx, long long W, long long stride, cudaStream_t s) {
  if (W <= 0) return cudaSuccess;
  k_iota<<<unsigned((W + 255) / 256), 256, 0, s>>>(off, idx, W, stride);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Eigenphases of large Wilson matrices on a cluster of GC_CTAS CTAs per loop: the
// same arithmetic as k_geig_big (Householder-Hessenberg, single-shift QR with the
// same shifts, rotations and deflation tests), organised so that one SM does not
// wait on one thread:
//  - Hessenberg: every CTA forms the Householder vector in its shared memory (same
//    data, same order, same bits); the left update is split over the columns, the
//    right update over the rows of the cluster; two cluster barriers per column.
//  - QR sweep in chunks of GC_W rotations: the first warp of CTA 0 chases the bulge
//    through the window rows [k0-1, kend+1] x columns [k0-1, kend] (kend = k0 + GC_W)
//    in shared memory and publishes the rotations; then every thread of the cluster
//    applies the chunk's row rotations to one column right of the window, or its
//    column rotations to one row above it, in order.  Right of the window only the
//    chunk's row rotations act and above it only its column rotations, so every
//    entry receives its rotations in the sequential order.
//  - The matrix lives in global memory and other SMs of the cluster write it: every
//    read bypasses L1 (ld.global.cg); the cluster barriers order the accesses.
// ---------------------------------------------------------------------------
constexpr int GC_CTAS = 4, GC_W = 16, GC_THREADS = 256;
constexpr int GC_WR = GC_W + 3, GC_WC = GC_W + 2;  // window rows, columns
constexpr int GC_MIN_P = 128;                      // smaller p: k_geig_big

struct GcCtl {
  double mu[4];  // the shift, as the solver's element type (16 bytes)
  int active, l, hi, fail;
};

// Block-wide double-float sum (`red` holds >= blockDim.x / 32 df).
__device__ __forceinline__ df block_sum_df(df v, df* red) {
  for (int o = 16; o > 0; o >>= 1) v = v + shfl_xor_df(v, o);
  const int w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[w] = v;
  __syncthreads();
  df t = red[0];
  for (int k = 1; k < nw; ++k) t = t + red[k];
  __syncthreads();
  return t;
}

// 1 / sqrt(a) to double-float accuracy: df_rsqrt and one more Newton step.
__device__ __forceinline__ df gc_rsqrt(df a) {
  const df y = df_rsqrt(a);
  return y * (df(1.5f) - df(0.5f) * (a * (y * y)));
}

// Magnitudes and exact power-of-two scalings on the leading floats: double-float has
// the float exponent range, so squares of entries below ~1e-19 (the trailing entries
// of a nearly singular Wilson matrix) would underflow.
__device__ __forceinline__ float abs_hi(cdf a) { return hypotf(a.re.hi, a.im.hi); }
__device__ __forceinline__ float cmax_hi(cdf a) { return fmaxf(fabsf(a.re.hi), fabsf(a.im.hi)); }
__device__ __forceinline__ cdf cscale(cdf a, float s) {
  return cdf(df(a.re.hi * s, a.re.lo * s), df(a.im.hi * s, a.im.lo * s));
}
// 2^-e with m = f 2^e, 1/2 <= f < 1 (m > 0 finite): scales m into [1/2, 1).
__device__ __forceinline__ float pow2_inv(float m) {
  int e;
  frexpf(m, &e);
  return ldexpf(1.f, -e);
}

// Element arithmetic of the cluster solver.  z64: the FP64 solver of geig.cuh
// (givens, geig_negligible_v, geig_shift).  cdf: the same steps in complex
// double-float on the FP32 pipe (mixed request): Givens from double-float reciprocal
// square roots; the deflation test of geig_negligible_v on the leading floats with
// eps = 2^-43 (double-float resolution 2^-48); the Wilkinson shift from the principal
// double-float square root; eigenphases by df_phase.
template <typename E>
struct GcA;
template <>
struct GcA<z64> {
  using R = double;
  __device__ static z64 ld(const z64* q) { return z64(__ldcg(&q->re), __ldcg(&q->im)); }
  __device__ static z64 zero() { return z64(0.0, 0.0); }
  __device__ static z64 one() { return z64(1.0, 0.0); }
  __device__ static R abs(z64 a) { return zabs(a); }
  __device__ static R sqrt_(R x) { return sqrt(x); }
  __device__ static R inv_sqrt(R x) { return 1.0 / sqrt(x); }
  __device__ static R div(R x, R y) { return x / y; }
  __device__ static bool positive(R x) { return x > 0.0; }
  __device__ static R bsum(R v, double* red) { return block_sum(v, red); }
  __device__ static z64 shfl_xor(z64 v, int o) {
    return z64(__shfl_xor_sync(0xffffffffu, v.re, o), __shfl_xor_sync(0xffffffffu, v.im, o));
  }
  __device__ static bool negligible(z64 h11, z64 h12, z64 h21, z64 h22) {
    return geig_negligible_v(h11, h12, h21, h22, 2.220446049250313e-16);
  }
  __device__ static z64 shift(z64 a, z64 b, z64 c, z64 d, int iter, z64 h2, bool has_h2) {
    return geig_shift(a, b, c, d, iter, has_h2 ? zabs(h2) : 0.0);
  }
  __device__ static void rot(z64 x, z64 y, R& c, z64& sr) { givens(x, y, c, sr); }
  __device__ static double phase(z64 z) { return atan2(z.im, z.re); }
};
template <>
struct GcA<cdf> {
  using R = df;
  __device__ static cdf ld(const cdf* q) {
    return cdf(df(__ldcg(&q->re.hi), __ldcg(&q->re.lo)), df(__ldcg(&q->im.hi), __ldcg(&q->im.lo)));
  }
  __device__ static cdf zero() { return cdf_zero(); }
  __device__ static cdf one() { return cdf(df(1.f), df(0.f)); }
  __device__ static R abs(cdf a) { return df_sqrt(abs2(a)); }
  __device__ static R sqrt_(R x) { return df_sqrt(x); }
  __device__ static R inv_sqrt(R x) { return gc_rsqrt(x); }
  __device__ static R div(R x, R y) { return df_div(x, y); }
  __device__ static bool positive(R x) { return x.hi > 0.f; }
  __device__ static R bsum(R v, double* red) { return block_sum_df(v, reinterpret_cast<df*>(red)); }
  __device__ static cdf shfl_xor(cdf v, int o) { return cdf(shfl_xor_df(v.re, o), shfl_xor_df(v.im, o)); }
  __device__ static bool negligible(cdf h11, cdf h12, cdf h21, cdf h22) {
    // 2^-43: above the noise floor a few double-float roundings leave on the
    // subdiagonal (a test at 2^-47 stalled short of deflation)
    const float eps = 1.1368683772161603e-13f;
    const float sub = abs_hi(h21), dia = abs_hi(h22) + abs_hi(h11);
    bool small = sub <= eps * dia || sub < 1e-36f;
    if (!small && sub <= dia) {
      const float x = abs_hi(h12);
      const float ab = fmaxf(sub, x), ba = fminf(sub, x);
      const float y = abs_hi(h11 - h22);
      const float aa = fmaxf(abs_hi(h22), y), bb = fminf(abs_hi(h22), y);
      const float sc = aa + ab;
      small = ba * (ab / sc) <= fmaxf(1e-36f, eps * (bb * (aa / sc)));
    }
    return small;
  }
  // computed on the 2 x 2 scaled by a power of two (the shift scales with it)
  __device__ static cdf shift(cdf a, cdf b, cdf c, cdf d, int iter, cdf h2, bool has_h2) {
    float m = fmaxf(fmaxf(cmax_hi(a), cmax_hi(b)), fmaxf(cmax_hi(c), cmax_hi(d)));
    if (has_h2) m = fmaxf(m, cmax_hi(h2));
    if (!(m > 0.f) || !(m < INFINITY)) return d;
    const float sc = pow2_inv(m), us = 1.f / sc;
    a = cscale(a, sc);
    b = cscale(b, sc);
    c = cscale(c, sc);
    d = cscale(d, sc);
    if (iter > 0 && iter % 12 == 0) {
      const df ex = abs(c) + (has_h2 ? abs(cscale(h2, sc)) : df(0.f));
      return cscale(d + cdf(df(0.75f) * ex, df(0.f)), us);
    }
    const cdf half = df(0.5f) * (a - d);
    const cdf sq = csqrt_df(half * half + b * c);
    const cdf m1 = d + half - sq, m2 = d + half + sq;
    return cscale(df_gt(abs2(m1 - d), abs2(m2 - d)) ? m2 : m1, us);
  }
  // computed on x, y scaled by a power of two (c and s do not depend on the scale)
  __device__ static void rot(cdf x, cdf y, R& c, cdf& sr) {
    const float m = fmaxf(cmax_hi(x), cmax_hi(y));
    if (!(m > 0.f)) {
      c = df(1.f);
      sr = cdf_zero();
      return;
    }
    const float sc = pow2_inv(m);
    x = cscale(x, sc);
    y = cscale(y, sc);
    const df ax2 = abs2(x), ay2 = abs2(y);
    if (ay2.hi == 0.f) {
      c = df(1.f);
      sr = cdf_zero();
      return;
    }
    if (ax2.hi == 0.f) {
      c = df(0.f);
      const df iy = gc_rsqrt(ay2);
      sr = cdf(y.re * iy, -(y.im * iy));
      return;
    }
    const df ir = gc_rsqrt(ax2 + ay2), iax = gc_rsqrt(ax2);
    c = ax2 * iax * ir;
    const cdf ux(x.re * iax, x.im * iax);
    sr = ir * (ux * conj(y));
  }
  __device__ static double phase(cdf z) { return df_phase(z); }
};

// geig_split_point with L1-bypassing loads, for the first warp.
template <typename E>
__device__ __forceinline__ int gc_split_point(const E* H, int p, int hi) {
  using A = GcA<E>;
  const int lane = threadIdx.x & 31;
  for (int base = hi; base >= 1; base -= 32) {
    const int l = base - lane;
    bool f = false;
    if (l >= 1)
      f = A::negligible(A::ld(H + (long long)(l - 1) * p + l - 1), A::ld(H + (long long)(l - 1) * p + l),
                        A::ld(H + (long long)l * p + l - 1), A::ld(H + (long long)l * p + l));
    const unsigned m = __ballot_sync(0xffffffffu, f);
    if (m) return base - (__ffs(m) - 1);
  }
  return 0;
}

// The bulge chase of rotations k0 .. kend-1 on the window (first warp of CTA 0).
template <typename E>
__device__ void gc_chase(E* H, int p, int l, int hi, int k0, int kend, E mu, E* win, E* rot) {
  using A = GcA<E>;
  using R = typename A::R;
  const int lane = threadIdx.x & 31;
  const int rlo = k0 > l ? k0 - 1 : l, rhi = min(kend + 1, hi), clo = rlo, chi = kend;
  const int nr = rhi - rlo + 1, nc = chi - clo + 1;
  for (int e = lane; e < nr * nc; e += 32) {
    const int r = e / nc, c = e - r * nc;
    win[r * GC_WC + c] = A::ld(H + (long long)(rlo + r) * p + clo + c);
  }
  __syncwarp();
#define GCW(r, c) win[((r) - rlo) * GC_WC + ((c) - clo)]
  for (int k = k0; k < kend; ++k) {
    const E x = k == l ? GCW(l, l) - mu : GCW(k, k - 1);
    const E y = k == l ? GCW(l + 1, l) : GCW(k + 1, k - 1);
    R c;
    E sr;
    A::rot(x, y, c, sr);  // every lane, same values
    const int cb = k > l ? k - 1 : l;
    for (int col = cb + lane; col <= chi; col += 32) {
      const E xv = GCW(k, col), yv = GCW(k + 1, col);
      GCW(k, col) = c * xv + sr * yv;
      GCW(k + 1, col) = c * yv - conj(sr) * xv;
    }
    __syncwarp();
    if (lane == 0 && k > l) GCW(k + 1, k - 1) = A::zero();
    __syncwarp();
    const int re = min(k + 2, hi);
    for (int row = rlo + lane; row <= re; row += 32) {
      const E xv = GCW(row, k), yv = GCW(row, k + 1);
      GCW(row, k) = c * xv + yv * conj(sr);
      GCW(row, k + 1) = c * yv - xv * sr;
    }
    __syncwarp();
    if (lane == 0) {
      rot[2 * (k - k0)] = E(c, R(0.0));
      rot[2 * (k - k0) + 1] = sr;
    }
  }
  for (int e = lane; e < nr * nc; e += 32) {
    const int r = e / nc, c = e - r * nc;
    H[(long long)(rlo + r) * p + clo + c] = win[r * GC_WC + c];
  }
#undef GCW
}

template <typename E>
__global__ void __launch_bounds__(GC_THREADS) k_geig_cluster(BigEigArgs a) {
  using A = GcA<E>;
  using R = typename A::R;
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char gsm[];
  const int p = a.p, tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5;
  E* vsh = reinterpret_cast<E*>(gsm);  // p: Householder vector
  E* win = vsh + p;                    // GC_WR x GC_WC window (CTA 0)
  E* rsh = win + GC_WR * GC_WC;        // 2 GC_W: the chunk's rotations
  __shared__ double red[32];
  const int rank = int(cluster.block_rank());
  const int lp = blockIdx.x / GC_CTAS;  // the cluster's loop: every CTA of it runs every
                                        // cluster barrier below
  const int gtid = rank * nt + tid, gnt = GC_CTAS * nt;
  const int nwarp = nt >> 5, gwarp = rank * nwarp + warp, gnwarp = GC_CTAS * nwarp;
  E* H = reinterpret_cast<E*>(a.W) + (long long)lp * a.sW;
  E* lam = reinterpret_cast<E*>(a.lam) + (long long)lp * p;
  E* rot = reinterpret_cast<E*>(a.vec) + (long long)lp * p;
  GcCtl* ctl = reinterpret_cast<GcCtl*>(a.ctl + 8LL * lp);
  if (rank == 0 && tid == 0) ctl->fail = 0;  // read by CTA 0 alone, at the end
  // --- Householder reduction to Hessenberg form
  for (int c = 0; c + 2 < p; ++c) {
    R nrm2 = R(0.0);
    for (int r = c + 1 + tid; r < p; r += nt) nrm2 = nrm2 + abs2(A::ld(H + (long long)r * p + c));
    nrm2 = A::bsum(nrm2, red);
    const E x0 = A::ld(H + (long long)(c + 1) * p + c);
    const R tail = nrm2 - abs2(x0);
    // a column already reduced is skipped; the barriers below run regardless, so the
    // CTAs of the cluster pass the same barriers whatever the data
    const bool work = A::positive(tail);
    const R nx = A::sqrt_(nrm2), ax0 = A::abs(x0);
    const E ph = A::positive(ax0) ? E(A::div(x0.re, ax0), A::div(x0.im, ax0)) : A::one();
    const R v0m = ax0 + nx, nv = work ? A::inv_sqrt(v0m * v0m + tail) : R(0.0);
    if (work)
      for (int r = c + 1 + tid; r < p; r += nt)
        vsh[r] = r == c + 1 ? E(nv * v0m * ph.re, nv * v0m * ph.im) : nv * A::ld(H + (long long)r * p + c);
    __syncthreads();
    // left: H <- (I - 2 v v^dagger) H on rows c+1.., the cluster's columns c+1..
    for (int col = c + 1 + gtid; work && col < p; col += gnt) {
      E w = A::zero();
#pragma unroll 4
      for (int r = c + 1; r < p; ++r) cfma_conj(w, vsh[r], A::ld(H + (long long)r * p + col));
#pragma unroll 4
      for (int r = c + 1; r < p; ++r) {
        E* h = H + (long long)r * p + col;
        *h = A::ld(h) - R(2.0) * (vsh[r] * w);
      }
    }
    cluster.sync();
    if (work && rank == 0)  // column c (every CTA has read it)
      for (int r = c + 1 + tid; r < p; r += nt) H[(long long)r * p + c] = r == c + 1 ? (-nx) * ph : A::zero();
    // right: H <- H (I - 2 v v^dagger) on columns c+1.., one warp per row of the cluster
    for (int row = gwarp; work && row < p; row += gnwarp) {
      E* hr = H + (long long)row * p;
      E w = A::zero();
      for (int k = c + 1 + lane; k < p; k += 32) cfma(w, A::ld(hr + k), vsh[k]);
      for (int o = 16; o > 0; o >>= 1) w = w + A::shfl_xor(w, o);
      for (int k = c + 1 + lane; k < p; k += 32) hr[k] = A::ld(hr + k) - R(2.0) * (w * conj(vsh[k]));
    }
    cluster.sync();
  }
  // --- shifted QR sweeps; the first warp of CTA 0 keeps the iteration state
  int hi_s = p - 1, iter = 0, total = 0;
  const int cap = 120 * p + 120;
  while (true) {
    if (rank == 0 && warp == 0) {
      int hi = hi_s, l = 0, active = 0, fail = 0;
      E mu = A::zero();
      while (hi >= 0) {
        if (hi == 0) {
          if (lane == 0) lam[0] = A::ld(H);
          hi = -1;
          break;
        }
        const int sl = gc_split_point(H, p, hi);
        if (lane == 0 && sl > 0) H[(long long)sl * p + sl - 1] = A::zero();
        __syncwarp();
        if (sl == hi) {
          if (lane == 0) lam[hi] = A::ld(H + (long long)hi * p + hi);
          --hi;
          iter = 0;
          continue;
        }
        mu = A::shift(A::ld(H + (long long)(hi - 1) * p + hi - 1), A::ld(H + (long long)(hi - 1) * p + hi),
                      A::ld(H + (long long)hi * p + hi - 1), A::ld(H + (long long)hi * p + hi), iter,
                      hi >= 2 ? A::ld(H + (long long)(hi - 1) * p + hi - 2) : A::zero(), hi >= 2);
        l = sl;
        active = 1;
        break;
      }
      ++iter;
      ++total;
      if (total > cap) {
        fail = 1;
        active = 0;
        hi = -1;
      }
      hi_s = hi;
      if (lane == 0) {
        *reinterpret_cast<E*>(ctl->mu) = mu;
        ctl->active = active;
        ctl->l = l;
        ctl->hi = hi;
        if (fail) ctl->fail = 1;
      }
    }
    cluster.sync();
    const int active = __ldcg(&ctl->active);
    if (!active) break;  // the same value in every CTA of the cluster
    const int l = __ldcg(&ctl->l), hi = __ldcg(&ctl->hi);
    const E mu = A::ld(reinterpret_cast<const E*>(ctl->mu));
    for (int k0 = l; k0 < hi; k0 += GC_W) {
      const int kend = min(k0 + GC_W, hi), nk = kend - k0;
      const int rlo = k0 > l ? k0 - 1 : l, chi = kend;
      if (rank == 0 && warp == 0) gc_chase(H, p, l, hi, k0, kend, mu, win, rot);
      cluster.sync();
      for (int e = tid; e < 2 * nk; e += nt) rsh[e] = A::ld(rot + e);
      __syncthreads();
      // right of the window: rows k0 .. kend of columns chi+1 .. hi, row rotations in
      // order; above it: columns k0 .. kend of rows l .. rlo-1, column rotations in order
      const int nA = hi - chi, nB = rlo - l;
      for (int t = gtid; t < nA + nB; t += gnt) {
        if (t < nA) {
          E* hc = H + (long long)k0 * p + chi + 1 + t;
          E v[GC_W + 1];
#pragma unroll
          for (int q = 0; q <= GC_W; ++q)
            if (q <= nk) v[q] = A::ld(hc + (long long)q * p);
#pragma unroll
          for (int q = 0; q < GC_W; ++q)
            if (q < nk) {
              const R c = rsh[2 * q].re;
              const E sr = rsh[2 * q + 1];
              const E x = v[q], y = v[q + 1];
              v[q] = c * x + sr * y;
              v[q + 1] = c * y - conj(sr) * x;
            }
#pragma unroll
          for (int q = 0; q <= GC_W; ++q)
            if (q <= nk) hc[(long long)q * p] = v[q];
        } else {
          E* hr = H + (long long)(l + t - nA) * p + k0;
          E v[GC_W + 1];
#pragma unroll
          for (int q = 0; q <= GC_W; ++q)
            if (q <= nk) v[q] = A::ld(hr + q);
#pragma unroll
          for (int q = 0; q < GC_W; ++q)
            if (q < nk) {
              const R c = rsh[2 * q].re;
              const E sr = rsh[2 * q + 1];
              const E x = v[q], y = v[q + 1];
              v[q] = c * x + y * conj(sr);
              v[q + 1] = c * y - x * sr;
            }
#pragma unroll
          for (int q = 0; q <= GC_W; ++q)
            if (q <= nk) hr[q] = v[q];
        }
      }
      cluster.sync();
    }
  }
  if (rank != 0) return;  // after the last cluster barrier
  // --- CTA 0: gaps, phases in ascending order
  const int i = a.i0 + lp;
  const long long k0 = (long long)i * a.N;
  if (a.min_gap) {
    double g = INFINITY;
    for (int j = tid; j < a.N; j += nt) g = fmin(g, a.gap[k0 + j]);
    g = block_min(g, red);
    if (tid == 0) a.min_gap[i] = g;
  }
  if (a.min_pso_gap && a.pso_gap) {
    double g = INFINITY;
    for (int j = tid; j < a.N; j += nt) g = fmin(g, a.pso_gap[k0 + j]);
    g = block_min(g, red);
    if (tid == 0) a.min_pso_gap[i] = g;
  }
  if (tid == 0 && __ldcg(&ctl->fail)) report(a.status, ST_ENOCONV, k0, 0.0);
  double* th = a.th + (long long)lp * p;
  int* ord = a.ord + (long long)lp * p;
  for (int c = tid; c < p; c += nt) th[c] = A::phase(A::ld(lam + c));
  __syncthreads();
  for (int c = tid; c < p; c += nt) {
    const double x = rank_key(th[c]);
    int rnk = 0;
    for (int d = 0; d < p; ++d) {
      const double y = rank_key(th[d]);
      rnk += (y < x) || (y == x && d < c);
    }
    ord[rnk] = c;
  }
  __syncthreads();
  for (int c = tid; c < p; c += nt) a.phases[(long long)i * p + c] = th[ord[c]];
}

template <typename E>
static cudaError_t launch_geig_cluster(const BigEigArgs& a, cudaStream_t s) {
  const size_t smem = (size_t(a.p) + GC_WR * GC_WC + 2 * GC_W) * sizeof(E);
  static size_t cached = 0;
  cudaError_t e = set_smem_once(k_geig_cluster<E>, smem, cached);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(unsigned(GC_CTAS * a.nl));
  cfg.blockDim = dim3(GC_THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = GC_CTAS;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_geig_cluster<E>, a);
}

bool geig_df_eligible(int p) { return p >= GC_MIN_P; }

cudaError_t launch_geig_big(const BigEigArgs& a, cudaStream_t s) {
  if (a.nl <= 0) return cudaSuccess;
  if (a.df) {
    if (!a.ctl || !geig_df_eligible(a.p)) return cudaErrorInvalidValue;
    return launch_geig_cluster<cdf>(a, s);
  }
  if (a.p < GC_MIN_P || !a.ctl) {
    k_geig_big<<<a.nl, 256, 0, s>>>(a);
    return cudaGetLastError();
  }
  return launch_geig_cluster<z64>(a, s);
}

}  // namespace bw
