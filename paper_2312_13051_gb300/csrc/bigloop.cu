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
#include <float.h>

#include <algorithm>
#include <cstring>

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

__global__ void __launch_bounds__(256) k_zgemm(GemmArgs g) {
  __shared__ z64 As[GK][GT];
  __shared__ z64 Bs[GK][GT];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int tiles_n = (g.n + GT - 1) / GT;
  const long long bl = g.b0 + blockIdx.y, b = g.kfirst + bl;
  const long long ba = g.a_next_N > 0 ? (b / g.a_next_N) * g.a_next_N + (b % g.a_next_N + 1) % g.a_next_N
                       : g.a_mod > 0  ? (b + g.a_shift) % g.a_mod
                                      : b;
  const int r0 = (blockIdx.x / tiles_n) * GT, c0 = (blockIdx.x % tiles_n) * GT;
  const z64* A = g.A + ba * g.sA;
  const z64* B = g.B + b * g.sB;
  z64* C = g.C + bl * g.sC;
  z64 acc[4][4];
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int y = 0; y < 4; ++y) acc[x][y] = z64(0.0, 0.0);
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
      z64 v(0.0, 0.0);
      if (gr < g.m && gk < g.k) {
        if (g.opA) {
          const z64 t = A[(long long)gk * g.lda + gr];
          v = z64(t.re, -t.im);
        } else {
          v = A[(long long)gr * g.lda + gk];
        }
      }
      As[kk][r] = v;
    }
    for (int e = tid; e < GK * GT; e += 256) {
      const int kk = e / GT, c = e - kk * GT;
      const int gc = c0 + c, gk = k0 + kk;
      Bs[kk][c] = (gc < g.n && gk < g.k) ? B[(long long)gk * g.ldb + gc] : z64(0.0, 0.0);
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < GK; ++kk) {
      z64 av[4], bv[4];
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

cudaError_t launch_zgemm(const GemmArgs& g, cudaStream_t s) {
  if (g.batch <= 0 || g.m <= 0 || g.n <= 0) return cudaSuccess;
  const long long tiles = (long long)((g.m + GT - 1) / GT) * ((g.n + GT - 1) / GT);
  if (tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
  for (long long b0 = 0; b0 < g.batch; b0 += 65535) {  // grid.y holds at most 65535
    GemmArgs h = g;
    h.b0 = b0;
    dim3 grid(unsigned(tiles), unsigned(std::min<long long>(65535, g.batch - b0)));
    k_zgemm<<<grid, 256, 0, s>>>(h);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
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

cudaError_t launch_geig_big(const BigEigArgs& a, cudaStream_t s) {
  if (a.nl <= 0) return cudaSuccess;
  k_geig_big<<<a.nl, 256, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace bw
