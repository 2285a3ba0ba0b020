// Loop kernels: overlaps, ordered products and eigenphases (Eq. 2), and the nested
// loop over Wannier states (Eq. 8).
//
//  - k_overlaps: M_j = U(k_{j+1})^dagger U(k_j) for every k-point of the plane, the
//                loop closing on j = 0 (optionally replaced by its unitary polar
//                factor).
//  - k_loops:    one CTA per transverse index: W = M_{N-1} ... M_0 (later k on the
//                left), general complex eigenvalues, theta = arg(lambda) ascending.
//                For the nested loop also the right eigenvectors nu of the chosen
//                sector, carried along the loop by nu_{j+1} = M_j nu_j (the loop
//                based at k_{j+1} is M_j W_j M_j^{-1}), orthonormalised, and the
//                Wannier states w = U(k_j) nu_j.
//  - k_nested:   one CTA per base point: product of w(i+1)^dagger w(i) along the
//                transverse direction (closed on i = 0) and its eigenphases.
//  - k_winding:  the winding of the summed Wannier centres over the transverse
//                direction (Eq. 6).
#include <float.h>

#include <cooperative_groups.h>
#include <cstring>
#include <type_traits>

#include "df32.cuh"
#include "geig.cuh"
#include "jacobi.cuh"
#include "launch.h"
#include "quad.cuh"

namespace bw {

__device__ __forceinline__ double phase_of(z64 z) { return atan2(z.im, z.re); }
__device__ __forceinline__ double phase_E(z64 z) { return phase_of(z); }
__device__ __forceinline__ double phase_E(cdf z) { return df_phase(z); }

// Planes stacked along the rows: the nested loop of base point b (of N_s N) runs over
// the rows of plane s = b / N and closes within it.
__host__ __device__ __forceinline__ int n_planes(const LoopArgs& a) { return a.N_s > 1 ? a.N_s : 1; }

// Ranks th[0..p) ascending (stable) into ord.
__device__ void rank_sort(const double* th, int p, int* ord) {
  for (int a = threadIdx.x; a < p; a += blockDim.x) {
    int rank = 0;
    const double x = rank_key(th[a]);
    for (int b = 0; b < p; ++b) {
      const double y = rank_key(th[b]);
      rank += (y < x) || (y == x && b < a);
    }
    ord[rank] = a;
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Overlaps
// ---------------------------------------------------------------------------
__global__ void k_overlaps(LoopArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int n = a.n, p = a.p, N = a.N, tid = threadIdx.x, nt = blockDim.x;
  const long long K = (long long)N * a.N_t;
  z64* Ms = reinterpret_cast<z64*>(smem);            // p x p
  z64* P = Ms + p * p;                               // p x p
  z64* Vp = P + p * p;                               // p x p
  z64* Tp = Vp + p * p;                              // p x p
  JacRot<double>* rot = reinterpret_cast<JacRot<double>*>(Tp + p * p);
  double* red = reinterpret_cast<double*>(rot + (p / 2 + 2));
  for (long long k = blockIdx.x; k < K; k += gridDim.x) {
    const int i = int(k / N), j = int(k - (long long)i * N);
    const long long kn = (long long)i * N + (j + 1 == N ? 0 : j + 1);
    const z64* Uh = a.U + k * (long long)n * p;
    const z64* Un = a.U + kn * (long long)n * p;
    z64* M = a.M + k * (long long)p * p;
    if (!a.unitarise) {
      for (int e = tid; e < p * p; e += nt) {
        const int r = e / p, c = e - r * p;
        z64 acc(0.0, 0.0);
        for (int q = 0; q < n; ++q) cfma_conj(acc, Un[q * p + r], Uh[q * p + c]);
        M[e] = acc;
      }
      continue;
    }
    for (int e = tid; e < p * p; e += nt) {
      const int r = e / p, c = e - r * p;
      z64 acc(0.0, 0.0);
      for (int q = 0; q < n; ++q) cfma_conj(acc, Un[q * p + r], Uh[q * p + c]);
      Ms[e] = acc;
    }
    __syncthreads();
    // polar factor: M (M^dagger M)^{-1/2} = M V diag(1/sigma) V^dagger
    for (int e = tid; e < p * p; e += nt) {
      const int r = e / p, c = e - r * p;
      z64 acc(0.0, 0.0);
      for (int q = 0; q < p; ++q) cfma_conj(acc, Ms[q * p + r], Ms[q * p + c]);
      P[e] = (r == c) ? z64(acc.re, 0.0) : acc;
    }
    __syncthreads();
    const int sw = jacobi_eigh<double>(P, Vp, p, p, a.max_sweeps, rot, red);
    if (sw < 0 && tid == 0) report(a.status, ST_ENOCONV, k, 0.0);
    // P <- V diag(1/sigma) V^dagger (sigma^2 on P's diagonal)
    for (int e = tid; e < p * p; e += nt) {
      const int r = e / p, c = e - r * p;
      z64 acc(0.0, 0.0);
      for (int q = 0; q < p; ++q) {
        const double s2 = P[q * p + q].re;
        const double w = s2 > 0.0 ? 1.0 / sqrt(s2) : 0.0;
        const z64 v = Vp[r * p + q] * conj(Vp[c * p + q]);
        acc = acc + w * v;
      }
      Tp[e] = acc;
    }
    __syncthreads();
    for (int e = tid; e < p * p; e += nt) {
      const int r = e / p, c = e - r * p;
      z64 acc(0.0, 0.0);
      for (int q = 0; q < p; ++q) cfma(acc, Ms[r * p + q], Tp[q * p + c]);
      M[e] = acc;
    }
    __syncthreads();
  }
}

// Mixed precision, p > 4: the overlaps in double-float on the FP32 pipe.  One CTA per
// k-point; the two FP64 state blocks pass through shared memory in chunks of
// OVL_ROWS rows, converted to double-float once per element, and each thread
// accumulates a 4 x 4 tile of M (four values of each block per row q feed sixteen
// products); M is written back in FP64.
constexpr int OVL_ROWS = 32, OVL_THREADS = 256;

__global__ void __launch_bounds__(OVL_THREADS, 1) k_overlaps_df(LoopArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int n = a.n, p = a.p, N = a.N, tid = threadIdx.x, pp = p * p;
  const long long K = (long long)N * a.N_t;
  cdf* Ah = reinterpret_cast<cdf*>(smem);        // OVL_ROWS x p, U(k_j)
  cdf* An = Ah + OVL_ROWS * p;                   // OVL_ROWS x p, U(k_{j+1})
  // thread (ty, tx) of a 16 x 16 grid owns rows ty + 16 u and columns tx + 16 v of M
  const int tx = tid & 15, ty = tid >> 4;
  for (long long k = blockIdx.x; k < K; k += gridDim.x) {
    const int i = int(k / N), j = int(k - (long long)i * N);
    const long long kn = (long long)i * N + (j + 1 == N ? 0 : j + 1);
    const z64* Uh = a.U + k * (long long)n * p;
    const z64* Un = a.U + kn * (long long)n * p;
    cdf acc[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) acc[u][v] = cdf_zero();
    for (int r0 = 0; r0 < n; r0 += OVL_ROWS) {
      const int rows = min(OVL_ROWS, n - r0);
      for (int e = tid; e < rows * p; e += OVL_THREADS) {
        Ah[e] = cdf_from(Uh[(long long)r0 * p + e]);
        An[e] = cdf_from(Un[(long long)r0 * p + e]);
      }
      __syncthreads();
      for (int q = 0; q < rows; ++q) {
        cdf an[4], ah[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int r = ty + 16 * u, c = tx + 16 * u;
          an[u] = r < p ? An[q * p + r] : cdf_zero();
          ah[u] = c < p ? Ah[q * p + c] : cdf_zero();
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) cfma_conj(acc[u][v], an[u], ah[v]);
      }
      __syncthreads();
    }
    z64* M = a.M + k * (long long)pp;
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const int r = ty + 16 * u, c = tx + 16 * v;
        if (r < p && c < p) M[r * p + c] = cdf_to_z64(acc[u][v]);
      }
  }
}

// ---------------------------------------------------------------------------
// Per-loop product, eigenphases and (nested) Wannier states
// ---------------------------------------------------------------------------
struct LoopSmem {
  size_t X, Y, Ms, G, lam, vec, th, key, ord, sh, red, total;
};

// df: room for one overlap matrix in double-float (the mixed request's product)
__host__ __device__ inline LoopSmem loop_layout(int p, int m, bool df = false) {
  auto al = [](size_t x) { return (x + 15) & ~size_t(15); };
  LoopSmem L;
  size_t o = 0;
  L.X = o; o = al(o + size_t(p) * p * sizeof(z64));
  L.Y = o; o = al(o + size_t(p) * p * sizeof(z64));
  L.Ms = o; o = al(o + (df ? size_t(p) * p * sizeof(cdf) : 0));
  L.G = o; o = al(o + size_t(m) * m * sizeof(z64));
  L.lam = o; o = al(o + size_t(p) * sizeof(z64));
  L.vec = o; o = al(o + size_t(p) * sizeof(z64));
  L.th = o; o = al(o + size_t(p) * sizeof(double));
  L.key = o; o = al(o + size_t(p) * sizeof(double));
  L.ord = o; o = al(o + size_t(p) * sizeof(int));
  L.sh = o; o = al(o + sizeof(GeigShared));
  L.red = o; o = al(o + 64 * sizeof(double));
  L.total = o;
  return L;
}

__global__ void k_loops(LoopArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int n = a.n, p = a.p, N = a.N, tid = threadIdx.x, nt = blockDim.x;
  const int m = a.nested ? a.m : 1;
  const LoopSmem L = loop_layout(p, m, a.df_overlaps != 0);
  z64* X = reinterpret_cast<z64*>(smem + L.X);
  z64* Y = reinterpret_cast<z64*>(smem + L.Y);
  z64* lam = reinterpret_cast<z64*>(smem + L.lam);
  z64* vec = reinterpret_cast<z64*>(smem + L.vec);
  double* th = reinterpret_cast<double*>(smem + L.th);
  double* key = reinterpret_cast<double*>(smem + L.key);
  int* ord = reinterpret_cast<int*>(smem + L.ord);
  GeigShared* sh = reinterpret_cast<GeigShared*>(smem + L.sh);
  double* red = reinterpret_cast<double*>(smem + L.red);

  for (int i = blockIdx.x; i < a.N_t; i += gridDim.x) {
    const long long k0 = (long long)i * N;
    // minimum gaps along the loop
    if (a.min_gap || a.min_pso_gap) {
      double g = INFINITY, gp = INFINITY;
      for (int j = tid; j < N; j += nt) {
        if (a.gap) g = fmin(g, a.gap[k0 + j]);
        if (a.pso_gap) gp = fmin(gp, a.pso_gap[k0 + j]);
      }
      g = block_min(g, red);
      gp = block_min(gp, red);
      if (tid == 0) {
        if (a.min_gap) a.min_gap[i] = g;
        if (a.min_pso_gap) a.min_pso_gap[i] = gp;
      }
    }
    // W = M_{N-1} ... M_0
    z64* W = X;
    z64* T = Y;
    if (a.df_overlaps) {
      // mixed request: the product in double-float on the FP32 pipe; each M_j is
      // staged in shared memory once, each thread advances four entries at a time
      cdf* Wd = reinterpret_cast<cdf*>(X);
      cdf* Td = reinterpret_cast<cdf*>(Y);
      cdf* Md = reinterpret_cast<cdf*>(smem + L.Ms);
      for (int e = tid; e < p * p; e += nt) {
        const int r = e / p, c = e - r * p;
        Wd[e] = cdf(df(r == c ? 1.f : 0.f), df(0.f));
      }
      for (int j = 0; j < N; ++j) {
        const z64* M = a.M + (k0 + j) * (long long)p * p;
        for (int e = tid; e < p * p; e += nt) Md[e] = cdf_from(M[e]);
        __syncthreads();
        for (int e0 = tid; e0 < p * p; e0 += 4 * nt) {
          cdf acc[4];
          int rr[4], cc[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int e = min(e0 + u * nt, p * p - 1);
            rr[u] = e / p;
            cc[u] = e - rr[u] * p;
            acc[u] = cdf_zero();
          }
          for (int q = 0; q < p; ++q)
#pragma unroll
            for (int u = 0; u < 4; ++u) cfma(acc[u], Md[rr[u] * p + q], Wd[q * p + cc[u]]);
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (e0 + u * nt < p * p) Td[e0 + u * nt] = acc[u];
        }
        __syncthreads();
        cdf* t = Wd; Wd = Td; Td = t;
      }
      // back to FP64 in place for the eigen-decomposition
      z64* Wz = reinterpret_cast<z64*>(Wd);
      for (int e = tid; e < p * p; e += nt) {
        const cdf v = Wd[e];
        Wz[e] = cdf_to_z64(v);
      }
      __syncthreads();
      W = Wz;
      T = Wz == X ? Y : X;
    } else {
      for (int e = tid; e < p * p; e += nt) {
        const int r = e / p, c = e - r * p;
        W[e] = z64(double(r == c), 0.0);
      }
      __syncthreads();
      for (int j = 0; j < N; ++j) {
        const z64* M = a.M + (k0 + j) * (long long)p * p;
        for (int e = tid; e < p * p; e += nt) {
          const int r = e / p, c = e - r * p;
          z64 acc(0.0, 0.0);
          for (int q = 0; q < p; ++q) cfma(acc, M[r * p + q], W[q * p + c]);
          T[e] = acc;
        }
        __syncthreads();
        z64* t = W; W = T; T = t;
      }
    }
    // eigen-decomposition (vectors for the nested loop); Z goes to T
    const int rc = geig(W, T, p, p, a.nested != 0, lam, vec, sh);
    if (rc != 0 && tid == 0) report(a.status, ST_ENOCONV, k0, 0.0);
    for (int c = tid; c < p; c += nt) th[c] = phase_of(lam[c]);
    __syncthreads();
    rank_sort(th, p, ord);
    for (int c = tid; c < p; c += nt) a.phases[(long long)i * p + c] = th[ord[c]];
    if (!a.nested) {
      __syncthreads();
      continue;
    }
    // sector: phases measured from `cut`, ascending (stable in eigenvalue index)
    const double two_pi = 6.283185307179586;
    for (int c = tid; c < p; c += nt) {
      double x = fmod(th[c] - a.cut, two_pi);
      if (x < 0.0) x += two_pi;
      if (x >= two_pi) x = 0.0;
      key[c] = x;
    }
    __syncthreads();
    rank_sort(key, p, ord);
    // Wannier gap: circular distance between sector and rest
    double wg = INFINITY;
    for (int e = tid; e < p * p; e += nt) {
      const int s = e / p, r = e - s * p;
      const bool in_s = s >= a.first && s < a.first + m;
      const bool in_r = !(r >= a.first && r < a.first + m);
      if (in_s && in_r) {
        double d = fabs(th[ord[s]] - th[ord[r]]);
        d = fmod(d, two_pi);
        d = fmin(d, two_pi - d);
        wg = fmin(wg, d);
      }
    }
    wg = block_min(wg, red);
    if (tid == 0) {
      if (a.min_wannier_gap) a.min_wannier_gap[i] = wg;
      if (!(wg > a.wannier_gap_tol)) report(a.status, ST_EWANGAP, k0, wg);
    }
    // nu_0 = Z[:, sector] -> X (W no longer needed), transport with Y as scratch
    z64* nu = (W == X) ? X : Y;
    z64* Zm = (W == X) ? Y : X;
    for (int e = tid; e < p * m; e += nt) {
      const int r = e / m, c = e - r * m;
      nu[e] = Zm[r * p + ord[a.first + c]];
    }
    __syncthreads();
    z64* nx = Zm;  // scratch for nu_{j+1}
    for (int j = 0; j < N; ++j) {
      // transport only; the sector basis of every base point is orthonormalised and
      // lifted to Wannier states by k_wannier, in parallel over all k-points (any
      // basis of the transported span is valid: the nested phases are gauge
      // invariant).  Columns are rescaled to unit norm so that the product cannot
      // drift in scale along the loop.
      for (int c = tid; c < m; c += nt) {
        double s2 = 0.0;
        for (int r = 0; r < p; ++r) s2 += abs2(nu[r * m + c]);
        const double inv = 1.0 / sqrt(s2);
        for (int r = 0; r < p; ++r) nu[r * m + c] = inv * nu[r * m + c];
      }
      __syncthreads();
      z64* dst = a.nu_buf + ((long long)j * a.N_t + i) * (long long)p * m;
      for (int e = tid; e < p * m; e += nt) dst[e] = nu[e];
      const z64* M = a.M + (k0 + j) * (long long)p * p;
      for (int e = tid; e < p * m; e += nt) {
        const int r = e / m, c = e - r * m;
        z64 acc(0.0, 0.0);
        for (int q = 0; q < p; ++q) cfma(acc, M[r * p + q], nu[q * m + c]);
        nx[e] = acc;
      }
      __syncthreads();
      z64* t = nu; nu = nx; nx = t;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Wannier states of every (base point j, transverse index i): the transported sector
// basis nu (p x m) orthonormalised by two Cholesky-QR passes (Gram matrix by the
// whole CTA, Cholesky factor by one warp, triangular solves one row per thread),
// then w = U(k_ij) nu.  One CTA per pair, all pairs independent.
// ---------------------------------------------------------------------------
// nu <- nu L^{-dagger} with G = nu^dagger nu = L L^dagger (L lower triangular, kept in
// the lower triangle of G); *ok = 0 on breakdown.
__device__ void cholqr_par(z64* nu, z64* G, int p, int m, int* ok) {
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int e = tid; e < m * m; e += nt) {
    const int x = e / m, y = e - x * m;
    z64 acc(0.0, 0.0);
    for (int r = 0; r < p; ++r) cfma_conj(acc, nu[r * m + x], nu[r * m + y]);
    G[e] = acc;  // G[x][y] = nu_x^dag nu_y
  }
  __syncthreads();
  __shared__ int chol_ok;
  chol_lower_warp(G, m, &chol_ok);  // warp-parallel factor, ends with a barrier
  if (!chol_ok && tid == 0) *ok = 0;
  // row q of nu: x L^dagger = q, i.e. L y = q^dagger (forward substitution), x = y^dagger
  for (int r = tid; r < p; r += nt) {
    z64* q = nu + r * m;
    for (int j = 0; j < m; ++j) {
      z64 y = conj(q[j]);
      for (int k = 0; k < j; ++k) y = y - G[j * m + k] * conj(q[k]);
      q[j] = conj((1.0 / G[j * m + j].re) * y);
    }
  }
  __syncthreads();
}

__global__ void k_wannier(LoopArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int n = a.n, p = a.p, m = a.m, N = a.N, tid = threadIdx.x, nt = blockDim.x;
  z64* nu = reinterpret_cast<z64*>(smem);  // p x m
  z64* G = nu + p * m;                     // m x m
  __shared__ int ok;
  const long long K = (long long)N * a.N_t;
  for (long long b = blockIdx.x; b < K; b += gridDim.x) {
    const int j = int(b / a.N_t), i = int(b - (long long)j * a.N_t);
    const z64* src = a.nu_buf + b * (long long)p * m;
    for (int e = tid; e < p * m; e += nt) nu[e] = src[e];
    if (tid == 0) ok = 1;
    __syncthreads();
    cholqr_par(nu, G, p, m, &ok);
    cholqr_par(nu, G, p, m, &ok);
    if (!ok && tid == 0) report(a.status, ST_ENOCONV, (long long)i * N + j, 0.0);
    const z64* Uk = a.U + ((long long)i * N + j) * (long long)n * p;
    z64* w = a.w + b * (long long)n * m;
    for (int e = tid; e < n * m; e += nt) {
      const int r = e / m, c = e - r * m;
      z64 acc(0.0, 0.0);
      for (int q = 0; q < p; ++q) cfma(acc, Uk[r * p + q], nu[q * m + c]);
      w[e] = acc;
    }
    __syncthreads();
  }
}

cudaError_t launch_wannier(const LoopArgs& a, cudaStream_t s) {
  const long long K = (long long)a.N * a.N_t;
  if (K <= 0 || !a.nu_buf) return cudaSuccess;
  const size_t sm = (size_t(a.p) * a.m + size_t(a.m) * a.m) * sizeof(z64);
  static size_t cached = 0;
  cudaError_t e = set_smem_once(k_wannier, sm, cached);
  if (e != cudaSuccess) return e;
  const long long cap = 152LL * 8;
  k_wannier<<<int(K < cap ? K : cap), 256, sm, s>>>(a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Nested loop per base point
// ---------------------------------------------------------------------------
__global__ void k_nested(LoopArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int n = a.n, m = a.m, Ns = n_planes(a), Nt = a.N_t / Ns, tid = threadIdx.x, nt = blockDim.x;
  const LoopSmem L = loop_layout(m, 1);
  z64* W = reinterpret_cast<z64*>(smem + L.X);
  z64* T = reinterpret_cast<z64*>(smem + L.Y);
  z64* lam = reinterpret_cast<z64*>(smem + L.lam);
  z64* vec = reinterpret_cast<z64*>(smem + L.vec);
  double* th = reinterpret_cast<double*>(smem + L.th);
  int* ord = reinterpret_cast<int*>(smem + L.ord);
  GeigShared* sh = reinterpret_cast<GeigShared*>(smem + L.sh);
  z64* Mt = reinterpret_cast<z64*>(smem + L.total);  // m x m after the layout
  for (int b = blockIdx.x; b < a.N * Ns; b += gridDim.x) {
    const int sp = b / a.N, j = b - sp * a.N;
    for (int e = tid; e < m * m; e += nt) {
      const int r = e / m, c = e - r * m;
      W[e] = z64(double(r == c), 0.0);
    }
    __syncthreads();
    const z64* wj = a.w + ((long long)j * a.N_t + (long long)sp * Nt) * n * m;
    for (int i = 0; i < Nt; ++i) {
      const z64* wa = wj + (long long)i * n * m;
      const z64* wb = wj + (long long)(i + 1 == Nt ? 0 : i + 1) * n * m;
      for (int e = tid; e < m * m; e += nt) {
        const int r = e / m, c = e - r * m;
        z64 acc(0.0, 0.0);
        for (int q = 0; q < n; ++q) cfma_conj(acc, wb[q * m + r], wa[q * m + c]);
        Mt[e] = acc;
      }
      __syncthreads();
      for (int e = tid; e < m * m; e += nt) {
        const int r = e / m, c = e - r * m;
        z64 acc(0.0, 0.0);
        for (int q = 0; q < m; ++q) cfma(acc, Mt[r * m + q], W[q * m + c]);
        T[e] = acc;
      }
      __syncthreads();
      z64* t = W; W = T; T = t;
    }
    const int rc = geig(W, T, m, m, false, lam, vec, sh);
    if (rc != 0 && tid == 0) report(a.status, ST_ENOCONV, b, 0.0);
    for (int c = tid; c < m; c += nt) th[c] = phase_of(lam[c]);
    __syncthreads();
    rank_sort(th, m, ord);
    for (int c = tid; c < m; c += nt) a.nested_out[(long long)b * m + c] = th[ord[c]];
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Small-p loop kernels: all overlaps of a loop in shared memory at once and a
// log-depth prefix product instead of a chain of dependent global loads.
// ---------------------------------------------------------------------------
constexpr int SCAN_P_MAX = 4;
constexpr size_t SCAN_SMEM_MAX = 96 * 1024;

// Element arithmetic of the scan kernels: complex FP64 (z64), or complex
// double-float (cdf) on the FP32 pipe for the mixed-precision few-band path, whose
// states arrive as double-float.  Eigenvalues of the final small matrices are taken
// in FP64 either way.
template <typename E>
struct Arith;
template <>
struct Arith<z64> {
  using R = double;
  __device__ static z64 zero() { return z64(0.0, 0.0); }
  __device__ static z64 one() { return z64(1.0, 0.0); }
  __device__ static z64 shfl_xor(z64 v, int o) {
    return z64(__shfl_xor_sync(0xffffffffu, v.re, o), __shfl_xor_sync(0xffffffffu, v.im, o));
  }
  __device__ static z64 from(z64 v) { return v; }
  __device__ static z64 to64(z64 v) { return v; }
  __device__ static double rsqrt(double x) { return 1.0 / sqrt(x); }
};
template <>
struct Arith<cdf> {
  using R = df;
  __device__ static cdf zero() { return cdf_zero(); }
  __device__ static cdf one() { return cdf(df(1.f), df(0.f)); }
  __device__ static cdf shfl_xor(cdf v, int o) {
    return cdf(shfl_xor_df(v.re, o), shfl_xor_df(v.im, o));
  }
  __device__ static cdf from(z64 v) { return cdf_from(v); }
  __device__ static z64 to64(cdf v) { return cdf_to_z64(v); }
  __device__ static df rsqrt(df x) { return df_rsqrt(x); }
};

// In-place inclusive prefix product over L matrices of size q x q, later index on the
// left: on return S[j] = A_j A_{j-1} ... A_0.  T is scratch of the same size.
// Returns the buffer holding the result (S or T).
template <typename E>
__device__ E* prefix_products(E* S, E* T, int L, int q) {
  const int qq = q * q;
  for (int d = 1; d < L; d <<= 1) {
    for (int e = threadIdx.x; e < L * qq; e += blockDim.x) {
      const int j = e / qq, rc = e - j * qq, r = rc / q, c = rc - r * q;
      if (j < d) {
        T[e] = S[e];
      } else {
        const E* A = S + j * qq;
        const E* B = S + (j - d) * qq;
        E acc = Arith<E>::zero();
        for (int k = 0; k < q; ++k) cfma(acc, A[r * q + k], B[k * q + c]);
        T[e] = acc;
      }
    }
    __syncthreads();
    E* t = S; S = T; T = t;
  }
  return S;
}

struct ScanSmem {
  size_t S, T, Nu, X, Y, lam, vec, th, key, ord, sh, red, total;
};

__host__ __device__ inline ScanSmem scan_layout(int L, int q, int n_nu) {
  auto al = [](size_t x) { return (x + 15) & ~size_t(15); };
  ScanSmem Z;
  size_t o = 0;
  Z.S = o; o = al(o + size_t(L) * q * q * sizeof(z64));
  Z.T = o; o = al(o + size_t(L) * q * q * sizeof(z64));
  Z.Nu = o; o = al(o + size_t(n_nu) * sizeof(z64));
  Z.X = o; o = al(o + size_t(q) * q * sizeof(z64));
  Z.Y = o; o = al(o + size_t(q) * q * sizeof(z64));
  Z.lam = o; o = al(o + size_t(q) * sizeof(z64));
  Z.vec = o; o = al(o + size_t(q) * sizeof(z64));
  Z.th = o; o = al(o + size_t(q) * sizeof(double));
  Z.key = o; o = al(o + size_t(q) * sizeof(double));
  Z.ord = o; o = al(o + size_t(q) * sizeof(int));
  Z.sh = o; o = al(o + sizeof(GeigShared));
  Z.red = o; o = al(o + 64 * sizeof(double));
  Z.total = o;
  return Z;
}

// Orders the eigenphases th[0..p) by their distance from `cut` (mod 2pi, stable),
// writes the Wannier gap of the sector [first, first+m) for loop i and reports a
// closed gap.  ord receives the ordering.  Every thread must call it.  The host
// passes cut reduced to [0, 2pi), so theta - cut lies in (-3pi, pi] and wraps by
// adding 2pi at most twice; two phases in (-pi, pi] differ by at most 2pi.  One warp
// takes the gap.
__device__ void nested_sector(const LoopArgs& a, const double* th, int p, int m, double* key,
                              int* ord, int i, long long k0) {
  const double two_pi = 6.283185307179586;
  for (int c = threadIdx.x; c < p; c += blockDim.x) {
    double x = th[c] - a.cut;
    if (x < 0.0) x += two_pi;
    if (x < 0.0) x += two_pi;
    if (x >= two_pi) x = 0.0;
    key[c] = x;
  }
  __syncthreads();
  rank_sort(key, p, ord);
  if (threadIdx.x < 32) {
    double wg = INFINITY;
    for (int e = threadIdx.x; e < p * p; e += 32) {
      const int s = e / p, r = e - s * p;
      const bool in_s = s >= a.first && s < a.first + m;
      const bool in_r = !(r >= a.first && r < a.first + m);
      if (in_s && in_r) {
        const double d = fabs(th[ord[s]] - th[ord[r]]);
        wg = fmin(wg, fmin(d, two_pi - d));
      }
    }
    for (int o = 16; o > 0; o >>= 1) wg = fmin(wg, __shfl_xor_sync(0xffffffffu, wg, o));
    if (threadIdx.x == 0) {
      if (a.min_wannier_gap) a.min_wannier_gap[i] = wg;
      if (!(wg > a.wannier_gap_tol)) report(a.status, ST_EWANGAP, k0, wg);
    }
  }
}

// One loop (transverse index i) of the scan kernels: overlaps from the loop's states
// Ul (N x n x p, global or shared memory), prefix products, eigenphases and, for the
// nested loop, the transported sector bases and Wannier states.  gl / pgl: the
// loop's N direct / PSO gaps (may be NULL).  Every thread of the CTA calls it.
template <typename E>
__device__ void scan_one_loop(const LoopArgs& a, int i, const E* Ul, const double* gl,
                              const double* pgl, unsigned char* smem) {
  using A = Arith<E>;
  const int n = a.n, p = a.p, N = a.N, tid = threadIdx.x, nt = blockDim.x;
  const int m = a.nested ? a.m : 1;
  const ScanSmem Z = scan_layout(N, p, a.nested ? N * p * m : 1);
  E* S = reinterpret_cast<E*>(smem + Z.S);
  E* T = reinterpret_cast<E*>(smem + Z.T);
  E* Nu = reinterpret_cast<E*>(smem + Z.Nu);
  E* wg = reinterpret_cast<E*>(a.w);
  z64* X = reinterpret_cast<z64*>(smem + Z.X);
  z64* Y = reinterpret_cast<z64*>(smem + Z.Y);
  z64* lam = reinterpret_cast<z64*>(smem + Z.lam);
  z64* vec = reinterpret_cast<z64*>(smem + Z.vec);
  double* th = reinterpret_cast<double*>(smem + Z.th);
  double* key = reinterpret_cast<double*>(smem + Z.key);
  int* ord = reinterpret_cast<int*>(smem + Z.ord);
  GeigShared* sh = reinterpret_cast<GeigShared*>(smem + Z.sh);
  double* red = reinterpret_cast<double*>(smem + Z.red);
  const int pp = p * p;
  {
    const long long k0 = (long long)i * N;
    if (a.min_gap || a.min_pso_gap) {  // one warp
      if (tid < 32) {
        double g = INFINITY, gp = INFINITY;
        for (int j = tid; j < N; j += 32) {
          if (gl) g = fmin(g, gl[j]);
          if (pgl) gp = fmin(gp, pgl[j]);
        }
        for (int o = 16; o > 0; o >>= 1) {
          g = fmin(g, __shfl_xor_sync(0xffffffffu, g, o));
          gp = fmin(gp, __shfl_xor_sync(0xffffffffu, gp, o));
        }
        if (tid == 0) {
          if (a.min_gap) a.min_gap[i] = g;
          if (a.min_pso_gap) a.min_pso_gap[i] = gp;
        }
      }
    }
    if (a.unitarise) {
      const z64* Mg = a.M + k0 * pp;
      for (int e = tid; e < N * pp; e += nt) S[e] = A::from(Mg[e]);
    } else {  // the overlaps of this loop, M_j = U(k_{j+1})^dagger U(k_j), closing on j = 0
      for (int e = tid; e < N * pp; e += nt) {
        const int jj = e / pp, rc = e - jj * pp, r = rc / p, c = rc - r * p;
        const E* Uh = Ul + jj * (long long)n * p;
        const E* Un = Ul + (jj + 1 == N ? 0 : jj + 1) * (long long)n * p;
        E acc = A::zero();
        for (int q = 0; q < n; ++q) cfma_conj(acc, Un[q * p + r], Uh[q * p + c]);
        S[e] = acc;
      }
    }
    __syncthreads();
    // P[j] = M_j ... M_0; the loop matrix is P[N-1]
    E* Pf = prefix_products(S, T, N, p);
    // eigenvalues (and for the nested loop right eigenvectors) of W = P[N-1]; at
    // p = 2 in closed form in the element arithmetic (the general solver's serial QR
    // sweeps dominate there), else by the FP64 general solver.  Ye: eigenvectors
    // as E for the transport.
    constexpr bool kDf = std::is_same<E, cdf>::value;
    E* Ye = reinterpret_cast<E*>(smem + Z.Y);
    if (p == 2) {
      if constexpr (kDf) {
        // eigenvalues on one thread; then the two eigenvectors (warp 0) and the two
        // phases (warp 1) in parallel
        cdf* lamd = reinterpret_cast<cdf*>(smem + Z.vec);
        const E* Wl = Pf + (N - 1) * pp;
        if (tid == 0) eig2_values_df(Wl, lamd);
        __syncthreads();
        if (tid < 2 && a.nested) eig2_vector_df(Wl, lamd[tid], tid, Ye);
        if (tid >= 32 && tid < 34) {
          lam[tid - 32] = cdf_to_z64(lamd[tid - 32]);
          th[tid - 32] = phase_of(lam[tid - 32]);
        }
      } else {
        if (tid == 0) eig2_closed(Pf + (N - 1) * pp, 2, lam, Y, a.nested != 0);
      }
      __syncthreads();
    } else {
      for (int e = tid; e < pp; e += nt) X[e] = A::to64(Pf[(N - 1) * pp + e]);
      __syncthreads();
      const int rc = geig(X, Y, p, p, a.nested != 0, lam, vec, sh);
      if (rc != 0 && tid == 0) report(a.status, ST_ENOCONV, k0, 0.0);
      if constexpr (kDf) {  // convert in place (same element size)
        __syncthreads();
        for (int e = tid; e < pp; e += nt) {
          const z64 v = Y[e];
          Ye[e] = A::from(v);
        }
      }
    }
    if (!(kDf && p == 2))
      for (int c = tid; c < p; c += nt) th[c] = phase_of(lam[c]);
    __syncthreads();
    rank_sort(th, p, ord);
    for (int c = tid; c < p; c += nt) a.phases[(long long)i * p + c] = th[ord[c]];
    __syncthreads();
    if (!a.nested) return;
    nested_sector(a, th, p, m, key, ord, i, k0);
    // nu_j = P[j-1] nu_0 (nu_0 = Y[:, sector]), one thread per base point j:
    // normalise the columns, then modified Gram-Schmidt (m <= SCAN_P_MAX)
    for (int j = tid; j < N; j += nt) {
      E* nu = Nu + (size_t)j * p * m;
      for (int r = 0; r < p; ++r)
        for (int c = 0; c < m; ++c) {
          const int col = ord[a.first + c];
          E acc = A::zero();
          if (j == 0) {
            acc = Ye[r * p + col];
          } else {
            const E* P = Pf + (size_t)(j - 1) * pp;
            for (int q = 0; q < p; ++q) cfma(acc, P[r * p + q], Ye[q * p + col]);
          }
          nu[r * m + c] = acc;
        }
      for (int c = 0; c < m; ++c) {
        for (int c2 = 0; c2 < c; ++c2) {
          E d = A::zero();
          for (int r = 0; r < p; ++r) cfma_conj(d, nu[r * m + c2], nu[r * m + c]);
          for (int r = 0; r < p; ++r) nu[r * m + c] = nu[r * m + c] - nu[r * m + c2] * d;
        }
        typename A::R s = abs2(nu[c]);
        for (int r = 1; r < p; ++r) s = s + abs2(nu[r * m + c]);
        s = A::rsqrt(s);
        for (int r = 0; r < p; ++r) nu[r * m + c] = s * nu[r * m + c];
      }
    }
    __syncthreads();
    // Wannier states w(j, i) = U(k_j) nu_j
    for (int e = tid; e < N * n * m; e += nt) {
      const int j = e / (n * m), rc2 = e - j * n * m, r = rc2 / m, c = rc2 - r * m;
      const E* Uk = Ul + j * (long long)n * p;
      const E* nu = Nu + (size_t)j * p * m;
      E acc = A::zero();
      for (int q = 0; q < p; ++q) cfma(acc, Uk[r * p + q], nu[q * m + c]);
      wg[((long long)j * a.N_t + i) * n * m + rc2] = acc;
    }
    __syncthreads();
  }
}

template <typename E>
__global__ void k_loops_scan(LoopArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const E* Ug = reinterpret_cast<const E*>(a.U);
  for (int i = blockIdx.x; i < a.N_t; i += gridDim.x) {
    const long long k0 = (long long)i * a.N;
    scan_one_loop<E>(a, i, Ug + k0 * a.n * a.p, a.gap ? a.gap + k0 : nullptr,
                     a.pso_gap ? a.pso_gap + k0 : nullptr, smem);
    __syncthreads();
  }
}

// Nested loop of one Wannier band at base point j: the loop matrix is the product
// of the scalar overlaps w(i+1)^dagger w(i) (any order), taken by the CTA's first
// warp straight from global memory; the other threads return at once.
template <typename E>
__device__ void nested_base_m1(const LoopArgs& a, int b) {
  using A = Arith<E>;
  const int n = a.n, Nt = a.N_t / n_planes(a), tid = threadIdx.x;
  if (tid >= 32) return;
  const int sp = b / a.N, j = b - sp * a.N;
  const E* wj = reinterpret_cast<const E*>(a.w) + ((long long)j * a.N_t + (long long)sp * Nt) * n;
  E prod = A::one();
  for (int i = tid; i < Nt; i += 32) {
    const E* wa = wj + (size_t)i * n;
    const E* wb = wj + (size_t)(i + 1 == Nt ? 0 : i + 1) * n;
    E acc = A::zero();
    for (int q = 0; q < n; ++q) cfma_conj(acc, wb[q], wa[q]);
    prod = prod * acc;
  }
  for (int o = 16; o > 0; o >>= 1) prod = prod * A::shfl_xor(prod, o);
  if (tid == 0) a.nested_out[b] = phase_E(prod);
}

// ---------------------------------------------------------------------------
// Mixed precision, four bands, two occupied, N <= 64: one CTA per loop solves the
// loop's N k-points (four lanes each, quad_df_occupied: double-float H(k), FP32
// Jacobi, double-float Newton refinement) into shared memory and runs the scan loop
// on them, so that the states never leave the SM.  The Bloch phases of the loop
// factor as exp(i 2pi (origin.R + (i trans.R mod N_t) / N_t)) exp(i 2pi (j loop.R
// mod N) / N): one table of N entries and one factor per translation, per CTA.
// ---------------------------------------------------------------------------
constexpr int FUSED_THREADS = 256;

struct FusedSmem {
  size_t U, g, cache, tab, rowf, lR, rowp, ent, col, hr, ht, total;
};

// The model plan (row pointers, entries, grouped hoppings) is staged in shared memory:
// each k-point walks it once, and global loads would put an L2 round trip on every
// step of that walk.
__host__ __device__ inline FusedSmem fused_layout(const ScanSmem& Z, int N, int nR, int n_ent,
                                                  int n_hop) {
  auto al = [](size_t x) { return (x + 15) & ~size_t(15); };
  FusedSmem F;
  size_t o = Z.total;
  F.U = o; o = al(o + size_t(N) * 4 * 2 * sizeof(cdf));
  F.g = o; o = al(o + size_t(N) * sizeof(double));
  F.cache = o; o = al(o + size_t(nR) * (FUSED_THREADS / 4) * sizeof(cdf));
  F.tab = o; o = al(o + size_t(N) * sizeof(cdf));
  F.rowf = o; o = al(o + size_t(nR) * sizeof(cdf));
  F.lR = o; o = al(o + size_t(nR) * sizeof(int));
  F.rowp = o; o = al(o + 5 * sizeof(int));
  F.ent = o; o = al(o + size_t(n_ent + 1) * sizeof(int));
  F.col = o; o = al(o + size_t(n_ent) * sizeof(int));
  F.hr = o; o = al(o + size_t(n_hop) * sizeof(int));
  F.ht = o; o = al(o + size_t(n_hop) * 4 * sizeof(float));
  F.total = o;
  return F;
}

// The loop of the fused kernel at p = 2 (and, nested, one Wannier band): the same
// steps as scan_one_loop with the sizes fixed and the work laid out on the states'
// four-lane groups (group j = tid / 4 holds k-point j, lane l its row l; Q0, Q1 are
// row l of U(k_j) in registers, Us the same states in shared memory).  Lane l of
// group j owns entry (l / 2, l % 2) of the 2 x 2 matrices: the overlap M_j, then the
// prefix product P_j = M_j ... M_0, formed by an inclusive scan over the eight groups
// of each warp (shuffles) and one over the warp totals (one warp), two CTA barriers
// in all.  Groups past N repeat the last k-point and write nothing; only the totals
// of warps followed by k-points are kept (Tw: 8 (ceil(N / 8) - 1) < 4 N entries).
__device__ void pair_loop_df(const LoopArgs& a, int i, const cdf* Us, const double* gs, cdf Q0,
                             cdf Q1, unsigned char* smem) {
  const int N = a.N, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int l = tid & 3, gw = lane >> 2, g4 = lane & ~3, r = l >> 1, c = l & 1;
  const int j = tid >> 2;
  const bool active = j < N;
  const int jj = active ? j : N - 1;
  const int nW = (N + 7) >> 3, eoff = 4 * (nW - 1);  // warps holding k-points
  const ScanSmem Z = scan_layout(N, 2, a.nested ? N * 2 * a.m : 1);
  cdf* Ps = reinterpret_cast<cdf*>(smem + Z.S);  // P_j entry e at Ps[4 j + e]
  cdf* Tw = reinterpret_cast<cdf*>(smem + Z.T);  // warp totals, then exclusive products at eoff
  cdf* Ye = reinterpret_cast<cdf*>(smem + Z.Y);
  cdf* lamd = reinterpret_cast<cdf*>(smem + Z.vec);
  int* ord = reinterpret_cast<int*>(smem + Z.ord);  // ord[0]: the sector's eigenvector
  const long long k0 = (long long)i * N;
  if (a.min_gap && tid < 32) {
    double g = INFINITY;
    for (int q = tid; q < N; q += 32) g = fmin(g, gs[q]);
    for (int o = 16; o > 0; o >>= 1) g = fmin(g, __shfl_xor_sync(0xffffffffu, g, o));
    if (tid == 0) a.min_gap[i] = g;
  }
  if (a.min_pso_gap && tid == 0) a.min_pso_gap[i] = INFINITY;
  // M_j[r][c] = sum_q conj(U(k_{j+1})[q][r]) U(k_j)[q][c], closing on j = 0
  const int jn = jj + 1 == N ? 0 : jj + 1;
  cdf x = cdf_zero();
#pragma unroll
  for (int q = 0; q < 4; ++q) cfma_conj(x, Us[(jn * 4 + q) * 2 + r], Us[(jj * 4 + q) * 2 + c]);
  // x <- x y over the groups of the warp: y from the group d earlier
  auto step = [&](cdf& v, int src4, bool take) {
    const cdf a0 = shfl_cdf(v, g4 + 2 * r), a1 = shfl_cdf(v, g4 + 2 * r + 1);
    const cdf b0 = shfl_cdf(v, src4 + c), b1 = shfl_cdf(v, src4 + 2 + c);
    if (take) {
      cdf y = cdf_zero();
      cfma(y, a0, b0);
      cfma(y, a1, b1);
      v = y;
    }
  };
#pragma unroll 1
  for (int d = 1; d < 8; d <<= 1) step(x, (g4 - 4 * d) & 31, gw >= d);
  if (gw == 7 && warp < nW - 1) Tw[warp * 4 + l] = x;
  __syncthreads();
  if (warp == 0 && nW > 1) {  // lane = 4 v + e holds entry e of warp v's total
    cdf t = gw < nW - 1 ? Tw[lane] : cdf_zero();
#pragma unroll 1
    for (int d = 1; d < 8; d <<= 1) step(t, (g4 - 4 * d) & 31, gw >= d);
    if (gw < nW - 1) Tw[eoff + 4 * gw + l] = t;  // the product before warp gw + 1
  }
  __syncthreads();
  if (warp > 0 && warp < nW) {  // P_j = (M_j ... M_{8 warp}) (M_{8 warp - 1} ... M_0)
    const cdf a0 = shfl_cdf(x, g4 + 2 * r), a1 = shfl_cdf(x, g4 + 2 * r + 1);
    const cdf* E = Tw + eoff + 4 * (warp - 1);
    cdf y = cdf_zero();
    cfma(y, a0, E[c]);
    cfma(y, a1, E[2 + c]);
    x = y;
  }
  if (active) Ps[4 * j + l] = x;
  __syncthreads();
  // eigenvalues of W = P_{N-1} on one thread; the two eigenvectors (warp 0) and the
  // two phases (warp 1) in parallel
  const cdf* Wl = Ps + 4 * (N - 1);
  if (tid == 0) eig2_values_df(Wl, lamd);
  __syncthreads();
  if (tid < 2 && a.nested) eig2_vector_df(Wl, lamd[tid], tid, Ye);
  if (tid >= 32 && tid < 64) {  // warp 1: the two phases, their order and the sector
    double t = 0.0;
    if (tid < 34) t = df_phase(lamd[tid - 32]);
    const double t1 = __shfl_sync(0xffffffffu, t, 1);
    if (tid == 32) {
      const double t0 = t;
      // ascending (stable, NaN last), as rank_sort orders p = 2 phases
      const bool sw = rank_key(t1) < rank_key(t0);
      a.phases[(long long)i * 2] = sw ? t1 : t0;
      a.phases[(long long)i * 2 + 1] = sw ? t0 : t1;
      if (a.nested) {
        // sector: position `first` in the order of (theta - cut) mod 2pi (as
        // nested_sector); its Wannier gap is the distance between the two phases
        const double two_pi = 6.283185307179586;
        double key0 = t0 - a.cut, key1 = t1 - a.cut;
        if (key0 < 0.0) key0 += two_pi;
        if (key0 < 0.0) key0 += two_pi;
        if (key0 >= two_pi) key0 = 0.0;
        if (key1 < 0.0) key1 += two_pi;
        if (key1 < 0.0) key1 += two_pi;
        if (key1 >= two_pi) key1 = 0.0;
        const int lo = rank_key(key1) < rank_key(key0) ? 1 : 0;
        ord[0] = a.first == 0 ? lo : 1 - lo;
        const double dd = fabs(t0 - t1), wgap = fmin(dd, two_pi - dd);
        if (a.min_wannier_gap) a.min_wannier_gap[i] = wgap;
        if (!(wgap > a.wannier_gap_tol)) report(a.status, ST_EWANGAP, k0, wgap);
      }
    }
  }
  __syncthreads();
  if (!a.nested) return;
  // nu_j = P_{j-1} nu_0 (nu_0: the sector's column of Ye), normalised; lanes l and
  // l + 2 of a group both form entry l % 2
  const int col = ord[0];
  cdf nu = Ye[c * 2 + col];
  if (jj > 0) {
    nu = cdf_zero();
    cfma(nu, Ps[4 * (jj - 1) + 2 * c], Ye[col]);
    cfma(nu, Ps[4 * (jj - 1) + 2 * c + 1], Ye[2 + col]);
  }
  const cdf nu_o = shfl_cdf(nu, lane ^ 1);
  const df s = c == 0 ? abs2(nu) + abs2(nu_o) : abs2(nu_o) + abs2(nu);
  const df inv = df_rsqrt(s);
  nu = inv * nu;
  // Wannier state w(j, i) = U(k_j) nu_j, row l on lane l
  const cdf n0 = shfl_cdf(nu, g4), n1 = shfl_cdf(nu, g4 + 1);
  cdf wv = cdf_zero();
  cfma(wv, Q0, n0);
  cfma(wv, Q1, n1);
  if (active) reinterpret_cast<cdf*>(a.w)[((long long)j * a.N_t + i) * 4 + l] = wv;
}

// The plan arrays as the kernel reads them: in global memory, or (inl != NULL) in the
// kernel's parameter copy of the plan, at the same offsets from dbase.
template <typename T>
__device__ __forceinline__ const T* plan_ptr(const T* p, const unsigned char* inl, const char* dbase) {
  return inl ? reinterpret_cast<const T*>(inl + (reinterpret_cast<const char*>(p) - dbase)) : p;
}

// Nested loop of one Wannier band at base point b for the fused kernel (n = 4,
// complex double-float states), by the whole CTA: thread (i, q) = (tid / 4, tid % 4)
// forms conj(w(i+1)[q]) w(i)[q] (every load of the base point in flight at once), the
// row's four lanes sum them, and the rows' overlaps multiply by shuffles in each warp
// and across the warps through shared memory (red: 8 cdf).
__device__ __forceinline__ void nested_base_m1_cta(const LoopArgs& a, int b, cdf* red) {
  const int Nt = a.N_t / n_planes(a), tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int sp = b / a.N, j = b - sp * a.N;
  const cdf* wj = reinterpret_cast<const cdf*>(a.w) + ((long long)j * a.N_t + (long long)sp * Nt) * 4;
  const cdf one(df(1.f), df(0.f));
  cdf prod = one;
  for (int i0 = 0; i0 < Nt; i0 += FUSED_THREADS / 4) {
    const int i = i0 + (tid >> 2), q = tid & 3;
    cdf z = cdf_zero();
    if (i < Nt) cfma_conj(z, wj[(size_t)(i + 1 == Nt ? 0 : i + 1) * 4 + q], wj[(size_t)i * 4 + q]);
    z = z + Arith<cdf>::shfl_xor(z, 1);
    z = z + Arith<cdf>::shfl_xor(z, 2);
    if (!(i < Nt)) z = one;
#pragma unroll 1
    for (int o = 4; o < 32; o <<= 1) z = z * Arith<cdf>::shfl_xor(z, o);
    if (lane == 0) red[warp] = z;
    __syncthreads();
    if (tid == 0)
#pragma unroll 1
      for (int w = 0; w < FUSED_THREADS / 32; ++w) prod = prod * red[w];
    __syncthreads();
  }
  if (tid == 0) a.nested_out[b] = df_phase(prod);
}

template <bool kNested1>
__device__ __forceinline__ void loops_fused_body(const StatesArgs& sa, const LoopArgs& a,
                                                 const unsigned char* inl, const char* dbase) {
  extern __shared__ __align__(16) unsigned char smem[];
  const DevModel& md = sa.model;
  const int N = a.N, Nt = a.N_t, nR = md.n_R, tid = threadIdx.x, nt = blockDim.x;
  constexpr int KPB = FUSED_THREADS / 4;
  const ScanSmem Z = scan_layout(N, 2, a.nested ? N * 2 * a.m : 1);
  const FusedSmem F = fused_layout(Z, N, nR, md.n_ent, md.n_hop);
  cdf* Us = reinterpret_cast<cdf*>(smem + F.U);
  int* s_rowp = reinterpret_cast<int*>(smem + F.rowp);
  int* s_ent = reinterpret_cast<int*>(smem + F.ent);
  int* s_col = reinterpret_cast<int*>(smem + F.col);
  int* s_hr = reinterpret_cast<int*>(smem + F.hr);
  float4* s_ht = reinterpret_cast<float4*>(smem + F.ht);
  const int* g_rowp = plan_ptr(sa.row_ptr, inl, dbase);
  const int* g_ent = plan_ptr(md.ent_start, inl, dbase);
  const int* g_col = plan_ptr(md.ent_col, inl, dbase);
  const int* g_hr = plan_ptr(md.hop_r, inl, dbase);
  const float* g_tdf = plan_ptr(md.hop_tdf, inl, dbase);
  const int* g_Rv = plan_ptr(md.Rv, inl, dbase);
  for (int e = tid; e < 5; e += nt) s_rowp[e] = g_rowp[e];
  for (int e = tid; e <= md.n_ent; e += nt) s_ent[e] = g_ent[e];
  for (int e = tid; e < md.n_ent; e += nt) s_col[e] = g_col[e];
  for (int h = tid; h < md.n_hop; h += nt) {
    s_hr[h] = g_hr[h];
    s_ht[h] = make_float4(g_tdf[4 * h], g_tdf[4 * h + 1], g_tdf[4 * h + 2], g_tdf[4 * h + 3]);
  }
  double* gs = reinterpret_cast<double*>(smem + F.g);
  cdf* cache = reinterpret_cast<cdf*>(smem + F.cache);
  cdf* tab = reinterpret_cast<cdf*>(smem + F.tab);
  cdf* rowf = reinterpret_cast<cdf*>(smem + F.rowf);
  int* lR = reinterpret_cast<int*>(smem + F.lR);
  for (int m = tid; m < N; m += nt) tab[m] = df_cispi_ratio(2 * m, N);  // e^{2 pi i m / N}
  const int l = tid & 3, kl = tid >> 2, base = (tid & 31) & ~3;
  const bool active = kl < N;
  const int j = active ? kl : N - 1;  // idle groups recompute the last k-point
  // the translation factors on the last warps, in parallel with the table above
  const int rbase = nt - 32 * ((nR + 31) / 32);
  for (int i = blockIdx.x; i < Nt; i += gridDim.x) {
    for (int r = tid - rbase; r >= 0 && r < nR; r += nt) {
      const int* Rv = g_Rv + 3 * r;
      double x = 0.0;
      int lq = 0, tq = 0, sq = 0;
      for (int dd = 0; dd < 3; ++dd) {
        x += sa.plane.origin[dd] * double(Rv[dd]);
        lq += int(sa.plane.loop_dir[dd]) * Rv[dd];
        tq += int(sa.plane.trans_dir[dd]) * Rv[dd];
        sq += sa.plane.sweep[dd] * Rv[dd];
      }
      x += double(pmod(plane_row_index(sa.plane, i, tq, sq), Nt)) / double(Nt);
      rowf[r] = df_cispi(2.0 * x);
      lR[r] = lq;
    }
    __syncthreads();
    for (int r = l; r < nR; r += 4) cache[r * KPB + kl] = rowf[r] * tab[pmod((long long)j * lR[r], N)];
    __syncwarp();
    // row l of H(k) in double-float
    cdf Hr[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) Hr[c] = cdf_zero();
    for (int e = s_rowp[l]; e < s_rowp[l + 1]; ++e) {
      cdf acc = cdf_zero();
      for (int h = s_ent[e]; h < s_ent[e + 1]; ++h) {
        const float4 t4 = s_ht[h];
        cfma(acc, cdf(df(t4.x, t4.y), df(t4.z, t4.w)), cache[s_hr[h] * KPB + kl]);
      }
      const int col = s_col[e];
#pragma unroll
      for (int c = 0; c < 4; ++c)
        if (c == col) Hr[c] = acc;
    }
    cdf Qf[2];
    double gap;
    const int sweeps = quad_df_occupied(Hr, l, base, sa.max_sweeps, Qf[0], Qf[1], gap);
    if (active) {
      Us[(j * 4 + l) * 2] = Qf[0];
      Us[(j * 4 + l) * 2 + 1] = Qf[1];
      if (l == 0) {
        const long long k = (long long)i * N + j;
        gs[j] = gap;
        if (sweeps < 0) report(sa.status, ST_ENOCONV, k, 0.0);
        if (!(gap > sa.gap_tol)) report(sa.status, ST_EGAP, k, gap);
      }
    }
    __syncthreads();
    if (!a.nested || a.m == 1)
      pair_loop_df(a, i, Us, gs, Qf[0], Qf[1], smem);
    else
      scan_one_loop<cdf>(a, i, Us, gs, nullptr, smem);
    __syncthreads();
  }
  if constexpr (kNested1) {
    // cooperative launch: every loop's Wannier states are written once the grid
    // has passed this barrier; then the nested loops of one Wannier band
    __threadfence();
    cooperative_groups::this_grid().sync();
    // the scan's scratch, free by now: S and T (2 N x 64 bytes, contiguous) hold 8 cdf
    cdf* red8 = reinterpret_cast<cdf*>(smem + Z.S);
    for (int b = blockIdx.x; b < a.N * n_planes(a); b += gridDim.x) nested_base_m1_cta(a, b, red8);
  }
}

template <bool kNested1>
__global__ void __launch_bounds__(FUSED_THREADS) k_loops_fused_df(StatesArgs sa, LoopArgs a) {
  loops_fused_body<kNested1>(sa, a, nullptr, nullptr);
}

template <bool kNested1>
__global__ void __launch_bounds__(FUSED_THREADS)
    k_loops_fused_df_inl(StatesArgs sa, LoopArgs a, const char* dbase, const __grid_constant__ FusedPlan plan) {
  loops_fused_body<kNested1>(sa, a, plan.bytes, dbase);
}

bool loops_fused_eligible(const LoopArgs& a, const DevModel& md) {
  if (!(a.n == 4 && a.p == 2 && a.N >= 1 && 4 * a.N <= FUSED_THREADS && loops_accept_df(a)))
    return false;
  const ScanSmem Z = scan_layout(a.N, 2, a.nested ? a.N * 2 * a.m : 1);
  return fused_layout(Z, a.N, md.n_R, md.n_ent, md.n_hop).total <= 96 * 1024;
}

cudaError_t launch_loops_fused_df(const StatesArgs& sa, const LoopArgs& a, cudaStream_t s,
                                  bool* nested_done, const void* plan_host, size_t plan_bytes,
                                  const void* plan_dev) {
  *nested_done = false;
  if (a.N_t <= 0) return cudaSuccess;
  const bool inl = plan_host && plan_bytes <= sizeof(FusedPlan);
  if (plan_host && !inl) return cudaErrorInvalidValue;
  FusedPlan fp;  // the kernel parameter (copied at launch)
  const char* dbase = static_cast<const char*>(plan_dev);
  if (inl) {
    std::memset(fp.bytes, 0, sizeof(fp.bytes));
    std::memcpy(fp.bytes, plan_host, plan_bytes);
  }
  const ScanSmem Z = scan_layout(a.N, 2, a.nested ? a.N * 2 * a.m : 1);
  const FusedSmem F = fused_layout(Z, a.N, sa.model.n_R, sa.model.n_ent, sa.model.n_hop);
  cudaError_t e;
  if (a.nested && a.m == 1) {
    // one cooperative launch for the loops and the nested loops when the whole grid
    // is resident at once (one CTA per loop)
    static size_t cached_c = 0, cached_ci = 0;
    if ((e = inl ? set_smem_once(k_loops_fused_df_inl<true>, F.total, cached_ci)
                 : set_smem_once(k_loops_fused_df<true>, F.total, cached_c)) != cudaSuccess)
      return e;
    // the device's SM count, cooperative support and the kernel's occupancy at this
    // shared-memory size, queried once per thread, device, variant and size
    struct Occ {
      int dev = -1, inl = -1, sms = 0, coop = 0, per_sm = 0;
      size_t smem = 0;
    };
    thread_local Occ occ;
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if (occ.dev != dev || occ.inl != int(inl) || occ.smem != F.total) {
      Occ q;
      q.dev = dev;
      q.inl = int(inl);
      q.smem = F.total;
      if ((e = cudaDeviceGetAttribute(&q.sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
      if ((e = cudaDeviceGetAttribute(&q.coop, cudaDevAttrCooperativeLaunch, dev)) != cudaSuccess) return e;
      if ((e = inl ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&q.per_sm, k_loops_fused_df_inl<true>,
                                                                    FUSED_THREADS, F.total)
                   : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&q.per_sm, k_loops_fused_df<true>,
                                                                    FUSED_THREADS, F.total)) != cudaSuccess)
        return e;
      occ = q;
    }
    const int sms = occ.sms, coop = occ.coop, per_sm = occ.per_sm;
    if (coop && (long long)per_sm * sms >= a.N_t) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(a.N_t);
      cfg.blockDim = dim3(FUSED_THREADS);
      cfg.dynamicSmemBytes = F.total;
      cfg.stream = s;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeCooperative;
      attr[0].val.cooperative = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      if ((e = inl ? cudaLaunchKernelEx(&cfg, k_loops_fused_df_inl<true>, sa, a, dbase, fp)
                   : cudaLaunchKernelEx(&cfg, k_loops_fused_df<true>, sa, a)) != cudaSuccess)
        return e;
      *nested_done = true;
      return cudaSuccess;
    }
  }
  if (inl) {
    static size_t cached_i = 0;
    if ((e = set_smem_once(k_loops_fused_df_inl<false>, F.total, cached_i)) != cudaSuccess) return e;
    k_loops_fused_df_inl<false><<<a.N_t, FUSED_THREADS, F.total, s>>>(sa, a, dbase, fp);
    return cudaGetLastError();
  }
  static size_t cached = 0;
  if ((e = set_smem_once(k_loops_fused_df<false>, F.total, cached)) != cudaSuccess) return e;
  k_loops_fused_df<false><<<a.N_t, FUSED_THREADS, F.total, s>>>(sa, a);
  return cudaGetLastError();
}

// Self-test of the double-float unit-circle helpers (df_cispi_ratio, df_cispi,
// df_phase) against the FP64 sincospi / atan2 of the CUDA math library; maxima by
// atomicMax on the bit patterns of the non-negative errors.
__device__ __forceinline__ void err_max(double* e, double v) {
  if (!(v <= 1.0)) v = 1.0;  // NaN or a gross error
  atomicMax(reinterpret_cast<unsigned long long*>(e), static_cast<unsigned long long>(__double_as_longlong(v)));
}

__global__ void k_selftest_unit_circle(double* err) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
  for (int e = tid; e < 64 * 64; e += nth) {  // (N, m)
    const int N = e / 64 + 1, m = e % 64;
    if (m >= N) continue;
    const cdf z = df_cispi_ratio(2 * m, N);
    double sn, cs;
    sincospi(2.0 * double(m) / double(N), &sn, &cs);
    err_max(err, fmax(fabs(df_to_double(z.re) - cs), fabs(df_to_double(z.im) - sn)));
  }
  for (int e = tid; e < 8192; e += nth) {
    const double t = -3.0 + 6.0 * double(e) / 8192.0;
    const cdf z = df_cispi(t);
    double sn, cs;
    sincospi(t, &sn, &cs);
    err_max(err + 1, fmax(fabs(df_to_double(z.re) - cs), fabs(df_to_double(z.im) - sn)));
  }
  for (int e = tid; e < 3 * 4096; e += nth) {
    const double rad = e < 4096 ? 0.5 : (e < 8192 ? 1.0 : 2.0);
    const double t = -1.0 + 2.0 * double(e % 4096 + 1) / 4096.0;  // (-1, 1] half-turns
    double sn, cs;
    sincospi(t, &sn, &cs);
    const cdf z(df_from_double(rad * cs), df_from_double(rad * sn));
    const double ref = atan2(df_to_double(z.im), df_to_double(z.re));
    const double d = fabs(df_phase(z) - ref);
    err_max(err + 2, fmin(d, 6.283185307179586 - d));
  }
}

cudaError_t launch_selftest_unit_circle(double* err, cudaStream_t s) {
  k_selftest_unit_circle<<<48, 256, 0, s>>>(err);
  return cudaGetLastError();
}

// Nested loop for small m: one CTA per base point, all Wannier states of the base
// point in shared memory, overlaps in parallel, product by prefix scan.
template <typename E>
__global__ void k_nested_scan(LoopArgs a) {
  using A = Arith<E>;
  extern __shared__ __align__(16) unsigned char smem[];
  const int n = a.n, m = a.m, Nt = a.N_t / n_planes(a), tid = threadIdx.x, nt = blockDim.x;
  const ScanSmem Z = scan_layout(Nt, m, Nt * n * m);
  E* S = reinterpret_cast<E*>(smem + Z.S);
  E* T = reinterpret_cast<E*>(smem + Z.T);
  E* Wn = reinterpret_cast<E*>(smem + Z.Nu);
  z64* X = reinterpret_cast<z64*>(smem + Z.X);
  z64* Y = reinterpret_cast<z64*>(smem + Z.Y);
  z64* lam = reinterpret_cast<z64*>(smem + Z.lam);
  z64* vec = reinterpret_cast<z64*>(smem + Z.vec);
  double* th = reinterpret_cast<double*>(smem + Z.th);
  int* ord = reinterpret_cast<int*>(smem + Z.ord);
  GeigShared* sh = reinterpret_cast<GeigShared*>(smem + Z.sh);
  const int mm2 = m * m, nm = n * m;
  for (int b = blockIdx.x; b < a.N * n_planes(a); b += gridDim.x) {
    const int sp = b / a.N, j = b - sp * a.N;
    const E* wj = reinterpret_cast<const E*>(a.w) + ((long long)j * a.N_t + (long long)sp * Nt) * nm;
    if (m == 1) {
      nested_base_m1<E>(a, b);
      continue;
    }
    for (int e = tid; e < Nt * nm; e += nt) Wn[e] = wj[e];
    __syncthreads();
    // A_i = w(i+1)^dagger w(i), closed on i = 0
    for (int e = tid; e < Nt * mm2; e += nt) {
      const int i = e / mm2, rc = e - i * mm2, r = rc / m, c = rc - r * m;
      const E* wa = Wn + (size_t)i * nm;
      const E* wb = Wn + (size_t)(i + 1 == Nt ? 0 : i + 1) * nm;
      E acc = A::zero();
      for (int q = 0; q < n; ++q) cfma_conj(acc, wb[q * m + r], wa[q * m + c]);
      S[e] = acc;
    }
    __syncthreads();
    E* Pf = prefix_products(S, T, Nt, m);
    for (int e = tid; e < mm2; e += nt) X[e] = A::to64(Pf[(Nt - 1) * mm2 + e]);
    __syncthreads();
    const int rc = geig(X, Y, m, m, false, lam, vec, sh);
    if (rc != 0 && tid == 0) report(a.status, ST_ENOCONV, b, 0.0);
    for (int c = tid; c < m; c += nt) th[c] = phase_of(lam[c]);
    __syncthreads();
    rank_sort(th, m, ord);
    for (int c = tid; c < m; c += nt) a.nested_out[(long long)b * m + c] = th[ord[c]];
    __syncthreads();
  }
}

static bool scan_loops_fit(const LoopArgs& a) {
  if (a.p > SCAN_P_MAX) return false;
  const int m = a.nested ? a.m : 1;
  return scan_layout(a.N, a.p, a.nested ? a.N * a.p * m : 1).total <= SCAN_SMEM_MAX;
}

static bool scan_nested_fit(const LoopArgs& a) {
  const int Nt = a.N_t / n_planes(a);
  return a.m <= SCAN_P_MAX && scan_layout(Nt, a.m, Nt * a.n * a.m).total <= SCAN_SMEM_MAX;
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
static int loop_threads(int p) { return p <= 4 ? 32 : (p <= 16 ? 64 : 128); }

bool loops_form_overlaps(const LoopArgs& a) { return !a.unitarise && scan_loops_fit(a); }

bool loops_transport_only(const LoopArgs& a) { return a.nested && !scan_loops_fit(a); }

bool loops_accept_df(const LoopArgs& a) {
  return !a.unitarise && scan_loops_fit(a) && (!a.nested || scan_nested_fit(a));
}

cudaError_t launch_overlaps(const LoopArgs& a, cudaStream_t s) {
  const long long K = (long long)a.N * a.N_t;
  if (K <= 0 || loops_form_overlaps(a)) return cudaSuccess;
  if (a.df_overlaps && !a.unitarise && a.p * a.p <= 16 * OVL_THREADS) {
    const size_t sm = 2 * size_t(OVL_ROWS) * a.p * sizeof(cdf);
    static size_t cached_df = 0;
    cudaError_t e = set_smem_once(k_overlaps_df, sm, cached_df);
    if (e != cudaSuccess) return e;
    const long long cap = 152LL * 8;
    k_overlaps_df<<<int(K < cap ? K : cap), OVL_THREADS, sm, s>>>(a);
    return cudaGetLastError();
  }
  const size_t sm = a.unitarise ? (4 * size_t(a.p) * a.p * sizeof(z64) +
                                   (a.p / 2 + 2) * sizeof(JacRot<double>) + 64 * sizeof(double))
                                : 0;
  static size_t cached = 0;
  cudaError_t e = set_smem_once(k_overlaps, sm, cached);
  if (e != cudaSuccess) return e;
  const long long cap = 152LL * 32;
  const int grid = int(K < cap ? K : cap);
  k_overlaps<<<grid, loop_threads(a.p), sm, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_loops(const LoopArgs& a, cudaStream_t s) {
  if (a.N_t <= 0) return cudaSuccess;
  if (scan_loops_fit(a)) {
    const ScanSmem Z = scan_layout(a.N, a.p, a.nested ? a.N * a.p * a.m : 1);
    if (a.u_df) {
      static size_t cached_df = 0;
      cudaError_t e = set_smem_once(k_loops_scan<cdf>, Z.total, cached_df);
      if (e != cudaSuccess) return e;
      k_loops_scan<cdf><<<a.N_t, 128, Z.total, s>>>(a);
      return cudaGetLastError();
    }
    static size_t cached_scan = 0;
    cudaError_t e = set_smem_once(k_loops_scan<z64>, Z.total, cached_scan);
    if (e != cudaSuccess) return e;
    k_loops_scan<z64><<<a.N_t, 128, Z.total, s>>>(a);
    return cudaGetLastError();
  }
  // the double-float product stages one more p x p matrix; without room for it the
  // product stays in FP64
  LoopArgs b = a;
  if (b.df_overlaps && loop_layout(b.p, b.nested ? b.m : 1, true).total > size_t(227) * 1024)
    b.df_overlaps = 0;
  const LoopSmem L = loop_layout(b.p, b.nested ? b.m : 1, b.df_overlaps != 0);
  static size_t cached = 0;
  cudaError_t e = set_smem_once(k_loops, L.total, cached);
  if (e != cudaSuccess) return e;
  k_loops<<<b.N_t, loop_threads(b.p), L.total, s>>>(b);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Winding of the hybrid Wannier centres (Eq. 6): s_i = sum_c theta[i][c] / 2pi is the
// total Wannier centre of row i in units of the lattice constant; the Chern (or
// spin-Chern) number is its net change across the transverse period, accumulated
// as sum_i wrap(s_{i+1} - s_i) over the cyclic grid (i = N_t - 1 steps to 0), where
// wrap(d) = d - rint(d) takes each increment to [-1/2, 1/2].  One CTA; the block
// sum runs in a fixed order, so the result is reproducible.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double wcc_row_sum(const double* phases, int i, int p) {
  double s = 0.0;
  for (int c = 0; c < p; ++c) s += phases[(long long)i * p + c];
  return s / 6.283185307179586;
}

__global__ void k_winding(const double* phases, int Nt, int p, double* sums, double* winding) {
  __shared__ double red[64];
  double acc = 0.0;
  for (int i = threadIdx.x; i < Nt; i += blockDim.x) {
    const double s0 = wcc_row_sum(phases, i, p);
    const double s1 = wcc_row_sum(phases, i + 1 == Nt ? 0 : i + 1, p);
    double d = s1 - s0;
    d -= rint(d);
    acc += d;
    if (sums) sums[i] = s0;
  }
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) *winding = acc;
}

cudaError_t launch_winding(const double* phases, int Nt, int p, double* sums, double* winding,
                           cudaStream_t s) {
  k_winding<<<1, 256, 0, s>>>(phases, Nt, p, sums, winding);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Plaquette Berry flux (the coupling-matrix method of the WSpinLine example): link
// variables from the determinants of the overlaps between neighbouring k-points,
//   Lx(j, i) = det U(j+1, i)^dag U(j, i),   Ly(j, i) = det U(j, i+1)^dag U(j, i),
// kept as unit complex numbers (phase only); the plaquette at (j, i), traversed
// k(j, i) -> k(j, i+1) -> k(j+1, i+1) -> k(j+1, i) -> k(j, i), has the Wilson loop
// determinant Ly(j, i) Lx(j, i+1) conj(Ly(j+1, i)) conj(Lx(j, i)) and its flux is the
// argument of that product, in (-pi, pi].  One CTA per k-point forms both overlaps in
// shared memory and takes each determinant's phase by LU with partial pivoting.
// ---------------------------------------------------------------------------
__global__ void k_plaquette_links(const z64* U, int n, int p, int N, int Nt, z64* Lx, z64* Ly) {
  extern __shared__ __align__(16) unsigned char smem[];
  z64* A = reinterpret_cast<z64*>(smem);
  __shared__ int piv;
  __shared__ z64 dsh;
  const int tid = threadIdx.x, nt = blockDim.x;
  const long long K = (long long)N * Nt;
  for (long long k = blockIdx.x; k < K; k += gridDim.x) {
    const int i = int(k / N), j = int(k - (long long)i * N);
    const z64* Uk = U + k * (long long)n * p;
    for (int dir = 0; dir < 2; ++dir) {
      const long long kb = dir == 0 ? (long long)i * N + (j + 1 == N ? 0 : j + 1)
                                    : (long long)(i + 1 == Nt ? 0 : i + 1) * N + j;
      const z64* Ub = U + kb * (long long)n * p;
      for (int e = tid; e < p * p; e += nt) {
        const int r = e / p, c = e - r * p;
        z64 acc(0.0, 0.0);
        for (int q = 0; q < n; ++q) cfma_conj(acc, Ub[(long long)q * p + r], Uk[(long long)q * p + c]);
        A[e] = acc;
      }
      if (tid == 0) dsh = z64(1.0, 0.0);
      __syncthreads();
      for (int c = 0; c < p; ++c) {
        if (tid == 0) {
          int best = c;
          double bmax = abs2(A[c * p + c]);
          for (int r = c + 1; r < p; ++r) {
            const double v = abs2(A[r * p + c]);
            if (v > bmax) {
              bmax = v;
              best = r;
            }
          }
          piv = best;
          const z64 pv = A[best * p + c];
          const double a = sqrt(bmax);
          z64 d = a > 0.0 ? dsh * z64(pv.re / a, pv.im / a) : z64(0.0, 0.0);
          if (best != c) d = z64(-d.re, -d.im);
          dsh = d;
        }
        __syncthreads();
        const int r0 = piv;
        if (r0 != c)
          for (int cc = c + tid; cc < p; cc += nt) {
            const z64 t = A[c * p + cc];
            A[c * p + cc] = A[r0 * p + cc];
            A[r0 * p + cc] = t;
          }
        __syncthreads();
        const z64 pv = A[c * p + c];
        const double pa = abs2(pv);
        for (int r = c + 1 + tid; r < p; r += nt) {  // multipliers A[r][c] / A[c][c]
          const z64 v = A[r * p + c];
          A[r * p + c] = pa > 0.0 ? z64((v.re * pv.re + v.im * pv.im) / pa, (v.im * pv.re - v.re * pv.im) / pa)
                                  : z64(0.0, 0.0);
        }
        __syncthreads();
        const int w = p - c - 1;
        for (int e = tid; e < w * w; e += nt) {
          const int r = c + 1 + e / w, cc = c + 1 + e % w;
          A[r * p + cc] = A[r * p + cc] - A[r * p + c] * A[c * p + cc];
        }
        __syncthreads();
      }
      if (tid == 0) (dir == 0 ? Lx : Ly)[k] = dsh;
      __syncthreads();
    }
  }
}

__global__ void k_plaquette_flux(const z64* Lx, const z64* Ly, int N, int Nt, double* flux) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= (long long)N * Nt) return;
  const int i = int(k / N), j = int(k - (long long)i * N);
  const int j1 = j + 1 == N ? 0 : j + 1, i1 = i + 1 == Nt ? 0 : i + 1;
  const z64 w = Ly[k] * Lx[(long long)i1 * N + j] * conj(Ly[(long long)i * N + j1]) * conj(Lx[k]);
  flux[k] = atan2(w.im, w.re);
}

// Sum of the fluxes / 2pi in a fixed order (one CTA), and per transverse row the
// minimum direct and PSO gaps.
__global__ void k_plaquette_sum(const double* flux, const double* gap, const double* pso_gap, int N,
                                int Nt, double* chern, double* min_gap, double* min_pso_gap) {
  __shared__ double red[64];
  const long long K = (long long)N * Nt;
  double acc = 0.0;
  for (long long k = threadIdx.x; k < K; k += blockDim.x) acc += flux[k];
  acc = block_sum(acc, red);
  if (threadIdx.x == 0 && chern) *chern = acc / 6.283185307179586;
  for (int i = threadIdx.x; i < Nt; i += blockDim.x) {
    double g = INFINITY, gp = INFINITY;
    for (int j = 0; j < N; ++j) {
      if (gap) g = fmin(g, gap[(long long)i * N + j]);
      if (pso_gap) gp = fmin(gp, pso_gap[(long long)i * N + j]);
    }
    if (min_gap) min_gap[i] = g;
    if (min_pso_gap) min_pso_gap[i] = gp;
  }
}

cudaError_t launch_plaquettes(const LoopArgs& a, z64* Lx, z64* Ly, double* flux, double* chern,
                              cudaStream_t s) {
  const long long K = (long long)a.N * a.N_t;
  if (K <= 0) return cudaSuccess;
  const size_t sm = size_t(a.p) * a.p * sizeof(z64);
  static size_t cached = 0;
  cudaError_t e = set_smem_once(k_plaquette_links, sm, cached);
  if (e != cudaSuccess) return e;
  const long long cap = 152LL * 16;
  k_plaquette_links<<<int(K < cap ? K : cap), a.p <= 8 ? 32 : 128, sm, s>>>(a.U, a.n, a.p, a.N, a.N_t, Lx, Ly);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return launch_plaquette_flux(a, Lx, Ly, flux, chern, s);
}

cudaError_t launch_plaquette_flux(const LoopArgs& a, const z64* Lx, const z64* Ly, double* flux,
                                  double* chern, cudaStream_t s) {
  const long long K = (long long)a.N * a.N_t;
  if (K <= 0) return cudaSuccess;
  k_plaquette_flux<<<int((K + 127) / 128), 128, 0, s>>>(Lx, Ly, a.N, a.N_t, flux);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_plaquette_sum<<<1, 256, 0, s>>>(flux, a.gap, a.pso_gap, a.N, a.N_t, chern, a.min_gap, a.min_pso_gap);
  return cudaGetLastError();
}

cudaError_t launch_nested(const LoopArgs& a, cudaStream_t s) {
  if (a.N <= 0) return cudaSuccess;
  const long long bases = (long long)a.N * n_planes(a);
  const int grid = int(bases < 152LL * 64 ? bases : 152LL * 64);
  if (scan_nested_fit(a)) {
    const int Nt = a.N_t / n_planes(a);
    const ScanSmem Z = scan_layout(Nt, a.m, Nt * a.n * a.m);
    if (a.u_df) {
      static size_t cached_df = 0;
      cudaError_t e = set_smem_once(k_nested_scan<cdf>, Z.total, cached_df);
      if (e != cudaSuccess) return e;
      k_nested_scan<cdf><<<grid, 128, Z.total, s>>>(a);
      return cudaGetLastError();
    }
    static size_t cached_scan = 0;
    cudaError_t e = set_smem_once(k_nested_scan<z64>, Z.total, cached_scan);
    if (e != cudaSuccess) return e;
    k_nested_scan<z64><<<grid, 128, Z.total, s>>>(a);
    return cudaGetLastError();
  }
  const LoopSmem L = loop_layout(a.m, 1);
  const size_t sm = L.total + size_t(a.m) * a.m * sizeof(z64);
  static size_t cached = 0;
  cudaError_t e = set_smem_once(k_nested, sm, cached);
  if (e != cudaSuccess) return e;
  k_nested<<<grid, loop_threads(a.m), sm, s>>>(a);
  return cudaGetLastError();
}

}  // namespace bw
