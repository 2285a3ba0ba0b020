// Per-k-point kernels: Bloch Hamiltonian, exact diagonalisation, occupied states.
//
//  - k_build_hk:      H(f) = sum_e t_e exp(i 2 pi f.R_e) |i_e><j_e| to global memory
//                     (Sec. I, the tight-binding Hamiltonian at each k).
//  - k_states_small:  one CTA per k-point, everything in shared memory: build H(k),
//                     Jacobi eigensolve, the lowest p eigenvectors and the direct gap
//                     (Sec. I "exact diagonalization"; Eq. 1 occupied bands), the
//                     optional FP64 refinement of an FP32 solve, and the optional
//                     projected-spin-operator sector (Sec. IV).
//  - k_eigh_small:    batched Hermitian eigensolver on caller matrices (uneven n).
#include <float.h>

#include "jacobi.cuh"
#include "launch.h"

namespace bw {

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

struct SmemLayout {
  size_t phs, A, V, H64, Q, HQ, C, G, Zg, lam, rho, order, order2, rot, red, total;
};

template <typename T>
__host__ __device__ inline SmemLayout states_layout(int n, int p, int nRs, bool mixed) {
  SmemLayout L;
  size_t o = 0;
  const int pp = p > 0 ? p : 1;
  L.phs = o; o = align16(o + size_t(nRs) * sizeof(z64));
  L.A = o; o = align16(o + size_t(n) * n * sizeof(cx<T>));
  L.V = o; o = align16(o + size_t(n) * n * sizeof(cx<T>));
  L.H64 = o; if (mixed) o = align16(o + size_t(n) * n * sizeof(z64));
  L.Q = o; o = align16(o + size_t(n) * pp * sizeof(z64));
  L.HQ = o; o = align16(o + size_t(n) * pp * sizeof(z64));
  L.C = o; if (mixed) o = align16(o + size_t(n) * pp * sizeof(z64));
  L.G = o; o = align16(o + size_t(pp) * pp * sizeof(z64));
  L.Zg = o; o = align16(o + size_t(pp) * pp * sizeof(z64));
  L.lam = o; o = align16(o + size_t(n) * sizeof(double));
  L.rho = o; o = align16(o + size_t(n) * sizeof(double));
  L.order = o; o = align16(o + size_t(n) * sizeof(int));
  L.order2 = o; o = align16(o + size_t(n) * sizeof(int));
  L.rot = o; o = align16(o + size_t(n / 2 + 2) * sizeof(JacRot<double>));
  L.red = o; o = align16(o + 64 * sizeof(double));
  L.total = o;
  return L;
}

// ---------------------------------------------------------------------------
// Bloch Hamiltonian to global memory: one CTA per k-point.
// ---------------------------------------------------------------------------
__global__ void k_build_hk(BuildArgs a) {
  __shared__ z64 phs[PHASE_CACHE];
  const DevModel& md = a.model;
  const int n = md.n, tid = threadIdx.x, nt = blockDim.x;
  const int nRs = min(md.n_R, PHASE_CACHE);
  for (long long k = blockIdx.x; k < a.K; k += gridDim.x) {
    const double f[3] = {a.f[3 * k], a.f[3 * k + 1], a.f[3 * k + 2]};
    for (int r = tid; r < nRs; r += nt) phs[r] = bloch_phase(f, md.Rv + 3 * r);
    const size_t nn = size_t(n) * n;
    if (a.complex64) {
      c32* H = reinterpret_cast<c32*>(a.H) + k * nn;
      for (size_t e = tid; e < nn; e += nt) H[e] = c32(0.f, 0.f);
    } else {
      z64* H = reinterpret_cast<z64*>(a.H) + k * nn;
      for (size_t e = tid; e < nn; e += nt) H[e] = z64(0.0, 0.0);
    }
    __syncthreads();
    for (int e = tid; e < md.n_ent; e += nt) {
      z64 acc(0.0, 0.0);
      for (int h = md.ent_start[e]; h < md.ent_start[e + 1]; ++h) {
        const int r = md.hop_r[h];
        const z64 ph = r < nRs ? phs[r] : bloch_phase(f, md.Rv + 3 * r);
        cfma(acc, md.hop_t[h], ph);
      }
      const size_t at = size_t(md.ent_row[e]) * n + md.ent_col[e];
      if (a.complex64)
        reinterpret_cast<c32*>(a.H)[k * nn + at] = ccast<float>(acc);
      else
        reinterpret_cast<z64*>(a.H)[k * nn + at] = acc;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Shared-memory helpers (FP64, block-wide)
// ---------------------------------------------------------------------------

// C (rows x cols) = A (rows x inner) * B (inner x cols), all row-major in smem.
__device__ void mm(const z64* A, const z64* B, z64* C, int rows, int inner, int cols) {
  for (int e = threadIdx.x; e < rows * cols; e += blockDim.x) {
    const int r = e / cols, c = e - r * cols;
    z64 acc(0.0, 0.0);
    for (int k = 0; k < inner; ++k) cfma(acc, A[r * inner + k], B[k * cols + c]);
    C[e] = acc;
  }
  __syncthreads();
}

// G (p x p) = Q^dagger Q for Q (n x p).
__device__ void gram(const z64* Q, z64* G, int n, int p) {
  for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
    const int a = e / p, b = e - a * p;
    z64 acc(0.0, 0.0);
    for (int r = 0; r < n; ++r) cfma_conj(acc, Q[r * p + a], Q[r * p + b]);
    G[e] = acc;
  }
  __syncthreads();
}

// One Cholesky-QR pass: Q <- Q L^{-dagger} with Q^dagger Q = L L^dagger.  G scratch p x p.
// Returns false when the Gram matrix is not positive definite.
__device__ bool cholqr(z64* Q, z64* G, int n, int p, int* flag) {
  gram(Q, G, n, p);
  chol_lower_warp(G, p, flag);
  if (!*flag) return false;
  // each row x of Q: solve x L^dagger = q, i.e. L y = q^dagger with x = y^dagger
  for (int r = threadIdx.x; r < n; r += blockDim.x) {
    z64* q = Q + r * p;
    for (int j = 0; j < p; ++j) {
      z64 y = conj(q[j]);
      for (int k = 0; k < j; ++k) y = y - G[j * p + k] * conj(q[k]);
      q[j] = conj((1.0 / G[j * p + j].re) * y);
    }
  }
  __syncthreads();
  return true;
}

// Rayleigh-Ritz of span(Q): Q <- Q Z (sorted), HQ <- H Q, rho ascending Ritz values.
// H (n x n) FP64; G, Zg (p x p), C (n x p) scratch.
__device__ bool ritz(const z64* H, z64* Q, z64* HQ, z64* C, z64* G, z64* Zg, double* rho,
                     int* ord, int n, int p, JacRot<double>* rot, double* red, int max_sweeps) {
  mm(H, Q, HQ, n, n, p);
  for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
    const int a = e / p, b = e - a * p;
    z64 acc(0.0, 0.0);
    for (int r = 0; r < n; ++r) cfma_conj(acc, Q[r * p + a], HQ[r * p + b]);
    G[e] = acc;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
    const int a = e / p, b = e - a * p;
    if (a < b) {
      const z64 x = G[a * p + b], y = conj(G[b * p + a]);
      const z64 h = 0.5 * (x + y);
      G[a * p + b] = h;
      G[b * p + a] = conj(h);
    } else if (a == b) {
      G[e] = z64(G[e].re, 0.0);
    }
  }
  __syncthreads();
  const int sw = jacobi_eigh<double>(G, Zg, p, p, max_sweeps, rot, red);
  sort_diag<double>(G, p, p, ord);
  for (int c = threadIdx.x; c < p; c += blockDim.x) rho[c] = G[ord[c] * p + ord[c]].re;
  // Q <- Q Zg[:, ord], HQ <- HQ Zg[:, ord], each through the scratch C
  for (int pass = 0; pass < 2; ++pass) {
    z64* X = pass == 0 ? Q : HQ;
    for (int e = threadIdx.x; e < n * p; e += blockDim.x) {
      const int r = e / p, c = e - r * p;
      z64 acc(0.0, 0.0);
      for (int k = 0; k < p; ++k) cfma(acc, X[r * p + k], Zg[k * p + ord[c]]);
      C[e] = acc;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n * p; e += blockDim.x) X[e] = C[e];
    __syncthreads();
  }
  return sw >= 0;
}

// Mixed precision: refine the lowest-p invariant subspace of the FP64 matrix H
// starting from an FP32 eigenbasis V (columns ordered by ord, eigenvalues lam).
// One Newton correction in the FP32 eigenbasis of the complement,
//   Q <- Q + V_u C,  C[a][i] = (V_u^dagger R)[a][i] / (G_ii - lam_{p+a}),
// with the FP64 residual R = H Q - Q G, G = Q^dagger H Q (its off-diagonal part is
// of the order of the FP32 error and enters the correction at second order), then
// Cholesky-QR.  The FP32 start is accurate to eps32 ||H|| / gap, the corrected
// subspace to about (eps32 ||H|| / gap)^2.  Returns the direct gap from FP64
// Rayleigh quotients of the p-th and (p+1)-th FP32 vectors; *ok = 0 when a
// Cholesky factorisation broke down.
__device__ double refine_mixed(const z64* H, const c32* V, const int* ord, const double* lam,
                               int n, int p, z64* Q, z64* HQ, z64* C, z64* G, z64* Zg,
                               double* rho, int* ord2, JacRot<double>* rot, double* red,
                               int max_sweeps, int* ok, int* flag) {
  const int tid = threadIdx.x, nt = blockDim.x;
  (void)Zg; (void)rho; (void)ord2; (void)rot; (void)max_sweeps;
  *ok = cholqr(Q, G, n, p, flag) ? 1 : 0;
  if (p < n) {
    mm(H, Q, HQ, n, n, p);
    // diagonal of G = Q^dagger H Q, then R = H Q - Q G (full G)
    for (int e = tid; e < p * p; e += nt) {
      const int a = e / p, b = e - a * p;
      z64 acc(0.0, 0.0);
      for (int r = 0; r < n; ++r) cfma_conj(acc, Q[r * p + a], HQ[r * p + b]);
      G[e] = acc;
    }
    __syncthreads();
    for (int e = tid; e < n * p; e += nt) {
      const int r = e / p, c = e - r * p;
      z64 acc = HQ[e];
      for (int q = 0; q < p; ++q) acc = acc - Q[r * p + q] * G[q * p + c];
      C[e] = acc;  // residual, kept in C
    }
    __syncthreads();
    const int nu = n - p;
    for (int e = tid; e < nu * p; e += nt) {
      const int a = e / p, i = e - a * p;
      const int col = ord[p + a];
      z64 acc(0.0, 0.0);
      for (int r = 0; r < n; ++r) cfma_conj(acc, ccast<double>(V[r * n + col]), C[r * p + i]);
      HQ[e] = (1.0 / (G[i * p + i].re - lam[col])) * acc;  // correction coefficients
    }
    __syncthreads();
    for (int e = tid; e < n * p; e += nt) {
      const int r = e / p, i = e - r * p;
      z64 acc = Q[e];
      for (int a = 0; a < nu; ++a) cfma(acc, ccast<double>(V[r * n + ord[p + a]]), HQ[a * p + i]);
      Q[e] = acc;
    }
    __syncthreads();
    if (!cholqr(Q, G, n, p, flag)) *ok = 0;
  }
  // gap from FP64 Rayleigh quotients of the FP32 vectors p-1 and p
  double gap = INFINITY;
  if (p < n) {
    double rq[2];
    for (int s = 0; s < 2; ++s) {
      const int col = ord[p - 1 + s];
      double num = 0.0, den = 0.0;
      for (int r = tid; r < n; r += nt) {
        z64 hv(0.0, 0.0);
        for (int c = 0; c < n; ++c) cfma(hv, H[r * n + c], ccast<double>(V[c * n + col]));
        const z64 v = ccast<double>(V[r * n + col]);
        num += v.re * hv.re + v.im * hv.im;
        den += abs2(v);
      }
      num = block_sum(num, red);
      den = block_sum(den, red);
      rq[s] = num / den;
    }
    gap = rq[1] - rq[0];
  }
  return gap;
}

// Projected spin operator sector (Sec. IV): S = U^dagger s U (p x p), eigh, keep the
// eigenvectors with eigenvalue sign `sign` (split at zero), or the p/2 lowest / highest
// (median); Us = U V_s written to `out` (n x p/2).
__device__ void pso_split(const z64* U, const DevOp& op, int sign, int median, int n, int p, z64* S,
                          z64* SV, int* ord, double* mu, JacRot<double>* rot, double* red,
                          int max_sweeps, z64* out, double* pso_out, double* pso_gap_out,
                          double pso_tol, DevStatus* st, long long k) {
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int e = tid; e < p * p; e += nt) {
    const int a = e / p, b = e - a * p;
    z64 acc(0.0, 0.0);
    for (int q = 0; q < op.nnz; ++q) {
      const z64 sv = op.val[q] * U[op.col[q] * p + b];
      cfma_conj(acc, U[op.row[q] * p + a], sv);
    }
    S[e] = acc;
  }
  __syncthreads();
  for (int e = tid; e < p * p; e += nt) {
    const int a = e / p, b = e - a * p;
    if (a < b) {
      const z64 h = 0.5 * (S[a * p + b] + conj(S[b * p + a]));
      S[a * p + b] = h;
      S[b * p + a] = conj(h);
    } else if (a == b) {
      S[e] = z64(S[e].re, 0.0);
    }
  }
  __syncthreads();
  const int sw = jacobi_eigh<double>(S, SV, p, p, max_sweeps, rot, red);
  sort_diag<double>(S, p, p, ord);
  for (int c = tid; c < p; c += nt) mu[c] = S[ord[c] * p + ord[c]].re;
  __syncthreads();
  const int h = p / 2;
  if (tid == 0) {
    int neg = 0;
    double g = INFINITY;
    for (int c = 0; c < p; ++c) {
      neg += mu[c] < 0.0;
      g = fmin(g, fabs(mu[c]));
    }
    if (median) {
      neg = h;
      g = mu[h] - mu[h - 1];
    }
    if (pso_out)
      for (int c = 0; c < p; ++c) pso_out[c] = mu[c];
    if (pso_gap_out) *pso_gap_out = g;
    if (sw < 0) report(st, ST_ENOCONV, k, 0.0);
    if (neg != h || !(g > pso_tol)) report(st, ST_EPSOGAP, k, g);
  }
  const int c0 = sign < 0 ? 0 : h;
  for (int e = tid; e < n * h; e += nt) {
    const int r = e / h, c = e - r * h;
    z64 acc(0.0, 0.0);
    for (int a = 0; a < p; ++a) cfma(acc, U[r * p + a], SV[a * p + ord[c0 + c]]);
    out[e] = acc;
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// One CTA per k-point: build, solve, (refine), (spin split), write.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_states_small(StatesArgs a, int p_out) {
  extern __shared__ __align__(16) unsigned char smem[];
  const DevModel& md = a.model;
  const int n = md.n, p = a.p, tid = threadIdx.x, nt = blockDim.x;
  const int nRs = min(md.n_R, PHASE_CACHE);
  const bool mixed = a.mixed != 0;
  const SmemLayout L = states_layout<T>(n, p, nRs, mixed);
  z64* phs = reinterpret_cast<z64*>(smem + L.phs);
  cx<T>* A = reinterpret_cast<cx<T>*>(smem + L.A);
  cx<T>* V = reinterpret_cast<cx<T>*>(smem + L.V);
  z64* H64 = reinterpret_cast<z64*>(smem + L.H64);
  z64* Q = reinterpret_cast<z64*>(smem + L.Q);
  z64* HQ = reinterpret_cast<z64*>(smem + L.HQ);
  z64* C = reinterpret_cast<z64*>(smem + L.C);
  z64* G = reinterpret_cast<z64*>(smem + L.G);
  z64* Zg = reinterpret_cast<z64*>(smem + L.Zg);
  double* lam = reinterpret_cast<double*>(smem + L.lam);
  double* rho = reinterpret_cast<double*>(smem + L.rho);
  int* ord = reinterpret_cast<int*>(smem + L.order);
  int* ord2 = reinterpret_cast<int*>(smem + L.order2);
  JacRot<double>* rot64 = reinterpret_cast<JacRot<double>*>(smem + L.rot);
  JacRot<T>* rot = reinterpret_cast<JacRot<T>*>(smem + L.rot);
  double* red = reinterpret_cast<double*>(smem + L.red);
  int* flag = reinterpret_cast<int*>(red + 40);

  for (long long k = blockIdx.x; k < a.K; k += gridDim.x) {
    double f[3];
    if (a.f) {
      f[0] = a.f[3 * k]; f[1] = a.f[3 * k + 1]; f[2] = a.f[3 * k + 2];
    } else {
      const int i = int(k / a.plane.N), j = int(k - (long long)i * a.plane.N);
      plane_f(a.plane, i, j, f);
    }
    for (int r = tid; r < nRs; r += nt) phs[r] = bloch_phase(f, md.Rv + 3 * r);
    for (int e = tid; e < n * n; e += nt) {
      A[e] = cx<T>(T(0), T(0));
      if (mixed) H64[e] = z64(0.0, 0.0);
    }
    __syncthreads();
    for (int e = tid; e < md.n_ent; e += nt) {
      z64 acc(0.0, 0.0);
      for (int h = md.ent_start[e]; h < md.ent_start[e + 1]; ++h) {
        const int r = md.hop_r[h];
        const z64 ph = r < nRs ? phs[r] : bloch_phase(f, md.Rv + 3 * r);
        cfma(acc, md.hop_t[h], ph);
      }
      const int at = md.ent_row[e] * n + md.ent_col[e];
      A[at] = ccast<T>(acc);
      if (mixed) H64[at] = acc;
    }
    __syncthreads();
    const int sw = jacobi_eigh<T>(A, V, n, n, a.max_sweeps, rot, red);
    sort_diag<T>(A, n, n, ord);
    for (int c = tid; c < n; c += nt) lam[c] = double(A[c * n + c].re);
    for (int e = tid; e < n * p; e += nt) {
      const int r = e / p, c = e - r * p;
      Q[e] = ccast<double>(V[r * n + ord[c]]);
    }
    __syncthreads();
    double gap;
    int ok = 1;
    if (!mixed) {
      gap = p < n ? lam[ord[p]] - lam[ord[p - 1]] : INFINITY;
    } else {
      gap = refine_mixed(H64, reinterpret_cast<const c32*>(V), ord, lam, n, p, Q, HQ, C, G, Zg,
                         rho, ord2, rot64, red, a.max_sweeps, &ok, flag);
    }
    if (tid == 0) {
      a.gap[k] = gap;
      if (sw < 0 || !ok) report(a.status, ST_ENOCONV, k, 0.0);
      if (!(gap > a.gap_tol)) report(a.status, ST_EGAP, k, gap);
    }
    z64* out = a.U + k * (long long)n * p_out;
    if (a.op.nnz > 0) {
      pso_split(Q, a.op, a.sign, a.pso_median, n, p, G, Zg, ord2, rho, rot64, red, a.max_sweeps, out,
                a.pso_evals ? a.pso_evals + k * p : nullptr, a.pso_gap ? a.pso_gap + k : nullptr,
                a.pso_gap_tol, a.status, k);
    } else {
      for (int e = tid; e < n * p; e += nt) out[e] = Q[e];
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Batched eigensolver on caller matrices (n <= SMALL_N_MAX): one CTA per matrix.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_eigh_small(EighArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int tid = threadIdx.x, nt = blockDim.x;
  for (long long b = blockIdx.x; b < a.batch; b += gridDim.x) {
    const int n = a.n_per[b];
    const int p = min(a.n_vec, n);
    const bool mixed = a.mixed != 0 && p > 0;
    const SmemLayout L = states_layout<T>(n, p, 0, mixed);
    cx<T>* A = reinterpret_cast<cx<T>*>(smem + L.A);
    cx<T>* V = reinterpret_cast<cx<T>*>(smem + L.V);
    z64* H64 = reinterpret_cast<z64*>(smem + L.H64);
    z64* Q = reinterpret_cast<z64*>(smem + L.Q);
    z64* HQ = reinterpret_cast<z64*>(smem + L.HQ);
    z64* C = reinterpret_cast<z64*>(smem + L.C);
    z64* G = reinterpret_cast<z64*>(smem + L.G);
    z64* Zg = reinterpret_cast<z64*>(smem + L.Zg);
    double* lam = reinterpret_cast<double*>(smem + L.lam);
    double* rho = reinterpret_cast<double*>(smem + L.rho);
    int* ord = reinterpret_cast<int*>(smem + L.order);
    int* ord2 = reinterpret_cast<int*>(smem + L.order2);
    JacRot<double>* rot64 = reinterpret_cast<JacRot<double>*>(smem + L.rot);
    JacRot<T>* rot = reinterpret_cast<JacRot<T>*>(smem + L.rot);
    double* red = reinterpret_cast<double*>(smem + L.red);
    int* flag = reinterpret_cast<int*>(red + 40);
    const z64* Hg = a.H + a.h_off[b];
    for (int e = tid; e < n * n; e += nt) {
      const int r = e / n, c = e - r * n;
      // Hermitian part of the input
      const z64 x = Hg[e], y = conj(Hg[c * n + r]);
      const z64 h = (r == c) ? z64(x.re, 0.0) : 0.5 * (x + y);
      A[e] = ccast<T>(h);
      if (mixed) H64[e] = h;
    }
    __syncthreads();
    const int sw = jacobi_eigh<T>(A, V, n, n, a.max_sweeps, rot, red);
    sort_diag<T>(A, n, n, ord);
    for (int c = tid; c < n; c += nt) lam[c] = double(A[c * n + c].re);
    __syncthreads();
    int ok = 1;
    if (mixed) {
      for (int e = tid; e < n * p; e += nt) {
        const int r = e / p, c = e - r * p;
        Q[e] = ccast<double>(V[r * n + ord[c]]);
      }
      __syncthreads();
      refine_mixed(H64, reinterpret_cast<const c32*>(V), ord, lam, n, p, Q, HQ, C, G, Zg, rho,
                   ord2, rot64, red, a.max_sweeps, &ok, flag);
      // individual eigenpairs: Rayleigh-Ritz on the refined subspace
      if (!ritz(H64, Q, HQ, C, G, Zg, rho, ord2, n, p, rot64, red, a.max_sweeps)) ok = 0;
    }
    double* ev = a.evals + a.e_off[b];
    for (int c = tid; c < n; c += nt) ev[c] = (mixed && c < p) ? rho[c] : lam[ord[c]];
    if (a.evecs && p > 0) {
      z64* out = a.evecs + a.v_off[b];
      for (int e = tid; e < n * p; e += nt) {
        const int r = e / p, c = e - r * p;
        out[e] = mixed ? Q[e] : ccast<double>(V[r * n + ord[c]]);
      }
    }
    if (tid == 0 && (sw < 0 || !ok)) report(a.status, ST_ENOCONV, b, 0.0);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
static int threads_for(int n) { return n <= 8 ? 32 : (n <= 16 ? 64 : 128); }

static int grid_for(long long units) {
  const long long cap = 152LL * 64;
  return int(units < cap ? (units > 0 ? units : 1) : cap);
}

cudaError_t launch_build_hk(const BuildArgs& a, cudaStream_t s) {
  if (a.K <= 0) return cudaSuccess;
  k_build_hk<<<grid_for(a.K), 256, 0, s>>>(a);
  return cudaGetLastError();
}

template <typename T>
static cudaError_t states_impl(const StatesArgs& a, int p_out, cudaStream_t s) {
  const int nRs = a.model.n_R < PHASE_CACHE ? a.model.n_R : PHASE_CACHE;
  const SmemLayout L = states_layout<T>(a.model.n, a.p, nRs, a.mixed != 0);
  static size_t cached = 0;
  cudaError_t e = set_smem_once(k_states_small<T>, L.total, cached);
  if (e != cudaSuccess) return e;
  k_states_small<T><<<grid_for(a.K), threads_for(a.model.n), L.total, s>>>(a, p_out);
  return cudaGetLastError();
}

cudaError_t launch_states_small(const StatesArgs& a, int p_out, cudaStream_t s) {
  if (a.K <= 0) return cudaSuccess;
  bool handled = false;
  const cudaError_t e = launch_states_tiny(a, p_out, s, &handled);
  if (handled || e != cudaSuccess) return e;
  return a.mixed ? states_impl<float>(a, p_out, s) : states_impl<double>(a, p_out, s);
}

template <typename T>
static cudaError_t eigh_impl(const EighArgs& a, int n_max, cudaStream_t s) {
  const SmemLayout L = states_layout<T>(n_max, a.n_vec < n_max ? a.n_vec : n_max, 0, a.mixed != 0);
  // the layout of the largest matrix bounds every smaller one
  static size_t cached = 0;
  cudaError_t e = set_smem_once(k_eigh_small<T>, L.total, cached);
  if (e != cudaSuccess) return e;
  k_eigh_small<T><<<grid_for(a.batch), threads_for(n_max), L.total, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_eigh_small(const EighArgs& a, int n_max, cudaStream_t s) {
  if (a.batch <= 0) return cudaSuccess;
  return a.mixed ? eigh_impl<float>(a, n_max, s) : eigh_impl<double>(a, n_max, s);
}

}  // namespace bw
