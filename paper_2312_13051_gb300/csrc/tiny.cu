// One thread per k-point for few-band models (n = 2 or 4): Bloch Hamiltonian,
// exact diagonalisation, optional FP64 refinement and projected-spin sector, all
// in registers (Sec. I "exact diagonalization", Eq. 1, Sec. IV).
//
// GB300's FP64 pipe serves a whole warp instruction at a time, so a kernel that
// gives one small matrix to a CTA pays for 32 lanes and uses a few.  Here every
// lane owns its own k-point: the matrix sizes are compile-time constants, loops
// unroll, and the arrays stay in registers.  The Bloch phases come from per-CTA
// tables: with an integer loop direction and an integer transverse direction,
// f(j, i).R = origin.R + j (loop.R) / N + i (trans.R) / N_t, so
// exp(i 2pi f.R) = exp(i 2pi origin.R) w_N^{(j loop.R) mod N} w_Nt^{(i trans.R) mod N_t}
// with w_M = exp(i 2pi / M) tabulated once per CTA.
#include <float.h>

#include "launch.h"

namespace bw {
namespace {

template <typename T>
__device__ __forceinline__ T teps();
template <>
__device__ __forceinline__ double teps<double>() { return 2.220446049250313e-16; }
template <>
__device__ __forceinline__ float teps<float>() { return 1.1920929e-7f; }

// Serial cyclic Jacobi on a Hermitian NN x NN matrix held in registers; V collects
// the rotations (same rotation formula and skip test as the block solver).  Returns the sweeps
// used or -1 without convergence.
template <int NN, typename T>
__device__ __forceinline__ int jac_serial(cx<T> (&A)[NN][NN], cx<T> (&V)[NN][NN], int max_sweeps) {
#pragma unroll
  for (int r = 0; r < NN; ++r)
#pragma unroll
    for (int c = 0; c < NN; ++c) V[r][c] = cx<T>(T(r == c), T(0));
  T fro = T(0);
#pragma unroll
  for (int r = 0; r < NN; ++r)
#pragma unroll
    for (int c = 0; c < NN; ++c) fro += abs2(A[r][c]);
  const T tol2 = T(64) * teps<T>() * teps<T>() * fro;
  for (int sweep = 0; sweep <= max_sweeps; ++sweep) {
    T off = T(0);
#pragma unroll
    for (int p = 0; p < NN; ++p)
#pragma unroll
      for (int q = p + 1; q < NN; ++q) off += T(2) * abs2(A[p][q]);
    if (off <= tol2 || fro == T(0)) return sweep;
    if (sweep == max_sweeps) break;
    bool rotated = false;
#pragma unroll
    for (int p = 0; p < NN; ++p)
#pragma unroll
      for (int q = p + 1; q < NN; ++q) {
        const cx<T> b = A[p][q];
        const T ab = sqrt(abs2(b));
        const T a = A[p][p].re, d = A[q][q].re;
        if (!(ab > T(4) * teps<T>() * sqrt(fabs(a) * fabs(d)) && ab > T(0))) continue;
        rotated = true;
        const T tau = (d - a) / (T(2) * ab);
        const T t = (tau >= T(0) ? T(1) : T(-1)) / (fabs(tau) + sqrt(T(1) + tau * tau));
        const T c = T(1) / sqrt(T(1) + t * t);
        const T s = t * c / ab;
        const cx<T> sc(s * b.re, s * b.im);
#pragma unroll
        for (int k = 0; k < NN; ++k) {
          const cx<T> ap = A[p][k], aq = A[q][k];
          A[p][k] = c * ap - sc * aq;
          A[q][k] = conj(sc) * ap + c * aq;
        }
#pragma unroll
        for (int k = 0; k < NN; ++k) {
          const cx<T> ap = A[k][p], aq = A[k][q];
          A[k][p] = c * ap - aq * conj(sc);
          A[k][q] = ap * sc + c * aq;
          const cx<T> vp = V[k][p], vq = V[k][q];
          V[k][p] = c * vp - vq * conj(sc);
          V[k][q] = vp * sc + c * vq;
        }
        A[p][q] = cx<T>(T(0), T(0));
        A[q][p] = cx<T>(T(0), T(0));
        A[p][p] = cx<T>(a - t * ab, T(0));
        A[q][q] = cx<T>(d + t * ab, T(0));
      }
    if (!rotated) return sweep + 1;
  }
  return -1;
}

// Columns of V sorted by ascending diagonal of A (stable): Vs[:, c], lam[c].
template <int NN, typename T>
__device__ __forceinline__ void sort_eig(const cx<T> (&A)[NN][NN], const cx<T> (&V)[NN][NN],
                                         cx<T> (&Vs)[NN][NN], T (&lam)[NN]) {
  int rank[NN];
#pragma unroll
  for (int a = 0; a < NN; ++a) {
    int r = 0;
#pragma unroll
    for (int b = 0; b < NN; ++b)
      r += (A[b][b].re < A[a][a].re) || (A[b][b].re == A[a][a].re && b < a);
    rank[a] = r;
  }
#pragma unroll
  for (int c = 0; c < NN; ++c) {
#pragma unroll
    for (int a = 0; a < NN; ++a)
      if (rank[a] == c) {
        lam[c] = A[a][a].re;
#pragma unroll
        for (int r = 0; r < NN; ++r) Vs[r][c] = V[r][a];
      }
  }
}

// One Cholesky-QR pass on the columns of Q (NN x PP) in FP64; false on breakdown.
template <int NN, int PP>
__device__ __forceinline__ bool cholqr_serial(z64 (&Q)[NN][PP]) {
  z64 L[PP][PP];
#pragma unroll
  for (int a = 0; a < PP; ++a)
#pragma unroll
    for (int b = 0; b <= a; ++b) {
      z64 g(0.0, 0.0);
#pragma unroll
      for (int r = 0; r < NN; ++r) cfma_conj(g, Q[r][b], Q[r][a]);  // G[a][b] = q_b^dag q_a ... conj
      L[a][b] = conj(g);                                            // G[a][b] = q_a^dag q_b
    }
  bool ok = true;
#pragma unroll
  for (int j = 0; j < PP; ++j) {
    double d = L[j][j].re;
#pragma unroll
    for (int k = 0; k < j; ++k) d -= abs2(L[j][k]);
    ok = ok && (d > 0.0);
    d = sqrt(fmax(d, 1e-300));
    L[j][j] = z64(d, 0.0);
#pragma unroll
    for (int i = j + 1; i < PP; ++i) {
      z64 s = L[i][j];
#pragma unroll
      for (int k = 0; k < j; ++k) s = s - L[i][k] * conj(L[j][k]);
      L[i][j] = (1.0 / d) * s;
    }
  }
#pragma unroll
  for (int r = 0; r < NN; ++r) {
    // row x of the new Q solves x L^dagger = q: L y = q^dagger, x = y^dagger
    z64 y[PP];
#pragma unroll
    for (int j = 0; j < PP; ++j) {
      z64 v = conj(Q[r][j]);
#pragma unroll
      for (int k = 0; k < j; ++k) v = v - L[j][k] * y[k];
      y[j] = (1.0 / L[j][j].re) * v;
    }
#pragma unroll
    for (int j = 0; j < PP; ++j) Q[r][j] = conj(y[j]);
  }
  return ok;
}


constexpr int TINY_THREADS = 32;

__device__ __forceinline__ int pmod(long long x, int m) {
  long long r = x % m;
  return int(r < 0 ? r + m : r);
}

// FP64 Rayleigh quotient v^dagger H v / v^dagger v of an FP32 vector.
template <int NN>
__device__ __forceinline__ double rq(const z64 (&H)[NN][NN], const c32 (&V)[NN][NN], int col) {
  double num = 0.0, den = 0.0;
#pragma unroll
  for (int r = 0; r < NN; ++r) {
    z64 hv(0.0, 0.0);
#pragma unroll
    for (int c = 0; c < NN; ++c) cfma(hv, H[r][c], ccast<double>(V[c][col]));
    const z64 v = ccast<double>(V[r][col]);
    num += v.re * hv.re + v.im * hv.im;
    den += abs2(v);
  }
  return num / den;
}

template <int NN, int PP, bool MIXED>
__global__ void __launch_bounds__(TINY_THREADS)
k_states_tiny(StatesArgs a, int use_tab) {
  extern __shared__ __align__(16) unsigned char smem[];
  const DevModel& md = a.model;
  const int tid = threadIdx.x, bd = blockDim.x, nR = md.n_R;
  const int N = a.plane.N, Nt = a.plane.N_t;
  z64* cache = reinterpret_cast<z64*>(smem);             // nR x bd
  z64* tabN = cache + nR * bd;                             // N
  z64* tabNt = tabN + (use_tab ? N : 0);                   // N_t
  z64* oph = tabNt + (use_tab ? Nt : 0);                   // nR
  int* lR = reinterpret_cast<int*>(oph + (use_tab ? nR : 0));
  int* tR = lR + (use_tab ? nR : 0);
  if (use_tab) {
    for (int m = tid; m < N; m += bd) {
      double s, c;
      sincospi(2.0 * double(m) / double(N), &s, &c);
      tabN[m] = z64(c, s);
    }
    for (int m = tid; m < Nt; m += bd) {
      double s, c;
      sincospi(2.0 * double(m) / double(Nt), &s, &c);
      tabNt[m] = z64(c, s);
    }
    for (int r = tid; r < nR; r += bd) {
      const int* R = md.Rv + 3 * r;
      double x = 0.0;
      int l = 0, t = 0;
      for (int d = 0; d < 3; ++d) {
        x += a.plane.origin[d] * double(R[d]);
        l += int(a.plane.loop_dir[d]) * R[d];
        t += int(a.plane.trans_dir[d]) * R[d];
      }
      double s, c;
      sincospi(2.0 * x, &s, &c);
      oph[r] = z64(c, s);
      lR[r] = l;
      tR[r] = t;
    }
    __syncthreads();
  }
  const long long k = (long long)blockIdx.x * bd + tid;
  if (k >= a.K) return;
  const int i = int(k / N), j = int(k - (long long)i * N);
  // Bloch phases of the distinct translations at this k-point
  if (use_tab) {
    for (int r = 0; r < nR; ++r)
      cache[r * bd + tid] = oph[r] * tabN[pmod((long long)j * lR[r], N)] *
                            tabNt[pmod((long long)i * tR[r], Nt)];
  } else {
    double f[3];
    if (a.f) {
      f[0] = a.f[3 * k]; f[1] = a.f[3 * k + 1]; f[2] = a.f[3 * k + 2];
    } else {
      plane_f(a.plane, i, j, f);
    }
    for (int r = 0; r < nR; ++r) cache[r * bd + tid] = bloch_phase(f, md.Rv + 3 * r);
  }
  // H(k) in FP64 registers
  z64 H[NN][NN];
#pragma unroll
  for (int r = 0; r < NN; ++r)
#pragma unroll
    for (int c = 0; c < NN; ++c) H[r][c] = z64(0.0, 0.0);
  for (int e = 0; e < md.n_ent; ++e) {
    z64 acc(0.0, 0.0);
    for (int h = md.ent_start[e]; h < md.ent_start[e + 1]; ++h)
      cfma(acc, md.hop_t[h], cache[md.hop_r[h] * bd + tid]);
    const int row = md.ent_row[e], col = md.ent_col[e];
#pragma unroll
    for (int r = 0; r < NN; ++r)
#pragma unroll
      for (int c = 0; c < NN; ++c)
        if (row == r && col == c) H[r][c] = acc;
  }
  z64 Q[NN][PP];
  double gap = INFINITY;
  bool ok = true;
  if (MIXED) {
    c32 A[NN][NN], V[NN][NN], Vs[NN][NN];
    float lam[NN];
#pragma unroll
    for (int r = 0; r < NN; ++r)
#pragma unroll
      for (int c = 0; c < NN; ++c) A[r][c] = ccast<float>(H[r][c]);
    ok = jac_serial<NN, float>(A, V, a.max_sweeps) >= 0;
    sort_eig<NN, float>(A, V, Vs, lam);
#pragma unroll
    for (int r = 0; r < NN; ++r)
#pragma unroll
      for (int c = 0; c < PP; ++c) Q[r][c] = ccast<double>(Vs[r][c]);
    ok = cholqr_serial<NN, PP>(Q) && ok;
    if (PP < NN) {
      // one Newton correction from the FP32 eigenbasis (see the block refinement)
      z64 HQ[NN][PP], G[PP][PP];
#pragma unroll
      for (int r = 0; r < NN; ++r)
#pragma unroll
        for (int c = 0; c < PP; ++c) {
          z64 acc(0.0, 0.0);
#pragma unroll
          for (int q = 0; q < NN; ++q) cfma(acc, H[r][q], Q[q][c]);
          HQ[r][c] = acc;
        }
#pragma unroll
      for (int x = 0; x < PP; ++x)
#pragma unroll
        for (int y = 0; y < PP; ++y) {
          z64 acc(0.0, 0.0);
#pragma unroll
          for (int r = 0; r < NN; ++r) cfma_conj(acc, Q[r][x], HQ[r][y]);
          G[x][y] = acc;
        }
#pragma unroll
      for (int r = 0; r < NN; ++r)
#pragma unroll
        for (int c = 0; c < PP; ++c) {
#pragma unroll
          for (int q = 0; q < PP; ++q) HQ[r][c] = HQ[r][c] - Q[r][q] * G[q][c];
        }
#pragma unroll
      for (int u = PP; u < NN; ++u)
#pragma unroll
        for (int c = 0; c < PP; ++c) {
          z64 acc(0.0, 0.0);
#pragma unroll
          for (int r = 0; r < NN; ++r) cfma_conj(acc, ccast<double>(Vs[r][u]), HQ[r][c]);
          acc = (1.0 / (G[c][c].re - double(lam[u]))) * acc;
#pragma unroll
          for (int r = 0; r < NN; ++r) cfma(Q[r][c], ccast<double>(Vs[r][u]), acc);
        }
      ok = cholqr_serial<NN, PP>(Q) && ok;
      gap = rq<NN>(H, Vs, PP) - rq<NN>(H, Vs, PP - 1);
    }
  } else {
    z64 A[NN][NN], V[NN][NN], Vs[NN][NN];
    double lam[NN];
#pragma unroll
    for (int r = 0; r < NN; ++r)
#pragma unroll
      for (int c = 0; c < NN; ++c) A[r][c] = H[r][c];
    ok = jac_serial<NN, double>(A, V, a.max_sweeps) >= 0;
    sort_eig<NN, double>(A, V, Vs, lam);
#pragma unroll
    for (int r = 0; r < NN; ++r)
#pragma unroll
      for (int c = 0; c < PP; ++c) Q[r][c] = Vs[r][c];
    if (PP < NN) gap = lam[PP] - lam[PP - 1];
  }
  a.gap[k] = gap;
  if (!ok) report(a.status, ST_ENOCONV, k, 0.0);
  if (!(gap > a.gap_tol)) report(a.status, ST_EGAP, k, gap);
  z64* out = a.U + k * (long long)NN * (a.op.nnz > 0 ? PP / 2 : PP);
  if (a.op.nnz > 0) {
    if (PP % 2 == 0) {
      // projected spin operator restricted to the occupied space (Sec. IV)
      z64 S[PP][PP], SV[PP][PP], SVs[PP][PP];
      double mu[PP];
#pragma unroll
      for (int x = 0; x < PP; ++x)
#pragma unroll
        for (int y = 0; y < PP; ++y) S[x][y] = z64(0.0, 0.0);
      for (int q = 0; q < a.op.nnz; ++q) {
        const int row = a.op.row[q], col = a.op.col[q];
        const z64 v = a.op.val[q];
        z64 qa[PP], qb[PP];
#pragma unroll
        for (int c = 0; c < PP; ++c) {
          qa[c] = z64(0.0, 0.0);
          qb[c] = z64(0.0, 0.0);
        }
#pragma unroll
        for (int r = 0; r < NN; ++r)
#pragma unroll
          for (int c = 0; c < PP; ++c) {
            if (r == row) qa[c] = Q[r][c];
            if (r == col) qb[c] = Q[r][c];
          }
#pragma unroll
        for (int x = 0; x < PP; ++x)
#pragma unroll
          for (int y = 0; y < PP; ++y) cfma_conj(S[x][y], qa[x], v * qb[y]);
      }
#pragma unroll
      for (int x = 0; x < PP; ++x) {
        S[x][x] = z64(S[x][x].re, 0.0);
#pragma unroll
        for (int y = x + 1; y < PP; ++y) {
          const z64 h = 0.5 * (S[x][y] + conj(S[y][x]));
          S[x][y] = h;
          S[y][x] = conj(h);
        }
      }
      const bool okp = jac_serial<PP, double>(S, SV, a.max_sweeps) >= 0;
      sort_eig<PP, double>(S, SV, SVs, mu);
      int neg = 0;
      double g = INFINITY;
#pragma unroll
      for (int c = 0; c < PP; ++c) {
        neg += mu[c] < 0.0;
        g = fmin(g, fabs(mu[c]));
        if (a.pso_evals) a.pso_evals[k * PP + c] = mu[c];
      }
      if (a.pso_gap) a.pso_gap[k] = g;
      if (!okp) report(a.status, ST_ENOCONV, k, 0.0);
      if (neg != PP / 2 || !(g > a.pso_gap_tol)) report(a.status, ST_EPSOGAP, k, g);
      const int c0 = a.sign < 0 ? 0 : PP / 2;
#pragma unroll
      for (int r = 0; r < NN; ++r)
#pragma unroll
        for (int c = 0; c < PP / 2; ++c) {
          z64 acc(0.0, 0.0);
#pragma unroll
          for (int q = 0; q < PP; ++q) {
            z64 sv = SVs[q][c];
            if (c0) sv = SVs[q][c + PP / 2];
            cfma(acc, Q[r][q], sv);
          }
          out[r * (PP / 2) + c] = acc;
        }
    }
  } else {
#pragma unroll
    for (int r = 0; r < NN; ++r)
#pragma unroll
      for (int c = 0; c < PP; ++c) out[r * PP + c] = Q[r][c];
  }
}

template <int NN, int PP, bool MIXED>
cudaError_t tiny_launch(const StatesArgs& a, int use_tab, size_t smem, cudaStream_t s) {
  static size_t cached = 0;
  cudaError_t e = set_smem_once(k_states_tiny<NN, PP, MIXED>, smem, cached);
  if (e != cudaSuccess) return e;
  const long long blocks = (a.K + TINY_THREADS - 1) / TINY_THREADS;
  k_states_tiny<NN, PP, MIXED><<<int(blocks), TINY_THREADS, smem, s>>>(a, use_tab);
  return cudaGetLastError();
}

template <int NN, int PP>
cudaError_t tiny_prec(const StatesArgs& a, int use_tab, size_t smem, cudaStream_t s) {
  return a.mixed ? tiny_launch<NN, PP, true>(a, use_tab, smem, s)
                 : tiny_launch<NN, PP, false>(a, use_tab, smem, s);
}

}  // namespace

// Few-band path: n in {2, 4}, at most TINY_R_MAX distinct translations.  Sets
// *handled = false (and launches nothing) when the problem is outside it.
cudaError_t launch_states_tiny(const StatesArgs& a, int p_out, cudaStream_t s, bool* handled) {
  *handled = false;
  const int n = a.model.n, p = a.p;
  if (!(n == 2 || n == 4) || p < 1 || p > n || a.model.n_R > TINY_R_MAX || a.K <= 0) return cudaSuccess;
  if (a.op.nnz > 0 && (p % 2 || p_out != p / 2)) return cudaSuccess;
  const int N = a.plane.N, Nt = a.plane.N_t;
  bool integer_plane = a.f == nullptr;
  for (int d = 0; d < 3; ++d)
    integer_plane = integer_plane && a.plane.trans_dir[d] == double((long long)a.plane.trans_dir[d]);
  const bool use_tab = integer_plane && (size_t(N) + Nt) <= 8192;
  size_t smem = size_t(a.model.n_R) * TINY_THREADS * sizeof(z64);
  if (use_tab) smem += (size_t(N) + Nt + a.model.n_R) * sizeof(z64) + 2 * a.model.n_R * sizeof(int);
  *handled = true;
  if (n == 2) {
    return p == 1 ? tiny_prec<2, 1>(a, use_tab, smem, s) : tiny_prec<2, 2>(a, use_tab, smem, s);
  }
  switch (p) {
    case 1: return tiny_prec<4, 1>(a, use_tab, smem, s);
    case 2: return tiny_prec<4, 2>(a, use_tab, smem, s);
    case 3: return tiny_prec<4, 3>(a, use_tab, smem, s);
    default: return tiny_prec<4, 4>(a, use_tab, smem, s);
  }
}

}  // namespace bw
