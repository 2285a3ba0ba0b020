// One thread per k-point for few-band models (n = 2 or 4): Bloch Hamiltonian,
// exact diagonalisation in FP64 and projected-spin sector, all in registers
// (Sec. I "exact diagonalization", Eq. 1, Sec. IV).
//
// GB300's FP64 pipe serves a whole warp instruction at a time, so a kernel that
// gives one small matrix to a CTA pays for 32 lanes and uses a few.  Here every
// lane owns its own k-point: the matrix sizes are compile-time constants, loops
// unroll, and the arrays stay in registers.  The Bloch phases come from per-CTA
// tables: with an integer loop direction and an integer transverse direction,
// f(j, i).R = origin.R + j (loop.R) / N + i (trans.R) / N_t, so
// exp(i 2pi f.R) = exp(i 2pi origin.R) w_N^{(j loop.R) mod N} w_Nt^{(i trans.R) mod N_t}
// with w_M = exp(i 2pi / M) tabulated once per CTA (in two levels for long grids).
#include <float.h>

#include "launch.h"
#include "quad.cuh"

namespace bw {
namespace {

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

constexpr int TINY_THREADS = 32;
// Above this many points a direction's phase table is split in two levels
// (w^m = w^{B (m / B)} w^{m mod B}, B ~ sqrt(M)), so that long grids keep the
// shared memory per CTA small.
constexpr int TAB_SPLIT = 512;

__host__ __device__ inline TabShape tab_shape(int M) {
  if (M <= TAB_SPLIT) return {M, 0};
  int B = 1;
  while (B * B < M) ++B;
  return {B, (M + B - 1) / B};
}

// Fills lo[0..B) and hi[0..H) with exp(i 2pi m / M).
__device__ void fill_tab(z64* lo, z64* hi, int M, TabShape t) {
  for (int m = threadIdx.x; m < t.B + t.H; m += blockDim.x) {
    const long long e = m < t.B ? m : (long long)(m - t.B) * t.B;
    double sn, cs;
    sincospi(2.0 * double(e) / double(M), &sn, &cs);
    *(m < t.B ? lo + m : hi + (m - t.B)) = z64(cs, sn);
  }
}

__device__ __forceinline__ z64 tab_at(const z64* lo, const z64* hi, TabShape t, int m) {
  if (t.H == 0) return lo[m];
  return hi[m / t.B] * lo[m % t.B];
}

template <int NN, int PP>
__global__ void __launch_bounds__(TINY_THREADS)
k_states_tiny(StatesArgs a, int use_tab) {
  extern __shared__ __align__(16) unsigned char smem[];
  const DevModel& md = a.model;
  const int tid = threadIdx.x, bd = blockDim.x, nR = md.n_R;
  const int N = a.plane.N, Nt = a.plane.N_t;
  const TabShape tN = tab_shape(N), tT = tab_shape(Nt);
  z64* cache = reinterpret_cast<z64*>(smem);             // nR x bd
  z64* tabN = cache + nR * bd;                             // tN.B + tN.H
  z64* tabNt = tabN + (use_tab ? tN.B + tN.H : 0);         // tT.B + tT.H
  z64* oph = tabNt + (use_tab ? tT.B + tT.H : 0);          // nR
  int* lR = reinterpret_cast<int*>(oph + (use_tab ? nR : 0));
  int* tR = lR + (use_tab ? nR : 0);
  int* sR = tR + (use_tab ? nR : 0);
  if (use_tab) {
    fill_tab(tabN, tabN + tN.B, N, tN);
    fill_tab(tabNt, tabNt + tT.B, Nt, tT);
    for (int r = tid; r < nR; r += bd) {
      const int* R = md.Rv + 3 * r;
      double x = 0.0;
      int l = 0, t = 0, sw = 0;
      for (int d = 0; d < 3; ++d) {
        x += a.plane.origin[d] * double(R[d]);
        l += int(a.plane.loop_dir[d]) * R[d];
        t += int(a.plane.trans_dir[d]) * R[d];
        sw += a.plane.sweep[d] * R[d];
      }
      double sn, cs;
      sincospi(2.0 * x, &sn, &cs);
      oph[r] = z64(cs, sn);
      lR[r] = l;
      tR[r] = t;
      sR[r] = sw;
    }
    __syncthreads();
  }
  const long long k = (long long)blockIdx.x * bd + tid;
  if (k >= a.K) return;
  const int i = int(k / N), j = int(k - (long long)i * N);
  // Bloch phases of the distinct translations at this k-point
  if (use_tab) {
    for (int r = 0; r < nR; ++r) {
      const int mN = pmod((long long)j * lR[r], N), mT = pmod(plane_row_index(a.plane, i, tR[r], sR[r]), Nt);
      cache[r * bd + tid] = oph[r] * tab_at(tabN, tabN + tN.B, tN, mN) * tab_at(tabNt, tabNt + tT.B, tT, mT);
    }
  } else {
    double f[3];
    if (a.f) {
      f[0] = a.f[3 * k]; f[1] = a.f[3 * k + 1]; f[2] = a.f[3 * k + 2];
    } else {
      plane_f(a.plane, i, j, f);
    }
    for (int r = 0; r < nR; ++r) cache[r * bd + tid] = bloch_phase(f, md.Rv + 3 * r);
  }
  z64 Q[NN][PP];
  double gap = INFINITY;
  bool ok = true;
  {
    // H(k) in FP64.  The mixed-precision request takes this FP64 solve as well: at
    // n <= 4 one thread's FP64 Jacobi costs no more than an FP32 solve plus the
    // FP64-grade refinement of its occupied block (measured), at full accuracy.
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
      if (a.pso_median) {
        neg = PP / 2;
        g = mu[PP / 2] - mu[PP / 2 - 1];
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

// ---------------------------------------------------------------------------
// Four lanes per k-point (n = 4, no spin split): lane l of a group of four
// consecutive lanes holds row l of H(k) and of the eigenvector matrix V.  A Jacobi
// sweep is three rounds; round R rotates the disjoint pairs {l, l ^ R} at once, the
// two lanes of a pair compute the same rotation (the stored matrix stays exactly
// Hermitian), partner rows travel by warp shuffles, and every lane applies both
// rotations of the round to the columns of its own rows.  Per lane this is about
// half the FP64 instructions of the one-thread version, which is what bounds the
// latency of a small grid (every FP64 warp instruction costs the same whatever
// the number of active lanes).
// ---------------------------------------------------------------------------
constexpr int QUAD_THREADS = 128;  // 32 k-points per CTA

template <int PP>
__global__ void __launch_bounds__(QUAD_THREADS) k_states_quad(StatesArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const DevModel& md = a.model;
  const int tid = threadIdx.x, nR = md.n_R;
  const int N = a.plane.N, Nt = a.plane.N_t;
  const TabShape tN = tab_shape(N), tT = tab_shape(Nt);
  constexpr int KPB = QUAD_THREADS / 4;
  z64* cache = reinterpret_cast<z64*>(smem);   // nR x KPB
  z64* tabN = cache + nR * KPB;
  z64* tabNt = tabN + tN.B + tN.H;
  z64* oph = tabNt + tT.B + tT.H;
  int* lR = reinterpret_cast<int*>(oph + nR);
  int* tR = lR + nR;
  int* sR = tR + nR;
  fill_tab(tabN, tabN + tN.B, N, tN);
  fill_tab(tabNt, tabNt + tT.B, Nt, tT);
  for (int r = tid; r < nR; r += blockDim.x) {
    const int* Rv = md.Rv + 3 * r;
    double x = 0.0;
    int lq = 0, tq = 0, sq = 0;
    for (int dd = 0; dd < 3; ++dd) {
      x += a.plane.origin[dd] * double(Rv[dd]);
      lq += int(a.plane.loop_dir[dd]) * Rv[dd];
      tq += int(a.plane.trans_dir[dd]) * Rv[dd];
      sq += a.plane.sweep[dd] * Rv[dd];
    }
    double sn, cs;
    sincospi(2.0 * x, &sn, &cs);
    oph[r] = z64(cs, sn);
    lR[r] = lq;
    tR[r] = tq;
    sR[r] = sq;
  }
  __syncthreads();
  const int l = tid & 3, kl = tid >> 2, base = (tid & 31) & ~3;
  const long long kraw = (long long)blockIdx.x * KPB + kl;
  const bool active = kraw < a.K;
  const long long k = active ? kraw : a.K - 1;  // idle groups recompute the last k-point
  const int i = int(k / N), j = int(k - (long long)i * N);
  for (int r = l; r < nR; r += 4) {
    const int mN = pmod((long long)j * lR[r], N), mT = pmod(plane_row_index(a.plane, i, tR[r], sR[r]), Nt);
    cache[r * KPB + kl] = oph[r] * tab_at(tabN, tabN + tN.B, tN, mN) * tab_at(tabNt, tabNt + tT.B, tT, mT);
  }
  __syncwarp();
  // row l of H(k)
  z64 Ar[4], Vr[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    Ar[c] = z64(0.0, 0.0);
    Vr[c] = z64(double(c == l), 0.0);
  }
  for (int e = a.row_ptr[l]; e < a.row_ptr[l + 1]; ++e) {
    z64 acc(0.0, 0.0);
    for (int h = md.ent_start[e]; h < md.ent_start[e + 1]; ++h)
      cfma(acc, md.hop_t[h], cache[md.hop_r[h] * KPB + kl]);
    const int col = md.ent_col[e];
#pragma unroll
    for (int c = 0; c < 4; ++c)
      if (c == col) Ar[c] = acc;
  }
  const int sweeps = quad_jacobi(Ar, Vr, l, base, a.max_sweeps);
  // eigenvalues of the group, ascending (stable)
  const double own = sel4(Ar, l).re;
  double lam[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) lam[c] = __shfl_sync(0xffffffffu, own, base + c);
  int ord[4];
#pragma unroll
  for (int x = 0; x < 4; ++x) {
    int rk = 0;
#pragma unroll
    for (int y = 0; y < 4; ++y) rk += (lam[y] < lam[x]) || (lam[y] == lam[x] && y < x);
#pragma unroll
    for (int c = 0; c < 4; ++c)
      if (rk == c) ord[c] = x;
  }
  if (!active) return;
  z64* out = a.U + k * 4LL * PP + l * PP;
#pragma unroll
  for (int c = 0; c < PP; ++c) out[c] = sel4(Vr, ord[c]);
  if (l == 0) {
    double gap = INFINITY;
    if (PP < 4) {
      double lp = lam[0], lm = lam[0];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        if (c == PP) lp = lam[ord[c]];
        if (c == PP - 1) lm = lam[ord[c]];
      }
      gap = lp - lm;
    }
    a.gap[k] = gap;
    if (sweeps < 0) report(a.status, ST_ENOCONV, k, 0.0);
    if (!(gap > a.gap_tol)) report(a.status, ST_EGAP, k, gap);
  }
}

// ---------------------------------------------------------------------------
// Mixed precision, four lanes per k-point (n = 4, p = 2, no spin split), with every step on
// the FP32 pipe: GB300 issues FP32 about 70x faster than FP64, and at small grids
// the FP64 kernel above is bound by its FP64 instruction count.
//  - Bloch phases and H(k) in double-float (two-level phase tables, exact products
//    of the double-float hopping amplitudes with the phases);
//  - FP32 Jacobi on the float part of H, made exactly Hermitian;
//  - one Newton correction of the occupied block Q in the FP32 eigenbasis, with the
//    residual R = H Q - Q rho in double-float: for each unoccupied FP32 vector z_a,
//    Q_c += z_a (z_a^dag R_c) / (rho_c - lam_a), rho_c = q_c^dag H q_c;
//  - one first-order Lowdin step Q <- Q - Q (Q^dag Q - I) / 2 with the Gram matrix
//    in double-float;
//  - the gap from double-float Ritz values of the refined occupied pair and of the
//    re-orthonormalised unoccupied pair (errors quadratic in the subspace errors,
//    whatever the splitting inside each pair).
// The occupied block leaves as complex double-float (hi, lo per part, 16 bytes like
// a complex128), accurate to about 1e-13, for the double-float loop kernels.
// ---------------------------------------------------------------------------
size_t quad_df_smem(int nR, int N, int Nt) {
  const TabShape tN = tab_shape_split(N), tT = tab_shape_split(Nt);
  return (size_t(nR) * (QUAD_THREADS / 4) + tN.B + tN.H + tT.B + tT.H + nR) * sizeof(cdf) +
         3 * size_t(nR) * sizeof(int);
}

template <int PP>
__global__ void __launch_bounds__(QUAD_THREADS) k_states_quad_df(StatesArgs a) {
  static_assert(PP == 2, "the double-float four-lane kernel serves two occupied bands");
  extern __shared__ __align__(16) unsigned char smem[];
  const DevModel& md = a.model;
  const int tid = threadIdx.x, nR = md.n_R;
  const int N = a.plane.N, Nt = a.plane.N_t;
  const TabShape tN = tab_shape_split(N), tT = tab_shape_split(Nt);
  constexpr int KPB = QUAD_THREADS / 4;
  cdf* cache = reinterpret_cast<cdf*>(smem);   // nR x KPB
  cdf* tabN = cache + nR * KPB;
  cdf* tabNt = tabN + tN.B + tN.H;
  cdf* oph = tabNt + tT.B + tT.H;
  int* lR = reinterpret_cast<int*>(oph + nR);
  int* tR = lR + nR;
  int* sR = tR + nR;
  fill_tab_df(tabN, tabN + tN.B, N, tN);
  fill_tab_df(tabNt, tabNt + tT.B, Nt, tT);
  for (int r = tid; r < nR; r += blockDim.x) {
    const int* Rv = md.Rv + 3 * r;
    double x = 0.0;
    int lq = 0, tq = 0, sq = 0;
    for (int dd = 0; dd < 3; ++dd) {
      x += a.plane.origin[dd] * double(Rv[dd]);
      lq += int(a.plane.loop_dir[dd]) * Rv[dd];
      tq += int(a.plane.trans_dir[dd]) * Rv[dd];
      sq += a.plane.sweep[dd] * Rv[dd];
    }
    double sn, cs;
    sincospi(2.0 * x, &sn, &cs);
    oph[r] = cdf_from(z64(cs, sn));
    lR[r] = lq;
    tR[r] = tq;
    sR[r] = sq;
  }
  __syncthreads();
  const int l = tid & 3, kl = tid >> 2, base = (tid & 31) & ~3;
  const long long kraw = (long long)blockIdx.x * KPB + kl;
  const bool active = kraw < a.K;
  const long long k = active ? kraw : a.K - 1;  // idle groups recompute the last k-point
  const int i = int(k / N), j = int(k - (long long)i * N);
  for (int r = l; r < nR; r += 4) {
    const int mN = pmod((long long)j * lR[r], N), mT = pmod(plane_row_index(a.plane, i, tR[r], sR[r]), Nt);
    cache[r * KPB + kl] = oph[r] * tab_at_df(tabN, tabN + tN.B, tN, mN) *
                          tab_at_df(tabNt, tabNt + tT.B, tT, mT);
  }
  __syncwarp();
  // row l of H(k) in double-float
  cdf Hr[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) Hr[c] = cdf_zero();
  for (int e = a.row_ptr[l]; e < a.row_ptr[l + 1]; ++e) {
    cdf acc = cdf_zero();
    for (int h = md.ent_start[e]; h < md.ent_start[e + 1]; ++h) {
      const float* t4 = md.hop_tdf + 4 * h;
      cfma(acc, cdf(df(t4[0], t4[1]), df(t4[2], t4[3])), cache[md.hop_r[h] * KPB + kl]);
    }
    const int col = md.ent_col[e];
#pragma unroll
    for (int c = 0; c < 4; ++c)
      if (c == col) Hr[c] = acc;
  }
  cdf Qf[PP];
  double gap;
  const int sweeps = quad_df_occupied(Hr, l, base, a.max_sweeps, Qf[0], Qf[1], gap);
  if (!active) return;
  cdf* out = reinterpret_cast<cdf*>(a.U) + k * 4LL * PP + l * PP;
#pragma unroll
  for (int c = 0; c < PP; ++c) out[c] = Qf[c];
  if (l == 0) {
    a.gap[k] = gap;
    if (sweeps < 0) report(a.status, ST_ENOCONV, k, 0.0);
    if (!(gap > a.gap_tol)) report(a.status, ST_EGAP, k, gap);
  }
}

template <int PP>
cudaError_t quad_df_launch(const StatesArgs& a, size_t smem, cudaStream_t s) {
  static size_t cached = 0;
  cudaError_t e = set_smem_once(k_states_quad_df<PP>, smem, cached);
  if (e != cudaSuccess) return e;
  const long long blocks = (a.K + QUAD_THREADS / 4 - 1) / (QUAD_THREADS / 4);
  k_states_quad_df<PP><<<int(blocks), QUAD_THREADS, smem, s>>>(a);
  return cudaGetLastError();
}

template <int PP>
cudaError_t quad_launch(const StatesArgs& a, size_t smem, cudaStream_t s) {
  static size_t cached = 0;
  cudaError_t e = set_smem_once(k_states_quad<PP>, smem, cached);
  if (e != cudaSuccess) return e;
  const long long blocks = (a.K + QUAD_THREADS / 4 - 1) / (QUAD_THREADS / 4);
  k_states_quad<PP><<<int(blocks), QUAD_THREADS, smem, s>>>(a);
  return cudaGetLastError();
}

template <int NN, int PP>
cudaError_t tiny_prec(const StatesArgs& a, int use_tab, size_t smem, cudaStream_t s) {
  static size_t cached = 0;
  cudaError_t e = set_smem_once(k_states_tiny<NN, PP>, smem, cached);
  if (e != cudaSuccess) return e;
  const long long blocks = (a.K + TINY_THREADS - 1) / TINY_THREADS;
  k_states_tiny<NN, PP><<<int(blocks), TINY_THREADS, smem, s>>>(a, use_tab);
  return cudaGetLastError();
}

}  // namespace

// The double-float four-lane kernel applies: mixed precision, n = 4, p = 2, no spin split,
// an integer plane (phase tables), at most TINY_R_MAX translations.
bool states_df_eligible(const StatesArgs& a, int p_out) {
  if (!a.mixed || a.f != nullptr || a.op.nnz > 0 || a.model.n != 4 || a.p != 2 ||
      p_out != a.p || a.model.n_R > TINY_R_MAX || a.K <= 0 || !a.row_ptr)
    return false;
  for (int d = 0; d < 3; ++d)
    if (a.plane.trans_dir[d] != double((long long)a.plane.trans_dir[d])) return false;
  return quad_df_smem(a.model.n_R, a.plane.N, a.plane.N_t) <= 48 * 1024;
}

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
  const TabShape tN = tab_shape(N), tT = tab_shape(Nt);
  const size_t tab = size_t(tN.B) + tN.H + tT.B + tT.H;
  const bool use_tab = integer_plane && tab <= 4096;
  size_t smem = size_t(a.model.n_R) * TINY_THREADS * sizeof(z64);
  if (use_tab) smem += (tab + a.model.n_R) * sizeof(z64) + 3 * a.model.n_R * sizeof(int);
  *handled = true;
  if (a.want_df)  // the caller checked states_df_eligible()
    return quad_df_launch<2>(a, quad_df_smem(a.model.n_R, N, Nt), s);
  // Small grids (under ~2 warps per SM partition with one thread per k-point) are
  // latency-bound: four lanes per k-point halve the FP64 instructions per lane.
  // Large grids are FP64-throughput-bound, where the one-thread kernel does less
  // total work.
  if (n == 4 && a.op.nnz == 0 && use_tab && a.row_ptr && a.K <= 8192) {
    const size_t qs = size_t(a.model.n_R) * (QUAD_THREADS / 4) * sizeof(z64) +
                      (tab + a.model.n_R) * sizeof(z64) + 3 * a.model.n_R * sizeof(int);
    switch (p) {
      case 1: return quad_launch<1>(a, qs, s);
      case 2: return quad_launch<2>(a, qs, s);
      case 3: return quad_launch<3>(a, qs, s);
      default: return quad_launch<4>(a, qs, s);
    }
  }
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
