// Four lanes per k-point for four-band models: lane l of a group of four
// consecutive lanes holds row l of H(k) and of the eigenvector matrix.  Shared by
// the states kernels (tiny.cu) and the fused mixed-precision loop kernel (loops.cu).
//
// A Jacobi sweep is three rounds; round R rotates the disjoint pairs {l, l ^ R} at
// once, the two lanes of a pair compute the same rotation, partner rows travel by
// warp shuffles, and every lane applies both rotations of the round to the columns
// of its own rows.  The mixed-precision solve (quad_df_occupied) runs the sweeps in
// FP32 on a double-float Hamiltonian and refines the occupied pair to double-float
// accuracy.
#pragma once

#include "common.cuh"
#include "df32.cuh"

namespace bw {

template <typename T>
__device__ __forceinline__ T teps();
template <>
__device__ __forceinline__ double teps<double>() { return 2.220446049250313e-16; }
template <>
__device__ __forceinline__ float teps<float>() { return 1.1920929e-7f; }

__device__ __forceinline__ int pmod(long long x, int m) {
  long long r = x % m;
  return int(r < 0 ? r + m : r);
}

struct TabShape {
  int B, H;  // low-level entries (w^0 .. w^{B-1}), high-level entries (w^{0}, w^{B}, ...)
};

template <typename T>
__device__ __forceinline__ cx<T> shfl_z(cx<T> v, int src) {
  return cx<T>(__shfl_sync(0xffffffffu, v.re, src), __shfl_sync(0xffffffffu, v.im, src));
}

// x[i] for a runtime i in [0, 4) without dynamic register indexing.
template <typename E>
__device__ __forceinline__ E sel4(const E (&x)[4], int i) {
  E r = x[0];
  if (i == 1) r = x[1];
  if (i == 2) r = x[2];
  if (i == 3) r = x[3];
  return r;
}

// Rotation of the Hermitian 2 x 2 block (a, b; conj b, d): c, s e^{i phi} and t as in
// the one-thread solver; false when the off-diagonal entry is negligible.
template <typename T>
__device__ __forceinline__ bool quad_angle(T a, T d, cx<T> b, T& c, cx<T>& sc, T& t, T& ab) {
  ab = sqrt(abs2(b));
  if (!(ab > T(4) * teps<T>() * sqrt(fabs(a) * fabs(d)) && ab > T(0))) return false;
  const T tau = (d - a) / (T(2) * ab);
  t = (tau >= T(0) ? T(1) : T(-1)) / (fabs(tau) + sqrt(T(1) + tau * tau));
  c = T(1) / sqrt(T(1) + t * t);
  const T s = t * c / ab;
  sc = cx<T>(s * b.re, s * b.im);
  return true;
}

// FP32 rotation from hardware reciprocal square roots and reciprocals (about 2 ulp):
// the FP32 sweeps only seed the double-float refinement, whose result does not
// depend on the last bits of the rotations.  The skip test compares squares.
template <>
__device__ __forceinline__ bool quad_angle<float>(float a, float d, c32 b, float& c, c32& sc, float& t,
                                                  float& ab) {
  const float b2 = abs2(b);
  const float e4 = 4.f * teps<float>();
  if (!(b2 > e4 * e4 * fabsf(a) * fabsf(d) && b2 > 0.f)) {
    ab = 0.f;
    return false;
  }
  const float inv_ab = rsqrtf(b2);
  ab = b2 * inv_ab;
  const float tau = 0.5f * (d - a) * inv_ab;
  t = copysignf(__frcp_rn(fabsf(tau) + sqrtf(fmaf(tau, tau, 1.f))), tau);
  if (tau == 0.f) t = 1.f;
  c = rsqrtf(fmaf(t, t, 1.f));
  const float s = t * c * inv_ab;
  sc = c32(s * b.re, s * b.im);
  return true;
}

template <int R, typename T>
__device__ __forceinline__ bool quad_round(cx<T> (&Ar)[4], cx<T> (&Vr)[4], int l, int base,
                                           bool frozen) {
  constexpr int Q = R == 1 ? 2 : 1;          // a lane of the other pair is l ^ Q
  constexpr int A0 = 0, A1 = R;              // pair containing index 0
  constexpr int B0 = R == 1 ? 2 : 1, B1 = R == 3 ? 2 : 3;  // the other pair
  const int partner = l ^ R;
  const bool is_p = l < partner;
  const T own_d = sel4(Ar, l).re;
  const T par_d = __shfl_sync(0xffffffffu, own_d, base + partner);
  const cx<T> bo = sel4(Ar, partner);
  const cx<T> b = is_p ? bo : conj(bo);      // A[p][q] from either row (exact Hermitian storage)
  const T a = is_p ? own_d : par_d, d = is_p ? par_d : own_d;
  T c = T(1), t = T(0), ab = T(0);
  cx<T> sc(T(0), T(0));
  const bool rot = !frozen && quad_angle(a, d, b, c, sc, t, ab);
  // rows: own row with the partner's
  cx<T> other[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) other[k] = shfl_z(Ar[k], base + partner);
  if (rot) {
    const cx<T> beta = is_p ? cx<T>(-sc.re, -sc.im) : conj(sc);
#pragma unroll
    for (int k = 0; k < 4; ++k) Ar[k] = c * Ar[k] + beta * other[k];
  }
  // columns: both rotations of the round on the own row of A and of V
  const T c2 = __shfl_sync(0xffffffffu, c, base + (l ^ Q));
  const cx<T> sc2 = shfl_z(sc, base + (l ^ Q));
  const bool mine_a = (l == A0 || l == A1);
  const T cA = mine_a ? c : c2, cB = mine_a ? c2 : c;
  const cx<T> sA = mine_a ? sc : sc2, sB = mine_a ? sc2 : sc;
  {
    const cx<T> ap = Ar[A0], aq = Ar[A1];
    Ar[A0] = cA * ap - aq * conj(sA);
    Ar[A1] = ap * sA + cA * aq;
    const cx<T> vp = Vr[A0], vq = Vr[A1];
    Vr[A0] = cA * vp - vq * conj(sA);
    Vr[A1] = vp * sA + cA * vq;
  }
  {
    const cx<T> ap = Ar[B0], aq = Ar[B1];
    Ar[B0] = cB * ap - aq * conj(sB);
    Ar[B1] = ap * sB + cB * aq;
    const cx<T> vp = Vr[B0], vq = Vr[B1];
    Vr[B0] = cB * vp - vq * conj(sB);
    Vr[B1] = vp * sB + cB * vq;
  }
  if (rot) {  // the annihilated entry and the new diagonal, as in the one-thread solver
    const cx<T> dnew(is_p ? a - t * ab : d + t * ab, T(0));
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (k == partner) Ar[k] = cx<T>(T(0), T(0));
      if (k == l) Ar[k] = dnew;
    }
  }
  return rot;
}

// Parallel-ordered Jacobi on the group's 4 x 4 matrix (lane l holds row l of A and
// of V, V starting as the identity).  Returns the sweeps used, or -1 without
// convergence within max_sweeps.  The warp's groups sweep together (the rounds
// shuffle across the whole warp): a converged group is frozen, its rotations the
// identity, until every group of the warp has converged.
template <typename T>
__device__ __forceinline__ int quad_jacobi(cx<T> (&Ar)[4], cx<T> (&Vr)[4], int l, int base,
                                           int max_sweeps) {
#pragma unroll
  for (int c = 0; c < 4; ++c) Vr[c] = cx<T>(T(c == l), T(0));
  T fro = T(0);
#pragma unroll
  for (int c = 0; c < 4; ++c) fro += abs2(Ar[c]);
  fro += __shfl_xor_sync(0xffffffffu, fro, 1);
  fro += __shfl_xor_sync(0xffffffffu, fro, 2);
  const T eps = teps<T>();
  const T tol2 = T(64) * eps * eps * fro;
  int done = -1;
  for (int sweep = 0; sweep <= max_sweeps; ++sweep) {
    T off = T(0);
#pragma unroll
    for (int c = 0; c < 4; ++c)
      if (c != l) off += abs2(Ar[c]);
    off += __shfl_xor_sync(0xffffffffu, off, 1);
    off += __shfl_xor_sync(0xffffffffu, off, 2);
    if (done < 0 && (off <= tol2 || fro == T(0))) done = sweep;
    if (__all_sync(0xffffffffu, done >= 0) || sweep == max_sweeps) break;
    const bool frozen = done >= 0;
    int rot = quad_round<1>(Ar, Vr, l, base, frozen);
    rot |= quad_round<2>(Ar, Vr, l, base, frozen);
    rot |= quad_round<3>(Ar, Vr, l, base, frozen);
    rot |= __shfl_xor_sync(0xffffffffu, rot, 1);
    rot |= __shfl_xor_sync(0xffffffffu, rot, 2);
    if (done < 0 && !rot) done = sweep + 1;
  }
  return done;
}

// Ascending order (stable) of the group's diagonal: lam[c] = A[c][c], ord[c] = the
// index of the c-th smallest.
template <typename T>
__device__ __forceinline__ void quad_order(const cx<T> (&Ar)[4], int l, int base, T (&lam)[4],
                                           int (&ord)[4]) {
  const T own = sel4(Ar, l).re;
#pragma unroll
  for (int c = 0; c < 4; ++c) lam[c] = __shfl_sync(0xffffffffu, own, base + c);
#pragma unroll
  for (int x = 0; x < 4; ++x) {
    int rk = 0;
#pragma unroll
    for (int y = 0; y < 4; ++y) rk += (lam[y] < lam[x]) || (lam[y] == lam[x] && y < x);
#pragma unroll
    for (int c = 0; c < 4; ++c)
      if (rk == c) ord[c] = x;
  }
}

__host__ __device__ inline TabShape tab_shape_split(int M) {
  int B = 1;
  while (B * B < M) ++B;
  return {B, (M + B - 1) / B};
}

__device__ inline void fill_tab_df(cdf* lo, cdf* hi, int M, TabShape t) {
  for (int m = threadIdx.x; m < t.B + t.H; m += blockDim.x) {
    const long long e = m < t.B ? m : (long long)(m - t.B) * t.B;
    double sn, cs;
    sincospi(2.0 * double(e) / double(M), &sn, &cs);
    *(m < t.B ? lo + m : hi + (m - t.B)) = cdf_from(z64(cs, sn));
  }
}

__device__ __forceinline__ cdf tab_at_df(const cdf* lo, const cdf* hi, TabShape t, int m) {
  return hi[m / t.B] * lo[m % t.B];
}

// Re(conj(x) y) with x exact in float, y double-float.
__device__ __forceinline__ df re_conj_dot(c32 x, cdf y) { return df_fma(df(x.re), y.re, x.im * y.im); }

__device__ __forceinline__ df group_sum_df(df v) {
  v = v + shfl_xor_df(v, 1);
  return v + shfl_xor_df(v, 2);
}

__device__ __forceinline__ c32 group_sum_c32(c32 v) {
  v.re += __shfl_xor_sync(0xffffffffu, v.re, 1);
  v.im += __shfl_xor_sync(0xffffffffu, v.im, 1);
  v.re += __shfl_xor_sync(0xffffffffu, v.re, 2);
  v.im += __shfl_xor_sync(0xffffffffu, v.im, 2);
  return v;
}

// The refinement below is written with rolled loops and register selects rather
// than unrolled code: it runs once per k-point on few warps per SM, where a long
// straight-line body stalls on instruction fetch.

// (H x)[l] for a double-float vector x held one entry per lane (x[q] in lane q).
__device__ __forceinline__ cdf quad_matvec(const cdf (&Hr)[4], cdf x, int base) {
  cdf acc = cdf_zero();
#pragma unroll 1
  for (int q = 0; q < 4; ++q) cfma(acc, sel4(Hr, q), shfl_cdf(x, base + q));
  return acc;
}

// First-order Lowdin step X <- X - X (X^dag X - I) / 2 for two vectors of the group,
// the Gram matrix in double-float (its deviation E from I is ~1e-7, so the
// correction X E / 2 itself is computed in FP32).
__device__ __forceinline__ void lowdin2(cdf& X0, cdf& X1) {
  float e00 = 0.f, e11 = 0.f;
  c32 e01(0.f, 0.f);
#pragma unroll 1
  for (int t = 0; t < 3; ++t) {  // (0, 0), (0, 1), (1, 1)
    const cdf xa = t == 2 ? X1 : X0, xb = t == 0 ? X0 : X1;
    cdf g = cdf_zero();
    cfma_conj(g, xa, xb);
    const df gre = group_sum_df(g.re) - df(t == 1 ? 0.f : 1.f), gim = group_sum_df(g.im);
    if (t == 0) e00 = gre.hi;
    if (t == 1) e01 = c32(gre.hi, gim.hi);
    if (t == 2) e11 = gre.hi;
  }
  const c32 x0(X0.re.hi, X0.im.hi), x1(X1.re.hi, X1.im.hi);
  const c32 c0 = c32(x0.re * e00, x0.im * e00) + x1 * conj(e01);
  const c32 c1 = x0 * e01 + c32(x1.re * e11, x1.im * e11);
  X0 = cdf(X0.re + df(-0.5f * c0.re), X0.im + df(-0.5f * c0.im));
  X1 = cdf(X1.re + df(-0.5f * c1.re), X1.im + df(-0.5f * c1.im));
}

// Eigenvalues lo <= hi of the 2 x 2 Hermitian Ritz matrix X^dag H X of two
// orthonormal vectors: (a + d) / 2 -+ sqrt(((a - d) / 2)^2 + |b|^2), in double-float.
__device__ __forceinline__ void ritz2(const cdf (&Hr)[4], cdf X0, cdf X1, int base, df& lo,
                                      df& hi) {
  cdf h0 = cdf_zero(), h1 = cdf_zero();
#pragma unroll 1
  for (int t = 0; t < 2; ++t) {
    const cdf h = quad_matvec(Hr, t ? X1 : X0, base);
    if (t == 0) h0 = h;
    if (t == 1) h1 = h;
  }
  df aa(0.f), dd(0.f), bre(0.f), bim(0.f);
#pragma unroll 1
  for (int t = 0; t < 3; ++t) {  // X0^dag h0, X1^dag h1, X0^dag h1
    cdf g = cdf_zero();
    cfma_conj(g, t == 1 ? X1 : X0, t == 0 ? h0 : h1);
    const df gre = group_sum_df(g.re);
    if (t == 0) aa = gre;
    if (t == 1) dd = gre;
    if (t == 2) {
      bre = gre;
      bim = group_sum_df(g.im);
    }
  }
  const df mean = df(0.5f) * (aa + dd), half = df(0.5f) * (aa - dd);
  const df r = df_sqrt(df_fma(half, half, df_fma(bre, bre, bim * bim)));
  lo = mean - r;
  hi = mean + r;
}

// Occupied pair of a four-band H(k) given as double-float rows (lane l holds row
// l): FP32 Jacobi on the float part of H, made exactly Hermitian; one Newton
// correction of the two lowest FP32 vectors q_c in the FP32 eigenbasis with the
// residual R = H q_c - q_c rho_c in double-float (q_c += z_a (z_a^dag R_c) /
// (rho_c - lam_a) over the unoccupied z_a); one first-order Lowdin step; the gap
// from the double-float Ritz values of the refined occupied pair and of the
// re-orthonormalised unoccupied pair (accurate whatever the splitting inside each
// pair).  Every lane of the warp must call it (warp shuffles).  Returns the Jacobi
// sweeps used (-1: no convergence); Q0, Q1 are row l of the occupied vectors.
__device__ __forceinline__ int quad_df_occupied(const cdf (&Hr)[4], int l, int base, int max_sweeps,
                                                cdf& Q0, cdf& Q1, double& gap) {
  c32 Ar[4], Vr[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) Ar[c] = c32(Hr[c].re.hi, c == l ? 0.f : Hr[c].im.hi);
#pragma unroll
  for (int cc = 0; cc < 4; ++cc) {
    const c32 v(Hr[cc].re.hi, Hr[cc].im.hi);  // own row, column cc
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const c32 t = shfl_z(v, base + c);     // A[c][cc] from lane c
      if (cc == l && c < l) Ar[c] = conj(t);
    }
  }
  const int sweeps = quad_jacobi(Ar, Vr, l, base, max_sweeps);
  float lam[4];
  int ord[4];
  quad_order(Ar, l, base, lam, ord);
  Q0 = Q1 = cdf_zero();
#pragma unroll 1
  for (int c = 0; c < 2; ++c) {
    const c32 q = sel4(Vr, ord[c]);
    const cdf hq = quad_matvec(Hr, cdf_from(q), base);
    const df rho = group_sum_df(re_conj_dot(q, hq));
    const cdf R(hq.re - q.re * rho, hq.im - q.im * rho);
    const c32 r32(R.re.hi, R.im.hi);
    c32 upd(0.f, 0.f);
#pragma unroll 1
    for (int aa = 2; aa < 4; ++aa) {
      const c32 z = sel4(Vr, ord[aa]);
      const c32 d = group_sum_c32(conj(z) * r32);
      const float den = rho.hi - sel4(lam, ord[aa]);
      const c32 coef = den != 0.f ? c32(d.re / den, d.im / den) : c32(0.f, 0.f);
      upd = upd + z * coef;
    }
    const cdf qn(df_two_sum(q.re, upd.re), df_two_sum(q.im, upd.im));
    if (c == 0) Q0 = qn;
    if (c == 1) Q1 = qn;
  }
  const cdf Z0 = cdf_from(sel4(Vr, ord[2])), Z1 = cdf_from(sel4(Vr, ord[3]));
  df occ_hi(0.f), un_lo(0.f);
#pragma unroll 1
  for (int t = 0; t < 2; ++t) {  // the occupied pair, then the unoccupied one
    cdf X0 = t ? Z0 : Q0, X1 = t ? Z1 : Q1;
    lowdin2(X0, X1);
    df lo, hi;
    ritz2(Hr, X0, X1, base, lo, hi);
    if (t == 0) {
      Q0 = X0;
      Q1 = X1;
      occ_hi = hi;
    } else {
      un_lo = lo;
    }
  }
  gap = df_to_double(un_lo - occ_hi);
  return sweeps;
}

}  // namespace bw
