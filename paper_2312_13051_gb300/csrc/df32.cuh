// Double-float arithmetic: a value is the unevaluated sum hi + lo of two floats with
// |lo| <= ulp(hi) / 2, about 48 significant bits (unit roundoff ~ 2^-47), computed
// on the FP32 pipe.  Built from error-free transformations: Knuth's TwoSum and
// Dekker's FastTwoSum for sums, the exact product a b = p + fma(a, b, -p) for
// products (Dekker 1971, "A floating-point technique for extending the available
// precision"), and one Newton correction of the float quotient / square root.
//
// GB300 runs FP32 about 70x faster than FP64; where the mixed path needs FP64-grade
// accuracy (the refinement residual) on data that fits the float exponent range,
// these operations take the FP32 pipe instead of the FP64 one.
#pragma once

#include "common.cuh"

namespace bw {

struct df {
  float hi, lo;
  __host__ __device__ df() = default;
  __host__ __device__ constexpr df(float h, float l = 0.f) : hi(h), lo(l) {}
};

// s + e = a + b exactly (any magnitudes).
__device__ __forceinline__ df df_two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  const float e = (a - (s - bb)) + (b - bb);
  return df(s, e);
}

// s + e = a + b exactly when |a| >= |b| (or a = 0).
__device__ __forceinline__ df df_fast_two_sum(float a, float b) {
  const float s = a + b;
  return df(s, b - (s - a));
}

__device__ __forceinline__ df df_from_double(double x) {
  const float h = float(x);
  return df(h, float(x - double(h)));
}

__device__ __forceinline__ double df_to_double(df x) { return double(x.hi) + double(x.lo); }

__device__ __forceinline__ df operator-(df a) { return df(-a.hi, -a.lo); }

// Accurate sum: both parts through TwoSum, then renormalised.
__device__ __forceinline__ df operator+(df a, df b) {
  df s = df_two_sum(a.hi, b.hi);
  const df t = df_two_sum(a.lo, b.lo);
  s.lo += t.hi;
  s = df_fast_two_sum(s.hi, s.lo);
  s.lo += t.lo;
  return df_fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ df operator-(df a, df b) { return a + (-b); }

__device__ __forceinline__ df operator*(df a, df b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
  return df_fast_two_sum(p, e);
}

__device__ __forceinline__ df operator*(float a, df b) {
  const float p = a * b.hi;
  float e = fmaf(a, b.hi, -p);
  e = fmaf(a, b.lo, e);
  return df_fast_two_sum(p, e);
}

// q = a / b: float quotient, corrected once from the double-float remainder.
__device__ __forceinline__ df df_div(df a, df b) {
  const float q0 = a.hi / b.hi;
  const df r = a - q0 * b;
  const float q1 = r.hi / b.hi;
  return df_fast_two_sum(q0, q1);
}

// sqrt(a), a >= 0: float root, corrected once (Newton step on s^2 = a).
__device__ __forceinline__ df df_sqrt(df a) {
  if (!(a.hi > 0.f)) return df(0.f, 0.f);
  const float s0 = sqrtf(a.hi);
  const float p = s0 * s0;
  const df r = a - df(p, fmaf(s0, s0, -p));  // a - s0^2, s0^2 exact
  const float s1 = r.hi / (2.f * s0);
  return df_fast_two_sum(s0, s1);
}

// Complex double-float.
struct cdf {
  df re, im;
  __host__ __device__ cdf() = default;
  __host__ __device__ constexpr cdf(df r, df i) : re(r), im(i) {}
};

__device__ __forceinline__ cdf cdf_from(z64 z) { return cdf(df_from_double(z.re), df_from_double(z.im)); }
__device__ __forceinline__ cdf cdf_from(c32 z) { return cdf(df(z.re), df(z.im)); }
__device__ __forceinline__ z64 cdf_to_z64(cdf z) { return z64(df_to_double(z.re), df_to_double(z.im)); }
__device__ __forceinline__ cdf conj(cdf a) { return cdf(a.re, -a.im); }
__device__ __forceinline__ cdf operator+(cdf a, cdf b) { return cdf(a.re + b.re, a.im + b.im); }
__device__ __forceinline__ cdf operator-(cdf a, cdf b) { return cdf(a.re - b.re, a.im - b.im); }
__device__ __forceinline__ cdf operator*(cdf a, cdf b) {
  return cdf(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
__device__ __forceinline__ cdf operator*(df s, cdf b) { return cdf(s * b.re, s * b.im); }
// |a|^2
__device__ __forceinline__ df abs2(cdf a) { return a.re * a.re + a.im * a.im; }

// a b + c: the product exactly (hi part) plus its first-order terms, one TwoSum with
// c and a final TwoSum; absolute error about 2^-46 (|a b| + |c|).
__device__ __forceinline__ df df_fma(df a, df b, df c) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
  const df s = df_two_sum(p, c.hi);
  return df_two_sum(s.hi, s.lo + (e + c.lo));
}

// acc += a b and acc += conj(a) b in double-float.
__device__ __forceinline__ void cfma(cdf& acc, cdf a, cdf b) {
  acc.re = df_fma(a.re, b.re, acc.re);
  acc.re = df_fma(-a.im, b.im, acc.re);
  acc.im = df_fma(a.re, b.im, acc.im);
  acc.im = df_fma(a.im, b.re, acc.im);
}

__device__ __forceinline__ void cfma_conj(cdf& acc, cdf a, cdf b) {
  acc.re = df_fma(a.re, b.re, acc.re);
  acc.re = df_fma(a.im, b.im, acc.re);
  acc.im = df_fma(a.re, b.im, acc.im);
  acc.im = df_fma(-a.im, b.re, acc.im);
}

// 1 / sqrt(a), a > 0: float estimate, one Newton step y <- y (3 - a y^2) / 2 in
// double-float.
__device__ __forceinline__ df df_rsqrt(df a) {
  const float y0 = rsqrtf(a.hi);
  const df y(y0, 0.f);
  const df t = a * (y * y);  // ~1
  const df corr = df(0.5f) * (df(3.f) - t);
  return y * corr;
}

__device__ __forceinline__ cdf cdf_zero() { return cdf(df(0.f, 0.f), df(0.f, 0.f)); }

__device__ __forceinline__ df df_abs(df a) { return a.hi < 0.f ? -a : a; }
__device__ __forceinline__ bool df_gt(df a, df b) { return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo); }

// Out-of-line copies of the larger operations for code that runs once per loop on
// one thread (the 2 x 2 eigen-decomposition below): called rather than inlined, each
// exists once in the kernel, so a cold instruction cache fetches less of it.
static __device__ __noinline__ cdf cmul_ool(cdf a, cdf b) { return a * b; }
static __device__ __noinline__ cdf cadd_ool(cdf a, cdf b) { return a + b; }
static __device__ __noinline__ cdf csub_ool(cdf a, cdf b) { return a - b; }
static __device__ __noinline__ df abs2_ool(cdf a) { return abs2(a); }
static __device__ __noinline__ df dfadd_ool(df a, df b) { return a + b; }
static __device__ __noinline__ df dfdiv_ool(df a, df b) { return df_div(a, b); }
static __device__ __noinline__ df dfsqrt_ool(df a) { return df_sqrt(a); }

// Principal complex square root: t = sqrt((|z| + |Re z|) / 2), then Im z / (2 t).
__device__ inline cdf csqrt_df(cdf z) {
  const df r = dfsqrt_ool(abs2_ool(z));
  if (!(r.hi > 0.f)) return cdf_zero();
  const df t = dfsqrt_ool(df(0.5f) * dfadd_ool(r, df_abs(z.re)));
  const df two_t = df(2.f) * t;
  if (z.re.hi >= 0.f) return cdf(t, dfdiv_ool(z.im, two_t));
  return cdf(dfdiv_ool(df_abs(z.im), two_t), z.im.hi >= 0.f ? t : -t);
}

// Closed-form eigenvalues of the 2 x 2 complex matrix H = [[a, b], [c, d]]
// (row-major) in double-float: lambda = (a + d)/2 +- sqrt(((a - d)/2)^2 + b c); the
// root of larger magnitude from the formula, the other as det / lambda_1 (no
// cancellation).
__device__ inline void eig2_values_df(const cdf* H, cdf* lam) {
  const cdf a = H[0], b = H[1], c = H[2], d = H[3];
  const cdf mid = df(0.5f) * cadd_ool(a, d), half = df(0.5f) * csub_ool(a, d);
  const cdf sq = csqrt_df(cadd_ool(cmul_ool(half, half), cmul_ool(b, c)));
  const cdf l1p = cadd_ool(mid, sq), l1m = csub_ool(mid, sq);
  const cdf l1 = df_gt(abs2_ool(l1m), abs2_ool(l1p)) ? l1m : l1p;
  const cdf det = csub_ool(cmul_ool(a, d), cmul_ool(b, c));
  cdf l2 = cdf_zero();
  const df den = abs2_ool(l1);
  if (den.hi > 0.f) {
    const cdf num = cmul_ool(det, conj(l1));
    l2 = cdf(dfdiv_ool(num.re, den), dfdiv_ool(num.im, den));
  }
  lam[0] = l1;
  lam[1] = l2;
}

// Unit right eigenvector of H for its eigenvalue l, written as column k of the
// row-major 2 x 2 Z: (b, l - a) or (l - d, c), whichever is longer (e_k when H is a
// multiple of I).
__device__ inline void eig2_vector_df(const cdf* H, cdf l, int k, cdf* Z) {
  const cdf a = H[0], b = H[1], c = H[2], d = H[3];
  cdf v0 = b, v1 = csub_ool(l, a);
  const cdf w0 = csub_ool(l, d), w1 = c;
  if (df_gt(dfadd_ool(abs2_ool(w0), abs2_ool(w1)), dfadd_ool(abs2_ool(v0), abs2_ool(v1)))) {
    v0 = w0;
    v1 = w1;
  }
  df nv = dfadd_ool(abs2_ool(v0), abs2_ool(v1));
  if (!(nv.hi > 0.f)) {
    v0 = cdf(df(k == 0 ? 1.f : 0.f), df(0.f));
    v1 = cdf(df(k == 0 ? 0.f : 1.f), df(0.f));
    nv = df(1.f);
  }
  const df inv = df_rsqrt(nv);
  Z[k] = inv * v0;
  Z[2 + k] = inv * v1;
}

// ---------------------------------------------------------------------------
// Unit-circle points and phases in double-float (FP32 pipe; GB300's FP64 pipe runs
// at 1/64 of the FP32 rate, so a transcendental on one thread of the latency-bound
// loop kernel costs microseconds in FP64).  Written from the textbook construction:
// reduction of the angle to |y| <= pi/4 plus a quarter turn, then the Taylor series of
// sin and cos about 0 by Horner's rule (truncated below 1e-17 at |y| = pi/4), every
// step with the accurate double-float sum and product; the phase of z refines a float
// estimate theta0 by the angle of z e^{-i theta0}, which is below 1e-6 in size, so
// its arctangent equals the ratio to 1e-20.  Errors ~5e-15 (sin, cos) and ~1e-14 rad
// (phase), at the double-float resolution.  Out of line: one copy of the code serves
// every caller, so a cold instruction cache fetches it once.
// ---------------------------------------------------------------------------

// A double constant as a double-float (used in constant expressions only).
__host__ __device__ constexpr df dfk(double x) { return df(float(x), float(x - double(float(x)))); }

// sin y and cos y, |y| <= pi/4 (a little beyond is harmless).
static __device__ __noinline__ void df_sincos_small(df y, df& s, df& c) {
  // sin y / y = sum_k (-1)^k z^k / (2k+1)!, k <= 8; cos y = sum_k (-1)^k z^k / (2k)!, k <= 9
  constexpr df s8 = dfk(1.0 / 355687428096000.0), s7 = dfk(-1.0 / 1307674368000.0),
               s6 = dfk(1.0 / 6227020800.0), s5 = dfk(-1.0 / 39916800.0), s4 = dfk(1.0 / 362880.0),
               s3 = dfk(-1.0 / 5040.0), s2 = dfk(1.0 / 120.0), s1 = dfk(-1.0 / 6.0);
  constexpr df c9 = dfk(-1.0 / 6402373705728000.0), c8 = dfk(1.0 / 20922789888000.0),
               c7 = dfk(-1.0 / 87178291200.0), c6 = dfk(1.0 / 479001600.0),
               c5 = dfk(-1.0 / 3628800.0), c4 = dfk(1.0 / 40320.0), c3 = dfk(-1.0 / 720.0),
               c2 = dfk(1.0 / 24.0);
  const df z = y * y;
  df ps = s8;
  ps = ps * z + s7;
  ps = ps * z + s6;
  ps = ps * z + s5;
  ps = ps * z + s4;
  ps = ps * z + s3;
  ps = ps * z + s2;
  ps = ps * z + s1;
  ps = ps * z + df(1.f);
  df pc = c9;
  pc = pc * z + c8;
  pc = pc * z + c7;
  pc = pc * z + c6;
  pc = pc * z + c5;
  pc = pc * z + c4;
  pc = pc * z + c3;
  pc = pc * z + c2;
  pc = pc * z + df(-0.5f);
  pc = pc * z + df(1.f);
  s = y * ps;
  c = pc;
}

// e^{i (q pi/2 + y)} from sin y, cos y.
__device__ __forceinline__ cdf df_cis_quarter(int q, df s, df c) {
  switch (q & 3) {
    case 0: return cdf(c, s);
    case 1: return cdf(-s, c);
    case 2: return cdf(-c, -s);
    default: return cdf(s, -c);
  }
}

// e^{i pi num / den}, den >= 1, |num| < 2^28 (exact reduction in integers).
static __device__ __noinline__ cdf df_cispi_ratio(int num, int den) {
  int k = num % (2 * den);
  if (k < 0) k += 2 * den;
  const int q = (4 * k + den) / (2 * den);  // nearest quarter turn
  const int n = 2 * k - q * den;            // y = pi n / (2 den), |n| <= den / 2
  constexpr df pi = dfk(3.141592653589793);
  const df r = df_div(df(float(n)), df(float(2 * den)));
  df sn, cs;
  df_sincos_small(pi * r, sn, cs);
  return df_cis_quarter(q, sn, cs);
}

// e^{i pi t} for a double t.
static __device__ __noinline__ cdf df_cispi(double t) {
  t -= 2.0 * rint(0.5 * t);  // exact: t in [-1, 1]
  const double qd = rint(2.0 * t);
  const double r = t - 0.5 * qd;  // exact, |r| <= 1/4
  constexpr df pi = dfk(3.141592653589793);
  df sn, cs;
  df_sincos_small(pi * df_from_double(r), sn, cs);
  return df_cis_quarter(int(qd), sn, cs);
}

// arg z in (-pi, pi] (as atan2), for z of modest dynamic range (both parts of the
// float exponent range); z = 0 and NaN take the FP64 atan2 of the leading parts.
static __device__ __noinline__ double df_phase(cdf z) {
  const float t0 = atan2f(z.im.hi, z.re.hi);
  if ((z.re.hi == 0.f && z.im.hi == 0.f) || !(t0 == t0)) return atan2(double(z.im.hi), double(z.re.hi));
  const int q = __float2int_rn(t0 * 0.636619772f);  // nearest quarter turn
  constexpr df hp = dfk(1.5707963267948966);
  const df y = df(t0) - df(float(q) * hp.hi, float(q) * hp.lo);  // q hp exact (|q| <= 2)
  df sn, cs;
  df_sincos_small(y, sn, cs);
  const cdf e = df_cis_quarter(q, sn, cs);  // e^{i t0}
  // z e^{-i t0} = (x c + y s) + i (y c - x s)
  const df xr = z.re * e.re + z.im * e.im;
  const df yr = z.im * e.re - z.re * e.im;
  double th = double(t0) + df_to_double(df_div(yr, xr));
  if (th > 3.141592653589793) th -= 6.283185307179586;
  if (th <= -3.141592653589793) th += 6.283185307179586;
  return th;
}

// Warp shuffle of a complex double-float.
__device__ __forceinline__ cdf shfl_cdf(cdf v, int src) {
  return cdf(df(__shfl_sync(0xffffffffu, v.re.hi, src), __shfl_sync(0xffffffffu, v.re.lo, src)),
             df(__shfl_sync(0xffffffffu, v.im.hi, src), __shfl_sync(0xffffffffu, v.im.lo, src)));
}

__device__ __forceinline__ df shfl_xor_df(df v, int m) {
  return df(__shfl_xor_sync(0xffffffffu, v.hi, m), __shfl_xor_sync(0xffffffffu, v.lo, m));
}

}  // namespace bw
