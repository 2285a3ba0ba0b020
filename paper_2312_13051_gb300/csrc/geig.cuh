// Block-wide eigensolver for a general complex matrix in shared memory (FP64).
//
// The Wilson matrix of Eq. 2 is a product of raw overlaps and is not unitary, so
// its eigenvalues need a general (non-Hermitian) solver: Householder reduction to
// upper Hessenberg form, then single-shift implicit QR sweeps with Givens
// rotations, Wilkinson shifts and deflation on small subdiagonals.  With vectors
// requested the rotations are applied to whole rows/columns, leaving the Schur
// form T = Z^dagger W Z; right eigenvectors are x = Z y with T y = lambda y solved
// by back substitution.
#pragma once

#include "common.cuh"

namespace bw {

struct GeigShared {
  z64 c0;        // Givens: G = [[c, s], [-conj(s), c]], c real (stored in c0.re)
  z64 s;
  z64 mu;
  int l, hi, active, fail, k;
  double scale;
};

__device__ __forceinline__ double zabs(z64 a) { return hypot(a.re, a.im); }

// Givens G with G [x; y] = [r; 0], c real >= 0: c = |x| / r, s = (x / |x|) conj(y) / r,
// r = sqrt(|x|^2 + |y|^2), from two reciprocal square roots (the entries of the
// Wilson matrices are O(1), far from the range where the squares over- or
// underflow; a square that underflows makes the rotation swap the two rows, still
// unitary, and the entry it leaves behind is set to zero by the caller).
__device__ __forceinline__ void givens(z64 x, z64 y, double& c, z64& s) {
  const double ax2 = abs2(x), ay2 = abs2(y);
  if (ay2 == 0.0) {
    c = 1.0;
    s = z64(0.0, 0.0);
    return;
  }
  if (ax2 == 0.0) {
    c = 0.0;
    const double iy = rsqrt(ay2);
    s = z64(y.re * iy, -y.im * iy);  // conj(y)/|y|
    return;
  }
  const double ir = rsqrt(ax2 + ay2), iax = rsqrt(ax2);
  c = ax2 * iax * ir;
  const z64 ux(x.re * iax, x.im * iax);
  s = ir * (ux * conj(y));
}

// Whether the subdiagonal entry H[l][l-1] is negligible: against the neighbouring
// diagonal entries, or by the product test of Ahues and Tisseur (its product with
// the superdiagonal small against the local separation of the diagonal entries).
__device__ __forceinline__ bool geig_negligible_v(z64 h11, z64 h12, z64 h21, z64 h22, double eps) {
  const double sub = zabs(h21);
  const double dia = zabs(h22) + zabs(h11);
  bool small = sub <= eps * dia || sub < 1e-300;
  if (!small && sub <= dia) {
    const double x = zabs(h12);
    const double ab = fmax(sub, x), ba = fmin(sub, x);
    const double y = zabs(h11 - h22);
    const double aa = fmax(zabs(h22), y), bb = fmin(zabs(h22), y);
    const double sc = aa + ab;
    small = ba * (ab / sc) <= fmax(1e-300, eps * (bb * (aa / sc)));
  }
  return small;
}

__device__ __forceinline__ bool geig_negligible(const z64* H, int ld, int l, double eps) {
  return geig_negligible_v(H[(l - 1) * ld + l - 1], H[(l - 1) * ld + l], H[l * ld + l - 1],
                           H[l * ld + l], eps);
}

// Shift of a QR sweep from the trailing 2 x 2 [[a, b], [c, d]] of the active window:
// its eigenvalue closest to d (Wilkinson); every 12th sweep without a deflation the
// exceptional shift d + 0.75 (|c| + sub2), sub2 = |H[hi-1][hi-2]| (0 when hi < 2).
__device__ __forceinline__ z64 geig_shift(z64 a, z64 b, z64 c, z64 d, int iter, double sub2) {
  if (iter > 0 && iter % 12 == 0) return d + z64(0.75 * (zabs(c) + sub2), 0.0);
  const z64 half = 0.5 * (a - d);
  const z64 disc = half * half + b * c;
  // complex sqrt
  const double r = zabs(disc);
  const double sr = sqrt(0.5 * (r + fabs(disc.re)));
  z64 sq;
  if (sr == 0.0) {
    sq = z64(0.0, 0.0);
  } else if (disc.re >= 0.0) {
    sq = z64(sr, disc.im / (2.0 * sr));
  } else {
    sq = z64(fabs(disc.im) / (2.0 * sr), disc.im >= 0.0 ? sr : -sr);
  }
  // mu = d + half -/+ sq, the one closer to d
  const z64 m1 = d + half - sq, m2 = d + half + sq;
  return (abs2(m1 - d) <= abs2(m2 - d)) ? m1 : m2;
}

// Largest l in [1, hi] whose subdiagonal entry is negligible, or 0: the first warp
// tests 32 subdiagonals at a time from hi down.  Every lane of the warp calls it.
__device__ __forceinline__ int geig_split_point(const z64* H, int ld, int hi, double eps) {
  const int lane = threadIdx.x & 31;
  for (int base = hi; base >= 1; base -= 32) {
    const int l = base - lane;
    const bool f = l >= 1 && geig_negligible(H, ld, l, eps);
    const unsigned m = __ballot_sync(0xffffffffu, f);
    if (m) return base - (__ffs(m) - 1);
  }
  return 0;
}

// Eigen-decomposition of H (p x p, leading dimension ld), destroyed on output.
// lam[p] receives the eigenvalues.  With want_vec, Z (p x p) receives the right
// eigenvectors as unit-norm columns; vec scratch needs p z64.  Returns 0, or -1
// when the QR iteration cap (120 p sweeps) is reached.
__device__ inline int geig(z64* H, z64* Z, int p, int ld, bool want_vec, z64* lam, z64* vec,
                    GeigShared* sh) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const double eps = 2.220446049250313e-16;
  if (want_vec)
    for (int e = tid; e < p * p; e += nt) {
      const int r = e / p, c = e - r * p;
      Z[r * ld + c] = z64(double(r == c), 0.0);
    }
  __syncthreads();
  // --- Householder reduction to Hessenberg form.  Column norms are block
  // reductions; the left update runs one thread per column and the right update one
  // warp per row, so that consecutive threads touch consecutive entries.
  __shared__ double hred[32];
  const int lane = tid & 31, warp = tid >> 5, nwarp = nt >> 5;
  for (int c = 0; c + 2 < p; ++c) {
    double nrm2 = 0.0;
    for (int r = c + 1 + tid; r < p; r += nt) nrm2 += abs2(H[r * ld + c]);
    nrm2 = block_sum(nrm2, hred);
    const z64 x0 = H[(c + 1) * ld + c];
    const double tail = nrm2 - abs2(x0);
    if (!(tail > 0.0)) {
      __syncthreads();
      continue;
    }
    const double nx = sqrt(nrm2), ax0 = zabs(x0);
    const z64 ph = ax0 > 0.0 ? z64(x0.re / ax0, x0.im / ax0) : z64(1.0, 0.0);
    // v = x - alpha e1, alpha = -|x| ph: v_0 = ph (|x0| + |x|), |v|^2 = (|x0| + |x|)^2 + tail
    const double v0m = ax0 + nx, nv = 1.0 / sqrt(v0m * v0m + tail);
    for (int r = c + 1 + tid; r < p; r += nt)
      vec[r] = r == c + 1 ? z64(nv * v0m * ph.re, nv * v0m * ph.im) : nv * H[r * ld + c];
    if (tid == 0) sh->mu = -nx * ph;
    __syncthreads();
    // left: H <- (I - 2 v v^dagger) H on rows c+1.., columns c+1.. (column c is set below)
    for (int col = c + 1 + tid; col < p; col += nt) {
      z64 w(0.0, 0.0);
      for (int r = c + 1; r < p; ++r) cfma_conj(w, vec[r], H[r * ld + col]);
      for (int r = c + 1; r < p; ++r) H[r * ld + col] = H[r * ld + col] - 2.0 * (vec[r] * w);
    }
    __syncthreads();
    // right: H <- H (I - 2 v v^dagger) on columns c+1..; Z likewise
    for (int row = warp; row < p; row += nwarp) {
      z64* hr = H + row * ld;
      z64 w(0.0, 0.0);
      for (int k = c + 1 + lane; k < p; k += 32) cfma(w, hr[k], vec[k]);
      for (int o = 16; o > 0; o >>= 1) {
        w.re += __shfl_xor_sync(0xffffffffu, w.re, o);
        w.im += __shfl_xor_sync(0xffffffffu, w.im, o);
      }
      for (int k = c + 1 + lane; k < p; k += 32) hr[k] = hr[k] - 2.0 * (w * conj(vec[k]));
      if (want_vec) {
        z64* zr = Z + row * ld;
        z64 wz(0.0, 0.0);
        for (int k = c + 1 + lane; k < p; k += 32) cfma(wz, zr[k], vec[k]);
        for (int o = 16; o > 0; o >>= 1) {
          wz.re += __shfl_xor_sync(0xffffffffu, wz.re, o);
          wz.im += __shfl_xor_sync(0xffffffffu, wz.im, o);
        }
        for (int k = c + 1 + lane; k < p; k += 32) zr[k] = zr[k] - 2.0 * (wz * conj(vec[k]));
      }
    }
    __syncthreads();
    for (int r = c + 1 + tid; r < p; r += nt) H[r * ld + c] = r == c + 1 ? sh->mu : z64(0.0, 0.0);
    __syncthreads();
  }
  // --- shifted QR on the Hessenberg matrix
  if (tid == 0) {
    sh->hi = p - 1;
    sh->fail = 0;
  }
  __syncthreads();
  int iter = 0, total = 0;
  const int cap = 120 * p + 120;
  while (true) {
    if (tid < 32) {  // the first warp finds the active block; its lane 0 sets the shift
      int hi = sh->hi;
      if (tid == 0) sh->active = 0;
      while (hi >= 0) {
        if (hi == 0) {
          if (tid == 0) lam[0] = H[0];
          hi = -1;
          break;
        }
        const int l = geig_split_point(H, ld, hi, eps);
        __syncwarp();
        if (tid == 0 && l > 0) H[l * ld + l - 1] = z64(0.0, 0.0);
        if (l == hi) {
          if (tid == 0) lam[hi] = H[hi * ld + hi];
          --hi;
          iter = 0;
          continue;
        }
        if (tid != 0) break;
        // shift from the trailing 2x2 of the active window
        const z64 mu = geig_shift(H[(hi - 1) * ld + hi - 1], H[(hi - 1) * ld + hi], H[hi * ld + hi - 1],
                                  H[hi * ld + hi], iter, hi >= 2 ? zabs(H[(hi - 1) * ld + hi - 2]) : 0.0);
        sh->mu = mu;
        sh->l = l;
        sh->active = 1;
        break;
      }
      if (tid == 0) {
        sh->hi = hi;
        ++iter;
        ++total;
        if (total > cap) {
          sh->fail = 1;
          sh->active = 0;
          sh->hi = -1;
        }
      }
    }
    __syncthreads();
    if (!sh->active) break;
    const int l = sh->l, hi = sh->hi;
    const int col_end = want_vec ? p - 1 : hi;
    const int row_beg = want_vec ? 0 : l;
    for (int k = l; k < hi; ++k) {
      if (tid == 0) {
        z64 x, y;
        if (k == l) {
          x = H[l * ld + l] - sh->mu;
          y = H[(l + 1) * ld + l];
        } else {
          x = H[k * ld + k - 1];
          y = H[(k + 1) * ld + k - 1];
        }
        double c;
        z64 s;
        givens(x, y, c, s);
        sh->c0 = z64(c, 0.0);
        sh->s = s;
      }
      __syncthreads();
      const double c = sh->c0.re;
      const z64 s = sh->s;
      // rows k, k+1: [rk; rk1] <- G [rk; rk1]
      const int cb = (k > l) ? k - 1 : l;
      for (int col = cb + tid; col <= col_end; col += nt) {
        const z64 x = H[k * ld + col], y = H[(k + 1) * ld + col];
        H[k * ld + col] = c * x + s * y;
        H[(k + 1) * ld + col] = c * y - conj(s) * x;
      }
      __syncthreads();
      if (tid == 0 && k > l) H[(k + 1) * ld + k - 1] = z64(0.0, 0.0);
      // columns k, k+1: H <- H G^dagger ; Z <- Z G^dagger
      const int re = min(k + 2, hi);
      for (int row = row_beg + tid; row <= re; row += nt) {
        const z64 x = H[row * ld + k], y = H[row * ld + k + 1];
        H[row * ld + k] = c * x + y * conj(s);
        H[row * ld + k + 1] = c * y - x * s;
      }
      if (want_vec)
        for (int row = tid; row < p; row += nt) {
          const z64 x = Z[row * ld + k], y = Z[row * ld + k + 1];
          Z[row * ld + k] = c * x + y * conj(s);
          Z[row * ld + k + 1] = c * y - x * s;
        }
      __syncthreads();
    }
  }
  const int fail = sh->fail;
  __syncthreads();
  if (fail) return -1;
  if (!want_vec) return 0;
  // --- right eigenvectors of the triangular T by back substitution; column k of
  // the result replaces column k of Z (T stays in H's upper triangle).
  double tn = 0.0;
  for (int e = tid; e < p * p; e += nt) {
    const int r = e / p, c = e - r * p;
    if (c >= r) tn = fmax(tn, zabs(H[r * ld + c]));
  }
  __shared__ double tmax[32];
  tn = -block_min(-tn, tmax);
  const double small = fmax(eps * tn, 1e-300);
  // Decreasing k: column k of X = Z[:, 0..k] y_k only uses columns <= k of the
  // original Z, which are untouched when columns are replaced from the right.
  for (int k = p - 1; k >= 0; --k) {
    if (tid == 0) {
      const z64 lk = H[k * ld + k];
      for (int r = k + 1; r < p; ++r) vec[r] = z64(0.0, 0.0);
      vec[k] = z64(1.0, 0.0);
      for (int r = k - 1; r >= 0; --r) {
        z64 acc(0.0, 0.0);
        for (int c = r + 1; c <= k; ++c) cfma(acc, H[r * ld + c], vec[c]);
        z64 den = H[r * ld + r] - lk;
        if (zabs(den) < small) den = z64(small, 0.0);
        const double dd = abs2(den);
        vec[r] = z64(-(acc.re * den.re + acc.im * den.im) / dd,
                     -(acc.im * den.re - acc.re * den.im) / dd);
      }
    }
    __syncthreads();
    double nrm = 0.0;
    z64 xr[4];
    int cnt = 0;
    for (int row = tid; row < p; row += nt, ++cnt) {
      z64 acc(0.0, 0.0);
      for (int c = 0; c <= k; ++c) cfma(acc, Z[row * ld + c], vec[c]);
      if (cnt < 4) xr[cnt] = acc;
      nrm += abs2(acc);
    }
    nrm = block_sum(nrm, tmax);
    const double inv = 1.0 / sqrt(nrm);
    cnt = 0;
    for (int row = tid; row < p; row += nt, ++cnt) Z[row * ld + k] = inv * xr[cnt];
    __syncthreads();
  }
  return 0;
}

// Principal complex square root.
__device__ __forceinline__ z64 csqrt64(z64 z) {
  const double r = zabs(z);
  if (r == 0.0) return z64(0.0, 0.0);
  const double t = sqrt(0.5 * (r + fabs(z.re)));
  if (z.re >= 0.0) return z64(t, z.im / (2.0 * t));
  return z64(fabs(z.im) / (2.0 * t), z.im >= 0.0 ? t : -t);
}

// Closed-form eigen-decomposition of a 2 x 2 complex matrix H = [[a, b], [c, d]]
// (leading dimension ld), one thread: lam[0..2), and with Z the unit right
// eigenvectors as columns.  lambda = (a + d)/2 +- sqrt(((a - d)/2)^2 + b c); the
// root of larger magnitude comes from the formula and the other from
// det / lambda_1, which avoids cancellation.  Eigenvector of lambda: (b, lambda - a)
// or (lambda - d, c), whichever is longer (e_1, e_2 when H is a multiple of I).
__device__ inline void eig2_closed(const z64* H, int ld, z64* lam, z64* Z, bool want_vec) {
  const z64 a = H[0], b = H[1], c = H[ld], d = H[ld + 1];
  const z64 mid = 0.5 * (a + d), half = 0.5 * (a - d);
  const z64 sq = csqrt64(half * half + b * c);
  const z64 l1p = mid + sq, l1m = mid - sq;
  const z64 l1 = abs2(l1p) >= abs2(l1m) ? l1p : l1m;
  const z64 det = a * d - b * c;
  z64 l2;
  if (abs2(l1) > 0.0) {
    const double den = abs2(l1);
    l2 = z64((det.re * l1.re + det.im * l1.im) / den, (det.im * l1.re - det.re * l1.im) / den);
  } else {
    l2 = z64(0.0, 0.0);
  }
  lam[0] = l1;
  lam[1] = l2;
  if (!want_vec) return;
  for (int k = 0; k < 2; ++k) {
    const z64 l = lam[k];
    z64 v0 = b, v1 = l - a;
    const z64 w0 = l - d, w1 = c;
    if (abs2(w0) + abs2(w1) > abs2(v0) + abs2(v1)) {
      v0 = w0;
      v1 = w1;
    }
    double nv = abs2(v0) + abs2(v1);
    if (!(nv > 0.0)) {
      v0 = z64(k == 0 ? 1.0 : 0.0, 0.0);
      v1 = z64(k == 0 ? 0.0 : 1.0, 0.0);
      nv = 1.0;
    }
    const double inv = 1.0 / sqrt(nv);
    Z[0 * ld + k] = inv * v0;
    Z[1 * ld + k] = inv * v1;
  }
}

}  // namespace bw
