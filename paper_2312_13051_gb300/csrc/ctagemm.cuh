// CTA-level building blocks of the large-n solver: a tiled complex GEMM with compensated
// sums for FP64-grade results (the plain FP32 products run on the tensor cores,
// tcgen05.cuh) and the application of a sequence of Householder reflectors, one at a
// time on column panels in shared memory (FP64) or in blocks (compact WY form) through
// tensor-core GEMMs (FP32).  Both keep operand reuse in shared memory instead of L2.
#pragma once

#include "common.cuh"
#include "tcgen05.cuh"

namespace bw {

// ---------------------------------------------------------------------------
// Compensated FP32 dot products (Ogita, Rump and Oishi, "Accurate sum and dot
// product", SIAM J. Sci. Comput. 26 (2005), algorithm Dot2): each product is split
// exactly into a + e with one FMA, the running sum is kept as hi + lo with an
// error-free two-sum, and the result is as accurate as a sum carried in twice the
// working precision.  GB300 runs FP32 ~70x faster than FP64, so this is the cheap
// way to the FP64-grade residuals the Newton correction needs.
// ---------------------------------------------------------------------------
struct DF {
  float hi, lo;
  __device__ __forceinline__ DF() : hi(0.f), lo(0.f) {}
  __device__ __forceinline__ void add_prod(float a, float b) {
    const float p = a * b;
    const float e = fmaf(a, b, -p);      // exact: a b = p + e
    const float s = hi + p;
    const float bp = s - hi;
    const float err = (hi - (s - bp)) + (p - bp);  // exact: hi + p = s + err
    hi = s;
    lo += err + e;
  }
  __device__ __forceinline__ void add(float x) { lo += x; }
  __device__ __forceinline__ double value() const { return double(hi) + double(lo); }
};

struct CDF {
  DF re, im;
  // acc += a * b with a = ah + al (FP64 split into two floats), b FP32
  __device__ __forceinline__ void add_prod(c32 ah, c32 al, c32 b) {
    re.add_prod(ah.re, b.re);
    re.add_prod(-ah.im, b.im);
    im.add_prod(ah.re, b.im);
    im.add_prod(ah.im, b.re);
    re.add(al.re * b.re - al.im * b.im);
    im.add(al.re * b.im + al.im * b.re);
  }
  // acc += conj(a) * b, both FP32
  __device__ __forceinline__ void add_cprod(c32 a, c32 b) {
    re.add_prod(a.re, b.re);
    re.add_prod(a.im, b.im);
    im.add_prod(a.re, b.im);
    im.add_prod(-a.im, b.re);
  }
  __device__ __forceinline__ z64 value() const { return z64(re.value(), im.value()); }
};


// Operand and accumulator policies of cta_gemm.
template <typename T>
struct GemmPlainT {  // C = A B in the precision of T
  using TA = cx<T>;
  using TB = cx<T>;
  using Acc = cx<T>;
  static constexpr bool kPrefetch = true;
  static __device__ __forceinline__ TA zero_a() { return TA(T(0), T(0)); }
  static __device__ __forceinline__ Acc zero() { return Acc(T(0), T(0)); }
  static __device__ __forceinline__ void mac(Acc& c, const TA& a, const TB& b) { cfma(c, a, b); }
};
struct SplitC {  // an FP64 value as the float pair hi + lo
  c32 hi, lo;
};
struct GemmSplitComp {  // C = A B, A an FP64 matrix as float pairs, compensated sums
  using TA = SplitC;
  using TB = c32;
  using Acc = CDF;
  static constexpr bool kPrefetch = false;  // compute-bound; its accumulators fill the registers
  static __device__ __forceinline__ TA zero_a() { return SplitC{c32(0.f, 0.f), c32(0.f, 0.f)}; }
  static __device__ __forceinline__ Acc zero() { return CDF(); }
  static __device__ __forceinline__ void mac(Acc& c, const TA& a, const TB& b) { c.add_prod(a.hi, a.lo, b); }
};
struct GemmGramComp {  // C = A^dag B (A passed unconjugated), compensated sums
  using TA = c32;
  using TB = c32;
  using Acc = CDF;
  static constexpr bool kPrefetch = false;
  static __device__ __forceinline__ TA zero_a() { return c32(0.f, 0.f); }
  static __device__ __forceinline__ Acc zero() { return CDF(); }
  static __device__ __forceinline__ void mac(Acc& c, const TA& a, const TB& b) { c.add_cprod(a, b); }
};

constexpr int CG_TILE = 64, CG_K = 16;
// Row length of the staged tiles: one element of padding, so that the staging stores
// of an operand whose k index is contiguous in memory (consecutive threads, rows kk
// apart) fall in different banks.
constexpr int CG_LD = CG_TILE + 1;
// Shared memory used by cta_gemm<Pol> (a 16 x 64 tile of each operand).
template <class Pol>
__host__ __device__ constexpr size_t cg_smem() {
  return CG_K * CG_LD * (sizeof(typename Pol::TA) + sizeof(typename Pol::TB));
}
constexpr size_t CG_SMEM = CG_K * CG_LD * (sizeof(SplitC) + sizeof(c32));  // the largest policy

// C(m, c) = sum_k A(m, k) B(k, c) (the policy's product and accumulator) for m < M,
// c < Ncol, k < K, computed by all blockDim.x == 256 threads of the CTA in 64 x 64
// output tiles (thread (ty, tx) owns rows ty + 16 i and columns tx + 16 j).
// la(m, k) and lb(k, c) return the operands (out-of-range indices are never
// requested); st(m, c, acc) consumes each result once.  A_K_CONTIG / B_C_CONTIG say
// which index of the operand is contiguous in memory, so that the staging loads
// are coalesced.  sm: cg_smem<Pol>() bytes.
template <class Pol, bool A_K_CONTIG, bool B_C_CONTIG, class LA, class LB, class ST>
__device__ void cta_gemm(int M, int Ncol, int K, LA la, LB lb, ST st, unsigned char* sm) {
  using TA = typename Pol::TA;
  using TB = typename Pol::TB;
  TA(*As)[CG_LD] = reinterpret_cast<TA(*)[CG_LD]>(sm);
  TB(*Bs)[CG_LD] = reinterpret_cast<TB(*)[CG_LD]>(sm + CG_K * CG_LD * sizeof(TA));
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  for (int m0 = 0; m0 < M; m0 += CG_TILE)
    for (int c0 = 0; c0 < Ncol; c0 += CG_TILE) {
      typename Pol::Acc acc[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = Pol::zero();
      // each thread moves PER elements of each operand per k-step; with Pol::kPrefetch
      // the next step's elements are loaded into registers before this step's products,
      // so that their global-memory latency overlaps the arithmetic
      constexpr int PER = CG_K * CG_TILE / 256;
      TA ra[PER];
      TB rb[PER];
      auto fetch = [&](int k0) {
#pragma unroll
        for (int s = 0; s < PER; ++s) {
          const int e = tid + 256 * s;
          int kk, mm, cc;
          if (A_K_CONTIG) {
            mm = e / CG_K;
            kk = e - mm * CG_K;
          } else {
            kk = e / CG_TILE;
            mm = e - kk * CG_TILE;
          }
          ra[s] = (m0 + mm < M && k0 + kk < K) ? la(m0 + mm, k0 + kk) : Pol::zero_a();
          if (B_C_CONTIG) {
            kk = e / CG_TILE;
            cc = e - kk * CG_TILE;
          } else {
            cc = e / CG_K;
            kk = e - cc * CG_K;
          }
          rb[s] = (c0 + cc < Ncol && k0 + kk < K) ? lb(k0 + kk, c0 + cc) : TB(0, 0);
        }
      };
      auto stage = [&]() {
#pragma unroll
        for (int s = 0; s < PER; ++s) {
          const int e = tid + 256 * s;
          int kk, mm, cc;
          if (A_K_CONTIG) {
            mm = e / CG_K;
            kk = e - mm * CG_K;
          } else {
            kk = e / CG_TILE;
            mm = e - kk * CG_TILE;
          }
          As[kk][mm] = ra[s];
          if (B_C_CONTIG) {
            kk = e / CG_TILE;
            cc = e - kk * CG_TILE;
          } else {
            cc = e / CG_K;
            kk = e - cc * CG_K;
          }
          Bs[kk][cc] = rb[s];
        }
      };
      if (Pol::kPrefetch) fetch(0);
      for (int k0 = 0; k0 < K; k0 += CG_K) {
        if (!Pol::kPrefetch) fetch(k0);
        stage();
        __syncthreads();
        if (Pol::kPrefetch && k0 + CG_K < K) fetch(k0 + CG_K);
#pragma unroll 2
        for (int kk = 0; kk < CG_K; ++kk) {
          TA av[4];
          TB bv[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) av[i] = As[kk][ty + 16 * i];
#pragma unroll
          for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tx + 16 * j];
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) Pol::mac(acc[i][j], av[i], bv[j]);
        }
        __syncthreads();
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int gm = m0 + ty + 16 * i, gc = c0 + tx + 16 * j;
          if (gm < M && gc < Ncol) st(gm, gc, acc[i][j]);
        }
    }
}

// Applies the reflectors P_c = I - 2 u_c u_c^dag, c = 0 .. n-3 (u_c in column c of
// A below the diagonal, rows c+1..n-1), to X (n x ncol, leading dimension ldx, in
// global memory): X <- P_{n-3} ... P_0 X (forward) or X <- P_0 ... P_{n-3} X
// (reverse), one reflector at a time.  X is processed in panels of PW columns held in
// shared memory; each reflector is read once per panel.  The FP64 back-transform
// uses this form: it does two thirds of the flops of the blocked form below, and the
// FP64 pipe, not latency, bounds it.  sm: reflect_smem<TX>(n, PW) bytes.
template <class TX>
__host__ __device__ inline size_t reflect_smem(int n, int PW) {
  return (size_t(n) * PW + n + 8 * size_t(PW)) * sizeof(cx<TX>);
}

template <int PW, class TA, class TX>
__device__ void cta_reflect_pw(const cx<TA>* A, int n, cx<TX>* X, int ncol, long long ldx, bool reverse,
                               unsigned char* smraw) {
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nwarp = nt >> 5;
  cx<TX>* P = reinterpret_cast<cx<TX>*>(smraw);  // n x PW panel
  cx<TX>* us = P + n * PW;                       // n
  cx<TX>* part = us + n;                         // nwarp (<= 8) x PW partial dot products
  for (int j0 = 0; j0 < ncol; j0 += PW) {
    const int w = min(PW, ncol - j0);
    for (int e = tid; e < n * PW; e += nt) {
      const int r = e / PW, j = e - r * PW;
      P[e] = j < w ? X[(long long)r * ldx + j0 + j] : cx<TX>(TX(0), TX(0));
    }
    for (int s = 0; s + 2 < n; ++s) {
      const int c = reverse ? n - 3 - s : s;
      for (int r = c + 1 + tid; r < n; r += nt) {
        const cx<TA> v = A[(long long)r * n + c];
        us[r] = cx<TX>(TX(v.re), TX(v.im));
      }
      __syncthreads();
      // partial w_j = sum_r conj(u_r) P[r][j]: warp k takes rows c+1+k, c+1+k+nwarp, ...
      if (lane < PW) {
        cx<TX> acc(TX(0), TX(0));
        for (int r = c + 1 + warp; r < n; r += nwarp) cfma_conj(acc, us[r], P[r * PW + lane]);
        part[warp * PW + lane] = acc;
      }
      __syncthreads();
      if (tid < PW) {
        cx<TX> t(TX(0), TX(0));
        for (int k = 0; k < nwarp; ++k) t = t + part[k * PW + tid];
        part[tid] = TX(2) * t;
      }
      __syncthreads();
      for (int e = (c + 1) * PW + tid; e < n * PW; e += nt) {
        const int r = e / PW, j = e - r * PW;
        P[e] = P[e] - us[r] * part[j];
      }
      __syncthreads();
    }
    for (int e = tid; e < n * PW; e += nt) {
      const int r = e / PW, j = e - r * PW;
      if (j < w) X[(long long)r * ldx + j0 + j] = P[e];
    }
    __syncthreads();
  }
}

// Panel width that fits `bytes` of shared memory (0: none fits).
template <class TX>
__host__ __device__ inline int reflect_pw(int n, size_t bytes) {
  for (int pw = 32; pw >= 1; pw >>= 1)
    if (reflect_smem<TX>(n, pw) <= bytes) return pw;
  return 0;
}

template <class TA, class TX>
__device__ void cta_reflect(const cx<TA>* A, int n, cx<TX>* X, int ncol, long long ldx, bool reverse,
                            unsigned char* sm, int pw) {
  switch (pw) {
    case 32: cta_reflect_pw<32>(A, n, X, ncol, ldx, reverse, sm); break;
    case 16: cta_reflect_pw<16>(A, n, X, ncol, ldx, reverse, sm); break;
    case 8: cta_reflect_pw<8>(A, n, X, ncol, ldx, reverse, sm); break;
    case 4: cta_reflect_pw<4>(A, n, X, ncol, ldx, reverse, sm); break;
    case 2: cta_reflect_pw<2>(A, n, X, ncol, ldx, reverse, sm); break;
    default: cta_reflect_pw<1>(A, n, X, ncol, ldx, reverse, sm); break;
  }
}

// ---------------------------------------------------------------------------
// Applies the reflectors P_c = I - 2 u_c u_c^dag, c = 0 .. n-3 (u_c in column c of A
// below the diagonal, rows c+1..n-1, unit norm) to X (n x ncol, leading dimension
// ldx, in global memory), in blocks of RW_NB (compact WY form, Schreiber
// and Van Loan, "A storage-efficient WY representation for products of Householder
// transformations", SIAM J. Sci. Stat. Comput. 10 (1989)): the product of the
// reflectors b .. b+nb-1,
//   P_b P_{b+1} ... P_{b+nb-1} = I - V T V^dag,
// V = [u_b ... u_{b+nb-1}] (n x nb, u_c zero above row c+1), T upper triangular with
// T_ii = 2 and T[0:i, i] = -2 T[0:i, 0:i] (V^dag V)[0:i, i].  Reverse (X <- P_0 ...
// P_{n-3} X) runs the blocks from last to first with X <- X - V (T (V^dag X)); forward
// (X <- P_{n-3} ... P_0 X, the adjoint product) runs them first to last with T^dag.
// Each block builds T once (a CTA GEMM and a triangular recurrence), then per chunk
// of RW_CW columns of X two CTA GEMMs and a triangular product: a few barriers per
// block instead of four per reflector.  Requires blockDim.x == 256.  Applies
// `ts`'s tensor memory (set up by the calling kernel, tcgen05.cuh).
// ---------------------------------------------------------------------------
constexpr int RW_NB = 32, RW_CW = 64;

// Shared memory of cta_reflect_wy: T, one chunk of W, and the tensor-core GEMM tiles.
__host__ __device__ inline size_t reflect_wy_smem() {
  return (size_t(RW_NB) * RW_NB + size_t(RW_NB) * RW_CW) * sizeof(c32) + tc::SMEM;
}

// FP32 (the mixed solver's precision); the three products of each block (V^dag V,
// V^dag X and X - V W) on the tensor cores.  Returns false when a tensor-core wait gave
// up (X is then incomplete).
__device__ inline bool cta_reflect_wy(const c32* A, int n, c32* X, int ncol, long long ldx, bool reverse,
                                      unsigned char* sm, tc::State& ts) {
  using C = c32;
  const int tid = threadIdx.x, lane = tid & 31;
  C* Tm = reinterpret_cast<C*>(sm);                 // RW_NB x RW_NB: V^dag V, then T
  C* W = Tm + RW_NB * RW_NB;                        // RW_NB x RW_CW
  unsigned char* gsm = reinterpret_cast<unsigned char*>(W + RW_NB * RW_CW);
  const int nrefl = n - 2;
  if (nrefl <= 0) return true;
  const int nblk = (nrefl + RW_NB - 1) / RW_NB;
  for (int bi = 0; bi < nblk; ++bi) {
    const int blk = reverse ? nblk - 1 - bi : bi;
    const int b0 = blk * RW_NB, bs = min(RW_NB, nrefl - b0);
    const int r0 = b0 + 1, rows = n - r0;            // rows where the block's vectors live
    // V[r][i] = u_{b0+i}[r] (zero for r <= b0 + i)
    auto v = [&](int r, int i) -> C {
      return r > b0 + i ? A[(long long)r * n + b0 + i] : C(0.f, 0.f);
    };
    // Gram matrix V^dag V
    if (!cta_cgemm_tc<false, true>(
            bs, bs, rows, [&](int i, int q) { return conj(v(r0 + q, i)); },
            [&](int q, int i) { return v(r0 + q, i); },
            [&](int i, int j, const C& g) { Tm[i * RW_NB + j] = g; }, gsm, ts))
      return false;
    __syncthreads();
    // T in place (one warp): column i from the columns before it
    if (tid < 32) {
      for (int i = 0; i < bs; ++i) {
        C t(0.f, 0.f);
        if (lane < i)
          for (int k = lane; k < i; ++k) cfma(t, Tm[lane * RW_NB + k], Tm[k * RW_NB + i]);
        __syncwarp();
        if (lane < i) Tm[lane * RW_NB + i] = -2.f * t;
        if (lane == 0) Tm[i * RW_NB + i] = C(2.f, 0.f);
        __syncwarp();
      }
    }
    __syncthreads();
    for (int c0 = 0; c0 < ncol; c0 += RW_CW) {
      const int cw = min(RW_CW, ncol - c0);
      // W = V^dag X[:, c0 : c0 + cw]
      if (!cta_cgemm_tc<false, true>(
              bs, cw, rows, [&](int i, int q) { return conj(v(r0 + q, i)); },
              [&](int q, int c) { return X[(long long)(r0 + q) * ldx + c0 + c]; },
              [&](int i, int c, const C& w) { W[i * RW_CW + c] = w; }, gsm, ts))
        return false;
      __syncthreads();
      // W <- T W (reverse) or T^dag W (forward), in place, one thread per column
      for (int c = tid; c < cw; c += blockDim.x) {
        if (reverse) {
          for (int i = 0; i < bs; ++i) {
            C acc(0.f, 0.f);
            for (int k = i; k < bs; ++k) cfma(acc, Tm[i * RW_NB + k], W[k * RW_CW + c]);
            W[i * RW_CW + c] = acc;
          }
        } else {
          for (int i = bs - 1; i >= 0; --i) {
            C acc(0.f, 0.f);
            for (int k = 0; k <= i; ++k) cfma(acc, conj(Tm[k * RW_NB + i]), W[k * RW_CW + c]);
            W[i * RW_CW + c] = acc;
          }
        }
      }
      __syncthreads();
      // X[:, chunk] <- X[:, chunk] - V W (rows r0 .. n-1)
      if (!cta_cgemm_tc<true, true>(
              rows, cw, bs, [&](int q, int i) { return v(r0 + q, i); },
              [&](int i, int c) { return W[i * RW_CW + c]; },
              [&](int q, int c, const C& y) {
                C& x = X[(long long)(r0 + q) * ldx + c0 + c];
                x = x - y;
              },
              gsm, ts))
        return false;
      __syncthreads();
    }
  }
  return true;
}

// The same compact-WY application with SIMT GEMMs in the precision of T: the FP64
// back-transform of large n, where a shared-memory panel of the one-reflector form
// would hold fewer than 16 columns and every panel would sweep all the reflectors.
template <typename T>
__host__ __device__ inline size_t reflect_wy_simt_smem() {
  return (size_t(RW_NB) * RW_NB + size_t(RW_NB) * RW_CW) * sizeof(cx<T>) + cg_smem<GemmPlainT<T>>();
}

template <typename T>
__device__ void cta_reflect_wy_simt(const cx<T>* A, int n, cx<T>* X, int ncol, long long ldx, bool reverse,
                               unsigned char* sm) {
  using C = cx<T>;
  const int tid = threadIdx.x, lane = tid & 31;
  C* Tm = reinterpret_cast<C*>(sm);                 // RW_NB x RW_NB: V^dag V, then T
  C* W = Tm + RW_NB * RW_NB;                        // RW_NB x RW_CW
  unsigned char* gsm = reinterpret_cast<unsigned char*>(W + RW_NB * RW_CW);
  const int nrefl = n - 2;
  if (nrefl <= 0) return;
  const int nblk = (nrefl + RW_NB - 1) / RW_NB;
  for (int bi = 0; bi < nblk; ++bi) {
    const int blk = reverse ? nblk - 1 - bi : bi;
    const int b0 = blk * RW_NB, bs = min(RW_NB, nrefl - b0);
    const int r0 = b0 + 1, rows = n - r0;            // rows where the block's vectors live
    // V[r][i] = u_{b0+i}[r] (zero for r <= b0 + i)
    auto v = [&](int r, int i) -> C {
      return r > b0 + i ? A[(long long)r * n + b0 + i] : C(T(0), T(0));
    };
    // Gram matrix V^dag V
    cta_gemm<GemmPlainT<T>, false, true>(
        bs, bs, rows, [&](int i, int q) { return conj(v(r0 + q, i)); },
        [&](int q, int i) { return v(r0 + q, i); },
        [&](int i, int j, const C& g) { Tm[i * RW_NB + j] = g; }, gsm);
    __syncthreads();
    // T in place (one warp): column i from the columns before it
    if (tid < 32) {
      for (int i = 0; i < bs; ++i) {
        C t(T(0), T(0));
        if (lane < i)
          for (int k = lane; k < i; ++k) cfma(t, Tm[lane * RW_NB + k], Tm[k * RW_NB + i]);
        __syncwarp();
        if (lane < i) Tm[lane * RW_NB + i] = T(-2) * t;
        if (lane == 0) Tm[i * RW_NB + i] = C(T(2), T(0));
        __syncwarp();
      }
    }
    __syncthreads();
    for (int c0 = 0; c0 < ncol; c0 += RW_CW) {
      const int cw = min(RW_CW, ncol - c0);
      // W = V^dag X[:, c0 : c0 + cw]
      cta_gemm<GemmPlainT<T>, false, true>(
          bs, cw, rows, [&](int i, int q) { return conj(v(r0 + q, i)); },
          [&](int q, int c) { return X[(long long)(r0 + q) * ldx + c0 + c]; },
          [&](int i, int c, const C& w) { W[i * RW_CW + c] = w; }, gsm);
      __syncthreads();
      // W <- T W (reverse) or T^dag W (forward), in place, one thread per column
      for (int c = tid; c < cw; c += blockDim.x) {
        if (reverse) {
          for (int i = 0; i < bs; ++i) {
            C acc(T(0), T(0));
            for (int k = i; k < bs; ++k) cfma(acc, Tm[i * RW_NB + k], W[k * RW_CW + c]);
            W[i * RW_CW + c] = acc;
          }
        } else {
          for (int i = bs - 1; i >= 0; --i) {
            C acc(T(0), T(0));
            for (int k = 0; k <= i; ++k) cfma(acc, conj(Tm[k * RW_NB + i]), W[k * RW_CW + c]);
            W[i * RW_CW + c] = acc;
          }
        }
      }
      __syncthreads();
      // X[:, chunk] <- X[:, chunk] - V W (rows r0 .. n-1)
      cta_gemm<GemmPlainT<T>, true, true>(
          rows, cw, bs, [&](int q, int i) { return v(r0 + q, i); },
          [&](int i, int c) { return W[i * RW_CW + c]; },
          [&](int q, int c, const C& y) {
            C& x = X[(long long)(r0 + q) * ldx + c0 + c];
            x = x - y;
          },
          gsm);
      __syncthreads();
    }
  }
}



}  // namespace bw
