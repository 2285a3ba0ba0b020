// Fifth-generation tensor cores (tcgen05, sm_103a) for the complex FP32 GEMMs of the
// large-n solver: operands staged by the CTA into shared memory, one thread issues
// tcgen05.mma, the accumulator lives in tensor memory (TMEM) and is read back with
// tcgen05.ld.
//
// A complex product C = A B (m x n, inner dimension k) runs as one real product of the
// embedding
//     [ Re A  -Im A ]   [ Re B ]     [ Re C ]
//     [ Im A   Re A ] x [ Im B ]  =  [ Im C ],
// so a 64 x 64 complex tile is a 128 x 64 real tile (M = 128 rows of TMEM lanes, 64
// columns).  FP32 accuracy from bf16 tensor cores: every operand is split into three
// bf16 pieces x = x0 + x1 + x2 (x0 = bf16(x), x1 = bf16(x - x0), x2 = bf16(x - x0 - x1);
// the differences are exact in FP32, and 3 x 8 significant bits hold an FP32
// significand), and every product keeps the eight terms a_i b_j with i + j <= 3
// (smallest first); the one dropped term, a2 b2, is ~2^-48 relative.  The products of
// bf16 values are exact.  Each chunk of 32 real terms is accumulated in TMEM in two
// accumulators, the seven cross products (smallest first) in one and a0 b0 alone in
// the other, so that no small term is added into a full-size sum inside the tensor
// core; the two are then added into FP32 registers.
//
// Shared-memory layout of a tile (no swizzle, K-major): rows in groups of 8, each group
// holding its K range as consecutive 8-row x 16-byte core matrices (8 bf16 per row).  The
// matrix descriptor's leading byte offset (LBO) is the distance between core matrices
// adjacent along K (128 bytes), its stride byte offset (SBO) the distance between 8-row
// groups (512 bytes: a chunk's 32 K values are four core matrices).
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

#include "common.cuh"

namespace bw {
namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = uint64_t((addr >> 4) & 0x3FFFu);
  d |= uint64_t((lbo >> 4) & 0x3FFFu) << 16;
  d |= uint64_t((sbo >> 4) & 0x3FFFu) << 32;
  d |= uint64_t(1) << 46;  // descriptor version; base offset 0, no swizzle
  return d;
}

// Instruction descriptor of kind::f16 with bf16 A and B and an FP32 accumulator, both
// operands K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(N >> 3) << 17) | (uint32_t(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

// The mbarrier completes once every MMA this thread issued before has finished.
__device__ __forceinline__ void commit(uint64_t* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
      smem_u32(mbar)));
}

__device__ __forceinline__ void mbar_init(uint64_t* mbar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)));
  asm volatile("fence.mbarrier_init.release.cluster;");
}

// Waits for the phase with the given parity, at most max_iter polls; false on time-out.
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity, int max_iter) {
  for (int it = 0; it < max_iter; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(mbar)), "r"(parity));
    if (ok) return true;
  }
  return false;
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;"); }
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;"); }

// TMEM allocation by one whole warp; the base address lands in *slot (shared memory).
__device__ __forceinline__ void alloc(uint32_t* slot, uint32_t cols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
               "r"(cols));
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}

__device__ __forceinline__ void dealloc(uint32_t tmem, uint32_t cols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(cols));
}

// 16 consecutive FP32 columns of this thread's TMEM lane (warp w of a warpgroup reads
// lanes 32 (w % 4) .. 32 (w % 4) + 31).
__device__ __forceinline__ void ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// x = x0 + x1 + x2 in bf16 (round to nearest; each difference is exact in FP32).
__device__ __forceinline__ void split3(float x, __nv_bfloat16 (&b)[3]) {
  b[0] = __float2bfloat16_rn(x);
  const float r1 = x - __bfloat162float(b[0]);
  b[1] = __float2bfloat16_rn(r1);
  b[2] = __float2bfloat16_rn(r1 - __bfloat162float(b[1]));
}

// Byte offset of real element (row, k) of a tile with 32 bf16 values per row (4 core
// matrices along K; SBO = 512).
__device__ __forceinline__ int off16(int row, int k) {
  return (row >> 3) * 512 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

constexpr int TILE = 64;                  // complex rows / columns per output tile
constexpr int KC = 16;                    // complex inner-dimension chunk (32 real)
constexpr int A_BYTES = 128 * 32 * 2;     // one bf16 piece of the embedded A chunk (8 KB)
constexpr int B_BYTES = 64 * 32 * 2;      // one bf16 piece of the embedded B chunk (4 KB)
constexpr size_t SMEM = 3 * A_BYTES + 3 * B_BYTES;  // 36 KB (the epilogue reuses it)
constexpr uint32_t TMEM_COLS = 128;     // two 128 x 64 FP32 accumulators
constexpr int WAIT_POLLS = 1 << 22;

// Per-CTA state: the TMEM base, the MMA-completion barrier and its phase, and whether a
// bounded wait ever gave up (then the CTA stops issuing MMAs).
struct State {
  uint32_t tmem;
  uint64_t* mbar;
  uint32_t phase;
  bool failed;
};

// Sets up a CTA's state: warp 0 allocates TMEM_COLS columns, thread 0 initialises the
// barrier.  slot and mbar live in shared memory.  Every thread calls it.
__device__ inline State setup(uint32_t* slot, uint64_t* mbar) {
  if (threadIdx.x == 0) mbar_init(mbar);
  if ((threadIdx.x >> 5) == 0) alloc(slot, TMEM_COLS);
  fence_before();
  __syncthreads();
  fence_after();
  return State{*slot, mbar, 0u, false};
}

__device__ inline void teardown(const State& s) {
  fence_before();
  __syncthreads();
  fence_after();
  if ((threadIdx.x >> 5) == 0) dealloc(s.tmem, TMEM_COLS);
}

}  // namespace tc

// C(m, c) = sum_k A(m, k) B(k, c), complex FP32 operands, on the tensor cores (see the
// file comment), for m < M, c < Ncol, k < K; la / lb / st as for cta_gemm.  All
// blockDim.x == 256 threads call it; sm holds tc::SMEM bytes, 16-byte aligned.  Returns
// false (and produces no outputs from then on) when an MMA did not complete within the
// bounded wait.
template <bool A_K_CONTIG, bool B_C_CONTIG, class LA, class LB, class ST>
__device__ bool cta_cgemm_tc(int M, int Ncol, int K, LA la, LB lb, ST st, unsigned char* sm, tc::State& s) {
  using namespace tc;
  unsigned char* Ap = sm;                    // pieces 0, 1, 2 of the embedded A chunk
  unsigned char* Bp = sm + 3 * A_BYTES;      // pieces 0, 1, 2 of the embedded B chunk
  // 128 x 64 FP32 epilogue staging, rows padded to 65 (33 KB over the operand buffers,
  // which are free once the tile's MMAs have completed)
  float* Dst = reinterpret_cast<float*>(sm);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // this thread's accumulators: TMEM lane 32 (warp % 4) + lane, columns col0 .. col0 + 31
  const int row = 32 * (warp & 3) + lane, col0 = 32 * (warp >> 2);
  const uint32_t taddr = s.tmem + (uint32_t(32 * (warp & 3)) << 16) + uint32_t(col0);
  constexpr uint32_t IDESC = idesc_bf16(128, 64);
  constexpr int PER = KC * TILE / 256;  // complex elements of each operand per thread per chunk
  for (int m0 = 0; m0 < M; m0 += TILE)
    for (int c0 = 0; c0 < Ncol; c0 += TILE) {
      if (s.failed) return false;
      float acc[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) acc[j] = 0.f;
      for (int k0 = 0; k0 < K; k0 += KC) {
#pragma unroll
        for (int q = 0; q < PER; ++q) {
          const int e = tid + 256 * q;
          int kk, mm;
          if (A_K_CONTIG) {
            mm = e / KC;
            kk = e - mm * KC;
          } else {
            kk = e / TILE;
            mm = e - kk * TILE;
          }
          const c32 a = (m0 + mm < M && k0 + kk < K) ? la(m0 + mm, k0 + kk) : c32(0.f, 0.f);
          __nv_bfloat16 re[3], im[3];
          split3(a.re, re);
          split3(a.im, im);
#pragma unroll
          for (int t = 0; t < 3; ++t) {
            unsigned char* P = Ap + t * A_BYTES;
            *reinterpret_cast<__nv_bfloat16*>(P + off16(mm, kk)) = re[t];
            *reinterpret_cast<__nv_bfloat16*>(P + off16(mm, KC + kk)) = __hneg(im[t]);
            *reinterpret_cast<__nv_bfloat16*>(P + off16(TILE + mm, kk)) = im[t];
            *reinterpret_cast<__nv_bfloat16*>(P + off16(TILE + mm, KC + kk)) = re[t];
          }
          int cc;
          if (B_C_CONTIG) {
            kk = e / TILE;
            cc = e - kk * TILE;
          } else {
            cc = e / KC;
            kk = e - cc * KC;
          }
          const c32 b = (c0 + cc < Ncol && k0 + kk < K) ? lb(k0 + kk, c0 + cc) : c32(0.f, 0.f);
          split3(b.re, re);
          split3(b.im, im);
#pragma unroll
          for (int t = 0; t < 3; ++t) {
            unsigned char* P = Bp + t * B_BYTES;
            *reinterpret_cast<__nv_bfloat16*>(P + off16(cc, kk)) = re[t];
            *reinterpret_cast<__nv_bfloat16*>(P + off16(cc, KC + kk)) = im[t];
          }
        }
        fence_async_smem();
        fence_before();
        __syncthreads();
        fence_after();
        if (tid == 0) {
          // pieces (i, j) with i + j <= 3: the seven cross products, smallest first, into
          // the first accumulator; a0 b0 alone into the second (columns 64 ..)
          constexpr int PI[8] = {1, 2, 0, 1, 2, 0, 1, 0}, PJ[8] = {2, 1, 2, 1, 0, 1, 0, 0};
          const uint32_t a0 = smem_u32(Ap), b0 = smem_u32(Bp);
#pragma unroll
          for (int t = 0; t < 8; ++t)
#pragma unroll
            for (int ks = 0; ks < 2; ++ks) {  // 16 real K values (two core matrices) per MMA
              const uint32_t o = ks * 256;
              const bool big = t == 7;
              mma_bf16(s.tmem + (big ? 64u : 0u), smem_desc(a0 + PI[t] * A_BYTES + o, 128, 512),
                       smem_desc(b0 + PJ[t] * B_BYTES + o, 128, 512), IDESC,
                       (big ? ks : (ks | t)) ? 1u : 0u);
            }
          commit(s.mbar);
        }
        // every thread waits for the chunk's MMAs before its shared memory is restaged
        const bool ok = mbar_wait(s.mbar, s.phase, WAIT_POLLS);
        s.phase ^= 1u;
        fence_after();
        if (!__syncthreads_and(ok)) {
          s.failed = true;
          return false;
        }
        // the chunk's partial sums into the FP32 register accumulators
        float v[16], w[16];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          ld16(taddr + uint32_t(16 * h), v);
          ld16(taddr + 64u + uint32_t(16 * h), w);
#pragma unroll
          for (int j = 0; j < 16; ++j) acc[16 * h + j] += w[j] + v[j];
        }
        fence_before();
        __syncthreads();  // TMEM read before the next chunk's first MMA overwrites it
        fence_after();
      }
      // epilogue: registers -> shared staging -> st (real part in row m, imaginary in 64 + m)
#pragma unroll
      for (int j = 0; j < 32; ++j) Dst[row * 65 + col0 + j] = acc[j];
      __syncthreads();
      for (int e = tid; e < TILE * TILE; e += 256) {
        const int mm = e / TILE, cc = e - mm * TILE;
        if (m0 + mm < M && c0 + cc < Ncol) st(m0 + mm, c0 + cc, c32(Dst[mm * 65 + cc], Dst[(TILE + mm) * 65 + cc]));
      }
      __syncthreads();
    }
  return true;
}

}  // namespace bw
