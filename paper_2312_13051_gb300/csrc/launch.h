// Internal launch interface between the host runtime and the kernel translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace bw {

// Largest n handled by the shared-memory Jacobi path.
constexpr int SMALL_N_MAX = 32;
// Largest n of the tridiagonal (large-n) path.
constexpr int LARGE_N_MAX = 4096;
// Largest p handled by the shared-memory loop kernels (Wilson matrix p x p).
constexpr int LOOP_P_MAX = 64;
// Distinct translations whose phases are cached in shared memory per k-point.
constexpr int PHASE_CACHE = 256;
// Distinct translations the one-thread-per-k-point path keeps per thread.
constexpr int TINY_R_MAX = 16;

struct StatesArgs {
  DevModel model;
  const int* row_ptr;   // n + 1: first plan entry of each row (entries sorted by row)
  DevPlane plane;       // used when f == nullptr
  const double* f;      // optional explicit k-points (K x 3)
  long long K;
  int p;                // occupied bands
  int mixed;            // 0: FP64 Jacobi, 1: FP32 Jacobi + FP64 refinement
  int max_sweeps;
  double gap_tol;
  // projected spin operator (optional)
  DevOp op;             // op.nnz == 0: no spin split
  int sign;
  double pso_gap_tol;
  int pso_median;       // sector = the p/2 lowest / highest PSO eigenvalues (split at the median)
  // outputs
  z64* U;               // K x n x p_out
  double* gap;          // K
  double* pso_evals;    // K x p (optional)
  double* pso_gap;      // K (optional)
  DevStatus* status;
  int want_df;          // write U as complex double-float (states_df_eligible() holds)
};

struct EighArgs {
  const z64* H;               // packed
  const long long* h_off;     // batch: offset of matrix b in z64 units
  const int* n_per;           // batch
  const long long* e_off;     // batch: offset into evals (doubles)
  const long long* v_off;     // batch: offset into evecs (z64)
  long long batch;
  int n_vec;
  int mixed;
  int max_sweeps;
  double* evals;
  z64* evecs;
  DevStatus* status;
};

struct BuildArgs {
  DevModel model;
  const double* f;  // K x 3
  long long K;
  int complex64;
  void* H;
};

struct LoopArgs {
  const z64* U;          // K x n x p
  z64* M;                // K x p x p (overlap scratch)
  int n, p, N, N_t;
  int unitarise;
  int max_sweeps;
  const double* gap;     // K (optional)
  const double* pso_gap; // K (optional)
  double* phases;        // N_t x p
  double* min_gap;       // N_t (optional)
  double* min_pso_gap;   // N_t (optional)
  // nested
  int nested;
  double cut;
  int first, m;
  double wannier_gap_tol;
  z64* w;                // N x N_t x n x m
  z64* nu_buf;           // N x N_t x p x m transported sector bases (sequential loop path), or NULL
  double* min_wannier_gap;  // N_t (optional)
  double* nested_out;    // N_s x N x m
  DevStatus* status;
  int N_s;               // planes stacked along the rows (N_t = N_s x rows per plane; 0 or 1: one)
  int u_df;              // U and w hold complex double-float (loops_accept_df() holds)
  int df_overlaps;       // mixed request: overlaps from the FP64 states in double-float
};

// Raises a kernel's dynamic shared-memory limit only when a launch needs more than
// any earlier one (so repeated and captured launches make no attribute call).
template <typename Kern>
inline cudaError_t set_smem_once(Kern kernel, size_t bytes, size_t& cached) {
  if (bytes <= cached) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes));
  if (e == cudaSuccess) cached = bytes;
  return e;
}

// Large-n occupied states over a wave of W k-points starting at k0 (see large.cu).
struct LargeArgs {
  DevModel model;
  DevPlane plane;
  const double* f;        // optional explicit k-points (K x 3)
  int n, p;
  int nval;               // eigenvalues of T' computed (>= p + 1 when p < n)
  int nvec;               // eigenvectors of T' computed
  int nbt;                // columns back-transformed (mixed: p + 1 when p < n)
  long long k0, W;
  long long kstride;      // k-point of wave slot kw: k0 + kw * kstride (0 means 1)
  int mixed;
  double gap_tol;
  // wave scratch
  void* A;                // W x n x n complex (T)
  void* dg;               // W x n (T)
  void* od;               // W x n (T)
  void* Dp;               // W x n complex (T)
  void* lam;              // W x nval (T)
  void* Z;                // W x n x nvec (T), row-major
  void* work;             // 6 n x (W nvec) (T), interleaved across threads
  void* X;                // W x n x nbt complex float (mixed)
  z64* Hent;              // W x n_ent (mixed): each slot holds the FP64 entry as two floats (hi, lo)
  z64* R64;               // W x n x p (mixed)
  c32* C32;               // W x n x p (mixed)
  z64* G64;               // W x p x p (mixed)
  const int* row_ptr;     // n + 1: first entry of each row in the plan
  // outputs
  z64* U;                 // W x n x p (wave-relative)
  double* gap;            // K (absolute k)
  DevStatus* status;
  // optional host callback after each stage launch (per-stage timing)
  void (*mark)(void*, const char*);
  void* mark_user;
  // explicit Hermitian matrices instead of a model (batched eigensolve): wave slot kw
  // holds matrix idx[k0 + kw] at Hin + h_off[that] (lower triangle read); the
  // refinement uses the dense matrix, and gap[k0 + kw] receives its gap
  const z64* Hin;
  const long long* h_off;
  const int* idx;
  int no_refine;          // mixed path without a block to refine (p = 0)
  int subspace_only;      // only the span of the nvec vectors matters (parallel clusters)
};

// Outputs of the batched eigensolve for one wave of the large path.
struct EighScatterArgs {
  const int* idx;         // wave slot -> matrix index (from idx + k0)
  long long k0, W;
  int n, nval, p, mixed;
  const void* lam;        // W x nval (T)
  const z64* U;           // W x n x p (refined / back-transformed block)
  const double* ritz;     // W x p (mixed: FP64 Ritz values), or NULL
  const long long* e_off;
  const long long* v_off;
  double* evals;
  z64* evecs;             // NULL: values only
};

// FP64 Rayleigh-Ritz of the refined block of explicit matrices (p <= 64):
// U <- U V, ritz = eigenvalues of U^dag H U (ascending).
cudaError_t launch_eigh_ritz(const LargeArgs& a, double* ritz, cudaStream_t s);
cudaError_t launch_eigh_scatter(const EighScatterArgs& e, cudaStream_t s);

// Batched complex GEMM C_b = op(A_b) B_b (row-major; op(A) is A or A^dagger), m x n
// result, inner dimension k; batch b (b = kfirst + the launch's batch index) uses
// A + b' sA, B + b sB, C + (b - kfirst) sC, where b' = b, or with a_next_N > 0 the next
// k-point of the same loop, (b / N) N + (b % N + 1) % N, or with a_mod > 0
// (b + a_shift) % a_mod (the k-point of the next transverse row).
struct GemmArgs {
  const z64* A;
  const z64* B;
  z64* C;
  int m, n, k;
  int opA;                // 0: A (m x k), 1: A^dagger (A stored k x m)
  long long lda, ldb, ldc;
  long long sA, sB, sC;
  long long a_next_N;
  long long batch;
  long long b0;           // first batch index of this launch (set by launch_zgemm)
  long long kfirst;       // absolute index of batch 0 for A and B (C stays relative)
  long long a_shift, a_mod;
};

// Eigenphases of nl Wilson matrices W (p x p, stride sW), loops i0 .. i0+nl-1.
struct BigEigArgs {
  z64* W;
  long long sW;
  int p, nl, i0, N;
  const double* gap;      // K (absolute k = i N + j)
  const double* pso_gap;  // K (spin-resolved loop), or NULL
  double* phases;         // N_t x p
  double* min_gap;        // N_t (optional)
  double* min_pso_gap;    // N_t (optional)
  z64* lam;               // nl x p scratch
  z64* vec;               // nl x p scratch
  double* th;             // nl x p scratch
  int* ord;               // nl x p scratch
  double* ctl;            // nl x 8 scratch (control block of the cluster solver)
  int df;                 // W (and lam) hold complex double-float: the cluster solver in
                          // double-float arithmetic (needs geig_df_eligible(p))
  DevStatus* status;
};
// True when the cluster eigenphase solver takes p (p >= 128); the double-float form
// (BigEigArgs::df) needs it.
bool geig_df_eligible(int p);

// Spin-resolved loop with many occupied bands (bigloop.cu).
// Y = sigma s U for a wave of W occupied blocks (n x p each), s a sparse operator in
// CSR form (rowp n + 1, col, val).
cudaError_t launch_spin_apply(const z64* U, z64* Y, long long W, int n, int p, const int* rowp,
                              const int* col, const z64* val, double sigma, cudaStream_t s);
// From the ascending eigenvalues nu (W x nval) of sigma S_occ per wave slot: the PSO
// eigenvalues mu = sigma nu ascending into pso_evals (K x p, optional, needs nval = p),
// the PSO gap into pso_gap[k] and BW_EPSOGAP unless it exceeds tol (h = p / 2): split
// at zero, gap min |nu_{h-1}|, |nu_h| and nu_{h-1} < 0 < nu_h required; split at the
// median (median != 0), gap nu_h - nu_{h-1}.
cudaError_t launch_pso_post(const double* nu, int nval, long long W, long long k0, int p,
                            double sigma, double tol, int median, double* pso_evals, double* pso_gap,
                            DevStatus* status, cudaStream_t s);

// off[t] = t stride, idx[t] = t for t < W (wave slot -> explicit matrix).
cudaError_t launch_iota(long long* off, int* idx, long long W, long long stride, cudaStream_t s);

// df: A, B and C hold complex double-float (cdf) instead of complex FP64.
cudaError_t launch_zgemm(const GemmArgs& g, cudaStream_t s, bool df = false);
// In place, count elements: complex FP64 -> complex double-float (to_cdf) or back.
cudaError_t launch_convert_cdf(z64* x, long long count, bool to_cdf, cudaStream_t s);
cudaError_t launch_geig_big(const BigEigArgs& a, cudaStream_t s);

// Launches every stage of the large-n solver for one wave.
cudaError_t launch_states_large(const LargeArgs& a, cudaStream_t s);

// Plaquette Berry flux of the states in a.U (K x n x p, p <= 64): link determinants
// (Lx, Ly: K unit complex numbers each, scratch), flux (N_t x N) and chern = sum / 2pi
// (device double); a.min_gap / a.min_pso_gap per transverse row from a.gap / a.pso_gap.
cudaError_t launch_plaquettes(const LoopArgs& a, z64* Lx, z64* Ly, double* flux, double* chern,
                              cudaStream_t s);

// Plaquette flux from precomputed link phases Lx, Ly (K unit complex numbers each):
// flux (N_t x N), chern = sum / 2pi, and a.min_gap / a.min_pso_gap per transverse row.
cudaError_t launch_plaquette_flux(const LoopArgs& a, const z64* Lx, const z64* Ly, double* flux,
                                  double* chern, cudaStream_t s);

// Plaquette Berry flux for p > 64 (bigloop.cu): link matrices of kb k-points at a time
// by the batched GEMM into Lmat (kb x p x p scratch), the phase of each determinant by
// LU with partial pivoting (one CTA per matrix), then launch_plaquette_flux.
cudaError_t launch_plaquettes_big(const LoopArgs& a, z64* Lmat, long long kb, z64* Lx, z64* Ly,
                                  double* flux, double* chern, cudaStream_t s);

// Phase of det(A_b) for nb p x p matrices (stride sA, overwritten by their LU factors).
cudaError_t launch_det_phase(z64* A, long long sA, int p, long long nb, z64* out, cudaStream_t s);

// Winding of the summed Wannier centres over the transverse direction (Eq. 6).
// Maximum errors of the double-float unit-circle helpers against FP64 (err: 3 device
// doubles, zeroed by the caller).
cudaError_t launch_selftest_unit_circle(double* err, cudaStream_t s);
cudaError_t launch_winding(const double* phases, int Nt, int p, double* sums, double* winding,
                           cudaStream_t s);

// Z2 index of a plane from its WCC spectrum (wcc.cu): rows 0 .. Nt / 2 of phases
// (Nt x p, each row ascending in [-pi, pi]); mid / width (Nt / 2 + 1) and crossings
// (Nt / 2) are written; *nu = total crossings mod 2, or -1 when a row was rejected
// (also reported as ST_EINVAL with the row index).
cudaError_t launch_z2(const double* phases, int Nt, int p, double* mid, double* width, int* crossings,
                      int* nu, DevStatus* status, cudaStream_t s);

cudaError_t launch_build_hk(const BuildArgs& a, cudaStream_t s);
cudaError_t launch_states_small(const StatesArgs& a, int p_out, cudaStream_t s);
cudaError_t launch_states_tiny(const StatesArgs& a, int p_out, cudaStream_t s, bool* handled);
// True when the mixed-precision double-float states kernel (n = 4) can serve the
// problem; with want_df set it writes U as complex double-float.
bool states_df_eligible(const StatesArgs& a, int p_out);
cudaError_t launch_eigh_small(const EighArgs& a, int n_max, cudaStream_t s);
// True when the loop kernel forms the overlaps itself (launch_overlaps then does nothing).
bool loops_form_overlaps(const LoopArgs& a);
cudaError_t launch_overlaps(const LoopArgs& a, cudaStream_t s);
cudaError_t launch_loops(const LoopArgs& a, cudaStream_t s);
cudaError_t launch_nested(const LoopArgs& a, cudaStream_t s);
// True when the nested loop kernel only transports the sector bases (into nu_buf)
// and launch_wannier forms the Wannier states.
bool loops_transport_only(const LoopArgs& a);
// True when the scan kernels serve both loops (no unitarised overlaps): they then
// also accept U in complex double-float (u_df).
bool loops_accept_df(const LoopArgs& a);
// Mixed precision, n = 4, p = 2, N <= 64 with the scan kernels: one kernel solves each
// loop's states and runs the loop (replaces launch_states_small + launch_loops; sa as
// for launch_states_small with want_df, a as for launch_loops with u_df).
bool loops_fused_eligible(const LoopArgs& a, const DevModel& md);
// *nested_done: the launch also ran the nested loops (one Wannier band, cooperative
// launch with the whole grid resident), so launch_nested must not run.
// plan_host (optional, at most FUSED_PLAN_BYTES): the hopping-list plan whose device
// copy sa.model / sa.row_ptr point into at plan_dev; the launch then carries the plan
// as a kernel parameter and nothing needs to be copied to plan_dev.
constexpr int FUSED_PLAN_BYTES = 2048;
struct alignas(16) FusedPlan {
  unsigned char bytes[FUSED_PLAN_BYTES];
};
cudaError_t launch_loops_fused_df(const StatesArgs& sa, const LoopArgs& a, cudaStream_t s,
                                  bool* nested_done, const void* plan_host = nullptr,
                                  size_t plan_bytes = 0, const void* plan_dev = nullptr);
// Orthonormalised Wannier states w from the transported bases in nu_buf (no-op without).
cudaError_t launch_wannier(const LoopArgs& a, cudaStream_t s);

}  // namespace bw
