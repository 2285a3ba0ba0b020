/*
 * berrywl.h -- C ABI of the GB300 (sm_103a) Wilson-loop library.
 *
 * The library computes Wannier-centre charges by discretised, path-ordered Wilson
 * loops (arXiv 2312.13051, Sec. II A, Eq. 2), hybrid Wannier centres over a plane
 * (Sec. II B, Eq. 3), the nested Wilson loop on a Wannier-band subspace (Sec. III,
 * Eq. 8) and the spin-resolved Wilson loop of a projected-spin-operator sector
 * (Sec. IV), for tight-binding models given as hopping lists.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Complex numbers are bw_c128 {re, im} (FP64), or {float re, im} where stated.
 *  - Matrices are row-major.  An eigenvector block U (n x p) stores U[r*p + c]
 *    (row r = orbital, column c = band), like numpy's V[:, :p].
 *  - The model (hopping list) and the spin operator are HOST arrays, read during
 *    the call: the library turns the list into its own device plan.  A context keeps
 *    a copy of the last list with its plan and reuses the plan while a later call
 *    passes an identical list (compared entry by entry, so edits in place are seen).
 *    Every other array argument is a DEVICE pointer owned by the caller.
 *  - Calls are asynchronous on `stream` (a cudaStream_t; NULL = legacy default
 *    stream).  The return value reports argument errors and launch failures only.
 *    Numerical conditions found on the device (closed gap, PSO gap, Wannier gap,
 *    no convergence) go to a sticky per-context status word; read it with
 *    bw_get_status(), which synchronises the stream.
 *  - Scratch memory comes from a per-context device arena bounded by the context's
 *    memory budget (BW_ENOMEM beyond it).  One context must not be used from two
 *    host threads at once; calls on different streams are ordered by the context.
 *  - Calls may be captured into a CUDA graph once the same call has run uncaptured on
 *    the context (so that its arena and staging buffer are large enough).  A replay
 *    re-reads the hopping list from the context's pinned staging buffer, so no other
 *    call may be issued on that context while its graphs are being replayed.
 *  - There is no CPU fallback: every numerical step runs in the library's CUDA
 *    kernels.  Without a usable CUDA device bw_create() fails with BW_ECUDA.
 */
#ifndef BERRYWL_H
#define BERRYWL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bw_ctx bw_ctx;

typedef enum {
  BW_OK = 0,
  BW_EINVAL = 1,    /* bad argument, non-Hermitian list, unsupported size          */
  BW_ENOMEM = 2,    /* scratch would exceed the context's memory budget            */
  BW_EGAP = 3,      /* direct gap lam_p - lam_{p-1} <= gap_tol at some k           */
  BW_EPSOGAP = 4,   /* PSO sector size != p/2, or min |PSO eigenvalue| <= tol      */
  BW_EWANGAP = 5,   /* Wannier (phase) gap around the nested sector <= tol         */
  BW_ENOCONV = 6,   /* an iterative eigensolver hit its iteration cap              */
  BW_ETIMEOUT = 7,  /* a bounded device-side wait gave up                          */
  BW_ECUDA = 8,     /* CUDA runtime error                                          */
  BW_ECANCELED = 9  /* request withdrawn before it ran (bw_server_cancel)          */
} bw_status;

typedef enum {
  BW_FP64 = 0,      /* every step in FP64                                          */
  BW_MIXED = 1      /* eigensolve in FP32, occupied block refined in FP64          */
} bw_precision;

typedef struct { double re, im; } bw_c128;

/* Tight-binding model, full hopping list (HOST arrays):
 *   H(f) = sum_e t[e] exp(i 2 pi f . R[e]) |i[e]><j[e]|
 * f in fractional reciprocal coordinates, R[e] integer translations (nnz x 3).
 * Every (i, j, R, t) must come with (j, i, -R, conj t); the list is checked and
 * rejected with BW_EINVAL when H(f) would not be Hermitian.  No orbital-position
 * phases are applied, so H(f + G) = H(f) for integer G (Sec. II A, periodic
 * condition psi(k) = psi(k + 2 pi / a)). */
typedef struct {
  int32_t n;              /* orbitals per (super)cell, >= 1                        */
  int64_t nnz;            /* entries in the list, >= 0                              */
  const int32_t* R;       /* nnz x 3                                                */
  const int32_t* i;       /* nnz, 0 <= i < n                                        */
  const int32_t* j;       /* nnz, 0 <= j < n                                        */
  const bw_c128* t;       /* nnz                                                    */
} bw_model;

/* Plane of k-points (Sec. II B, vec(t1, t2) in units of the reciprocal vectors):
 *   f(j, i) = origin + (j / N) loop_dir + (i / N_t) trans_dir,  j < N, i < N_t.
 * loop_dir is an integer vector so each loop closes on the k-point it started from
 * (Eq. 2); the loop reuses the eigenvectors of j = 0 at j = N.  For the nested loop
 * trans_dir must be an integer vector as well (closure along the second direction).
 * k-point index k = i * N + j. */
typedef struct {
  double origin[3];
  int32_t loop_dir[3];
  double trans_dir[3];
  int32_t N;              /* points per loop, >= 1                                  */
  int32_t N_t;            /* transverse points, >= 1                                */
} bw_plane;

/* A stack of N_s parallel planes (Sec. III: the nested loop as a function of k_z;
 * Sec. II B: the weak and strong Z2 indices of a 3D crystal from the planes k_a = 0 and
 * k_a = 1/2): plane s, 0 <= s < N_s, is `plane` with its origin moved by
 * (s / N_s) sweep_dir,
 *   f(j, i, s) = origin + (j / N) loop_dir + (i / N_t) trans_dir + (s / N_s) sweep_dir.
 * sweep_dir is an integer reciprocal vector (N_s planes over one period; N_s = 2 with
 * sweep_dir = e_z gives k_z = 0 and k_z = 1/2).  Every plane's loops run in the same
 * launches.  Outputs are plane-major: row s N_t + i of a per-row output belongs to
 * transverse point i of plane s; k-point index k = (s N_t + i) N + j. */
typedef struct {
  bw_plane plane;         /* plane s = 0; N_t transverse points per plane              */
  int32_t sweep_dir[3];
  int32_t N_s;            /* planes, >= 1                                             */
} bw_plane_stack;

/* Options.  A negative tolerance selects the default. */
typedef struct {
  double gap_tol;         /* direct gap; default 1e-6 * max(1, max|t|)              */
  double pso_gap_tol;     /* min |PSO eigenvalue|; default 1e-6                     */
  double wannier_gap_tol; /* phase gap around the nested sector; default 1e-6 rad   */
  int32_t unitarise;      /* 1: replace each overlap by its unitary polar factor    */
  int32_t max_sweeps;     /* Jacobi sweep cap; 0 = default (30)                     */
  int32_t pso_split;      /* PSO sector (Sec. IV): 0 = the eigenvalues of sign `sign`
                             (split at zero, p/2 of them required; gap min |mu|);
                             1 = the p/2 lowest (sign -1) or highest (+1) eigenvalues
                             (split at the median; gap mu_{p/2} - mu_{p/2-1})      */
} bw_opts;

/* Context: binds device `device`, allocates nothing yet.  mem_budget_bytes bounds
 * the scratch arena (0 = 90% of the device's free memory at creation). */
bw_status bw_create(bw_ctx** out, int device, size_t mem_budget_bytes);
void bw_destroy(bw_ctx* ctx);

/* Message of the last failure on this context (argument error or device status,
 * with the failing k index).  Valid until the next call on the context. */
const char* bw_last_error(const bw_ctx* ctx);

/* Synchronises `stream`, returns and clears the sticky device status of the calls
 * issued so far (BW_OK, BW_EGAP, BW_EPSOGAP, BW_EWANGAP or BW_ENOCONV).  When
 * k_index is non-NULL it receives the first failing k-point index (or -1). */
bw_status bw_get_status(bw_ctx* ctx, void* stream, int64_t* k_index);

/* Per-kernel timing.  With profiling enabled, CUDA events are recorded around every
 * kernel launch of each call (as external events under stream capture, so replays of
 * a captured graph are timed as well).  No paper counterpart: measurement only. */
bw_status bw_set_profiling(bw_ctx* ctx, int enable);

/* Self-test of the double-float unit-circle arithmetic that the mixed four-band loop
 * kernel uses in place of FP64 transcendentals (phase tables e^{2 pi i m / N}, Bloch
 * factors e^{i pi t}, eigenphases arg z): runs it on the device against the FP64
 * sincospi / atan2 of the CUDA math library and writes three maximum absolute errors
 * to max_err (host, 3 doubles): e^{2 pi i m / N} for 1 <= N <= 64, 0 <= m < N;
 * e^{i pi t} on 8192 points of [-3, 3); arg z (circular distance, radians) on 4096
 * angles x radii 0.5, 1, 2.  Synchronous.  No paper counterpart: verification only. */
bw_status bw_selftest_unit_circle(bw_ctx* ctx, double* max_err);

/* Waits for the last timing event of the most recent profiled call (or replay) and
 * writes up to `max` kernel names (32 bytes each, NUL-terminated; may be NULL) and
 * durations in milliseconds (may be NULL).  Returns the count, -1 on error. */
int bw_profile_read(bw_ctx* ctx, int max, char* names, double* ms);

/* Step 1, Bloch Hamiltonian (Sec. I: H(k) from the hopping list).
 * f: DEVICE, K x 3 doubles.  H_out: DEVICE, K x n x n complex, complex128
 * (complex64 = 0) or complex64 pairs of floats (complex64 = 1). */
bw_status bw_build_hk(bw_ctx* ctx, const bw_model* model, const double* f, int64_t K,
                      int complex64, void* H_out, void* stream);

/* Step 2, exact diagonalisation (Sec. I), batched with uneven sizes.
 * H: DEVICE, matrices packed back to back (matrix b holds n_per[b]^2 complex128,
 * row-major, Hermitian; for n > 32 only the lower triangle is read, for n <= 32 the
 * full matrix).  n_per: HOST, batch sizes.  evals: DEVICE, sum(n_per)
 * doubles, ascending per matrix.  evecs: DEVICE, sum(n_per[b] * n_vec) complex128,
 * matrix b's lowest n_vec eigenvectors as an n x n_vec row-major block (NULL: values
 * only).  BW_MIXED: FP32 solve, lowest n_vec block refined in FP64 (needs
 * n_vec < n and a gap above it; for n > 32 also n_vec <= 64), the other eigenvalues
 * to FP32 accuracy.  n <= 32: one shared-memory Jacobi solve per matrix; n > 32:
 * Householder tridiagonalisation, bisection and inverse iteration, matrices of equal
 * size in waves.  1 <= n <= 4096, 0 <= n_vec <= n. */
bw_status bw_eigh_batched(bw_ctx* ctx, const void* H, const int32_t* n_per, int64_t batch,
                          int32_t n_vec, bw_precision prec, double* evals, void* evecs,
                          void* stream);

/* Hybrid Wannier centres (Sec. II B, Eq. 3, BerryEasy's WSurf): for each transverse
 * index i the Wilson loop along loop_dir of the lowest p bands,
 *   W_i = M_{N-1} ... M_1 M_0,   M_j = U(k_{j+1})^dagger U(k_j),  U(k_N) = U(k_0)
 * (Eq. 2, later k multiplied from the left), and its eigenphases theta in (-pi, pi].
 * phases: DEVICE, N_t x p doubles, ascending per row (xbar = theta / 2pi).
 * min_gap: DEVICE, N_t doubles, min over the loop of lam_p - lam_{p-1} (may be NULL).
 * 1 <= p <= n. */
bw_status bw_wilson_loop(bw_ctx* ctx, const bw_model* model, const bw_plane* plane,
                         int32_t p, bw_precision prec, const bw_opts* opts,
                         double* phases, double* min_gap, void* stream);

/* Nested Wilson loop (Sec. III, Eq. 8, BerryEasy's WNWL).  For each base point
 * k_j of the first loop: the right eigenvectors nu of the loop started at k_j,
 * ordered by phase measured from `cut` (mod 2pi, ascending); the sector
 * [first, first + m) spans the Wannier states w = U(k_j) nu (orthonormalised);
 * their Wilson loop along trans_dir (closed on i = 0) gives the nested phases.
 * phases: DEVICE, N_t x p (first loop, as bw_wilson_loop).  nested: DEVICE, N x m,
 * ascending per base point.  min_wannier_gap: DEVICE, N_t doubles: circular phase
 * distance between the sector and the other phases (may be NULL).  min_gap as in
 * bw_wilson_loop (may be NULL).  1 <= m, 0 <= first, first + m <= p. */
bw_status bw_nested_wilson_loop(bw_ctx* ctx, const bw_model* model, const bw_plane* plane,
                                int32_t p, double cut, int32_t first, int32_t m,
                                bw_precision prec, const bw_opts* opts, double* phases,
                                double* nested, double* min_wannier_gap, double* min_gap,
                                void* stream);

/* Spin-resolved Wilson loop (Sec. IV, BerryEasy's WSpinSurf / spin_spectrum).
 * At each k the projected spin operator restricted to the occupied space,
 * S_occ = U^dagger s U (p x p), is diagonalised; its eigenvectors with eigenvalue
 * of sign `sign` (-1: C_down, +1: C_up) form the sector U_s = U V_s, which must
 * hold p/2 states at every k with min |eigenvalue| > pso_gap_tol (else
 * BW_EPSOGAP).  The Wilson loop of U_s as in bw_wilson_loop.  For n > 32 and
 * p > 64, S_occ is formed by a batched GEMM and diagonalised in FP64 on the
 * tridiagonal path in both precisions, and the loop runs as batched GEMMs.
 * spin_op: HOST, n x n complex128 Hermitian (e.g. diag(1,-1,-1,1) = s3 (x) t3).
 * phases: DEVICE, N_t x p/2.  pso_evals: DEVICE, K x p ascending (may be NULL).
 * min_pso_gap, min_gap: DEVICE, N_t doubles each (may be NULL).  p even. */
bw_status bw_spin_resolved_wilson_loop(bw_ctx* ctx, const bw_model* model,
                                       const bw_plane* plane, int32_t p,
                                       const bw_c128* spin_op, int32_t sign,
                                       bw_precision prec, const bw_opts* opts,
                                       double* phases, double* pso_evals,
                                       double* min_pso_gap, double* min_gap, void* stream);

/* The three loop entry points over a stack of planes (bw_plane_stack): the results of
 * the single-plane calls for every plane, in one pass.  phases: DEVICE, N_s N_t x p
 * (N_s N_t x p/2 for the spin-resolved loop); min_gap, min_wannier_gap, min_pso_gap:
 * DEVICE, N_s N_t (may be NULL); nested: DEVICE, N_s N x m (row s N + j: base point j of
 * plane s; each nested loop closes within its plane); pso_evals: DEVICE, N_s N_t N x p
 * (may be NULL).  Limits and statuses as for the single-plane calls; a NULL stack or
 * N_s < 1 is BW_EINVAL; the device status reports k-point indices k = (s N_t + i) N + j
 * and nested base points s N + j. */
bw_status bw_wilson_loop_stack(bw_ctx* ctx, const bw_model* model, const bw_plane_stack* stack,
                               int32_t p, bw_precision prec, const bw_opts* opts, double* phases,
                               double* min_gap, void* stream);
bw_status bw_nested_wilson_loop_stack(bw_ctx* ctx, const bw_model* model, const bw_plane_stack* stack,
                                      int32_t p, double cut, int32_t first, int32_t m,
                                      bw_precision prec, const bw_opts* opts, double* phases,
                                      double* nested, double* min_wannier_gap, double* min_gap,
                                      void* stream);
bw_status bw_spin_resolved_wilson_loop_stack(bw_ctx* ctx, const bw_model* model,
                                             const bw_plane_stack* stack, int32_t p,
                                             const bw_c128* spin_op, int32_t sign, bw_precision prec,
                                             const bw_opts* opts, double* phases, double* pso_evals,
                                             double* min_pso_gap, double* min_gap, void* stream);

/* Plaquette Berry flux (the coupling-matrix method of BerryEasy's WSpinLine, used in
 * the disordered-quadrupole example of Sec. IV A): the plane's grid is cut into N x N_t
 * plaquettes; plaquette (j, i) has corners k(j, i), k(j+1, i), k(j+1, i+1), k(j, i+1)
 * (both directions close cyclically, so trans_dir must be an integer vector) and its
 * integrated Berry flux is the argument of the determinant of the Wilson loop of the
 * occupied states around it, traversed k(j, i) -> k(j, i+1) -> k(j+1, i+1) ->
 * k(j+1, i) -> k(j, i) with Eq. 2 overlaps; with this orientation the total flux / 2pi
 * equals the Eq. 6 winding of the same states (the Chern number).  With spin_op
 * (HOST, n x n, may be NULL) the states are the PSO sector of sign `sign` as in
 * bw_spin_resolved_wilson_loop, and the total is the spin-Chern number C_down
 * (sign -1) or C_up (+1).
 * flux: DEVICE, N_t x N doubles in (-pi, pi] (row i, column j).  chern: DEVICE, one
 * double, sum(flux) / 2pi (may be NULL).  min_gap, min_pso_gap: DEVICE, N_t doubles
 * per transverse row (may be NULL; min_pso_gap only with spin_op).  Up to 64 bands in
 * the loop (p, or p/2 with a spin operator) each k-point's two link determinants come
 * from overlaps and LU in shared memory; beyond, the link matrices are formed by a
 * batched GEMM in blocks of 256 k-points and each determinant's phase by LU with
 * partial pivoting in global memory (one CTA per matrix). */
bw_status bw_plaquette_flux(bw_ctx* ctx, const bw_model* model, const bw_plane* plane, int32_t p,
                            const bw_c128* spin_op, int32_t sign, bw_precision prec,
                            const bw_opts* opts, double* flux, double* chern, double* min_gap,
                            double* min_pso_gap, void* stream);

/* Winding of the hybrid Wannier centres over the transverse direction (Sec. II B,
 * Eq. 6: C = sum_n xbar_n(k_y = 2 pi) - sum_n xbar_n(k_y = 0), in units of the
 * lattice constant).  For the rows of `phases` (N_t x p, as written by the loop
 * entry points, theta in radians) s_i = sum_c theta[i][c] / 2pi, and the winding is
 * sum_i wrap(s_{i+1} - s_i) over the cyclic transverse grid (row N_t - 1 steps to
 * row 0), wrap(d) = d - rint(d).  It is the Chern number of the loop's bands (of the
 * PSO sector for the spin-resolved loop) when the grid resolves each step of the
 * summed centre to less than half a lattice constant; the result is an integer up to
 * rounding.  phases: DEVICE.  sums: DEVICE, N_t doubles (may be NULL).  winding:
 * DEVICE, one double.  Asynchronous on `stream`; no scratch memory. */
bw_status bw_winding(bw_ctx* ctx, const double* phases, int32_t N_t, int32_t p, double* sums,
                     double* winding, void* stream);

/* Z2 index of a time-reversal-symmetric plane from the connectivity of its hybrid
 * Wannier centres (Sec. II B after Eq. 7: the WCCs of a non-trivial plane run across
 * the whole cell between the time-reversal-invariant lines t2 = 0 and t2 = 1/2;
 * Sec. II C reads it for supercells with vacancies; the weak and strong indices of a
 * 3D crystal are those of its high-symmetry planes).  The connectivity is read by the
 * largest-gap construction of Soluyanov and Vanderbilt (Phys. Rev. B 83, 235401
 * (2011)):
 *   x = theta / 2pi, plus 1 when negative;
 *   for rows i = 0 .. N_t/2 the widest circular gap between the sorted x (gaps
 *   x[q+1] - x[q], then (x[0] + 1) - x[p-1]; the first widest wins a tie) and its
 *   midpoint z_i = x[q] + gap/2 (minus 1 when it reaches 1), in FP64;
 *   crossings[i] = the number of x of row i + 1 strictly between z_i and z_{i+1};
 *   nu = sum of crossings mod 2.
 * The reading is a heuristic on a finite grid: it needs the midpoint to move less than
 * the WCCs around it between rows (refine N_t when `width` gets small).
 * phases: DEVICE, N_t x p as the loop entry points write them (row i at t2 = i / N_t,
 * each row ascending in [-pi, pi]); N_t even, p >= 1; rows 0 .. N_t/2 are read.
 * nu: DEVICE, one int32: 0 or 1, or -1 when a row is not ascending in [-pi, pi] (then
 * the device status is BW_EINVAL with the row index; bw_get_status reports it).
 * crossings: DEVICE, N_t/2 int32 (may be NULL).  mid, width: DEVICE, N_t/2 + 1
 * doubles, the midpoint and the width of each row's widest gap (may be NULL; NULL
 * outputs take scratch from the context).  Asynchronous on `stream`. */
bw_status bw_z2_largest_gap(bw_ctx* ctx, const double* phases, int32_t N_t, int32_t p, int32_t* nu,
                            int32_t* crossings, double* mid, double* width, void* stream);

/* Allocation-free Wilson loop (no counterpart in the paper: it serves callers).
 * Some callers cannot let a library allocate device memory: programs that give all
 * device memory to their own pool under a hard cap, plugins running inside another
 * program's CUDA context, or latency-critical loops where cudaMalloc / cudaFree
 * would block on or synchronise the device.  This entry point computes the Wilson
 * loop of bw_wilson_loop (same arguments and outputs, no context) without
 * allocating: all scratch lives in one fixed 8 MiB device array inside the library,
 * which every GPU that loads the library holds until the process exits.
 *  - BW_FP64 runs the kernels bw_wilson_loop runs and gives the same results bit for
 *    bit.  BW_MIXED runs the FP32 solve with FP64 refinement and FP64 overlaps (not
 *    the double-float kernels bw_wilson_loop uses where they apply), so mixed results
 *    agree with bw_wilson_loop within the mixed-precision tolerance (both within
 *    1e-6 rad of the FP64 result), not bit for bit.
 *  - The problem must fit in the array: 16 K n p + 8 K bytes (K = N * N_t) plus the
 *    hopping-list plan, plus 16 K p^2 bytes for the overlaps when the loop kernel
 *    does not form them itself (unitarise set, or p > 4 or a loop too long for the
 *    scan kernel); larger problems return BW_ENOMEM with a message, before anything
 *    runs.  n <= 32 and p <= 64.
 *  - Runs on the current CUDA device, in the context current on the calling thread.
 *    The first call in each context (normally once per device) looks up the array's
 *    device address there (cudaGetSymbolAddress); make that first call before any
 *    stream capture on that device.
 *  - Every call uses the same array and finds the previous call's data in it; the
 *    call clears its status word itself.  Calls whose work overlaps on the GPU
 *    (other host threads, other streams) race on the array: serialise them.
 *  - The call waits for `stream` before returning and returns the device status of
 *    its own work (BW_EGAP etc.) as well as argument errors.
 *  - err (may be NULL) receives a NUL-terminated message of at most err_len bytes.
 * phases, min_gap: DEVICE, caller-owned, as for bw_wilson_loop. */
bw_status bw_wilson_loop_noalloc(const bw_model* model, const bw_plane* plane, int32_t p,
                                 bw_precision prec, const bw_opts* opts, double* phases,
                                 double* min_gap, void* stream, char* err, size_t err_len);

/* Scratch bytes bw_wilson_loop would reserve on this context for the problem (the
 * context's memory budget bounds it: a smaller budget runs the loops in smaller
 * blocks).  Validates the arguments like bw_wilson_loop; no device work. */
bw_status bw_wilson_loop_workspace(bw_ctx* ctx, const bw_model* model, const bw_plane* plane,
                                   int32_t p, bw_precision prec, const bw_opts* opts,
                                   size_t* bytes);

/* ---------------------------------------------------------------------------
 * Request server (no counterpart in the paper: serving many Wilson-loop requests,
 * e.g. disorder realisations and supercells of different sizes, on one GPU).
 *
 * The server owns one device memory pool (allocated once at creation), up to
 * max_slots contexts with one CUDA stream each, and a worker thread.  A submitted
 * request is validated and sized on the caller's thread, queued, and admitted when
 * a slot is free and the pool holds its scratch and outputs (at most half of the
 * pool per request); requests arriving while others run are admitted as soon as
 * slots and memory free up, and their kernels overlap on the GPU.  A request that
 * does not fit yet lets later, smaller ones through.  Each request computes exactly
 * what bw_wilson_loop computes; its results are copied to the caller's HOST buffers,
 * which must stay valid until the request is collected by bw_server_poll or
 * bw_server_wait.  The server functions may be called from any one host thread.
 * --------------------------------------------------------------------------- */
typedef struct bw_server bw_server;

typedef struct {
  int64_t id;
  int32_t status;         /* bw_status of the request (argument, device or CUDA error) */
  int32_t reserved;
  int64_t k_index;        /* k-point index of a device-side status, else -1         */
  double latency_ms;      /* submit -> results in the caller's buffers                */
  double queue_ms;        /* submit -> admission                                      */
  double device_ms;       /* first to last operation on the slot's stream             */
  char message[128];      /* error text (empty when status is BW_OK)                  */
} bw_request_info;

/* mem_budget_bytes = 0: 80 % of the free device memory.  1 <= max_slots <= 64. */
bw_status bw_server_create(bw_server** out, int device, int32_t max_slots,
                           size_t mem_budget_bytes);
/* Stops admitting, waits for the requests on the GPU, drops queued ones. */
void bw_server_destroy(bw_server* server);
const char* bw_server_last_error(const bw_server* server);
/* Queues a Wilson loop (arguments as bw_wilson_loop; model copied).  phases: HOST,
 * N_t x p doubles; min_gap: HOST, N_t doubles (may be NULL).  *id receives the
 * request id.  Returns argument errors and BW_ENOMEM (larger than the pool). */
bw_status bw_server_submit(bw_server* server, const bw_model* model, const bw_plane* plane,
                           int32_t p, bw_precision prec, const bw_opts* opts,
                           double* phases, double* min_gap, int64_t* id);
/* Collects up to max finished requests (in completion order) without blocking;
 * returns their number, or -1 on bad arguments. */
int bw_server_poll(bw_server* server, bw_request_info* done, int max);
/* Blocks until request id finishes (BW_ETIMEOUT after timeout_s seconds) and
 * collects it into *info (may be NULL). */
bw_status bw_server_wait(bw_server* server, int64_t id, double timeout_s, bw_request_info* info);
/* Requests queued or running. */
int64_t bw_server_outstanding(bw_server* server);
/* Withdraws a request that is still queued (not yet admitted): it completes at once
 * with status BW_ECANCELED and is collected like any other (bw_server_poll /
 * bw_server_wait); its host buffers are not written.  A request already admitted
 * runs to completion (kernels are not interrupted): BW_EINVAL, as for an unknown or
 * already finished id. */
bw_status bw_server_cancel(bw_server* server, int64_t id);

#ifdef __cplusplus
}
#endif

#endif /* BERRYWL_H */
