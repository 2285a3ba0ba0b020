// Host runtime of the C ABI: context, scratch arena, hopping-list plans, entry points.
//
// A hopping list arrives as host arrays and is turned into a device plan: the
// distinct translations R (their phases are evaluated once per k-point), and the
// distinct (row, col) entries of H, each owning the hoppings that sum into it.
// The plan groups duplicate (i, j, R) hoppings, and rejects lists for which
// H(f) would not be Hermitian (every (i, j, R) must match (j, i, -R) conjugated).
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include <cuda.h>

#include "../../include/berrywl.h"
#include "launch.h"

using bw::z64;

// Timing marks kept per call (kernel launches of one call, in order).
constexpr int kProfMax = 1024;
// Internal status returned by reserve() in a workspace query (never reaches a caller).
constexpr bw_status kQueryDone = bw_status(100);

struct bw_ctx {
  int device = 0;
  size_t budget = 0;
  char* arena = nullptr;
  size_t arena_cap = 0;
  size_t arena_off = 0;
  bw::DevStatus* status = nullptr;
  char* staging = nullptr;
  size_t staging_cap = 0;
  cudaEvent_t upload_ev = nullptr;
  bool upload_pending = false;
  cudaEvent_t done_ev = nullptr;
  cudaStream_t last_stream = nullptr;
  bool have_last = false;
  std::string err;
  // arena supplied by the owner (a server slot): never grown or freed here
  bool external_arena = false;
  // workspace query: reserve() records the bytes and stops the call
  bool query_only = false;
  size_t query_bytes = 0;
  // per-kernel timing (bw_set_profiling)
  bool prof = false;
  int prof_n = 0;
  const char* prof_names[kProfMax] = {};
  cudaEvent_t prof_ev[kProfMax + 1] = {};
  // the last hopping list's plan (a PlanCache, see plan_and_blob), owned
  void* plan_cache = nullptr;
};

namespace {

bw_status fail(bw_ctx* c, bw_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  return s;
}

bw_status cuda_fail(bw_ctx* c, cudaError_t e, const char* where) {
  return fail(c, BW_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define BW_CUDA(call, where)                         \
  do {                                               \
    cudaError_t e_ = (call);                         \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, where); \
  } while (0)

size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

// Host blob whose segments are copied to the device in one transfer.
struct Blob {
  std::vector<char> data;
  size_t add(const void* src, size_t bytes) {
    const size_t off = al256(data.size());
    data.resize(off + std::max<size_t>(bytes, 1));
    if (bytes) std::memcpy(data.data() + off, src, bytes);
    return off;
  }
  template <typename T>
  size_t add(const std::vector<T>& v) { return add(v.data(), v.size() * sizeof(T)); }
};

struct HostPlan {
  int n = 0, n_R = 0, n_ent = 0;
  std::vector<int> Rv, ent_row, ent_col, ent_start, hop_r, row_ptr;
  std::vector<z64> hop_t;
  double tmax = 0.0;
  size_t o_Rv, o_row, o_col, o_start, o_r, o_t, o_tdf, o_rowptr;
};

bw_status make_plan(bw_ctx* ctx, const bw_model* m, HostPlan& P) {
  if (!m) return fail(ctx, BW_EINVAL, "model is NULL");
  if (m->n < 1) return fail(ctx, BW_EINVAL, "model.n = %d < 1", m->n);
  if (m->nnz < 0 || m->nnz > (int64_t(1) << 31) - 2)
    return fail(ctx, BW_EINVAL, "model.nnz = %lld out of range", (long long)m->nnz);
  const int64_t nnz = m->nnz;
  if (nnz > 0 && (!m->R || !m->i || !m->j || !m->t))
    return fail(ctx, BW_EINVAL, "model arrays are NULL");
  const int n = m->n;
  P.n = n;
  for (int64_t e = 0; e < nnz; ++e) {
    if (m->i[e] < 0 || m->i[e] >= n || m->j[e] < 0 || m->j[e] >= n)
      return fail(ctx, BW_EINVAL, "hopping %lld has orbital index out of [0, %d)", (long long)e, n);
    if (!std::isfinite(m->t[e].re) || !std::isfinite(m->t[e].im))
      return fail(ctx, BW_EINVAL, "hopping %lld has a non-finite amplitude", (long long)e);
    P.tmax = std::max(P.tmax, std::hypot(m->t[e].re, m->t[e].im));
  }
  // distinct translations
  std::vector<std::array<int, 3>> Rs(nnz);
  for (int64_t e = 0; e < nnz; ++e) Rs[e] = {m->R[3 * e], m->R[3 * e + 1], m->R[3 * e + 2]};
  std::vector<std::array<int, 3>> U(Rs);
  std::sort(U.begin(), U.end());
  U.erase(std::unique(U.begin(), U.end()), U.end());
  P.n_R = int(U.size());
  P.Rv.resize(3 * U.size());
  for (size_t r = 0; r < U.size(); ++r)
    for (int d = 0; d < 3; ++d) P.Rv[3 * r + d] = U[r][d];
  auto rid = [&](const std::array<int, 3>& R) -> int {
    auto it = std::lower_bound(U.begin(), U.end(), R);
    return (it != U.end() && *it == R) ? int(it - U.begin()) : -1;
  };
  std::vector<int> hr(nnz);
  for (int64_t e = 0; e < nnz; ++e) hr[e] = rid(Rs[e]);
  // group hoppings by (i, j, r), summing duplicates, in a deterministic order
  std::vector<int64_t> idx(nnz);
  std::iota(idx.begin(), idx.end(), 0);
  std::sort(idx.begin(), idx.end(), [&](int64_t a, int64_t b) {
    if (m->i[a] != m->i[b]) return m->i[a] < m->i[b];
    if (m->j[a] != m->j[b]) return m->j[a] < m->j[b];
    if (hr[a] != hr[b]) return hr[a] < hr[b];
    return a < b;
  });
  struct Grp { int i, j, r; z64 t; };
  std::vector<Grp> g;
  for (int64_t q = 0; q < nnz; ++q) {
    const int64_t e = idx[q];
    const z64 t(m->t[e].re, m->t[e].im);
    if (!g.empty() && g.back().i == m->i[e] && g.back().j == m->j[e] && g.back().r == hr[e])
      g.back().t = g.back().t + t;
    else
      g.push_back({m->i[e], m->j[e], hr[e], t});
  }
  // Hermiticity: t(i, j, R) = conj t(j, i, -R)
  const double tol = 1e-12 * std::max(1.0, P.tmax);
  auto find = [&](int i, int j, int r) -> const Grp* {
    auto it = std::lower_bound(g.begin(), g.end(), Grp{i, j, r, z64(0, 0)}, [](const Grp& a, const Grp& b) {
      if (a.i != b.i) return a.i < b.i;
      if (a.j != b.j) return a.j < b.j;
      return a.r < b.r;
    });
    return (it != g.end() && it->i == i && it->j == j && it->r == r) ? &*it : nullptr;
  };
  for (const Grp& x : g) {
    const std::array<int, 3>& R = U[x.r];
    const int rn = rid({-R[0], -R[1], -R[2]});
    const Grp* y = rn >= 0 ? find(x.j, x.i, rn) : nullptr;
    const z64 yt = y ? y->t : z64(0.0, 0.0);
    if (std::hypot(x.t.re - yt.re, x.t.im + yt.im) > tol)
      return fail(ctx, BW_EINVAL,
                  "hopping list is not Hermitian: (i=%d, j=%d, R=(%d,%d,%d)) has no conjugate partner",
                  x.i, x.j, R[0], R[1], R[2]);
  }
  // entries
  for (size_t q = 0; q < g.size(); ++q) {
    if (q == 0 || g[q].i != g[q - 1].i || g[q].j != g[q - 1].j) {
      P.ent_row.push_back(g[q].i);
      P.ent_col.push_back(g[q].j);
      P.ent_start.push_back(int(q));
    }
    P.hop_r.push_back(g[q].r);
    P.hop_t.push_back(g[q].t);
  }
  P.ent_start.push_back(int(g.size()));
  P.n_ent = int(P.ent_row.size());
  // first entry of each row (entries are sorted by row)
  P.row_ptr.assign(n + 1, 0);
  for (int e = 0; e < P.n_ent; ++e) P.row_ptr[P.ent_row[e] + 1]++;
  for (int r = 0; r < n; ++r) P.row_ptr[r + 1] += P.row_ptr[r];
  return BW_OK;
}

void plan_to_blob(HostPlan& P, Blob& b) {
  P.o_Rv = b.add(P.Rv);
  P.o_row = b.add(P.ent_row);
  P.o_col = b.add(P.ent_col);
  P.o_start = b.add(P.ent_start);
  P.o_r = b.add(P.hop_r);
  P.o_t = b.add(P.hop_t);
  std::vector<float> tdf(4 * P.hop_t.size());
  for (size_t h = 0; h < P.hop_t.size(); ++h) {
    const double v[2] = {P.hop_t[h].re, P.hop_t[h].im};
    for (int c = 0; c < 2; ++c) {
      const float hi = float(v[c]);
      tdf[4 * h + 2 * c] = hi;
      tdf[4 * h + 2 * c + 1] = float(v[c] - double(hi));
    }
  }
  P.o_tdf = b.add(tdf);
  P.o_rowptr = b.add(P.row_ptr);
}

// The plan of the last hopping list seen on a context, with a copy of that list:
// building a plan sorts and groups the list, which for a many-band model (~10^6
// hoppings) costs more host time than the GPU work of a call, and a caller usually
// passes the same model call after call (planes, precisions, loop kinds).  A list is
// reused only when it matches the copy entry by entry.
struct PlanCache {
  int32_t n = 0;
  int64_t nnz = -1;
  std::vector<int32_t> R, i, j;
  std::vector<bw_c128> t;
  HostPlan P;
  Blob blob;
};

bool same_model(const PlanCache& c, const bw_model* m) {
  if (c.n != m->n || c.nnz != m->nnz) return false;
  const size_t nz = size_t(m->nnz);
  if (nz == 0) return true;
  return std::memcmp(c.R.data(), m->R, 3 * nz * sizeof(int32_t)) == 0 &&
         std::memcmp(c.i.data(), m->i, nz * sizeof(int32_t)) == 0 &&
         std::memcmp(c.j.data(), m->j, nz * sizeof(int32_t)) == 0 &&
         std::memcmp(c.t.data(), m->t, nz * sizeof(bw_c128)) == 0;
}

// make_plan + plan_to_blob, through the context's cache; *P and *blob point into the
// cache and stay valid until the next call on the context.
bw_status plan_and_blob(bw_ctx* ctx, const bw_model* m, const HostPlan** P, const Blob** blob) {
  PlanCache* c = static_cast<PlanCache*>(ctx->plan_cache);
  if (!(m && c && same_model(*c, m))) {
    HostPlan fresh;
    bw_status st = make_plan(ctx, m, fresh);
    if (st) return st;
    if (!c) {
      c = new PlanCache();
      ctx->plan_cache = c;
    }
    c->nnz = -1;  // invalid until the copy below is complete
    c->blob = Blob();
    plan_to_blob(fresh, c->blob);
    c->P = std::move(fresh);
    const size_t nz = size_t(m->nnz);
    c->R.assign(m->R, m->R + (nz ? 3 * nz : 0));
    c->i.assign(m->i, m->i + nz);
    c->j.assign(m->j, m->j + nz);
    c->t.assign(m->t, m->t + nz);
    c->n = m->n;
    c->nnz = m->nnz;
  }
  *P = &c->P;
  *blob = &c->blob;
  return BW_OK;
}

void plan_cache_free(bw_ctx* ctx) {
  delete static_cast<PlanCache*>(ctx->plan_cache);
  ctx->plan_cache = nullptr;
}

bw::DevModel dev_model(const HostPlan& P, const char* base) {
  bw::DevModel d;
  d.n = P.n;
  d.n_R = P.n_R;
  d.n_ent = P.n_ent;
  d.n_hop = int(P.hop_t.size());
  d.Rv = reinterpret_cast<const int*>(base + P.o_Rv);
  d.ent_row = reinterpret_cast<const int*>(base + P.o_row);
  d.ent_col = reinterpret_cast<const int*>(base + P.o_col);
  d.ent_start = reinterpret_cast<const int*>(base + P.o_start);
  d.hop_r = reinterpret_cast<const int*>(base + P.o_r);
  d.hop_t = reinterpret_cast<const z64*>(base + P.o_t);
  d.hop_tdf = reinterpret_cast<const float*>(base + P.o_tdf);
  return d;
}

struct HostOp {
  std::vector<int> row, col, rowp;  // entries sorted by row; rowp: CSR row pointers (n + 1)
  std::vector<z64> val;
  size_t o_row, o_col, o_val, o_rowp;
};

bw_status make_op(bw_ctx* ctx, const bw_c128* S, int n, HostOp& op) {
  if (!S) return fail(ctx, BW_EINVAL, "spin operator is NULL");
  double smax = 0.0;
  for (int64_t e = 0; e < int64_t(n) * n; ++e) smax = std::max(smax, std::hypot(S[e].re, S[e].im));
  const double tol = 1e-12 * std::max(1.0, smax);
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < n; ++c) {
      const bw_c128 a = S[int64_t(r) * n + c], b = S[int64_t(c) * n + r];
      if (!std::isfinite(a.re) || !std::isfinite(a.im))
        return fail(ctx, BW_EINVAL, "spin operator has a non-finite entry");
      if (std::hypot(a.re - b.re, a.im + b.im) > tol)
        return fail(ctx, BW_EINVAL, "spin operator is not Hermitian at (%d, %d)", r, c);
      if (a.re != 0.0 || a.im != 0.0) {
        op.row.push_back(r);
        op.col.push_back(c);
        op.val.push_back(z64(a.re, a.im));
      }
    }
  if (op.val.empty()) return fail(ctx, BW_EINVAL, "spin operator is zero");
  op.rowp.assign(n + 1, 0);
  for (int r : op.row) op.rowp[r + 1]++;
  for (int r = 0; r < n; ++r) op.rowp[r + 1] += op.rowp[r];
  return BW_OK;
}

bool capturing(cudaStream_t s) {
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &st) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return st == cudaStreamCaptureStatusActive;
}

// Orders this call after the previous one when the stream changes.  Under stream
// capture nothing is waited on or recorded: the caller orders the captured graph.
void begin_call(bw_ctx* ctx, cudaStream_t s) {
  cudaSetDevice(ctx->device);
  if (!capturing(s) && ctx->have_last && ctx->last_stream != s)
    cudaStreamWaitEvent(s, ctx->done_ev, 0);
  ctx->arena_off = 0;
  ctx->prof_n = 0;
}

void end_call(bw_ctx* ctx, cudaStream_t s) {
  if (capturing(s)) return;
  cudaEventRecord(ctx->done_ev, s);
  ctx->last_stream = s;
  ctx->have_last = true;
}

// Timing marks around kernel launches (recorded as external events under capture,
// so that replays of a captured graph can be timed too).
void prof_mark(bw_ctx* ctx, cudaStream_t s, const char* name) {
  if (!ctx->prof || ctx->prof_n >= kProfMax) return;
  const int i = ctx->prof_n;
  if (!ctx->prof_ev[0])
    for (auto& e : ctx->prof_ev) cudaEventCreate(&e);
  ctx->prof_names[i] = name;
  cudaEventRecordWithFlags(ctx->prof_ev[i + 1], s, capturing(s) ? cudaEventRecordExternal : 0);
  ctx->prof_n = i + 1;
}

// Records the start mark before the first kernel of a call.
struct MarkHook {
  bw_ctx* ctx;
  cudaStream_t s;
};

void mark_hook(void* user, const char* name) {
  MarkHook* h = static_cast<MarkHook*>(user);
  prof_mark(h->ctx, h->s, name);
}

void prof_start(bw_ctx* ctx, cudaStream_t s) {
  if (!ctx->prof) return;
  if (!ctx->prof_ev[0])
    for (auto& e : ctx->prof_ev) cudaEventCreate(&e);
  cudaEventRecordWithFlags(ctx->prof_ev[0], s, capturing(s) ? cudaEventRecordExternal : 0);
}

// Makes sure the arena holds `bytes`; growing it waits for outstanding work.
bw_status reserve(bw_ctx* ctx, size_t bytes, cudaStream_t s) {
  if (ctx->query_only) {
    ctx->query_bytes = bytes;
    return kQueryDone;
  }
  if (ctx->external_arena && bytes > ctx->arena_cap)
    return fail(ctx, BW_ENOMEM, "call needs %zu bytes of scratch, the attached arena holds %zu", bytes,
                ctx->arena_cap);
  if (bytes > ctx->budget)
    return fail(ctx, BW_ENOMEM, "call needs %zu bytes of scratch, budget is %zu", bytes, ctx->budget);
  if (bytes <= ctx->arena_cap) return BW_OK;
  if (capturing(s))
    return fail(ctx, BW_EINVAL, "scratch arena must grow during stream capture: run the call once "
                "uncaptured first");
  BW_CUDA(cudaStreamSynchronize(s), "cudaStreamSynchronize");
  if (ctx->have_last) BW_CUDA(cudaStreamSynchronize(ctx->last_stream), "cudaStreamSynchronize");
  if (ctx->arena) cudaFree(ctx->arena);
  ctx->arena = nullptr;
  ctx->arena_cap = 0;
  size_t cap = std::min(ctx->budget, std::max(bytes + bytes / 4, size_t(64) << 20));
  cudaError_t e = cudaMalloc(&ctx->arena, cap);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, BW_ENOMEM, "cudaMalloc of %zu bytes failed: %s", cap, cudaGetErrorString(e));
  }
  ctx->arena_cap = cap;
  return BW_OK;
}

char* carve(bw_ctx* ctx, size_t bytes) {
  const size_t off = al256(ctx->arena_off);
  ctx->arena_off = off + al256(std::max<size_t>(bytes, 1));
  return ctx->arena + off;
}

// Copies the blob to `dst` on stream s through the pinned staging buffer.
bw_status upload(bw_ctx* ctx, const Blob& b, char* dst, cudaStream_t s) {
  const size_t bytes = b.data.size();
  if (!bytes) return BW_OK;
  const bool cap = capturing(s);
  if (ctx->upload_pending && !cap) {
    BW_CUDA(cudaEventSynchronize(ctx->upload_ev), "cudaEventSynchronize");
    ctx->upload_pending = false;
  }
  if (bytes > ctx->staging_cap) {
    if (cap)
      return fail(ctx, BW_EINVAL, "staging buffer must grow during stream capture: run the call "
                  "once uncaptured first");
    if (ctx->staging) cudaFreeHost(ctx->staging);
    ctx->staging = nullptr;
    ctx->staging_cap = 0;
    const size_t cap = std::max(bytes, size_t(1) << 20);
    BW_CUDA(cudaMallocHost(&ctx->staging, cap), "cudaMallocHost");
    ctx->staging_cap = cap;
  }
  std::memcpy(ctx->staging, b.data.data(), bytes);
  BW_CUDA(cudaMemcpyAsync(dst, ctx->staging, bytes, cudaMemcpyHostToDevice, s), "cudaMemcpyAsync");
  if (!cap) {
    BW_CUDA(cudaEventRecord(ctx->upload_ev, s), "cudaEventRecord");
    ctx->upload_pending = true;
  }
  return BW_OK;
}

struct Opts {
  double gap_tol, pso_gap_tol, wannier_gap_tol;
  int unitarise, max_sweeps;
  int pso_median;  // bw_opts.pso_split (0 or 1; anything else is rejected by the callers)
};

Opts resolve_opts(const bw_opts* o, double tmax) {
  Opts r;
  r.gap_tol = (o && o->gap_tol >= 0.0) ? o->gap_tol : 1e-6 * std::max(1.0, tmax);
  r.pso_gap_tol = (o && o->pso_gap_tol >= 0.0) ? o->pso_gap_tol : 1e-6;
  r.wannier_gap_tol = (o && o->wannier_gap_tol >= 0.0) ? o->wannier_gap_tol : 1e-6;
  r.unitarise = o ? o->unitarise : 0;
  r.max_sweeps = (o && o->max_sweeps > 0) ? o->max_sweeps : 30;
  r.pso_median = o ? o->pso_split : 0;
  return r;
}

bw_status check_plane(bw_ctx* ctx, const bw_plane* pl, bool nested) {
  if (!pl) return fail(ctx, BW_EINVAL, "plane is NULL");
  if (pl->N < 1 || pl->N_t < 1) return fail(ctx, BW_EINVAL, "plane needs N >= 1 and N_t >= 1");
  if (int64_t(pl->N) * pl->N_t > (int64_t(1) << 31))
    return fail(ctx, BW_EINVAL, "plane has too many k-points");
  for (int d = 0; d < 3; ++d)
    if (!std::isfinite(pl->origin[d]) || !std::isfinite(pl->trans_dir[d]))
      return fail(ctx, BW_EINVAL, "plane has non-finite coordinates");
  if (nested)
    for (int d = 0; d < 3; ++d)
      if (pl->trans_dir[d] != std::round(pl->trans_dir[d]))
        return fail(ctx, BW_EINVAL, "nested loop needs an integer trans_dir to close");
  return BW_OK;
}

// One plane, or a stack of N_s parallel planes flattened into N_s N_t rows: `flat` is
// the plane with N_t = all rows, which sizes every buffer; the kernels take plane and
// transverse point from the row (bw::DevPlane).
struct PlaneX {
  bw_plane flat;
  int N_s = 1, N_tp = 0;
  int sweep[3] = {0, 0, 0};
};

bw_status stack_planes(bw_ctx* ctx, const bw_plane* pl, const int32_t* sweep, int N_s, PlaneX& X) {
  if (N_s < 1) return fail(ctx, BW_EINVAL, "need N_s >= 1 planes (N_s = %d)", N_s);
  if (int64_t(pl->N_t) * N_s > (int64_t(1) << 30) ||
      int64_t(pl->N) * pl->N_t * N_s > (int64_t(1) << 31))
    return fail(ctx, BW_EINVAL, "plane stack has too many k-points");
  X.flat = *pl;
  X.flat.N_t = pl->N_t * N_s;
  X.N_s = N_s;
  X.N_tp = pl->N_t;
  for (int d = 0; d < 3; ++d) X.sweep[d] = (sweep && N_s > 1) ? sweep[d] : 0;
  return BW_OK;
}

bw::DevPlane dev_plane(const PlaneX& X) {
  const bw_plane* pl = &X.flat;
  bw::DevPlane d;
  for (int k = 0; k < 3; ++k) {
    d.origin[k] = pl->origin[k];
    d.loop_dir[k] = double(pl->loop_dir[k]);
    d.trans_dir[k] = pl->trans_dir[k];
    d.sweep[k] = X.sweep[k];
  }
  d.N = pl->N;
  d.N_t = pl->N_t;
  d.N_s = X.N_s;
  d.N_tp = X.N_tp;
  return d;
}

// Projected-spin split of waves of occupied blocks (Sec. IV) for n > 32: the
// occupied-space operator S = U^dagger (sigma s U) of every k-point of a wave by one
// sparse application and one batched GEMM, its FP64 eigen-decomposition on the
// tridiagonal path (sigma = +1 for the sector s < 0, -1 for s > 0, so the sector is
// the lowest p/2 eigenvectors V of sigma S), the PSO gap check, and the sector
// states U V by a second GEMM.  pso_split_bytes: scratch per wave slot.
struct PsoSplit {
  int n = 0, p = 0, pl = 0, pnval = 0;
  double sigma = 1.0, tol = 0.0;
  int median = 0;
  z64 *Yw = nullptr, *Sw = nullptr, *Vw = nullptr;
  const int* rowp = nullptr;
  const int* col = nullptr;
  const z64* val = nullptr;
  double* pso_evals = nullptr;
  double* psog = nullptr;
  bw::LargeArgs ps;
};

size_t pso_split_bytes(int n, int p, bool want_evals) {
  const int pl = p / 2, pnval = want_evals ? p : pl + 1;
  const size_t d8 = sizeof(double);
  return al256(size_t(n) * p * sizeof(z64)) + 2 * al256(size_t(p) * p * sizeof(z64)) +
         al256(size_t(p) * pl * sizeof(z64)) + 2 * al256(size_t(p) * d8) + al256(size_t(p) * 2 * d8) +
         al256(size_t(pnval) * d8) + al256(size_t(pl) * p * d8) + al256(size_t(pl) * 6 * p * d8) +
         sizeof(long long) + sizeof(int);
}

bw_status pso_split_setup(bw_ctx* ctx, PsoSplit& X, long long Wv, int n, int p, const HostOp& op,
                          const char* dblob, int sign, double tol, double* pso_evals, double* psog,
                          MarkHook* hook, cudaStream_t s) {
  X.n = n;
  X.p = p;
  X.pl = p / 2;
  X.pnval = pso_evals ? p : X.pl + 1;
  X.sigma = sign < 0 ? 1.0 : -1.0;
  X.tol = tol;
  X.pso_evals = pso_evals;
  X.psog = psog;
  const size_t d8 = sizeof(double);
  X.Yw = reinterpret_cast<z64*>(carve(ctx, Wv * al256(size_t(n) * p * sizeof(z64))));
  X.Sw = reinterpret_cast<z64*>(carve(ctx, Wv * al256(size_t(p) * p * sizeof(z64))));
  X.Vw = reinterpret_cast<z64*>(carve(ctx, Wv * al256(size_t(p) * X.pl * sizeof(z64))));
  long long* h_off = reinterpret_cast<long long*>(carve(ctx, Wv * sizeof(long long)));
  int* idx = reinterpret_cast<int*>(carve(ctx, Wv * sizeof(int)));
  BW_CUDA(bw::launch_iota(h_off, idx, Wv, (long long)al256(size_t(p) * p * sizeof(z64)) / long(sizeof(z64)), s),
          "index kernel");
  bw::LargeArgs& ps = X.ps;
  std::memset(&ps, 0, sizeof(ps));
  ps.n = p;
  ps.p = X.pl;
  ps.nval = X.pnval;
  ps.nvec = X.pl;
  ps.nbt = X.pl;
  ps.mixed = 0;
  ps.gap = psog;
  ps.status = ctx->status;
  ps.A = carve(ctx, Wv * al256(size_t(p) * p * sizeof(z64)));
  ps.dg = carve(ctx, Wv * al256(size_t(p) * d8));
  ps.od = carve(ctx, Wv * al256(size_t(p) * d8));
  ps.Dp = carve(ctx, Wv * al256(size_t(p) * 2 * d8));
  ps.lam = carve(ctx, Wv * al256(size_t(X.pnval) * d8));
  ps.Z = carve(ctx, Wv * al256(size_t(X.pl) * p * d8));
  ps.work = carve(ctx, Wv * al256(size_t(X.pl) * 6 * p * d8));
  ps.U = X.Vw;
  ps.mark = mark_hook;
  ps.mark_user = hook;
  ps.subspace_only = 1;  // the sector's span is what the loop needs
  ps.Hin = X.Sw;
  ps.h_off = h_off;
  ps.idx = idx;
  X.rowp = reinterpret_cast<const int*>(dblob + op.o_rowp);
  X.col = reinterpret_cast<const int*>(dblob + op.o_col);
  X.val = reinterpret_cast<const z64*>(dblob + op.o_val);
  return BW_OK;
}

// One wave: Uw holds Wn occupied blocks (n x p) of k-points k0 .. k0 + Wn - 1; the
// sector states go to dst (n x p/2 per k-point).
bw_status pso_split_wave(bw_ctx* ctx, PsoSplit& X, const z64* Uw, long long Wn, long long k0, z64* dst,
                         cudaStream_t s) {
  const int n = X.n, p = X.p, pl = X.pl;
  // S slots at the stride of the eigensolver's matrix index; sigma s U as written by the
  // spin kernel and V as written by the back-transform are packed
  const long long sS = (long long)al256(size_t(p) * p * sizeof(z64)) / long(sizeof(z64));
  const long long sY = (long long)n * p, sV = (long long)p * pl;
  BW_CUDA(bw::launch_spin_apply(Uw, X.Yw, Wn, n, p, X.rowp, X.col, X.val, X.sigma, s), "spin operator kernel");
  bw::GemmArgs g;
  std::memset(&g, 0, sizeof(g));
  g.A = Uw; g.B = X.Yw; g.C = X.Sw;
  g.m = p; g.n = p; g.k = n; g.opA = 1;
  g.lda = p; g.ldb = p; g.ldc = p;
  g.sA = (long long)n * p; g.sB = sY; g.sC = sS;
  g.batch = Wn;
  BW_CUDA(bw::launch_zgemm(g, s), "spin operator GEMM");
  X.ps.k0 = 0;
  X.ps.W = Wn;
  BW_CUDA(bw::launch_states_large(X.ps, s), "spin operator eigensolve");
  BW_CUDA(bw::launch_pso_post(reinterpret_cast<const double*>(X.ps.lam), X.pnval, Wn, k0, p, X.sigma, X.tol,
                              X.median, X.pso_evals, X.psog, ctx->status, s),
          "spin sector check");
  std::memset(&g, 0, sizeof(g));
  g.A = Uw; g.B = X.Vw; g.C = dst;
  g.m = n; g.n = pl; g.k = p; g.opA = 0;
  g.lda = p; g.ldb = pl; g.ldc = pl;
  g.sA = (long long)n * p; g.sB = sV; g.sC = (long long)n * pl;
  g.batch = Wn;
  BW_CUDA(bw::launch_zgemm(g, s), "sector states GEMM");
  return BW_OK;
}

// Wilson loop with many occupied bands (p > LOOP_P_MAX, n > SMALL_N_MAX).  The
// Wilson matrix no longer fits in shared memory, so the loop runs as batched GEMMs
// (FP64, or double-float on the FP32 pipe in the mixed request):
// for a block of nl loops (their k-points are contiguous, k = i N + j) the states are
// solved in waves of up to 2048 k-points, one GEMM forms every overlap
// M_j = U(k_{j+1})^dagger U(k_j) of the block (closing on U(k_0), Eq. 2), N - 1 GEMMs
// form W = M_{N-1} ... M_0 for all loops of the block at once, and one CTA per loop
// takes the eigenphases.  Memory per loop: N n x p states, N + 2 p x p matrices;
// the solver's per-k-point scratch is per wave.  The block shrinks to fit the budget.
// With a spin operator (Sec. IV) each wave also forms S = U^dagger (sigma s U) by
// one sparse application and one GEMM, diagonalises it in FP64 on the tridiagonal
// path (sigma = +1 for the sector s < 0, -1 for s > 0: the sector is the lowest p/2
// eigenvectors V of sigma S), checks the PSO gap, and keeps the sector states U V;
// the loop then runs on those p/2 columns.
bw_status run_big_loop(bw_ctx* ctx, const HostPlan& P, const Blob& blob, const PlaneX& PX,
                       int p, bool mx, const Opts& o, double* phases, double* min_gap,
                       cudaStream_t s, const HostOp* op = nullptr, int sign = -1,
                       double* pso_evals = nullptr, double* min_pso_gap = nullptr) {
  const bw_plane* plane = &PX.flat;
  const int n = P.n, N = plane->N, Nt = plane->N_t;
  const bool spin = op != nullptr;
  const int pl = spin ? p / 2 : p;  // columns the loop runs on
  const long long K = (long long)N * Nt;
  const size_t ts = mx ? sizeof(float) : sizeof(double);
  const int nval = mx ? n : std::min(n, p + 1), nvec = mx ? n : p;
  const int nbt = mx ? std::min(n, p + 1) : p;
  const size_t sz_A = al256(size_t(n) * n * 2 * ts), sz_v = al256(size_t(n) * ts),
               sz_D = al256(size_t(n) * 2 * ts), sz_lam = al256(size_t(nval) * ts),
               sz_Z = al256(size_t(nvec) * n * ts), sz_wk = al256(size_t(nvec) * 6 * n * ts),
               sz_X = mx ? al256(size_t(n) * nbt * sizeof(bw::c32)) : 0,
               sz_He = mx ? al256(size_t(P.n_ent) * sizeof(z64)) : 0,
               sz_R = mx ? al256(size_t(n) * p * sizeof(z64)) : 0,
               sz_C = mx ? al256(size_t(n) * p * sizeof(bw::c32)) : 0,
               sz_G = mx ? al256(size_t(p) * p * sizeof(z64)) : 0;
  // spin split, per wave slot: the occupied block and the split's scratch
  const size_t sp_U = spin ? al256(size_t(n) * p * sizeof(z64)) : 0;
  const size_t per_k = sz_A + 2 * sz_v + sz_D + sz_lam + sz_Z + sz_wk + sz_X + sz_He + sz_R + sz_C +
                       sz_G + sp_U + (spin ? pso_split_bytes(n, p, pso_evals != nullptr) : 0);
  const size_t bUk = size_t(n) * pl * sizeof(z64), bPk = size_t(pl) * pl * sizeof(z64);
  const size_t bEl = size_t(pl) * (2 * sizeof(z64) + sizeof(double) + sizeof(int)) + 8 * sizeof(double);
  const size_t per_loop = size_t(N) * (bUk + bPk) + 2 * bPk + bEl;
  size_t total = al256(blob.data.size()) + (spin ? 2 : 1) * al256(size_t(K) * sizeof(double)) + 48 * 256;
  const size_t avail = ctx->budget > total ? ctx->budget - total : 0;
  long long Wv = std::min<long long>(K, 2048);
  while (Wv > 1 && size_t(Wv) * per_k + per_loop > avail) Wv /= 2;
  const size_t left = avail > size_t(Wv) * per_k ? avail - size_t(Wv) * per_k : 0;
  const int nl_max = int(std::min<long long>(Nt, std::max<long long>(1, (long long)(left / per_loop))));
  Wv = std::min<long long>(Wv, (long long)nl_max * N);
  total += size_t(Wv) * per_k + size_t(nl_max) * per_loop;
  bw_status st;
  if ((st = reserve(ctx, total, s))) return st;
  char* dblob = carve(ctx, blob.data.size());
  double* gap = reinterpret_cast<double*>(carve(ctx, size_t(K) * sizeof(double)));
  double* psog = spin ? reinterpret_cast<double*>(carve(ctx, size_t(K) * sizeof(double))) : nullptr;
  if ((st = upload(ctx, blob, dblob, s))) return st;
  z64* Ublk = reinterpret_cast<z64*>(carve(ctx, size_t(nl_max) * N * bUk));
  z64* Mblk = reinterpret_cast<z64*>(carve(ctx, size_t(nl_max) * N * bPk));
  z64* Wbuf[2];
  for (auto& w : Wbuf) w = reinterpret_cast<z64*>(carve(ctx, size_t(nl_max) * bPk));
  z64* e_lam = reinterpret_cast<z64*>(carve(ctx, nl_max * size_t(pl) * sizeof(z64)));
  z64* e_vec = reinterpret_cast<z64*>(carve(ctx, nl_max * size_t(pl) * sizeof(z64)));
  double* e_th = reinterpret_cast<double*>(carve(ctx, nl_max * size_t(pl) * sizeof(double)));
  int* e_ord = reinterpret_cast<int*>(carve(ctx, nl_max * size_t(pl) * sizeof(int)));
  double* e_ctl = reinterpret_cast<double*>(carve(ctx, nl_max * 8 * sizeof(double)));

  bw::LargeArgs lg;
  std::memset(&lg, 0, sizeof(lg));
  lg.model = dev_model(P, dblob);
  lg.plane = dev_plane(PX);
  lg.n = n;
  lg.p = p;
  lg.nval = nval;
  lg.nvec = nvec;
  lg.nbt = nbt;
  lg.mixed = mx;
  lg.gap_tol = o.gap_tol;
  lg.row_ptr = reinterpret_cast<const int*>(dblob + P.o_rowptr);
  lg.gap = gap;
  lg.status = ctx->status;
  lg.A = carve(ctx, Wv * sz_A);
  lg.dg = carve(ctx, Wv * sz_v);
  lg.od = carve(ctx, Wv * sz_v);
  lg.Dp = carve(ctx, Wv * sz_D);
  lg.lam = carve(ctx, Wv * sz_lam);
  lg.Z = carve(ctx, Wv * sz_Z);
  lg.work = carve(ctx, Wv * sz_wk);
  if (mx) {
    lg.X = carve(ctx, Wv * sz_X);
    lg.Hent = reinterpret_cast<z64*>(carve(ctx, Wv * sz_He));
    lg.R64 = reinterpret_cast<z64*>(carve(ctx, Wv * sz_R));
    lg.C32 = reinterpret_cast<bw::c32*>(carve(ctx, Wv * sz_C));
    lg.G64 = reinterpret_cast<z64*>(carve(ctx, Wv * sz_G));
  }
  MarkHook hook{ctx, s};
  lg.mark = mark_hook;
  lg.mark_user = &hook;
  // spin split of a wave: the wave's occupied blocks, then the sector states
  z64* Uw = nullptr;
  PsoSplit X;
  if (spin) {
    Uw = reinterpret_cast<z64*>(carve(ctx, Wv * sp_U));
    if ((st = pso_split_setup(ctx, X, Wv, n, p, *op, dblob, sign, o.pso_gap_tol, pso_evals, psog, &hook, s)))
      return st;
    X.median = o.pso_median;
  }
  prof_start(ctx, s);
  const long long sU = (long long)n * pl, sP = (long long)pl * pl;
  for (int i0 = 0; i0 < Nt; i0 += nl_max) {
    const int nl = std::min(nl_max, Nt - i0);
    const long long kb = (long long)i0 * N, Kb = (long long)nl * N;
    for (long long w0 = 0; w0 < Kb; w0 += Wv) {
      const long long Wn = std::min(Wv, Kb - w0);
      lg.k0 = kb + w0;
      lg.W = Wn;
      lg.U = spin ? Uw : Ublk + w0 * sU;
      BW_CUDA(bw::launch_states_large(lg, s), "large-n states kernels");
      if (!spin) continue;
      if ((st = pso_split_wave(ctx, X, Uw, Wn, kb + w0, Ublk + w0 * sU, s))) return st;
      prof_mark(ctx, s, "pso_split");
    }
    // mixed request: the overlaps and loop products in complex double-float on the
    // FP32 pipe (the states converted in place; W converted back for the eigenphases)
    if (mx) BW_CUDA(bw::launch_convert_cdf(Ublk, Kb * sU, true, s), "state conversion");
    // every overlap of the block: batch b = l N + j, A = U(k_{j+1}) (closing on j = 0)
    bw::GemmArgs g;
    std::memset(&g, 0, sizeof(g));
    g.A = Ublk; g.B = Ublk; g.C = Mblk;
    g.m = pl; g.n = pl; g.k = n; g.opA = 1;
    g.lda = pl; g.ldb = pl; g.ldc = pl;
    g.sA = sU; g.sB = sU; g.sC = sP;
    g.a_next_N = N;
    g.batch = Kb;
    BW_CUDA(bw::launch_zgemm(g, s, mx), "overlap GEMM");
    prof_mark(ctx, s, "overlaps");
    // W = M_{N-1} ... M_0 for the nl loops at once
    const z64* Wcur = Mblk;  // M_0 of loop l at Mblk + l N pl^2
    long long sWcur = (long long)N * sP;
    for (int j = 1; j < N; ++j) {
      z64* Wout = Wbuf[j & 1];
      std::memset(&g, 0, sizeof(g));
      g.A = Mblk + (long long)j * sP; g.B = Wcur; g.C = Wout;
      g.m = pl; g.n = pl; g.k = pl; g.opA = 0;
      g.lda = pl; g.ldb = pl; g.ldc = pl;
      g.sA = (long long)N * sP; g.sB = sWcur; g.sC = sP;
      g.batch = nl;
      BW_CUDA(bw::launch_zgemm(g, s, mx), "loop-product GEMM");
      Wcur = Wout;
      sWcur = sP;
    }
    // the eigenphases in double-float as well when the cluster solver takes p; else W
    // back to FP64 (nl consecutive p x p matrices: sWcur = sP, or N sP = sP at N = 1)
    const bool df_eig = mx && bw::geig_df_eligible(pl);
    if (mx && !df_eig)
      BW_CUDA(bw::launch_convert_cdf(const_cast<z64*>(Wcur), nl * sP, false, s), "W conversion");
    if (N > 1) prof_mark(ctx, s, "loops");
    bw::BigEigArgs e;
    std::memset(&e, 0, sizeof(e));
    e.W = const_cast<z64*>(Wcur);
    e.sW = sWcur;
    e.p = pl;
    e.nl = nl;
    e.i0 = i0;
    e.N = N;
    e.gap = gap;
    e.pso_gap = psog;
    e.phases = phases;
    e.min_gap = min_gap;
    e.min_pso_gap = min_pso_gap;
    e.lam = e_lam;
    e.vec = e_vec;
    e.th = e_th;
    e.ord = e_ord;
    e.ctl = e_ctl;
    e.df = df_eig ? 1 : 0;
    e.status = ctx->status;
    BW_CUDA(bw::launch_geig_big(e, s), "eigenphase kernel");
    prof_mark(ctx, s, "eigenphases");
  }
  end_call(ctx, s);
  return BW_OK;
}

// Shared driver of the three loop entry points.
enum class LoopKind { Plain, Nested, Spin, Plaquette };

bw_status run_loop(bw_ctx* ctx, LoopKind kind, const bw_model* model, const bw_plane* user_plane,
                   int p, bw_precision prec, const bw_opts* opts, const bw_c128* spin_op,
                   int sign, double cut, int first, int m, double* phases, double* min_gap,
                   double* nested_out, double* min_wgap, double* pso_evals, double* min_pso_gap,
                   cudaStream_t s, double* chern_out = nullptr, const int32_t* sweep = nullptr,
                   int N_s = 1) {
  if (!ctx) return BW_EINVAL;
  ctx->err.clear();
  // the PSO split runs for the spin-resolved loop and for the flux of a spin sector
  const bool spin = kind == LoopKind::Spin || (kind == LoopKind::Plaquette && spin_op != nullptr);
  bw_status st = check_plane(ctx, user_plane, kind == LoopKind::Nested || kind == LoopKind::Plaquette);
  if (st) return st;
  PlaneX PX;
  if ((st = stack_planes(ctx, user_plane, sweep, N_s, PX))) return st;
  if (kind == LoopKind::Plaquette && PX.N_s > 1) return fail(ctx, BW_EINVAL, "plaquette flux takes one plane");
  const bw_plane* plane = &PX.flat;
  if (prec != BW_FP64 && prec != BW_MIXED) return fail(ctx, BW_EINVAL, "unknown precision %d", int(prec));
  if (!phases) return fail(ctx, BW_EINVAL, "phases output is NULL");
  const HostPlan* Pc = nullptr;
  const Blob* Bc = nullptr;
  if ((st = plan_and_blob(ctx, model, &Pc, &Bc))) return st;
  const HostPlan& P = *Pc;
  const int n = P.n;
  if (p < 1 || p > n) return fail(ctx, BW_EINVAL, "need 1 <= p <= n (p = %d, n = %d)", p, n);
  if (n > bw::LARGE_N_MAX)
    return fail(ctx, BW_EINVAL, "n = %d exceeds the largest supported size %d", n, bw::LARGE_N_MAX);
  const bool large = n > bw::SMALL_N_MAX;
  int p_eff = p;
  HostOp op;
  if (spin) {
    if (p % 2) return fail(ctx, BW_EINVAL, "spin-resolved loop needs an even p (p = %d)", p);
    if (sign != -1 && sign != 1) return fail(ctx, BW_EINVAL, "sign must be -1 or +1");
    if ((st = make_op(ctx, spin_op, n, op))) return st;
    p_eff = p / 2;
  }
  if (kind == LoopKind::Nested) {
    if (!nested_out) return fail(ctx, BW_EINVAL, "nested output is NULL");
    if (m < 1 || first < 0 || first + m > p)
      return fail(ctx, BW_EINVAL, "nested sector [first, first+m) = [%d, %d) outside [0, %d)", first,
                  first + m, p);
    if (!std::isfinite(cut)) return fail(ctx, BW_EINVAL, "cut is not finite");
  }
  if (kind == LoopKind::Nested && p_eff > bw::LOOP_P_MAX)
    return fail(ctx, BW_EINVAL, "nested loop supports p <= %d (p = %d)", bw::LOOP_P_MAX, p_eff);
  // many occupied bands: batched-GEMM loops (the spin-resolved one from p > 64 at
  // large n, where the split runs on the tridiagonal path)
  const bool big = (kind == LoopKind::Plain && p_eff > bw::LOOP_P_MAX) ||
                   (kind == LoopKind::Spin && large && p > 64);
  const Opts o = resolve_opts(opts, P.tmax);
  if (o.unitarise && p_eff > 32) return fail(ctx, BW_EINVAL, "unitarise supports p <= 32");
  if (o.pso_median != 0 && o.pso_median != 1)
    return fail(ctx, BW_EINVAL, "pso_split must be 0 (split at zero) or 1 (at the median), got %d",
                o.pso_median);
  const long long K = (long long)plane->N * plane->N_t;
  // the plan's blob, with the spin operator appended for the loops that split by it
  Blob blob_op;
  if (spin) {
    blob_op = *Bc;
    op.o_row = blob_op.add(op.row);
    op.o_col = blob_op.add(op.col);
    op.o_val = blob_op.add(op.val);
    op.o_rowp = blob_op.add(op.rowp);
  }
  const Blob& blob = spin ? blob_op : *Bc;
  if (big) {
    begin_call(ctx, s);
    if (kind == LoopKind::Spin)
      return run_big_loop(ctx, P, blob, PX, p, prec == BW_MIXED, o, phases, min_gap, s, &op, sign,
                          pso_evals, min_pso_gap);
    return run_big_loop(ctx, P, blob, PX, p, prec == BW_MIXED, o, phases, min_gap, s);
  }
  const size_t bU = al256(size_t(K) * n * p_eff * sizeof(z64));
  const size_t bGap = al256(size_t(K) * sizeof(double));
  // overlap scratch; the plaquette flux needs none up to p = 64 (links in shared memory)
  // and blocks of link matrices beyond
  const long long kb_links = std::min<long long>(K, 256);
  const size_t bM = kind != LoopKind::Plaquette ? al256(size_t(K) * p_eff * p_eff * sizeof(z64))
                    : p_eff > bw::LOOP_P_MAX   ? al256(size_t(kb_links) * p_eff * p_eff * sizeof(z64))
                                               : 0;
  const size_t bW = kind == LoopKind::Nested ? al256(size_t(K) * n * m * sizeof(z64)) : 0;
  bool transport_only = false;
  if (kind == LoopKind::Nested) {
    bw::LoopArgs q;
    std::memset(&q, 0, sizeof(q));
    q.n = n;
    q.p = p_eff;
    q.N = plane->N;
    q.N_t = plane->N_t;
    q.N_s = PX.N_s;
    q.nested = 1;
    q.m = m;
    transport_only = bw::loops_transport_only(q);
  }
  const size_t bNu = transport_only ? al256(size_t(K) * p_eff * m * sizeof(z64)) : 0;
  const size_t bPso = spin ? al256(size_t(K) * sizeof(double)) : 0;
  const size_t bLink = kind == LoopKind::Plaquette ? al256(size_t(K) * sizeof(z64)) : 0;
  size_t total = al256(blob.data.size()) + bU + bGap + bM + bW + bNu + bPso + 2 * bLink + 4096;
  // large n: per-k-point scratch of the tridiagonal solver, processed in waves
  const bool mx = prec == BW_MIXED;
  const size_t ts = mx ? sizeof(float) : sizeof(double);
  const int nval = mx ? n : std::min(n, p + 1), nvec = mx ? n : p;
  const int nbt = mx ? std::min(n, p + 1) : p;
  const size_t sz_A = al256(size_t(n) * n * 2 * ts), sz_v = al256(size_t(n) * ts),
               sz_D = al256(size_t(n) * 2 * ts), sz_lam = al256(size_t(nval) * ts),
               sz_Z = al256(size_t(nvec) * n * ts), sz_wk = al256(size_t(nvec) * 6 * n * ts),
               sz_X = mx ? al256(size_t(n) * nbt * sizeof(bw::c32)) : 0,
               sz_He = mx ? al256(size_t(P.n_ent) * sizeof(z64)) : 0,
               sz_R = mx ? al256(size_t(n) * p * sizeof(z64)) : 0,
               sz_C = mx ? al256(size_t(n) * p * sizeof(bw::c32)) : 0,
               sz_G = mx ? al256(size_t(p) * p * sizeof(z64)) : 0,
               sz_Uf = spin ? al256(size_t(n) * p * sizeof(z64)) : 0;
  const size_t per_k = sz_A + 2 * sz_v + sz_D + sz_lam + sz_Z + sz_wk + sz_X + sz_He + sz_R + sz_C +
                       sz_G + sz_Uf + (spin && large ? pso_split_bytes(n, p, pso_evals != nullptr) : 0);
  long long Wv = 0;
  if (large) {
    const size_t avail = ctx->budget > total ? (ctx->budget - total) / 2 : 0;
    Wv = std::min<long long>(K, std::max<long long>(1, (long long)(avail / per_k)));
    Wv = std::min<long long>(Wv, 2048);
    total += size_t(Wv) * per_k + 16 * 256;
  }
  begin_call(ctx, s);
  if ((st = reserve(ctx, total, s))) return st;
  char* dblob = carve(ctx, blob.data.size());
  z64* U = reinterpret_cast<z64*>(carve(ctx, bU));
  double* gap = reinterpret_cast<double*>(carve(ctx, bGap));
  z64* M = reinterpret_cast<z64*>(carve(ctx, bM));
  z64* w = bW ? reinterpret_cast<z64*>(carve(ctx, bW)) : nullptr;
  z64* nu_buf = bNu ? reinterpret_cast<z64*>(carve(ctx, bNu)) : nullptr;
  double* psog = bPso ? reinterpret_cast<double*>(carve(ctx, bPso)) : nullptr;
  z64* Lx = bLink ? reinterpret_cast<z64*>(carve(ctx, bLink)) : nullptr;
  z64* Ly = bLink ? reinterpret_cast<z64*>(carve(ctx, bLink)) : nullptr;

  bw::StatesArgs sa;
  std::memset(&sa, 0, sizeof(sa));
  sa.model = dev_model(P, dblob);
  sa.row_ptr = reinterpret_cast<const int*>(dblob + P.o_rowptr);
  sa.plane = dev_plane(PX);
  sa.f = nullptr;
  sa.K = K;
  sa.p = p;
  sa.mixed = prec == BW_MIXED;
  sa.max_sweeps = o.max_sweeps;
  sa.gap_tol = o.gap_tol;
  sa.op.nnz = 0;
  if (spin) {
    sa.op.nnz = int(op.val.size());
    sa.op.row = reinterpret_cast<const int*>(dblob + op.o_row);
    sa.op.col = reinterpret_cast<const int*>(dblob + op.o_col);
    sa.op.val = reinterpret_cast<const z64*>(dblob + op.o_val);
    sa.sign = sign;
    sa.pso_gap_tol = o.pso_gap_tol;
    sa.pso_median = o.pso_median;
    sa.pso_evals = pso_evals;
    sa.pso_gap = psog;
  }
  sa.U = U;
  sa.gap = gap;
  sa.status = ctx->status;
  // Mixed precision with four bands and the scan loop kernels: states, overlaps and
  // loop products in double-float on the FP32 pipe (U and w as complex double-float)
  bool use_df = false, fused = false;
  if (!large && sa.mixed && (kind == LoopKind::Plain || kind == LoopKind::Nested)) {
    bw::LoopArgs q;
    std::memset(&q, 0, sizeof(q));
    q.n = n;
    q.p = p_eff;
    q.N = plane->N;
    q.N_t = plane->N_t;
    q.N_s = PX.N_s;
    q.unitarise = o.unitarise;
    q.nested = kind == LoopKind::Nested;
    q.m = m;
    use_df = bw::loops_accept_df(q) && bw::states_df_eligible(sa, p_eff);
    fused = use_df && bw::loops_fused_eligible(q, sa.model);
  }
  sa.want_df = use_df ? 1 : 0;
  // a small plan rides along as a parameter of the fused kernel (no copy to dblob)
  const bool plan_inline = fused && blob.data.size() <= sizeof(bw::FusedPlan);
  if (!plan_inline && (st = upload(ctx, blob, dblob, s))) return st;
  prof_start(ctx, s);
  if (fused) {
    // states are solved inside the loop kernel below
  } else if (!large) {
    BW_CUDA(bw::launch_states_small(sa, p_eff, s), "states kernel");
  } else {
    bw::LargeArgs lg;
    std::memset(&lg, 0, sizeof(lg));
    lg.model = sa.model;
    lg.plane = sa.plane;
    lg.n = n;
    lg.p = p;
    lg.nval = nval;
    lg.nvec = nvec;
    lg.nbt = nbt;
    lg.mixed = mx;
    lg.gap_tol = o.gap_tol;
    lg.row_ptr = reinterpret_cast<const int*>(dblob + P.o_rowptr);
    lg.gap = gap;
    lg.status = ctx->status;
    lg.A = carve(ctx, Wv * sz_A);
    lg.dg = carve(ctx, Wv * sz_v);
    lg.od = carve(ctx, Wv * sz_v);
    lg.Dp = carve(ctx, Wv * sz_D);
    lg.lam = carve(ctx, Wv * sz_lam);
    lg.Z = carve(ctx, Wv * sz_Z);
    lg.work = carve(ctx, Wv * sz_wk);
    if (mx) {
      lg.X = carve(ctx, Wv * sz_X);
      lg.Hent = reinterpret_cast<z64*>(carve(ctx, Wv * sz_He));
      lg.R64 = reinterpret_cast<z64*>(carve(ctx, Wv * sz_R));
      lg.C32 = reinterpret_cast<bw::c32*>(carve(ctx, Wv * sz_C));
      lg.G64 = reinterpret_cast<z64*>(carve(ctx, Wv * sz_G));
    }
    z64* Ufull = reinterpret_cast<z64*>(carve(ctx, Wv * sz_Uf));
    PsoSplit X;
    MarkHook hook{ctx, s};
    lg.mark = mark_hook;
    lg.mark_user = &hook;
    if (spin && (st = pso_split_setup(ctx, X, Wv, n, p, op, dblob, sign, o.pso_gap_tol, pso_evals, psog,
                                      &hook, s)))
      return st;
    X.median = o.pso_median;
    for (long long k0 = 0; k0 < K; k0 += Wv) {
      lg.k0 = k0;
      lg.W = std::min(Wv, K - k0);
      // the wave's occupied blocks go straight to U, or through the spin split
      lg.U = spin ? Ufull : U + k0 * (long long)n * p;
      BW_CUDA(bw::launch_states_large(lg, s), "large-n states kernels");
      if (spin) {
        if ((st = pso_split_wave(ctx, X, Ufull, lg.W, k0, U + k0 * (long long)n * p_eff, s))) return st;
        prof_mark(ctx, s, "pso_split");
      }
    }
  }
  if (!large && !fused) prof_mark(ctx, s, "states");

  bw::LoopArgs la;
  std::memset(&la, 0, sizeof(la));
  la.U = U;
  la.M = M;
  la.n = n;
  la.p = p_eff;
  la.N = plane->N;
  la.N_t = plane->N_t;
  la.N_s = PX.N_s;
  la.unitarise = o.unitarise;
  la.max_sweeps = o.max_sweeps;
  la.gap = gap;
  la.pso_gap = psog;
  la.phases = phases;
  la.min_gap = min_gap;
  la.min_pso_gap = min_pso_gap;
  la.status = ctx->status;
  la.u_df = use_df ? 1 : 0;
  la.df_overlaps = mx ? 1 : 0;
  if (kind == LoopKind::Plaquette) {
    if (p_eff <= bw::LOOP_P_MAX)
      BW_CUDA(bw::launch_plaquettes(la, Lx, Ly, phases, chern_out, s), "plaquette kernels");
    else
      BW_CUDA(bw::launch_plaquettes_big(la, M, kb_links, Lx, Ly, phases, chern_out, s),
              "plaquette link GEMM and determinant kernels");
    prof_mark(ctx, s, "plaquettes");
    end_call(ctx, s);
    return BW_OK;
  }
  if (kind == LoopKind::Nested) {
    la.nested = 1;
    // the kernels measure phases from cut as (theta - cut) wrapped into [0, 2 pi)
    double cr = std::fmod(cut, 6.283185307179586);
    if (cr < 0.0) cr += 6.283185307179586;
    la.cut = cr;
    la.first = first;
    la.m = m;
    la.wannier_gap_tol = o.wannier_gap_tol;
    la.w = w;
    la.nu_buf = nu_buf;
    la.min_wannier_gap = min_wgap;
    la.nested_out = nested_out;
  }
  bool nested_done = false;
  if (fused) {
    BW_CUDA(bw::launch_loops_fused_df(sa, la, s, &nested_done, plan_inline ? blob.data.data() : nullptr,
                                      blob.data.size(), dblob),
            "fused states and loop kernel");
  } else {
    if (!bw::loops_form_overlaps(la)) {
      BW_CUDA(bw::launch_overlaps(la, s), "overlap kernel");
      prof_mark(ctx, s, "overlaps");
    }
    BW_CUDA(bw::launch_loops(la, s), "loop kernel");
  }
  prof_mark(ctx, s, "loops");
  if (la.nu_buf) {
    BW_CUDA(bw::launch_wannier(la, s), "Wannier-state kernel");
    prof_mark(ctx, s, "wannier");
  }
  if (kind == LoopKind::Nested && !nested_done) {
    BW_CUDA(bw::launch_nested(la, s), "nested kernel");
    prof_mark(ctx, s, "nested");
  }
  end_call(ctx, s);
  return BW_OK;
}

}  // namespace

extern "C" {

bw_status bw_create(bw_ctx** out, int device, size_t mem_budget_bytes) {
  if (!out) return BW_EINVAL;
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || count == 0) {
    cudaGetLastError();
    return BW_ECUDA;
  }
  if (device < 0 || device >= count) return BW_EINVAL;
  bw_ctx* ctx = new bw_ctx();
  ctx->device = device;
  cudaError_t e = cudaSetDevice(device);
  if (e == cudaSuccess) e = cudaMalloc(&ctx->status, sizeof(bw::DevStatus));
  if (e == cudaSuccess) e = cudaMemset(ctx->status, 0, sizeof(bw::DevStatus));
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->upload_ev, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->done_ev, cudaEventDisableTiming);
  size_t fr = 0, tot = 0;
  if (e == cudaSuccess) e = cudaMemGetInfo(&fr, &tot);
  if (e != cudaSuccess) {
    bw_destroy(ctx);
    return BW_ECUDA;
  }
  ctx->budget = mem_budget_bytes ? mem_budget_bytes : size_t(0.9 * double(fr));
  *out = ctx;
  return BW_OK;
}

void bw_destroy(bw_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  if (ctx->arena && !ctx->external_arena) cudaFree(ctx->arena);
  if (ctx->status) cudaFree(ctx->status);
  if (ctx->staging) cudaFreeHost(ctx->staging);
  if (ctx->upload_ev) cudaEventDestroy(ctx->upload_ev);
  if (ctx->done_ev) cudaEventDestroy(ctx->done_ev);
  for (auto& e : ctx->prof_ev)
    if (e) cudaEventDestroy(e);
  plan_cache_free(ctx);
  delete ctx;
}

const char* bw_last_error(const bw_ctx* ctx) { return ctx ? ctx->err.c_str() : "no context"; }

bw_status bw_set_profiling(bw_ctx* ctx, int enable) {
  if (!ctx) return BW_EINVAL;
  ctx->prof = enable != 0;
  return BW_OK;
}

bw_status bw_selftest_unit_circle(bw_ctx* ctx, double* max_err) {
  if (!ctx) return BW_EINVAL;
  ctx->err.clear();
  if (!max_err) return fail(ctx, BW_EINVAL, "max_err is NULL");
  BW_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
  double* d = nullptr;
  BW_CUDA(cudaMalloc(&d, 3 * sizeof(double)), "cudaMalloc");
  cudaError_t e = cudaMemset(d, 0, 3 * sizeof(double));
  if (e == cudaSuccess) e = bw::launch_selftest_unit_circle(d, nullptr);
  if (e == cudaSuccess) e = cudaMemcpy(max_err, d, 3 * sizeof(double), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return fail(ctx, BW_ECUDA, "self-test: %s", cudaGetErrorString(e));
  return BW_OK;
}

int bw_profile_read(bw_ctx* ctx, int max, char* names, double* ms) {
  if (!ctx || max < 0) return -1;
  if (ctx->prof_n <= 0) return 0;
  if (cudaEventSynchronize(ctx->prof_ev[ctx->prof_n]) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  // durations summed per kernel name, in order of first appearance
  const char* seen[128];
  double tot[128];
  int nu = 0;
  for (int i = 0; i < ctx->prof_n; ++i) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, ctx->prof_ev[i], ctx->prof_ev[i + 1]) != cudaSuccess) {
      cudaGetLastError();
      return -1;
    }
    int u = 0;
    while (u < nu && std::strcmp(seen[u], ctx->prof_names[i]) != 0) ++u;
    if (u == nu) {
      seen[nu] = ctx->prof_names[i];
      tot[nu++] = 0.0;
    }
    tot[u] += double(t);
  }
  const int n = std::min(nu, max);
  for (int i = 0; i < n; ++i) {
    if (ms) ms[i] = tot[i];
    if (names) {
      std::strncpy(names + 32 * i, seen[i], 31);
      names[32 * i + 31] = 0;
    }
  }
  return n;
}

bw_status bw_get_status(bw_ctx* ctx, void* stream, int64_t* k_index) {
  if (!ctx) return BW_EINVAL;
  cudaSetDevice(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  BW_CUDA(cudaStreamSynchronize(s), "cudaStreamSynchronize");
  bw::DevStatus h;
  BW_CUDA(cudaMemcpy(&h, ctx->status, sizeof(h), cudaMemcpyDeviceToHost), "cudaMemcpy status");
  if (k_index) *k_index = h.code ? h.k_index : -1;
  if (h.code) {
    static const char* names[] = {"OK", "EINVAL", "ENOMEM", "EGAP", "EPSOGAP", "EWANGAP",
                                  "ENOCONV", "ETIMEOUT", "ECUDA", "ECANCELED"};
    const char* nm = (h.code >= 0 && h.code <= 9) ? names[h.code] : "?";
    fail(ctx, bw_status(h.code), "device status %s at k index %lld (value %.6e)", nm, h.k_index, h.value);
    BW_CUDA(cudaMemset(ctx->status, 0, sizeof(bw::DevStatus)), "cudaMemset status");
  }
  return bw_status(h.code);
}

bw_status bw_build_hk(bw_ctx* ctx, const bw_model* model, const double* f, int64_t K,
                      int complex64, void* H_out, void* stream) {
  if (!ctx) return BW_EINVAL;
  ctx->err.clear();
  if (K < 0) return fail(ctx, BW_EINVAL, "K < 0");
  if (K > 0 && (!f || !H_out)) return fail(ctx, BW_EINVAL, "f or H_out is NULL");
  const HostPlan* Pc = nullptr;
  const Blob* Bc = nullptr;
  bw_status st = plan_and_blob(ctx, model, &Pc, &Bc);
  if (st) return st;
  const HostPlan& P = *Pc;
  const Blob& blob = *Bc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  begin_call(ctx, s);
  if ((st = reserve(ctx, al256(blob.data.size()) + 4096, s))) return st;
  char* dblob = carve(ctx, blob.data.size());
  if ((st = upload(ctx, blob, dblob, s))) return st;
  bw::BuildArgs a;
  a.model = dev_model(P, dblob);
  a.f = f;
  a.K = K;
  a.complex64 = complex64 ? 1 : 0;
  a.H = H_out;
  prof_start(ctx, s);
  BW_CUDA(bw::launch_build_hk(a, s), "build kernel");
  prof_mark(ctx, s, "build_hk");
  end_call(ctx, s);
  return BW_OK;
}

bw_status bw_winding(bw_ctx* ctx, const double* phases, int32_t N_t, int32_t p, double* sums,
                     double* winding, void* stream) {
  if (!ctx) return BW_EINVAL;
  ctx->err.clear();
  if (N_t < 1 || p < 1) return fail(ctx, BW_EINVAL, "need N_t >= 1 and p >= 1 (N_t = %d, p = %d)", N_t, p);
  if (!phases || !winding) return fail(ctx, BW_EINVAL, "phases or winding is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  begin_call(ctx, s);
  prof_start(ctx, s);
  BW_CUDA(bw::launch_winding(phases, N_t, p, sums, winding, s), "winding kernel");
  prof_mark(ctx, s, "winding");
  end_call(ctx, s);
  return BW_OK;
}

bw_status bw_z2_largest_gap(bw_ctx* ctx, const double* phases, int32_t N_t, int32_t p, int32_t* nu,
                            int32_t* crossings, double* mid, double* width, void* stream) {
  if (!ctx) return BW_EINVAL;
  ctx->err.clear();
  if (N_t < 2 || N_t % 2 || p < 1)
    return fail(ctx, BW_EINVAL, "need an even N_t >= 2 and p >= 1 (N_t = %d, p = %d)", N_t, p);
  if (!phases || !nu) return fail(ctx, BW_EINVAL, "phases or nu is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t h = size_t(N_t / 2);
  const size_t need = (crossings ? 0 : al256(h * sizeof(int32_t))) +
                      (mid ? 0 : al256((h + 1) * sizeof(double))) +
                      (width ? 0 : al256((h + 1) * sizeof(double)));
  begin_call(ctx, s);
  if (need) {
    bw_status st = reserve(ctx, need, s);
    if (st) return st;
    if (!crossings) crossings = reinterpret_cast<int32_t*>(carve(ctx, h * sizeof(int32_t)));
    if (!mid) mid = reinterpret_cast<double*>(carve(ctx, (h + 1) * sizeof(double)));
    if (!width) width = reinterpret_cast<double*>(carve(ctx, (h + 1) * sizeof(double)));
  }
  prof_start(ctx, s);
  BW_CUDA(bw::launch_z2(phases, N_t, p, mid, width, crossings, nu, ctx->status, s), "z2 kernels");
  prof_mark(ctx, s, "z2");
  end_call(ctx, s);
  return BW_OK;
}

bw_status bw_eigh_batched(bw_ctx* ctx, const void* H, const int32_t* n_per, int64_t batch,
                          int32_t n_vec, bw_precision prec, double* evals, void* evecs,
                          void* stream) {
  if (!ctx) return BW_EINVAL;
  ctx->err.clear();
  if (batch < 0) return fail(ctx, BW_EINVAL, "batch < 0");
  if (batch == 0) return BW_OK;
  if (!H || !n_per || !evals) return fail(ctx, BW_EINVAL, "H, n_per or evals is NULL");
  if (prec != BW_FP64 && prec != BW_MIXED) return fail(ctx, BW_EINVAL, "unknown precision");
  if (n_vec < 0) return fail(ctx, BW_EINVAL, "n_vec < 0");
  const bool mx = prec == BW_MIXED;
  int n_max_small = 0;
  std::vector<long long> ho(batch), eo(batch), vo(batch);
  std::vector<long long> ho_s, eo_s, vo_s;
  std::vector<int> np_s, large_idx;
  long long h = 0, ev = 0, vv = 0;
  for (int64_t b = 0; b < batch; ++b) {
    const int n = n_per[b];
    if (n < 1 || n > bw::LARGE_N_MAX)
      return fail(ctx, BW_EINVAL, "matrix %lld has n = %d outside [1, %d]", (long long)b, n, bw::LARGE_N_MAX);
    if (n_vec > n) return fail(ctx, BW_EINVAL, "n_vec = %d exceeds n = %d of matrix %lld", n_vec, n, (long long)b);
    if (n > bw::SMALL_N_MAX && mx && n_vec > 0 && (n_vec >= n || n_vec > 64))
      return fail(ctx, BW_EINVAL, "mixed precision for n > %d needs n_vec < n and n_vec <= 64 "
                  "(matrix %lld: n = %d, n_vec = %d)", bw::SMALL_N_MAX, (long long)b, n, n_vec);
    ho[b] = h;
    eo[b] = ev;
    vo[b] = vv;
    if (n <= bw::SMALL_N_MAX) {
      n_max_small = std::max(n_max_small, n);
      ho_s.push_back(h);
      eo_s.push_back(ev);
      vo_s.push_back(vv);
      np_s.push_back(n);
    } else {
      large_idx.push_back(int(b));
    }
    h += (long long)n * n;
    ev += n;
    vv += (long long)n * n_vec;
  }
  // large matrices grouped by size (one solver configuration per size)
  std::stable_sort(large_idx.begin(), large_idx.end(),
                   [&](int x, int y) { return n_per[x] < n_per[y]; });
  Blob blob;
  const size_t o_h = blob.add(ho_s), o_e = blob.add(eo_s), o_v = blob.add(vo_s), o_n = blob.add(np_s);
  const size_t o_ha = blob.add(ho), o_ea = blob.add(eo), o_va = blob.add(vo), o_li = blob.add(large_idx);
  // scratch of the largest group's wave
  struct Group { int n, first, count; };
  std::vector<Group> groups;
  for (size_t g = 0; g < large_idx.size();) {
    size_t e = g;
    while (e < large_idx.size() && n_per[large_idx[e]] == n_per[large_idx[g]]) ++e;
    groups.push_back({n_per[large_idx[g]], int(g), int(e - g)});
    g = e;
  }
  auto per_k_bytes = [&](int n) {
    const int p = n_vec;
    const bool refine = mx && p > 0;
    const size_t ts = mx ? sizeof(float) : sizeof(double);
    const int nval = n, nvec = mx ? (refine ? n : 0) : p, nbt = refine ? p + 1 : p;
    size_t b = al256(size_t(n) * n * 2 * ts) + 2 * al256(size_t(n) * ts) + al256(size_t(n) * 2 * ts) +
               al256(size_t(nval) * ts) + al256(size_t(nvec) * n * ts) + al256(size_t(nvec) * 6 * n * ts);
    if (refine)
      b += al256(size_t(n) * nbt * sizeof(bw::c32)) + al256(size_t(n) * n * sizeof(z64)) +
           al256(size_t(n) * p * sizeof(z64)) + al256(size_t(n) * p * sizeof(bw::c32)) +
           al256(size_t(p) * p * sizeof(z64));
    b += al256(size_t(n) * std::max(p, 1) * sizeof(z64)) + al256(sizeof(double)) +
         al256(size_t(std::max(p, 1)) * sizeof(double));
    return b;
  };
  const size_t fixed = al256(blob.data.size()) + 4096;
  long long Wv = 0;
  size_t wave_bytes = 0;
  for (const Group& g : groups) {
    const size_t pk = per_k_bytes(g.n);
    const size_t avail = ctx->budget > fixed ? (ctx->budget - fixed) / 2 : 0;
    long long w = std::min<long long>(g.count, std::min<long long>(2048, (long long)(avail / pk)));
    w = std::max<long long>(w, 1);
    Wv = std::max(Wv, w);
    wave_bytes = std::max(wave_bytes, size_t(w) * (pk + 24 * 256));
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  begin_call(ctx, s);
  bw_status st;
  if ((st = reserve(ctx, fixed + wave_bytes, s))) return st;
  char* d = carve(ctx, blob.data.size());
  if ((st = upload(ctx, blob, d, s))) return st;
  prof_start(ctx, s);
  if (!np_s.empty()) {
    bw::EighArgs a;
    a.H = static_cast<const z64*>(H);
    a.h_off = reinterpret_cast<const long long*>(d + o_h);
    a.e_off = reinterpret_cast<const long long*>(d + o_e);
    a.v_off = reinterpret_cast<const long long*>(d + o_v);
    a.n_per = reinterpret_cast<const int*>(d + o_n);
    a.batch = (long long)np_s.size();
    a.n_vec = n_vec;
    a.mixed = mx;
    a.max_sweeps = 30;
    a.evals = evals;
    a.evecs = static_cast<z64*>(evecs);
    a.status = ctx->status;
    BW_CUDA(bw::launch_eigh_small(a, n_max_small, s), "eigh kernel");
    prof_mark(ctx, s, "eigh");
  }
  const size_t mark = ctx->arena_off;
  for (const Group& g : groups) {
    ctx->arena_off = mark;
    const int n = g.n, p = n_vec;
    const bool refine = mx && p > 0;
    const size_t ts = mx ? sizeof(float) : sizeof(double);
    const size_t pk = per_k_bytes(n);
    const size_t avail = ctx->budget > fixed ? (ctx->budget - fixed) / 2 : 0;
    const long long W = std::max<long long>(1, std::min<long long>(g.count, std::min<long long>(2048, (long long)(avail / pk))));
    bw::LargeArgs lg;
    std::memset(&lg, 0, sizeof(lg));
    lg.model.n = n;
    lg.n = n;
    lg.p = p;
    lg.nval = n;
    lg.nvec = mx ? (refine ? n : 0) : p;
    lg.nbt = refine ? p + 1 : p;
    lg.mixed = mx;
    lg.no_refine = mx && !refine;
    lg.gap_tol = 0.0;
    lg.status = ctx->status;
    lg.Hin = static_cast<const z64*>(H);
    lg.h_off = reinterpret_cast<const long long*>(d + o_ha);
    lg.idx = reinterpret_cast<const int*>(d + o_li);
    lg.A = carve(ctx, W * al256(size_t(n) * n * 2 * ts));
    lg.dg = carve(ctx, W * al256(size_t(n) * ts));
    lg.od = carve(ctx, W * al256(size_t(n) * ts));
    lg.Dp = carve(ctx, W * al256(size_t(n) * 2 * ts));
    lg.lam = carve(ctx, W * al256(size_t(n) * ts));
    lg.Z = carve(ctx, W * al256(size_t(lg.nvec) * n * ts));
    lg.work = carve(ctx, W * al256(size_t(lg.nvec) * 6 * n * ts));
    if (refine) {
      lg.X = carve(ctx, W * al256(size_t(n) * lg.nbt * sizeof(bw::c32)));
      lg.Hent = reinterpret_cast<z64*>(carve(ctx, W * al256(size_t(n) * n * sizeof(z64))));
      lg.R64 = reinterpret_cast<z64*>(carve(ctx, W * al256(size_t(n) * p * sizeof(z64))));
      lg.C32 = reinterpret_cast<bw::c32*>(carve(ctx, W * al256(size_t(n) * p * sizeof(bw::c32))));
      lg.G64 = reinterpret_cast<z64*>(carve(ctx, W * al256(size_t(p) * p * sizeof(z64))));
    }
    lg.U = reinterpret_cast<z64*>(carve(ctx, W * al256(size_t(n) * std::max(p, 1) * sizeof(z64))));
    // the refinement's gap test uses gap[k0 + kw]: one slot per matrix of the group
    lg.gap = reinterpret_cast<double*>(carve(ctx, size_t(large_idx.size()) * sizeof(double)));
    double* ritz = reinterpret_cast<double*>(carve(ctx, W * al256(size_t(std::max(p, 1)) * sizeof(double))));
    MarkHook hook{ctx, s};
    lg.mark = mark_hook;
    lg.mark_user = &hook;
    for (long long w0 = 0; w0 < g.count; w0 += W) {
      lg.k0 = g.first + w0;
      lg.W = std::min<long long>(W, g.count - w0);
      BW_CUDA(bw::launch_states_large(lg, s), "large-n eigensolver kernels");
      if (refine) {
        BW_CUDA(bw::launch_eigh_ritz(lg, ritz, s), "Rayleigh-Ritz kernel");
        prof_mark(ctx, s, "eigh_ritz");
      }
      bw::EighScatterArgs e;
      e.idx = lg.idx;
      e.k0 = lg.k0;
      e.W = lg.W;
      e.n = n;
      e.nval = n;
      e.p = p;
      e.mixed = mx;
      e.lam = lg.lam;
      e.U = lg.U;
      e.ritz = refine ? ritz : nullptr;
      e.e_off = reinterpret_cast<const long long*>(d + o_ea);
      e.v_off = reinterpret_cast<const long long*>(d + o_va);
      e.evals = evals;
      e.evecs = static_cast<z64*>(evecs);
      BW_CUDA(bw::launch_eigh_scatter(e, s), "eigh scatter kernel");
      prof_mark(ctx, s, "eigh_scatter");
    }
  }
  end_call(ctx, s);
  return BW_OK;
}

bw_status bw_wilson_loop(bw_ctx* ctx, const bw_model* model, const bw_plane* plane, int32_t p,
                         bw_precision prec, const bw_opts* opts, double* phases, double* min_gap,
                         void* stream) {
  return run_loop(ctx, LoopKind::Plain, model, plane, p, prec, opts, nullptr, 0, 0.0, 0, 0, phases,
                  min_gap, nullptr, nullptr, nullptr, nullptr, static_cast<cudaStream_t>(stream));
}

bw_status bw_nested_wilson_loop(bw_ctx* ctx, const bw_model* model, const bw_plane* plane,
                                int32_t p, double cut, int32_t first, int32_t m,
                                bw_precision prec, const bw_opts* opts, double* phases,
                                double* nested, double* min_wannier_gap, double* min_gap,
                                void* stream) {
  return run_loop(ctx, LoopKind::Nested, model, plane, p, prec, opts, nullptr, 0, cut, first, m,
                  phases, min_gap, nested, min_wannier_gap, nullptr, nullptr,
                  static_cast<cudaStream_t>(stream));
}

bw_status bw_plaquette_flux(bw_ctx* ctx, const bw_model* model, const bw_plane* plane, int32_t p,
                            const bw_c128* spin_op, int32_t sign, bw_precision prec,
                            const bw_opts* opts, double* flux, double* chern, double* min_gap,
                            double* min_pso_gap, void* stream) {
  if (ctx && !flux) {
    ctx->err.clear();
    return fail(ctx, BW_EINVAL, "flux output is NULL");
  }
  return run_loop(ctx, LoopKind::Plaquette, model, plane, p, prec, opts, spin_op, sign, 0.0, 0, 0,
                  flux, min_gap, nullptr, nullptr, nullptr, spin_op ? min_pso_gap : nullptr,
                  static_cast<cudaStream_t>(stream), chern);
}

bw_status bw_wilson_loop_stack(bw_ctx* ctx, const bw_model* model, const bw_plane_stack* stack,
                               int32_t p, bw_precision prec, const bw_opts* opts, double* phases,
                               double* min_gap, void* stream) {
  if (ctx && !stack) {
    ctx->err.clear();
    return fail(ctx, BW_EINVAL, "plane stack is NULL");
  }
  return run_loop(ctx, LoopKind::Plain, model, stack ? &stack->plane : nullptr, p, prec, opts, nullptr, 0,
                  0.0, 0, 0, phases, min_gap, nullptr, nullptr, nullptr, nullptr,
                  static_cast<cudaStream_t>(stream), nullptr, stack ? stack->sweep_dir : nullptr,
                  stack ? stack->N_s : 1);
}

bw_status bw_nested_wilson_loop_stack(bw_ctx* ctx, const bw_model* model, const bw_plane_stack* stack,
                                      int32_t p, double cut, int32_t first, int32_t m,
                                      bw_precision prec, const bw_opts* opts, double* phases,
                                      double* nested, double* min_wannier_gap, double* min_gap,
                                      void* stream) {
  if (ctx && !stack) {
    ctx->err.clear();
    return fail(ctx, BW_EINVAL, "plane stack is NULL");
  }
  return run_loop(ctx, LoopKind::Nested, model, stack ? &stack->plane : nullptr, p, prec, opts, nullptr, 0,
                  cut, first, m, phases, min_gap, nested, min_wannier_gap, nullptr, nullptr,
                  static_cast<cudaStream_t>(stream), nullptr, stack ? stack->sweep_dir : nullptr,
                  stack ? stack->N_s : 1);
}

bw_status bw_spin_resolved_wilson_loop_stack(bw_ctx* ctx, const bw_model* model,
                                             const bw_plane_stack* stack, int32_t p,
                                             const bw_c128* spin_op, int32_t sign, bw_precision prec,
                                             const bw_opts* opts, double* phases, double* pso_evals,
                                             double* min_pso_gap, double* min_gap, void* stream) {
  if (ctx && !stack) {
    ctx->err.clear();
    return fail(ctx, BW_EINVAL, "plane stack is NULL");
  }
  return run_loop(ctx, LoopKind::Spin, model, stack ? &stack->plane : nullptr, p, prec, opts, spin_op, sign,
                  0.0, 0, 0, phases, min_gap, nullptr, nullptr, pso_evals, min_pso_gap,
                  static_cast<cudaStream_t>(stream), nullptr, stack ? stack->sweep_dir : nullptr,
                  stack ? stack->N_s : 1);
}

bw_status bw_spin_resolved_wilson_loop(bw_ctx* ctx, const bw_model* model, const bw_plane* plane,
                                       int32_t p, const bw_c128* spin_op, int32_t sign,
                                       bw_precision prec, const bw_opts* opts, double* phases,
                                       double* pso_evals, double* min_pso_gap, double* min_gap,
                                       void* stream) {
  return run_loop(ctx, LoopKind::Spin, model, plane, p, prec, opts, spin_op, sign, 0.0, 0, 0,
                  phases, min_gap, nullptr, nullptr, pso_evals, min_pso_gap,
                  static_cast<cudaStream_t>(stream));
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free Wilson loop.
//
// Some callers cannot let a library allocate device memory: a host program that
// hands all device memory to its own pool under a hard cap, a plugin that runs
// inside another program's CUDA context, or a latency-critical loop where
// cudaMalloc / cudaFree would block on (or implicitly synchronise) the device.
// For them bw_wilson_loop_noalloc runs the kernels of bw_wilson_loop with all of
// its scratch (the hopping-list plan, the occupied states, the overlaps when the
// loop kernel does not form them itself, the gaps and the status word) in one
// fixed file-scope device array.  The array is part of the library image: every
// device that loads the library holds it until the process exits.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kNoAllocScratchBytes = size_t(8) << 20;  // 8 MiB
constexpr int kNoAllocMaxContexts = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// A __device__ array has one instance in every CUDA context that loads the library
// (a device's primary context, or a context the caller created with the driver
// API), each at its own address.  The address is looked up once per context, with
// that context current, and kept under the context's unique id (cuCtxGetId; ids are
// never reused within a process, unlike context handles).
using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

struct NoAllocSlot {
  unsigned long long ctx_id;
  char* base;
};

std::mutex g_noalloc_mu;
NoAllocSlot g_noalloc_slot[kNoAllocMaxContexts];
int g_noalloc_slots = 0;
CtxGetCurrentFn g_cu_ctx_get_current = nullptr;
CtxGetIdFn g_cu_ctx_get_id = nullptr;

// Driver-API functions through the runtime's entry-point query (no link against the
// driver library).  Called with g_noalloc_mu held.
bw_status noalloc_driver_entry_points(bw_ctx* ctx) {
  if (g_cu_ctx_get_current && g_cu_ctx_get_id) return BW_OK;
  void* f1 = nullptr;
  void* f2 = nullptr;
  cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = q1;
  BW_CUDA(cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1),
          "cudaGetDriverEntryPointByVersion(cuCtxGetCurrent)");
  BW_CUDA(cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2),
          "cudaGetDriverEntryPointByVersion(cuCtxGetId)");
  if (q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
    return fail(ctx, BW_ECUDA, "the CUDA driver does not provide cuCtxGetCurrent / cuCtxGetId");
  g_cu_ctx_get_current = reinterpret_cast<CtxGetCurrentFn>(f1);
  g_cu_ctx_get_id = reinterpret_cast<CtxGetIdFn>(f2);
  return BW_OK;
}

// Id of the context current on this thread; 0 when none is current yet.
bw_status noalloc_context_id(bw_ctx* ctx, unsigned long long* id) {
  *id = 0;
  CUcontext c = nullptr;
  if (g_cu_ctx_get_current(&c) != CUDA_SUCCESS)
    return fail(ctx, BW_ECUDA, "cuCtxGetCurrent failed");
  if (c && g_cu_ctx_get_id(c, id) != CUDA_SUCCESS) return fail(ctx, BW_ECUDA, "cuCtxGetId failed");
  return BW_OK;
}

// Device address of the fixed array in the context current on this thread.  The
// host-side name g_noalloc_scratch is only a stand-in for the symbol and must never
// reach a kernel; the address comes from cudaGetSymbolAddress, looked up the first
// time each context calls (with no context current yet, the runtime makes the
// current device's primary context current during the lookup).
bw_status noalloc_base(bw_ctx* ctx, char** out) {
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  bw_status st = noalloc_driver_entry_points(ctx);
  if (st) return st;
  unsigned long long id = 0;
  if ((st = noalloc_context_id(ctx, &id))) return st;
  for (int i = 0; id && i < g_noalloc_slots; ++i)
    if (g_noalloc_slot[i].ctx_id == id) {
      *out = g_noalloc_slot[i].base;
      return BW_OK;
    }
  void* p = nullptr;
  BW_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch), "cudaGetSymbolAddress");
  if (!id && (st = noalloc_context_id(ctx, &id))) return st;
  if (id && g_noalloc_slots < kNoAllocMaxContexts) g_noalloc_slot[g_noalloc_slots++] = {id, static_cast<char*>(p)};
  *out = static_cast<char*>(p);
  return BW_OK;
}

bw_status noalloc_run(bw_ctx* ctx, const bw_model* model, const bw_plane* plane, int p,
                      bw_precision prec, const bw_opts* opts, double* phases, double* min_gap,
                      cudaStream_t s) {
  bw_status st = check_plane(ctx, plane, false);
  if (st) return st;
  PlaneX PX;
  if ((st = stack_planes(ctx, plane, nullptr, 1, PX))) return st;
  if (prec != BW_FP64 && prec != BW_MIXED) return fail(ctx, BW_EINVAL, "unknown precision %d", int(prec));
  if (!phases) return fail(ctx, BW_EINVAL, "phases output is NULL");
  HostPlan P;
  if ((st = make_plan(ctx, model, P))) return st;
  const int n = P.n;
  if (p < 1 || p > n) return fail(ctx, BW_EINVAL, "need 1 <= p <= n (p = %d, n = %d)", p, n);
  if (n > bw::SMALL_N_MAX)
    return fail(ctx, BW_EINVAL, "n = %d exceeds the largest supported size %d", n, bw::SMALL_N_MAX);
  if (p > bw::LOOP_P_MAX) return fail(ctx, BW_EINVAL, "p = %d exceeds %d", p, bw::LOOP_P_MAX);
  const Opts o = resolve_opts(opts, P.tmax);
  if (o.unitarise && p > 32) return fail(ctx, BW_EINVAL, "unitarise supports p <= 32");
  const long long K = (long long)plane->N * plane->N_t;
  Blob blob;
  plan_to_blob(P, blob);
  bw::LoopArgs la;
  std::memset(&la, 0, sizeof(la));
  la.n = n;
  la.p = p;
  la.N = plane->N;
  la.N_t = plane->N_t;
  la.unitarise = o.unitarise;
  la.max_sweeps = o.max_sweeps;
  // the scan loop kernel forms the overlaps itself: no overlap buffer then
  const bool need_M = !bw::loops_form_overlaps(la);
  const size_t bStat = al256(sizeof(bw::DevStatus));
  const size_t bBlob = al256(blob.data.size());
  const size_t bU = al256(size_t(K) * n * p * sizeof(z64));
  const size_t bGap = al256(size_t(K) * sizeof(double));
  const size_t bM = need_M ? al256(size_t(K) * p * p * sizeof(z64)) : 0;
  const size_t total = bStat + bBlob + bU + bGap + bM;
  if (total > kNoAllocScratchBytes)
    return fail(ctx, BW_ENOMEM,
                "this problem needs %zu bytes of scratch; the fixed scratch of "
                "bw_wilson_loop_noalloc holds %zu bytes (K * n * p * 16 + K * 8 + the "
                "hopping-list plan, plus K * p * p * 16 when the loop kernel does not form the "
                "overlaps itself, must fit)",
                total, kNoAllocScratchBytes);
  char* base = nullptr;
  if ((st = noalloc_base(ctx, &base))) return st;
  bw::DevStatus* status = reinterpret_cast<bw::DevStatus*>(base);
  char* dblob = base + bStat;
  z64* U = reinterpret_cast<z64*>(dblob + bBlob);
  double* gap = reinterpret_cast<double*>(reinterpret_cast<char*>(U) + bU);
  z64* M = need_M ? reinterpret_cast<z64*>(reinterpret_cast<char*>(gap) + bGap) : nullptr;
  // The array keeps the previous call's contents: the status word must start at zero.
  BW_CUDA(cudaMemsetAsync(status, 0, sizeof(bw::DevStatus), s), "cudaMemsetAsync");
  BW_CUDA(cudaMemcpyAsync(dblob, blob.data.data(), blob.data.size(), cudaMemcpyHostToDevice, s),
          "cudaMemcpyAsync");

  bw::StatesArgs sa;
  std::memset(&sa, 0, sizeof(sa));
  sa.model = dev_model(P, dblob);
  sa.row_ptr = reinterpret_cast<const int*>(dblob + P.o_rowptr);
  sa.plane = dev_plane(PX);
  sa.K = K;
  sa.p = p;
  sa.mixed = prec == BW_MIXED;
  sa.max_sweeps = o.max_sweeps;
  sa.gap_tol = o.gap_tol;
  sa.U = U;
  sa.gap = gap;
  sa.status = status;
  BW_CUDA(bw::launch_states_small(sa, p, s), "states kernel");
  la.U = U;
  la.M = M;
  la.gap = gap;
  la.phases = phases;
  la.min_gap = min_gap;
  la.status = status;
  BW_CUDA(bw::launch_overlaps(la, s), "overlap kernel");
  BW_CUDA(bw::launch_loops(la, s), "loop kernel");
  // Read the status word behind the kernels on the caller's stream, then wait for that
  // stream alone (the copy of the host list above is complete by then as well).
  bw::DevStatus h;
  BW_CUDA(cudaMemcpyAsync(&h, status, sizeof(h), cudaMemcpyDeviceToHost, s), "cudaMemcpyAsync status");
  BW_CUDA(cudaStreamSynchronize(s), "cudaStreamSynchronize");
  if (h.code) {
    static const char* names[] = {"OK", "EINVAL", "ENOMEM", "EGAP", "EPSOGAP", "EWANGAP",
                                  "ENOCONV", "ETIMEOUT", "ECUDA", "ECANCELED"};
    const char* nm = (h.code >= 0 && h.code <= 9) ? names[h.code] : "?";
    return fail(ctx, bw_status(h.code), "device status %s at k index %lld (value %.6e)", nm,
                h.k_index, h.value);
  }
  return BW_OK;
}

}  // namespace

extern "C" bw_status bw_wilson_loop_noalloc(const bw_model* model, const bw_plane* plane,
                                            int32_t p, bw_precision prec, const bw_opts* opts,
                                            double* phases, double* min_gap, void* stream,
                                            char* err, size_t err_len) {
  bw_ctx tmp;  // host-side message holder only; no device resources
  const bw_status st = noalloc_run(&tmp, model, plane, p, prec, opts, phases, min_gap,
                                   static_cast<cudaStream_t>(stream));
  if (err && err_len) {
    std::strncpy(err, tmp.err.c_str(), err_len - 1);
    err[err_len - 1] = 0;
  }
  return st;
}

extern "C" bw_status bw_wilson_loop_workspace(bw_ctx* ctx, const bw_model* model,
                                              const bw_plane* plane, int32_t p, bw_precision prec,
                                              const bw_opts* opts, size_t* bytes) {
  if (!ctx || !bytes) return BW_EINVAL;
  double dummy = 0.0;
  ctx->query_only = true;
  ctx->query_bytes = 0;
  const bw_status st = run_loop(ctx, LoopKind::Plain, model, plane, p, prec, opts, nullptr, 0, 0.0, 0,
                                0, &dummy, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr);
  ctx->query_only = false;
  if (st == kQueryDone) {
    *bytes = ctx->query_bytes;
    return BW_OK;
  }
  return st == BW_OK ? BW_EINVAL : st;
}

namespace bw_internal {

bw_status attach_arena(bw_ctx* ctx, void* base, size_t cap) {
  if (!ctx) return BW_EINVAL;
  if (ctx->arena && !ctx->external_arena) {
    cudaSetDevice(ctx->device);
    cudaFree(ctx->arena);
  }
  ctx->arena = static_cast<char*>(base);
  ctx->arena_cap = cap;
  ctx->external_arena = true;
  ctx->budget = cap;
  return BW_OK;
}

bw_status reserve_staging(bw_ctx* ctx, size_t bytes) {
  if (bytes <= ctx->staging_cap) return BW_OK;
  cudaSetDevice(ctx->device);
  if (ctx->staging) cudaFreeHost(ctx->staging);
  ctx->staging = nullptr;
  ctx->staging_cap = 0;
  BW_CUDA(cudaMallocHost(&ctx->staging, bytes), "cudaMallocHost");
  ctx->staging_cap = bytes;
  return BW_OK;
}

bw_status clear_status_async(bw_ctx* ctx, cudaStream_t s) {
  BW_CUDA(cudaMemsetAsync(ctx->status, 0, sizeof(bw::DevStatus), s), "cudaMemsetAsync status");
  return BW_OK;
}

bw_status status_to_host_async(bw_ctx* ctx, void* pinned_dst, cudaStream_t s) {
  BW_CUDA(cudaMemcpyAsync(pinned_dst, ctx->status, sizeof(bw::DevStatus), cudaMemcpyDeviceToHost, s),
          "cudaMemcpyAsync status");
  return BW_OK;
}

const char* last_error(const bw_ctx* ctx) { return ctx->err.c_str(); }

}  // namespace bw_internal
