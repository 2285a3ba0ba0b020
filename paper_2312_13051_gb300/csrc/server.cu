// Request server: continuous batching of Wilson-loop solves on one GPU.
//
// A request (hopping list, plane, p, precision) is admitted when a slot is free and
// a contiguous region of the server's device pool holds its scratch and outputs;
// requests that arrive while others run are admitted as soon as slots and memory
// free up, so their kernels overlap on the device (one CUDA stream per slot).  The
// pool is allocated once at creation, so admission never calls cudaMalloc or
// cudaFree (which would synchronise the device under the other slots' work).
// A worker thread launches admitted requests, watches the slots' completion events,
// copies results to the caller's host buffers and releases the memory.
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/berrywl.h"
#include "internal.h"

namespace {

using Clock = std::chrono::steady_clock;

size_t al256s(size_t x) { return (x + 255) & ~size_t(255); }

struct Request {
  int64_t id = 0;
  int32_t n = 0;
  std::vector<int32_t> R, I, J;
  std::vector<bw_c128> T;
  bw_plane plane{};
  int32_t p = 0;
  bw_precision prec = BW_FP64;
  bw_opts opts{};
  bool has_opts = false;
  double* out_phases = nullptr;  // caller host buffers
  double* out_gap = nullptr;
  size_t scratch = 0, total = 0, off = 0;
  Clock::time_point t_submit, t_admit, t_done;
  float device_ms = 0.f;
  bw_status status = BW_OK;
  int64_t k_index = -1;
  std::string err;
};

struct Slot {
  bw_ctx* ctx = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t ev_start = nullptr, ev_end = nullptr;
  double* h_out = nullptr;  // pinned: phases then gap
  size_t h_cap = 0;
  unsigned char* h_status = nullptr;  // pinned copy of the device status word
  Request* req = nullptr;
};

// First-fit allocator over [0, cap) in 256-byte units, free list kept sorted.
struct Pool {
  std::map<size_t, size_t> free_;  // offset -> size
  void init(size_t cap) { free_.clear(); free_[0] = cap; }
  bool take(size_t bytes, size_t& off) {
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < bytes) continue;
      off = it->first;
      const size_t rest = it->second - bytes;
      free_.erase(it);
      if (rest) free_[off + bytes] = rest;
      return true;
    }
    return false;
  }
  void give(size_t off, size_t bytes) {
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
};

}  // namespace

struct bw_server {
  int device = 0;
  size_t budget = 0, per_request = 0;
  char* pool_base = nullptr;
  Pool pool;
  std::vector<Slot> slots;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> queue;
  std::map<int64_t, Request*> done;
  std::vector<int64_t> done_order;
  std::thread worker;
  bool stop = false;
  int64_t next_id = 1;
  std::mutex qmu;
  bw_ctx* qctx = nullptr;  // workspace queries only
  std::string err;
};

namespace {

bw_status server_fail(bw_server* s, bw_status st, const char* msg) {
  if (s) s->err = msg;
  return st;
}

// Launches an admitted request on its slot (worker thread, outside the lock).
void launch(bw_server* sv, Slot& sl, Request* r) {
  char* base = sv->pool_base + r->off;
  const size_t out_ph = size_t(r->plane.N_t) * r->p, out_all = out_ph + size_t(r->plane.N_t);
  double* d_out = reinterpret_cast<double*>(base + al256s(r->scratch));
  bw_internal::attach_arena(sl.ctx, base, r->scratch);
  cudaEventRecord(sl.ev_start, sl.stream);
  bw_status st = bw_internal::clear_status_async(sl.ctx, sl.stream);
  if (st == BW_OK) {
    bw_model m;
    m.n = r->n;
    m.nnz = int64_t(r->T.size());
    m.R = r->R.data();
    m.i = r->I.data();
    m.j = r->J.data();
    m.t = r->T.data();
    st = bw_wilson_loop(sl.ctx, &m, &r->plane, r->p, r->prec, r->has_opts ? &r->opts : nullptr, d_out,
                        d_out + out_ph, sl.stream);
    if (st != BW_OK) r->err = bw_internal::last_error(sl.ctx);
  }
  r->status = st;
  if (st == BW_OK) {
    cudaMemcpyAsync(sl.h_out, d_out, out_all * sizeof(double), cudaMemcpyDeviceToHost, sl.stream);
    bw_internal::status_to_host_async(sl.ctx, sl.h_status, sl.stream);
  }
  cudaEventRecord(sl.ev_end, sl.stream);
}

// Completes the request of a slot whose end event has fired (under the lock).
void complete(bw_server* sv, Slot& sl) {
  Request* r = sl.req;
  r->t_done = Clock::now();
  cudaEventElapsedTime(&r->device_ms, sl.ev_start, sl.ev_end);
  if (r->status == BW_OK) {
    int code = 0;
    long long k = -1;
    std::memcpy(&code, sl.h_status, sizeof(int));
    std::memcpy(&k, sl.h_status + 8, sizeof(long long));
    if (code != 0) {
      r->status = bw_status(code);
      r->k_index = k;
      char buf[128];
      std::snprintf(buf, sizeof(buf), "device status %d at k index %lld", code, k);
      r->err = buf;
    }
    const size_t out_ph = size_t(r->plane.N_t) * r->p;
    std::memcpy(r->out_phases, sl.h_out, out_ph * sizeof(double));
    if (r->out_gap) std::memcpy(r->out_gap, sl.h_out + out_ph, size_t(r->plane.N_t) * sizeof(double));
  }
  sv->pool.give(r->off, r->total);
  sl.req = nullptr;
  sv->done[r->id] = r;
  sv->done_order.push_back(r->id);
}

void worker_main(bw_server* sv) {
  cudaSetDevice(sv->device);
  std::vector<std::pair<Slot*, Request*>> admit;
  while (true) {
    admit.clear();
    {
      std::unique_lock<std::mutex> lk(sv->mu);
      bool progressed = false;
      int busy = 0;
      for (auto& sl : sv->slots) {
        if (!sl.req) continue;
        const cudaError_t q = cudaEventQuery(sl.ev_end);
        if (q == cudaErrorNotReady) {
          ++busy;
          continue;
        }
        if (q != cudaSuccess) {
          cudaGetLastError();
          sl.req->status = BW_ECUDA;
          sl.req->err = cudaGetErrorString(q);
        }
        complete(sv, sl);
        progressed = true;
      }
      if (progressed) sv->cv_done.notify_all();
      if (sv->stop) {
        if (busy == 0) break;
      } else {
        // admission in arrival order; a request that does not fit yet lets later,
        // smaller ones through (memory-admitted continuous batching)
        for (auto it = sv->queue.begin(); it != sv->queue.end();) {
          Slot* free_slot = nullptr;
          for (auto& sl : sv->slots)
            if (!sl.req) {
              free_slot = &sl;
              break;
            }
          if (!free_slot) break;
          size_t off = 0;
          if (!sv->pool.take((*it)->total, off)) {
            ++it;
            continue;
          }
          Request* r = *it;
          r->off = off;
          r->t_admit = Clock::now();
          free_slot->req = r;
          admit.emplace_back(free_slot, r);
          it = sv->queue.erase(it);
        }
      }
      if (admit.empty() && !progressed)
        sv->cv_work.wait_for(lk, std::chrono::microseconds(busy ? 20 : 500));
    }
    for (auto& a : admit) launch(sv, *a.first, a.second);
  }
}

}  // namespace

extern "C" {

bw_status bw_server_create(bw_server** out, int device, int32_t max_slots, size_t mem_budget_bytes) {
  if (!out || max_slots < 1 || max_slots > 64) return BW_EINVAL;
  *out = nullptr;
  bw_server* sv = new bw_server();
  sv->device = device;
  if (cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    delete sv;
    return BW_ECUDA;
  }
  size_t fr = 0, tot = 0;
  cudaMemGetInfo(&fr, &tot);
  sv->budget = al256s(mem_budget_bytes ? mem_budget_bytes : size_t(0.8 * double(fr)));
  // one request may take at most half of the pool, so that two large ones overlap
  sv->per_request = sv->budget / 2;
  bw_status st = bw_create(&sv->qctx, device, sv->per_request);
  if (st != BW_OK) {
    delete sv;
    return st;
  }
  cudaError_t e = cudaMalloc(&sv->pool_base, sv->budget);
  if (e != cudaSuccess) {
    cudaGetLastError();
    bw_destroy(sv->qctx);
    delete sv;
    return BW_ENOMEM;
  }
  sv->pool.init(sv->budget);
  sv->slots.resize(max_slots);
  for (auto& sl : sv->slots) {
    if ((st = bw_create(&sl.ctx, device, 0)) != BW_OK) break;
    bw_internal::attach_arena(sl.ctx, sv->pool_base, 0);
    if ((st = bw_internal::reserve_staging(sl.ctx, size_t(8) << 20)) != BW_OK) break;
    if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&sl.ev_start) != cudaSuccess || cudaEventCreate(&sl.ev_end) != cudaSuccess ||
        cudaMallocHost(&sl.h_out, size_t(4) << 20) != cudaSuccess ||
        cudaMallocHost(&sl.h_status, 64) != cudaSuccess) {
      st = BW_ECUDA;
      break;
    }
    sl.h_cap = (size_t(4) << 20) / sizeof(double);
  }
  if (st != BW_OK) {
    cudaGetLastError();
    bw_server_destroy(sv);
    return st;
  }
  sv->worker = std::thread(worker_main, sv);
  *out = sv;
  return BW_OK;
}

void bw_server_destroy(bw_server* sv) {
  if (!sv) return;
  if (sv->worker.joinable()) {
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      sv->stop = true;
    }
    sv->cv_work.notify_all();
    sv->worker.join();
  }
  cudaSetDevice(sv->device);
  for (Request* r : sv->queue) delete r;
  for (auto& kv : sv->done) delete kv.second;
  for (auto& sl : sv->slots) {
    if (sl.stream) cudaStreamSynchronize(sl.stream);
    if (sl.ctx) bw_destroy(sl.ctx);
    if (sl.stream) cudaStreamDestroy(sl.stream);
    if (sl.ev_start) cudaEventDestroy(sl.ev_start);
    if (sl.ev_end) cudaEventDestroy(sl.ev_end);
    if (sl.h_out) cudaFreeHost(sl.h_out);
    if (sl.h_status) cudaFreeHost(sl.h_status);
  }
  if (sv->pool_base) cudaFree(sv->pool_base);
  if (sv->qctx) bw_destroy(sv->qctx);
  delete sv;
}

const char* bw_server_last_error(const bw_server* sv) { return sv ? sv->err.c_str() : "no server"; }

bw_status bw_server_submit(bw_server* sv, const bw_model* model, const bw_plane* plane, int32_t p,
                           bw_precision prec, const bw_opts* opts, double* phases, double* min_gap,
                           int64_t* id) {
  if (!sv || !model || !plane || !phases || !id) return BW_EINVAL;
  if (model->nnz < 0 || (model->nnz > 0 && (!model->R || !model->i || !model->j || !model->t)))
    return server_fail(sv, BW_EINVAL, "hopping list arrays are NULL");
  size_t ws = 0;
  {
    // validates the request and sizes its scratch (host work only)
    std::lock_guard<std::mutex> lk(sv->qmu);
    const bw_status st = bw_wilson_loop_workspace(sv->qctx, model, plane, p, prec, opts, &ws);
    if (st != BW_OK) return server_fail(sv, st, bw_last_error(sv->qctx));
  }
  const size_t n_out = size_t(plane->N_t) * (size_t(p) + 1);
  if (n_out > sv->slots[0].h_cap) return server_fail(sv, BW_EINVAL, "result larger than a slot's host buffer");
  Request* r = new Request();
  r->n = model->n;
  const size_t nnz = size_t(model->nnz);
  r->R.assign(model->R, model->R + 3 * nnz);
  r->I.assign(model->i, model->i + nnz);
  r->J.assign(model->j, model->j + nnz);
  r->T.assign(model->t, model->t + nnz);
  r->plane = *plane;
  r->p = p;
  r->prec = prec;
  if (opts) {
    r->opts = *opts;
    r->has_opts = true;
  }
  r->out_phases = phases;
  r->out_gap = min_gap;
  r->scratch = ws;
  r->total = al256s(ws) + al256s(n_out * sizeof(double));
  if (r->total > sv->budget) {
    delete r;
    return server_fail(sv, BW_ENOMEM, "request needs more device memory than the server's pool");
  }
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    r->id = sv->next_id++;
    r->t_submit = Clock::now();
    sv->queue.push_back(r);
    *id = r->id;
  }
  sv->cv_work.notify_all();
  return BW_OK;
}

namespace {
void fill_info(const Request* r, bw_request_info* info) {
  using ms = std::chrono::duration<double, std::milli>;
  info->id = r->id;
  info->status = int32_t(r->status);
  info->reserved = 0;
  info->k_index = r->k_index;
  info->latency_ms = ms(r->t_done - r->t_submit).count();
  info->queue_ms = ms(r->t_admit - r->t_submit).count();
  info->device_ms = r->device_ms;
  std::snprintf(info->message, sizeof(info->message), "%s", r->err.c_str());
}
}  // namespace

int bw_server_poll(bw_server* sv, bw_request_info* out, int max) {
  if (!sv || max < 0 || (max > 0 && !out)) return -1;
  std::lock_guard<std::mutex> lk(sv->mu);
  int n = 0;
  auto it = sv->done_order.begin();
  for (; it != sv->done_order.end() && n < max; ++it, ++n) {
    Request* r = sv->done[*it];
    fill_info(r, out + n);
    sv->done.erase(*it);
    delete r;
  }
  sv->done_order.erase(sv->done_order.begin(), it);
  return n;
}

bw_status bw_server_wait(bw_server* sv, int64_t id, double timeout_s, bw_request_info* info) {
  if (!sv) return BW_EINVAL;
  std::unique_lock<std::mutex> lk(sv->mu);
  const auto until = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                        std::chrono::duration<double>(timeout_s > 0 ? timeout_s : 0.0));
  while (!sv->done.count(id)) {
    bool known = false;
    for (Request* r : sv->queue) known |= r->id == id;
    for (auto& sl : sv->slots) known |= sl.req && sl.req->id == id;
    if (!known) return server_fail(sv, BW_EINVAL, "unknown request id (already collected?)");
    if (sv->cv_done.wait_until(lk, until) == std::cv_status::timeout && !sv->done.count(id))
      return BW_ETIMEOUT;
  }
  Request* r = sv->done[id];
  if (info) fill_info(r, info);
  sv->done.erase(id);
  for (auto it = sv->done_order.begin(); it != sv->done_order.end(); ++it)
    if (*it == id) {
      sv->done_order.erase(it);
      break;
    }
  delete r;
  return BW_OK;
}

bw_status bw_server_cancel(bw_server* sv, int64_t id) {
  if (!sv) return BW_EINVAL;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    Request* r = nullptr;
    for (auto it = sv->queue.begin(); it != sv->queue.end(); ++it)
      if ((*it)->id == id) {
        r = *it;
        sv->queue.erase(it);
        break;
      }
    if (!r) {
      for (auto& sl : sv->slots)
        if (sl.req && sl.req->id == id)
          return server_fail(sv, BW_EINVAL, "request is already running on the GPU; it runs to completion");
      return server_fail(sv, BW_EINVAL, "unknown request id (finished, collected or never submitted)");
    }
    r->t_admit = r->t_done = Clock::now();
    r->status = BW_ECANCELED;
    r->err = "cancelled before admission";
    sv->done[r->id] = r;
    sv->done_order.push_back(r->id);
  }
  sv->cv_done.notify_all();
  return BW_OK;
}

int64_t bw_server_outstanding(bw_server* sv) {
  if (!sv) return -1;
  std::lock_guard<std::mutex> lk(sv->mu);
  int64_t n = int64_t(sv->queue.size());
  for (auto& sl : sv->slots) n += sl.req != nullptr;
  return n;
}

}  // extern "C"
