// Serving loop: a persistent request queue on one GPU that admits solve requests of different
// grid levels, ranks and loads as they arrive, by device-memory budget and free worker slot, and
// runs the admitted ones concurrently.
//
// Structure:
//  - W worker threads, each with its own library context on its own non-blocking CUDA stream,
//    so the kernels of different requests overlap on the device (continuous batching: a request
//    is admitted the moment a slot and enough of the budget are free, not when a batch closes);
//  - each worker's cooperative kernels are sized to 1/W of the SMs (tnfem_ctx::sm_share), so the
//    grids of all workers can be resident together whatever order the hardware starts them in;
//  - each worker allocates stream-ordered from the device's memory pool, so a request's
//    allocations and frees do not call cudaMalloc / cudaFree (which would synchronise the device
//    and serialise the workers);
//  - admission: requests wait in arrival order; the head is admitted when a worker is idle and
//    the sum of the admitted requests' memory estimates stays within the budget (one request is
//    always admitted when nothing else runs, so an over-budget request fails on its own budget
//    check instead of blocking the queue);
//  - the solution cores are copied to host memory by the worker, so a request's result outlives
//    the worker's device buffers and the caller needs no context.
// Requests are independent AMEn solves (Section 5.4, Algorithm 2) of independently built
// operators and loads (Algorithm 1, Section 5.3); the loop adds scheduling only.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.h"

namespace {

double now_us() {
  return std::chrono::duration<double, std::micro>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// Device allocations of a worker: stream-ordered (cudaMallocAsync / cudaFreeAsync on the worker's
// stream) from the device's memory pool, whose release threshold keeps freed memory cached, so a
// request's allocations and frees neither call cudaMalloc / cudaFree nor synchronise the device.
void* stream_alloc(size_t bytes, void* user) {
  void* p = nullptr;
  if (cudaMallocAsync(&p, bytes, static_cast<cudaStream_t>(user)) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}
void stream_free(void* p, void* user) { cudaFreeAsync(p, static_cast<cudaStream_t>(user)); }

struct Request {
  uint64_t id = 0;
  tnfem_grid grid{};
  tnfem_material mat{};
  std::vector<tnfem_load> loads;
  std::vector<std::vector<double>> amp, phase;  // owned copies of the Fourier arrays
  std::vector<std::vector<int>> wave;
  tnfem_solve_opts opts{};
  size_t est = 0;
  // result
  bool done = false;
  tnfem_status status = TNFEM_OK;
  std::string err;
  tnfem_solve_info info{};
  std::vector<int> ranks, modes;
  std::vector<double> cores;
  size_t peak_bytes = 0;
  int worker = -1;
  double t_submit = 0, t_start = 0, t_end = 0;
};

}  // namespace

struct tnfem_server {
  int device = 0;
  int workers = 1;
  size_t budget = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> queue;                              // submitted, not yet admitted
  std::unordered_map<uint64_t, std::unique_ptr<Request>> reqs;
  size_t admitted_bytes = 0;
  int running = 0;
  bool stopping = false;
  uint64_t next_id = 1;
  std::vector<std::thread> threads;
  std::vector<std::string> worker_err;
  std::atomic<int> ready{0};
  double t0 = 0;  // server start (steady clock, us)
};

namespace tnfem {

// Estimate (with margin) of the device memory one solve request holds at its peak, calibrated on
// GB300 measurements of the peak bytes a context held (tnfem_memory_stats) while building and
// solving (serving's `peak_bytes` reports the measured value next to it):
//  - the sweep holds environments and work arrays sized by the rank cap R (+ the enrichment rank):
//    about 0.09 MiB x R^2 in 2D (430 MiB at R = 68, 900 MiB at R = 100, nearly independent of the
//    levels), scaled by the operator rank ratio (about 340 / 53) in 3D;
//  - in 3D the operator's device rounding dominates (raw Kronecker-sum ranks 441 - 576): 0.3 - 0.5
//    GiB at 2^3 nodes per axis, 18.4 GiB at 2^5, 19.1 GiB at 2^6, 25.1 GiB at 2^7; larger grids are
//    extrapolated at +3.4 GiB per level, with a further factor 1.5 from 2^8 on (raw rank 576).
size_t serve_estimate_bytes(const tnfem_grid& g, const tnfem_solve_opts& o) {
  const double MiB = 1024.0 * 1024.0, GiB = 1024.0 * MiB;
  const int d = g.levels + 1;
  // no bond of the train can exceed min(product of the modes left of it, product right of it)
  double rmax_bond = 1.0, left = g.dim;
  for (int k = 1; k < d; ++k) {
    const double right = std::pow((double)(1 << g.dim), d - k);
    rmax_bond = std::max(rmax_bond, std::min(left, right));
    left *= (double)(1 << g.dim);
  }
  const double R = std::min((double)o.rank_cap, rmax_bond) + std::max(0, o.kickrank);
  double sweep = 48.0 * MiB + 0.095 * MiB * R * R + 2.0 * MiB * d;
  double build = 0.0;
  if (g.dim == 3) {
    sweep *= 342.0 / 53.0;
    const int L = g.levels;
    if (L <= 3) build = 0.6 * GiB;
    else if (L <= 5) build = 18.4 * GiB;
    else build = (18.4 + 3.4 * (L - 5)) * GiB * (L >= 8 ? 1.5 : 1.0);
  }
  if (g.mapped == 2) {
    // general quadrilateral: the build's device TT-SVD holds about four copies of the dense stencil
    // coefficients (36 doubles per node), and the operator's ranks (up to ~100) are about three
    // times the box operator's, which the sweep's environments scale with
    build = 4.0 * 36.0 * 8.0 * std::pow(4.0, g.levels);
    sweep *= 3.0;
  }
  // + 128 MiB: a served 2D request (2^8, cap 16) held 174 MiB where a standalone solve held 57
  return (size_t)(1.25 * std::max(sweep, build) + 128.0 * MiB);
}

}  // namespace tnfem

namespace {

void run_request(tnfem_ctx* ctx, Request* r) {
  tnfem_mpo* A = nullptr;
  tnfem_tt* f = nullptr;
  tnfem_tt* u = nullptr;
  tnfem_memory_stats(ctx, nullptr, nullptr, 1);
  tnfem_status st = tnfem_build_stiffness(ctx, &r->grid, &r->mat, &A);
  if (st == TNFEM_OK) st = tnfem_build_load(ctx, &r->grid, &r->mat, r->loads.data(), (int)r->loads.size(), &f);
  if (st == TNFEM_OK) {
    st = tnfem_solve(ctx, A, f, &r->opts, nullptr, &u, &r->info);
    if (u) {
      int nc = 0;
      r->ranks.assign(64, 0);
      r->modes.assign(63, 0);
      tnfem_status e = tnfem_tt_export(ctx, u, &nc, r->ranks.data(), r->modes.data(), nullptr);
      if (e == TNFEM_OK) {
        size_t tot = 0;
        for (int k = 0; k < nc; ++k) tot += (size_t)r->ranks[k] * r->modes[k] * r->ranks[k + 1];
        r->cores.resize(tot);
        e = tnfem_tt_export(ctx, u, &nc, r->ranks.data(), r->modes.data(), r->cores.data());
      }
      r->ranks.resize(nc + 1);
      r->modes.resize(nc);
      if (e != TNFEM_OK && (st == TNFEM_OK || st == TNFEM_E_NOT_CONVERGED)) st = e;
    }
  }
  if (st != TNFEM_OK) r->err = tnfem_last_error(ctx);
  size_t peak = 0;
  tnfem_memory_stats(ctx, nullptr, &peak, 0);
  r->peak_bytes = peak;
  tnfem_free_tt(u);
  tnfem_free_tt(f);
  tnfem_free_mpo(A);
  r->status = st;
}

void worker_main(tnfem_server* s, int w) {
  tnfem_ctx* ctx = nullptr;
  cudaStream_t stream = nullptr;
  std::string err;
  if (cudaSetDevice(s->device) != cudaSuccess || cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    err = "worker: CUDA stream creation failed";
  } else if (tnfem_create(s->device, stream, stream_alloc, stream_free, stream, &ctx) != TNFEM_OK) {
    err = "worker: context creation failed";
  } else {
    ctx->sm_share = std::max(1, tnfem::coop_sms(ctx) / std::max(1, s->workers));
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->worker_err[w] = err;
  }
  s->ready.fetch_add(1);
  s->cv_done.notify_all();
  if (!ctx) {
    if (stream) cudaStreamDestroy(stream);
    return;
  }
  for (;;) {
    Request* r = nullptr;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_work.wait(lk, [&] {
        if (s->stopping) return true;
        if (s->queue.empty()) return false;
        Request* h = s->queue.front();
        return s->running == 0 || s->admitted_bytes + h->est <= s->budget;
      });
      if (s->queue.empty() && s->stopping) break;
      if (s->stopping && !s->queue.empty()) {
        // drain: requests still queued at stop fail without running
        Request* h = s->queue.front();
        s->queue.pop_front();
        h->status = TNFEM_E_INVALID;
        h->err = "server stopped before the request was admitted";
        h->done = true;
        s->cv_done.notify_all();
        continue;
      }
      r = s->queue.front();
      s->queue.pop_front();
      s->admitted_bytes += r->est;
      ++s->running;
    }
    r->worker = w;
    r->t_start = now_us();
    run_request(ctx, r);
    r->t_end = now_us();
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->admitted_bytes -= r->est;
      --s->running;
      r->done = true;
    }
    s->cv_done.notify_all();
    s->cv_work.notify_all();
  }
  tnfem_destroy(ctx);
  cudaStreamSynchronize(stream);
  cudaStreamDestroy(stream);
}

}  // namespace

using namespace tnfem;

extern "C" {

tnfem_status tnfem_server_budget(const tnfem_server* s, size_t* bytes) {
  if (!s || !bytes) return TNFEM_E_INVALID;
  *bytes = s->budget;
  return TNFEM_OK;
}

tnfem_status tnfem_serve_estimate(const tnfem_grid* grid, const tnfem_solve_opts* opts, size_t* bytes) {
  if (!grid || !opts || !bytes) return TNFEM_E_INVALID;
  *bytes = serve_estimate_bytes(*grid, *opts);
  return TNFEM_OK;
}

tnfem_status tnfem_server_start(int device, int workers, size_t hbm_budget, tnfem_server** out) {
  if (!out) return TNFEM_E_INVALID;
  *out = nullptr;
  if (workers < 1 || workers > 64) return TNFEM_E_INVALID;
  if (cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return TNFEM_E_CUDA;
  }
  auto* s = new (std::nothrow) tnfem_server();
  if (!s) return TNFEM_E_NOMEM;
  s->device = device;
  s->workers = workers;
  s->budget = hbm_budget;
  s->t0 = now_us();
  if (s->budget == 0) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
      cudaGetLastError();
      delete s;
      return TNFEM_E_CUDA;
    }
    s->budget = fr / 10 * 8;  // 80% of what is free now
  }
  // freed device memory stays in the device's pool up to the budget (no release at each sync)
  cudaMemPool_t mp = nullptr;
  if (cudaDeviceGetDefaultMemPool(&mp, device) == cudaSuccess) {
    uint64_t thr = s->budget;
    cudaMemPoolSetAttribute(mp, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  cudaGetLastError();
  s->worker_err.assign(workers, std::string());
  for (int w = 0; w < workers; ++w) s->threads.emplace_back(worker_main, s, w);
  {
    std::unique_lock<std::mutex> lk(s->mu);
    s->cv_done.wait(lk, [&] { return s->ready.load() == workers; });
  }
  for (const auto& e : s->worker_err)
    if (!e.empty()) {
      tnfem_server_stop(s);
      return TNFEM_E_CUDA;
    }
  *out = s;
  return TNFEM_OK;
}

tnfem_status tnfem_submit(tnfem_server* s, const tnfem_grid* grid, const tnfem_material* mat, const tnfem_load* loads,
                          int n_loads, const tnfem_solve_opts* opts, uint64_t* id) {
  if (!s || !grid || !mat || !opts || !id || n_loads < 0 || (n_loads > 0 && !loads)) return TNFEM_E_INVALID;
  if (grid->dim != 2 && grid->dim != 3) return TNFEM_E_INVALID;
  if (grid->levels < 1 || grid->levels > 20) return TNFEM_E_INVALID;
  auto r = std::make_unique<Request>();
  r->grid = *grid;
  r->mat = *mat;
  r->opts = *opts;
  r->loads.assign(loads, loads + n_loads);
  for (auto& ld : r->loads) {
    // a train lives in the caller's context and may be freed before the request runs
    if (ld.kind == TNFEM_LOAD_NODAL_TT) return TNFEM_E_INVALID;
    if (ld.kind == TNFEM_LOAD_FOURIER) {
      if (ld.n_modes < 0 || (ld.n_modes > 0 && (!ld.amp || !ld.wave || !ld.phase))) return TNFEM_E_INVALID;
      r->amp.emplace_back(ld.amp, ld.amp + (size_t)grid->dim * ld.n_modes);
      r->wave.emplace_back(ld.wave, ld.wave + (size_t)grid->dim * ld.n_modes);
      r->phase.emplace_back(ld.phase, ld.phase + ld.n_modes);
      ld.amp = r->amp.back().data();
      ld.wave = r->wave.back().data();
      ld.phase = r->phase.back().data();
    }
  }
  r->est = serve_estimate_bytes(r->grid, r->opts);
  r->t_submit = now_us();
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stopping) return TNFEM_E_INVALID;
  r->id = s->next_id++;
  *id = r->id;
  s->queue.push_back(r.get());
  s->reqs[r->id] = std::move(r);
  s->cv_work.notify_all();
  return TNFEM_OK;
}

tnfem_status tnfem_wait(tnfem_server* s, uint64_t id, int64_t timeout_us, tnfem_request_info* out) {
  if (!s) return TNFEM_E_INVALID;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return TNFEM_E_INVALID;
  Request* r = it->second.get();
  auto pred = [&] { return r->done; };
  if (timeout_us < 0) s->cv_done.wait(lk, pred);
  else if (!s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), pred)) return TNFEM_E_TIMEOUT;
  if (out) {
    memset(out, 0, sizeof(*out));
    out->status = r->status;
    out->info = r->info;
    out->queued_us = r->t_start - r->t_submit;
    out->run_us = r->t_end - r->t_start;
    out->latency_us = r->t_end - r->t_submit;
    out->start_us = r->t_start - s->t0;
    out->end_us = r->t_end - s->t0;
    out->worker = r->worker;
    out->est_bytes = r->est;
    out->peak_bytes = r->peak_bytes;
    out->ncores = (int)r->modes.size();
    for (int k = 0; k < out->ncores && k < 63; ++k) out->modes[k] = r->modes[k];
    for (int k = 0; k < (int)r->ranks.size() && k < 64; ++k) out->ranks[k] = r->ranks[k];
    out->result_doubles = r->cores.size();
    snprintf(out->message, sizeof(out->message), "%s", r->err.c_str());
  }
  return TNFEM_OK;
}

tnfem_status tnfem_result_take(tnfem_server* s, uint64_t id, double* cores) {
  if (!s) return TNFEM_E_INVALID;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end() || !it->second->done) return TNFEM_E_INVALID;
  if (cores && !it->second->cores.empty())
    memcpy(cores, it->second->cores.data(), it->second->cores.size() * sizeof(double));
  s->reqs.erase(it);
  return TNFEM_OK;
}

tnfem_status tnfem_cancel(tnfem_server* s, uint64_t id) {
  if (!s) return TNFEM_E_INVALID;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return TNFEM_E_INVALID;
  Request* r = it->second.get();
  auto q = std::find(s->queue.begin(), s->queue.end(), r);
  if (q == s->queue.end()) return TNFEM_E_INVALID;  // already running or done
  s->queue.erase(q);
  r->status = TNFEM_E_INVALID;
  r->err = "cancelled before admission";
  r->t_start = r->t_end = now_us();
  r->done = true;
  s->cv_done.notify_all();
  return TNFEM_OK;
}

tnfem_status tnfem_server_stats(tnfem_server* s, int* queued, int* running, size_t* admitted_bytes) {
  if (!s) return TNFEM_E_INVALID;
  std::lock_guard<std::mutex> lk(s->mu);
  if (queued) *queued = (int)s->queue.size();
  if (running) *running = s->running;
  if (admitted_bytes) *admitted_bytes = s->admitted_bytes;
  return TNFEM_OK;
}

tnfem_status tnfem_server_stop(tnfem_server* s) {
  if (!s) return TNFEM_E_INVALID;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stopping = true;
  }
  s->cv_work.notify_all();
  for (auto& t : s->threads)
    if (t.joinable()) t.join();
  delete s;
  return TNFEM_OK;
}

}  // extern "C"
