// Sampled launch timing.  When enabled, every `prof_every`-th launch of a kernel class is
// bracketed by two CUDA events recorded on the context's stream, together with that launch's
// algorithmic flops and bytes; tnfem_profile_read synchronises, resolves the pending event pairs
// into per-class sums and returns the events to a pool.  Sampling keeps the event overhead small
// on the launch-dense Krylov loop while still timing every kind of launch the sweep makes.
#include "internal.h"

namespace tnfem {

namespace {

cudaEvent_t take_event(tnfem_ctx* ctx) {
  if (!ctx->prof_pool.empty()) {
    cudaEvent_t e = ctx->prof_pool.back();
    ctx->prof_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  TN_CHECK_CUDA(cudaEventCreate(&e));
  return e;
}

}  // namespace

}  // namespace tnfem

struct tnfem_ctx::KTimerPool {
  tnfem::KTimer* dev = nullptr;
  int cap = 0, used = 0;
};

namespace tnfem {

namespace {
__global__ void ktimer_init_kernel(KTimer* t, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    t[i] = KTimer{~0ull, 0ull, 0ull, 0u, 0u};
}
constexpr int kTimerSlots = 4096;
}  // namespace

// Allocate (once) and reset the timer slots; only outside stream capture.
void ktimers_reset(tnfem_ctx* ctx) {
  if (!ctx->ktimers) {
    auto* p = new tnfem_ctx::KTimerPool();
    try {
      p->dev = static_cast<KTimer*>(dalloc(ctx, kTimerSlots * sizeof(KTimer)));
    } catch (...) {
      delete p;
      throw;
    }
    p->cap = kTimerSlots;
    ctx->ktimers = p;
  }
  ktimer_init_kernel<<<(kTimerSlots + 255) / 256, 256, 0, ctx->stream>>>(ctx->ktimers->dev, kTimerSlots);
  ctx->ktimers->used = 0;
  ctx->prof_timers.clear();
}

KTimer* prof_ktimer(tnfem_ctx* ctx, int cls, double flops, double bytes) {
  if (ctx->prof_every <= 0 || !ctx->ktimers || cls < 0 || cls >= TNFEM_PROF_CLASSES) return nullptr;
  // the sampling decision is taken when the launch is issued (or captured: then every replay of
  // the captured launch is timed); outside graphs the sampled launch is timed on the device too,
  // so host launch gaps never enter its duration
  if (ctx->prof_seen[cls] % ctx->prof_every != 0) return nullptr;
  tnfem_ctx::KTimerPool* p = ctx->ktimers;
  if (p->used >= p->cap) {
    if (ctx->capturing) return nullptr;
    prof_resolve(ctx);  // read and recycle the slots (outside capture only)
  }
  const int slot = p->used++;
  ctx->prof_timers.push_back(tnfem_ctx::ProfTimer{slot, cls, flops, bytes});
  return p->dev + slot;
}

ProfScope::ProfScope(tnfem_ctx* c, int cls, double flops, double bytes, bool device_timed) : ctx(c) {
  if (ctx->prof_every <= 0 || cls < 0 || cls >= TNFEM_PROF_CLASSES) return;
  if (device_timed) {  // the kernel times itself (KTimer); only count the launch
    ctx->prof_seen[cls]++;
    return;
  }
  // launches captured into a graph are credited per replay by the graph and timed on the device
  // (prof_ktimer); not bracketed by events here
  if (ctx->capturing) {
    ctx->prof_seen[cls]++;
    return;
  }
  long long seen = ctx->prof_seen[cls]++;
  if (seen % ctx->prof_every != 0) return;
  tnfem_ctx::ProfEv ev{take_event(ctx), take_event(ctx), cls, flops, bytes};
  TN_CHECK_CUDA(cudaEventRecord(ev.a, ctx->stream));
  ctx->prof_pending.push_back(ev);
  idx = (int)ctx->prof_pending.size() - 1;
}

void prof_set_work(tnfem_ctx* ctx, int idx, double flops, double bytes) {
  if (idx < 0 || idx >= (int)ctx->prof_pending.size()) return;
  ctx->prof_pending[idx].flops = flops;
  ctx->prof_pending[idx].bytes = bytes;
}

ProfScope::~ProfScope() {
  if (idx < 0) return;
  // a failed record only loses this sample; destructors must not throw
  if (cudaEventRecord(ctx->prof_pending[idx].b, ctx->stream) != cudaSuccess) {
    cudaGetLastError();
    ctx->prof_pending[idx].cls = -1;
  }
}

void prof_resolve(tnfem_ctx* ctx) {
  if (!ctx->prof_timers.empty()) {
    tnfem_ctx::KTimerPool* p = ctx->ktimers;
    std::vector<KTimer> h(p->used);
    TN_CHECK_CUDA(cudaStreamSynchronize(ctx->stream));
    TN_CHECK_CUDA(cudaMemcpy(h.data(), p->dev, p->used * sizeof(KTimer), cudaMemcpyDeviceToHost));
    for (const auto& t : ctx->prof_timers) {
      const KTimer& k = h[t.slot];
      ctx->prof_sampled[t.cls] += k.count;
      ctx->prof_ms[t.cls] += k.total_ns * 1e-6;
      ctx->prof_flops[t.cls] += t.flops * k.count;
      ctx->prof_bytes[t.cls] += t.bytes * k.count;
    }
    ktimers_reset(ctx);
  }
  if (ctx->prof_pending.empty()) return;
  TN_CHECK_CUDA(cudaStreamSynchronize(ctx->stream));
  for (auto& ev : ctx->prof_pending) {
    if (ev.cls >= 0) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, ev.a, ev.b) == cudaSuccess) {
        ctx->prof_sampled[ev.cls] += 1;
        ctx->prof_ms[ev.cls] += ms;
        ctx->prof_flops[ev.cls] += ev.flops;
        ctx->prof_bytes[ev.cls] += ev.bytes;
      } else {
        cudaGetLastError();
      }
    }
    ctx->prof_pool.push_back(ev.a);
    ctx->prof_pool.push_back(ev.b);
  }
  ctx->prof_pending.clear();
}

void prof_release(tnfem_ctx* ctx) {
  if (ctx->ktimers) {
    dfree(ctx, ctx->ktimers->dev);
    delete ctx->ktimers;
    ctx->ktimers = nullptr;
  }
  ctx->prof_timers.clear();
  for (auto& ev : ctx->prof_pending) {
    cudaEventDestroy(ev.a);
    cudaEventDestroy(ev.b);
  }
  ctx->prof_pending.clear();
  for (cudaEvent_t e : ctx->prof_pool) cudaEventDestroy(e);
  ctx->prof_pool.clear();
}

}  // namespace tnfem

using namespace tnfem;

extern "C" {

tnfem_status tnfem_profile_start(tnfem_ctx* ctx, int every) {
  if (!ctx) return TNFEM_E_INVALID;
  try {
    prof_resolve(ctx);
  } catch (const Error& e) {
    ctx->err = e.what();
    return e.status;
  }
  ctx->prof_every = every > 0 ? every : 0;
  if (ctx->prof_every > 0) {
    try {
      ktimers_reset(ctx);
    } catch (const Error& e) {
      ctx->err = e.what();
      return e.status;
    }
  }
  for (int c = 0; c < TNFEM_PROF_CLASSES; ++c) {
    ctx->prof_seen[c] = ctx->prof_sampled[c] = 0;
    ctx->prof_ms[c] = ctx->prof_flops[c] = ctx->prof_bytes[c] = 0.0;
  }
  return TNFEM_OK;
}

tnfem_status tnfem_profile_read(tnfem_ctx* ctx, int cls, long long* launches, long long* sampled, double* ms,
                                double* flops, double* bytes) {
  if (!ctx || cls < 0 || cls >= TNFEM_PROF_CLASSES) return TNFEM_E_INVALID;
  try {
    prof_resolve(ctx);
  } catch (const Error& e) {
    ctx->err = e.what();
    return e.status;
  }
  if (launches) *launches = ctx->prof_seen[cls];
  if (sampled) *sampled = ctx->prof_sampled[cls];
  if (ms) *ms = ctx->prof_ms[cls];
  if (flops) *flops = ctx->prof_flops[cls];
  if (bytes) *bytes = ctx->prof_bytes[cls];
  return TNFEM_OK;
}

}  // extern "C"

// ---- arithmetic peaks --------------------------------------------------------------------------
// Register-resident FMA chains (8 independent chains per thread, no memory traffic) over a grid of
// 8 CTAs of 256 threads per SM: the CUDA-core FMA rate the contraction kernels can approach.
namespace tnfem {
namespace {

template <typename T>
__global__ void __launch_bounds__(256) fma_peak_kernel(T* out, int iters, T seed) {
  T a[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) a[c] = seed + (T)(threadIdx.x + c);
  const T b = (T)0.999999, d = (T)1e-7;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < 8; ++c) a[c] = fma(a[c], b, d);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < 8; ++c) s += a[c];
  if (s == (T)-1) out[0] = s;  // never true; keeps the chains live
}

}  // namespace
}  // namespace tnfem

extern "C" tnfem_status tnfem_measure_fma_peak(tnfem_ctx* ctx, int precision, double* tflops) {
  if (!ctx || !tflops || (precision != 0 && precision != 1)) return TNFEM_E_INVALID;
  try {
    int sms = 0;
    TN_CHECK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
    const int blocks = sms * 8, threads = 256;
    const int iters = precision == 0 ? 2048 : 65536;
    cudaEvent_t e0, e1;
    TN_CHECK_CUDA(cudaEventCreate(&e0));
    TN_CHECK_CUDA(cudaEventCreate(&e1));
    float ms = 0.f;
    for (int rep = 0; rep < 2; ++rep) {  // the first launch warms up clocks and code
      TN_CHECK_CUDA(cudaEventRecord(e0, ctx->stream));
      if (precision == 0)
        fma_peak_kernel<double><<<blocks, threads, 0, ctx->stream>>>(reinterpret_cast<double*>(ctx->scratch), iters,
                                                                      1.0);
      else
        fma_peak_kernel<float><<<blocks, threads, 0, ctx->stream>>>(reinterpret_cast<float*>(ctx->scratch), iters,
                                                                     1.0f);
      count_launch(ctx);
      TN_CHECK_CUDA(cudaEventRecord(e1, ctx->stream));
      TN_CHECK_CUDA(cudaEventSynchronize(e1));
      TN_CHECK_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const double flops = 2.0 * 8.0 * iters * (double)blocks * threads;
    *tflops = ms > 0 ? flops / (ms * 1e-3) * 1e-12 : 0.0;
  } catch (const Error& e) {
    ctx->err = e.what();
    cudaGetLastError();
    return e.status;
  }
  return TNFEM_OK;
}
