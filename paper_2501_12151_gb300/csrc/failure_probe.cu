// Failure-detection probe: a cooperative kernel whose CTAs pass `rounds` grid barriers of
// grid_sync.cuh with a caller-chosen wait bound, one CTA optionally arriving late at the first.
// With a delay beyond the bound the waiting CTAs give up, flag the error in the barrier word and
// leave; the late CTA sees the flag on arrival and leaves too.  Every wait (the delay and each
// barrier poll) is bounded by the global timer, so the kernel ends in about max(delay, bound)
// and the context stays usable.  This checks, on the device, the timeout path that the solver's
// cooperative kernels (fused CG, SVD, enrichment QR) rely on; it is not a step of the method.
#include "grid_sync.cuh"
#include "internal.h"

namespace tnfem {
namespace {

__global__ void barrier_probe_kernel(GridSync* gs, int late_cta, unsigned long long late_ns,
                                     unsigned long long limit_ns, int rounds, int* failed) {
  unsigned int idx = 0;
  for (int r = 0; r < rounds; ++r) {
    if (r == 0 && (int)blockIdx.x == late_cta && threadIdx.x == 0) {
      const unsigned long long t0 = global_ns();
      while (global_ns() - t0 < late_ns) __nanosleep(10000);
    }
    if (!grid_sync(gs, idx, limit_ns)) {
      if (threadIdx.x == 0) atomicOr(failed, 1);
      return;
    }
  }
}

}  // namespace
}  // namespace tnfem

using namespace tnfem;

extern "C" tnfem_status tnfem_op_barrier_probe(tnfem_ctx* ctx, int ctas, int late_cta, double late_ms,
                                               double limit_ms) {
  if (!ctx) return TNFEM_E_INVALID;
  tnfem_status st = TNFEM_OK;
  try {
    int sms = 0;
    TN_CHECK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
    TN_REQUIRE(ctas >= 1 && ctas <= sms, "ctas must be in [1, number of SMs]");
    TN_REQUIRE(late_cta >= -1 && late_cta < ctas, "late_cta must be -1 (none) or a CTA index");
    TN_REQUIRE(late_ms >= 0.0 && late_ms <= 1000.0, "late_ms must be in [0, 1000]");
    TN_REQUIRE(limit_ms >= 0.01 && limit_ms <= 2000.0, "limit_ms must be in [0.01, 2000]");
    // barrier state and the failure flag in the context's scratch (GridSync first, flag after)
    GridSync* gs = reinterpret_cast<GridSync*>(ctx->scratch + kScratchDoubles - 1024);
    int* failed = reinterpret_cast<int*>(ctx->scratch + kScratchDoubles - 1020);
    TN_CHECK_CUDA(cudaMemsetAsync(gs, 0, 64, ctx->stream));
    unsigned long long late_ns = (unsigned long long)(late_ms * 1e6);
    unsigned long long limit_ns = (unsigned long long)(limit_ms * 1e6);
    int rounds = 3;
    void* args[] = {&gs, &late_cta, &late_ns, &limit_ns, &rounds, &failed};
    TN_CHECK_CUDA(cudaLaunchCooperativeKernel(reinterpret_cast<void*>(barrier_probe_kernel), dim3(ctas), dim3(32),
                                              args, 0, ctx->stream));
    count_launch(ctx);
    int h = 0;
    TN_CHECK_CUDA(cudaMemcpyAsync(&h, failed, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    TN_CHECK_CUDA(cudaStreamSynchronize(ctx->stream));
    if (h) throw Error(TNFEM_E_TIMEOUT, "barrier probe: a grid barrier wait ran out");
    ctx->err.clear();
  } catch (const Error& e) {
    ctx->err = e.what();
    if (e.status == TNFEM_E_CUDA) cudaGetLastError();
    st = e.status;
  }
  return st;
}
