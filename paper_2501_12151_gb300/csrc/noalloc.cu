// Local matvec (step a4) for callers that cannot allocate device memory.
//
// Code that runs where cudaMalloc is off limits -- inside a CUDA stream capture that must not
// grow the memory pool, under an allocator owned by a host framework that forbids foreign
// allocations, or in a real-time loop that may not block on the driver -- still needs the
// contraction.  This variant takes its intermediates from a file-scope device array instead of
// allocating them: the operator copy with swapped mode indices, the two stage products and the
// split-K partials of the three chained GEMMs.
//
// The array is a static __device__ symbol, so every GPU that loads the library holds it (32 MiB)
// until the process exits.  Host code cannot use the symbol's name as a device address; the first
// call on each device (made with that device current) looks the address up with
// cudaGetSymbolAddress and caches it, so that first call should come before any stream capture.
// The cached address belongs to the device's primary context: a cudaDeviceReset between calls
// frees the array with that context, so the device must not be reset while this entry point is
// in use (a reset is not detected).
// Every call shares the array and overwrites it; calls whose work overlaps on the GPU (several
// streams, several host threads) race on it and must be serialised by the caller.  Nothing in the
// array has to start at zero: every element a call reads was written earlier by the same call.
#include <mutex>

#include "internal.h"

namespace {

constexpr long long kScratchDoubles = TNFEM_NOALLOC_SCRATCH_DOUBLES;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_matvec_scratch[kScratchDoubles];

std::mutex g_scratch_mu;
double* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on `device` (current), looked up once per device.
cudaError_t scratch_address(int device, double** out) {
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_matvec_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[device] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[device];
  return cudaSuccess;
}

}  // namespace

extern "C" tnfem_status tnfem_op_local_matvec_noalloc(void* stream, int r0, int n, int r1, int a0, int a1,
                                                      const double* PhiL, const double* A, const double* PhiR,
                                                      const double* x, double* y) {
  if (!PhiL || !A || !PhiR || !x || !y) return TNFEM_E_INVALID;
  if (r0 < 1 || n < 1 || r1 < 1 || a0 < 1 || a1 < 1) return TNFEM_E_INVALID;
  const long long ap = (long long)a0 * n * n * a1;
  const long long t1 = (long long)r0 * a0 * n * r1;
  const long long t2 = (long long)r0 * n * a1 * r1;
  // the three chained GEMMs need the operator copy, both stage products and some split-K room
  if (ap + t1 + t2 + 1024 > kScratchDoubles) return TNFEM_E_INVALID;
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess || device < 0 || device >= kMaxDevices) {
    cudaGetLastError();
    return TNFEM_E_CUDA;
  }
  double* scratch = nullptr;
  if (scratch_address(device, &scratch) != cudaSuccess) {
    cudaGetLastError();
    return TNFEM_E_CUDA;
  }
  // a context on the stack: no allocation, no profiling, launches counted locally
  tnfem_ctx ctx;
  ctx.device = device;
  ctx.stream = static_cast<cudaStream_t>(stream);
  try {
    double* Ap = scratch;
    double* ws = scratch + ((ap + 31) / 32) * 32;
    const size_t ws_elems = (size_t)(kScratchDoubles - (ws - scratch));
    tnfem::transpose4_mid<double>(&ctx, Ap, A, a0, n, n, a1);
    tnfem::local_matvec<double>(&ctx, r0, n, r1, a0, a1, PhiL, Ap, PhiR, x, y, ws, ws_elems);
  } catch (const tnfem::Error& e) {
    cudaGetLastError();
    return e.status;
  } catch (...) {
    return TNFEM_E_INVALID;
  }
  return TNFEM_OK;
}
