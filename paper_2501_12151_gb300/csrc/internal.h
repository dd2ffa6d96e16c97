// Internal declarations of the tnfem library: context, device buffers, tensor trains and the
// kernel launchers shared by the host drivers.  Not part of the public ABI (include/tnfem.h).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <stdexcept>
#include <string>
#include <unordered_map>
#include <vector>

#include "tnfem.h"

namespace tnfem {

// ---- errors ----------------------------------------------------------------------------------

struct Error : public std::runtime_error {
  tnfem_status status;
  Error(tnfem_status s, const std::string& m) : std::runtime_error(m), status(s) {}
};

#define TN_CHECK_CUDA(call)                                                                   \
  do {                                                                                        \
    cudaError_t _e = (call);                                                                  \
    if (_e != cudaSuccess)                                                                    \
      throw ::tnfem::Error(TNFEM_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(_e)); \
  } while (0)

#define TN_REQUIRE(cond, msg)                                             \
  do {                                                                    \
    if (!(cond)) throw ::tnfem::Error(TNFEM_E_INVALID, std::string(msg)); \
  } while (0)

}  // namespace tnfem

// ---- context ---------------------------------------------------------------------------------

struct tnfem_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  tnfem_alloc_fn alloc_fn = nullptr;
  tnfem_free_fn free_fn = nullptr;
  void* user = nullptr;
  std::string err;
  long long launches = 0;
  // per-context scratch for reductions and small device scalars
  double* scratch = nullptr;  // kScratchDoubles doubles
  // pinned host staging for small device->host reads
  double* host_pinned = nullptr;
  // sampled launch timing (see tnfem_profile_start): events around every `prof_every`-th launch
  // of each kernel class, resolved on tnfem_profile_read
  struct ProfEv {
    cudaEvent_t a, b;
    int cls;
    double flops, bytes;
  };
  bool capturing = false;  // launches are being captured into a graph
  bool tensor_cores = false;  // binary32 GEMMs on tcgen05 (three-term TF32) instead of CUDA cores
  bool df64 = false;          // large binary64 GEMMs in double-binary32 arithmetic (gemm_df_kernel)
  bool own_stream = false; // `stream` was created by the context (caller passed NULL)
  int prof_every = 0;
  long long prof_seen[TNFEM_PROF_CLASSES] = {};
  long long prof_sampled[TNFEM_PROF_CLASSES] = {};
  double prof_ms[TNFEM_PROF_CLASSES] = {};
  double prof_flops[TNFEM_PROF_CLASSES] = {};
  double prof_bytes[TNFEM_PROF_CLASSES] = {};
  std::vector<ProfEv> prof_pending;
  std::vector<cudaEvent_t> prof_pool;
  // device-side timers of sampled launches captured into graphs (see tnfem::KTimer)
  struct ProfTimer {
    int slot;
    int cls;
    double flops, bytes;
  };
  struct KTimerPool;
  KTimerPool* ktimers = nullptr;
  std::vector<ProfTimer> prof_timers;
  // device-memory accounting: bytes held through dalloc, their high-water mark, and the budget
  // (0: none) above which an allocation fails with TNFEM_E_BUDGET
  size_t mem_budget = 0, mem_in_use = 0, mem_peak = 0;
  std::unordered_map<void*, size_t> mem_sizes;
  // SMs this context's cooperative (grid-barrier) kernels may fill (0: all).  Contexts whose work
  // overlaps on one GPU (the serving loop's workers) each take a share, so that all their
  // cooperative grids can be resident at once whatever order the hardware schedules them in.
  int sm_share = 0;
};

namespace tnfem {

constexpr int kScratchDoubles = 1 << 16;
// binary64 GEMMs with at least this many multiply-adds run in double-binary32 when ctx->df64
// (tnfem_op_gemm_f64 engine 1; the solve does not use it, see the engine's description)
constexpr double kDfMinMnk = 1 << 20;
// the mixed solve paths take the double-binary32 route for tolerances from this value up
constexpr double kDfTolMin = 1e-7;
// device flag (in the context's scratch) set by a double-binary32 GEMM whose output was not finite
inline int* df_overflow_flag(tnfem_ctx* ctx) { return reinterpret_cast<int*>(ctx->scratch + kScratchDoubles - 520); }
constexpr int kReduceBlocks = 304;  // 2 x 152 SMs: partial sums of one reduction

// SM count of the context's device, capped by ctx->sm_share (grid sizing of cooperative kernels)
int coop_sms(tnfem_ctx* ctx);
void* dalloc(tnfem_ctx* ctx, size_t bytes);
void dfree(tnfem_ctx* ctx, void* p);
void sync(tnfem_ctx* ctx);
inline void count_launch(tnfem_ctx* ctx, int n = 1) { ctx->launches += n; }

// Brackets one kernel launch of class `cls` with a pair of events on the context's stream when
// profiling samples it; `flops` / `bytes` are the launch's algorithmic work and traffic.
struct ProfScope {
  tnfem_ctx* ctx;
  int idx = -1;
  ProfScope(tnfem_ctx* c, int cls, double flops, double bytes, bool device_timed = false);
  ~ProfScope();
};
// Set the algorithmic work of the sampled launch `idx` (ProfScope::idx; ignored when < 0), for
// launches whose work is known only after they ran.
void prof_set_work(tnfem_ctx* ctx, int idx, double flops, double bytes);

// Device-side duration of one kernel launch, accumulated over every execution of that launch
// (including each replay of a graph that captured it): the first CTA to start records the
// global timer, every CTA records its end, and the last CTA to finish adds end - start to
// `total_ns` and increments `count`.  Used for launches inside CUDA graphs, where events cannot
// bracket single kernels.
struct KTimer {
  unsigned long long start, end, total_ns;
  unsigned int arrived, count;
};
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void ktimer_begin(KTimer* t) {
  if (t && threadIdx.x == 0) atomicMin(&t->start, global_ns());
}
// Call once per CTA after its last store (all threads of the CTA reach it).
__device__ __forceinline__ void ktimer_end(KTimer* t) {
  if (!t) return;
  __syncthreads();
  if (threadIdx.x == 0) {
    atomicMax(&t->end, global_ns());
    __threadfence();
    const unsigned int nblk = gridDim.x * gridDim.y * gridDim.z;
    if (atomicAdd(&t->arrived, 1u) == nblk - 1) {
      __threadfence();
      const unsigned long long s = atomicAdd(&t->start, 0ull), e = atomicAdd(&t->end, 0ull);
      t->total_ns += e - s;
      t->count += 1;
      t->start = ~0ull;
      t->end = 0ull;
      t->arrived = 0u;
    }
  }
}
// A sampled launch that is being captured into a graph gets a timer slot (nullptr otherwise).
KTimer* prof_ktimer(tnfem_ctx* ctx, int cls, double flops, double bytes);
void prof_resolve(tnfem_ctx* ctx);
void prof_release(tnfem_ctx* ctx);
void check_launch(tnfem_ctx* ctx, const char* what);

// RAII device array
template <typename T>
struct DArr {
  tnfem_ctx* ctx = nullptr;
  T* p = nullptr;
  size_t n = 0;
  DArr() = default;
  DArr(tnfem_ctx* c, size_t count) : ctx(c), n(count) {
    p = count ? static_cast<T*>(dalloc(c, count * sizeof(T))) : nullptr;
  }
  DArr(const DArr&) = delete;
  DArr& operator=(const DArr&) = delete;
  DArr(DArr&& o) noexcept : ctx(o.ctx), p(o.p), n(o.n) { o.p = nullptr; o.n = 0; }
  DArr& operator=(DArr&& o) noexcept {
    if (this != &o) { release(); ctx = o.ctx; p = o.p; n = o.n; o.p = nullptr; o.n = 0; }
    return *this;
  }
  ~DArr() { release(); }
  void release() { if (p) dfree(ctx, p); p = nullptr; n = 0; }
  void ensure(tnfem_ctx* c, size_t count) {
    if (count > n) { release(); ctx = c; p = static_cast<T*>(dalloc(c, count * sizeof(T))); n = count; }
  }
};

// ---- kernel launchers (kernels_blas.cu) ------------------------------------------------------

// Strided batched GEMM: C(m,n) = alpha * sum_k A(m,k) B(k,n) + beta * C(m,n) for each batch b,
// A(m,k) = A[b*sAb + m*sAm + k*sAk], B(k,n) = B[b*sBb + k*sBk + n*sBn],
// C(m,n) = C[b*sCb + m*sCm + n*sCn].  `work` (nullable) enables split-K through a deterministic
// two-pass reduction; it must hold splits*batch*M*N elements.
struct GemmDesc {
  int M, N, K, batch;
  long long sAm, sAk, sAb, sBk, sBn, sBb, sCm, sCn, sCb;
};
template <typename T>
void gemm(tnfem_ctx* ctx, const GemmDesc& g, T alpha, const T* A, const T* B, T beta, T* C,
          T* work = nullptr, size_t work_elems = 0, const int* skip = nullptr);

// C = alpha * sum over splits of work + beta * C (split-K epilogue, work [split][batch][M][N])
template <typename T>
void splitk_reduce(tnfem_ctx* ctx, const GemmDesc& g, T alpha, T beta, T* C, const T* work, int splits,
                   const int* skip);
template <typename T> void fill(tnfem_ctx* ctx, T* x, T v, size_t n);
template <typename T> void copy(tnfem_ctx* ctx, T* dst, const T* src, size_t n);
template <typename T> void axpby(tnfem_ctx* ctx, T* y, T a, const T* x, T b, size_t n);  // y = a x + b y
template <typename T> void scale(tnfem_ctx* ctx, T* x, T a, size_t n);
void convert_d2f(tnfem_ctx* ctx, float* dst, const double* src, size_t n);
void convert_f2d(tnfem_ctx* ctx, double* dst, const float* src, size_t n);
// Partial sums of x.y into part[0..kReduceBlocks) (deterministic order).
template <typename T> void dot_partials(tnfem_ctx* ctx, const T* x, const T* y, size_t n, double* part);
// Host-side dot / norm (synchronising).
template <typename T> double dot(tnfem_ctx* ctx, const T* x, const T* y, size_t n);
template <typename T> double nrm2(tnfem_ctx* ctx, const T* x, size_t n);
// out[c][b][a] = in[a][b][c] for a [A][B][C] array (used to flip tensor-train cores)
template <typename T> void transpose3(tnfem_ctx* ctx, T* out, const T* in, int A, int B, int C);
// out[d][b][c][a] = in[a][b][c][d] (flip operator cores)
template <typename T> void transpose4_outer(tnfem_ctx* ctx, T* out, const T* in, int A, int B, int C, int D);
// out[a][j][i][d] = in[a][i][j][d] (swap the two middle indices)
template <typename T> void transpose4_mid(tnfem_ctx* ctx, T* out, const T* in, int A, int B, int C, int D);
// 2D transpose: out[n][m] = in[m][n]
template <typename T> void transpose2(tnfem_ctx* ctx, T* out, const T* in, int m, int n);

// ---- dense factorizations (kernels_la.cu) ----------------------------------------------------

// Reduced Householder QR of row-major m x n matrix A (overwritten as workspace):
// Q [m][k], R [k][n], k = min(m, n).
template <typename T>
void qr(tnfem_ctx* ctx, int m, int n, T* A, T* Q, T* R, T* work);
size_t qr_work_elems(int m, int n);
// QR of the m x (rk + w) row-major A = [U | W] whose first rk columns are orthonormal (m >= rk + w):
// Q [m][rk + w], R [rk + w][rk + w] as qr() gives them, up to the basis of the W part (block
// Gram-Schmidt against U, with a Householder fallback when W lies inside span(U)); A is
// overwritten.  work holds qr_ext_work_elems(m, rk, w) elements; with less, or w < 1, or rk < 1,
// this is qr().  Synchronises the stream.
size_t qr_ext_work_elems(int m, int rk, int w);
template <typename T>
void qr_ext(tnfem_ctx* ctx, int m, int rk, int w, T* A, T* Q, T* R, T* work, size_t work_elems);
// Thin SVD by one-sided Jacobi of row-major m x n matrix (m >= n), A overwritten:
// U [m][n] (unit columns, sign fixed), S [n] descending, Vt [n][n].
template <typename T>
void svd(tnfem_ctx* ctx, int m, int n, T* A, T* U, T* S, T* Vt, T* work);
size_t svd_work_elems(int m, int n);

}  // namespace tnfem

// ---- tensor trains ---------------------------------------------------------------------------

struct tnfem_tt {
  tnfem_ctx* ctx = nullptr;
  int d = 0;
  std::vector<int> n;       // modes, size d
  std::vector<int> r;       // ranks, size d+1
  std::vector<double*> core;
  std::vector<size_t> cap;  // capacity (elements) of each core
  ~tnfem_tt();
};

struct tnfem_mpo {
  tnfem_ctx* ctx = nullptr;
  int d = 0;
  std::vector<int> n;       // modes
  std::vector<int> a;       // ranks, size d+1
  std::vector<double*> core;        // [a0][n][n][a1]
  // Derived copies used by the sweep (built by mpo_prepare): cores with the two mode indices
  // swapped, [a0][j][i][a1], in the given and in the flipped orientation (cores reversed,
  // [a1][j][i][a0]), in binary64 and binary32.
  std::vector<double*> p64[2];
  std::vector<float*> p32[2];
  bool prepared = false;
  ~tnfem_mpo();
};

namespace tnfem {

tnfem_tt* tt_new(tnfem_ctx* ctx, const std::vector<int>& n, const std::vector<int>& r,
                 const std::vector<size_t>* cap = nullptr);
void tt_set_core(tnfem_tt* x, int k, int r0, int r1);  // change rank, keep buffer if it fits
tnfem_tt* tt_clone(const tnfem_tt* x);
tnfem_mpo* mpo_new(tnfem_ctx* ctx, const std::vector<int>& n, const std::vector<int>& a);
void mpo_prepare(tnfem_mpo* A);
// random Gaussian core entries from a counter-based generator (splitmix64 + Box-Muller)
void fill_gaussian(tnfem_ctx* ctx, double* x, size_t n, uint64_t seed, uint64_t stream_id);
// dst[(off0+a)][i][(off1+b)] = s * src[a][i][b] inside a [R0][n][R1] array
void block_copy3(tnfem_ctx* ctx, double* dst, int R0, int n, int R1, int off0, int off1,
                 const double* src, int r0, int r1, double s);
// dst[i][c] = src[i*ld + c] * s[c], c < ncols (s is a device array)
void scale_cols(tnfem_ctx* ctx, double* dst, const double* src, int rows, int ld, int ncols,
                const double* s);
int truncation_rank(const std::vector<double>& S, double delta, int rmax);
size_t tt_bytes(const tnfem_tt* x);
size_t mpo_bytes(const tnfem_mpo* A);

// TT algebra on the device (tt_ops.cu)
tnfem_tt* tt_round(tnfem_ctx* ctx, const tnfem_tt* x, double eps, int rmax);
// TT-SVD of a dense host array (row-major, modes[0] slowest) on the device, left to right, each
// unfolding through the QR of its transpose and the SVD of the small factor, truncated to
// eps / sqrt(d-1) ||array|| per bond; unfoldings of at most 64 rows keep an identity core
tnfem_tt* tt_from_full(tnfem_ctx* ctx, const double* host, const std::vector<int>& modes, double eps);
tnfem_tt* tt_axpy(tnfem_ctx* ctx, const tnfem_tt* x, double beta, const tnfem_tt* y);
tnfem_tt* mpo_apply(tnfem_ctx* ctx, const tnfem_mpo* A, const tnfem_tt* x);
double tt_dot(tnfem_ctx* ctx, const tnfem_tt* x, const tnfem_tt* y);
double tt_norm(tnfem_ctx* ctx, const tnfem_tt* x);
double energy_norm(tnfem_ctx* ctx, const tnfem_mpo* A, const tnfem_tt* u, const tnfem_tt* v);
// a9's global relative residual ||f - A u|| / ||f|| from dense expansions (tt_ops.cu); for grids
// with at most 2^22 unknowns whose expansion times the largest rank fits 2^28 doubles
size_t dense_elems(const tnfem_tt* x);
double residual_norm_dense(tnfem_ctx* ctx, const tnfem_mpo* A, const tnfem_tt* f, const tnfem_tt* u);
// MPO rounding (as a train with mode n^2)
tnfem_mpo* mpo_round(tnfem_ctx* ctx, const tnfem_mpo* A, double eps, int rmax);

// Contractions shared by the sweep and the entry points (contract.cu)
template <typename T>
struct Workspace;
// y = local matvec; T1/T2 workspaces sized by local_ws_elems
size_t local_ws_elems(int r0, int n, int r1, int a0, int a1);
template <typename T>
void local_matvec(tnfem_ctx* ctx, int r0, int n, int r1, int a0, int a1, const T* PhiL,
                  const T* A, const T* PhiR, const T* x, T* y, T* ws, size_t ws_elems,
                  const int* skip = nullptr);
// Left environment update, operator: out[b',g,b] = sum y[a',i,b'] Phi[a',beta,a] A[beta,i,j,g] x[a,j,b]
template <typename T>
void env_left(tnfem_ctx* ctx, int ry0, int ry1, int rx0, int rx1, int n, int a0, int a1,
              const T* Phi, const T* y, const T* A, const T* x, T* out, T* ws, size_t ws_elems);
// Left environment update, vector: out[b',d] = sum y[a',i,b'] Psi[a',c] f[c,i,d]
template <typename T>
void env_left_vec(tnfem_ctx* ctx, int ry0, int ry1, int rf0, int rf1, int n, const T* Psi,
                  const T* y, const T* f, T* out, T* ws, size_t ws_elems);
// Local right-hand side g = alpha * (sum PsiL[a',c] f[c,i,d] PsiR[b',d]) + beta * g
template <typename T>
void local_rhs(tnfem_ctx* ctx, int r0, int n, int r1, int rf0, int rf1, const T* PsiL,
               const T* f, const T* PsiR, T* g, T* ws, size_t ws_elems, T alpha = T(1),
               T beta = T(0));
// Rectangular local operator application with separate bra (ry) and ket (rx) ranks:
// y[a',i,b'] = alpha * sum PhiL[a',beta,a] A[beta,i,j,g] PhiR[b',g,b] x[a,j,b] + beta_ * y
template <typename T>
void local_apply(tnfem_ctx* ctx, int ry0, int ry1, int rx0, int rx1, int n, int a0, int a1,
                 const T* PhiL, const T* Ap, const T* PhiR, const T* x, T* y, T alpha, T beta,
                 T* ws, size_t ws_elems, const int* skip = nullptr);

}  // namespace tnfem
