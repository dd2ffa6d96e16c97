// The AMEn sweep (alternating minimal energy; the solver of Section 5.4 / Algorithm 2) on the
// device.  One class drives one solve of A x = b, where the right-hand side is a sum of
// "sources" b = sum_s c_s S_s, each S_s either a tensor train v or an operator-times-train A u.
// The binary64 solve has the single source f; the mixed-precision refinement solves the
// correction equation A e = f - A u with sources (f, +1) and (A u, -1), whose projections are
// formed in binary64 while the sweep itself (environments, local matvecs, conjugate
// gradients, QR, SVD) runs in precision T.
//
// Per core k of a sweep (current orientation):
//   1. g = projection of b onto the current interfaces of x            (sources, binary64)
//   2. local residual ||g - B x_k|| / ||g||, B = PhiL A_k PhiR       (three-stage contraction)
//   3. B y = g by conjugate gradients, B symmetric positive definite (device-side control flow)
//   4. SVD of y as (r0 n) x r1, truncation tol/sqrt(d) (Frobenius, relative) and rank cap
//   5. enrichment: residual projected on (x left, z right) appended to the kept singular
//      vectors, re-orthogonalised by QR; z core <- leading left singular vectors of the residual
//      projected on z's interfaces (kickrank of them)
//   6. the non-orthogonal factor moves into core k+1; left environments of bond k+1 are updated
// A backward sweep is the same forward sweep over the flipped train (cores reversed and
// transposed); environments are stored per bond and side and are reused across the flip.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <memory>

#include <nvtx3/nvToolsExt.h>

#include "amen.h"
#include "cg_fused.h"
#include "internal.h"
#include "precond.h"
#include "tc_gemm.h"
#include "tc_matvec.h"

namespace tnfem {

namespace {

constexpr int RT = 256;

// Sum of np per-block partials, computed by warp 0 only and broadcast through shared memory:
// binary64 arithmetic is scarce on this part, so the block's other warps do none of it.
__device__ __forceinline__ double block_reduce_partials(const double* __restrict__ part, int np, double* sh) {
  if (threadIdx.x < 32) {
    double s = 0.0;
    for (int i = threadIdx.x; i < np; i += 32) s += part[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) sh[0] = s;
  }
  __syncthreads();
  const double t = sh[0];
  __syncthreads();
  return t;
}

__device__ __forceinline__ void block_partial_out(double s, double* sh, double* out) {
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += sh[i];
    out[blockIdx.x] = t;
  }
}

template <typename T>
__global__ void __launch_bounds__(RT) cg_init_kernel(const T* __restrict__ g, const T* __restrict__ Bx,
                                                     T* __restrict__ r, T* __restrict__ p, size_t N,
                                                     double* __restrict__ part) {
  __shared__ double sh[32];
  double s = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
    T v = g[i] - Bx[i];
    r[i] = v;
    p[i] = v;
    s += (double)v * (double)v;
  }
  block_partial_out(s, sh, part);
}

template <typename T>
__global__ void __launch_bounds__(RT) cg_dot_kernel(const T* __restrict__ x, const T* __restrict__ y, size_t N,
                                                    double* __restrict__ part, const int* __restrict__ ctl) {
  if (ctl[0]) return;
  __shared__ double sh[32];
  double s = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x)
    s += (double)x[i] * (double)y[i];
  block_partial_out(s, sh, part);
}

// Stop test on r.r (partials part_rr), then alpha = r.z / pAp; x += alpha p; r -= alpha Ap;
// partial sums of the new r.r.  Without a preconditioner z = r and part_rz aliases part_rr.
// The three sums and alpha are formed by warp 0 and broadcast.
// ctl[0]: 0 running, 1 converged, 2 breakdown; ctl[1]: iterations done
template <typename T>
__global__ void __launch_bounds__(RT) cg_update1_kernel(T* __restrict__ x, T* __restrict__ r, const T* __restrict__ p,
                                                        const T* __restrict__ Ap, size_t N,
                                                        const double* __restrict__ part_rr, int np_rr,
                                                        const double* __restrict__ part_rz, int np_rz,
                                                        const double* __restrict__ part_pAp, int np_pap,
                                                        double* __restrict__ part_rr_new, int* __restrict__ ctl,
                                                        double stop2) {
  if (ctl[0]) return;
  __shared__ double sh[32];
  __shared__ double s_alpha;
  __shared__ int s_state;
  if (threadIdx.x < 32) {
    double rr = 0.0, rz = 0.0, pap = 0.0;
    for (int i = threadIdx.x; i < np_rr; i += 32) rr += part_rr[i];
    for (int i = threadIdx.x; i < np_rz; i += 32) rz += part_rz[i];
    for (int i = threadIdx.x; i < np_pap; i += 32) pap += part_pAp[i];
    for (int o = 16; o > 0; o >>= 1) {
      rr += __shfl_xor_sync(0xffffffffu, rr, o);
      rz += __shfl_xor_sync(0xffffffffu, rz, o);
      pap += __shfl_xor_sync(0xffffffffu, pap, o);
    }
    if (threadIdx.x == 0) {
      int state = 0;
      if (rr <= stop2) state = 1;
      else if (!(pap > 0.0) || !isfinite(pap) || !(rz > 0.0)) state = 2;
      s_state = state;
      s_alpha = state == 0 ? rz / pap : 0.0;
    }
  }
  __syncthreads();
  if (s_state) {
    if (blockIdx.x == 0 && threadIdx.x == 0) ctl[0] = s_state;
    return;
  }
  const T alpha = (T)s_alpha;
  double s = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
    x[i] += alpha * p[i];
    T v = r[i] - alpha * Ap[i];
    r[i] = v;
    s += (double)v * (double)v;
  }
  block_partial_out(s, sh, part_rr_new);
  if (blockIdx.x == 0 && threadIdx.x == 0) ctl[1] += 1;
}

// p = z + beta p with beta = (r.z)_new / (r.z)_old
template <typename T>
__global__ void __launch_bounds__(RT) cg_update2_kernel(T* __restrict__ p, const T* __restrict__ z, size_t N,
                                                        const double* __restrict__ part_rz_new,
                                                        const double* __restrict__ part_rz, int np_rz,
                                                        const int* __restrict__ ctl) {
  if (ctl[0]) return;
  __shared__ double s_beta;
  if (threadIdx.x < 32) {
    double rn = 0.0, ro = 0.0;
    for (int i = threadIdx.x; i < np_rz; i += 32) {
      rn += part_rz_new[i];
      ro += part_rz[i];
    }
    for (int o = 16; o > 0; o >>= 1) {
      rn += __shfl_xor_sync(0xffffffffu, rn, o);
      ro += __shfl_xor_sync(0xffffffffu, ro, o);
    }
    if (threadIdx.x == 0) s_beta = rn / ro;
  }
  __syncthreads();
  const T beta = (T)s_beta;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x)
    p[i] = z[i] + beta * p[i];
}

// d = a - b (precision T), partial sums of d.d
template <typename T>
__global__ void __launch_bounds__(RT) diff_kernel(T* __restrict__ d, const T* __restrict__ a, const T* __restrict__ b,
                                                  size_t N, double* __restrict__ part) {
  __shared__ double sh[32];
  double s = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
    T v = a[i] - b[i];
    d[i] = v;
    s += (double)v * (double)v;
  }
  block_partial_out(s, sh, part);
}

// out[i][c] = src[i*ld + c], c < ncols
template <typename T>
__global__ void pack_cols_kernel(T* __restrict__ out, const T* __restrict__ src, int rows, int ld, int ncols,
                                 int out_ld, int out_off) {
  long long total = (long long)rows * ncols;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    int i = (int)(t / ncols), c = (int)(t % ncols);
    out[(long long)i * out_ld + out_off + c] = src[(long long)i * ld + c];
  }
}

// M[i][:] *= s[i] for i < rows (row scaling by singular values)
template <typename T>
__global__ void scale_rows_kernel(T* __restrict__ M, const T* __restrict__ s, int rows, int cols) {
  long long total = (long long)rows * cols;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x)
    M[t] *= s[t / cols];
}

__global__ void sum_partials_kernel(const double* __restrict__ part, double* __restrict__ out) {
  __shared__ double sh[32];
  double s = block_reduce_partials(part, kReduceBlocks, sh);
  if (threadIdx.x == 0) *out = s;
}

// dst = (float)(src * s)
__global__ void scale_to_float_kernel(float* __restrict__ dst, const double* __restrict__ src, double s, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    dst[i] = (float)(src[i] * s);
}

// y += s * (double)d
__global__ void add_scaled_float_kernel(double* __restrict__ y, const float* __restrict__ d, double s, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] += s * (double)d[i];
}

inline int nblk(long long n) { return (int)std::max<long long>(1, std::min<long long>((n + RT - 1) / RT, kReduceBlocks)); }

template <typename T> struct Prec;
template <> struct Prec<double> {
  static const double* A(const tnfem_mpo* M, int o, int k) { return M->p64[o][k]; }
};
template <> struct Prec<float> {
  static const float* A(const tnfem_mpo* M, int o, int k) { return M->p32[o][k]; }
};

template <typename S, typename D>
void convert_any(tnfem_ctx* ctx, D* dst, const S* src, size_t n) {
  if constexpr (std::is_same<S, D>::value) copy<D>(ctx, dst, src, n);
  else if constexpr (std::is_same<S, double>::value) convert_d2f(ctx, dst, src, n);
  else convert_f2d(ctx, dst, src, n);
}

}  // namespace

// ------------------------------------------------------------------------------------------------

// A captured sequence of launches on the context's stream, replayed as one CUDA graph launch.
// Launch and profiling counters of the captured kernels are credited on every replay.
struct ChunkGraph {
  cudaGraphExec_t exec = nullptr;
  long long kernels = 0;
  long long seen[TNFEM_PROF_CLASSES] = {};
  ChunkGraph() = default;
  ChunkGraph(const ChunkGraph&) = delete;
  ChunkGraph& operator=(const ChunkGraph&) = delete;
  ~ChunkGraph() {
    if (exec) cudaGraphExecDestroy(exec);
  }
  template <typename F>
  void capture(tnfem_ctx* ctx, F&& body) {
    const long long l0 = ctx->launches;
    long long s0[TNFEM_PROF_CLASSES];
    for (int c = 0; c < TNFEM_PROF_CLASSES; ++c) s0[c] = ctx->prof_seen[c];
    TN_CHECK_CUDA(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
    ctx->capturing = true;
    cudaGraph_t g = nullptr;
    try {
      body();
    } catch (...) {
      ctx->capturing = false;
      cudaStreamEndCapture(ctx->stream, &g);
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      throw;
    }
    ctx->capturing = false;
    TN_CHECK_CUDA(cudaStreamEndCapture(ctx->stream, &g));
    kernels = ctx->launches - l0;
    ctx->launches = l0;
    for (int c = 0; c < TNFEM_PROF_CLASSES; ++c) {
      seen[c] = ctx->prof_seen[c] - s0[c];
      ctx->prof_seen[c] = s0[c];
    }
    bool ok = false;
    if (exec) {
      cudaGraphExecUpdateResultInfo info;
      ok = cudaGraphExecUpdate(exec, g, &info) == cudaSuccess;
      if (!ok) {
        cudaGetLastError();
        cudaGraphExecDestroy(exec);
        exec = nullptr;
      }
    }
    if (!ok) {
      cudaError_t e = cudaGraphInstantiate(&exec, g, 0);
      if (e != cudaSuccess) {
        exec = nullptr;
        cudaGraphDestroy(g);
        throw Error(TNFEM_E_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
      }
    }
    cudaGraphDestroy(g);
  }
  void launch(tnfem_ctx* ctx) {
    TN_CHECK_CUDA(cudaGraphLaunch(exec, ctx->stream));
    ctx->launches += kernels;
    for (int c = 0; c < TNFEM_PROF_CLASSES; ++c) ctx->prof_seen[c] += seen[c];
  }
};

template <typename T>
class Amen {
 public:
  ~Amen() {
    if (nvtx_open_) nvtxRangePop();  // a solve that ended by an exception mid-phase
  }
  Amen(tnfem_ctx* ctx, const tnfem_mpo* A, const std::vector<AmenSource>& src, const AmenParams& prm,
       const tnfem_tt* x0)
      : ctx_(ctx), A_(A), src_(src), prm_(prm) {
    d_ = A->d;
    n_ = A->n;
    setup(x0);
  }

  void run(AmenStats& st);
  tnfem_tt* take_result();

 private:
  // bond/core mapping between the current orientation and the stored (original) one
  int oc(int k) const { return o_ == 0 ? k : d_ - 1 - k; }     // original core of current core k
  int ob(int b) const { return o_ == 0 ? b : d_ - b; }         // original bond of current bond b
  int ncur(int k) const { return n_[oc(k)]; }
  int acur(int b) const { return A_->a[ob(b)]; }
  const T* Acur(int k) const { return Prec<T>::A(A_, o_, k); }
  const double* A64cur(int k) const { return A_->p64[o_][k]; }
  // environments: fam -> side (0: left of original bond, 1: right) -> original bond
  T*& envT(int fam, int side, int bond) { return envT_[fam][side][bond]; }
  double*& envS(int fam, int side, int bond) { return envS_[side][fam][bond]; }
  // current-orientation left / right environment of current core k
  int side_left() const { return o_ == 0 ? 0 : 1; }
  int side_right() const { return o_ == 0 ? 1 : 0; }
  T* EL(int fam, int k) { return envT(fam, side_left(), ob(k)); }
  T* ER(int fam, int k) { return envT(fam, side_right(), ob(k + 1)); }
  double* SL(int fam, int k) { return envS(fam, side_left(), ob(k)); }
  double* SR(int fam, int k) { return envS(fam, side_right(), ob(k + 1)); }
  // source cores in the current orientation
  const double* srccore(int s, int k) const {
    return o_ == 0 ? src_[s].v->core[k] : srcflip_[s][k];
  }
  int srcrank(int s, int b) const { return src_[s].v->r[ob(b)]; }

  void setup(const tnfem_tt* x0);
  void flip();
  void orthogonalize_left(std::vector<T*>& cores, std::vector<int>& r, std::vector<size_t>& cap);
  void envs_at(int k, bool with_z);  // compute left envs of bond k+1 from core k
  void core_step(int k, AmenStats& st);
  int cg(int k, T* y, const T* g, double gnorm, double rtol);
  // buffers of one preconditioned conjugate-gradient run in precision U
  template <typename U>
  struct CgBufs {
    U *Bx, *r, *p, *Ap, *z, *ws;
    size_t wsn;
    bool pre;
  };
  template <typename U>
  bool setup_pre(int r0, int n, int r1, int a0, int a1, const U* PL, const U* Ak, const U* PR, DArr<U>& work);
  template <typename U>
  int pcg_run(int r0, int n, int r1, int a0, int a1, const U* PL, const U* Ak, const U* PR, U* y, const U* g,
              double gnorm, double rtol, const CgBufs<U>& b);
  int cg_local_mixed(int k, T* y, const T* g, double gnorm, double rtol);
  // a bounded wait inside a tensor-core kernel ran out (recorded on the device)
  void check_tc_error() {
    if (ctx_->tensor_cores && tc_gemm_error(ctx_) != 0)
      throw Error(TNFEM_E_TIMEOUT, "tensor-core kernel: bounded wait expired");
  }
  void source_proj(int k, bool bra_z_left, bool bra_z_right, double* out, int ry0, int ry1);
  double* bra64(bool z, int k, int r0, int r1);
  void count_apply(int ry0, int ry1, int rx0, int rx1, int n, int a0, int a1) {
    flops_ += 2.0 * ry0 * a0 * rx0 * n * rx1 + 2.0 * ry0 * rx1 * a0 * n * n * a1 + 2.0 * ry0 * n * a1 * rx1 * ry1;
  }

  tnfem_ctx* ctx_;
  const tnfem_mpo* A_;
  std::vector<AmenSource> src_;
  AmenParams prm_;
  int d_ = 0;
  int o_ = 0;
  std::vector<int> n_;
  // x and z cores, stored per original core, holding the current orientation's data
  std::vector<T*> xc_, zc_;
  std::vector<size_t> xcap_, zcap_;
  std::vector<int> rx_, rz_;  // ranks in the current orientation
  std::vector<int> capx_, capz_;  // rank caps per original bond
  // binary64 copies of the bra cores for the source projections (T = float only)
  std::vector<double*> x64_, z64_;
  // flipped source cores
  std::vector<std::vector<double*>> srcflip_;
  // environments
  std::vector<T*> envT_[2][2];                // fam 0: x A x, fam 1: z A x
  std::vector<std::vector<double*>> envS_[2];  // [side][fam] ... see setup
  std::vector<std::vector<double*>> envS_store_;
  // work
  std::vector<std::unique_ptr<DArr<T>>> keepT_;
  std::vector<std::unique_ptr<DArr<double>>> keepD_;
  DArr<T> wsT_, y_, g_, Bx_, r_, p_, Ap_, tmpA_, tmpB_, U_, S_, Vt_, Ue_, Q_, R_, Vn_, svdw_, qrw_, crz_, crs_, nxt_;
  DArr<double> ws64_, g64_, c64_, part_;
  DArr<int> ctl_;
  DArr<T> z_, bjw_;     // preconditioned residual, block-Jacobi set-up workspace
  DArr<float> bjP_;     // block-Jacobi inverses
  long long precond_solves_ = 0;
  // binary32 shadow of the local solve (binary64 sweep with binary32 local solves)
  DArr<float> PL32_, PR32_, g32_, y32_, Bx32_, r32_, p32_, Ap32_, z32_, ws32_, bjw32_;
  DArr<double> d64_;
  long long local_refines_ = 0;
  // Per original core: consecutive visits whose first binary32 correction was confirmed (binary64
  // residual) to have met its target with a factor-2 margin.  From two on, the confirming binary64
  // matvec is skipped except on every fourth sweep; the sweep's own binary64 residual before each
  // local solve still decides convergence, so a skipped check can cost sweeps, never accuracy.
  std::vector<int> trust_;
  int sweep_ = 0;
  long long breakdowns_ = 0;
  bool init_r_ready_ = false;  // r_ holds g - B x_k of the current core step (norm init_rn_)
  bool last_cg_converged_ = false;  // the last conjugate-gradient run met its tolerance
  // per-phase wall time (device-synchronised at each phase boundary when tracing is on)
  bool trace_ = false;
  int cur_phase_ = -1;
  std::chrono::steady_clock::time_point phase_t0_;
  double phase_ms_[kPhases] = {};
  void phase(int next) {
    // NVTX ranges name the phases for a profiler (ncu --nvtx); no cost when no tool is attached
    static const char* const kNames[kPhases] = {"tnfem rhs projection", "tnfem local residual", "tnfem local solve",
                                                "tnfem truncated svd", "tnfem enrichment", "tnfem environments",
                                                "tnfem other"};
    if (nvtx_open_) nvtxRangePop();
    nvtx_open_ = next >= 0;
    if (nvtx_open_) nvtxRangePushA(kNames[next]);
    if (!trace_) return;
    sync(ctx_);
    const auto now = std::chrono::steady_clock::now();
    if (cur_phase_ >= 0) phase_ms_[cur_phase_] += std::chrono::duration<double, std::milli>(now - phase_t0_).count();
    cur_phase_ = next;
    phase_t0_ = now;
  }
  bool nvtx_open_ = false;           // an NVTX phase range is open
  long long fallbacks_ = 0;          // binary32 local solves finished in binary64
  double init_rn_ = 0.0;
  ChunkGraph graph_[2];  // conjugate-gradient chunk graphs, binary32 / binary64
  FusedCg fcg_;          // the conjugate-gradient loop as one persistent kernel
  TcMatvec tcmv_;        // binary32 local matvec on the tensor cores (packed operands)
  bool tcmv_on_ = false; // tcmv_ holds the current local system
  // local matvec of the current local system in precision U
  template <typename U>
  void matvec(int r0, int n, int r1, int a0, int a1, const U* PL, const U* Ak, const U* PR, const U* in, U* out,
              U* ws, size_t wsn, const int* skip) {
    if constexpr (std::is_same<U, float>::value) {
      if (tcmv_on_) {
        tcmv_.apply(ctx_, in, out, skip);
        return;
      }
    }
    local_matvec<U>(ctx_, r0, n, r1, a0, a1, PL, Ak, PR, in, out, ws, wsn, skip);
  }
  double* host_ = nullptr;
  double flops_ = 0.0;
  long long iters_ = 0;
  double max_res_ = 0.0, max_dx_ = 0.0;
};

// envS_ indexing: envS_[side][fam][bond] with fam = 2*s + (0: bra x, 1: bra z)

template <typename T>
void Amen<T>::setup(const tnfem_tt* x0) {
  const int d = d_;
  const int R = prm_.rmax, kick = prm_.kick;
  // rank caps per original bond: bounded by the mode products on either side (+ kick slack)
  capx_.assign(d + 1, 1);
  capz_.assign(d + 1, 1);
  for (int b = 1; b < d; ++b) {
    double lp = 1, rp = 1;
    for (int k = 0; k < b; ++k) lp = std::min(lp * n_[k], 1e9);
    for (int k = b; k < d; ++k) rp = std::min(rp * n_[k], 1e9);
    int mp = (int)std::min(lp, rp);
    capx_[b] = std::max(1, std::min(R, mp) + 2 * kick);
    if (x0) capx_[b] = std::max(capx_[b], x0->r[b]);
    capz_[b] = std::max(1, std::min(std::max(kick, 1), mp));
  }
  xc_.assign(d, nullptr);
  zc_.assign(d, nullptr);
  xcap_.assign(d, 0);
  zcap_.assign(d, 0);
  x64_.assign(d, nullptr);
  z64_.assign(d, nullptr);
  size_t maxcore = 0, maxloc = 0, maxws = 0, maxenvT = 0;
  int maxr = 1;
  for (int k = 0; k < d; ++k) {
    xcap_[k] = (size_t)capx_[k] * n_[k] * capx_[k + 1];
    zcap_[k] = (size_t)capz_[k] * n_[k] * capz_[k + 1];
    keepT_.emplace_back(new DArr<T>(ctx_, xcap_[k]));
    xc_[k] = keepT_.back()->p;
    keepT_.emplace_back(new DArr<T>(ctx_, zcap_[k]));
    zc_[k] = keepT_.back()->p;
    if (!std::is_same<T, double>::value) {
      keepD_.emplace_back(new DArr<double>(ctx_, xcap_[k]));
      x64_[k] = keepD_.back()->p;
      keepD_.emplace_back(new DArr<double>(ctx_, zcap_[k]));
      z64_[k] = keepD_.back()->p;
    }
    maxcore = std::max(maxcore, xcap_[k]);
    maxr = std::max(maxr, capx_[k + 1]);
    // both orientations use this core, with its operator ranks swapped in the flipped one
    int a0 = std::max(A_->a[k], A_->a[k + 1]), a1 = a0;
    maxws = std::max(maxws, local_ws_elems(std::max(capx_[k], capx_[k + 1]), n_[k],
                                           std::max(capx_[k], capx_[k + 1]), a0, a1));
    for (size_t s = 0; s < src_.size(); ++s) {
      const tnfem_tt* v = src_[s].v;
      int rv = std::max(v->r[k], v->r[k + 1]);
      int rr = std::max(std::max(capx_[k], capx_[k + 1]), rv);
      maxws = std::max(maxws, local_ws_elems(rr, n_[k], rr, a0, a1));
    }
  }
  for (int b = 0; b <= d; ++b) maxenvT = std::max(maxenvT, (size_t)capx_[b] * A_->a[b] * capx_[b]);
  maxloc = maxcore;
  // environments (binary T): x A x and z A x, both sides of every bond
  for (int fam = 0; fam < 2; ++fam)
    for (int side = 0; side < 2; ++side) {
      envT_[fam][side].assign(d + 1, nullptr);
      for (int b = 0; b <= d; ++b) {
        size_t sz = fam == 0 ? (size_t)capx_[b] * A_->a[b] * capx_[b] : (size_t)capz_[b] * A_->a[b] * capx_[b];
        keepT_.emplace_back(new DArr<T>(ctx_, std::max<size_t>(sz, 1)));
        envT_[fam][side][b] = keepT_.back()->p;
      }
    }
  // source environments (binary64): per source, bra x and bra z
  const int nf = 2 * (int)src_.size();
  for (int side = 0; side < 2; ++side) {
    envS_[side].assign(nf, std::vector<double*>(d + 1, nullptr));
    for (int f = 0; f < nf; ++f) {
      const AmenSource& S = src_[f / 2];
      for (int b = 0; b <= d; ++b) {
        int rb = (f % 2 == 0) ? capx_[b] : capz_[b];
        size_t sz = (size_t)rb * S.v->r[b] * (S.is_op ? A_->a[b] : 1);
        keepD_.emplace_back(new DArr<double>(ctx_, std::max<size_t>(sz, 1)));
        envS_[side][f][b] = keepD_.back()->p;
      }
    }
  }
  // flipped source cores
  srcflip_.assign(src_.size(), std::vector<double*>(d, nullptr));
  for (size_t s = 0; s < src_.size(); ++s) {
    const tnfem_tt* v = src_[s].v;
    for (int k = 0; k < d; ++k) {
      size_t sz = (size_t)v->r[k] * v->n[k] * v->r[k + 1];
      keepD_.emplace_back(new DArr<double>(ctx_, sz));
      srcflip_[s][d - 1 - k] = keepD_.back()->p;
      transpose3<double>(ctx_, srcflip_[s][d - 1 - k], v->core[k], v->r[k], v->n[k], v->r[k + 1]);
    }
  }
  // work buffers
  wsT_ = DArr<T>(ctx_, maxws);
  ws64_ = DArr<double>(ctx_, maxws);
  y_ = DArr<T>(ctx_, maxloc);
  g_ = DArr<T>(ctx_, maxloc);
  Bx_ = DArr<T>(ctx_, maxloc);
  r_ = DArr<T>(ctx_, maxloc);
  p_ = DArr<T>(ctx_, maxloc);
  Ap_ = DArr<T>(ctx_, maxloc);
  tmpA_ = DArr<T>(ctx_, maxloc + maxenvT);
  tmpB_ = DArr<T>(ctx_, maxloc + maxenvT);
  g64_ = DArr<double>(ctx_, maxloc);
  c64_ = DArr<double>(ctx_, maxloc);
  const int maxm = 8 * 4096;
  (void)maxm;
  size_t maxmn = maxloc + 64;
  U_ = DArr<T>(ctx_, maxmn + (size_t)maxr * maxr * 64);
  S_ = DArr<T>(ctx_, 4096);
  Vt_ = DArr<T>(ctx_, maxmn + (size_t)maxr * maxr * 64);
  Ue_ = DArr<T>(ctx_, 2 * maxmn + (size_t)maxr * 64 * 8);
  Q_ = DArr<T>(ctx_, 2 * maxmn + (size_t)maxr * 64 * 8);
  R_ = DArr<T>(ctx_, (size_t)(maxr + 64) * (maxr + 64) * 4);
  Vn_ = DArr<T>(ctx_, maxmn + (size_t)maxr * maxr * 4);
  svdw_ = DArr<T>(ctx_, 2 * maxmn + (size_t)(maxr + 64) * (maxr + 64) * 8 + 4096);
  qrw_ = DArr<T>(ctx_, 8192);
  crz_ = DArr<T>(ctx_, maxmn);
  crs_ = DArr<T>(ctx_, maxmn);
  nxt_ = DArr<T>(ctx_, maxmn + (size_t)maxr * maxr * 64);
  part_ = DArr<double>(ctx_, 6 * kReduceBlocks + 8);
  z_ = DArr<T>(ctx_, maxloc);
  d64_ = DArr<double>(ctx_, maxloc + 8);
  if (prm_.local_mixed && std::is_same<T, double>::value) {
    PL32_ = DArr<float>(ctx_, maxenvT);
    PR32_ = DArr<float>(ctx_, maxenvT);
    g32_ = DArr<float>(ctx_, maxloc);
    y32_ = DArr<float>(ctx_, maxloc);
    Bx32_ = DArr<float>(ctx_, maxloc);
    r32_ = DArr<float>(ctx_, maxloc);
    p32_ = DArr<float>(ctx_, maxloc);
    Ap32_ = DArr<float>(ctx_, maxloc);
    z32_ = DArr<float>(ctx_, maxloc);
    ws32_ = DArr<float>(ctx_, maxws);
  }
  ctl_ = DArr<int>(ctx_, 4);
  host_ = ctx_->host_pinned;

  // initial x: given start, or a seeded rank-2 Gaussian train; z: seeded rank-kick train
  rx_.assign(d + 1, 1);
  rz_.assign(d + 1, 1);
  for (int b = 1; b < d; ++b) {
    rx_[b] = x0 ? x0->r[b] : std::min(2, capx_[b]);
    rz_[b] = capz_[b];
  }
  for (int k = 0; k < d; ++k) {
    size_t sx = (size_t)rx_[k] * n_[k] * rx_[k + 1];
    size_t sz = (size_t)rz_[k] * n_[k] * rz_[k + 1];
    DArr<double> tmp(ctx_, std::max(sx, sz));
    if (x0) copy<double>(ctx_, tmp.p, x0->core[k], sx);
    else fill_gaussian(ctx_, tmp.p, sx, prm_.seed, 2 * k);
    convert_any<double, T>(ctx_, xc_[k], tmp.p, sx);
    fill_gaussian(ctx_, tmp.p, sz, prm_.seed, 2 * k + 1);
    convert_any<double, T>(ctx_, zc_[k], tmp.p, sz);
    sync(ctx_);
  }
  // boundary environments are 1
  for (int fam = 0; fam < 2; ++fam)
    for (int side = 0; side < 2; ++side) {
      fill<T>(ctx_, envT_[fam][side][0], T(1), 1);
      fill<T>(ctx_, envT_[fam][side][d], T(1), 1);
    }
  for (int side = 0; side < 2; ++side)
    for (int f = 0; f < nf; ++f) {
      fill<double>(ctx_, envS_[side][f][0], 1.0, 1);
      fill<double>(ctx_, envS_[side][f][d], 1.0, 1);
    }
  // right environments for the first forward sweep: left environments of the flipped train
  flip();
  orthogonalize_left(xc_, rx_, xcap_);
  orthogonalize_left(zc_, rz_, zcap_);
  for (int k = 0; k < d - 1; ++k) envs_at(k, prm_.kick > 0);
  flip();
}

// Transpose every x and z core in place (through a scratch buffer) and reverse the ranks.
template <typename T>
void Amen<T>::flip() {
  const int d = d_;
  for (int k = 0; k < d; ++k) {
    // current core k lives in original slot oc(k); after the flip it is current core d-1-k
    int slot = oc(k);
    int r0 = rx_[k], n = n_[slot], r1 = rx_[k + 1];
    transpose3<T>(ctx_, tmpA_.p, xc_[slot], r0, n, r1);
    copy<T>(ctx_, xc_[slot], tmpA_.p, (size_t)r0 * n * r1);
    int z0 = rz_[k], z1 = rz_[k + 1];
    transpose3<T>(ctx_, tmpA_.p, zc_[slot], z0, n, z1);
    copy<T>(ctx_, zc_[slot], tmpA_.p, (size_t)z0 * n * z1);
  }
  std::reverse(rx_.begin(), rx_.end());
  std::reverse(rz_.begin(), rz_.end());
  o_ ^= 1;
}

template <typename T>
void Amen<T>::orthogonalize_left(std::vector<T*>& cores, std::vector<int>& r, std::vector<size_t>& cap) {
  const int d = d_;
  for (int k = 0; k < d - 1; ++k) {
    int slot = oc(k), nslot = oc(k + 1);
    int r0 = r[k], n = n_[slot], r1 = r[k + 1];
    int m = r0 * n, kq = std::min(m, r1);
    copy<T>(ctx_, Ue_.p, cores[slot], (size_t)m * r1);
    qr<T>(ctx_, m, r1, Ue_.p, Q_.p, R_.p, qrw_.p);
    int n2 = n_[nslot], r2 = r[k + 2];
    TN_REQUIRE((size_t)kq * n2 * r2 <= cap[nslot], "orthogonalize: capacity");
    GemmDesc g{kq, n2 * r2, r1, 1, r1, 1, 0, (long long)n2 * r2, 1, 0, (long long)n2 * r2, 1, 0};
    gemm<T>(ctx_, g, T(1), R_.p, cores[nslot], T(0), nxt_.p);
    copy<T>(ctx_, cores[slot], Q_.p, (size_t)m * kq);
    copy<T>(ctx_, cores[nslot], nxt_.p, (size_t)kq * n2 * r2);
    r[k + 1] = kq;
  }
  sync(ctx_);
}

template <typename T>
double* Amen<T>::bra64(bool z, int k, int r0, int r1) {
  int slot = oc(k);
  T* c = z ? zc_[slot] : xc_[slot];
  if constexpr (std::is_same<T, double>::value) {
    return c;
  } else {
    double* d = z ? z64_[slot] : x64_[slot];
    convert_f2d(ctx_, d, c, (size_t)r0 * n_[slot] * r1);
    return d;
  }
}

// Left environments of current bond k+1 from current core k (all families).
template <typename T>
void Amen<T>::envs_at(int k, bool with_z) {
  const int n = ncur(k), a0 = acur(k), a1 = acur(k + 1);
  const int r0 = rx_[k], r1 = rx_[k + 1];
  const int slot = oc(k);
  const int sl = side_left();
  T* xk = xc_[slot];
  env_left<T>(ctx_, r0, r1, r0, r1, n, a0, a1, EL(0, k), xk, Acur(k), xk, envT(0, sl, ob(k + 1)), wsT_.p, wsT_.n);
  count_apply(r0, r1, r0, r1, n, a0, a1);
  if (with_z) {
    const int z0 = rz_[k], z1 = rz_[k + 1];
    env_left<T>(ctx_, z0, z1, r0, r1, n, a0, a1, EL(1, k), zc_[slot], Acur(k), xk, envT(1, sl, ob(k + 1)), wsT_.p,
                wsT_.n);
    count_apply(z0, z1, r0, r1, n, a0, a1);
  }
  for (size_t s = 0; s < src_.size(); ++s) {
    for (int bz = 0; bz < (with_z ? 2 : 1); ++bz) {
      const int f = 2 * (int)s + bz;
      const int b0 = bz ? rz_[k] : r0, b1 = bz ? rz_[k + 1] : r1;
      double* bra = bra64(bz == 1, k, b0, b1);
      const int v0 = srcrank((int)s, k), v1 = srcrank((int)s, k + 1);
      if (src_[s].is_op) {
        env_left<double>(ctx_, b0, b1, v0, v1, n, a0, a1, SL(f, k), bra, A64cur(k), srccore((int)s, k),
                         envS(f, sl, ob(k + 1)), ws64_.p, ws64_.n);
      } else {
        env_left_vec<double>(ctx_, b0, b1, v0, v1, n, SL(f, k), bra, srccore((int)s, k), envS(f, sl, ob(k + 1)),
                             ws64_.p, ws64_.n);
      }
    }
  }
}

// out (binary64, ry0 x n x ry1) = sum_s c_s * projection of source s onto the bra interfaces
// (x or z on the left, x or z on the right).
template <typename T>
void Amen<T>::source_proj(int k, bool zl, bool zr, double* out, int ry0, int ry1) {
  const int n = ncur(k), a0 = acur(k), a1 = acur(k + 1);
  for (size_t s = 0; s < src_.size(); ++s) {
    const int fl = 2 * (int)s + (zl ? 1 : 0), fr = 2 * (int)s + (zr ? 1 : 0);
    const double beta = s == 0 ? 0.0 : 1.0;
    const int v0 = srcrank((int)s, k), v1 = srcrank((int)s, k + 1);
    if (src_[s].is_op) {
      local_apply<double>(ctx_, ry0, ry1, v0, v1, n, a0, a1, SL(fl, k), A64cur(k), SR(fr, k), srccore((int)s, k), out,
                          src_[s].coef, beta, ws64_.p, ws64_.n);
      count_apply(ry0, ry1, v0, v1, n, a0, a1);
    } else {
      local_rhs<double>(ctx_, ry0, n, ry1, v0, v1, SL(fl, k), srccore((int)s, k), SR(fr, k), out, ws64_.p, ws64_.n,
                        src_[s].coef, beta);
    }
  }
}

template <typename T>
template <typename U>
bool Amen<T>::setup_pre(int r0, int n, int r1, int a0, int a1, const U* PL, const U* Ak, const U* PR, DArr<U>& work) {
  if (!prm_.precond || !bj_fits(r0, n, r1) || !bj_worth_it(r0, n)) return false;
  work.ensure(ctx_, bj_work_elems(r0, n, r1, a0, a1));
  bjP_.ensure(ctx_, (size_t)r1 * r0 * n * r0 * n);
  const bool ok = bj_setup<U>(ctx_, r0, n, r1, a0, a1, PL, Ak, PR, bjP_.p, work.p, work.n, ctl_.p + 2);
  if (ok) ++precond_solves_;
  return ok;
}

// Preconditioned conjugate gradients on B y = g from the given y, to ||g - B y|| <= rtol ||g||.
// Control flow stays on the device (ctl); the host reads two integers after every chunk of 8
// iterations.  On a capturable stream the chunk is captured once per local solve into a CUDA
// graph (updated in place when the previous solve's graph has the same topology) and replayed,
// so the host issues one graph launch instead of ~60 kernel launches per chunk.
template <typename T>
template <typename U>
int Amen<T>::pcg_run(int r0, int n, int r1, int a0, int a1, const U* PL, const U* Ak, const U* PR, U* y,
                     const U* g, double gnorm, double rtol, const CgBufs<U>& b) {
  const size_t N = (size_t)r0 * n * r1;
  const bool tc_mv = std::is_same<U, float>::value && tcmv_on_;
  if (prm_.fused_cg && !tc_mv) {
    // the whole preconditioned CG loop as one persistent cooperative kernel
    const FcgPlan pl = fcg_.plan<U>(ctx_, r0, n, r1, a0, a1, b.pre);
    if (pl.ok) {
      int state = 0;
      const double stop2 = rtol * rtol * gnorm * gnorm;
      const int done = fcg_.run<U>(ctx_, pl, r0, n, r1, a0, a1, PL, Ak, PR, b.pre ? bjP_.p : nullptr, g, y, stop2,
                                   prm_.local_maxit, &state);
      last_cg_converged_ = state == 1;
      for (int i = 0; i <= done; ++i) count_apply(r0, r1, r0, r1, n, a0, a1);
      if (state == 2) {
        // Loss of positive curvature (rounding in a binary32 solve of an ill-conditioned system):
        // the iterate of the last completed step is kept and the sweep carries on.
        ++breakdowns_;
        if (b.pre && done < 2) {
          CgBufs<U> plain = b;
          plain.pre = false;
          return done + pcg_run<U>(r0, n, r1, a0, a1, PL, Ak, PR, y, g, gnorm, rtol, plain);
        }
      }
      return done;
    }
  }
  double* prr[2] = {part_.p, part_.p + kReduceBlocks};
  double* prz_b[2] = {part_.p + 2 * kReduceBlocks, part_.p + 3 * kReduceBlocks};
  double* ppap = part_.p + 4 * kReduceBlocks;
  int* ctl = ctl_.p;
  U* z = b.pre ? b.z : b.r;
  double** prz = b.pre ? prz_b : prr;
  TN_CHECK_CUDA(cudaMemsetAsync(ctl, 0, 4 * sizeof(int), ctx_->stream));
  matvec<U>(r0, n, r1, a0, a1, PL, Ak, PR, y, b.Bx, b.ws, b.wsn, nullptr);
  count_apply(r0, r1, r0, r1, n, a0, a1);
  // blocks of the vector kernels: ~8 elements per thread (the vectors are short); the
  // preconditioner works block by block over b
  const int nb = (int)std::max<long long>(1, std::min<long long>(kReduceBlocks, ((long long)N + 2047) / 2048));
  // preconditioner apply: up to 4 CTAs per block b (rows split), at most kReduceBlocks CTAs
  const int nbj = std::max(1, std::min(kReduceBlocks, r1 * std::max(1, std::min(4, kReduceBlocks / std::max(1, r1)))));
  const int np_rz = b.pre ? nbj : nb;
  cg_init_kernel<U><<<nb, RT, 0, ctx_->stream>>>(g, b.Bx, b.r, b.p, N, prr[0]);
  count_launch(ctx_);
  if (b.pre) bj_apply<U>(ctx_, r0, n, r1, bjP_.p, b.r, b.z, b.p, prz[0], nullptr, nbj);
  const double stop2 = rtol * rtol * gnorm * gnorm;
  constexpr int kChunk = 8;  // even: the partial-sum buffers are back at index 0 after a chunk
  auto chunk = [&]() {
    int cur = 0;
    for (int c = 0; c < kChunk; ++c) {
      const int nx = cur ^ 1;
      matvec<U>(r0, n, r1, a0, a1, PL, Ak, PR, b.p, b.Ap, b.ws, b.wsn, ctl);
      {
        ProfScope ps(ctx_, TNFEM_PROF_KRYLOV, 2.0 * N, 2.0 * N * sizeof(U));
        cg_dot_kernel<U><<<nb, RT, 0, ctx_->stream>>>(b.p, b.Ap, N, ppap, ctl);
      }
      {
        ProfScope ps(ctx_, TNFEM_PROF_KRYLOV, 6.0 * N, 6.0 * N * sizeof(U));
        cg_update1_kernel<U><<<nb, RT, 0, ctx_->stream>>>(y, b.r, b.p, b.Ap, N, prr[cur], nb, prz[cur], np_rz, ppap,
                                                          nb, prr[nx], ctl, stop2);
      }
      if (b.pre) bj_apply<U>(ctx_, r0, n, r1, bjP_.p, b.r, b.z, nullptr, prz[nx], ctl, nbj);
      {
        ProfScope ps(ctx_, TNFEM_PROF_KRYLOV, 2.0 * N, 3.0 * N * sizeof(U));
        cg_update2_kernel<U><<<nb, RT, 0, ctx_->stream>>>(b.p, z, N, prz[nx], prz[cur], np_rz, ctl);
      }
      count_launch(ctx_, 3);
      cur = nx;
    }
  };
  ChunkGraph& cgph = graph_[sizeof(U) == 8 ? 1 : 0];
  const bool use_graph = prm_.graphs && ctx_->stream != nullptr;
  if (use_graph) cgph.capture(ctx_, chunk);
  int done_it = 0;
  const int maxit = prm_.local_maxit;
  int it = 0;
  while (it < maxit) {
    if (use_graph) cgph.launch(ctx_);
    else chunk();
    it += kChunk;
    check_launch(ctx_, "cg");
    int h[2];
    TN_CHECK_CUDA(cudaMemcpyAsync(h, ctl, 2 * sizeof(int), cudaMemcpyDeviceToHost, ctx_->stream));
    sync(ctx_);
    done_it = h[1];
    last_cg_converged_ = h[0] == 1;
    if (h[0] == 2) {
      // Loss of positive curvature (rounding in a binary32 solve of an ill-conditioned system):
      // the iterate of the last completed step is kept and the sweep carries on.
      ++breakdowns_;
      if (b.pre && done_it < 2) {
        // the binary32 block inverses were not positive definite: retry unpreconditioned
        CgBufs<U> plain = b;
        plain.pre = false;
        for (int i = 0; i < done_it; ++i) count_apply(r0, r1, r0, r1, n, a0, a1);
        return done_it + pcg_run<U>(r0, n, r1, a0, a1, PL, Ak, PR, y, g, gnorm, rtol, plain);
      }
      break;
    }
    if (h[0]) break;
  }
  for (int i = 0; i < done_it; ++i) count_apply(r0, r1, r0, r1, n, a0, a1);
  return done_it;
}

template <typename T>
int Amen<T>::cg(int k, T* y, const T* g, double gnorm, double rtol) {
  if (prm_.local_mixed && std::is_same<T, double>::value) return cg_local_mixed(k, y, g, gnorm, rtol);
  const int n = ncur(k), a0 = acur(k), a1 = acur(k + 1);
  const int r0 = rx_[k], r1 = rx_[k + 1];
  const T* PL = EL(0, k);
  const T* PR = ER(0, k);
  const T* Ak = Acur(k);
  const bool pre = setup_pre<T>(r0, n, r1, a0, a1, PL, Ak, PR, bjw_);
  CgBufs<T> b{Bx_.p, r_.p, p_.p, Ap_.p, z_.p, wsT_.p, wsT_.n, pre};
  if constexpr (std::is_same<T, float>::value) {
    if (ctx_->tensor_cores) {
      tcmv_.plan(ctx_, r0, n, r1, a0, a1);
      tcmv_.prepare(ctx_, PL, Ak, PR);
      tcmv_on_ = true;
    }
  }
  int it = 0;
  try {
    it = pcg_run<T>(r0, n, r1, a0, a1, PL, Ak, PR, y, g, gnorm, rtol, b);
  } catch (...) {
    tcmv_on_ = false;
    throw;
  }
  tcmv_on_ = false;
  check_tc_error();
  return it;
}

// Binary64 sweep, binary32 local solves: iterative refinement of the local system against its
// binary64 residual.  Each step solves B d = r / ||r|| by binary32 preconditioned CG (interfaces
// and operator core rounded to binary32) and updates y += ||r|| d in binary64, until the binary64
// local residual meets rtol.
template <typename T>
int Amen<T>::cg_local_mixed(int k, T* y, const T* g, double gnorm, double rtol) {
  if constexpr (!std::is_same<T, double>::value) {
    (void)k; (void)y; (void)g; (void)gnorm; (void)rtol;
    throw Error(TNFEM_E_INVALID, "binary32 local solves need a binary64 sweep");
  } else {
    const int n = ncur(k), a0 = acur(k), a1 = acur(k + 1);
    const int r0 = rx_[k], r1 = rx_[k + 1];
    const size_t N = (size_t)r0 * n * r1;
    const double* PL = EL(0, k);
    const double* PR = ER(0, k);
    const double* Ak = Acur(k);
    convert_d2f(ctx_, PL32_.p, PL, (size_t)r0 * a0 * r0);
    convert_d2f(ctx_, PR32_.p, PR, (size_t)r1 * a1 * r1);
    const float* A32 = A_->p32[o_][k];
    const bool pre = setup_pre<float>(r0, n, r1, a0, a1, PL32_.p, A32, PR32_.p, bjw32_);
    CgBufs<float> b{Bx32_.p, r32_.p, p32_.p, Ap32_.p, z32_.p, ws32_.p, ws32_.n, pre};
    if (ctx_->tensor_cores) {
      tcmv_.plan(ctx_, r0, n, r1, a0, a1);
      tcmv_.prepare(ctx_, PL32_.p, A32, PR32_.p);
      tcmv_on_ = true;
    }
    struct Off {  // the tensor-core operands belong to this local system only
      bool& f;
      ~Off() { f = false; }
    } off{tcmv_on_};
    int iters = 0;
    double prev = 0.0;
    const bool have_r0 = init_r_ready_;  // the sweep step already formed r = g - B y for this y
    init_r_ready_ = false;
    bool stalled = false;
    const int slot = oc(k);
    if ((int)trust_.size() < d_) trust_.assign(d_, 0);
    for (int step = 0; step < 12; ++step) {
      double rn;
      if (step == 1 && trust_[slot] >= 2 && sweep_ % 4 != 3) break;  // confirmation skipped
      if (step == 0 && have_r0) {
        rn = init_rn_;
      } else {
        // binary64 residual r = g - B y
        local_matvec<double>(ctx_, r0, n, r1, a0, a1, PL, Ak, PR, y, Bx_.p, wsT_.p, wsT_.n);
        count_apply(r0, r1, r0, r1, n, a0, a1);
        diff_kernel<double><<<kReduceBlocks, RT, 0, ctx_->stream>>>(r_.p, g, Bx_.p, N, part_.p + 5 * kReduceBlocks);
        sum_partials_kernel<<<1, RT, 0, ctx_->stream>>>(part_.p + 5 * kReduceBlocks, d64_.p + N);
        count_launch(ctx_, 2);
        double rn2 = 0;
        TN_CHECK_CUDA(cudaMemcpyAsync(&rn2, d64_.p + N, sizeof(double), cudaMemcpyDeviceToHost, ctx_->stream));
        sync(ctx_);
        rn = std::sqrt(rn2);
      }
      if (!(rn > rtol * gnorm)) {
        if (step == 1) trust_[slot] = rn <= 0.5 * rtol * gnorm ? trust_[slot] + 1 : 0;
        break;
      }
      if (step > 0) trust_[slot] = 0;  // one binary32 correction was not enough
      if (step > 0 && !(rn < 0.5 * prev)) {  // stagnation: binary32 cannot reduce it further
        stalled = true;
        break;
      }
      prev = rn;
      ++local_refines_;
      // d solves B d = r / ||r|| in binary32 to the reduction still needed (not below 1e-6)
      scale_to_float_kernel<<<nblk((long long)N), RT, 0, ctx_->stream>>>(g32_.p, r_.p, 1.0 / rn, N);
      count_launch(ctx_);
      fill<float>(ctx_, y32_.p, 0.0f, N);
      const double need = rtol * gnorm / rn;
      iters += pcg_run<float>(r0, n, r1, a0, a1, PL32_.p, A32, PR32_.p, y32_.p, g32_.p, 1.0,
                              std::max(1e-6, 0.5 * need), b);
      add_scaled_float_kernel<<<nblk((long long)N), RT, 0, ctx_->stream>>>(y, y32_.p, rn, N);
      count_launch(ctx_);
    }
    if (stalled) {
      // binary32 cannot reduce this system's residual any further (its conditioning exceeds what
      // binary32 products resolve): finish the local solve in binary64 from the current y
      ++fallbacks_;
      const bool pre64 = setup_pre<double>(r0, n, r1, a0, a1, PL, Ak, PR, bjw_);
      CgBufs<double> b64{Bx_.p, r_.p, p_.p, Ap_.p, z_.p, wsT_.p, wsT_.n, pre64};
      iters += pcg_run<double>(r0, n, r1, a0, a1, PL, Ak, PR, y, g, gnorm, rtol, b64);
    }
    check_tc_error();
    return iters;
  }
}

template <typename T>
void Amen<T>::core_step(int k, AmenStats& st) {
  const int d = d_;
  const int n = ncur(k), a0 = acur(k), a1 = acur(k + 1);
  const int r0 = rx_[k], r1 = rx_[k + 1];
  const int slot = oc(k);
  const size_t N = (size_t)r0 * n * r1;
  T* xk = xc_[slot];
  const T* Ak = Acur(k);
  // 1. projected right-hand side
  phase(kPhaseRhs);
  source_proj(k, false, false, g64_.p, r0, r1);
  convert_any<double, T>(ctx_, g_.p, g64_.p, N);
  const double gnorm = nrm2<double>(ctx_, g64_.p, N);
  // 2. local residual before the solve
  phase(kPhaseResidual);
  local_matvec<T>(ctx_, r0, n, r1, a0, a1, EL(0, k), Ak, ER(0, k), xk, Bx_.p, wsT_.p, wsT_.n);
  count_apply(r0, r1, r0, r1, n, a0, a1);
  diff_kernel<T><<<kReduceBlocks, RT, 0, ctx_->stream>>>(r_.p, g_.p, Bx_.p, N, part_.p);
  sum_partials_kernel<<<1, RT, 0, ctx_->stream>>>(part_.p, c64_.p);
  count_launch(ctx_, 2);
  double rn2 = 0;
  TN_CHECK_CUDA(cudaMemcpyAsync(&rn2, c64_.p, sizeof(double), cudaMemcpyDeviceToHost, ctx_->stream));
  sync(ctx_);
  if (!std::isfinite(gnorm) || !std::isfinite(rn2))
    throw Error(TNFEM_E_NUMERIC, "non-finite local right-hand side or residual at core " + std::to_string(k) +
                                     " (NaN/Inf in the operator, the load, the start or an environment)");
  const double res = gnorm > 0 ? std::sqrt(rn2) / gnorm : 0.0;
  max_res_ = std::max(max_res_, res);
  // r_ now holds g - B x_k; the binary32-local-solve path starts its refinement from it
  init_rn_ = std::sqrt(rn2);
  init_r_ready_ = true;
  // 3. local solve (a zero projected load has the zero local solution)
  phase(kPhaseSolve);
  if (gnorm > 0) copy<T>(ctx_, y_.p, xk, N);
  else fill<T>(ctx_, y_.p, T(0), N);
  if (res > prm_.tol / prm_.resid_damp && gnorm > 0) {
    // the local system is solved to a fraction of its own starting residual (not below tol / 2):
    // the sweep's accuracy is set by the truncation, so tighter local solves only cost iterations
    const double rtol = std::max(prm_.tol / prm_.resid_damp, prm_.local_rtol * res);
    iters_ += cg(k, y_.p, g_.p, gnorm, rtol);
    diff_kernel<T><<<kReduceBlocks, RT, 0, ctx_->stream>>>(r_.p, y_.p, xk, N, part_.p);
    sum_partials_kernel<<<1, RT, 0, ctx_->stream>>>(part_.p, c64_.p);
    count_launch(ctx_, 2);
    double dn2 = 0;
    TN_CHECK_CUDA(cudaMemcpyAsync(&dn2, c64_.p, sizeof(double), cudaMemcpyDeviceToHost, ctx_->stream));
    sync(ctx_);
    const double yn = nrm2<T>(ctx_, y_.p, N);
    if (!std::isfinite(dn2) || !std::isfinite(yn))
      throw Error(TNFEM_E_NUMERIC, "non-finite local solution at core " + std::to_string(k));
    if (yn > 0) max_dx_ = std::max(max_dx_, std::sqrt(dn2) / yn);
  }
  if (k == d - 1) {
    copy<T>(ctx_, xk, y_.p, N);
    return;
  }
  // 4. truncated SVD of y as (r0 n) x r1
  phase(kPhaseSvd);
  const int m = r0 * n;
  int p;
  if (m >= r1) {
    copy<T>(ctx_, Ue_.p, y_.p, N);
    svd<T>(ctx_, m, r1, Ue_.p, U_.p, S_.p, Vt_.p, svdw_.p);
    p = r1;  // U: m x p, Vt: p x r1
  } else {
    transpose2<T>(ctx_, Ue_.p, y_.p, m, r1);                   // r1 x m
    svd<T>(ctx_, r1, m, Ue_.p, Q_.p, S_.p, R_.p, svdw_.p);     // Q: r1 x m, R: m x m
    transpose2<T>(ctx_, U_.p, R_.p, m, m);                     // U = R^T: m x m
    transpose2<T>(ctx_, Vt_.p, Q_.p, r1, m);                   // Vt = Q^T: m x r1
    p = m;
  }
  std::vector<double> S(p);
  {
    std::vector<T> St(p);
    TN_CHECK_CUDA(cudaMemcpyAsync(St.data(), S_.p, p * sizeof(T), cudaMemcpyDeviceToHost, ctx_->stream));
    sync(ctx_);
    double s2 = 0;
    for (int i = 0; i < p; ++i) { S[i] = (double)St[i]; s2 += S[i] * S[i]; }
    const double delta = prm_.tol / std::sqrt((double)d) * std::sqrt(s2);
    st.last_rank_trunc = truncation_rank(S, delta, prm_.rmax);
  }
  const int rk = st.last_rank_trunc;
  // V = diag(S[:rk]) Vt[:rk, :]  (rk x r1), in place in Vt
  scale_rows_kernel<T><<<nblk((long long)rk * r1), RT, 0, ctx_->stream>>>(Vt_.p, S_.p, rk, r1);
  count_launch(ctx_);
  // U_rk packed (m x rk) into the first rk columns of Ue (leading dimension rk + rz1)
  const int rz1 = rz_[k + 1];
  const int kick = prm_.kick;
  const int ue_cols = rk + (kick > 0 ? rz1 : 0);
  pack_cols_kernel<T><<<nblk((long long)m * rk), RT, 0, ctx_->stream>>>(Ue_.p, U_.p, m, p, rk, ue_cols, 0);
  count_launch(ctx_);
  int kq = rk;
  T* Vnew = Vt_.p;  // kq x r1
  if (kick > 0) {
    phase(kPhaseEnrich);
    // yt = U_rk V (m x r1)
    GemmDesc gy{m, r1, rk, 1, ue_cols, 1, 0, r1, 1, 0, r1, 1, 0};
    gemm<T>(ctx_, gy, T(1), Ue_.p, Vt_.p, T(0), y_.p);
    const int z0 = rz_[k];
    // crs = PhiL A PhiZR yt - b projected on (x left, z right)   (r0 x n x rz1)
    source_proj(k, false, true, c64_.p, r0, rz1);
    convert_any<double, T>(ctx_, crs_.p, c64_.p, (size_t)r0 * n * rz1);
    if (4 * rz1 <= r1) {
      // the right interface is narrow (kickrank columns): contract it first by applying the flipped
      // operator core to the transposed train, y^T[b',i,a'] = PhiZR A^T PhiL x^T, which costs
      // O(r^2 a (n + a) rz) instead of the O(r^2 n^2 a^2) of the left-first order
      T* xt = tmpA_.p;
      T* yt2 = tmpB_.p;
      transpose3<T>(ctx_, xt, y_.p, r0, n, r1);  // [r1][n][r0]
      const T* Af = Prec<T>::A(A_, o_ ^ 1, d - 1 - k);
      local_apply<T>(ctx_, rz1, r0, r1, r0, n, a1, a0, ER(1, k), Af, EL(0, k), xt, yt2, T(1), T(0), wsT_.p, wsT_.n);
      transpose3<T>(ctx_, xt, yt2, rz1, n, r0);  // [r0][n][rz1]
      axpby<T>(ctx_, crs_.p, T(1), xt, T(-1), (size_t)r0 * n * rz1);
    } else {
      local_apply<T>(ctx_, r0, rz1, r0, r1, n, a0, a1, EL(0, k), Ak, ER(1, k), y_.p, crs_.p, T(1), T(-1), wsT_.p,
                     wsT_.n);
    }
    count_apply(r0, rz1, r0, r1, n, a0, a1);
    // crz = PhiZL A PhiZR yt - b projected on z's interfaces   (z0 x n x rz1)
    source_proj(k, true, true, c64_.p, z0, rz1);
    convert_any<double, T>(ctx_, crz_.p, c64_.p, (size_t)z0 * n * rz1);
    local_apply<T>(ctx_, z0, rz1, r0, r1, n, a0, a1, EL(1, k), Ak, ER(1, k), y_.p, crz_.p, T(1), T(-1), wsT_.p,
                   wsT_.n);
    count_apply(z0, rz1, r0, r1, n, a0, a1);
    // new z core: leading left singular vectors of crz as (z0 n) x rz1
    const int mz = z0 * n;
    int kz = std::min(kick, std::min(mz, rz1));
    kz = std::max(1, std::min(kz, capz_[ob(k + 1)]));
    if (mz >= rz1) {
      svd<T>(ctx_, mz, rz1, crz_.p, Q_.p, S_.p, R_.p, svdw_.p);  // Q: mz x rz1
      pack_cols_kernel<T><<<nblk((long long)mz * kz), RT, 0, ctx_->stream>>>(zc_[slot], Q_.p, mz, rz1, kz, kz, 0);
    } else {
      transpose2<T>(ctx_, nxt_.p, crz_.p, mz, rz1);                 // rz1 x mz
      svd<T>(ctx_, rz1, mz, nxt_.p, Q_.p, S_.p, R_.p, svdw_.p);     // R: mz x mz (right vectors)
      transpose2<T>(ctx_, nxt_.p, R_.p, mz, mz);                     // left vectors of crz
      pack_cols_kernel<T><<<nblk((long long)mz * kz), RT, 0, ctx_->stream>>>(zc_[slot], nxt_.p, mz, mz, kz, kz, 0);
    }
    count_launch(ctx_);
    rz_[k + 1] = kz;
    // enrichment block into Ue's last rz1 columns, then QR
    pack_cols_kernel<T><<<nblk((long long)m * rz1), RT, 0, ctx_->stream>>>(Ue_.p, crs_.p, m, rz1, rz1, ue_cols, rk);
    count_launch(ctx_);
    // U_rk has orthonormal columns: only the rz1 enrichment columns need orthogonalising
    qr_ext<T>(ctx_, m, rk, rz1, Ue_.p, Q_.p, R_.p, qrw_.p, qrw_.n);
    kq = std::min(m, ue_cols);
    // Vnew = R[:, :rk] V   (kq x r1)
    GemmDesc gv{kq, r1, rk, 1, ue_cols, 1, 0, r1, 1, 0, r1, 1, 0};
    gemm<T>(ctx_, gv, T(1), R_.p, Vt_.p, T(0), Vn_.p);
    Vnew = Vn_.p;
    TN_REQUIRE((size_t)m * kq <= xcap_[slot], "enriched core exceeds capacity");
    copy<T>(ctx_, xk, Q_.p, (size_t)m * kq);
  } else {
    // x_k = U_rk
    copy<T>(ctx_, xk, Ue_.p, (size_t)m * rk);
  }
  // 6. x_{k+1} <- Vnew x_{k+1}
  phase(kPhaseEnv);
  const int nslot = oc(k + 1);
  const int n2 = ncur(k + 1), r2 = rx_[k + 2];
  TN_REQUIRE((size_t)kq * n2 * r2 <= xcap_[nslot], "next core exceeds capacity");
  GemmDesc gn{kq, n2 * r2, r1, 1, r1, 1, 0, (long long)n2 * r2, 1, 0, (long long)n2 * r2, 1, 0};
  gemm<T>(ctx_, gn, T(1), Vnew, xc_[nslot], T(0), nxt_.p);
  copy<T>(ctx_, xc_[nslot], nxt_.p, (size_t)kq * n2 * r2);
  rx_[k + 1] = kq;
  envs_at(k, kick > 0);
}

template <typename T>
void Amen<T>::run(AmenStats& st) {
  const int d = d_;
  st = AmenStats();
  trace_ = getenv("TNFEM_TRACE") != nullptr;
  double res_hist[2] = {0.0, 0.0};  // largest local residuals of the two previous sweeps
  trust_.assign(d, 0);
  for (int sweep = 0; sweep < prm_.max_sweeps; ++sweep) {
    sweep_ = sweep;
    max_res_ = 0.0;
    max_dx_ = 0.0;
    for (int k = 0; k < d && !st.timed_out; ++k) {
      core_step(k, st);
      if (prm_.has_deadline && std::chrono::steady_clock::now() > prm_.deadline) st.timed_out = true;
    }
    st.sweeps = sweep + 1;
    st.max_res = max_res_;
    st.max_dx = max_dx_;
    if (st.timed_out) break;
    if (prm_.verbose)
      fprintf(stderr, "[tnfem] sweep %d: max res %.3e max dx %.3e rank %d iters %lld refines %lld fallbacks %lld\n",
              sweep, max_res_, max_dx_, *std::max_element(rx_.begin(), rx_.end()), iters_, local_refines_, fallbacks_);
    flip();
    if (max_res_ <= prm_.tol || max_dx_ <= prm_.tol) {
      st.converged = true;
      break;
    }
    // Stagnation at the truncation floor: the local residuals no longer fall (the SVD truncation
    // re-creates them every step) and the core updates are within a small factor of tol, so more
    // sweeps would only move the iterate by amounts of the order of the truncation itself.
    if (sweep >= 2 && max_dx_ <= prm_.stall_dx * prm_.tol &&
        max_res_ >= 0.5 * std::min(res_hist[0], res_hist[1])) {
      st.converged = true;
      break;
    }
    res_hist[0] = res_hist[1];
    res_hist[1] = max_res_;
  }
  phase(kPhaseOther);
  if (o_ == 1) flip();
  phase(-1);
  for (int i = 0; i < kPhases; ++i) st.phase_ms[i] = phase_ms_[i];
  st.local_iters = iters_;
  st.flops = flops_;
  st.max_rank = *std::max_element(rx_.begin(), rx_.end());
}

template <typename T>
tnfem_tt* Amen<T>::take_result() {
  TN_REQUIRE(o_ == 0, "result requested in flipped orientation");
  tnfem_tt* u = tt_new(ctx_, n_, rx_);
  for (int k = 0; k < d_; ++k)
    convert_any<T, double>(ctx_, u->core[k], xc_[k], (size_t)rx_[k] * n_[k] * rx_[k + 1]);
  sync(ctx_);
  return u;
}

tnfem_tt* amen_solve(tnfem_ctx* ctx, const tnfem_mpo* A, const std::vector<AmenSource>& src, const AmenParams& prm,
                     const tnfem_tt* x0, bool single, AmenStats& st) {
  mpo_prepare(const_cast<tnfem_mpo*>(A));
  if (single) {
    Amen<float> s(ctx, A, src, prm, x0);
    s.run(st);
    return s.take_result();
  }
  Amen<double> s(ctx, A, src, prm, x0);
  s.run(st);
  return s.take_result();
}

}  // namespace tnfem
