// C ABI of the library (include/tnfem.h): argument checks, handle bookkeeping and the two solve
// drivers (binary64 AMEn, and binary32 AMEn inside binary64 iterative refinement).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <memory>

#include "amen.h"
#include "builder.h"
#include "cg_fused.h"
#include "precond.h"
#include "internal.h"
#include "tc_gemm.h"
#include "tc_matvec.h"

using namespace tnfem;

namespace {

// sets the binary32 GEMM engine for the duration of one call
struct EngineScope {
  tnfem_ctx* ctx;
  bool saved;
  EngineScope(tnfem_ctx* c, int engine) : ctx(c), saved(c->tensor_cores) { c->tensor_cores = engine == 1; }
  ~EngineScope() { ctx->tensor_cores = saved; }
};

// large binary64 GEMMs in double-binary32 arithmetic for the scope's duration
struct DfScope {
  tnfem_ctx* ctx;
  bool saved;
  DfScope(tnfem_ctx* c, bool on) : ctx(c), saved(c->df64) { c->df64 = on; }
  ~DfScope() { ctx->df64 = saved; }
};

template <typename F>
tnfem_status guard(tnfem_ctx* ctx, F&& f) {
  try {
    f();
    if (ctx) ctx->err.clear();
    return TNFEM_OK;
  } catch (const Error& e) {
    if (ctx) ctx->err = e.what();
    if (e.status == TNFEM_E_CUDA) cudaGetLastError();
    return e.status;
  } catch (const std::bad_alloc&) {
    if (ctx) ctx->err = "host allocation failed";
    return TNFEM_E_NOMEM;
  } catch (const std::exception& e) {
    if (ctx) ctx->err = e.what();
    return TNFEM_E_INVALID;
  }
}

void check_grid(const tnfem_grid* g) {
  TN_REQUIRE(g, "grid is null");
  TN_REQUIRE(g->dim == 2 || g->dim == 3, "grid.dim must be 2 or 3");
  TN_REQUIRE(g->levels >= 1 && g->levels <= 20, "grid.levels must be in [1, 20]");
  TN_REQUIRE(g->mapped >= 0 && g->mapped <= 2, "grid.mapped must be 0, 1 or 2");
  if (!g->mapped)
    for (int d = 0; d < g->dim; ++d) TN_REQUIRE(g->hi[d] > g->lo[d], "grid box is degenerate");
  if (g->mapped == 2) check_quad(*g);
}

void check_material(const tnfem_material* m) {
  TN_REQUIRE(m, "material is null");
  TN_REQUIRE(m->E[0] > 0 && m->E[1] > 0, "Young's modulus must be positive");
  TN_REQUIRE(m->nu >= 0.0 && m->nu < 0.5, "Poisson's ratio must be in [0, 0.5)");
}

tnfem_mpo* upload_mpo(tnfem_ctx* ctx, const HTrain& h, int ncomp, int dim) {
  const int d = (int)h.c.size();
  std::vector<int> n(d), a(d + 1);
  a[0] = 1;
  for (int k = 0; k < d; ++k) {
    n[k] = (k == 0) ? ncomp : (1 << dim);
    a[k + 1] = h.c[k].r1;
  }
  tnfem_mpo* A = mpo_new(ctx, n, a);
  try {
    for (int k = 0; k < d; ++k)
      TN_CHECK_CUDA(cudaMemcpyAsync(A->core[k], h.c[k].v.data(), h.c[k].v.size() * sizeof(double),
                                    cudaMemcpyHostToDevice, ctx->stream));
    sync(ctx);
  } catch (...) {
    delete A;
    throw;
  }
  return A;
}

tnfem_tt* upload_tt(tnfem_ctx* ctx, const HTrain& h, int ncomp, int dim) {
  const int d = (int)h.c.size();
  std::vector<int> n(d), r(d + 1);
  r[0] = 1;
  for (int k = 0; k < d; ++k) {
    n[k] = (k == 0) ? ncomp : (1 << dim);
    r[k + 1] = h.c[k].r1;
  }
  tnfem_tt* x = tt_new(ctx, n, r);
  try {
    for (int k = 0; k < d; ++k)
      TN_CHECK_CUDA(cudaMemcpyAsync(x->core[k], h.c[k].v.data(), h.c[k].v.size() * sizeof(double),
                                    cudaMemcpyHostToDevice, ctx->stream));
    sync(ctx);
  } catch (...) {
    delete x;
    throw;
  }
  return x;
}

// General quadrilateral (grid.mapped == 2): the dense stencil coefficients or load values are
// built on the host, their TT comes from a TT-SVD on the device; the operator train (rank 9 x the
// coefficients') is formed on the host and rounded on the device like the box operators.
std::vector<int> quad_modes(int L, int first, int last) {
  std::vector<int> m(1, first);
  m.insert(m.end(), L, 4);
  if (last) m.push_back(last);
  return m;
}

HTrain download_train(tnfem_ctx* ctx, const tnfem_tt* x) {
  HTrain h;
  for (int k = 0; k < x->d; ++k) {
    HCore c{x->r[k], x->n[k], x->r[k + 1], std::vector<double>((size_t)x->r[k] * x->n[k] * x->r[k + 1])};
    TN_CHECK_CUDA(cudaMemcpyAsync(c.v.data(), x->core[k], c.v.size() * sizeof(double), cudaMemcpyDeviceToHost,
                                  ctx->stream));
    h.c.push_back(std::move(c));
  }
  sync(ctx);
  return h;
}

// a host train with arbitrary modes, rounded on the device and brought back
HTrain round_on_device(tnfem_ctx* ctx, const HTrain& h, double eps) {
  const int d = (int)h.c.size();
  std::vector<int> n(d), r(d + 1, 1);
  for (int k = 0; k < d; ++k) {
    n[k] = h.c[k].N;
    r[k + 1] = h.c[k].r1;
  }
  std::unique_ptr<tnfem_tt> x(tt_new(ctx, n, r));
  for (int k = 0; k < d; ++k)
    TN_CHECK_CUDA(cudaMemcpyAsync(x->core[k], h.c[k].v.data(), h.c[k].v.size() * sizeof(double),
                                  cudaMemcpyHostToDevice, ctx->stream));
  sync(ctx);
  std::unique_ptr<tnfem_tt> y(tt_round(ctx, x.get(), eps, 1 << 20));
  return download_train(ctx, y.get());
}

tnfem_mpo* build_quad_operator(tnfem_ctx* ctx, const tnfem_grid& g, const tnfem_material& mat, bool mass) {
  HTrain coef;
  {
    std::vector<double> full;
    quad_operator_coefficients(g, mat, mass, full, nullptr);
    std::unique_ptr<tnfem_tt> ct(tt_from_full(ctx, full.data(), quad_modes(g.levels, 4, 9), 1e-14));
    coef = download_train(ctx, ct.get());
  }
  const HTrain B = round_on_device(ctx, quad_stage_axis1(coef), 1e-14);
  tnfem_mpo* raw = upload_mpo(ctx, quad_stage_axis0(B), 2, 2);
  tnfem_mpo* A = nullptr;
  try {
    A = mpo_round(ctx, raw, 1e-14, 1 << 20);
  } catch (...) {
    delete raw;
    throw;
  }
  delete raw;
  return A;
}

// value of a train at one multi-index: product of core slices
__global__ void eval_kernel(int d, const double* const* __restrict__ cores, const int* __restrict__ ranks,
                            const int* __restrict__ modes, const int* __restrict__ idx, int npts,
                            double* __restrict__ out, int rmax) {
  extern __shared__ double sh[];
  double* v = sh;
  double* w = sh + rmax;
  for (int p = blockIdx.x; p < npts; p += gridDim.x) {
    if (threadIdx.x == 0) v[0] = 1.0;
    __syncthreads();
    for (int k = 0; k < d; ++k) {
      const int r0 = ranks[k], r1 = ranks[k + 1], s = idx[(long long)p * d + k];
      const double* c = cores[k] + (long long)s * r1;
      for (int t = threadIdx.x; t < r1; t += blockDim.x) {
        double acc = 0.0;
        for (int a = 0; a < r0; ++a) acc += v[a] * c[(long long)a * modes[k] * r1 + t];
        w[t] = acc;
      }
      __syncthreads();
      for (int t = threadIdx.x; t < r1; t += blockDim.x) v[t] = w[t];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[p] = v[0];
    __syncthreads();
  }
}

// evaluate u at (component, node) pairs given as per-core mode indices
std::vector<double> eval_points(tnfem_ctx* ctx, const tnfem_tt* u, const std::vector<int>& idx, int npts) {
  const int d = u->d;
  std::vector<double> out(npts);
  if (npts == 0) return out;
  DArr<double*> dcores(ctx, d);
  DArr<int> dr(ctx, d + 1), dn(ctx, d), didx(ctx, idx.size());
  DArr<double> dout(ctx, npts);
  int rmax = *std::max_element(u->r.begin(), u->r.end());
  TN_CHECK_CUDA(cudaMemcpyAsync(dcores.p, u->core.data(), d * sizeof(double*), cudaMemcpyHostToDevice, ctx->stream));
  TN_CHECK_CUDA(cudaMemcpyAsync(dr.p, u->r.data(), (d + 1) * sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
  TN_CHECK_CUDA(cudaMemcpyAsync(dn.p, u->n.data(), d * sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
  TN_CHECK_CUDA(cudaMemcpyAsync(didx.p, idx.data(), idx.size() * sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
  int blocks = std::min(npts, 152 * 8);
  eval_kernel<<<blocks, 128, 2 * rmax * sizeof(double), ctx->stream>>>(d, dcores.p, dr.p, dn.p, didx.p, npts, dout.p,
                                                                         rmax);
  count_launch(ctx);
  check_launch(ctx, "eval");
  TN_CHECK_CUDA(cudaMemcpyAsync(out.data(), dout.p, npts * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  sync(ctx);
  return out;
}

// per-core mode indices of (component c, node i_0..i_{D-1}) on the QTT layout
void qtt_index(int D, int L, int c, const int64_t* node, int* out) {
  out[0] = c;
  for (int k = 1; k <= L; ++k) {
    int s = 0;
    for (int dd = 0; dd < D; ++dd) s = s * 2 + (int)((node[dd] >> (L - k)) & 1);
    out[k] = s;
  }
}

int grid_dim_of(const tnfem_tt* u) {
  int m = u->n.size() > 1 ? u->n[1] : 2;
  return m == 8 ? 3 : 2;
}

tnfem_tt* mixed_solve(tnfem_ctx* ctx, const tnfem_mpo* A, const tnfem_tt* f, const tnfem_solve_opts* o,
                      const tnfem_tt* x0, tnfem_solve_info* info, bool& converged, bool has_deadline,
                      std::chrono::steady_clock::time_point deadline, bool& timed_out) {
  // binary32 inner AMEn on A e = f - A u with binary64 source projections, binary64 rounding of u + e
  AmenParams ip;
  ip.tol = std::max(1e-5, std::min(1e-3, o->refine_tol * 1e2));
  ip.rmax = o->rank_cap;
  ip.kick = o->kickrank;
  ip.max_sweeps = std::max(2, std::min(o->max_sweeps, 12));
  ip.local_maxit = o->local_maxit > 0 ? o->local_maxit : 500;
  ip.seed = o->seed;
  ip.precond = o->no_precond == 0;
  ip.local_rtol = o->local_rtol < 0 ? kLocalRtolDefault : o->local_rtol;
  ip.fused_cg = o->cg_engine == 0;
  ip.verbose = getenv("TNFEM_VERBOSE") != nullptr;
  ip.has_deadline = has_deadline;
  ip.deadline = deadline;
  tnfem_tt* u = x0 ? tt_clone(x0) : nullptr;
  const double fnorm = energy_norm(ctx, A, f, nullptr);  // scale reference (any norm works)
  (void)fnorm;
  double est = 1.0;
  int refines = 0;
  converged = false;
  long long iters = 0;
  double flops = 0;
  int sweeps = 0;
  AmenStats st;
  for (int it = 0; it < std::max(1, o->max_refine); ++it) {
    std::vector<AmenSource> src;
    src.push_back(AmenSource{f, false, 1.0});
    if (u) src.push_back(AmenSource{u, true, -1.0});
    ip.seed = o->seed + 7919ull * it;
    tnfem_tt* e = amen_solve(ctx, A, src, ip, nullptr, true, st);
    sweeps += st.sweeps;
    iters += st.local_iters;
    flops += st.flops;
    ++refines;
    if (!u) {
      u = tt_round(ctx, e, o->tol, o->rank_cap);
      delete e;
      est = 1.0;
    } else {
      const double en = energy_norm(ctx, A, e, nullptr);
      tnfem_tt* s = tt_axpy(ctx, u, 1.0, e);
      delete e;
      tnfem_tt* un = tt_round(ctx, s, o->tol, o->rank_cap);
      delete s;
      delete u;
      u = un;
      const double un_e = energy_norm(ctx, A, u, nullptr);
      est = un_e > 0 ? en / un_e : 0.0;
      if (est <= o->refine_tol) {
        converged = true;
        break;
      }
    }
    if (st.timed_out || (has_deadline && std::chrono::steady_clock::now() > deadline)) {
      timed_out = true;
      break;
    }
  }
  if (info) {
    info->sweeps = sweeps;
    info->refines = refines;
    info->local_iters = iters;
    info->flops = flops;
    info->max_res = st.max_res;
    info->max_dx = st.max_dx;
    info->energy_err_est = est;
  }
  return u;
}

}  // namespace

namespace tnfem {

// fused local CG of tnfem_op_local_cg in precision U
template <typename U>
void op_local_cg(tnfem_ctx* ctx, int precond, int r0, int n, int r1, int a0, int a1, const U* PhiL, const U* A,
                 const U* PhiR, const U* g, U* x, double rtol, int maxit, int* iters, int* state) {
  const size_t N = (size_t)r0 * n * r1;
  DArr<U> Ap(ctx, (size_t)a0 * n * n * a1);
  transpose4_mid<U>(ctx, Ap.p, A, a0, n, n, a1);
  DArr<float> P;
  if (precond) {
    TN_REQUIRE(bj_fits(r0, n, r1), "block-Jacobi preconditioner: blocks too large");
    DArr<U> work(ctx, bj_work_elems(r0, n, r1, a0, a1));
    P = DArr<float>(ctx, (size_t)r1 * r0 * n * r0 * n);
    DArr<int> flag(ctx, 1);
    TN_REQUIRE(bj_setup<U>(ctx, r0, n, r1, a0, a1, PhiL, Ap.p, PhiR, P.p, work.p, work.n, flag.p),
               "block-Jacobi preconditioner: a block is not positive definite");
  }
  FusedCg f;
  const FcgPlan pl = f.plan<U>(ctx, r0, n, r1, a0, a1, precond != 0);
  TN_REQUIRE(pl.ok, "fused conjugate gradients: shape outside the kernel's limits");
  const double gn = nrm2<U>(ctx, g, N);
  *iters = f.run<U>(ctx, pl, r0, n, r1, a0, a1, PhiL, Ap.p, PhiR, precond ? P.p : nullptr, g, x,
                    rtol * rtol * gn * gn, maxit, state);
}

}  // namespace tnfem

extern "C" {

tnfem_status tnfem_create(int device, void* stream, tnfem_alloc_fn alloc_fn, tnfem_free_fn free_fn, void* user,
                          tnfem_ctx** out) {
  if (!out) return TNFEM_E_INVALID;
  *out = nullptr;
  auto* ctx = new (std::nothrow) tnfem_ctx();
  if (!ctx) return TNFEM_E_NOMEM;
  tnfem_status st = guard(ctx, [&] {
    TN_CHECK_CUDA(cudaSetDevice(device));
    ctx->device = device;
    ctx->stream = static_cast<cudaStream_t>(stream);
    if (!ctx->stream) {
      // a private stream that synchronises with the legacy default stream like NULL does, and
      // that (unlike NULL) can be captured into CUDA graphs
      TN_CHECK_CUDA(cudaStreamCreate(&ctx->stream));
      ctx->own_stream = true;
    }
    ctx->alloc_fn = alloc_fn;
    ctx->free_fn = free_fn;
    ctx->user = user;
    ctx->scratch = static_cast<double*>(dalloc(ctx, kScratchDoubles * sizeof(double)));
    TN_CHECK_CUDA(cudaMemsetAsync(ctx->scratch, 0, kScratchDoubles * sizeof(double), ctx->stream));
    TN_CHECK_CUDA(cudaStreamSynchronize(ctx->stream));
    TN_CHECK_CUDA(cudaMallocHost(&ctx->host_pinned, 4096));
  });
  if (st != TNFEM_OK) {
    if (ctx->scratch) dfree(ctx, ctx->scratch);
    if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
    return st;
  }
  *out = ctx;
  return TNFEM_OK;
}

void tnfem_destroy(tnfem_ctx* ctx) {
  if (!ctx) return;
  prof_release(ctx);
  if (ctx->scratch) dfree(ctx, ctx->scratch);
  if (ctx->host_pinned) cudaFreeHost(ctx->host_pinned);
  if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
}

const char* tnfem_last_error(const tnfem_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

tnfem_status tnfem_set_stream(tnfem_ctx* ctx, void* stream) {
  if (!ctx) return TNFEM_E_INVALID;
  if (!stream) {
    if (!ctx->own_stream) {
      if (cudaStreamCreate(&ctx->stream) != cudaSuccess) {
        cudaGetLastError();
        ctx->err = "cudaStreamCreate failed";
        return TNFEM_E_CUDA;
      }
      ctx->own_stream = true;
    }
    return TNFEM_OK;
  }
  if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
  ctx->own_stream = false;
  ctx->stream = static_cast<cudaStream_t>(stream);
  return TNFEM_OK;
}

long long tnfem_kernel_launches(const tnfem_ctx* ctx) { return ctx ? ctx->launches : 0; }

tnfem_status tnfem_set_hbm_budget(tnfem_ctx* ctx, size_t bytes) {
  if (!ctx) return TNFEM_E_INVALID;
  ctx->mem_budget = bytes;
  return TNFEM_OK;
}

tnfem_status tnfem_memory_stats(tnfem_ctx* ctx, size_t* in_use, size_t* peak, int reset_peak) {
  if (!ctx) return TNFEM_E_INVALID;
  if (reset_peak) ctx->mem_peak = ctx->mem_in_use;
  if (in_use) *in_use = ctx->mem_in_use;
  if (peak) *peak = ctx->mem_peak;
  return TNFEM_OK;
}

tnfem_status tnfem_build_stiffness(tnfem_ctx* ctx, const tnfem_grid* grid, const tnfem_material* mat,
                                   tnfem_mpo** out) {
  if (!ctx || !out) return TNFEM_E_INVALID;
  *out = nullptr;
  return guard(ctx, [&] {
    check_grid(grid);
    check_material(mat);
    if (grid->mapped == 2) {
      *out = build_quad_operator(ctx, *grid, *mat, false);
      return;
    }
    double s = 0;
    HTrain h = stiffness_train(*grid, *mat, &s);
    tnfem_mpo* raw = upload_mpo(ctx, h, grid->dim, grid->dim);
    tnfem_mpo* A = nullptr;
    try {
      A = mpo_round(ctx, raw, 1e-14, 1 << 20);
    } catch (...) {
      delete raw;
      throw;
    }
    delete raw;
    *out = A;
  });
}

namespace {

tnfem_mpo* mass_operator(tnfem_ctx* ctx, const tnfem_grid& g) {
  if (g.mapped == 2) {
    const tnfem_material any{{1.0, 1.0}, 1e300, 0.3};
    return build_quad_operator(ctx, g, any, true);
  }
  std::unique_ptr<tnfem_mpo> raw(upload_mpo(ctx, mass_train(g), g.dim, g.dim));
  return mpo_round(ctx, raw.get(), 1e-14, 1 << 20);
}

// f += P (M f0) for each nodal-train load (Section 5.3), on the device
tnfem_tt* add_nodal_loads(tnfem_ctx* ctx, const tnfem_grid& g, const std::vector<const tnfem_tt*>& nodal,
                          tnfem_tt* f_in) {
  std::unique_ptr<tnfem_tt> f(f_in);
  std::unique_ptr<tnfem_mpo> M(mass_operator(ctx, g));
  std::unique_ptr<tnfem_mpo> P(upload_mpo(ctx, projector_train(g), g.dim, g.dim));
  for (const tnfem_tt* f0 : nodal) {
    std::unique_ptr<tnfem_tt> mf(mpo_apply(ctx, M.get(), f0));
    std::unique_ptr<tnfem_tt> mfr(tt_round(ctx, mf.get(), 1e-14, 1 << 20));
    std::unique_ptr<tnfem_tt> pmf(mpo_apply(ctx, P.get(), mfr.get()));
    std::unique_ptr<tnfem_tt> sum(tt_axpy(ctx, f.get(), 1.0, pmf.get()));
    f.reset(tt_round(ctx, sum.get(), 1e-14, 1 << 20));
  }
  return f.release();
}

}  // namespace

tnfem_status tnfem_build_mass(tnfem_ctx* ctx, const tnfem_grid* grid, tnfem_mpo** out) {
  if (!ctx || !out) return TNFEM_E_INVALID;
  *out = nullptr;
  return guard(ctx, [&] {
    check_grid(grid);
    *out = mass_operator(ctx, *grid);
  });
}

tnfem_status tnfem_build_load(tnfem_ctx* ctx, const tnfem_grid* grid, const tnfem_material* mat,
                              const tnfem_load* loads, int n_loads, tnfem_tt** out) {
  if (!ctx || !out) return TNFEM_E_INVALID;
  *out = nullptr;
  return guard(ctx, [&] {
    check_grid(grid);
    check_material(mat);
    TN_REQUIRE(n_loads >= 0 && (n_loads == 0 || loads), "loads array");
    // nodal-train loads go through the mass operator on the device; the rest is built on the host
    std::vector<tnfem_load> analytic;
    std::vector<const tnfem_tt*> nodal;
    for (int i = 0; i < n_loads; ++i) {
      if (loads[i].kind != TNFEM_LOAD_NODAL_TT) {
        analytic.push_back(loads[i]);
        continue;
      }
      const tnfem_tt* f0 = loads[i].nodal;
      TN_REQUIRE(f0, "nodal-train load without a train");
      TN_REQUIRE(f0->ctx == ctx, "nodal-train load: the train belongs to another context");
      TN_REQUIRE(f0->d == grid->levels + 1 && f0->n[0] == grid->dim, "nodal-train load does not match the grid");
      for (int k = 1; k < f0->d; ++k) TN_REQUIRE(f0->n[k] == (1 << grid->dim), "nodal-train load does not match the grid");
      nodal.push_back(f0);
    }
    const int na = (int)analytic.size();
    tnfem_tt* f = nullptr;
    if (grid->mapped == 2) {
      std::vector<double> full;
      quad_load_values(*grid, *mat, analytic.data(), na, full);
      f = tt_from_full(ctx, full.data(), quad_modes(grid->levels, 2, 0), 1e-14);
    } else {
      std::unique_ptr<tnfem_tt> raw(upload_tt(ctx, load_train(*grid, *mat, analytic.data(), na), grid->dim, grid->dim));
      f = tt_round(ctx, raw.get(), 1e-14, 1 << 20);
    }
    *out = nodal.empty() ? f : add_nodal_loads(ctx, *grid, nodal, f);
  });
}

tnfem_status tnfem_solve(tnfem_ctx* ctx, const tnfem_mpo* A, const tnfem_tt* f, const tnfem_solve_opts* opts,
                         const tnfem_tt* x0, tnfem_tt** u, tnfem_solve_info* info) {
  if (!ctx || !u) return TNFEM_E_INVALID;
  *u = nullptr;
  bool converged = false, timed_out = false;
  tnfem_status st = guard(ctx, [&] {
    TN_REQUIRE(A && f && opts, "null operator, load or options");
    TN_REQUIRE(A->d == f->d, "operator and load have different core counts");
    for (int k = 0; k < A->d; ++k) TN_REQUIRE(A->n[k] == f->n[k], "operator and load modes differ");
    if (x0) {
      TN_REQUIRE(x0->d == f->d, "x0 core count");
      for (int k = 0; k < A->d; ++k) TN_REQUIRE(x0->n[k] == f->n[k], "x0 modes differ");
    }
    TN_REQUIRE(opts->tol > 0 && opts->rank_cap >= 1 && opts->kickrank >= 0 && opts->max_sweeps >= 1,
               "solve options out of range");
    TN_REQUIRE(opts->precision == TNFEM_FP64 || opts->precision == TNFEM_MIXED ||
                   opts->precision == TNFEM_MIXED_LOCAL || opts->precision == TNFEM_MIXED_TF32,
               "precision");
    TN_REQUIRE(opts->timeout_us >= 0, "timeout_us must be >= 0");
    sync(ctx);
    EngineScope es(ctx, (opts->tensor_cores || opts->precision == TNFEM_MIXED_TF32) ? 1 : 0);
    // Mixed paths at a loose tolerance run their large binary64 contractions in double-binary32
    // arithmetic (binary32 FMAs issue at 64x the binary64 rate on this part): its ~2^-47 noise,
    // amplified by the local systems' conditioning, stays orders of magnitude below a tolerance of
    // 1e-7 or looser, whereas at 1e-9 it stalled the stopping rule (measured).  A contraction whose
    // values leave the binary32 range sets a flag, and the solve is then repeated in binary64.
    const bool df_route = (opts->precision == TNFEM_MIXED_LOCAL || opts->precision == TNFEM_MIXED_TF32) &&
                          opts->tol >= kDfTolMin;
    DfScope dfs(ctx, df_route);
    if (df_route) TN_CHECK_CUDA(cudaMemsetAsync(df_overflow_flag(ctx), 0, sizeof(int), ctx->stream));
    auto t0 = std::chrono::steady_clock::now();
    const bool has_deadline = opts->timeout_us > 0;
    const auto deadline = t0 + std::chrono::microseconds(opts->timeout_us);
    tnfem_tt* res = nullptr;
    if (info) memset(info, 0, sizeof(*info));
    if (opts->precision == TNFEM_FP64 || opts->precision == TNFEM_MIXED_LOCAL ||
        opts->precision == TNFEM_MIXED_TF32) {
      AmenParams p;
      p.tol = opts->tol;
      p.rmax = opts->rank_cap;
      p.kick = opts->kickrank;
      p.max_sweeps = opts->max_sweeps;
      p.local_maxit = opts->local_maxit > 0 ? opts->local_maxit : 500;
      p.seed = opts->seed;
      p.precond = opts->no_precond == 0;
      p.local_rtol = opts->local_rtol < 0 ? kLocalRtolDefault : opts->local_rtol;
      p.fused_cg = opts->cg_engine == 0;
      p.local_mixed = opts->precision != TNFEM_FP64;
      p.verbose = getenv("TNFEM_VERBOSE") != nullptr;
      p.has_deadline = has_deadline;
      p.deadline = deadline;
      AmenStats s;
      res = amen_solve(ctx, A, {AmenSource{f, false, 1.0}}, p, x0, false, s);
      if (df_route) {
        int ovf = 0;
        TN_CHECK_CUDA(cudaMemcpyAsync(&ovf, df_overflow_flag(ctx), sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
        sync(ctx);
        if (ovf) {  // a value outside the binary32 range: the whole solve again in binary64
          delete res;
          res = nullptr;
          ctx->df64 = false;
          s = AmenStats();
          res = amen_solve(ctx, A, {AmenSource{f, false, 1.0}}, p, x0, false, s);
        }
      }
      converged = s.converged;
      timed_out = s.timed_out;
      if (info) {
        info->sweeps = s.sweeps;
        info->local_iters = s.local_iters;
        info->max_res = s.max_res;
        info->max_dx = s.max_dx;
        info->flops = s.flops;
        for (int i = 0; i < 7; ++i) info->t_phase_ms[i] = s.phase_ms[i];
      }
    } else {
      res = mixed_solve(ctx, A, f, opts, x0, info, converged, has_deadline, deadline, timed_out);
    }
    sync(ctx);
    auto t1 = std::chrono::steady_clock::now();
    if (info) {
      info->t_solve_ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
      info->max_rank = *std::max_element(res->r.begin(), res->r.end());
      info->bytes_A = mpo_bytes(A);
      info->bytes_f = tt_bytes(f);
      info->bytes_u = tt_bytes(res);
      info->converged = converged ? 1 : 0;
    }
    *u = res;
  });
  if (st == TNFEM_OK && timed_out) {
    ctx->err = "solve stopped at its timeout_us";
    return TNFEM_E_TIMEOUT;
  }
  if (st == TNFEM_OK && !converged) {
    ctx->err = "solve stopped before reaching the tolerance";
    return TNFEM_E_NOT_CONVERGED;
  }
  return st;
}

tnfem_status tnfem_eval_displacement(tnfem_ctx* ctx, const tnfem_tt* u, const int64_t* nodes, int64_t n, double* out) {
  if (!ctx) return TNFEM_E_INVALID;
  return guard(ctx, [&] {
    TN_REQUIRE(u && (n == 0 || (nodes && out)), "null argument");
    TN_REQUIRE(n >= 0 && n < (1ll << 31), "point count out of range");
    const int D = u->n[0], L = u->d - 1;
    TN_REQUIRE(D == 2 || D == 3, "train is not on the elasticity layout");
    TN_REQUIRE(L >= 1 && u->n[1] == (1 << D), "train is not on the elasticity layout");
    const int64_t N = 1ll << L;
    std::vector<int> idx((size_t)n * D * u->d);
    for (int64_t p = 0; p < n; ++p) {
      for (int d = 0; d < D; ++d) TN_REQUIRE(nodes[p * D + d] >= 0 && nodes[p * D + d] < N, "node index out of range");
      for (int c = 0; c < D; ++c) qtt_index(D, L, c, nodes + p * D, &idx[((size_t)p * D + c) * u->d]);
    }
    std::vector<double> v = eval_points(ctx, u, idx, (int)(n * D));
    memcpy(out, v.data(), v.size() * sizeof(double));
  });
}

tnfem_status tnfem_eval_strain(tnfem_ctx* ctx, const tnfem_tt* u, const tnfem_grid* grid, const int64_t* elems,
                               int64_t n, double* out) {
  if (!ctx) return TNFEM_E_INVALID;
  return guard(ctx, [&] {
    check_grid(grid);
    TN_REQUIRE(u && (n == 0 || (elems && out)), "null argument");
    const int D = grid->dim, L = grid->levels;
    TN_REQUIRE(u->d == L + 1 && u->n[0] == D, "train does not match the grid");
    const int64_t N = 1ll << L;
    const int nc = 1 << D;
    std::vector<int64_t> nodes((size_t)n * nc * D);
    for (int64_t p = 0; p < n; ++p)
      for (int a = 0; a < nc; ++a)
        for (int d = 0; d < D; ++d) {
          int64_t e = elems[p * D + d];
          TN_REQUIRE(e >= 0 && e < N - 1, "element index out of range");
          nodes[((size_t)p * nc + a) * D + d] = e + ((a >> (D - 1 - d)) & 1);
        }
    std::vector<double> vals((size_t)n * nc * D);
    if (n) {
      std::vector<int> idx((size_t)n * nc * D * u->d);
      for (int64_t q = 0; q < n * nc; ++q)
        for (int c = 0; c < D; ++c) qtt_index(D, L, c, &nodes[(size_t)q * D], &idx[((size_t)q * D + c) * u->d]);
      vals = eval_points(ctx, u, idx, (int)(n * nc * D));
    }
    // gradient at the element centre: d N_a / d x_d = xi_{a,d} 2^{1-D} / h_d on a box; on a mapped
    // grid the same on the unit box (h = 1 / (N - 1)), then d/dx_e = sum_d Jinv[d][e] d/dxi_d
    std::vector<double> h(D);
    for (int d = 0; d < D; ++d) h[d] = grid->mapped ? 1.0 / (N - 1) : (grid->hi[d] - grid->lo[d]) / (N - 1);
    double Jinv[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    if (grid->mapped == 1) grid_affine_inverse(*grid, Jinv, nullptr);
    const int ns = D == 2 ? 3 : 6;
    for (int64_t p = 0; p < n; ++p) {
      double gr[3][3] = {{0}};
      for (int a = 0; a < nc; ++a)
        for (int c = 0; c < D; ++c) {
          double v = vals[((size_t)p * nc + a) * D + c];
          for (int d = 0; d < D; ++d) {
            double xi = ((a >> (D - 1 - d)) & 1) ? 1.0 : -1.0;
            gr[c][d] += v * xi * std::pow(2.0, 1 - D) / h[d];
          }
        }
      if (grid->mapped == 2) {
        // the element's own Jacobian, frozen at its centre as in the assembly
        double Ji[2][2];
        quad_element_inverse(*grid, elems[p * D], elems[p * D + 1], Ji);
        for (int i = 0; i < 2; ++i)
          for (int j = 0; j < 2; ++j) Jinv[i][j] = Ji[i][j];
      }
      if (grid->mapped) {
        double gp[3][3] = {{0}};
        for (int c = 0; c < D; ++c)
          for (int e = 0; e < D; ++e)
            for (int d = 0; d < D; ++d) gp[c][e] += Jinv[d][e] * gr[c][d];
        for (int c = 0; c < D; ++c)
          for (int e = 0; e < D; ++e) gr[c][e] = gp[c][e];
      }
      double* o = out + p * ns;
      if (D == 2) {
        o[0] = gr[0][0];
        o[1] = gr[1][1];
        o[2] = 0.5 * (gr[0][1] + gr[1][0]);
      } else {
        o[0] = gr[0][0];
        o[1] = gr[1][1];
        o[2] = gr[2][2];
        o[3] = 0.5 * (gr[1][2] + gr[2][1]);
        o[4] = 0.5 * (gr[0][2] + gr[2][0]);
        o[5] = 0.5 * (gr[0][1] + gr[1][0]);
      }
    }
  });
}

tnfem_status tnfem_energy_norm(tnfem_ctx* ctx, const tnfem_mpo* A, const tnfem_tt* u, const tnfem_tt* v, double* out) {
  if (!ctx) return TNFEM_E_INVALID;
  return guard(ctx, [&] {
    TN_REQUIRE(A && u && out, "null argument");
    TN_REQUIRE(A->d == u->d && (!v || v->d == u->d), "core count mismatch");
    *out = energy_norm(ctx, A, u, v);
  });
}

tnfem_status tnfem_tt_dot(tnfem_ctx* ctx, const tnfem_tt* x, const tnfem_tt* y, double* out) {
  if (!ctx) return TNFEM_E_INVALID;
  return guard(ctx, [&] {
    TN_REQUIRE(x && y && out, "null argument");
    *out = tt_dot(ctx, x, y);
  });
}

tnfem_status tnfem_tt_norm(tnfem_ctx* ctx, const tnfem_tt* x, double* out) {
  if (!ctx) return TNFEM_E_INVALID;
  return guard(ctx, [&] {
    TN_REQUIRE(x && out, "null argument");
    *out = tt_norm(ctx, x);
  });
}

namespace {
double residual_norm_train(tnfem_ctx* ctx, const tnfem_mpo* A, const tnfem_tt* f, const tnfem_tt* u) {
  tnfem_tt* Au = mpo_apply(ctx, A, u);
  tnfem_tt* r = nullptr;
  double out = 0;
  try {
    r = tt_axpy(ctx, f, -1.0, Au);
    const double rn = tt_norm(ctx, r);
    const double fn = tt_norm(ctx, f);
    out = fn > 0 ? rn / fn : rn;
  } catch (...) {
    tnfem_free_tt(Au);
    tnfem_free_tt(r);
    throw;
  }
  tnfem_free_tt(Au);
  tnfem_free_tt(r);
  return out;
}

void check_residual_args(const tnfem_mpo* A, const tnfem_tt* f, const tnfem_tt* u, const double* out) {
  TN_REQUIRE(A && f && u && out, "null argument");
  TN_REQUIRE(A->d == u->d && f->d == u->d, "operator, load and solution have different core counts");
  for (int k = 0; k < u->d; ++k) TN_REQUIRE(A->n[k] == u->n[k] && f->n[k] == u->n[k], "modes differ");
}
}  // namespace

tnfem_status tnfem_residual_norm(tnfem_ctx* ctx, const tnfem_mpo* A, const tnfem_tt* f, const tnfem_tt* u,
                                 double* out) {
  if (!ctx) return TNFEM_E_INVALID;
  return guard(ctx, [&] {
    check_residual_args(A, f, u, out);
    const size_t N = dense_elems(u);
    size_t rk = 1;
    for (int k = 0; k <= u->d; ++k) rk = std::max({rk, (size_t)A->a[k], (size_t)u->r[k], (size_t)f->r[k]});
    if (N <= (1ull << 22) && N * rk <= (1ull << 28)) *out = residual_norm_dense(ctx, A, f, u);
    else *out = residual_norm_train(ctx, A, f, u);
  });
}

tnfem_status tnfem_residual_norm_train(tnfem_ctx* ctx, const tnfem_mpo* A, const tnfem_tt* f, const tnfem_tt* u,
                                       double* out) {
  if (!ctx) return TNFEM_E_INVALID;
  return guard(ctx, [&] {
    check_residual_args(A, f, u, out);
    *out = residual_norm_train(ctx, A, f, u);
  });
}

tnfem_status tnfem_tt_round(tnfem_ctx* ctx, const tnfem_tt* x, double eps, int rmax, tnfem_tt** out) {
  if (!ctx || !out) return TNFEM_E_INVALID;
  *out = nullptr;
  return guard(ctx, [&] {
    TN_REQUIRE(x && eps >= 0 && rmax >= 1, "bad arguments");
    *out = tt_round(ctx, x, eps, rmax);
  });
}

tnfem_status tnfem_tt_axpy(tnfem_ctx* ctx, const tnfem_tt* x, double beta, const tnfem_tt* y, tnfem_tt** out) {
  if (!ctx || !out) return TNFEM_E_INVALID;
  *out = nullptr;
  return guard(ctx, [&] {
    TN_REQUIRE(x && y, "null argument");
    *out = tt_axpy(ctx, x, beta, y);
  });
}

tnfem_status tnfem_mpo_apply(tnfem_ctx* ctx, const tnfem_mpo* A, const tnfem_tt* x, tnfem_tt** out) {
  if (!ctx || !out) return TNFEM_E_INVALID;
  *out = nullptr;
  return guard(ctx, [&] {
    TN_REQUIRE(A && x, "null argument");
    *out = mpo_apply(ctx, A, x);
  });
}

static tnfem_status export_cores(tnfem_ctx* ctx, int d, const std::vector<int>& r, const std::vector<int>& n,
                                 const std::vector<double*>& core, int mult, int* ncores, int* ranks, int* modes,
                                 double* cores) {
  return guard(ctx, [&] {
    TN_REQUIRE(ncores, "ncores is null");
    *ncores = d;
    if (ranks) for (int k = 0; k <= d; ++k) ranks[k] = r[k];
    if (modes) for (int k = 0; k < d; ++k) modes[k] = n[k];
    if (cores) {
      size_t off = 0;
      for (int k = 0; k < d; ++k) {
        size_t sz = (size_t)r[k] * n[k] * (mult ? n[k] : 1) * r[k + 1];
        TN_CHECK_CUDA(cudaMemcpyAsync(cores + off, core[k], sz * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
        off += sz;
      }
      sync(ctx);
    }
  });
}

tnfem_status tnfem_tt_export(tnfem_ctx* ctx, const tnfem_tt* x, int* ncores, int* ranks, int* modes, double* cores) {
  if (!ctx || !x) return TNFEM_E_INVALID;
  return export_cores(ctx, x->d, x->r, x->n, x->core, 0, ncores, ranks, modes, cores);
}

tnfem_status tnfem_mpo_export(tnfem_ctx* ctx, const tnfem_mpo* A, int* ncores, int* ranks, int* modes, double* cores) {
  if (!ctx || !A) return TNFEM_E_INVALID;
  return export_cores(ctx, A->d, A->a, A->n, A->core, 1, ncores, ranks, modes, cores);
}

tnfem_status tnfem_tt_import(tnfem_ctx* ctx, int ncores, const int* ranks, const int* modes, const double* cores,
                             tnfem_tt** out) {
  if (!ctx || !out) return TNFEM_E_INVALID;
  *out = nullptr;
  return guard(ctx, [&] {
    TN_REQUIRE(ncores >= 1 && ncores <= 63 && ranks && modes && cores, "bad import arguments");
    TN_REQUIRE(ranks[0] == 1 && ranks[ncores] == 1, "boundary ranks must be 1");
    std::vector<int> n(modes, modes + ncores), r(ranks, ranks + ncores + 1);
    for (int k = 0; k < ncores; ++k) TN_REQUIRE(n[k] >= 1 && r[k + 1] >= 1, "modes and ranks must be positive");
    tnfem_tt* x = tt_new(ctx, n, r);
    size_t off = 0;
    try {
      for (int k = 0; k < ncores; ++k) {
        size_t sz = (size_t)r[k] * n[k] * r[k + 1];
        TN_CHECK_CUDA(cudaMemcpyAsync(x->core[k], cores + off, sz * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
        off += sz;
      }
      sync(ctx);
    } catch (...) {
      delete x;
      throw;
    }
    *out = x;
  });
}

tnfem_status tnfem_mpo_import(tnfem_ctx* ctx, int ncores, const int* ranks, const int* modes, const double* cores,
                              tnfem_mpo** out) {
  if (!ctx || !out) return TNFEM_E_INVALID;
  *out = nullptr;
  return guard(ctx, [&] {
    TN_REQUIRE(ncores >= 1 && ncores <= 63 && ranks && modes && cores, "bad import arguments");
    TN_REQUIRE(ranks[0] == 1 && ranks[ncores] == 1, "boundary ranks must be 1");
    std::vector<int> n(modes, modes + ncores), a(ranks, ranks + ncores + 1);
    for (int k = 0; k < ncores; ++k) TN_REQUIRE(n[k] >= 1 && a[k + 1] >= 1, "modes and ranks must be positive");
    tnfem_mpo* A = mpo_new(ctx, n, a);
    size_t off = 0;
    try {
      for (int k = 0; k < ncores; ++k) {
        size_t sz = (size_t)a[k] * n[k] * n[k] * a[k + 1];
        TN_CHECK_CUDA(cudaMemcpyAsync(A->core[k], cores + off, sz * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
        off += sz;
      }
      sync(ctx);
    } catch (...) {
      delete A;
      throw;
    }
    *out = A;
  });
}

static tnfem_status host_export(const HTrain& h, int dim, bool op, int* ncores, int* ranks, int* modes,
                                double* cores) {
  TN_REQUIRE(ncores, "ncores is null");
  const int d = (int)h.c.size();
  *ncores = d;
  if (ranks) {
    ranks[0] = 1;
    for (int k = 0; k < d; ++k) ranks[k + 1] = h.c[k].r1;
  }
  if (modes)
    for (int k = 0; k < d; ++k) modes[k] = (k == 0) ? dim : (1 << dim);
  if (cores) {
    size_t off = 0;
    for (int k = 0; k < d; ++k) {
      memcpy(cores + off, h.c[k].v.data(), h.c[k].v.size() * sizeof(double));
      off += h.c[k].v.size();
    }
  }
  (void)op;
  return TNFEM_OK;
}

tnfem_status tnfem_host_stiffness(const tnfem_grid* grid, const tnfem_material* mat, int* ncores, int* ranks,
                                  int* modes, double* cores, double* shift) {
  return guard(nullptr, [&] {
    check_grid(grid);
    check_material(mat);
    double s = 0;
    HTrain h = stiffness_train(*grid, *mat, &s);
    if (shift) *shift = s;
    host_export(h, grid->dim, true, ncores, ranks, modes, cores);
  });
}

tnfem_status tnfem_host_mass(const tnfem_grid* grid, int* ncores, int* ranks, int* modes, double* cores) {
  return guard(nullptr, [&] {
    check_grid(grid);
    HTrain h = mass_train(*grid);
    host_export(h, grid->dim, true, ncores, ranks, modes, cores);
  });
}

tnfem_status tnfem_host_load(const tnfem_grid* grid, const tnfem_material* mat, const tnfem_load* loads, int n_loads,
                             int* ncores, int* ranks, int* modes, double* cores) {
  return guard(nullptr, [&] {
    check_grid(grid);
    check_material(mat);
    TN_REQUIRE(n_loads >= 0 && (n_loads == 0 || loads), "loads array");
    HTrain h = load_train(*grid, *mat, loads, n_loads);
    host_export(h, grid->dim, false, ncores, ranks, modes, cores);
  });
}

void tnfem_free_tt(tnfem_tt* x) { delete x; }
void tnfem_free_mpo(tnfem_mpo* A) { delete A; }

tnfem_status tnfem_op_local_matvec(tnfem_ctx* ctx, int r0, int n, int r1, int a0, int a1, const double* PhiL,
                                   const double* A, const double* PhiR, const double* x, double* y) {
  if (!ctx) return TNFEM_E_INVALID;
  return guard(ctx, [&] {
    TN_REQUIRE(PhiL && A && PhiR && x && y, "null pointer");
    TN_REQUIRE(r0 >= 1 && r1 >= 1 && n >= 1 && a0 >= 1 && a1 >= 1, "sizes must be positive");
    DArr<double> Ap(ctx, (size_t)a0 * n * n * a1);
    transpose4_mid<double>(ctx, Ap.p, A, a0, n, n, a1);
    DArr<double> ws(ctx, local_ws_elems(r0, n, r1, a0, a1));
    local_matvec<double>(ctx, r0, n, r1, a0, a1, PhiL, Ap.p, PhiR, x, y, ws.p, ws.n);
    sync(ctx);
  });
}

tnfem_status tnfem_op_local_cg(tnfem_ctx* ctx, int precision, int precond, int r0, int n, int r1, int a0, int a1,
                               const void* PhiL, const void* A, const void* PhiR, const void* g, void* x,
                               double rtol, int maxit, int* iters, int* state) {
  if (!ctx) return TNFEM_E_INVALID;
  return guard(ctx, [&] {
    TN_REQUIRE(PhiL && A && PhiR && g && x && iters && state, "null pointer");
    TN_REQUIRE(r0 >= 1 && r1 >= 1 && n >= 1 && a0 >= 1 && a1 >= 1, "sizes must be positive");
    TN_REQUIRE(n <= 8, "mode size above 8");
    TN_REQUIRE(maxit >= 0 && rtol >= 0.0, "maxit and rtol must be non-negative");
    if (precision == TNFEM_FP64)
      tnfem::op_local_cg<double>(ctx, precond, r0, n, r1, a0, a1, (const double*)PhiL, (const double*)A,
                          (const double*)PhiR, (const double*)g, (double*)x, rtol, maxit, iters, state);
    else
      tnfem::op_local_cg<float>(ctx, precond, r0, n, r1, a0, a1, (const float*)PhiL, (const float*)A, (const float*)PhiR,
                         (const float*)g, (float*)x, rtol, maxit, iters, state);
    sync(ctx);
  });
}

tnfem_status tnfem_op_gemm_f64(tnfem_ctx* ctx, int engine, int M, int N, int K, int batch, long long sAm,
                               long long sAk, long long sAb, long long sBk, long long sBn, long long sBb,
                               long long sCm, long long sCn, long long sCb, double alpha, const double* A,
                               const double* B, double beta, double* C) {
  if (!ctx) return TNFEM_E_INVALID;
  return guard(ctx, [&] {
    TN_REQUIRE(A && B && C, "null pointer");
    TN_REQUIRE(engine == 0 || engine == 1, "engine must be 0 (binary64) or 1 (double-binary32)");
    TN_REQUIRE(M >= 1 && N >= 1 && K >= 1 && batch >= 1, "sizes must be positive");
    DfScope dfs(ctx, engine == 1);
    GemmDesc g{M, N, K, batch, sAm, sAk, sAb, sBk, sBn, sBb, sCm, sCn, sCb};
    const size_t work = (size_t)64 * batch * M * N;
    DArr<double> w(ctx, std::min<size_t>(work, (size_t)1 << 25));
    TN_CHECK_CUDA(cudaMemsetAsync(df_overflow_flag(ctx), 0, sizeof(int), ctx->stream));
    gemm<double>(ctx, g, alpha, A, B, beta, C, w.p, w.n);
    int ovf = 0;
    TN_CHECK_CUDA(cudaMemcpyAsync(&ovf, df_overflow_flag(ctx), sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    sync(ctx);
    TN_REQUIRE(ovf == 0, "double-binary32 GEMM: a value outside the binary32 range");
  });
}

tnfem_status tnfem_op_gemm_f32(tnfem_ctx* ctx, int engine, int M, int N, int K, int batch, long long sAm,
                               long long sAk, long long sAb, long long sBk, long long sBn, long long sBb,
                               long long sCm, long long sCn, long long sCb, float alpha, const float* A,
                               const float* B, float beta, float* C) {
  if (!ctx) return TNFEM_E_INVALID;
  return guard(ctx, [&] {
    TN_REQUIRE(A && B && C, "null pointer");
    TN_REQUIRE(engine == 0 || engine == 1, "engine must be 0 (CUDA cores) or 1 (tensor cores)");
    TN_REQUIRE(M >= 1 && N >= 1 && K >= 1 && batch >= 1, "sizes must be positive");
    EngineScope es(ctx, engine);
    GemmDesc g{M, N, K, batch, sAm, sAk, sAb, sBk, sBn, sBb, sCm, sCn, sCb};
    const size_t work = (size_t)64 * batch * M * N;
    DArr<float> w(ctx, std::min<size_t>(work, (size_t)1 << 26));
    gemm<float>(ctx, g, alpha, A, B, beta, C, w.p, w.n);
    sync(ctx);
  });
}

tnfem_status tnfem_op_local_matvec_f32(tnfem_ctx* ctx, int engine, int r0, int n, int r1, int a0, int a1,
                                       const float* PhiL, const float* A, const float* PhiR, const float* x,
                                       float* y) {
  if (!ctx) return TNFEM_E_INVALID;
  return guard(ctx, [&] {
    TN_REQUIRE(PhiL && A && PhiR && x && y, "null pointer");
    TN_REQUIRE(engine >= 0 && engine <= 2, "engine must be 0 (CUDA cores), 1 or 2 (tensor cores)");
    TN_REQUIRE(r0 >= 1 && r1 >= 1 && n >= 1 && a0 >= 1 && a1 >= 1, "sizes must be positive");
    EngineScope es(ctx, engine == 0 ? 0 : 1);
    DArr<float> Ap(ctx, (size_t)a0 * n * n * a1);
    transpose4_mid<float>(ctx, Ap.p, A, a0, n, n, a1);
    if (engine == 2) {
      TcMatvec mv;
      mv.plan(ctx, r0, n, r1, a0, a1);
      mv.prepare(ctx, PhiL, Ap.p, PhiR);
      mv.apply(ctx, x, y, nullptr);
      sync(ctx);
      TN_REQUIRE(tc_gemm_error(ctx) == 0, "tensor-core kernel: bounded wait expired");
      return;
    }
    DArr<float> ws(ctx, local_ws_elems(r0, n, r1, a0, a1));
    local_matvec<float>(ctx, r0, n, r1, a0, a1, PhiL, Ap.p, PhiR, x, y, ws.p, ws.n);
    sync(ctx);
  });
}

tnfem_status tnfem_op_env_left(tnfem_ctx* ctx, int ry0, int ry1, int rx0, int rx1, int n, int a0, int a1,
                               const double* Phi, const double* y, const double* A, const double* x, double* out) {
  if (!ctx) return TNFEM_E_INVALID;
  return guard(ctx, [&] {
    TN_REQUIRE(Phi && y && A && x && out, "null pointer");
    TN_REQUIRE(ry0 >= 1 && ry1 >= 1 && rx0 >= 1 && rx1 >= 1 && n >= 1 && a0 >= 1 && a1 >= 1, "sizes must be positive");
    DArr<double> Ap(ctx, (size_t)a0 * n * n * a1);
    transpose4_mid<double>(ctx, Ap.p, A, a0, n, n, a1);
    int rr = std::max(std::max(ry0, ry1), std::max(rx0, rx1));
    DArr<double> ws(ctx, local_ws_elems(rr, n, rr, a0, a1));
    env_left<double>(ctx, ry0, ry1, rx0, rx1, n, a0, a1, Phi, y, Ap.p, x, out, ws.p, ws.n);
    sync(ctx);
  });
}

tnfem_status tnfem_op_qr(tnfem_ctx* ctx, int m, int n, const double* Ain, double* Q, double* R) {
  if (!ctx) return TNFEM_E_INVALID;
  return guard(ctx, [&] {
    TN_REQUIRE(Ain && Q && R && m >= 1 && n >= 1, "bad arguments");
    DArr<double> A(ctx, (size_t)m * n), w(ctx, qr_work_elems(m, n));
    copy<double>(ctx, A.p, Ain, (size_t)m * n);
    qr<double>(ctx, m, n, A.p, Q, R, w.p);
    sync(ctx);
  });
}

tnfem_status tnfem_op_qr_ext(tnfem_ctx* ctx, int m, int rk, int w, double* A, double* Q, double* R) {
  if (!ctx) return TNFEM_E_INVALID;
  return guard(ctx, [&] {
    TN_REQUIRE(A && Q && R, "null pointer");
    TN_REQUIRE(rk >= 1 && w >= 1 && m >= rk + w, "needs rk >= 1, w >= 1 and m >= rk + w");
    DArr<double> work(ctx, qr_ext_work_elems(m, rk, w) + qr_work_elems(m, rk + w));
    qr_ext<double>(ctx, m, rk, w, A, Q, R, work.p, work.n);
    sync(ctx);
  });
}

tnfem_status tnfem_op_svd(tnfem_ctx* ctx, int m, int n, const double* Ain, double* U, double* S, double* Vt) {
  if (!ctx) return TNFEM_E_INVALID;
  return guard(ctx, [&] {
    TN_REQUIRE(Ain && U && S && Vt && m >= n && n >= 1, "bad arguments (needs m >= n >= 1)");
    DArr<double> A(ctx, (size_t)m * n), w(ctx, svd_work_elems(m, n));
    copy<double>(ctx, A.p, Ain, (size_t)m * n);
    svd<double>(ctx, m, n, A.p, U, S, Vt, w.p);
    sync(ctx);
  });
}

}  // extern "C"
