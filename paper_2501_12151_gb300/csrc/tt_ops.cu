// Tensor-train data structures and TT algebra on the device: rounding (left-to-right
// Householder QR, then right-to-left truncated SVD, Section 4 Eq. qr), exact sums and
// operator-times-train products, inner products, norms and the energy norm of a difference.
#include <algorithm>
#include <climits>
#include <cmath>

#include "internal.h"

using namespace tnfem;

tnfem_tt::~tnfem_tt() {
  for (double* p : core)
    if (p) dfree(ctx, p);
}

tnfem_mpo::~tnfem_mpo() {
  for (double* p : core)
    if (p) dfree(ctx, p);
  for (int o = 0; o < 2; ++o) {
    for (double* p : p64[o])
      if (p) dfree(ctx, p);
    for (float* p : p32[o])
      if (p) dfree(ctx, p);
  }
}

namespace tnfem {

void* dalloc(tnfem_ctx* ctx, size_t bytes) {
  if (bytes == 0) bytes = 8;
  bytes = (bytes + 255) & ~size_t(255);
  if (ctx->mem_budget && ctx->mem_in_use + bytes > ctx->mem_budget)
    throw Error(TNFEM_E_BUDGET, "device-memory budget of " + std::to_string(ctx->mem_budget) + " bytes exceeded (" +
                                    std::to_string(ctx->mem_in_use) + " held, " + std::to_string(bytes) + " requested)");
  void* p = nullptr;
  if (ctx->alloc_fn) {
    p = ctx->alloc_fn(bytes, ctx->user);
    if (!p) throw Error(TNFEM_E_NOMEM, "device allocation callback failed for " + std::to_string(bytes) + " bytes");
  } else {
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      throw Error(TNFEM_E_NOMEM, "cudaMalloc(" + std::to_string(bytes) + "): " + cudaGetErrorString(e));
    }
  }
  ctx->mem_sizes[p] = bytes;
  ctx->mem_in_use += bytes;
  ctx->mem_peak = std::max(ctx->mem_peak, ctx->mem_in_use);
  return p;
}

void dfree(tnfem_ctx* ctx, void* p) {
  if (!p) return;
  auto it = ctx->mem_sizes.find(p);
  if (it != ctx->mem_sizes.end()) {
    ctx->mem_in_use -= it->second;
    ctx->mem_sizes.erase(it);
  }
  if (ctx->free_fn) ctx->free_fn(p, ctx->user);
  else cudaFree(p);
}

int coop_sms(tnfem_ctx* ctx) {
  int v = 0;
  TN_CHECK_CUDA(cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, ctx->device));
  return ctx->sm_share > 0 ? std::min(v, ctx->sm_share) : v;
}

void sync(tnfem_ctx* ctx) { TN_CHECK_CUDA(cudaStreamSynchronize(ctx->stream)); }

tnfem_tt* tt_new(tnfem_ctx* ctx, const std::vector<int>& n, const std::vector<int>& r,
                 const std::vector<size_t>* cap) {
  auto* x = new tnfem_tt();
  x->ctx = ctx;
  x->d = (int)n.size();
  x->n = n;
  x->r = r;
  x->core.assign(x->d, nullptr);
  x->cap.assign(x->d, 0);
  try {
    for (int k = 0; k < x->d; ++k) {
      size_t need = (size_t)r[k] * n[k] * r[k + 1];
      size_t c = cap ? std::max(need, (*cap)[k]) : need;
      x->core[k] = static_cast<double*>(dalloc(ctx, c * sizeof(double)));
      x->cap[k] = c;
    }
  } catch (...) {
    delete x;
    throw;
  }
  return x;
}

void tt_set_core(tnfem_tt* x, int k, int r0, int r1) {
  size_t need = (size_t)r0 * x->n[k] * r1;
  if (need > x->cap[k]) {
    double* p = static_cast<double*>(dalloc(x->ctx, need * sizeof(double)));
    dfree(x->ctx, x->core[k]);
    x->core[k] = p;
    x->cap[k] = need;
  }
  x->r[k] = r0;
  x->r[k + 1] = r1;
}

tnfem_tt* tt_clone(const tnfem_tt* x) {
  tnfem_tt* y = tt_new(x->ctx, x->n, x->r);
  for (int k = 0; k < x->d; ++k)
    copy<double>(x->ctx, y->core[k], x->core[k], (size_t)x->r[k] * x->n[k] * x->r[k + 1]);
  return y;
}

tnfem_mpo* mpo_new(tnfem_ctx* ctx, const std::vector<int>& n, const std::vector<int>& a) {
  auto* A = new tnfem_mpo();
  A->ctx = ctx;
  A->d = (int)n.size();
  A->n = n;
  A->a = a;
  A->core.assign(A->d, nullptr);
  try {
    for (int k = 0; k < A->d; ++k)
      A->core[k] = static_cast<double*>(dalloc(ctx, (size_t)a[k] * n[k] * n[k] * a[k + 1] * sizeof(double)));
  } catch (...) {
    delete A;
    throw;
  }
  return A;
}

void mpo_prepare(tnfem_mpo* A) {
  if (A->prepared) return;
  tnfem_ctx* ctx = A->ctx;
  const int d = A->d;
  for (int o = 0; o < 2; ++o) {
    A->p64[o].assign(d, nullptr);
    A->p32[o].assign(d, nullptr);
  }
  size_t maxc = 0;
  for (int k = 0; k < d; ++k) maxc = std::max(maxc, (size_t)A->a[k] * A->n[k] * A->n[k] * A->a[k + 1]);
  DArr<double> tmp(ctx, maxc);
  for (int k = 0; k < d; ++k) {
    const int a0 = A->a[k], n = A->n[k], a1 = A->a[k + 1];
    const size_t sz = (size_t)a0 * n * n * a1;
    // given orientation: [a0][j][i][a1]
    A->p64[0][k] = static_cast<double*>(dalloc(ctx, sz * sizeof(double)));
    transpose4_mid<double>(ctx, A->p64[0][k], A->core[k], a0, n, n, a1);
    // flipped orientation: core d-1-k of the flipped train is [a1][n][n][a0]; swap its modes too
    const int kf = d - 1 - k;
    A->p64[1][kf] = static_cast<double*>(dalloc(ctx, sz * sizeof(double)));
    transpose4_outer<double>(ctx, tmp.p, A->core[k], a0, n, n, a1);  // [a1][i][j][a0]
    transpose4_mid<double>(ctx, A->p64[1][kf], tmp.p, a1, n, n, a0);  // [a1][j][i][a0]
    for (int o = 0; o < 2; ++o) {
      int kk = o == 0 ? k : kf;
      A->p32[o][kk] = static_cast<float*>(dalloc(ctx, sz * sizeof(float)));
      convert_d2f(ctx, A->p32[o][kk], A->p64[o][kk], sz);
    }
    sync(ctx);
  }
  A->prepared = true;
}

size_t tt_bytes(const tnfem_tt* x) {
  size_t s = 0;
  for (int k = 0; k < x->d; ++k) s += (size_t)x->r[k] * x->n[k] * x->r[k + 1] * sizeof(double);
  return s;
}

size_t mpo_bytes(const tnfem_mpo* A) {
  size_t s = 0;
  for (int k = 0; k < A->d; ++k) s += (size_t)A->a[k] * A->n[k] * A->n[k] * A->a[k + 1] * sizeof(double);
  return s;
}

// ---- random cores ------------------------------------------------------------------------------

namespace {

__device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void gaussian_kernel(double* x, size_t n, uint64_t seed, uint64_t sid) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    uint64_t key = splitmix64(seed ^ splitmix64(sid * 0x100000001B3ull + i));
    uint64_t a = splitmix64(key), b = splitmix64(key ^ 0xD1B54A32D192ED03ull);
    // uniform in (0, 1]: 53 random bits
    double u1 = ((a >> 11) + 1.0) * (1.0 / 9007199254740992.0);
    double u2 = (b >> 11) * (1.0 / 9007199254740992.0);
    x[i] = sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
  }
}

__global__ void block_copy3_kernel(double* __restrict__ dst, int R0, int n, int R1, int off0, int off1,
                                   const double* __restrict__ src, int r0, int r1, double s) {
  long long total = (long long)r0 * n * r1;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    int b = (int)(t % r1);
    long long q = t / r1;
    int i = (int)(q % n);
    int a = (int)(q / n);
    dst[((long long)(off0 + a) * n + i) * R1 + off1 + b] = s * src[t];
  }
}

// out[(beta a)][i][(g b)] = sum_j A[beta][i][j][g] x[a][j][b]
__global__ void mpo_apply_kernel(double* __restrict__ out, const double* __restrict__ A,
                                 const double* __restrict__ x, int a0, int n, int a1, int r0, int r1) {
  long long total = (long long)a0 * r0 * n * a1 * r1;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    int b = (int)(t % r1);
    long long q = t / r1;
    int g = (int)(q % a1);
    q /= a1;
    int i = (int)(q % n);
    q /= n;
    int a = (int)(q % r0);
    int be = (int)(q / r0);
    double s = 0.0;
    const double* Ar = A + (((long long)be * n + i) * n) * a1 + g;
    const double* xr = x + (long long)a * n * r1 + b;
    for (int j = 0; j < n; ++j) s += Ar[(long long)j * a1] * xr[(long long)j * r1];
    out[t] = s;
  }
}

// dst[i][c] = src[i*ld + c] * s[c] for c < ncols
__global__ void scale_cols_kernel(double* __restrict__ dst, const double* __restrict__ src, int rows,
                                  int ld, int ncols, const double* __restrict__ s) {
  long long total = (long long)rows * ncols;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    int i = (int)(t / ncols), c = (int)(t % ncols);
    dst[t] = src[(long long)i * ld + c] * s[c];
  }
}

inline int gblocks(long long n) { return (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, 152 * 16)); }

}  // namespace

void fill_gaussian(tnfem_ctx* ctx, double* x, size_t n, uint64_t seed, uint64_t sid) {
  if (!n) return;
  gaussian_kernel<<<gblocks((long long)n), 256, 0, ctx->stream>>>(x, n, seed, sid);
  count_launch(ctx);
  check_launch(ctx, "gaussian");
}

void block_copy3(tnfem_ctx* ctx, double* dst, int R0, int n, int R1, int off0, int off1, const double* src,
                 int r0, int r1, double s) {
  long long total = (long long)r0 * n * r1;
  if (!total) return;
  block_copy3_kernel<<<gblocks(total), 256, 0, ctx->stream>>>(dst, R0, n, R1, off0, off1, src, r0, r1, s);
  count_launch(ctx);
  check_launch(ctx, "block_copy3");
}

void scale_cols(tnfem_ctx* ctx, double* dst, const double* src, int rows, int ld, int ncols, const double* s) {
  if ((long long)rows * ncols == 0) return;
  scale_cols_kernel<<<gblocks((long long)rows * ncols), 256, 0, ctx->stream>>>(dst, src, rows, ld, ncols, s);
  count_launch(ctx);
  check_launch(ctx, "scale_cols");
}

// Truncation rank: smallest r whose discarded tail sum_{i>=r} s_i^2 <= delta^2, capped.
int truncation_rank(const std::vector<double>& S, double delta, int rmax) {
  int n = (int)S.size();
  std::vector<double> tail(n + 1, 0.0);
  for (int i = n - 1; i >= 0; --i) tail[i] = tail[i + 1] + S[i] * S[i];
  int r = n;
  for (int i = 0; i < n; ++i) {
    if (std::sqrt(tail[i]) <= delta) { r = i; break; }
  }
  r = std::max(1, std::min(r, rmax));
  return r;
}

// ---- rounding --------------------------------------------------------------------------------

// Left-orthogonalise cores 0..d-2 of y in place (y has room for the ranks it gets).
static void orthogonalize_left_inplace(tnfem_ctx* ctx, tnfem_tt* y) {
  const int d = y->d;
  size_t maxw = 0;
  for (int k = 0; k < d; ++k) maxw = std::max(maxw, (size_t)y->r[k] * y->n[k] * y->r[k + 1]);
  DArr<double> A(ctx, maxw), Q(ctx, maxw), R(ctx, maxw + 64), tmp(ctx, maxw), qw(ctx, 4096 + maxw / 16);
  for (int k = 0; k < d - 1; ++k) {
    const int r0 = y->r[k], n = y->n[k], r1 = y->r[k + 1];
    const int m = r0 * n, kk = std::min(m, r1);
    copy<double>(ctx, A.p, y->core[k], (size_t)m * r1);
    qw.ensure(ctx, qr_work_elems(m, r1));
    qr<double>(ctx, m, r1, A.p, Q.p, R.p, qw.p);
    // next core <- R * next   (kk x r1) (r1 x n2 r2)
    const int n2 = y->n[k + 1], r2 = y->r[k + 2];
    GemmDesc g{kk, n2 * r2, r1, 1, r1, 1, 0, (long long)n2 * r2, 1, 0, (long long)n2 * r2, 1, 0};
    tmp.ensure(ctx, (size_t)kk * n2 * r2);
    gemm<double>(ctx, g, 1.0, R.p, y->core[k + 1], 0.0, tmp.p);
    tt_set_core(y, k, r0, kk);
    copy<double>(ctx, y->core[k], Q.p, (size_t)m * kk);
    tt_set_core(y, k + 1, kk, r2);
    copy<double>(ctx, y->core[k + 1], tmp.p, (size_t)kk * n2 * r2);
  }
  sync(ctx);
}

tnfem_tt* tt_round(tnfem_ctx* ctx, const tnfem_tt* x, double eps, int rmax) {
  const int d = x->d;
  tnfem_tt* y = tt_clone(x);
  try {
    if (d == 1) return y;
    orthogonalize_left_inplace(ctx, y);
    const double nrm = nrm2<double>(ctx, y->core[d - 1], (size_t)y->r[d - 1] * y->n[d - 1] * y->r[d]);
    const double delta = eps / std::sqrt((double)(d - 1)) * nrm;
    std::vector<double> S;
    for (int k = d - 1; k >= 1; --k) {
      const int r0 = y->r[k], n = y->n[k], r1 = y->r[k + 1];
      const int w = n * r1;  // M = core as r0 x w
      const int p = std::min(r0, w);
      DArr<double> Mt(ctx, (size_t)r0 * w), U(ctx, (size_t)std::max(r0, w) * p), Sd(ctx, p + 8),
          Vt(ctx, (size_t)p * p), sw(ctx, svd_work_elems(std::max(r0, w), p));
      DArr<double> left(ctx, (size_t)r0 * p), right(ctx, (size_t)p * w);
      if (w >= r0) {
        // M^T (w x r0) = U S Vt  =>  M = Vt^T S U^T: new core = U^T (rows), left factor Vt^T S
        transpose2<double>(ctx, Mt.p, y->core[k], r0, w);
        if (w >= 8 * r0 && r0 >= 64) {
          // far taller than wide (the operator cores of the 3D rounding): QR first, the Jacobi SVD
          // of the small R factor, U = Q U_R (the SVD's rotations then run on r0-long columns)
          DArr<double> Qt(ctx, (size_t)w * r0), Rt(ctx, (size_t)r0 * r0), UR(ctx, (size_t)r0 * r0),
              qw(ctx, qr_work_elems(w, r0));
          qr<double>(ctx, w, r0, Mt.p, Qt.p, Rt.p, qw.p);
          svd<double>(ctx, r0, r0, Rt.p, UR.p, Sd.p, Vt.p, sw.p);
          GemmDesc gu{w, r0, r0, 1, r0, 1, 0, r0, 1, 0, r0, 1, 0};
          gemm<double>(ctx, gu, 1.0, Qt.p, UR.p, 0.0, U.p);
        } else {
          svd<double>(ctx, w, r0, Mt.p, U.p, Sd.p, Vt.p, sw.p);
        }
        transpose2<double>(ctx, right.p, U.p, w, p);     // p x w
        transpose2<double>(ctx, left.p, Vt.p, p, p);     // r0 x p (= Vt^T)
      } else {
        // M (r0 x w), r0 > w: M = U S Vt: new core = Vt, left factor U S
        copy<double>(ctx, Mt.p, y->core[k], (size_t)r0 * w);
        svd<double>(ctx, r0, w, Mt.p, U.p, Sd.p, Vt.p, sw.p);
        copy<double>(ctx, right.p, Vt.p, (size_t)p * w);
        copy<double>(ctx, left.p, U.p, (size_t)r0 * p);
      }
      S.assign(p, 0.0);
      TN_CHECK_CUDA(cudaMemcpyAsync(S.data(), Sd.p, p * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
      sync(ctx);
      const int rk = truncation_rank(S, delta, rmax);
      // LS = left[:, :rk] * diag(S[:rk])  (r0 x rk), applied to the previous core
      DArr<double> LS(ctx, (size_t)r0 * rk);
      scale_cols(ctx, LS.p, left.p, r0, p, rk, Sd.p);
      const int r_prev = y->r[k - 1], n_prev = y->n[k - 1];
      DArr<double> nc(ctx, (size_t)r_prev * n_prev * rk);
      GemmDesc g2{r_prev * n_prev, rk, r0, 1, r0, 1, 0, rk, 1, 0, rk, 1, 0};
      gemm<double>(ctx, g2, 1.0, y->core[k - 1], LS.p, 0.0, nc.p);
      // new core k = right[:rk] (rk x w)
      tt_set_core(y, k, rk, r1);
      copy<double>(ctx, y->core[k], right.p, (size_t)rk * w);
      tt_set_core(y, k - 1, r_prev, rk);
      copy<double>(ctx, y->core[k - 1], nc.p, (size_t)r_prev * n_prev * rk);
      sync(ctx);
    }
  } catch (...) {
    delete y;
    throw;
  }
  return y;
}

tnfem_tt* tt_from_full(tnfem_ctx* ctx, const double* host, const std::vector<int>& modes, double eps) {
  const int d = (int)modes.size();
  TN_REQUIRE(d >= 1, "tt_from_full: no modes");
  size_t total = 1;
  for (int m : modes) total *= (size_t)m;
  TN_REQUIRE(total <= (size_t)INT_MAX, "tt_from_full: array too large");
  DArr<double> C(ctx, total);
  TN_CHECK_CUDA(cudaMemcpyAsync(C.p, host, total * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  const double nrm = nrm2<double>(ctx, C.p, total);
  const double delta = eps / std::sqrt((double)std::max(1, d - 1)) * nrm;
  std::vector<DArr<double>> cores;
  std::vector<int> r(d + 1, 1);
  size_t rest = total;
  int rk = 1;
  for (int k = 0; k < d - 1; ++k) {
    rest /= (size_t)modes[k];
    const int m = rk * modes[k], ri = (int)rest;
    if (m <= 64 && m <= ri) {
      // an unfolding with at most 64 rows keeps the identity core (exact, rank = rows); the
      // array itself is then already the next unfolding
      std::vector<double> I((size_t)m * m, 0.0);
      for (int i = 0; i < m; ++i) I[(size_t)i * m + i] = 1.0;
      DArr<double> core(ctx, (size_t)m * m);
      TN_CHECK_CUDA(cudaMemcpyAsync(core.p, I.data(), I.size() * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
      sync(ctx);
      cores.push_back(std::move(core));
      rk = r[k + 1] = m;
      continue;
    }
    const int q = std::min(m, ri);
    DArr<double> U(ctx, (size_t)m * q), Sd(ctx, q + 8), Vt(ctx, (size_t)q * q), next;
    std::vector<double> S(q);
    int keep;
    if (m <= ri) {
      // C (m x rest): C^T = Q R, R^T = U S Vt, so C = U S Vt Q^T
      DArr<double> Q(ctx, rest * m), R(ctx, (size_t)m * m);
      {
        DArr<double> Ct(ctx, rest * m), qw(ctx, qr_work_elems(ri, m));
        transpose2<double>(ctx, Ct.p, C.p, m, ri);
        qr<double>(ctx, ri, m, Ct.p, Q.p, R.p, qw.p);
      }
      DArr<double> Rt(ctx, (size_t)m * m), sw(ctx, svd_work_elems(m, m));
      transpose2<double>(ctx, Rt.p, R.p, m, m);
      svd<double>(ctx, m, m, Rt.p, U.p, Sd.p, Vt.p, sw.p);
      TN_CHECK_CUDA(cudaMemcpyAsync(S.data(), Sd.p, q * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
      sync(ctx);
      keep = truncation_rank(S, delta, 1 << 20);
      // next = diag(S) Vt[:keep] Q^T = (Q V[:, :keep] diag(S))^T, keep x rest
      DArr<double> V(ctx, (size_t)m * m), VS(ctx, (size_t)m * keep);
      transpose2<double>(ctx, V.p, Vt.p, m, m);
      scale_cols(ctx, VS.p, V.p, m, m, keep, Sd.p);
      next = DArr<double>(ctx, (size_t)keep * rest);
      GemmDesc g{keep, ri, m, 1, 1, keep, 0, 1, m, 0, ri, 1, 0};
      gemm<double>(ctx, g, 1.0, VS.p, Q.p, 0.0, next.p);
    } else {
      // more rows than columns: C = U S Vt directly
      DArr<double> sw(ctx, svd_work_elems(m, ri));
      svd<double>(ctx, m, ri, C.p, U.p, Sd.p, Vt.p, sw.p);
      TN_CHECK_CUDA(cudaMemcpyAsync(S.data(), Sd.p, q * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
      sync(ctx);
      keep = truncation_rank(S, delta, 1 << 20);
      DArr<double> V(ctx, (size_t)ri * ri), VS(ctx, (size_t)ri * keep);
      transpose2<double>(ctx, V.p, Vt.p, ri, ri);
      scale_cols(ctx, VS.p, V.p, ri, ri, keep, Sd.p);
      next = DArr<double>(ctx, (size_t)keep * rest);
      transpose2<double>(ctx, next.p, VS.p, ri, keep);
    }
    // core = U[:, :keep]  (m x keep)
    DArr<double> ones(ctx, keep), core(ctx, (size_t)m * keep);
    fill<double>(ctx, ones.p, 1.0, keep);
    scale_cols(ctx, core.p, U.p, m, q, keep, ones.p);
    sync(ctx);
    cores.push_back(std::move(core));
    C = std::move(next);
    rk = r[k + 1] = keep;
  }
  cores.push_back(std::move(C));
  tnfem_tt* y = tt_new(ctx, modes, r);
  for (int k = 0; k < d; ++k) copy<double>(ctx, y->core[k], cores[k].p, (size_t)r[k] * modes[k] * r[k + 1]);
  sync(ctx);
  return y;
}

tnfem_mpo* mpo_round(tnfem_ctx* ctx, const tnfem_mpo* A, double eps, int rmax) {
  std::vector<int> nn(A->d);
  for (int k = 0; k < A->d; ++k) nn[k] = A->n[k] * A->n[k];
  tnfem_tt* x = tt_new(ctx, nn, A->a);
  tnfem_tt* y = nullptr;
  tnfem_mpo* B = nullptr;
  try {
    for (int k = 0; k < A->d; ++k)
      copy<double>(ctx, x->core[k], A->core[k], (size_t)A->a[k] * nn[k] * A->a[k + 1]);
    y = tt_round(ctx, x, eps, rmax);
    B = mpo_new(ctx, A->n, y->r);
    for (int k = 0; k < A->d; ++k)
      copy<double>(ctx, B->core[k], y->core[k], (size_t)y->r[k] * nn[k] * y->r[k + 1]);
    sync(ctx);
  } catch (...) {
    delete x;
    delete y;
    delete B;
    throw;
  }
  delete x;
  delete y;
  return B;
}

// ---- sums, products, inner products ------------------------------------------------------------

tnfem_tt* tt_axpy(tnfem_ctx* ctx, const tnfem_tt* x, double beta, const tnfem_tt* y) {
  TN_REQUIRE(x->d == y->d, "tt_axpy: different number of cores");
  for (int k = 0; k < x->d; ++k) TN_REQUIRE(x->n[k] == y->n[k], "tt_axpy: mode mismatch");
  const int d = x->d;
  std::vector<int> r(d + 1);
  r[0] = 1;
  r[d] = 1;
  for (int k = 1; k < d; ++k) r[k] = x->r[k] + y->r[k];
  if (d == 1) r[1] = 1;
  tnfem_tt* z = tt_new(ctx, x->n, r);
  try {
    for (int k = 0; k < d; ++k) {
      const int n = x->n[k];
      const size_t sz = (size_t)r[k] * n * r[k + 1];
      if (d == 1) {
        copy<double>(ctx, z->core[0], x->core[0], sz);
        axpby<double>(ctx, z->core[0], beta, y->core[0], 1.0, sz);
        continue;
      }
      fill<double>(ctx, z->core[k], 0.0, sz);
      const int xo0 = 0, xo1 = 0;
      const int yo0 = (k == 0) ? 0 : x->r[k];
      const int yo1 = (k == d - 1) ? 0 : x->r[k + 1];
      block_copy3(ctx, z->core[k], r[k], n, r[k + 1], xo0, xo1, x->core[k], x->r[k], x->r[k + 1], 1.0);
      block_copy3(ctx, z->core[k], r[k], n, r[k + 1], yo0, yo1, y->core[k], y->r[k], y->r[k + 1],
                  k == 0 ? beta : 1.0);
    }
    sync(ctx);
  } catch (...) {
    delete z;
    throw;
  }
  return z;
}

tnfem_tt* mpo_apply(tnfem_ctx* ctx, const tnfem_mpo* A, const tnfem_tt* x) {
  TN_REQUIRE(A->d == x->d, "mpo_apply: core count mismatch");
  const int d = x->d;
  std::vector<int> r(d + 1);
  for (int k = 0; k <= d; ++k) r[k] = A->a[k] * x->r[k];
  for (int k = 0; k < d; ++k) TN_REQUIRE(A->n[k] == x->n[k], "mpo_apply: mode mismatch");
  tnfem_tt* y = tt_new(ctx, x->n, r);
  try {
    for (int k = 0; k < d; ++k) {
      long long total = (long long)r[k] * x->n[k] * r[k + 1];
      mpo_apply_kernel<<<gblocks(total), 256, 0, ctx->stream>>>(y->core[k], A->core[k], x->core[k], A->a[k],
                                                                 x->n[k], A->a[k + 1], x->r[k], x->r[k + 1]);
      count_launch(ctx);
      check_launch(ctx, "mpo_apply");
    }
    sync(ctx);
  } catch (...) {
    delete y;
    throw;
  }
  return y;
}

double tt_dot(tnfem_ctx* ctx, const tnfem_tt* x, const tnfem_tt* y) {
  TN_REQUIRE(x->d == y->d, "tt_dot: core count mismatch");
  const int d = x->d;
  size_t maxe = 1, maxw = 1;
  for (int k = 0; k <= d; ++k) maxe = std::max(maxe, (size_t)x->r[k] * y->r[k]);
  for (int k = 0; k < d; ++k) maxw = std::max(maxw, (size_t)x->r[k] * x->n[k] * y->r[k + 1]);
  DArr<double> E0(ctx, maxe), E1(ctx, maxe), ws(ctx, maxw * 2 + 64 * maxe + 1024);
  fill<double>(ctx, E0.p, 1.0, 1);
  for (int k = 0; k < d; ++k) {
    env_left_vec<double>(ctx, x->r[k], x->r[k + 1], y->r[k], y->r[k + 1], x->n[k], E0.p, x->core[k],
                         y->core[k], E1.p, ws.p, ws.n);
    std::swap(E0.p, E1.p);
  }
  double v = 0;
  TN_CHECK_CUDA(cudaMemcpyAsync(&v, E0.p, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  sync(ctx);
  return v;
}

double tt_norm(tnfem_ctx* ctx, const tnfem_tt* x) {
  tnfem_tt* y = tt_clone(x);
  double v = 0;
  try {
    orthogonalize_left_inplace(ctx, y);
    const int d = y->d;
    v = nrm2<double>(ctx, y->core[d - 1], (size_t)y->r[d - 1] * y->n[d - 1] * y->r[d]);
  } catch (...) {
    delete y;
    throw;
  }
  delete y;
  return v;
}

double energy_norm(tnfem_ctx* ctx, const tnfem_mpo* A, const tnfem_tt* u, const tnfem_tt* v) {
  tnfem_tt* dlt = v ? tt_axpy(ctx, u, -1.0, v) : tt_clone(u);
  double out = 0;
  try {
    // orthogonalise the difference so that its last core carries the (small) difference itself
    orthogonalize_left_inplace(ctx, dlt);
    mpo_prepare(const_cast<tnfem_mpo*>(A));
    const int d = dlt->d;
    size_t maxe = 1, maxws = 1;
    for (int k = 0; k <= d; ++k) maxe = std::max(maxe, (size_t)dlt->r[k] * A->a[k] * dlt->r[k]);
    for (int k = 0; k < d; ++k)
      maxws = std::max(maxws, local_ws_elems(dlt->r[k], dlt->n[k], dlt->r[k + 1], A->a[k], A->a[k + 1]));
    DArr<double> E0(ctx, maxe), E1(ctx, maxe), ws(ctx, maxws);
    fill<double>(ctx, E0.p, 1.0, 1);
    for (int k = 0; k < d; ++k) {
      env_left<double>(ctx, dlt->r[k], dlt->r[k + 1], dlt->r[k], dlt->r[k + 1], dlt->n[k], A->a[k], A->a[k + 1],
                       E0.p, dlt->core[k], A->p64[0][k], dlt->core[k], E1.p, ws.p, ws.n);
      std::swap(E0.p, E1.p);
    }
    double q = 0;
    TN_CHECK_CUDA(cudaMemcpyAsync(&q, E0.p, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    sync(ctx);
    out = std::sqrt(std::max(q, 0.0));
  } catch (...) {
    delete dlt;
    throw;
  }
  delete dlt;
  return out;
}

// ---- global residual on the dense expansion ---------------------------------------------------
//
// a9's confirmation ||f - A u||_2 / ||f||_2 for grids whose unknowns fit the device as a dense
// vector (the 2^10 x 2^10 benchmark: 2.1M unknowns): u and f are expanded to dense vectors in the
// QTT index order (i_0 most significant) by a chain of GEMMs, A u is formed densely by applying the
// operator cores one at a time (a batched GEMM per core, intermediate [outputs so far][rank]
// [inputs left]), and the residual is an explicit difference of dense vectors, so nothing cancels
// beyond the rounding of A u itself.

namespace {

// out[((i * a1 + g) * a0 + a) * n + j] = in[((a * n + i) * n + j) * a1 + g]
__global__ void mpo_core_perm_kernel(double* __restrict__ out, const double* __restrict__ in, int a0, int n, int a1) {
  const long long total = (long long)a0 * n * n * a1;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    long long r = t;
    const int g = (int)(r % a1);
    r /= a1;
    const int j = (int)(r % n);
    r /= n;
    const int i = (int)(r % n);
    const int a = (int)(r / n);
    out[(((long long)i * a1 + g) * a0 + a) * n + j] = in[t];
  }
}

}  // namespace

// dense expansion of a train into `out` (prod of modes entries); `tmp` holds as many
size_t dense_elems(const tnfem_tt* x) {
  size_t N = 1;
  for (int k = 0; k < x->d; ++k) N *= (size_t)x->n[k];
  return N;
}

void tt_full_device(tnfem_ctx* ctx, const tnfem_tt* x, double* out, double* tmp, size_t cap) {
  // V_k [(o, i), r'] = V_{k-1} [o, r] . core_k [r, (i, r')]
  double* cur = tmp;
  double* nxt = out;
  size_t rows = 1;
  fill<double>(ctx, cur, 1.0, 1);
  for (int k = 0; k < x->d; ++k) {
    const int r0 = x->r[k], n = x->n[k], r1 = x->r[k + 1];
    TN_REQUIRE(rows * n * r1 <= cap, "dense expansion: buffer too small");
    GemmDesc g{(int)rows, n * r1, r0, 1, r0, 1, 0, (long long)n * r1, 1, 0, (long long)n * r1, 1, 0};
    TN_REQUIRE(rows < (1ull << 31), "dense expansion: too many rows");
    gemm<double>(ctx, g, 1.0, cur, x->core[k], 0.0, nxt);
    rows *= n;
    std::swap(cur, nxt);
  }
  if (cur != out) copy<double>(ctx, out, cur, rows);
}

double residual_norm_dense(tnfem_ctx* ctx, const tnfem_mpo* A, const tnfem_tt* f, const tnfem_tt* u) {
  const int d = u->d;
  const size_t N = dense_elems(u);
  int amax = 1;
  for (int k = 0; k <= d; ++k) amax = std::max(amax, A->a[k]);
  int rmax = 1;
  for (int k = 0; k <= d; ++k) rmax = std::max({rmax, u->r[k], f->r[k]});
  const size_t cap = N * (size_t)std::max(amax, rmax);
  DArr<double> X(ctx, cap), Y(ctx, cap), F(ctx, N);
  tt_full_device(ctx, f, F.p, X.p, cap);
  tt_full_device(ctx, u, Y.p, X.p, cap);  // u dense in Y
  // state T [o][alpha][rest] in X / Y alternately: start with T = u (o = 1, alpha = 1, rest = N)
  double* T = Y.p;
  double* Tn = X.p;
  size_t no = 1, rest = N;
  for (int k = 0; k < d; ++k) {
    const int a0 = A->a[k], n = A->n[k], a1 = A->a[k + 1];
    DArr<double> Ap(ctx, (size_t)a0 * n * n * a1);
    mpo_core_perm_kernel<<<std::max(1, std::min(1216, (int)((Ap.n + 255) / 256))), 256, 0, ctx->stream>>>(Ap.p, A->core[k],
                                                                                                         a0, n, a1);
    count_launch(ctx);
    check_launch(ctx, "mpo_core_perm");
    const size_t restn = rest / n;
    if (no <= restn) {
      // batch over the outputs o: T'[o][(i,b)][s] = Ap[(i,b)][(a,j)] . T[o][(a,j)][s]
      TN_REQUIRE(no < 65536, "dense residual: batch too large");
      GemmDesc g{n * a1, (int)restn, a0 * n, (int)no, (long long)a0 * n, 1, 0, (long long)restn, 1,
                 (long long)a0 * n * restn, (long long)restn, 1, (long long)n * a1 * restn};
      gemm<double>(ctx, g, 1.0, Ap.p, T, 0.0, Tn);
    } else {
      // batch over the remaining inputs s: rows o, T'[o][(i,b)][s] = T[o][(a,j)][s] . Ap^T
      TN_REQUIRE(restn < 65536, "dense residual: batch too large");
      GemmDesc g{(int)no, n * a1, a0 * n, (int)restn, (long long)a0 * n * restn, (long long)restn, 1, 1,
                 (long long)a0 * n, 0, (long long)n * a1 * restn, (long long)restn, 1};
      gemm<double>(ctx, g, 1.0, T, Ap.p, 0.0, Tn);
    }
    no *= n;
    rest = restn;
    std::swap(T, Tn);
  }
  // T = A u (a_d = 1, rest = 1), dense in the same order as F: r = F - A u
  axpby<double>(ctx, T, 1.0, F.p, -1.0, N);  // T <- F - T
  const double rn = nrm2<double>(ctx, T, N);
  const double fn = nrm2<double>(ctx, F.p, N);
  return fn > 0 ? rn / fn : rn;
}

}  // namespace tnfem
