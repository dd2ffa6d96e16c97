// The sweep's contractions expressed as three chained strided GEMMs each:
//
//   local matvec (a4):  y[a',i,b'] = sum PhiL[a',beta,a] A[beta,i,j,g] PhiR[b',g,b] x[a,j,b]
//   left environment (a2/a8):  Phi'[b',g,b] = sum y[a',i,b'] Phi[a',beta,a] A[beta,i,j,g] x[a,j,b]
//
// stage 1  T1[a',beta,j,b] = PhiL . x            (r0 a0) x r0 x (n r1)
// stage 2  T2[a',i,g,b]    = T1 . A  per a'      batched r1 x (a0 n) x (n a1)
// stage 3  y               = T2 . PhiR           (r0 n) x (a1 r1) x r1
//
// The operator core enters stage 2 through its copy permuted to [beta][j][i][g] so that the
// contracted pair (beta, j) has a single stride.  Every layout below is row-major.
#include <algorithm>

#include "internal.h"

namespace tnfem {

size_t local_ws_elems(int r0, int n, int r1, int a0, int a1) {
  size_t t1 = (size_t)r0 * a0 * n * r1;
  size_t t2 = (size_t)r0 * n * a1 * r1;
  size_t out = (size_t)r0 * n * r1 + (size_t)r1 * a1 * r1;
  // split-K partials: two copies of a stage-1/2 product or 64 copies of a stage-3 output
  return t1 + t2 + std::max(2 * std::max(t1, t2), 64 * out) + 64;
}

namespace {

template <typename T>
void stage12(tnfem_ctx* ctx, int ry0, int rx0, int rx1, int n, int a0, int a1, const T* Phi,
             const T* Ap, const T* x, T* T1, T* T2, T* work, size_t work_elems,
             const int* skip = nullptr) {
  // stage 1: T1[(a',beta)][(j,b)] = sum_a Phi[(a',beta)][a] x[a][(j,b)]
  GemmDesc g1{ry0 * a0, n * rx1, rx0, 1, rx0, 1, 0, (long long)n * rx1, 1, 0, (long long)n * rx1, 1, 0};
  gemm<T>(ctx, g1, T(1), Phi, x, T(0), T1, work, work_elems, skip);
  // stage 2 (batch a'): T2[a'][(i,g)][b] = sum_{kappa=(beta,j)} T1[a'][kappa][b] Ap[kappa][(i,g)]
  GemmDesc g2{rx1, n * a1, a0 * n, ry0,
              1, rx1, (long long)a0 * n * rx1,
              (long long)n * a1, 1, 0,
              1, rx1, (long long)n * a1 * rx1};
  gemm<T>(ctx, g2, T(1), T1, Ap, T(0), T2, work, work_elems, skip);
}

}  // namespace

template <typename T>
void local_apply(tnfem_ctx* ctx, int ry0, int ry1, int rx0, int rx1, int n, int a0, int a1, const T* PhiL,
                 const T* Ap, const T* PhiR, const T* x, T* y, T alpha, T beta, T* ws, size_t ws_elems,
                 const int* skip) {
  T* T1 = ws;
  T* T2 = T1 + (size_t)ry0 * a0 * n * rx1;
  T* work = T2 + (size_t)ry0 * n * a1 * rx1;
  size_t used = (size_t)(work - ws);
  TN_REQUIRE(ws_elems > used, "local_apply: workspace too small");
  size_t work_elems = ws_elems - used;
  stage12<T>(ctx, ry0, rx0, rx1, n, a0, a1, PhiL, Ap, x, T1, T2, work, work_elems, skip);
  // stage 3: y[(a',i)][b'] = sum_{kappa=(g,b)} T2[(a',i)][kappa] PhiR[b'][kappa]
  GemmDesc g3{ry0 * n, ry1, a1 * rx1, 1, (long long)a1 * rx1, 1, 0, 1, (long long)a1 * rx1, 0, ry1, 1, 0};
  gemm<T>(ctx, g3, alpha, T2, PhiR, beta, y, work, work_elems, skip);
}

template <typename T>
void local_matvec(tnfem_ctx* ctx, int r0, int n, int r1, int a0, int a1, const T* PhiL, const T* Ap,
                  const T* PhiR, const T* x, T* y, T* ws, size_t ws_elems, const int* skip) {
  local_apply<T>(ctx, r0, r1, r0, r1, n, a0, a1, PhiL, Ap, PhiR, x, y, T(1), T(0), ws, ws_elems, skip);
}

template <typename T>
void env_left(tnfem_ctx* ctx, int ry0, int ry1, int rx0, int rx1, int n, int a0, int a1, const T* Phi,
              const T* y, const T* Ap, const T* x, T* out, T* ws, size_t ws_elems) {
  T* T1 = ws;
  T* T2 = T1 + (size_t)ry0 * a0 * n * rx1;
  T* work = T2 + (size_t)ry0 * n * a1 * rx1;
  size_t used = (size_t)(work - ws);
  TN_REQUIRE(ws_elems > used, "env_left: workspace too small");
  size_t work_elems = ws_elems - used;
  stage12<T>(ctx, ry0, rx0, rx1, n, a0, a1, Phi, Ap, x, T1, T2, work, work_elems);
  // stage 3: out[b'][(g,b)] = sum_{kappa=(a',i)} y[kappa][b'] T2[kappa][(g,b)]
  GemmDesc g3{ry1, a1 * rx1, ry0 * n, 1, 1, ry1, 0, (long long)a1 * rx1, 1, 0, (long long)a1 * rx1, 1, 0};
  gemm<T>(ctx, g3, T(1), y, T2, T(0), out, work, work_elems);
}

template <typename T>
void env_left_vec(tnfem_ctx* ctx, int ry0, int ry1, int rf0, int rf1, int n, const T* Psi, const T* y,
                  const T* f, T* out, T* ws, size_t ws_elems) {
  T* Tm = ws;
  T* work = Tm + (size_t)ry0 * n * rf1;
  size_t used = (size_t)(work - ws);
  TN_REQUIRE(ws_elems > used, "env_left_vec: workspace too small");
  size_t work_elems = ws_elems - used;
  GemmDesc g1{ry0, n * rf1, rf0, 1, rf0, 1, 0, (long long)n * rf1, 1, 0, (long long)n * rf1, 1, 0};
  gemm<T>(ctx, g1, T(1), Psi, f, T(0), Tm, work, work_elems);
  GemmDesc g2{ry1, rf1, ry0 * n, 1, 1, ry1, 0, rf1, 1, 0, rf1, 1, 0};
  gemm<T>(ctx, g2, T(1), y, Tm, T(0), out, work, work_elems);
}

template <typename T>
void local_rhs(tnfem_ctx* ctx, int r0, int n, int r1, int rf0, int rf1, const T* PsiL, const T* f,
               const T* PsiR, T* g, T* ws, size_t ws_elems, T alpha, T beta) {
  T* Tm = ws;
  T* work = Tm + (size_t)r0 * n * rf1;
  size_t used = (size_t)(work - ws);
  TN_REQUIRE(ws_elems > used, "local_rhs: workspace too small");
  size_t work_elems = ws_elems - used;
  GemmDesc g1{r0, n * rf1, rf0, 1, rf0, 1, 0, (long long)n * rf1, 1, 0, (long long)n * rf1, 1, 0};
  gemm<T>(ctx, g1, T(1), PsiL, f, T(0), Tm, work, work_elems);
  GemmDesc g2{r0 * n, r1, rf1, 1, rf1, 1, 0, 1, rf1, 0, r1, 1, 0};
  gemm<T>(ctx, g2, alpha, Tm, PsiR, beta, g, work, work_elems);
}

#define TN_INST_C(T)                                                                              \
  template void local_apply<T>(tnfem_ctx*, int, int, int, int, int, int, int, const T*, const T*,  \
                               const T*, const T*, T*, T, T, T*, size_t, const int*);             \
  template void local_matvec<T>(tnfem_ctx*, int, int, int, int, int, const T*, const T*, const T*, \
                                const T*, T*, T*, size_t, const int*);                             \
  template void env_left<T>(tnfem_ctx*, int, int, int, int, int, int, int, const T*, const T*,     \
                            const T*, const T*, T*, T*, size_t);                                   \
  template void env_left_vec<T>(tnfem_ctx*, int, int, int, int, int, const T*, const T*, const T*, \
                                T*, T*, size_t);                                                   \
  template void local_rhs<T>(tnfem_ctx*, int, int, int, int, int, const T*, const T*, const T*,    \
                             T*, T*, size_t, T, T);
TN_INST_C(double)
TN_INST_C(float)

}  // namespace tnfem
