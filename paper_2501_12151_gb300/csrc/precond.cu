// Block-Jacobi preconditioner of the local systems of the sweep (step a5).
//
// The local matrix of core k is B = sum_{beta,gamma} PhiL[:,beta,:] (x) A_k[beta,:,:,gamma] (x)
// PhiR[:,gamma,:], acting on a core x[a][j][b].  Its diagonal blocks in the right bond index b,
//
//   P_b[(a',i),(a,j)] = sum_{beta,gamma} PhiL[a',beta,a] A_k[beta,i,j,gamma] PhiR[b,gamma,b],
//
// are principal submatrices of the symmetric positive definite B, hence SPD themselves; the
// preconditioner is M^{-1} = blockdiag_b(P_b^{-1}).  The blocks keep the left interface and the
// current core exactly and the right interface only through its diagonal, which is where most of
// the fine-level ill-conditioning of the QTT elasticity operator sits in a left-to-right sweep.
//
// Set-up: two GEMMs form all blocks at once, a permutation kernel gathers and symmetrises them
// into [b][(a',i)][(a,j)] binary32 storage, and one CTA per block inverts it by Gauss-Jordan
// elimination without pivoting (stable for SPD matrices).  Apply: one CTA per block multiplies
// the block inverse with the block's strided slice of the residual, fused with the partial sums
// of r.z that conjugate gradients needs.
#include <atomic>
#include <algorithm>

#include "internal.h"
#include "precond.h"

namespace tnfem {

namespace {

constexpr int PT = 256;
constexpr size_t kInvertSmemMax = 220 * 1024;  // blocks up to this size are inverted in shared memory

// dR[b][g] = PhiR[b][g][b]
template <typename T>
__global__ void bj_diag_kernel(const T* __restrict__ PhiR, int r1, int a1, T* __restrict__ dR) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < r1 * a1; t += gridDim.x * blockDim.x) {
    int b = t / a1, g = t % a1;
    dR[t] = PhiR[((long long)b * a1 + g) * r1 + b];
  }
}

// Pb[b][(a',i)][(a,j)] = 0.5 (Pfull[a'][a][j][i][b] + Pfull[a][a'][i][j][b])
template <typename T>
__global__ void bj_gather_kernel(float* __restrict__ Pb, const T* __restrict__ Pfull, int r0, int n, int r1) {
  const int m = r0 * n;
  const long long total = (long long)r1 * m * m;
  const long long s_a = (long long)r0 * n * n * r1;  // stride of a' in Pfull
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int q = (int)(t % m);
    const long long rest = t / m;
    const int p = (int)(rest % m);
    const int b = (int)(rest / m);
    const int ap = p / n, i = p % n, a = q / n, j = q % n;
    const T v1 = Pfull[ap * s_a + (((long long)a * n + j) * n + i) * r1 + b];
    const T v2 = Pfull[a * s_a + (((long long)ap * n + i) * n + j) * r1 + b];
    Pb[t] = (float)(0.5 * ((double)v1 + (double)v2));
  }
}

// In-place Gauss-Jordan inversion of the m x m block blockIdx.x (SPD, no pivoting).  A pivot
// that is not positive marks the block as failed in flag[0]; its contents are then meaningless
// and the caller does not use the preconditioner.  With `in_smem` the block is copied into shared
// memory for the elimination and written back at the end.
__global__ void __launch_bounds__(1024) bj_invert_kernel(float* __restrict__ Pb, int m, int* __restrict__ flag,
                                                         int in_smem) {
  extern __shared__ float sh[];
  float* col = sh;       // column k before the step
  float* rowk = sh + m;  // row k after scaling
  float* Mg = Pb + (long long)blockIdx.x * m * m;
  float* M = in_smem ? sh + 2 * m : Mg;
  const long long mm = (long long)m * m;
  if (in_smem) {
    for (long long t = threadIdx.x; t < mm; t += blockDim.x) M[t] = Mg[t];
    __syncthreads();
  }
  __shared__ float s_p;
  for (int k = 0; k < m; ++k) {
    for (int i = threadIdx.x; i < m; i += blockDim.x) col[i] = M[(long long)i * m + k];
    __syncthreads();
    if (threadIdx.x == 0) {
      const float piv = col[k];
      if (!(piv > 0.0f) || !isfinite(piv)) {
        atomicExch(flag, 1);
        s_p = 0.0f;
      } else {
        s_p = 1.0f / piv;
      }
    }
    __syncthreads();
    const float p = s_p;
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
      const float v = (j == k ? 1.0f : M[(long long)k * m + j]) * p;
      rowk[j] = v;
      M[(long long)k * m + j] = v;
    }
    __syncthreads();
    // rows i != k: M[i][j] = (j == k ? 0 : M[i][j]) - col[i] rowk[j]; threads walk (i, j) with
    // j fastest, stepping i and j incrementally
    int i = threadIdx.x / m, j = threadIdx.x % m;
    const int di = blockDim.x / m, dj = blockDim.x % m;
    for (long long t = threadIdx.x; t < mm; t += blockDim.x) {
      if (i != k) {
        const float old = (j == k) ? 0.0f : M[t];
        M[t] = old - col[i] * rowk[j];
      }
      i += di;
      j += dj;
      if (j >= m) { j -= m; ++i; }
    }
    __syncthreads();
  }
  if (in_smem) {
    for (long long t = threadIdx.x; t < mm; t += blockDim.x) Mg[t] = M[t];
  }
}

// z[(a',i)][b] = sum_q Pinv_b[(a',i)][q] r[q][b]; partial sums of r.z per CTA into part[blockIdx.x]
// (every one of the gridDim.x entries is written); with p_out != nullptr also p = z.  CTA c takes
// block b = c % r1 and the row slice c / r1 of `split` equal slices, so a preconditioner block is
// spread over `split` CTAs.
template <typename T>
__global__ void __launch_bounds__(PT) bj_apply_kernel(const float* __restrict__ Pinv, const T* __restrict__ r,
                                                      T* __restrict__ z, T* __restrict__ p_out, int m, int r1,
                                                      int split, double* __restrict__ part,
                                                      const int* __restrict__ ctl) {
  if (ctl && ctl[0]) return;
  // The block products run in binary32 for either precision of the solve: the preconditioner is
  // only an approximation of B^{-1}, and binary64 FMA throughput is scarce on this part.  The r.z
  // partials that conjugate gradients needs are accumulated in binary64 from the stored values.
  extern __shared__ float rbf[];  // m values of this block's slice of r
  __shared__ double red[PT / 32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double acc_rz = 0.0;
  const int per = (m + split - 1) / split;
  for (int c = blockIdx.x; c < r1 * split; c += gridDim.x) {
    const int b = c % r1, slice = c / r1;
    const int row0 = slice * per, row1 = min(m, row0 + per);
    __syncthreads();
    for (int q = threadIdx.x; q < m; q += blockDim.x) rbf[q] = (float)r[(long long)q * r1 + b];
    __syncthreads();
    const float* P = Pinv + (long long)b * m * m;
    for (int row = row0 + warp; row < row1; row += PT / 32) {
      const float* pr = P + (long long)row * m;
      float s = 0.f;
      for (int q = lane; q < m; q += 32) s = fmaf(pr[q], rbf[q], s);
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) {
        const T zv = (T)s;
        z[(long long)row * r1 + b] = zv;
        if (p_out) p_out[(long long)row * r1 + b] = zv;
        acc_rz += (double)r[(long long)row * r1 + b] * (double)zv;
      }
    }
  }
  // lane 0 of each warp holds a partial; reduce over warps
  if (lane == 0) red[warp] = acc_rz;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < PT / 32; ++w) t += red[w];
    part[blockIdx.x] = t;
  }
}

}  // namespace

bool bj_fits(int r0, int n, int r1) {
  const long long m = (long long)r0 * n;
  return m <= kBlockJacobiMaxM && (long long)r1 * m * m <= kBlockJacobiMaxElems;
}

bool bj_worth_it(int r0, int n) {
  const size_t m = (size_t)r0 * n;
  return (m * m + 2 * m) * sizeof(float) <= kInvertSmemMax || m <= 512;
}

size_t bj_work_elems(int r0, int n, int r1, int a0, int a1) {
  const size_t m = (size_t)r0 * n;
  const size_t t1 = (size_t)a0 * n * n * r1;
  const size_t full = (size_t)r1 * m * m;
  return (size_t)r1 * a1 + t1 + full + 64;
}

template <typename T>
bool bj_setup(tnfem_ctx* ctx, int r0, int n, int r1, int a0, int a1, const T* PhiL, const T* Ap, const T* PhiR,
              float* Pinv, T* work, size_t work_elems, int* flag) {
  if (!bj_fits(r0, n, r1)) return false;
  TN_REQUIRE(work_elems >= bj_work_elems(r0, n, r1, a0, a1), "block-Jacobi workspace too small");
  const int m = r0 * n;
  T* dR = work;
  T* T1 = dR + (size_t)r1 * a1;
  T* Pfull = T1 + (size_t)a0 * n * n * r1;
  {
    ProfScope ps(ctx, TNFEM_PROF_OTHER, 0.0, (double)r1 * a1 * sizeof(T));
    bj_diag_kernel<T><<<std::max(1, std::min(152, (r1 * a1 + 255) / 256)), 256, 0, ctx->stream>>>(PhiR, r1, a1, dR);
    count_launch(ctx);
  }
  // T1[(beta,j,i)][b] = sum_g Ap[(beta,j,i)][g] dR[b][g]
  GemmDesc g1{a0 * n * n, r1, a1, 1, a1, 1, 0, 1, a1, 0, r1, 1, 0};
  gemm<T>(ctx, g1, T(1), Ap, dR, T(0), T1);
  // Pfull[a'][a][(j,i,b)] = sum_beta PhiL[a'][beta][a] T1[beta][(j,i,b)]   (batch a')
  const long long nb = (long long)n * n * r1;
  GemmDesc g2{r0, (int)nb, a0, r0, 1, r0, (long long)a0 * r0, nb, 1, 0, nb, 1, (long long)r0 * nb};
  gemm<T>(ctx, g2, T(1), PhiL, T1, T(0), Pfull);
  const long long total = (long long)r1 * m * m;
  {
    ProfScope ps(ctx, TNFEM_PROF_OTHER, 0.0, (double)total * (2 * sizeof(T) + sizeof(float)));
    bj_gather_kernel<T><<<(int)std::min<long long>(152 * 8, (total + 255) / 256), 256, 0, ctx->stream>>>(Pinv, Pfull,
                                                                                                        r0, n, r1);
    count_launch(ctx);
  }
  TN_CHECK_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), ctx->stream));
  {
    // the block stays on chip for the elimination when it fits
    const size_t smem_full = ((size_t)m * m + 2 * m) * sizeof(float);
    const int in_smem = smem_full <= kInvertSmemMax ? 1 : 0;
    static std::atomic<unsigned long long> attr_set{0};  // one bit per device
    const unsigned long long bit = 1ull << (ctx->device & 63);
    if (in_smem && !(attr_set & bit)) {
      TN_CHECK_CUDA(cudaFuncSetAttribute(bj_invert_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kInvertSmemMax));
      attr_set |= bit;
    }
    ProfScope ps(ctx, TNFEM_PROF_OTHER, 2.0 * r1 * (double)m * m * m, (double)total * sizeof(float));
    bj_invert_kernel<<<r1, 1024, in_smem ? smem_full : 2 * m * sizeof(float), ctx->stream>>>(Pinv, m, flag, in_smem);
    count_launch(ctx);
  }
  check_launch(ctx, "block-Jacobi set-up");
  int h = 0;
  TN_CHECK_CUDA(cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  sync(ctx);
  return h == 0;
}

template <typename T>
void bj_apply(tnfem_ctx* ctx, int r0, int n, int r1, const float* Pinv, const T* r, T* z, T* p_out, double* part,
              const int* ctl, int nblocks) {
  const int m = r0 * n;
  ProfScope ps(ctx, TNFEM_PROF_KRYLOV, 2.0 * r1 * (double)m * m, (double)r1 * m * m * sizeof(float));
  const int split = std::max(1, nblocks / std::max(1, r1));
  bj_apply_kernel<T><<<nblocks, PT, m * sizeof(float), ctx->stream>>>(Pinv, r, z, p_out, m, r1, split, part, ctl);
  count_launch(ctx);
}

template bool bj_setup<double>(tnfem_ctx*, int, int, int, int, int, const double*, const double*, const double*,
                               float*, double*, size_t, int*);
template bool bj_setup<float>(tnfem_ctx*, int, int, int, int, int, const float*, const float*, const float*, float*,
                              float*, size_t, int*);
template void bj_apply<double>(tnfem_ctx*, int, int, int, const float*, const double*, double*, double*, double*,
                               const int*, int);
template void bj_apply<float>(tnfem_ctx*, int, int, int, const float*, const float*, float*, float*, double*,
                              const int*, int);

}  // namespace tnfem
