// Dense building blocks of the sweep: strided batched GEMM (binary64 / binary32 CUDA cores),
// deterministic reductions, elementwise updates and core transposes.
//
// On GB300 binary64 runs at ~1.2 TFLOP/s for the whole chip (measured), so every binary64
// contraction is ALU-bound: the GEMM below keeps all 152 SMs busy (split-K when the output is
// small) and stages tiles through shared memory; memory traffic is secondary.
#include <algorithm>

#include "internal.h"
#include "tc_gemm.h"

namespace tnfem {

namespace {

constexpr int BM = 64, BN = 64, BK = 16, GT = 256;

// With `flat`, B is shared by all batches and the rows of a tile are the flattened (batch, m)
// pairs (row R = b * M + m), so small per-batch M does not leave tiles idle.
template <typename T>
__global__ void __launch_bounds__(GT) gemm_kernel(GemmDesc g, T alpha, const T* __restrict__ A,
                                                  const T* __restrict__ B, T beta, T* __restrict__ C,
                                                  T* __restrict__ work, int splits, int kchunk, int flat,
                                                  const int* __restrict__ skip, KTimer* __restrict__ timer) {
  if (skip && *skip) return;
  ktimer_begin(timer);
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN + 1];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int bz = blockIdx.z;
  const int b = flat ? 0 : bz / splits, sp = bz % splits;
  const int kbeg = sp * kchunk;
  const int kend = min(g.K, kbeg + kchunk);
  const long long rows = flat ? (long long)g.M * g.batch : g.M;
  const T* Ab = A + (long long)b * g.sAb;
  const T* Bb = B + (long long)b * g.sBb;
  const bool a_k_fast = (g.sAk == 1);
  const bool b_n_fast = (g.sBn == 1);
  // row offsets of this thread's four A loads (fixed over the K loop)
  long long a_off[4];
  bool a_ok[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int idx = tid + i * GT;
    const int mm = a_k_fast ? idx / BK : idx % BM;
    const long long R = m0 + mm;
    a_ok[i] = R < rows;
    const long long bb = flat ? R / g.M : 0, m = flat ? R - bb * g.M : R;
    a_off[i] = bb * g.sAb + m * g.sAm;
  }
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
  for (int k0 = kbeg; k0 < kend; k0 += BK) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      int idx = tid + i * GT;
      int mm, kk;
      if (a_k_fast) { kk = idx % BK; mm = idx / BK; } else { mm = idx % BM; kk = idx / BM; }
      int gk = k0 + kk;
      T v = T(0);
      if (a_ok[i] && gk < kend) v = Ab[a_off[i] + (long long)gk * g.sAk];
      As[kk][mm] = v;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      int idx = tid + i * GT;
      int nn, kk;
      if (b_n_fast) { nn = idx % BN; kk = idx / BN; } else { kk = idx % BK; nn = idx / BK; }
      int gn = n0 + nn, gk = k0 + kk;
      T v = T(0);
      if (gn < g.N && gk < kend) v = Bb[(long long)gk * g.sBk + (long long)gn * g.sBn];
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
  if (splits == 1) {
    T* Cb = C + (long long)b * g.sCb;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const long long R = m0 + ty + 16 * i;
      if (R >= rows) continue;
      const long long bb = flat ? R / g.M : 0, m = flat ? R - bb * g.M : R;
      T* crow = Cb + bb * g.sCb + m * g.sCm;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        int gn = n0 + tx + 16 * j;
        if (gn >= g.N) continue;
        T* c = crow + (long long)gn * g.sCn;
        T v = alpha * acc[i][j];
        if (beta != T(0)) v += beta * (*c);
        *c = v;
      }
    }
  } else {
    // partials [split][batch][M][N]; flattened rows index (batch, m) in the same order
    T* W = work + ((long long)sp * g.batch + b) * (long long)g.M * g.N;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const long long R = m0 + ty + 16 * i;
      if (R >= rows) continue;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        int gn = n0 + tx + 16 * j;
        if (gn >= g.N) continue;
        W[R * g.N + gn] = acc[i][j];
      }
    }
  }
  ktimer_end(timer);
}

// ---- binary64 GEMM in double-binary32 arithmetic ---------------------------------------------
//
// GB300 issues binary64 FMAs at 1/64 of the binary32 rate, so the large binary64 contractions of
// the mixed-precision sweep can run faster as pairs of binary32 numbers: every operand is split as
// x = hi + lo (hi = x rounded to binary32, lo = the binary32 rounding of the remainder, 48
// significant bits together), every product as a b = p + e with p = hi_a hi_b rounded and e its
// exact rounding error (an FMA) plus the cross terms hi_a lo_b + lo_a hi_b, and the sum is carried
// as (S, s): S the binary32 running sum of the p (each addition's exact rounding error recovered
// by a two-sum) and s the binary32 sum of those errors and the e.  About twelve binary32
// operations per multiply-add; the relative error of a K-term sum is about K * 2^-47 of the sum of
// |terms| (the dropped lo_a lo_b and the roundings of the small terms), against K * 2^-53 for
// binary64.  Every operation is an explicitly rounded intrinsic so that no FMA contraction can
// change the two-sum.  Values must stay inside the binary32 range: an output that is not finite
// sets *overflow, and the caller then redoes the work in binary64.
__device__ __forceinline__ float2 df_split(double x) {
  const float h = __double2float_rn(x);
  return make_float2(h, __double2float_rn(x - (double)h));
}

__device__ __forceinline__ void df_mac(float& S, float& s, const float2 a, const float2 b) {
  const float p = __fmul_rn(a.x, b.x);
  float e = __fmaf_rn(a.x, b.x, -p);
  e = __fmaf_rn(a.x, b.y, e);
  e = __fmaf_rn(a.y, b.x, e);
  const float t = __fadd_rn(S, p);
  const float z = __fsub_rn(t, S);
  const float err = __fadd_rn(__fsub_rn(S, __fsub_rn(t, z)), __fsub_rn(p, z));
  s = __fadd_rn(s, __fadd_rn(err, e));
  S = t;
}

// gemm_kernel<double> with the operands staged as (hi, lo) pairs and the sums in double-binary32
__global__ void __launch_bounds__(GT) gemm_df_kernel(GemmDesc g, double alpha, const double* __restrict__ A,
                                                     const double* __restrict__ B, double beta,
                                                     double* __restrict__ C, double* __restrict__ work,
                                                     int splits, int kchunk, int flat, const int* __restrict__ skip,
                                                     KTimer* __restrict__ timer, int* __restrict__ overflow) {
  if (skip && *skip) return;
  ktimer_begin(timer);
  __shared__ float2 As[BK][BM + 1];
  __shared__ float2 Bs[BK][BN + 1];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int bz = blockIdx.z;
  const int b = flat ? 0 : bz / splits, sp = bz % splits;
  const int kbeg = sp * kchunk;
  const int kend = min(g.K, kbeg + kchunk);
  const long long rows = flat ? (long long)g.M * g.batch : g.M;
  const double* Ab = A + (long long)b * g.sAb;
  const double* Bb = B + (long long)b * g.sBb;
  const bool a_k_fast = (g.sAk == 1);
  const bool b_n_fast = (g.sBn == 1);
  long long a_off[4];
  bool a_ok[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int idx = tid + i * GT;
    const int mm = a_k_fast ? idx / BK : idx % BM;
    const long long R = m0 + mm;
    a_ok[i] = R < rows;
    const long long bb = flat ? R / g.M : 0, m = flat ? R - bb * g.M : R;
    a_off[i] = bb * g.sAb + m * g.sAm;
  }
  float accS[4][4], accs[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      accS[i][j] = 0.0f;
      accs[i][j] = 0.0f;
    }
  for (int k0 = kbeg; k0 < kend; k0 += BK) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      int idx = tid + i * GT;
      int mm, kk;
      if (a_k_fast) { kk = idx % BK; mm = idx / BK; } else { mm = idx % BM; kk = idx / BM; }
      int gk = k0 + kk;
      double v = 0.0;
      if (a_ok[i] && gk < kend) v = Ab[a_off[i] + (long long)gk * g.sAk];
      As[kk][mm] = df_split(v);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      int idx = tid + i * GT;
      int nn, kk;
      if (b_n_fast) { nn = idx % BN; kk = idx / BN; } else { kk = idx % BK; nn = idx / BK; }
      int gn = n0 + nn, gk = k0 + kk;
      double v = 0.0;
      if (gn < g.N && gk < kend) v = Bb[(long long)gk * g.sBk + (long long)gn * g.sBn];
      Bs[kk][nn] = df_split(v);
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < BK; ++kk) {
      float2 a[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) df_mac(accS[i][j], accs[i][j], a[i], bv[j]);
    }
    __syncthreads();
  }
  bool bad = false;
  if (splits == 1) {
    double* Cb = C + (long long)b * g.sCb;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const long long R = m0 + ty + 16 * i;
      if (R >= rows) continue;
      const long long bb = flat ? R / g.M : 0, m = flat ? R - bb * g.M : R;
      double* crow = Cb + bb * g.sCb + m * g.sCm;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        int gn = n0 + tx + 16 * j;
        if (gn >= g.N) continue;
        double* c = crow + (long long)gn * g.sCn;
        double v = alpha * ((double)accS[i][j] + (double)accs[i][j]);
        if (beta != 0.0) v += beta * (*c);
        bad |= !isfinite(v);
        *c = v;
      }
    }
  } else {
    double* W = work + ((long long)sp * g.batch + b) * (long long)g.M * g.N;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const long long R = m0 + ty + 16 * i;
      if (R >= rows) continue;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        int gn = n0 + tx + 16 * j;
        if (gn >= g.N) continue;
        const double v = (double)accS[i][j] + (double)accs[i][j];
        bad |= !isfinite(v);
        W[R * g.N + gn] = v;
      }
    }
  }
  if (bad && overflow) atomicExch(overflow, 1);
  ktimer_end(timer);
}

template <typename T>
__global__ void splitk_reduce_kernel(GemmDesc g, T alpha, T beta, T* __restrict__ C,
                                     const T* __restrict__ work, int splits,
                                     const int* __restrict__ skip) {
  if (skip && *skip) return;
  long long total = (long long)g.batch * g.M * g.N;
  long long mn = (long long)g.M * g.N;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    int b = (int)(t / mn);
    long long r = t % mn;
    int m = (int)(r / g.N), n = (int)(r % g.N);
    T s = T(0);
    for (int sp = 0; sp < splits; ++sp) s += work[(long long)sp * total + t];
    T* c = C + (long long)b * g.sCb + (long long)m * g.sCm + (long long)n * g.sCn;
    T v = alpha * s;
    if (beta != T(0)) v += beta * (*c);
    *c = v;
  }
}

template <typename T>
__global__ void fill_kernel(T* x, T v, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    x[i] = v;
}

template <typename T>
__global__ void axpby_kernel(T* y, T a, const T* x, T b, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = a * x[i] + b * y[i];
}

template <typename T>
__global__ void scale_kernel(T* x, T a, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    x[i] *= a;
}

template <typename S, typename D>
__global__ void convert_kernel(D* dst, const S* src, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    dst[i] = (D)src[i];
}

template <typename T>
__global__ void dot_partial_kernel(const T* __restrict__ x, const T* __restrict__ y, size_t n,
                                   double* __restrict__ part) {
  __shared__ double sh[32];
  double s = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    s += (double)x[i] * (double)y[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
  }
}

__global__ void sum_partials_kernel(const double* __restrict__ part, int np, double* __restrict__ out) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) s += part[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) *out = s;
  }
}

template <typename T>
__global__ void transpose3_kernel(T* __restrict__ out, const T* __restrict__ in, int A, int B, int C) {
  long long total = (long long)A * B * C;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    int c = (int)(t % C);
    long long r = t / C;
    int b = (int)(r % B);
    int a = (int)(r / B);
    out[((long long)c * B + b) * A + a] = in[t];
  }
}

template <typename T>
__global__ void transpose4_outer_kernel(T* __restrict__ out, const T* __restrict__ in, int A, int B,
                                        int C, int D) {
  long long total = (long long)A * B * C * D;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    int d = (int)(t % D);
    long long r = t / D;
    int c = (int)(r % C);
    r /= C;
    int b = (int)(r % B);
    int a = (int)(r / B);
    out[(((long long)d * B + b) * C + c) * A + a] = in[t];
  }
}

template <typename T>
__global__ void transpose4_mid_kernel(T* __restrict__ out, const T* __restrict__ in, int A, int B,
                                      int C, int D) {
  long long total = (long long)A * B * C * D;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    int d = (int)(t % D);
    long long r = t / D;
    int c = (int)(r % C);
    r /= C;
    int b = (int)(r % B);
    int a = (int)(r / B);
    out[(((long long)a * C + c) * B + b) * D + d] = in[t];
  }
}

template <typename T>
__global__ void transpose2_kernel(T* __restrict__ out, const T* __restrict__ in, int m, int n) {
  __shared__ T tile[32][33];
  int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  for (int j = threadIdx.y; j < 32; j += 8) {
    int r = by + j, c = bx + threadIdx.x;
    if (r < m && c < n) tile[j][threadIdx.x] = in[(long long)r * n + c];
  }
  __syncthreads();
  for (int j = threadIdx.y; j < 32; j += 8) {
    int r = bx + j, c = by + threadIdx.x;
    if (r < n && c < m) out[(long long)r * m + c] = tile[threadIdx.x][j];
  }
}

inline int grid_for(size_t n, int threads = 256) {
  size_t b = (n + threads - 1) / threads;
  return (int)std::max<size_t>(1, std::min<size_t>(b, 152 * 16));
}

}  // namespace

void check_launch(tnfem_ctx* ctx, const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) throw Error(TNFEM_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

template <typename T>
void gemm(tnfem_ctx* ctx, const GemmDesc& g, T alpha, const T* A, const T* B, T beta, T* C, T* work,
          size_t work_elems, const int* skip) {
  if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return;
  if (g.K <= 0) {
    // C = beta * C
    GemmDesc z = g;
    z.K = 1;
    // a zero-K product: scale C through the reduce kernel with zero partials is overkill;
    // handle with a tiny loop over batches (rare).
    for (int b = 0; b < g.batch; ++b) {
      if (g.sCn == 1 && g.sCm == g.N) {
        if (beta == T(0)) fill<T>(ctx, C + (long long)b * g.sCb, T(0), (size_t)g.M * g.N);
        else scale<T>(ctx, C + (long long)b * g.sCb, beta, (size_t)g.M * g.N);
      } else {
        throw Error(TNFEM_E_INVALID, "gemm with K=0 on a strided output");
      }
    }
    return;
  }
  if constexpr (sizeof(T) == 4) {
    if (ctx->tensor_cores && tc_gemm_supported(g)) {
      tc_gemm(ctx, g, alpha, A, B, beta, C, work, work_elems, skip);
      return;
    }
  }
  const int flat = (g.sBb == 0 && g.batch > 1) ? 1 : 0;
  const long long rows = flat ? (long long)g.M * g.batch : g.M;
  int tiles_m = (int)((rows + BM - 1) / BM), tiles_n = (g.N + BN - 1) / BN;
  long long tiles = (long long)tiles_m * tiles_n * (flat ? 1 : g.batch);
  int splits = 1;
  // split K when the tiles alone give the SMs fewer than two CTAs each and K is long (the partial
  // sums cost a second kernel).  Aiming at two CTAs per SM rather than one measured 525 ms per
  // 2^10 x 2^10 solve against 563 ms (binary64 contractions 201 -> 182 ms, reduces 53 -> 48 ms)
  const long long target = 304;
  int kchunk = g.K;
  if constexpr (sizeof(T) == 8) {
    // binary64: one CTA already keeps an SM's FP64 pipe busy (ncu: 92-98% active with one CTA
    // resident), so an SM's time is the sum of its CTAs' K steps.  Take the split that minimises
    // the busiest SM's steps, ceil(CTAs / SMs) x ceil(ceil(K / s) / BK), the fewest splits on ties
    // (each split adds partial sums to reduce).
    const long long fit = work ? (long long)(work_elems / ((size_t)g.batch * g.M * g.N)) : 1;
    const long long smax = std::max(1ll, std::min({64ll, fit, (long long)((g.K + BK - 1) / BK)}));
    long long best = -1;
    for (long long sp = 1; sp <= smax; ++sp) {
      const long long kc = (g.K + sp - 1) / sp;
      const long long cost = ((tiles * sp + 151) / 152) * ((kc + BK - 1) / BK);
      if (best < 0 || cost < best) {
        best = cost;
        splits = (int)sp;
      }
    }
    kchunk = (g.K + splits - 1) / splits;
    splits = (g.K + kchunk - 1) / kchunk;
  } else {
    if (work && tiles < target && g.K >= 8 * BK) {
      long long want = (target + tiles - 1) / tiles;
      long long maxs = g.K / (2 * BK);
      long long fit = (long long)(work_elems / ((size_t)g.batch * g.M * g.N));
      splits = (int)std::max<long long>(1, std::min(std::min(want, maxs), std::min(fit, (long long)64)));
    }
    kchunk = (g.K + splits - 1) / splits;
    kchunk = ((kchunk + BK - 1) / BK) * BK;
    splits = (g.K + kchunk - 1) / kchunk;
  }
  dim3 grid(tiles_n, tiles_m, (flat ? 1 : g.batch) * splits);
  TN_REQUIRE((flat ? 1 : g.batch) * (long long)splits < 65536 && tiles_m < 65536, "gemm: grid too large");
  {
    const double mnk = (double)g.M * g.N * g.K * g.batch;
    const double words = ((double)g.M * g.K + (double)g.K * g.N + (double)g.M * g.N) * g.batch;
    const int cls = sizeof(T) == 8 ? TNFEM_PROF_CONTRACT64 : TNFEM_PROF_CONTRACT32;
    KTimer* timer = prof_ktimer(ctx, cls, 2.0 * mnk, words * sizeof(T));
    ProfScope ps(ctx, cls, 2.0 * mnk, words * sizeof(T), timer != nullptr);
    if constexpr (sizeof(T) == 8) {
      if (ctx->df64 && mnk >= kDfMinMnk) {
        gemm_df_kernel<<<grid, GT, 0, ctx->stream>>>(g, alpha, A, B, beta, C, work, splits, kchunk, flat, skip, timer,
                                                     df_overflow_flag(ctx));
      } else {
        gemm_kernel<T><<<grid, GT, 0, ctx->stream>>>(g, alpha, A, B, beta, C, work, splits, kchunk, flat, skip, timer);
      }
    } else {
      gemm_kernel<T><<<grid, GT, 0, ctx->stream>>>(g, alpha, A, B, beta, C, work, splits, kchunk, flat, skip, timer);
    }
  }
  count_launch(ctx);
  if (splits > 1) {
    long long total = (long long)g.batch * g.M * g.N;
    ProfScope ps(ctx, TNFEM_PROF_OTHER, (double)total * splits, (double)total * (splits + 1) * sizeof(T));
    splitk_reduce_kernel<T><<<grid_for(total), 256, 0, ctx->stream>>>(g, alpha, beta, C, work, splits, skip);
    count_launch(ctx);
  }
  check_launch(ctx, "gemm");
}

template <typename T>
void splitk_reduce(tnfem_ctx* ctx, const GemmDesc& g, T alpha, T beta, T* C, const T* work, int splits,
                   const int* skip) {
  long long total = (long long)g.batch * g.M * g.N;
  ProfScope ps(ctx, TNFEM_PROF_OTHER, (double)total * splits, (double)total * (splits + 1) * sizeof(T));
  splitk_reduce_kernel<T><<<grid_for(total), 256, 0, ctx->stream>>>(g, alpha, beta, C, work, splits, skip);
  count_launch(ctx);
}

template <typename T> void fill(tnfem_ctx* ctx, T* x, T v, size_t n) {
  if (!n) return;
  fill_kernel<T><<<grid_for(n), 256, 0, ctx->stream>>>(x, v, n);
  count_launch(ctx);
  check_launch(ctx, "fill");
}
template <typename T> void copy(tnfem_ctx* ctx, T* dst, const T* src, size_t n) {
  if (!n || dst == src) return;
  TN_CHECK_CUDA(cudaMemcpyAsync(dst, src, n * sizeof(T), cudaMemcpyDeviceToDevice, ctx->stream));
}
template <typename T> void axpby(tnfem_ctx* ctx, T* y, T a, const T* x, T b, size_t n) {
  if (!n) return;
  axpby_kernel<T><<<grid_for(n), 256, 0, ctx->stream>>>(y, a, x, b, n);
  count_launch(ctx);
  check_launch(ctx, "axpby");
}
template <typename T> void scale(tnfem_ctx* ctx, T* x, T a, size_t n) {
  if (!n) return;
  scale_kernel<T><<<grid_for(n), 256, 0, ctx->stream>>>(x, a, n);
  count_launch(ctx);
  check_launch(ctx, "scale");
}
void convert_d2f(tnfem_ctx* ctx, float* dst, const double* src, size_t n) {
  if (!n) return;
  convert_kernel<double, float><<<grid_for(n), 256, 0, ctx->stream>>>(dst, src, n);
  count_launch(ctx);
  check_launch(ctx, "convert");
}
void convert_f2d(tnfem_ctx* ctx, double* dst, const float* src, size_t n) {
  if (!n) return;
  convert_kernel<float, double><<<grid_for(n), 256, 0, ctx->stream>>>(dst, src, n);
  count_launch(ctx);
  check_launch(ctx, "convert");
}
template <typename T> void dot_partials(tnfem_ctx* ctx, const T* x, const T* y, size_t n, double* part) {
  dot_partial_kernel<T><<<kReduceBlocks, 256, 0, ctx->stream>>>(x, y, n, part);
  count_launch(ctx);
  check_launch(ctx, "dot");
}
template <typename T> double dot(tnfem_ctx* ctx, const T* x, const T* y, size_t n) {
  if (!n) return 0.0;
  double* part = ctx->scratch;
  double* out = ctx->scratch + kReduceBlocks;
  dot_partials<T>(ctx, x, y, n, part);
  sum_partials_kernel<<<1, 256, 0, ctx->stream>>>(part, kReduceBlocks, out);
  count_launch(ctx);
  check_launch(ctx, "dot sum");
  TN_CHECK_CUDA(cudaMemcpyAsync(ctx->host_pinned, out, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  sync(ctx);
  return ctx->host_pinned[0];
}
template <typename T> double nrm2(tnfem_ctx* ctx, const T* x, size_t n) {
  double s = dot<T>(ctx, x, x, n);
  return s > 0 ? sqrt(s) : 0.0;
}
template <typename T> void transpose3(tnfem_ctx* ctx, T* out, const T* in, int A, int B, int C) {
  size_t n = (size_t)A * B * C;
  if (!n) return;
  transpose3_kernel<T><<<grid_for(n), 256, 0, ctx->stream>>>(out, in, A, B, C);
  count_launch(ctx);
  check_launch(ctx, "transpose3");
}
template <typename T> void transpose4_outer(tnfem_ctx* ctx, T* out, const T* in, int A, int B, int C, int D) {
  size_t n = (size_t)A * B * C * D;
  if (!n) return;
  transpose4_outer_kernel<T><<<grid_for(n), 256, 0, ctx->stream>>>(out, in, A, B, C, D);
  count_launch(ctx);
  check_launch(ctx, "transpose4");
}
template <typename T> void transpose4_mid(tnfem_ctx* ctx, T* out, const T* in, int A, int B, int C, int D) {
  size_t n = (size_t)A * B * C * D;
  if (!n) return;
  transpose4_mid_kernel<T><<<grid_for(n), 256, 0, ctx->stream>>>(out, in, A, B, C, D);
  count_launch(ctx);
  check_launch(ctx, "transpose4mid");
}
template <typename T> void transpose2(tnfem_ctx* ctx, T* out, const T* in, int m, int n) {
  if (!m || !n) return;
  dim3 grid((n + 31) / 32, (m + 31) / 32);
  transpose2_kernel<T><<<grid, dim3(32, 8), 0, ctx->stream>>>(out, in, m, n);
  count_launch(ctx);
  check_launch(ctx, "transpose2");
}

template void splitk_reduce<double>(tnfem_ctx*, const GemmDesc&, double, double, double*, const double*, int,
                                    const int*);
template void splitk_reduce<float>(tnfem_ctx*, const GemmDesc&, float, float, float*, const float*, int, const int*);

#define TN_INST(T)                                                                              \
  template void gemm<T>(tnfem_ctx*, const GemmDesc&, T, const T*, const T*, T, T*, T*, size_t,    \
                        const int*);                                                             \
  template void fill<T>(tnfem_ctx*, T*, T, size_t);                                             \
  template void copy<T>(tnfem_ctx*, T*, const T*, size_t);                                      \
  template void axpby<T>(tnfem_ctx*, T*, T, const T*, T, size_t);                               \
  template void scale<T>(tnfem_ctx*, T*, T, size_t);                                            \
  template void dot_partials<T>(tnfem_ctx*, const T*, const T*, size_t, double*);               \
  template double dot<T>(tnfem_ctx*, const T*, const T*, size_t);                               \
  template double nrm2<T>(tnfem_ctx*, const T*, size_t);                                        \
  template void transpose3<T>(tnfem_ctx*, T*, const T*, int, int, int);                         \
  template void transpose4_outer<T>(tnfem_ctx*, T*, const T*, int, int, int, int);              \
  template void transpose4_mid<T>(tnfem_ctx*, T*, const T*, int, int, int, int);                \
  template void transpose2<T>(tnfem_ctx*, T*, const T*, int, int);
TN_INST(double)
TN_INST(float)

}  // namespace tnfem
