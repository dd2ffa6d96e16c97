// Dense factorizations used by the sweep's orthogonalisation and truncation steps:
// Householder QR (the reduced QR of Section 4, Eq. qr) and the one-sided Jacobi (Hestenes)
// SVD used for TT truncation.  Binary64 runs at ~2 FMAs per clock per SM on this part, so the
// larger factorizations are spread over SMs: a thread-block cluster with the columns in
// distributed shared memory (qr_cluster_kernel, svd_cluster_kernel) or a cooperative grid with a
// bounded grid barrier (svd_coop_kernel, qr_ext_coop_kernel); small ones run on one CTA
// (qr_kernel, qr_blk_kernel, svd_kernel).  Cluster and CTA barriers are hardware barriers that
// every thread reaches the same number of times; the grid barriers give up after a bounded wait
// and report it.
#include <atomic>
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cfloat>

#include <cooperative_groups.h>

#include "grid_sync.cuh"
#include "internal.h"

namespace tnfem {

namespace {

constexpr int LT = 1024;
constexpr size_t kSvdSmemMax = 200 * 1024;  // working copies of the Jacobi SVD up to this size stay on chip
constexpr int kSvdCoopMinN = 16;             // binary64 SVDs with at least this many columns use svd_coop_kernel

template <typename T> __device__ __forceinline__ T eps_of();
template <> __device__ __forceinline__ double eps_of<double>() { return 2.220446049250313e-16; }
template <> __device__ __forceinline__ float eps_of<float>() { return 1.1920929e-7f; }

template <typename T>
__device__ T block_sum(T v, T* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  if (w == 0) {
    v = (l < (int)(blockDim.x >> 5)) ? sh[l] : T(0);
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (l == 0) sh[32] = v;
  }
  __syncthreads();
  return sh[32];
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// A: m x n row-major, overwritten by the Householder vectors (below the diagonal) and R.
// tau: k scalars.  Q: m x k row-major (explicit), R: k x n row-major.
// The whole CTA (any multiple of 32 threads) takes part.
template <typename T>
__device__ void qr_body(int m, int n, T* __restrict__ A, T* __restrict__ Q, T* __restrict__ R, T* __restrict__ tau) {
  __shared__ T sh[33];
  __shared__ T s_beta, s_tau, s_v0;
  const int k = min(m, n);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int j = 0; j < k; ++j) {
    T part = T(0);
    for (int i = j + 1 + threadIdx.x; i < m; i += blockDim.x) {
      T v = A[(long long)i * n + j];
      part += v * v;
    }
    T tail = block_sum(part, sh);
    if (threadIdx.x == 0) {
      T alpha = A[(long long)j * n + j];
      if (tail == T(0)) {
        s_tau = T(0);
        s_beta = alpha;
        s_v0 = T(1);
      } else {
        T nx = sqrt(alpha * alpha + tail);
        T beta = alpha >= T(0) ? -nx : nx;
        s_tau = (beta - alpha) / beta;
        s_v0 = alpha - beta;
        s_beta = beta;
      }
      tau[j] = s_tau;
    }
    __syncthreads();
    const T tj = s_tau, v0 = s_v0;
    // scale the vector: v = [1, x_{j+1..}/v0]
    if (tj != T(0)) {
      for (int i = j + 1 + threadIdx.x; i < m; i += blockDim.x) A[(long long)i * n + j] /= v0;
    }
    __syncthreads();
    if (threadIdx.x == 0) A[(long long)j * n + j] = s_beta;
    // apply H = I - tau v v^T to trailing columns, one warp per column
    if (tj != T(0)) {
      for (int c = j + 1 + warp; c < n; c += nw) {
        T w = T(0);
        for (int i = j + lane; i < m; i += 32) {
          T vi = (i == j) ? T(1) : A[(long long)i * n + j];
          w += vi * A[(long long)i * n + c];
        }
        w = warp_sum(w) * tj;
        for (int i = j + lane; i < m; i += 32) {
          T vi = (i == j) ? T(1) : A[(long long)i * n + j];
          A[(long long)i * n + c] -= w * vi;
        }
      }
    }
    __syncthreads();
  }
  // R = upper triangle of the first k rows
  for (long long t = threadIdx.x; t < (long long)k * n; t += blockDim.x) {
    int i = (int)(t / n), c = (int)(t % n);
    R[t] = (c >= i) ? A[(long long)i * n + c] : T(0);
  }
  // Q = H_0 ... H_{k-1} [I_k; 0]
  for (long long t = threadIdx.x; t < (long long)m * k; t += blockDim.x) {
    int i = (int)(t / k), c = (int)(t % k);
    Q[t] = (i == c) ? T(1) : T(0);
  }
  __syncthreads();
  for (int j = k - 1; j >= 0; --j) {
    const T tj = tau[j];
    if (tj == T(0)) continue;
    for (int c = j + warp; c < k; c += nw) {
      T w = T(0);
      for (int i = j + lane; i < m; i += 32) {
        T vi = (i == j) ? T(1) : A[(long long)i * n + j];
        w += vi * Q[(long long)i * k + c];
      }
      w = warp_sum(w) * tj;
      for (int i = j + lane; i < m; i += 32) {
        T vi = (i == j) ? T(1) : A[(long long)i * n + j];
        Q[(long long)i * k + c] -= w * vi;
      }
    }
    __syncthreads();
  }
}

template <typename T>
__global__ void __launch_bounds__(LT) qr_kernel(int m, int n, T* __restrict__ A, T* __restrict__ Q,
                                                T* __restrict__ R, T* __restrict__ tau) {
  qr_body(m, n, A, Q, R, tau);
}

// Blocked Householder QR for m >= n (the same reflectors as qr_body, grouped into panels of nb
// columns in the compact WY form H_p0 ... H_p0+nb-1 = I - V T V^T).  The matrix is transposed into
// the Q buffer (column-major, W[c][i] = A[i][c], so every column access is coalesced).  Each panel
// is factorised in shared memory (nb x m), T is formed from tau and V^T V, and the trailing
// columns take the whole panel at once, A_c <- (I - V T^T V^T) A_c: two passes over each
// trailing column per panel instead of two per reflector, with nb independent sums in flight.
// Q = prod_p (I - V_p T_p V_p^T) [I; 0] is accumulated column-major in the A buffer, panels
// last to first, and transposed into Q.
constexpr int kQrNbMax = 8;
constexpr size_t kQrBlkMinElems = 32768;      // smaller matrices stay on qr_kernel
constexpr int kQrClMinN = 16;                 // QRs with at least this many columns go to the cluster kernel
constexpr size_t kQrClSmemMax = 200 * 1024;   // its columns, Q columns and reflector on chip
constexpr size_t kQrSmemMax = 200 * 1024;  // panel of qr_blk_kernel on chip
constexpr int QBT = 512;                   // threads of qr_blk_kernel

template <typename T>
__device__ void qr_blk_load_v(int m, int p0, int pb, const T* __restrict__ W, T* __restrict__ Vs) {
  // panel columns with the reflector form: zero above the diagonal, unit diagonal, vector below
  for (long long t = threadIdx.x; t < (long long)pb * m; t += blockDim.x) {
    const int c = (int)(t / m), i = (int)(t % m);
    const int j = p0 + c;
    Vs[t] = (i < j) ? T(0) : (i == j ? T(1) : W[(long long)j * m + i]);
  }
}

// T (pb x pb, upper triangular, row-major in Ts) of the panel whose vectors are in Vs.
template <typename T>
__device__ void qr_blk_form_t(int m, int p0, int pb, const T* __restrict__ Vs, const T* __restrict__ tau,
                              T* __restrict__ Ys, T* __restrict__ Ts) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int pr = warp; pr < pb * pb; pr += nw) {
    const int a = pr / pb, b = pr % pb;
    if (a >= b) continue;
    const T* va = Vs + (long long)a * m;
    const T* vb = Vs + (long long)b * m;
    T y = T(0);
    for (int i = p0 + b + lane; i < m; i += 32) y += va[i] * vb[i];
    y = warp_sum(y);
    if (lane == 0) Ys[a * kQrNbMax + b] = y;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int b = 0; b < pb; ++b) {
      const T tb = tau[p0 + b];
      Ts[b * kQrNbMax + b] = tb;
      for (int a = 0; a < b; ++a) {
        T acc = T(0);
        for (int c = a; c < b; ++c) acc += Ts[a * kQrNbMax + c] * Ys[c * kQrNbMax + b];
        Ts[a * kQrNbMax + b] = -tb * acc;
      }
    }
  }
  __syncthreads();
}

template <typename T>
__device__ __forceinline__ void qr_blk_body(int m, int n, int nb, T* __restrict__ A, T* __restrict__ Q,
                                            T* __restrict__ R, T* __restrict__ tau) {
  extern __shared__ __align__(16) unsigned char qb_smem[];
  T* Vs = reinterpret_cast<T*>(qb_smem);  // [nb][m] the current panel
  __shared__ T sh[33];
  __shared__ T s_beta, s_tau, s_v0;
  __shared__ T Ys[kQrNbMax * kQrNbMax], Ts[kQrNbMax * kQrNbMax];
  const int k = n;  // m >= n
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  T* W = Q;
  for (long long t = threadIdx.x; t < (long long)m * n; t += blockDim.x) {
    const int c = (int)(t / m), i = (int)(t % m);
    W[t] = A[(long long)i * n + c];
  }
  __syncthreads();
  for (int p0 = 0; p0 < k; p0 += nb) {
    const int pb = min(nb, k - p0);
    for (long long t = threadIdx.x; t < (long long)pb * m; t += blockDim.x) Vs[t] = W[(long long)p0 * m + t];
    __syncthreads();
    // unblocked Householder steps inside the panel
    for (int jj = 0; jj < pb; ++jj) {
      const int j = p0 + jj;
      T* vj = Vs + (long long)jj * m;
      T part = T(0);
      for (int i = j + 1 + threadIdx.x; i < m; i += blockDim.x) {
        const T v = vj[i];
        part += v * v;
      }
      const T tail = block_sum(part, sh);
      if (threadIdx.x == 0) {
        const T alpha = vj[j];
        if (tail == T(0)) {
          s_tau = T(0);
          s_beta = alpha;
          s_v0 = T(1);
        } else {
          const T nx = sqrt(alpha * alpha + tail);
          const T beta = alpha >= T(0) ? -nx : nx;
          s_tau = (beta - alpha) / beta;
          s_v0 = alpha - beta;
          s_beta = beta;
        }
        tau[j] = s_tau;
      }
      __syncthreads();
      const T tj = s_tau, v0 = s_v0;
      if (tj != T(0))
        for (int i = j + 1 + threadIdx.x; i < m; i += blockDim.x) vj[i] /= v0;
      __syncthreads();
      if (tj != T(0)) {
        for (int cc = jj + 1 + warp; cc < pb; cc += nw) {
          T* vc = Vs + (long long)cc * m;
          T w = (lane == 0) ? vc[j] : T(0);  // the unit entry of v at row j
          for (int i = j + 1 + lane; i < m; i += 32) w += vj[i] * vc[i];
          w = warp_sum(w) * tj;
          if (lane == 0) vc[j] -= w;
          for (int i = j + 1 + lane; i < m; i += 32) vc[i] -= w * vj[i];
        }
      }
      __syncthreads();
      if (threadIdx.x == 0) vj[j] = s_beta;
      __syncthreads();
    }
    // write the factorised panel back (R above and on the diagonal, vectors below)
    for (long long t = threadIdx.x; t < (long long)pb * m; t += blockDim.x) W[(long long)p0 * m + t] = Vs[t];
    __syncthreads();
    if (p0 + pb >= n) break;
    qr_blk_load_v(m, p0, pb, W, Vs);
    __syncthreads();
    qr_blk_form_t(m, p0, pb, Vs, tau, Ys, Ts);
    // trailing columns: A_c <- A_c - V (T^T (V^T A_c))
    for (int c = p0 + pb + warp; c < n; c += nw) {
      T* ac = W + (long long)c * m;
      T w[kQrNbMax];
#pragma unroll
      for (int t = 0; t < kQrNbMax; ++t) w[t] = T(0);
      for (int i = p0 + lane; i < m; i += 32) {
        const T a = ac[i];
#pragma unroll
        for (int t = 0; t < kQrNbMax; ++t)
          if (t < pb) w[t] += Vs[(long long)t * m + i] * a;
      }
#pragma unroll
      for (int t = 0; t < kQrNbMax; ++t)
        if (t < pb) w[t] = warp_sum(w[t]);
      // w <- T^T w in place (entry b needs w[a] for a <= b: descending b)
#pragma unroll
      for (int b = kQrNbMax - 1; b >= 0; --b) {
        if (b >= pb) continue;
        T acc = T(0);
#pragma unroll
        for (int a = 0; a <= b; ++a) acc += Ts[a * kQrNbMax + b] * w[a];
        w[b] = acc;
      }
      for (int i = p0 + lane; i < m; i += 32) {
        T sacc = T(0);
#pragma unroll
        for (int t = 0; t < kQrNbMax; ++t)
          if (t < pb) sacc += Vs[(long long)t * m + i] * w[t];
        ac[i] -= sacc;
      }
    }
    __syncthreads();
  }
  for (long long t = threadIdx.x; t < (long long)k * n; t += blockDim.x) {
    const int i = (int)(t / n), c = (int)(t % n);
    R[t] = (c >= i) ? W[(long long)c * m + i] : T(0);
  }
  // Q = prod_p (I - V_p T_p V_p^T) [I_k; 0], column-major in the A buffer, panels last to first
  T* QW = A;
  for (long long t = threadIdx.x; t < (long long)m * k; t += blockDim.x) {
    const int c = (int)(t / m), i = (int)(t % m);
    QW[t] = (i == c) ? T(1) : T(0);
  }
  __syncthreads();
  const int np = (k + nb - 1) / nb;
  for (int pi = np - 1; pi >= 0; --pi) {
    const int p0 = pi * nb, pb = min(nb, k - p0);
    qr_blk_load_v(m, p0, pb, W, Vs);
    __syncthreads();
    qr_blk_form_t(m, p0, pb, Vs, tau, Ys, Ts);
    for (int c = p0 + warp; c < k; c += nw) {
      T* qc = QW + (long long)c * m;
      T w[kQrNbMax];
#pragma unroll
      for (int t = 0; t < kQrNbMax; ++t) w[t] = T(0);
      for (int i = p0 + lane; i < m; i += 32) {
        const T a = qc[i];
#pragma unroll
        for (int t = 0; t < kQrNbMax; ++t)
          if (t < pb) w[t] += Vs[(long long)t * m + i] * a;
      }
#pragma unroll
      for (int t = 0; t < kQrNbMax; ++t)
        if (t < pb) w[t] = warp_sum(w[t]);
      // w <- T w in place (entry a needs w[b] for b >= a: ascending a)
#pragma unroll
      for (int a = 0; a < kQrNbMax; ++a) {
        if (a >= pb) continue;
        T acc = T(0);
#pragma unroll
        for (int b = a; b < kQrNbMax; ++b)
          if (b < pb) acc += Ts[a * kQrNbMax + b] * w[b];
        w[a] = acc;
      }
      for (int i = p0 + lane; i < m; i += 32) {
        T sacc = T(0);
#pragma unroll
        for (int t = 0; t < kQrNbMax; ++t)
          if (t < pb) sacc += Vs[(long long)t * m + i] * w[t];
        qc[i] -= sacc;
      }
    }
    __syncthreads();
  }
  for (long long t = threadIdx.x; t < (long long)m * k; t += blockDim.x) {
    const int i = (int)(t / k), c = (int)(t % k);
    Q[t] = QW[(long long)c * m + i];
  }
}

template <typename T>
__global__ void __launch_bounds__(QBT) qr_blk_kernel(int m, int n, int nb, T* __restrict__ A, T* __restrict__ Q,
                                                     T* __restrict__ R, T* __restrict__ tau) {
  qr_blk_body<T>(m, n, nb, A, Q, R, tau);
}

// The same factorisation of `gridDim.x` independent m x n blocks (block b at A + b sA, its factors
// at Q + b sQ, R + b sR, its Householder scalars at tau + b sT): the first level of the
// tall-skinny QR below, one CTA per row block.
template <typename T>
__global__ void __launch_bounds__(QBT) qr_blk_batched_kernel(int m, int n, int nb, T* __restrict__ A, long long sA,
                                                             T* __restrict__ Q, long long sQ, T* __restrict__ R,
                                                             long long sR, T* __restrict__ tau, long long sT) {
  const long long b = blockIdx.x;
  qr_blk_body<T>(m, n, nb, A + b * sA, Q + b * sQ, R + b * sR, tau + b * sT);
}

// Householder QR (m >= n) on one thread-block cluster, with qr_kernel's arithmetic in qr_kernel's
// order (column norm, dot products, updates), so its factors equal qr_kernel's bit for bit.  Binary64 arithmetic runs at a few
// operations per clock per SM on this part, so a single CTA is bound by its own FP64 pipe (a
// 1152 x 72 factorisation with its Q is ~12 M FMAs, ~3 ms on one SM).  Here column c lives in the
// shared memory of CTA c mod C, column-major; at step j the owner of column j forms the reflector
// (the same arithmetic as qr_body), the cluster barrier publishes it, every CTA copies v_j through
// distributed shared memory and applies it to its own trailing columns.  Q = H_0 ... H_{n-1} [I; 0]
// is then accumulated column by column in each owner, reading the final reflectors remotely
// (no barrier between steps: the factors are read-only by then).
constexpr int CQT = 256;          // threads per CTA of qr_cluster_kernel
constexpr int kQrClColMax = 16;   // columns per CTA at most

template <typename T>
__global__ void __launch_bounds__(CQT) qr_cluster_kernel(int m, int n, const T* __restrict__ A, T* __restrict__ Q,
                                                         T* __restrict__ R) {
  namespace cgr = cooperative_groups;
  cgr::cluster_group cluster = cgr::this_cluster();
  extern __shared__ __align__(16) unsigned char qc_smem[];
  const int C = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  const int ncol = (n + C - 1) / C;
  T* Wl = reinterpret_cast<T*>(qc_smem);  // [ncol][m] own columns: factors (R above, v below)
  T* QWl = Wl + (size_t)ncol * m;         // [ncol][m] own columns of Q
  T* sv = QWl + (size_t)ncol * m;         // [m] the reflector of the current step
  __shared__ T taul[kQrClColMax];
  __shared__ T sh[33];
  __shared__ T s_beta, s_v0;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int nown = (n - rank + C - 1) / C;  // columns rank, rank + C, ... below n
  for (int lc = 0; lc < nown; ++lc) {
    const int c = lc * C + rank;
    for (int i = threadIdx.x; i < m; i += blockDim.x) Wl[(size_t)lc * m + i] = A[(size_t)i * n + c];
  }
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    const int o = j % C, lj = j / C;
    if (rank == o) {
      T* wj = Wl + (size_t)lj * m;
      // the column norm in qr_kernel's order (LT threads striding the column, a shuffle tree per
      // warp, then over the warps), so that both kernels produce the same bits
      for (int vw = warp; vw < LT / 32; vw += nw) {
        T part = T(0);
        for (int i = j + 1 + vw * 32 + lane; i < m; i += LT) {
          const T v = wj[i];
          part += v * v;
        }
        for (int off = 16; off > 0; off >>= 1) part += __shfl_down_sync(0xffffffffu, part, off);
        if (lane == 0) sh[vw] = part;
      }
      __syncthreads();
      if (warp == 0) {
        T v = sh[lane];
        for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
        if (lane == 0) sh[32] = v;
      }
      __syncthreads();
      const T tail = sh[32];
      if (threadIdx.x == 0) {
        const T alpha = wj[j];
        if (tail == T(0)) {
          taul[lj] = T(0);
          s_beta = alpha;
          s_v0 = T(1);
        } else {
          const T nx = sqrt(alpha * alpha + tail);
          const T beta = alpha >= T(0) ? -nx : nx;
          taul[lj] = (beta - alpha) / beta;
          s_v0 = alpha - beta;
          s_beta = beta;
        }
      }
      __syncthreads();
      const T v0 = s_v0;
      if (taul[lj] != T(0))
        for (int i = j + 1 + threadIdx.x; i < m; i += blockDim.x) wj[i] /= v0;
      if (threadIdx.x == 0) wj[j] = s_beta;
    }
    cluster.sync();
    const T tj = *cluster.map_shared_rank(taul + lj, o);
    if (tj != T(0)) {
      const T* wo = cluster.map_shared_rank(Wl, o) + (size_t)lj * m;
      for (int i = j + 1 + threadIdx.x; i < m; i += blockDim.x) sv[i] = wo[i];
      __syncthreads();
      for (int lc = (j + 1 - rank + C - 1) / C + warp; lc < nown; lc += nw) {
        T* wc = Wl + (size_t)lc * m;
        T w = T(0);
        for (int i = j + lane; i < m; i += 32) w += ((i == j) ? T(1) : sv[i]) * wc[i];
        w = warp_sum(w) * tj;
        for (int i = j + lane; i < m; i += 32) wc[i] -= w * ((i == j) ? T(1) : sv[i]);
      }
    }
    __syncthreads();
  }
  cluster.sync();
  // R rows 0..n-1 of the own columns
  for (int lc = 0; lc < nown; ++lc) {
    const int c = lc * C + rank;
    for (int i = threadIdx.x; i < n; i += blockDim.x) R[(size_t)i * n + c] = (i <= c) ? Wl[(size_t)lc * m + i] : T(0);
  }
  // Q columns owned here: H_0 ... H_{n-1} e_c, reflectors applied last to first
  for (int lc = 0; lc < nown; ++lc) {
    const int c = lc * C + rank;
    for (int i = threadIdx.x; i < m; i += blockDim.x) QWl[(size_t)lc * m + i] = (i == c) ? T(1) : T(0);
  }
  __syncthreads();
  for (int j = n - 1; j >= 0; --j) {
    const int o = j % C, lj = j / C;
    const T tj = *cluster.map_shared_rank(taul + lj, o);
    if (tj == T(0)) continue;
    const T* wo = cluster.map_shared_rank(Wl, o) + (size_t)lj * m;
    for (int i = j + 1 + threadIdx.x; i < m; i += blockDim.x) sv[i] = wo[i];
    __syncthreads();
    // columns c >= j (columns below j are still e_c, which H_j leaves unchanged)
    for (int lc = (j - rank + C - 1) / C + warp; lc < nown; lc += nw) {
      T* qc = QWl + (size_t)lc * m;
      T w = T(0);
      for (int i = j + lane; i < m; i += 32) w += ((i == j) ? T(1) : sv[i]) * qc[i];
      w = warp_sum(w) * tj;
      for (int i = j + lane; i < m; i += 32) qc[i] -= w * ((i == j) ? T(1) : sv[i]);
    }
    __syncthreads();
  }
  for (int lc = 0; lc < nown; ++lc) {
    const int c = lc * C + rank;
    for (int i = threadIdx.x; i < m; i += blockDim.x) Q[(size_t)i * n + c] = QWl[(size_t)lc * m + i];
  }
  cluster.sync();  // no CTA leaves while another may still read its reflectors
}

// Jacobi rotation (cs, sn) annihilating the off-diagonal c of the column-pair Gram block
// [[a, c], [c, b]]: t = tan(theta) is the smaller root of c t^2 + (b - a) t - c = 0,
// t = 2c / (d + sign(d) sqrt(d^2 + 4c^2)) with d = b - a, evaluated in binary32 on power-of-two
// scaled d and c (binary64 division and square root are long sequences on this part); cs and sn
// are then formed in binary64 from t, so the rotation is orthogonal to binary64 rounding whatever
// the accuracy of t, and an inexact angle only leaves a residual c' ~ 1e-7 c for the next sweep.
// A t that vanished in binary32 falls back to the binary64 formula.
__device__ __forceinline__ void jacobi_rotation(double a, double b, double c, double& cs, double& sn) {
  const double d = b - a;
  int e = 0;
  frexp(fmax(fabs(d), fabs(c)), &e);
  const float d32 = (float)ldexp(d, -e), c32 = (float)ldexp(c, -e);
  const float r = sqrtf(d32 * d32 + 4.0f * c32 * c32);
  double t = (double)(2.0f * c32 / (d32 >= 0.0f ? d32 + r : d32 - r));
  if (!(t != 0.0) || !isfinite(t)) {
    const double zeta = d / (2.0 * c);
    t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
  }
  cs = rsqrt(1.0 + t * t);
  sn = cs * t;
}
__device__ __forceinline__ void jacobi_rotation(float a, float b, float c, float& cs, float& sn) {
  const float zeta = (b - a) / (2.0f * c);
  const float t = (zeta >= 0.0f ? 1.0f : -1.0f) / (fabsf(zeta) + sqrtf(1.0f + zeta * zeta));
  cs = rsqrtf(1.0f + t * t);
  sn = cs * t;
}

// One-sided Jacobi SVD.  G: m x n column-major work copy of A, V: n x n column-major.
// With use_smem the working copies G, V and sig live in dynamic shared memory (when they fit);
// otherwise in the global work buffers passed in.
template <typename T>
__global__ void __launch_bounds__(LT) svd_kernel(int m, int n, const T* __restrict__ A, T* __restrict__ U,
                                                 T* __restrict__ S, T* __restrict__ Vt,
                                                 T* Gg, T* Vg, T* sigg, int max_sweeps, int use_smem) {
  extern __shared__ __align__(16) unsigned char svd_smem[];
  T* G = use_smem ? reinterpret_cast<T*>(svd_smem) : Gg;
  T* V = use_smem ? G + (size_t)m * n : Vg;
  T* sig = use_smem ? V + (size_t)n * n : sigg;
  __shared__ int s_rot;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (long long t = threadIdx.x; t < (long long)m * n; t += blockDim.x) {
    int i = (int)(t / n), j = (int)(t % n);
    G[(long long)j * m + i] = A[t];
  }
  for (long long t = threadIdx.x; t < (long long)n * n; t += blockDim.x) {
    int i = (int)(t % n), j = (int)(t / n);
    V[t] = (i == j) ? T(1) : T(0);
  }
  __syncthreads();
  const int np = n + (n & 1);  // players, with a dummy when n is odd
  const T tol = eps_of<T>() * (T)4;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    if (threadIdx.x == 0) s_rot = 0;
    __syncthreads();
    for (int r = 0; r < np - 1; ++r) {
      for (int pi = warp; pi < np / 2; pi += nw) {
        int p, q;
        if (pi == 0) { p = r; q = np - 1; }
        else { p = (r + pi) % (np - 1); q = (r - pi + (np - 1)) % (np - 1); }
        if (p >= n || q >= n) continue;
        if (p > q) { int t = p; p = q; q = t; }
        T* gp = G + (long long)p * m;
        T* gq = G + (long long)q * m;
        T a = T(0), b = T(0), c = T(0);
        for (int i = lane; i < m; i += 32) {
          T x = gp[i], y = gq[i];
          a += x * x; b += y * y; c += x * y;
        }
        a = warp_sum(a); b = warp_sum(b); c = warp_sum(c);
        if (c == T(0) || a == T(0) || b == T(0)) continue;
        // the rotation is computed by one lane and broadcast (see jacobi_rotation: binary64
        // square roots and divisions are long sequences, and binary64 throughput is scarce)
        T cs = T(1), sn = T(0);
        int rotate = 0;
        if (lane == 0) {
          const T tiny = sizeof(T) == 8 ? T(1e-140) : T(1e-17);
          rotate = (a > tiny && b > tiny) ? (c * c > tol * tol * a * b) : (fabs(c) > tol * sqrt(a * b));
          if (rotate) jacobi_rotation(a, b, c, cs, sn);
        }
        rotate = __shfl_sync(0xffffffffu, rotate, 0);
        if (!rotate) continue;
        cs = __shfl_sync(0xffffffffu, cs, 0);
        sn = __shfl_sync(0xffffffffu, sn, 0);
        for (int i = lane; i < m; i += 32) {
          T x = gp[i], y = gq[i];
          gp[i] = cs * x - sn * y;
          gq[i] = sn * x + cs * y;
        }
        T* vp = V + (long long)p * n;
        T* vq = V + (long long)q * n;
        for (int i = lane; i < n; i += 32) {
          T x = vp[i], y = vq[i];
          vp[i] = cs * x - sn * y;
          vq[i] = sn * x + cs * y;
        }
        if (lane == 0) atomicAdd(&s_rot, 1);
      }
      __syncthreads();
    }
    int rot = s_rot;
    __syncthreads();
    if (rot == 0) break;
  }
  // singular values
  for (int j = warp; j < n; j += nw) {
    T s = T(0);
    for (int i = lane; i < m; i += 32) s += G[(long long)j * m + i] * G[(long long)j * m + i];
    s = warp_sum(s);
    if (lane == 0) sig[j] = sqrt(s);
  }
  __syncthreads();
  // order: rank by descending value, ties by index
  for (int j = warp; j < n; j += nw) {
    const T sj = sig[j];
    int pos = 0;
    for (int i = lane; i < n; i += 32) {
      T si = sig[i];
      pos += (si > sj || (si == sj && i < j)) ? 1 : 0;
    }
    for (int o = 16; o > 0; o >>= 1) pos += __shfl_xor_sync(0xffffffffu, pos, o);
    // sign: make the entry of largest magnitude of u_j positive
    T best = T(-1);
    int bi = 0;
    for (int i = lane; i < m; i += 32) {
      T v = fabs(G[(long long)j * m + i]);
      if (v > best) { best = v; bi = i; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      T ob = __shfl_xor_sync(0xffffffffu, best, o);
      int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    T sgn = (G[(long long)j * m + bi] < T(0)) ? T(-1) : T(1);
    T inv = sj > T(0) ? sgn / sj : T(0);
    for (int i = lane; i < m; i += 32) U[(long long)i * n + pos] = G[(long long)j * m + i] * inv;
    for (int i = lane; i < n; i += 32) Vt[(long long)pos * n + i] = sgn * V[(long long)j * n + i];
    if (lane == 0) S[pos] = sj;
  }
}

// ---- multi-CTA one-sided Jacobi --------------------------------------------------------------
// The same rotations as svd_kernel, but each pair of a round is handled by its own CTA (four warps),
// so the binary64 work of a round is spread over as many SMs as there are pairs; rounds are
// separated by a grid barrier.  The kernel is launched cooperatively (all CTAs resident), and
// every barrier wait is bounded: on expiry the CTA sets err, and every CTA leaves at the next
// barrier check without writing outputs.

struct GridBar {
  unsigned int count;  // GridSync: arrivals
  unsigned int gen;    // GridSync: completed barriers | error bit
  int err;
  int rot[127];  // rotations per sweep (zeroed before the launch)
  int prof;      // nonzero: svd_coop_kernel accumulates SM cycles per stage of a round into tcyc
  int pad;
  unsigned long long tcyc[6];  // sums over CTAs: sums, rotation, update, barrier, rounds, (spare)
};

constexpr int CT = 128;  // threads per CTA of the cooperative kernels: four warps, all four SM partitions

// every wait bounded (see grid_sync.cuh); a failure is also recorded in err for the host
__device__ __forceinline__ bool grid_barrier(GridBar* bar, unsigned int& idx) {
  const bool ok = grid_sync(reinterpret_cast<GridSync*>(bar), idx);
  if (!ok && threadIdx.x == 0) atomicExch(&bar->err, 1);
  return ok;
}

template <typename T>
__global__ void __launch_bounds__(CT) svd_coop_kernel(int m, int n, const T* __restrict__ A, T* __restrict__ U,
                                                      T* __restrict__ S, T* __restrict__ Vt, T* G, T* V, T* sig,
                                                      int max_sweeps, GridBar* bar) {
  __shared__ T red[3][CT / 32];
  __shared__ T s_cs, s_sn;
  __shared__ int s_rot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int cta = blockIdx.x, ncta = gridDim.x;
  unsigned int bidx = 0;  // grid barriers passed
  // copy-in: G column-major, V = I (rows spread over CTAs)
  for (long long t = (long long)cta * CT + tid; t < (long long)m * n; t += (long long)ncta * CT) {
    const int i = (int)(t / n), j = (int)(t % n);
    G[(long long)j * m + i] = A[t];
  }
  for (long long t = (long long)cta * CT + tid; t < (long long)n * n; t += (long long)ncta * CT) {
    const int i = (int)(t % n), j = (int)(t / n);
    V[t] = (i == j) ? T(1) : T(0);
  }
  if (!grid_barrier(bar, bidx)) return;
  const int np = n + (n & 1);
  const T tol = eps_of<T>() * (T)4;
  const T tiny = sizeof(T) == 8 ? T(1e-140) : T(1e-17);
  const int sweeps = min(max_sweeps, 127);
  // optional stage timing (thread 0): sums, rotation, update, barrier
  const bool tp = bar->prof != 0 && tid == 0;
  long long tm = tp ? clock64() : 0, tc[5] = {0, 0, 0, 0, 0};
  auto mark = [&](int slot) {
    if (tp) {
      const long long t = clock64();
      tc[slot] += t - tm;
      tm = t;
    }
  };
  for (int sweep = 0; sweep < sweeps; ++sweep) {
    for (int r = 0; r < np - 1; ++r) {
      if (tp) ++tc[4];
      for (int pi = cta; pi < np / 2; pi += ncta) {
        int p, q;
        if (pi == 0) { p = r; q = np - 1; }
        else { p = (r + pi) % (np - 1); q = (r - pi + (np - 1)) % (np - 1); }
        if (p >= n || q >= n) continue;
        if (p > q) { int t = p; p = q; q = t; }
        T* gp = G + (long long)p * m;
        T* gq = G + (long long)q * m;
        T a = T(0), b = T(0), c = T(0);
        for (int i = tid; i < m; i += CT) {
          T x = gp[i], y = gq[i];
          a += x * x; b += y * y; c += x * y;
        }
        a = warp_sum(a); b = warp_sum(b); c = warp_sum(c);
        if (lane == 0) {
          red[0][warp] = a;
          red[1][warp] = b;
          red[2][warp] = c;
        }
        __syncthreads();
        mark(0);
        if (tid == 0) {
          a = b = c = T(0);
          for (int w = 0; w < CT / 32; ++w) {
            a += red[0][w];
            b += red[1][w];
            c += red[2][w];
          }
          int rotate = 0;
          if (c != T(0) && a != T(0) && b != T(0)) {
            rotate = (a > tiny && b > tiny) ? (c * c > tol * tol * a * b) : (fabs(c) > tol * sqrt(a * b));
          }
          if (rotate) {
            T cs, sn;
            jacobi_rotation(a, b, c, cs, sn);
            s_cs = cs;
            s_sn = sn;
            atomicAdd(&bar->rot[sweep], 1);
          }
          s_rot = rotate;
        }
        __syncthreads();
        mark(1);
        if (!s_rot) continue;
        const T cs = s_cs, sn = s_sn;
        for (int i = tid; i < m; i += CT) {
          T x = gp[i], y = gq[i];
          gp[i] = cs * x - sn * y;
          gq[i] = sn * x + cs * y;
        }
        T* vp = V + (long long)p * n;
        T* vq = V + (long long)q * n;
        for (int i = tid; i < n; i += CT) {
          T x = vp[i], y = vq[i];
          vp[i] = cs * x - sn * y;
          vq[i] = sn * x + cs * y;
        }
        __syncthreads();
        mark(2);
      }
      if (!grid_barrier(bar, bidx)) return;
      mark(3);
    }
    if (*((volatile int*)&bar->rot[sweep]) == 0) break;
  }
  if (tp)
    for (int i = 0; i < 5; ++i) atomicAdd(&bar->tcyc[i], (unsigned long long)tc[i]);
  // singular values, then (after a barrier) ranks, signs and outputs; columns spread over the
  // warps of all CTAs
  const int gw = cta * (CT / 32) + warp, nwarp = ncta * (CT / 32);
  for (int j = gw; j < n; j += nwarp) {
    T s = T(0);
    for (int i = lane; i < m; i += 32) s += G[(long long)j * m + i] * G[(long long)j * m + i];
    s = warp_sum(s);
    if (lane == 0) sig[j] = sqrt(s);
  }
  if (!grid_barrier(bar, bidx)) return;
  for (int j = gw; j < n; j += nwarp) {
    const T sj = sig[j];
    int pos = 0;
    for (int i = lane; i < n; i += 32) {
      T si = sig[i];
      pos += (si > sj || (si == sj && i < j)) ? 1 : 0;
    }
    for (int o = 16; o > 0; o >>= 1) pos += __shfl_xor_sync(0xffffffffu, pos, o);
    T best = T(-1);
    int bi = 0;
    for (int i = lane; i < m; i += 32) {
      T v = fabs(G[(long long)j * m + i]);
      if (v > best) { best = v; bi = i; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      T ob = __shfl_xor_sync(0xffffffffu, best, o);
      int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    T sgn = (G[(long long)j * m + bi] < T(0)) ? T(-1) : T(1);
    T inv = sj > T(0) ? sgn / sj : T(0);
    for (int i = lane; i < m; i += 32) U[(long long)i * n + pos] = G[(long long)j * m + i] * inv;
    for (int i = lane; i < n; i += 32) Vt[(long long)pos * n + i] = sgn * V[(long long)j * n + i];
    if (lane == 0) S[pos] = sj;
  }
}

// ---- one-sided Jacobi inside one thread-block cluster --------------------------------------------
// The rotations of svd_coop_kernel, with every column resident in the shared memory of its owner
// CTA (column j in CTA j mod C) and reached by the other CTAs of the cluster through distributed
// shared memory; rounds are separated by the hardware cluster barrier instead of a grid barrier
// in L2.  Each CTA has two groups of four warps, each group taking one column pair per round
// (pairs b, b + 2C, ... for slot b = 2 rank + group), so C = ceil(pairs / 2) CTAs hold a round.
// Every thread of every CTA runs the same rounds and sweeps (the stop decision reads one counter
// after a cluster barrier), so the barrier counts agree by construction.
constexpr int CLT = 256;  // threads per CTA of the cluster SVD: two groups of four warps

template <typename T>
__global__ void __launch_bounds__(CLT) svd_cluster_kernel(int m, int n, const T* __restrict__ A, T* __restrict__ U,
                                                          T* __restrict__ S, T* __restrict__ Vt, int max_sweeps) {
  namespace cgr = cooperative_groups;
  cgr::cluster_group cluster = cgr::this_cluster();
  extern __shared__ __align__(16) unsigned char cl_smem[];
  const int C = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  const int ncol = (n + C - 1) / C;           // columns owned per CTA (at most)
  T* Gl = reinterpret_cast<T*>(cl_smem);      // [ncol][m]
  T* Vl = Gl + (size_t)ncol * m;              // [ncol][n]
  T* sig = Vl + (size_t)ncol * n;             // [n] (CTA 0's copy is the shared one)
  __shared__ int rot[128];                    // rotations per sweep (CTA 0's copy is the shared one)
  __shared__ T red[2][3][4];
  __shared__ T s_cs[2], s_sn[2];
  __shared__ int s_rot[2];
  const int tid = threadIdx.x, grp = tid >> 7, gt = tid & 127, gw = gt >> 5, lane = tid & 31;
  auto colG = [&](int j) -> T* { return cluster.map_shared_rank(Gl, j % C) + (size_t)(j / C) * m; };
  auto colV = [&](int j) -> T* { return cluster.map_shared_rank(Vl, j % C) + (size_t)(j / C) * n; };
  // the four warps of one group meet at a named barrier (ids 1, 2)
  auto group_sync = [&]() { asm volatile("bar.sync %0, 128;" ::"r"(grp + 1) : "memory"); };
  // copy-in of the owned columns, V = I
  for (int lj = 0; lj * C + rank < n; ++lj) {
    const int j = lj * C + rank;
    for (int i = tid; i < m; i += CLT) Gl[(size_t)lj * m + i] = A[(size_t)i * n + j];
    for (int i = tid; i < n; i += CLT) Vl[(size_t)lj * n + i] = i == j ? T(1) : T(0);
  }
  for (int i = tid; i < 128; i += CLT) rot[i] = 0;
  cluster.sync();
  int* rot0 = cluster.map_shared_rank(rot, 0);
  const int np = n + (n & 1);
  const int npairs = np / 2;
  const T tol = eps_of<T>() * (T)4;
  const T tiny = sizeof(T) == 8 ? T(1e-140) : T(1e-17);
  const int sweeps = min(max_sweeps, 127);
  for (int sweep = 0; sweep < sweeps; ++sweep) {
    for (int r = 0; r < np - 1; ++r) {
      for (int pi = 2 * rank + grp; pi < npairs; pi += 2 * C) {
        int p, q;
        if (pi == 0) { p = r; q = np - 1; }
        else { p = (r + pi) % (np - 1); q = (r - pi + (np - 1)) % (np - 1); }
        if (p >= n || q >= n) continue;  // uniform within the group
        if (p > q) { int t = p; p = q; q = t; }
        T* gp = colG(p);
        T* gq = colG(q);
        T a = T(0), b = T(0), c = T(0);
        for (int i = gt; i < m; i += 128) {
          T x = gp[i], y = gq[i];
          a += x * x; b += y * y; c += x * y;
        }
        a = warp_sum(a); b = warp_sum(b); c = warp_sum(c);
        if (lane == 0) {
          red[grp][0][gw] = a;
          red[grp][1][gw] = b;
          red[grp][2][gw] = c;
        }
        group_sync();
        if (gt == 0) {
          a = (red[grp][0][0] + red[grp][0][1]) + (red[grp][0][2] + red[grp][0][3]);
          b = (red[grp][1][0] + red[grp][1][1]) + (red[grp][1][2] + red[grp][1][3]);
          c = (red[grp][2][0] + red[grp][2][1]) + (red[grp][2][2] + red[grp][2][3]);
          int rotate = 0;
          if (c != T(0) && a != T(0) && b != T(0)) {
            rotate = (a > tiny && b > tiny) ? (c * c > tol * tol * a * b) : (fabs(c) > tol * sqrt(a * b));
          }
          if (rotate) {
            T cs, sn;
            jacobi_rotation(a, b, c, cs, sn);
            s_cs[grp] = cs;
            s_sn[grp] = sn;
            atomicAdd(rot0 + sweep, 1);
          }
          s_rot[grp] = rotate;
        }
        group_sync();
        if (s_rot[grp]) {
          const T cs = s_cs[grp], sn = s_sn[grp];
          for (int i = gt; i < m; i += 128) {
            T x = gp[i], y = gq[i];
            gp[i] = cs * x - sn * y;
            gq[i] = sn * x + cs * y;
          }
          T* vp = colV(p);
          T* vq = colV(q);
          for (int i = gt; i < n; i += 128) {
            T x = vp[i], y = vq[i];
            vp[i] = cs * x - sn * y;
            vq[i] = sn * x + cs * y;
          }
        }
        group_sync();  // red / s_* are reused by the group's next pair
      }
      cluster.sync();
    }
    const int done = *((volatile int*)(rot0 + sweep)) == 0;
    if (done) break;
  }
  // singular values of the owned columns into CTA 0's sig, then ranks, signs and outputs
  T* sig0 = cluster.map_shared_rank(sig, 0);
  const int warp = tid >> 5, nw = CLT / 32;
  for (int lj = warp; lj * C + rank < n; lj += nw) {
    const int j = lj * C + rank;
    const T* g = Gl + (size_t)lj * m;
    T sacc = T(0);
    for (int i = lane; i < m; i += 32) sacc += g[i] * g[i];
    sacc = warp_sum(sacc);
    if (lane == 0) sig0[j] = sqrt(sacc);
  }
  cluster.sync();
  for (int lj = warp; lj * C + rank < n; lj += nw) {
    const int j = lj * C + rank;
    const T* g = Gl + (size_t)lj * m;
    const T* v = Vl + (size_t)lj * n;
    const T sj = sig0[j];
    int pos = 0;
    for (int i = lane; i < n; i += 32) {
      const T si = sig0[i];
      pos += (si > sj || (si == sj && i < j)) ? 1 : 0;
    }
    for (int o = 16; o > 0; o >>= 1) pos += __shfl_xor_sync(0xffffffffu, pos, o);
    T best = T(-1);
    int bi = 0;
    for (int i = lane; i < m; i += 32) {
      const T val = fabs(g[i]);
      if (val > best) { best = val; bi = i; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      T ob = __shfl_xor_sync(0xffffffffu, best, o);
      int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    const T sgn = (g[bi] < T(0)) ? T(-1) : T(1);
    const T inv = sj > T(0) ? sgn / sj : T(0);
    for (int i = lane; i < m; i += 32) U[(size_t)i * n + pos] = g[i] * inv;
    for (int i = lane; i < n; i += 32) Vt[(size_t)pos * n + i] = sgn * v[i];
    if (lane == 0) S[pos] = sj;
  }
  cluster.sync();  // CTA 0's sig and rot stay alive until every CTA is done reading them
}

// ---- QR of [U | W] with U orthonormal ---------------------------------------------------------
// Q, R of the m x (rk + w) matrix A = [U | W] (row-major, leading dimension rk + w) when its first
// rk columns are orthonormal (the left singular vectors of the sweep's truncation, step a7): W is
// orthogonalised against U by block Gram-Schmidt, twice, W = U C + W''; W'' = Q_w R_w by
// Householder QR (one CTA); then A = [U | Q_w] [[I, C], [0, R_w]], the same factorisation as the
// Householder QR of A up to the basis of the W part.  When W'' lies numerically inside span(U)
// the QR of W'' completes it with directions that need not be orthogonal to U; that is detected
// (max |U^T Q_w| > 1e-10) and CTA 0 then takes the Householder QR of the projected (same-span)
// A' = Q R' instead, with R corrected so that Q R = A still holds.  One cooperative launch, grid
// barriers between the phases, every wait bounded.
template <typename T>
__global__ void __launch_bounds__(CT) qr_ext_coop_kernel(int m, int rk, int w, T* __restrict__ A, T* __restrict__ Q,
                                                         T* __restrict__ R, T* __restrict__ work, GridBar* bar) {
  const int ld = rk + w;
  const int tid = threadIdx.x, lane = tid & 31;
  unsigned int bidx = 0;  // grid barriers passed
  const int gwarp = blockIdx.x * (CT / 32) + (tid >> 5), nwarp = gridDim.x * (CT / 32);
  const int gthr = blockIdx.x * CT + tid, nthr = gridDim.x * CT;
  T* Cp = work;                    // [rk][w] this pass's coefficients
  T* Ca = Cp + (size_t)rk * w;     // [rk][w] accumulated coefficients
  T* Wc = Ca + (size_t)rk * w;     // [m][w] remainder, contiguous
  T* Qw = Wc + (size_t)m * w;      // [m][w]
  T* Rw = Qw + (size_t)m * w;      // [w][w]
  T* tau = Rw + (size_t)w * w;     // [max(w, ld)]
  T* emax = tau + ld;              // [nwarp]
  const T* U = A;
  T* W = A + rk;
  for (int pass = 0; pass < 2; ++pass) {
    for (int it = gwarp; it < rk * w; it += nwarp) {
      const int k = it / w, j = it - k * w;
      T sacc = T(0);
      for (int i = lane; i < m; i += 32) sacc += U[(size_t)i * ld + k] * W[(size_t)i * ld + j];
      sacc = warp_sum(sacc);
      if (lane == 0) {
        Cp[it] = sacc;
        Ca[it] = pass == 0 ? sacc : Ca[it] + sacc;
      }
    }
    if (!grid_barrier(bar, bidx)) return;
    for (int t = gthr; t < m * w; t += nthr) {
      const int i = t / w, j = t - i * w;
      T sacc = T(0);
      for (int k = 0; k < rk; ++k) sacc += U[(size_t)i * ld + k] * Cp[k * w + j];
      W[(size_t)i * ld + j] -= sacc;
    }
    if (!grid_barrier(bar, bidx)) return;
  }
  if (blockIdx.x == 0) {
    for (int t = tid; t < m * w; t += CT) Wc[t] = W[(size_t)(t / w) * ld + t % w];
    __syncthreads();
    qr_body(m, w, Wc, Qw, Rw, tau);
  }
  if (!grid_barrier(bar, bidx)) return;
  // orthogonality of Q_w to U
  T mx = T(0);
  for (int it = gwarp; it < rk * w; it += nwarp) {
    const int k = it / w, j = it - k * w;
    T sacc = T(0);
    for (int i = lane; i < m; i += 32) sacc += U[(size_t)i * ld + k] * Qw[(size_t)i * w + j];
    mx = fmax(mx, fabs(warp_sum(sacc)));
  }
  if (lane == 0) emax[gwarp] = mx;
  if (!grid_barrier(bar, bidx)) return;
  T worst = T(0);
  for (int i = 0; i < nwarp; ++i) worst = fmax(worst, emax[i]);
  if (worst <= T(1e-10)) {
    // Q = [U | Q_w], R = [[I, C], [0, R_w]]
    for (int t = gthr; t < m * ld; t += nthr) {
      const int i = t / ld, c = t - i * ld;
      Q[t] = c < rk ? U[(size_t)i * ld + c] : Qw[(size_t)i * w + (c - rk)];
    }
    for (int t = gthr; t < ld * ld; t += nthr) {
      const int i = t / ld, c = t - i * ld;
      T v;
      if (i < rk) v = c < rk ? (i == c ? T(1) : T(0)) : Ca[i * w + (c - rk)];
      else v = c < rk ? T(0) : Rw[(i - rk) * w + (c - rk)];
      R[t] = v;
    }
  } else if (blockIdx.x == 0) {
    // A' = [U | W''] = Q R'; A = A' + [0 | U C] and U = Q R'[:, :rk], so R = R' + [0 | R'[:, :rk] C]
    qr_body(m, ld, A, Q, R, tau);
    __syncthreads();
    for (int t = tid; t < rk * w; t += CT) {
      const int i = t / w, j = t - i * w;
      T sacc = T(0);
      for (int k = i; k < rk; ++k) sacc += R[(size_t)i * ld + k] * Ca[k * w + j];
      R[(size_t)i * ld + rk + j] += sacc;
    }
  }
}

}  // namespace

size_t qr_work_elems(int m, int n) { return (size_t)std::min(m, n) + 8; }
size_t svd_work_elems(int m, int n) { return (size_t)m * n + (size_t)n * n + (size_t)n + 8; }

// QR on one cluster (qr_cluster_kernel); false when the shape or the device does not allow it.
template <typename T>
static bool qr_cluster(tnfem_ctx* ctx, int m, int n, const T* A, T* Q, T* R) {
  if (m < n || n < kQrClMinN) return false;
  const int C = std::min(16, (n + 3) / 4);
  const int ncol = (n + C - 1) / C;
  if (C < 2 || ncol > kQrClColMax) return false;
  const size_t smem = ((size_t)2 * ncol + 1) * m * sizeof(T);
  if (smem > kQrClSmemMax) return false;
  static std::atomic<unsigned long long> attr_set{0};  // one bit per device
  const unsigned long long bit = 1ull << (ctx->device & 63);
  if (!(attr_set & bit)) {
    if (cudaFuncSetAttribute(qr_cluster_kernel<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess ||
        cudaFuncSetAttribute(qr_cluster_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kQrClSmemMax) !=
            cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    attr_set |= bit;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C);
  cfg.blockDim = dim3(CQT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = ctx->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int nclusters = 0;
  if (cudaOccupancyMaxActiveClusters(&nclusters, qr_cluster_kernel<T>, &cfg) != cudaSuccess || nclusters < 1) {
    cudaGetLastError();
    return false;
  }
  if (cudaLaunchKernelEx(&cfg, qr_cluster_kernel<T>, m, n, (const T*)A, Q, R) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return true;
}

// Tall-skinny QR (TSQR) for matrices whose columns do not fit one CTA's shared memory (the
// unfoldings of the 3D operator's cores in its rounding, ~28k x 441): the rows are cut into
// blocks of about 2n rows, each block is factorised by its own CTA (qr_blk_batched_kernel), the
// stacked R factors are factorised the same way recursively, and each block of Q is its block
// Q factor times the matching n x n block of the next level's Q (batched GEMM).  Every level is
// Householder QR, so Q has orthonormal columns to rounding whatever the rank of A.
template <typename T>
void qr_tall(tnfem_ctx* ctx, int m, int n, T* A, T* Q, T* R);

template <typename T>
static void qr_blk_batch(tnfem_ctx* ctx, int rows, int n, int count, T* A, T* Q, T* R, T* tau) {
  const int nb = (int)std::min<size_t>(kQrNbMax, kQrSmemMax / ((size_t)rows * sizeof(T)));
  TN_REQUIRE(nb >= 1, "qr_tall: row block too long");
  const size_t smem = (size_t)nb * rows * sizeof(T);
  static std::atomic<unsigned long long> attr_set{0};  // one bit per device
  const unsigned long long bit = 1ull << (ctx->device & 63);
  if (!(attr_set & bit)) {
    TN_CHECK_CUDA(cudaFuncSetAttribute(qr_blk_batched_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kQrSmemMax));
    attr_set |= bit;
  }
  qr_blk_batched_kernel<T><<<count, QBT, smem, ctx->stream>>>(rows, n, nb, A, (long long)rows * n, Q,
                                                               (long long)rows * n, R, (long long)n * n, tau, n);
  count_launch(ctx);
  check_launch(ctx, "qr_tall");
}

template <typename T>
void qr_tall(tnfem_ctx* ctx, int m, int n, T* A, T* Q, T* R) {
  const int b = 2 * n;           // rows per block
  const int B = m / b;           // blocks; the last one takes the remaining rows (b .. 2b - 1)
  const int last = m - (B - 1) * b;
  DArr<T> Qb(ctx, (size_t)m * n), Rs(ctx, (size_t)B * n * n), tau(ctx, (size_t)B * n + 8);
  if (B > 1) qr_blk_batch<T>(ctx, b, n, B - 1, A, Qb.p, Rs.p, tau.p);
  qr_blk_batch<T>(ctx, last, n, 1, A + (size_t)(B - 1) * b * n, Qb.p + (size_t)(B - 1) * b * n,
                  Rs.p + (size_t)(B - 1) * n * n, tau.p + (size_t)(B - 1) * n);
  // next level: the stacked R factors (B n x n)
  DArr<T> Q2(ctx, (size_t)B * n * n);
  const int m2 = B * n;
  if (m2 >= 4 * n && (size_t)m2 * sizeof(T) > kQrSmemMax / kQrNbMax) {
    qr_tall<T>(ctx, m2, n, Rs.p, Q2.p, R);
  } else {
    DArr<T> w(ctx, qr_work_elems(m2, n));
    qr<T>(ctx, m2, n, Rs.p, Q2.p, R, w.p);
  }
  // Q block i = Qb_i (rows_i x n) . Q2_i (n x n)
  if (B > 1) {
    GemmDesc g{b, n, n, B - 1, n, 1, (long long)b * n, n, 1, (long long)n * n, n, 1, (long long)b * n};
    gemm<T>(ctx, g, T(1), Qb.p, Q2.p, T(0), Q);
  }
  GemmDesc gl{last, n, n, 1, n, 1, 0, n, 1, 0, n, 1, 0};
  gemm<T>(ctx, gl, T(1), Qb.p + (size_t)(B - 1) * b * n, Q2.p + (size_t)(B - 1) * n * n, T(0),
          Q + (size_t)(B - 1) * b * n);
}

template <typename T>
void qr(tnfem_ctx* ctx, int m, int n, T* A, T* Q, T* R, T* work) {
  if (m <= 0 || n <= 0) return;
  const int k = std::min(m, n);
  // columns too long for the one-CTA panel and far taller than wide: the tall-skinny QR
  if (m >= 8 * n && n >= 16 && (size_t)m * sizeof(T) * kQrNbMax > kQrSmemMax && !ctx->capturing) {
    qr_tall<T>(ctx, m, n, A, Q, R);
    return;
  }
  ProfScope ps(ctx, TNFEM_PROF_QR, 4.0 * m * n * (double)k, (double)(2 * m * n + m * k + k * n) * sizeof(T));
  if (qr_cluster<T>(ctx, m, n, A, Q, R)) {
    count_launch(ctx);
    check_launch(ctx, "qr");
    return;
  }
  const int nb = (int)std::min<size_t>(kQrNbMax, kQrSmemMax / ((size_t)m * sizeof(T)));
  if (m >= n && nb >= 1 && (size_t)m * n >= kQrBlkMinElems) {
    const size_t smem = (size_t)nb * m * sizeof(T);
    if (smem > 48 * 1024)
      TN_CHECK_CUDA(cudaFuncSetAttribute(qr_blk_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    qr_blk_kernel<T><<<1, QBT, smem, ctx->stream>>>(m, n, nb, A, Q, R, work);
  } else {
    qr_kernel<T><<<1, LT, 0, ctx->stream>>>(m, n, A, Q, R, work);
  }
  count_launch(ctx);
  check_launch(ctx, "qr");
}

size_t qr_ext_work_elems(int m, int rk, int w) {
  return 2 * (size_t)rk * w + 2 * (size_t)m * w + (size_t)w * w + (size_t)(rk + w) + 64 * (CT / 32) + 8;
}

template <typename T>
void qr_ext(tnfem_ctx* ctx, int m, int rk, int w, T* A, T* Q, T* R, T* work, size_t work_elems) {
  const int ld = rk + w;
  if (w < 1 || rk < 1 || m < ld || work_elems < qr_ext_work_elems(m, rk, w)) {
    qr<T>(ctx, m, ld, A, Q, R, work);
    return;
  }
  GridBar* bar = reinterpret_cast<GridBar*>(ctx->scratch + kScratchDoubles - 512);
  TN_CHECK_CUDA(cudaMemsetAsync(bar, 0, sizeof(GridBar), ctx->stream));
  int dev_sms = 0;
  dev_sms = coop_sms(ctx);
  int ncta = std::max(1, std::min({64, dev_sms, (rk * w + (CT / 32) - 1) / (CT / 32)}));
  void* args[] = {&m, &rk, &w, &A, &Q, &R, &work, &bar};
  {
    ProfScope ps(ctx, TNFEM_PROF_QR, 8.0 * m * rk * (double)w, (double)(2 * m * ld + ld * ld) * sizeof(T));
    TN_CHECK_CUDA(cudaLaunchCooperativeKernel(reinterpret_cast<void*>(qr_ext_coop_kernel<T>), dim3(ncta), dim3(CT),
                                              args, 0, ctx->stream));
  }
  count_launch(ctx);
  check_launch(ctx, "qr");
  int err = 0;
  TN_CHECK_CUDA(cudaMemcpyAsync(&err, &bar->err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  sync(ctx);
  if (err) throw Error(TNFEM_E_TIMEOUT, "qr: a grid barrier wait expired");
}

// TNFEM_SVD_PROF set: Jacobi sweeps of every cooperative SVD, reported at process exit.
struct SvdStats {
  bool on = getenv("TNFEM_SVD_PROF") != nullptr;
  long long calls = 0, sweeps = 0, mn = 0;
  int hist[16] = {};
  double cyc[5] = {};  // per CTA: sums, rotation, update, barrier cycles; rounds
  void add(int m, int n, int sw) {
    ++calls;
    sweeps += sw;
    mn += (long long)m * n;
    ++hist[std::min(sw, 15)];
  }
  ~SvdStats() {
    if (!on || calls == 0) return;
    fprintf(stderr, "[tnfem] cooperative SVD: %lld calls, %.2f sweeps per call (incl. the checking sweep), mean m*n %.0f; sweeps histogram:",
            calls, (double)sweeps / calls, (double)mn / calls);
    for (int i = 0; i < 16; ++i)
      if (hist[i]) fprintf(stderr, " %d:%d", i, hist[i]);
    fprintf(stderr, "\n");
    if (cyc[4] > 0)
      fprintf(stderr, "[tnfem] cooperative SVD SM cycles per round (mean over CTAs): sums %.0f rotation %.0f update %.0f barrier %.0f\n",
              cyc[0] / cyc[4], cyc[1] / cyc[4], cyc[2] / cyc[4], cyc[3] / cyc[4]);
  }
};
SvdStats& svd_stats() {
  static SvdStats st;
  return st;
}

// The binary64 SVD on one thread-block cluster (svd_cluster_kernel); false when the shape or the
// device does not allow it (more than 16 CTAs, shared memory, no cluster of that size resident),
// and the caller takes the cooperative kernel.
template <typename T>
bool svd_cluster(tnfem_ctx* ctx, int m, int n, const T* A, T* U, T* S, T* Vt, int max_sweeps) {
  const int np = n + (n & 1);
  const int C = (np / 2 + 1) / 2;
  if (C < 2 || C > 16) return false;
  const int ncol = (n + C - 1) / C;
  const size_t smem = ((size_t)ncol * (m + n) + n) * sizeof(T);
  constexpr size_t kMax = 160 * 1024;
  if (smem > kMax) return false;
  static std::atomic<unsigned long long> attr_set{0};  // one bit per device
  const unsigned long long bit = 1ull << (ctx->device & 63);
  if (!(attr_set & bit)) {
    if (cudaFuncSetAttribute(svd_cluster_kernel<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
            cudaSuccess ||
        cudaFuncSetAttribute(svd_cluster_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMax) !=
            cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    attr_set |= bit;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C);
  cfg.blockDim = dim3(CLT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = ctx->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int nclusters = 0;
  if (cudaOccupancyMaxActiveClusters(&nclusters, svd_cluster_kernel<T>, &cfg) != cudaSuccess || nclusters < 1) {
    cudaGetLastError();
    return false;
  }
  {
    ProfScope ps(ctx, TNFEM_PROF_SVD, 0.0, (double)(2 * m * n + 2 * n * n) * sizeof(T));
    if (cudaLaunchKernelEx(&cfg, svd_cluster_kernel<T>, m, n, A, U, S, Vt, max_sweeps) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
  }
  count_launch(ctx);
  check_launch(ctx, "svd");
  return true;
}

template <typename T>
void svd(tnfem_ctx* ctx, int m, int n, T* A, T* U, T* S, T* Vt, T* work) {
  if (m <= 0 || n <= 0) return;
  TN_REQUIRE(m >= n, "svd: needs m >= n");
  T* G = work;
  T* V = G + (size_t)m * n;
  T* sig = V + (size_t)n * n;
  if (sizeof(T) == 8 && n >= kSvdCoopMinN && !svd_stats().on && svd_cluster<T>(ctx, m, n, A, U, S, Vt, 60)) return;
  if (sizeof(T) == 8 && n >= kSvdCoopMinN) {
    // binary64 with enough pairs per round: spread the rounds over SMs
    GridBar* bar = reinterpret_cast<GridBar*>(ctx->scratch + kScratchDoubles - 512);
    TN_CHECK_CUDA(cudaMemsetAsync(bar, 0, sizeof(GridBar), ctx->stream));
    if (svd_stats().on) {
      const int one = 1;
      TN_CHECK_CUDA(cudaMemcpyAsync(&bar->prof, &one, sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
    }
    int ncta = (n + (n & 1)) / 2;
    int dev_sms = 0;
    dev_sms = coop_sms(ctx);
    ncta = std::max(1, std::min(ncta, dev_sms));
    int max_sweeps = 60;
    void* args[] = {&m, &n, &A, &U, &S, &Vt, &G, &V, &sig, &max_sweeps, &bar};
    {
      ProfScope ps(ctx, TNFEM_PROF_SVD, 0.0, (double)(2 * m * n + 2 * n * n) * sizeof(T));
      TN_CHECK_CUDA(cudaLaunchCooperativeKernel(reinterpret_cast<void*>(svd_coop_kernel<T>), dim3(ncta), dim3(CT),
                                                args, 0, ctx->stream));
    }
    count_launch(ctx);
    check_launch(ctx, "svd");
    int err = 0;
    TN_CHECK_CUDA(cudaMemcpyAsync(&err, &bar->err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    sync(ctx);
    if (err) throw Error(TNFEM_E_TIMEOUT, "svd: a grid barrier wait expired");
    if (svd_stats().on) {
      // sweeps done = index of the first sweep without a rotation, plus that checking sweep
      int rot[127];
      TN_CHECK_CUDA(cudaMemcpy(rot, bar->rot, sizeof(rot), cudaMemcpyDeviceToHost));
      int sw = 0;
      while (sw < max_sweeps && sw < 127 && rot[sw] != 0) ++sw;
      svd_stats().add(m, n, std::min(sw + 1, max_sweeps));
      unsigned long long tc[6];
      TN_CHECK_CUDA(cudaMemcpy(tc, bar->tcyc, sizeof(tc), cudaMemcpyDeviceToHost));
      for (int i = 0; i < 5; ++i) svd_stats().cyc[i] += (double)tc[i] / ncta;
    }
    return;
  }
  ProfScope ps(ctx, TNFEM_PROF_SVD, 0.0, (double)(2 * m * n + 2 * n * n) * sizeof(T));
  const size_t smem = ((size_t)m * n + (size_t)n * n + n) * sizeof(T);
  const int use_smem = smem <= kSvdSmemMax ? 1 : 0;
  static std::atomic<unsigned long long> attr_set{0};  // one bit per device
  const unsigned long long bit = 1ull << (ctx->device & 63);
  if (use_smem && !(attr_set & bit)) {
    TN_CHECK_CUDA(cudaFuncSetAttribute(svd_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSvdSmemMax));
    attr_set |= bit;
  }
  svd_kernel<T><<<1, LT, use_smem ? smem : 0, ctx->stream>>>(m, n, A, U, S, Vt, G, V, sig, sizeof(T) == 8 ? 60 : 40,
                                                            use_smem);
  count_launch(ctx);
  check_launch(ctx, "svd");
}

template void qr<double>(tnfem_ctx*, int, int, double*, double*, double*, double*);
template void qr<float>(tnfem_ctx*, int, int, float*, float*, float*, float*);
template void svd<double>(tnfem_ctx*, int, int, double*, double*, double*, double*, double*);
template void qr_ext<double>(tnfem_ctx*, int, int, int, double*, double*, double*, double*, size_t);
template void qr_ext<float>(tnfem_ctx*, int, int, int, float*, float*, float*, float*, size_t);
template void svd<float>(tnfem_ctx*, int, int, float*, float*, float*, float*, float*);

}  // namespace tnfem
