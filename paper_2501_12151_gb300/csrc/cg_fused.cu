// Preconditioned conjugate gradients on one local system of the sweep (step a5 of the AMEn
// iteration, Section 4) as one persistent cooperative kernel.
//
// The local matrix of core k is B = PhiL (x) A_k (x) PhiR, applied to a core x[a][j][b] in three
// contractions (see contract.cu).  A CG pass here is three phases separated by grid barriers:
//
//   phase 1  T1[a'][beta][j][b] = sum_a PhiL[a'][beta][a] p[a][j][b]
//            tiles of the (r0 a0) x (n r1) product; the direction update p = z + beta p of this
//            pass is formed in shared memory from the staged z and p tiles, and written out by
//            the tiles of the first tile row;
//   phase 2  item (a', g-slice): T2[i][g][b] = sum_{beta,j} T1[a'][beta][j][b] A[beta][j][i][g]
//            for the slice's g into shared memory, then the slice's share of
//            (B p)[a'][i][b'] = sum_{g,b} T2[i][g][b] PhiR[b'][g][b] and of p.Bp;
//   phase 3  item (b, row slice): r = r - alpha B p on the block b (the g-slice shares summed),
//            z = P_b^{-1} r on the slice's rows (block Jacobi, see precond.cu), x += alpha p, and
//            the slice's shares of r.r and r.z.
//
// The first pass forms r = g - B x the same way, with x in place of p.  The scalars alpha, beta
// and the stop test r.r <= stop2 are formed by every CTA from the same partial sums in the same
// order, so every CTA takes the same branch.  Partial sums are accumulated in binary64; the
// block products of the preconditioner run in binary32, as in precond.cu.
//
// Data movement.  Before the launch the system's operators are repacked once into the layouts the
// phases read (PhiL transposed, A and PhiR cut into the g-slices, every row padded to a multiple
// of four elements), and the iteration's vectors live in padded internal buffers (r and the B p
// shares block-major in b).  Every operand block an item needs is then a run of 16-byte aligned
// rows, copied global -> shared with cp.async.cg (L2 only) in double-buffered K chunks.  Within an
// item, the 4 x 4 register tiles of the output need fewer threads than the CTA has when the tile
// is small; the threads then form two groups that take alternate k of each chunk, and the groups'
// accumulators are summed through shared memory at the end.
//
// A CG iteration thus costs three grid barriers (two-level, see grid_sync.cuh) and no launch.
// Every barrier wait is bounded: on expiry the CTA records the error and leaves, and so does every
// other CTA at its next barrier.
#include <atomic>
#include <algorithm>
#include <cstdio>
#include <cstdlib>

#include "cg_fused.h"
#include "grid_sync.cuh"

namespace tnfem {

namespace {

constexpr int FT = 256;                      // threads per CTA
constexpr int kTL = 64;                      // row stride of a staged tile chunk (elements)
constexpr int kRCB = 8192;                   // binary32 preconditioner elements staged at once

__host__ __device__ inline int rup4(int v) { return (v + 3) & ~3; }

// Grid barrier state in the ctl buffer (see grid_sync.cuh): GridSync at ctl + 4, one arrival
// counter per group of CTAs at ctl + 64 + 32 g (separate 128-byte lines).
constexpr int kCtlInts = 64 + 32 * kGridGroupsMax;  // ints of the ctl buffer

// Staging sizes per precision: K chunk of phase 2 (double-buffered) and phase 1, and the elements
// of one buffer of a PhiR slice (phase 2, second contraction).
template <typename U> struct FcgCfg;
template <> struct FcgCfg<float> {
  static constexpr int KC = 32, KC1 = 64, PRB = 7168;
};
template <> struct FcgCfg<double> {
  static constexpr int KC = 16, KC1 = 32, PRB = 2048;
};

// Padded sizes and workspace offsets (elements of U) of one plan.
struct FcgDims {
  int M1, N1, M1p, N1p, r1p, K2, rows2p, K3p, m, mp;
  size_t oPLt, oApk, oPRk, oT1, oY, oR, oZ, oP, total, zero_from;
};

__host__ __device__ inline FcgDims fcg_dims(int r0, int n, int r1, int a0, int S, int gw) {
  FcgDims d;
  d.M1 = r0 * a0;
  d.N1 = n * r1;
  d.M1p = rup4(d.M1);
  d.N1p = rup4(d.N1);
  d.r1p = rup4(r1);
  d.K2 = a0 * n;
  d.rows2p = rup4(n * gw);
  d.K3p = rup4(gw * r1);
  d.m = r0 * n;
  d.mp = rup4(d.m);
  size_t o = 0;
  d.oPLt = o; o += (size_t)r0 * d.M1p;
  d.oApk = o; o += (size_t)S * d.K2 * d.rows2p;
  d.oPRk = o; o += (size_t)S * r1 * d.K3p;
  d.zero_from = o;
  d.oT1 = o; o += (size_t)d.M1 * n * d.r1p;
  d.oY = o; o += (size_t)S * r1 * d.mp;
  d.oR = o; o += (size_t)2 * r1 * d.mp;
  d.oZ = o; o += (size_t)r0 * d.N1p;
  d.oP = o; o += (size_t)2 * r0 * d.N1p;
  d.total = o;
  return d;
}

template <typename U>
struct FcgArgs {
  int r0, n, r1, a0, a1;
  int tr1, tc1, n1, S, gw, n2, split, n3, maxit;
  double stop2;
  const U* g;
  const float* Pinv;
  U* x;
  U* ws;          // packed operators and the iteration's vectors (fcg_dims layout)
  double* parts;  // pap [n2], rr [2][n3], rz [2][n3]
  int* ctl;       // [0] state, [1] iterations; GridSync at ctl + 4; group counters from ctl + 64
  unsigned long long* tprof;  // nullable: SM cycles per phase summed over CTAs (7 slots), then passes
};

__device__ __forceinline__ bool fcg_sync(int* ctl, unsigned int& idx) {
  return grid_sync_groups(reinterpret_cast<GridSync*>(ctl + 4), reinterpret_cast<unsigned int*>(ctl + 64), idx);
}

__device__ __forceinline__ float ldcg(const float* p) { return __ldcg(p); }
__device__ __forceinline__ double ldcg(const double* p) { return __ldcg(p); }

__device__ __forceinline__ void ld4(const float* p, float (&v)[4]) {
  const float4 t = *reinterpret_cast<const float4*>(p);
  v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void ld4(const double* p, double (&v)[4]) {
  const double2 a = *reinterpret_cast<const double2*>(p);
  const double2 b = *reinterpret_cast<const double2*>(p + 2);
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}

__device__ __forceinline__ float fmaU(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmaU(double a, double b, double c) { return fma(a, b, c); }

template <typename V>
__device__ __forceinline__ V warp_allsum(V v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum of part[0..cnt) in a fixed order, formed by the calling warp and returned to all its lanes;
// each lane requests up to 16 of its values at once (one round trip for up to 512 partials).
__device__ __forceinline__ double warp0_sum(const double* part, int cnt) {
  const int lane = threadIdx.x & 31;
  double s = 0.0;
  for (int base = 0; base < cnt; base += 512) {
    double v[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int i = base + lane + 32 * j;
      v[j] = i < cnt ? __ldcg(part + i) : 0.0;
    }
#pragma unroll
    for (int j = 0; j < 16; ++j) s += v[j];
  }
  return warp_allsum(s);
}

// Block-wide sums of two values; the totals are valid in thread 0.
__device__ __forceinline__ void block_sum2(double& a, double& b, double* red) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  a = warp_allsum(a);
  b = warp_allsum(b);
  if (lane == 0) {
    red[warp] = a;
    red[FT / 32 + warp] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double ta = 0.0, tb = 0.0;
    for (int w = 0; w < FT / 32; ++w) {
      ta += red[w];
      tb += red[FT / 32 + w];
    }
    a = ta;
    b = tb;
  }
  __syncthreads();
}

// ---- asynchronous copies ---------------------------------------------------------------------

// 16 bytes global -> shared, L2 only (both addresses 16-byte aligned)
__device__ __forceinline__ void cp16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
               "l"((unsigned long long)__cvta_generic_to_global(src))
               : "memory");
}
// one element (4 or 8 bytes), for the unaligned external vectors x and g
__device__ __forceinline__ void cp1(float* dst, const float* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
               "l"((unsigned long long)__cvta_generic_to_global(src))
               : "memory");
}
__device__ __forceinline__ void cp1(double* dst, const double* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
               "l"((unsigned long long)__cvta_generic_to_global(src))
               : "memory");
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cpa_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// rows x w4 elements (w4 a multiple of 4) from src (row stride lds) to dst (row stride ldd), in
// 16-byte pieces; every row start 16-byte aligned on both sides.  Thread t copies piece t % per of
// rows t / per, t / per + FT / per, ... (per = pieces of a row; one division per call).
template <typename U>
__device__ __forceinline__ void copy_rows(U* dst, int ldd, const U* src, size_t lds, int rows, int w4) {
  constexpr int E = 16 / sizeof(U);  // elements per piece
  const int per = w4 / E;
  if (per <= 0) return;
  if (per > FT) {
    for (int e = threadIdx.x; e < rows * per; e += FT) {
      const int r = e / per, c = (e - r * per) * E;
      cp16(dst + (size_t)r * ldd + c, src + (size_t)r * lds + c);
    }
    return;
  }
  const int rstep = FT / per;
  const int r0 = threadIdx.x / per;
  if (r0 >= rstep) return;
  const int c = (threadIdx.x - r0 * per) * E;
  for (int r = r0; r < rows; r += rstep) cp16(dst + (size_t)r * ldd + c, src + (size_t)r * lds + c);
}
// cnt elements (a multiple of 16 bytes) from src to dst, both 16-byte aligned
template <typename U>
__device__ __forceinline__ void copy_flat(U* dst, const U* src, int cnt) {
  constexpr int E = 16 / sizeof(U);
  for (int e = threadIdx.x; e < cnt / E; e += FT) cp16(dst + e * E, src + e * E);
}

// ---- register tiles --------------------------------------------------------------------------
//
// Output tile rows x cols (<= 64 each) from k-major operands As[k][m] and Bs[k][c] (row stride
// kTL).  Thread (ty, tx) of its group holds the 4 x 4 block at rows 4 ty.., columns 4 tx..; when
// the tile needs at most half the CTA's warps, two groups split the k of every chunk and their
// accumulators are summed at the end (tile_reduce).
struct Mk {
  int gx, grp, ngrp, ty, tx;
  bool act;
};

__device__ __forceinline__ Mk mk_setup(int rows, int cols) {
  Mk k;
  k.gx = (cols + 3) >> 2;
  const int gy = (rows + 3) >> 2;
  const int thr = k.gx * gy;
  const int wneed = (thr + 31) >> 5;
  k.ngrp = wneed * 2 <= FT / 32 ? 2 : 1;
  const int gsz = wneed * 32;
  k.grp = threadIdx.x / gsz;
  const int tt = threadIdx.x - k.grp * gsz;
  k.ty = tt / k.gx;
  k.tx = tt - k.ty * k.gx;
  k.act = k.grp < k.ngrp && tt < thr;
  return k;
}

// acc += sum over the k of [0, kc) that belong to the thread's group (NG groups take alternate k)
template <typename U, int NG>
__device__ __forceinline__ void tile_fma_g(const U* as, const U* bs, int kc, const Mk& mk, U (&acc)[4][4]) {
  const U* pa = as + 4 * mk.ty + mk.grp * kTL;
  const U* pb = bs + 4 * mk.tx + mk.grp * kTL;
#pragma unroll 4
  for (int kk = mk.grp; kk < kc; kk += NG, pa += NG * kTL, pb += NG * kTL) {
    U a[4], b[4];
    ld4(pa, a);
    ld4(pb, b);
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = fmaU(a[i], b[j], acc[i][j]);
  }
}
template <typename U>
__device__ __forceinline__ void tile_fma(const U* as, const U* bs, int kc, const Mk& mk, U (&acc)[4][4]) {
  if (mk.ngrp == 2) tile_fma_g<U, 2>(as, bs, kc, mk, acc);
  else tile_fma_g<U, 1>(as, bs, kc, mk, acc);
}

// Sum the second group's accumulators into the first's through red (>= 64 x 64 elements, free).
template <typename U>
__device__ __forceinline__ void tile_reduce(const Mk& mk, U (&acc)[4][4], U* red) {
  if (mk.ngrp < 2) return;
  __syncthreads();
  if (mk.act && mk.grp == 1) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) red[(4 * mk.ty + i) * 64 + 4 * mk.tx + j] = acc[i][j];
  }
  __syncthreads();
  if (mk.act && mk.grp == 0) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] += red[(4 * mk.ty + i) * 64 + 4 * mk.tx + j];
  }
}

// Phase 2, second contraction on one staged chunk of PhiR rows: for the chunk's nb rows b',
// out[i][b'] = sum_{k<K3} T2s[i][k] buf[b'][k] (i < NN), two b' per warp with the lanes along k;
// lane 0 stores the shares and accumulates p.Bp (PN = row a' of p, unused in the first pass).
template <typename U, int NN>
__device__ __forceinline__ void stage3(const U* T2s, const U* buf, int K3, int K3p, int nb, int b0, int r1,
                                       U* Ybase, int mp, const U* PN, bool first, double& pap) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int bl = 2 * warp; bl < nb; bl += 2 * (FT / 32)) {
    const bool two = bl + 1 < nb;
    const U* p0 = buf + (size_t)bl * K3p;
    const U* p1 = two ? p0 + K3p : p0;
    U s0[NN], s1[NN];
#pragma unroll
    for (int i = 0; i < NN; ++i) {
      s0[i] = U(0);
      s1[i] = U(0);
    }
    for (int k = lane; k < K3; k += 32) {
      const U w0 = p0[k], w1 = p1[k];
#pragma unroll
      for (int i = 0; i < NN; ++i) {
        const U t = T2s[i * K3 + k];
        s0[i] = fmaU(t, w0, s0[i]);
        s1[i] = fmaU(t, w1, s1[i]);
      }
    }
#pragma unroll
    for (int i = 0; i < NN; ++i) {
      s0[i] = warp_allsum(s0[i]);
      s1[i] = warp_allsum(s1[i]);
    }
    if (lane == 0) {
      const int bpp = b0 + bl;
#pragma unroll
      for (int i = 0; i < NN; ++i) {
        Ybase[(size_t)bpp * mp + i] = s0[i];
        if (!first) pap += (double)PN[i * r1 + bpp] * (double)s0[i];
        if (two) {
          Ybase[(size_t)(bpp + 1) * mp + i] = s1[i];
          if (!first) pap += (double)PN[i * r1 + bpp + 1] * (double)s1[i];
        }
      }
    }
  }
}

// Shared-memory bytes of the kernel for one plan (the phases reuse one region).
template <typename U>
__host__ __device__ inline size_t fcg_smem_bytes(int r1, int m, int S, int per) {
  using C = FcgCfg<U>;
  const size_t p1 = (size_t)3 * C::KC1 * kTL * sizeof(U);
  const size_t p2 = ((size_t)4 * C::KC * kTL + (size_t)64 * r1 + rup4(8 * r1) + 2 * C::PRB) * sizeof(U);
  const int mp = rup4(m);
  const int rc = max(1, min(per, kRCB / max(1, mp)));
  const size_t p3 = ((size_t)(S + 2) * mp + 2 * (size_t)rup4(per)) * sizeof(U) + (size_t)mp * sizeof(float) +
                    (size_t)rc * mp * sizeof(float);
  size_t mx = p1 > p2 ? p1 : p2;
  mx = mx > p3 ? mx : p3;
  return mx + 64;
}

// ---- operator repacking (once per local system) ------------------------------------------------

template <typename U>
__global__ void fcg_pack_kernel(int r0, int n, int r1, int a0, int a1, int S, int gw, const U* __restrict__ PL,
                                const U* __restrict__ Ap, const U* __restrict__ PR, U* __restrict__ ws) {
  const FcgDims d = fcg_dims(r0, n, r1, a0, S, gw);
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  // PhiL^T: PLt[a][(a', beta)] (row stride M1p)
  for (long long t = t0; t < (long long)r0 * d.M1p; t += stride) {
    const int a = (int)(t / d.M1p), mm = (int)(t - (long long)a * d.M1p);
    ws[d.oPLt + t] = mm < d.M1 ? PL[(size_t)mm * r0 + a] : U(0);
  }
  // A slices: Apk[s][kappa][(i, g)] (row stride rows2p), g fastest within the slice
  for (long long t = t0; t < (long long)S * d.K2 * d.rows2p; t += stride) {
    const int row = (int)(t % d.rows2p);
    const long long rest = t / d.rows2p;
    const int kap = (int)(rest % d.K2), s = (int)(rest / d.K2);
    const int g0 = s * gw, gc = min(gw, a1 - g0);
    U v = U(0);
    if (row < n * gc) {
      const int i = row / gc, gl = row - i * gc;
      v = Ap[(size_t)kap * n * a1 + i * a1 + g0 + gl];
    }
    ws[d.oApk + t] = v;
  }
  // PhiR slices: PRk[s][b'][(g, b)] (row stride K3p)
  for (long long t = t0; t < (long long)S * r1 * d.K3p; t += stride) {
    const int k = (int)(t % d.K3p);
    const long long rest = t / d.K3p;
    const int bp = (int)(rest % r1), s = (int)(rest / r1);
    const int g0 = s * gw, gc = min(gw, a1 - g0);
    ws[d.oPRk + t] = k < gc * r1 ? PR[(size_t)bp * a1 * r1 + (size_t)g0 * r1 + k] : U(0);
  }
}

// ---- the kernel ------------------------------------------------------------------------------

template <typename U>
__global__ void __launch_bounds__(FT, 2) fcg_kernel(const FcgArgs<U> A) {
  using Cfg = FcgCfg<U>;
  constexpr int KC = Cfg::KC, KC1 = Cfg::KC1, PRB = Cfg::PRB;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  U* sm = reinterpret_cast<U*>(smem_raw);
  __shared__ double red[2 * (FT / 32)];
  __shared__ double s_sc[2];
  __shared__ double s_sum[3];
  __shared__ int s_state;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int r0 = A.r0, n = A.n, r1 = A.r1, a1 = A.a1;
  const FcgDims D = fcg_dims(r0, n, r1, A.a0, A.S, A.gw);
  const int M1 = D.M1, N1 = D.N1, m = D.m, mp = D.mp;
  const U* PLt = A.ws + D.oPLt;
  const U* Apk = A.ws + D.oApk;
  const U* PRk = A.ws + D.oPRk;
  U* T1 = A.ws + D.oT1;
  U* Y = A.ws + D.oY;
  U* const R0v = A.ws + D.oR;
  U* const R1v = R0v + (size_t)r1 * mp;
  U* Z = A.ws + D.oZ;
  U* const P0v = A.ws + D.oP;
  U* const P1v = P0v + (size_t)r0 * D.N1p;
  double* ppap = A.parts;
  double* prr = A.parts + A.n2;             // [2][n3]
  double* prz = A.parts + A.n2 + 2 * A.n3;  // [2][n3]
  U beta = U(0);
  int it = 0;
  int state = 0;
  unsigned int bidx = 0;  // grid barriers passed
  // optional phase timing (thread 0 of every CTA): work and barrier wait of each phase
  const bool tp = A.tprof != nullptr && threadIdx.x == 0;
  long long tmark = tp ? clock64() : 0;
  long long tacc[7] = {0, 0, 0, 0, 0, 0, 0};
  auto mark = [&](int slot) {
    if (tp) {
      const long long t = clock64();
      tacc[slot] += t - tmark;
      tmark = t;
    }
  };
  int passes = 0;
  for (int pass = 0;; ++pass) {
    const bool first = pass == 0;
    const int par = pass & 1;
    U* pnew = par ? P1v : P0v;
    const U* pold = par ? P0v : P1v;
    ++passes;

    // ---- phase 1: T1 = PhiL . p with p = z + beta p_old formed in shared memory ------------------
    {
      U* as = sm;                 // [KC1][kTL]  PhiL^T rows a, columns (a', beta)
      U* bz = as + KC1 * kTL;     // [KC1][kTL]  z (or x), then p
      U* bp = bz + KC1 * kTL;     // [KC1][kTL]  p_old
      const int nc1 = (N1 + A.tc1 - 1) / A.tc1;
      for (int item = blockIdx.x; item < A.n1; item += gridDim.x) {
        const int mt = item / nc1, ct = item - mt * nc1;
        const int row0 = mt * A.tr1, col0 = ct * A.tc1;
        const int rows = min(A.tr1, M1 - row0), cols = min(A.tc1, N1 - col0);
        const int rows4 = rup4(rows), cols4 = rup4(cols);
        const bool own = mt == 0;
        const Mk mk = mk_setup(rows, cols);
        U acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = U(0);
        for (int k0 = 0; k0 < r0; k0 += KC1) {
          const int kc = min(KC1, r0 - k0);
          __syncthreads();
          copy_rows<U>(as, kTL, PLt + (size_t)k0 * D.M1p + row0, D.M1p, kc, rows4);
          if (first) {
            const int cc = threadIdx.x & 63;
            for (int kb = threadIdx.x >> 6; kb < kc; kb += FT / 64) {
              if (cc < cols) cp1(bz + kb * kTL + cc, A.x + (size_t)(k0 + kb) * N1 + col0 + cc);
              else if (cc < cols4) bz[kb * kTL + cc] = U(0);
            }
          } else {
            copy_rows<U>(bz, kTL, Z + (size_t)k0 * D.N1p + col0, D.N1p, kc, cols4);
            if (pass > 1) copy_rows<U>(bp, kTL, pold + (size_t)k0 * D.N1p + col0, D.N1p, kc, cols4);
          }
          cpa_commit();
          cpa_wait<0>();
          __syncthreads();
          if (!first) {
            const int cc = threadIdx.x & 63;
            if (cc < cols) {
              for (int kb = threadIdx.x >> 6; kb < kc; kb += FT / 64) {
                const U v = pass == 1 ? bz[kb * kTL + cc] : fmaU(beta, bp[kb * kTL + cc], bz[kb * kTL + cc]);
                bz[kb * kTL + cc] = v;
                if (own) pnew[(size_t)(k0 + kb) * D.N1p + col0 + cc] = v;
              }
            }
            __syncthreads();
          }
          if (mk.act) tile_fma<U>(as, bz, kc, mk, acc);
        }
        tile_reduce<U>(mk, acc, sm + KC1 * kTL);  // the staged z/p buffers are free now
        if (mk.act && mk.grp == 0) {
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              const int rr = 4 * mk.ty + i, cc = 4 * mk.tx + j;
              if (rr < rows && cc < cols) {
                const int c = col0 + cc;
                const int jj = c / r1, b = c - jj * r1;
                T1[((size_t)(row0 + rr) * n + jj) * D.r1p + b] = acc[i][j];
              }
            }
        }
      }
    }
    mark(0);
    if (!fcg_sync(A.ctl, bidx)) return;
    mark(1);

    // ---- phase 2: per (a', g-slice) T2 = T1[a'] . A, then its share of B p and p.Bp --------------
    {
      U* As = sm;                        // [2][KC][kTL]
      U* Bs = As + 2 * KC * kTL;         // [2][KC][kTL]
      U* T2s = Bs + 2 * KC * kTL;        // [64][r1]
      U* PN = T2s + 64 * r1;             // [N1p] row a' of p
      U* PRs = PN + rup4(8 * r1);        // [2][PRB]
      const int K2 = D.K2;
      for (int item = blockIdx.x; item < A.n2; item += gridDim.x) {
        const int ap = item / A.S, gs = item - ap * A.S;
        const int g0 = gs * A.gw, gc = min(A.gw, a1 - g0);
        const int rows = n * gc;  // (i, g) with g fastest; <= 64 by the plan
        const int rows4 = rup4(rows);
        const U* Aslice = Apk + (size_t)gs * K2 * D.rows2p;
        const U* T1a = T1 + (size_t)ap * K2 * D.r1p;
        // the second contraction's operands do not depend on the first: row a' of p and the first
        // PhiR chunk are requested now and arrive while T2 is formed
        const int K3 = gc * r1;
        int nbc = max(1, min(r1, PRB / D.K3p));
        if (nbc > FT / 16 && nbc < r1) nbc -= nbc % (FT / 16);  // whole rounds of the warps (2 b' each)
        const int nchk = (r1 + nbc - 1) / nbc;
        const U* PRslice = PRk + (size_t)gs * r1 * D.K3p;
        auto issue3 = [&](int c) {
          const int b0 = c * nbc, nb = min(nbc, r1 - b0);
          copy_flat<U>(PRs + (c & 1) * PRB, PRslice + (size_t)b0 * D.K3p, nb * D.K3p);
          cpa_commit();
        };
        __syncthreads();
        if (!first) copy_flat<U>(PN, pnew + (size_t)ap * D.N1p, D.N1p);
        issue3(0);
        for (int c0 = 0; c0 < r1; c0 += 64) {
          const int cols = min(64, r1 - c0), cols4 = rup4(cols);
          const Mk mk = mk_setup(rows, cols);
          U acc[4][4];
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = U(0);
          const int nch = (K2 + KC - 1) / KC;
          auto issue = [&](int c) {
            const int k0 = c * KC, kc = min(KC, K2 - k0);
            copy_rows<U>(As + (c & 1) * KC * kTL, kTL, Aslice + (size_t)k0 * D.rows2p, D.rows2p, kc, rows4);
            copy_rows<U>(Bs + (c & 1) * KC * kTL, kTL, T1a + (size_t)k0 * D.r1p + c0, D.r1p, kc, cols4);
            cpa_commit();
          };
          issue(0);
          for (int c = 0; c < nch; ++c) {
            if (c + 1 < nch) {
              issue(c + 1);
              cpa_wait<1>();
            } else {
              cpa_wait<0>();
            }
            __syncthreads();
            const int kc = min(KC, K2 - c * KC);
            if (mk.act) tile_fma<U>(As + (c & 1) * KC * kTL, Bs + (c & 1) * KC * kTL, kc, mk, acc);
            __syncthreads();
          }
          tile_reduce<U>(mk, acc, As);  // the chunk buffers (4 KC kTL >= 64 x 64) are free
          if (mk.act && mk.grp == 0) {
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
              for (int j = 0; j < 4; ++j) {
                const int rr = 4 * mk.ty + i, cc = 4 * mk.tx + j;
                if (rr < rows && cc < cols) T2s[rr * r1 + c0 + cc] = acc[i][j];
              }
          }
          __syncthreads();  // the reduction buffer is the next tile's chunk buffer
        }
        mark(2);  // (timing only: the items' two contractions are accumulated in separate slots)
        // (B p)[a'][i][b'] share: sum over k = (g - g0, b) of T2s[i][k] PhiR[b'][g0 + .][.], with
        // the slice's PhiR rows staged nbc b' at a time (chunk 0 requested at the item's start)
        double pap = 0.0, unused = 0.0;
        for (int c = 0; c < nchk; ++c) {
          if (c + 1 < nchk) {
            issue3(c + 1);
            cpa_wait<1>();
          } else {
            cpa_wait<0>();
          }
          __syncthreads();  // T2s complete (first chunk) and this chunk's PhiR staged
          const U* buf = PRs + (c & 1) * PRB;
          const int b0 = c * nbc, nb = min(nbc, r1 - b0);
          U* Ybase = Y + (size_t)gs * r1 * mp + ap * n;
          switch (n) {
            case 1: stage3<U, 1>(T2s, buf, K3, D.K3p, nb, b0, r1, Ybase, mp, PN, first, pap); break;
            case 2: stage3<U, 2>(T2s, buf, K3, D.K3p, nb, b0, r1, Ybase, mp, PN, first, pap); break;
            case 3: stage3<U, 3>(T2s, buf, K3, D.K3p, nb, b0, r1, Ybase, mp, PN, first, pap); break;
            case 4: stage3<U, 4>(T2s, buf, K3, D.K3p, nb, b0, r1, Ybase, mp, PN, first, pap); break;
            case 5: stage3<U, 5>(T2s, buf, K3, D.K3p, nb, b0, r1, Ybase, mp, PN, first, pap); break;
            case 6: stage3<U, 6>(T2s, buf, K3, D.K3p, nb, b0, r1, Ybase, mp, PN, first, pap); break;
            case 7: stage3<U, 7>(T2s, buf, K3, D.K3p, nb, b0, r1, Ybase, mp, PN, first, pap); break;
            default: stage3<U, 8>(T2s, buf, K3, D.K3p, nb, b0, r1, Ybase, mp, PN, first, pap); break;
          }
          __syncthreads();  // the buffer is refilled two chunks later
        }
        block_sum2(pap, unused, red);
        if (threadIdx.x == 0) ppap[item] = pap;
      }
    }
    mark(3);
    if (!fcg_sync(A.ctl, bidx)) return;
    mark(4);

    // ---- phase 3: alpha; r -= alpha B p; z = M^{-1} r; x += alpha p; r.r and r.z shares -------------
    U alpha = U(0);
    if (!first) {
      // the two sums on two warps, then the decision on thread 0
      if (warp == 0) {
        const double v = warp0_sum(ppap, A.n2);
        if (lane == 0) s_sum[0] = v;
      } else if (warp == 1) {
        const double v = warp0_sum(prz + (par ^ 1) * A.n3, A.n3);
        if (lane == 0) s_sum[1] = v;
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        const double pap = s_sum[0], rz = s_sum[1];
        const bool bad = !(pap > 0.0) || !isfinite(pap) || !(rz > 0.0);
        s_state = bad ? 2 : 0;
        s_sc[0] = bad ? 0.0 : rz / pap;
      }
      __syncthreads();
      if (s_state == 2) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
          A.ctl[0] = 2;
          A.ctl[1] = it;
        }
        return;
      }
      alpha = (U)s_sc[0];
    }
    {
      const int S = A.S;
      const int per = (m + A.split - 1) / A.split;
      const int rc = max(1, min(per, kRCB / mp));
      U* Rg = sm;                                        // [(1 + S) mp]: r_old (or g), S shares of B p
      U* rs = Rg + (size_t)(S + 1) * mp;                 // [mp] new residual of the block
      U* xs = rs + mp;                                   // [per] x on the item's rows
      U* ps = xs + rup4(per);                            // [per] p on the item's rows
      float* rf = reinterpret_cast<float*>(ps + rup4(per));  // [mp] binary32 copy of rs
      float* Pr = rf + mp;                               // [rc][m] preconditioner rows
      const U* rold = par ? R0v : R1v;
      U* rdst = par ? R1v : R0v;
      const bool pal = (m & 3) == 0;  // preconditioner rows 16-byte aligned
      for (int item = blockIdx.x; item < A.n3; item += gridDim.x) {
        const int b = item % r1, sl = item / r1;
        const int row0 = sl * per, row1 = min(m, row0 + per);
        __syncthreads();
        if (first) {
          for (int q = threadIdx.x; q < m; q += FT) cp1(Rg + q, A.g + (size_t)q * r1 + b);
        } else {
          copy_flat<U>(Rg, rold + (size_t)b * mp, mp);
        }
        for (int s = 0; s < S; ++s) copy_flat<U>(Rg + (size_t)(s + 1) * mp, Y + ((size_t)s * r1 + b) * mp, mp);
        if (!first) {
          // x and p on the item's rows (strided in b): staged with the rest, not loaded per row
          for (int q = threadIdx.x; q < row1 - row0; q += FT) {
            const int row = row0 + q, a = row / n, j = row - a * n;
            cp1(xs + q, A.x + (size_t)row * r1 + b);
            cp1(ps + q, pnew + (size_t)a * D.N1p + j * r1 + b);
          }
        }
        // the first chunk of preconditioner rows travels with them
        auto issue_p = [&](int rc0, int nr) {
          const float* P = A.Pinv + ((size_t)b * m + rc0) * m;
          if (pal) {
            copy_flat<float>(Pr, P, nr * m);
          } else {
            for (int e = threadIdx.x; e < nr * m; e += FT) cp1(Pr + e, P + e);
          }
        };
        if (A.Pinv && row0 < row1) issue_p(row0, min(rc, row1 - row0));
        cpa_commit();
        cpa_wait<0>();
        __syncthreads();
        for (int q = threadIdx.x; q < m; q += FT) {
          U ys = U(0);
          for (int s = 1; s <= S; ++s) ys += Rg[(size_t)s * mp + q];
          const U v = first ? Rg[q] - ys : Rg[q] - alpha * ys;
          rs[q] = v;
          rf[q] = (float)v;
        }
        double pr = 0.0, pz = 0.0;
        for (int rc0 = row0; rc0 < row1; rc0 += rc) {
          const int nr = min(rc, row1 - rc0);
          __syncthreads();  // rs complete; Pr free
          if (A.Pinv && rc0 > row0) {
            issue_p(rc0, nr);
            cpa_commit();
            cpa_wait<0>();
            __syncthreads();
          }
          for (int rl = warp; rl < nr; rl += FT / 32) {
            const int row = rc0 + rl;
            U zv;
            if (A.Pinv) {
              const float* pr_row = Pr + (size_t)rl * m;
              float acc = 0.0f;
              for (int q = lane; q < m; q += 32) acc = fmaf(pr_row[q], rf[q], acc);
              zv = (U)warp_allsum(acc);
            } else {
              zv = rs[row];
            }
            if (lane == 0) {
              const int a = row / n, j = row - a * n;
              const size_t zi = (size_t)a * D.N1p + j * r1 + b;
              const U rv = rs[row];
              rdst[(size_t)b * mp + row] = rv;
              Z[zi] = zv;
              if (!first) A.x[(size_t)row * r1 + b] = xs[row - row0] + alpha * ps[row - row0];
              pr += (double)rv * (double)rv;
              pz += (double)rv * (double)zv;
            }
          }
        }
        block_sum2(pr, pz, red);
        if (threadIdx.x == 0) {
          prr[par * A.n3 + item] = pr;
          prz[par * A.n3 + item] = pz;
        }
      }
    }
    if (!first) ++it;
    mark(5);
    if (!fcg_sync(A.ctl, bidx)) return;

    // ---- stop test and beta of the next pass -----------------------------------------------
    if (warp < 3) {
      const double* src = warp == 0 ? prr + par * A.n3 : warp == 1 ? prz + par * A.n3 : prz + (par ^ 1) * A.n3;
      const double v = (warp == 2 && first) ? 1.0 : warp0_sum(src, A.n3);
      if (lane == 0) s_sum[warp] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      const double rr = s_sum[0], rzn = s_sum[1], rzo = s_sum[2];
      int st = 0;
      if (rr <= A.stop2) st = 1;
      else if (it >= A.maxit) st = 3;
      s_state = st;
      s_sc[1] = first ? 0.0 : rzn / rzo;
    }
    __syncthreads();
    mark(6);
    if (s_state) {
      state = s_state == 1 ? 1 : 0;
      break;
    }
    beta = (U)s_sc[1];
  }
  if (tp) {
    for (int i = 0; i < 7; ++i) atomicAdd(A.tprof + i, (unsigned long long)tacc[i]);
    atomicAdd(A.tprof + 7, (unsigned long long)passes);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    A.ctl[0] = state;
    A.ctl[1] = it;
  }
}

int sm_count(tnfem_ctx* ctx) { return coop_sms(ctx); }

}  // namespace

FusedCg::~FusedCg() {
  if (prof_on_ && prof_passes_ > 0) {
    static const char* names[7] = {"phase 1",   "barrier 1", "phase 2 T2", "phase 2 Bp",
                                   "barrier 2", "phase 3",   "barrier 3"};
    fprintf(stderr, "[tnfem] fused CG: %.0f passes; SM cycles per pass (mean over CTAs):", prof_passes_);
    for (int i = 0; i < 7; ++i) fprintf(stderr, " %s %.0f", names[i], prof_cycles_[i] / prof_passes_);
    fprintf(stderr, "\n");
  }
  if (ctx_) {
    if (tprof_) dfree(ctx_, tprof_);
    if (ws_) dfree(ctx_, ws_);
    if (parts_) dfree(ctx_, parts_);
    if (ctl_) dfree(ctx_, ctl_);
    if (host_) cudaFreeHost(host_);
  }
}

void FusedCg::ensure(tnfem_ctx* ctx, size_t parts, size_t ws_bytes) {
  if (ctx_ && ctx_ != ctx) throw Error(TNFEM_E_INVALID, "fused CG state used with another context");
  ctx_ = ctx;
  if (!ctl_) {
    prof_on_ = getenv("TNFEM_FCG_PROF") != nullptr;
    if (prof_on_) tprof_ = static_cast<unsigned long long*>(dalloc(ctx, 8 * sizeof(unsigned long long)));
    ctl_ = static_cast<int*>(dalloc(ctx, kCtlInts * sizeof(int)));
    TN_CHECK_CUDA(cudaMallocHost(reinterpret_cast<void**>(&host_), 16 * sizeof(int)));
  }
  if (parts_n_ < parts) {
    if (parts_) dfree(ctx, parts_);
    parts_ = nullptr;
    parts_n_ = 0;
    parts_ = static_cast<double*>(dalloc(ctx, parts * sizeof(double)));
    parts_n_ = parts;
  }
  if (ws_bytes_ < ws_bytes) {
    if (ws_) dfree(ctx, ws_);
    ws_ = nullptr;
    ws_bytes_ = 0;
    ws_ = dalloc(ctx, ws_bytes);
    ws_bytes_ = ws_bytes;
  }
}

template <typename U>
FcgPlan FusedCg::plan(tnfem_ctx* ctx, int r0, int n, int r1, int a0, int a1, bool pre) {
  (void)pre;
  FcgPlan pl;
  if (n < 1 || n > 8 || r0 < 1 || r1 < 1 || a0 < 1 || a1 < 1) return pl;
  if (rup4(r1) > FcgCfg<U>::PRB) return pl;  // one b' row of a PhiR slice must fit a staging buffer
  const int m = r0 * n;
  static std::atomic<unsigned long long> attr_set[2];  // one bit per device and precision
  const unsigned long long bit = 1ull << (ctx->device & 63);
  const int which = sizeof(U) == 8 ? 1 : 0;
  constexpr int kSmemMax = 160 * 1024;
  if (!(attr_set[which] & bit)) {
    TN_CHECK_CUDA(cudaFuncSetAttribute(fcg_kernel<U>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemMax));
    attr_set[which] |= bit;
  }
  const int nsm = sm_count(ctx);
  auto occupancy = [&](size_t smem) {
    int occ = 0;
    if (smem > (size_t)kSmemMax) return 0;
    TN_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fcg_kernel<U>, FT, smem));
    return occ;
  };
  // widest g-slice: n * width <= 64 rows and width * r1 (padded) within a PhiR staging buffer
  int gwmax = std::max(1, std::min(a1, 64 / n));
  while (gwmax > 1 && rup4(gwmax * r1) > FcgCfg<U>::PRB) --gwmax;
  if (rup4(gwmax * r1) > FcgCfg<U>::PRB) return pl;
  const int S0 = (a1 + gwmax - 1) / gwmax;
  int occ = occupancy(fcg_smem_bytes<U>(r1, m, S0, m));
  if (occ < 1) return pl;
  long long slots = (long long)occ * nsm;
  // phase 1: columns in near-equal tiles (multiples of 4) of at most 64; rows (a multiple of 4,
  // at most 64) so that the tiles take the fewest rounds of the resident CTAs, then the fewest rows
  const int M1 = r0 * a0, N1 = n * r1;
  const int nc1 = (N1 + 63) / 64;
  const int tc1 = std::min(64, rup4((N1 + nc1 - 1) / nc1));
  const long long ncol1 = (N1 + tc1 - 1) / tc1;
  long long best1 = -1;
  for (int tr = 4; tr <= 64; tr += 4) {
    const long long items = (long long)((M1 + tr - 1) / tr) * ncol1;
    const long long cost = ((items + slots - 1) / slots) * (std::min(tr, rup4(M1)) + 16);
    if (best1 < 0 || cost < best1) {
      best1 = cost;
      pl.tr1 = tr;
      pl.n1 = (int)items;
    }
  }
  pl.tc1 = tc1;
  // phase 2: the slicing of g with the fewest rounds of the resident CTAs x rows per item
  long long best2 = -1;
  for (int S = S0; S <= a1; ++S) {
    const int gw = (a1 + S - 1) / S;
    if ((a1 + gw - 1) / gw != S) continue;  // the same slicing as a smaller S
    const long long items = (long long)r0 * S;
    const long long cost = ((items + slots - 1) / slots) * (rup4(n * gw) + 8) * ((r1 + 63) / 64);
    if (best2 < 0 || cost < best2) {
      best2 = cost;
      pl.S = S;
      pl.gw = gw;
      pl.n2 = (int)items;
    }
    if (items > 4 * slots) break;
  }
  // phase 3: split each block's rows so that the items fill the resident CTAs (>= 8 rows each)
  pl.split = (int)std::max<long long>(1, std::min<long long>(slots / r1, (m + 7) / 8));
  pl.n3 = r1 * pl.split;
  pl.smem = fcg_smem_bytes<U>(r1, m, pl.S, (m + pl.split - 1) / pl.split);
  occ = occupancy(pl.smem);
  if (occ < 1) return pl;
  slots = (long long)occ * nsm;
  pl.ncta = (int)std::min<long long>(slots, std::max({pl.n1, pl.n2, pl.n3}));
  pl.ws_bytes = fcg_dims(r0, n, r1, a0, pl.S, pl.gw).total * sizeof(U) + 256;
  pl.ok = pl.ncta >= 1;
  return pl;
}

template <typename U>
int FusedCg::run(tnfem_ctx* ctx, const FcgPlan& pl, int r0, int n, int r1, int a0, int a1, const U* PL,
                 const U* Ap, const U* PR, const float* Pinv, const U* g, U* x, double stop2, int maxit,
                 int* state) {
  TN_REQUIRE(pl.ok, "fused CG: no plan for this system");
  ensure(ctx, (size_t)pl.n2 + 4 * (size_t)pl.n3, pl.ws_bytes);
  const FcgDims D = fcg_dims(r0, n, r1, a0, pl.S, pl.gw);
  U* ws = static_cast<U*>(ws_);
  // repack the operators; zero the vectors (their padding must stay finite)
  {
    const long long work = std::max<long long>({(long long)r0 * D.M1p, (long long)pl.S * D.K2 * D.rows2p,
                                                (long long)pl.S * r1 * D.K3p});
    const int blocks = (int)std::max<long long>(1, std::min<long long>(1216, (work + 255) / 256));
    fcg_pack_kernel<U><<<blocks, 256, 0, ctx->stream>>>(r0, n, r1, a0, a1, pl.S, pl.gw, PL, Ap, PR, ws);
    count_launch(ctx);
    TN_CHECK_CUDA(cudaMemsetAsync(ws + D.zero_from, 0, (D.total - D.zero_from) * sizeof(U), ctx->stream));
  }
  FcgArgs<U> a;
  a.r0 = r0; a.n = n; a.r1 = r1; a.a0 = a0; a.a1 = a1;
  a.tr1 = pl.tr1; a.tc1 = pl.tc1; a.n1 = pl.n1; a.S = pl.S; a.gw = pl.gw; a.n2 = pl.n2;
  a.split = pl.split; a.n3 = pl.n3; a.maxit = std::max(0, maxit);
  a.stop2 = stop2;
  a.g = g; a.Pinv = Pinv; a.x = x; a.ws = ws;
  a.parts = parts_;
  a.ctl = ctl_;
  a.tprof = nullptr;
  if (prof_on_) {
    a.tprof = tprof_;
    TN_CHECK_CUDA(cudaMemsetAsync(tprof_, 0, 8 * sizeof(unsigned long long), ctx->stream));
  }
  TN_CHECK_CUDA(cudaMemsetAsync(ctl_, 0, kCtlInts * sizeof(int), ctx->stream));
  void* args[] = {&a};
  int pidx = -1;
  {
    ProfScope ps(ctx, sizeof(U) == 8 ? TNFEM_PROF_CG64 : TNFEM_PROF_CG32, 0.0, 0.0);
    pidx = ps.idx;
    TN_CHECK_CUDA(cudaLaunchCooperativeKernel(reinterpret_cast<void*>(fcg_kernel<U>), dim3(pl.ncta), dim3(FT), args,
                                              pl.smem, ctx->stream));
  }
  count_launch(ctx);
  check_launch(ctx, "fused conjugate gradients");
  TN_CHECK_CUDA(cudaMemcpyAsync(host_, ctl_, 8 * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  sync(ctx);
  if (static_cast<unsigned int>(host_[4 + 1]) & kGridErrBit)
    throw Error(TNFEM_E_TIMEOUT, "fused conjugate gradients: a grid barrier wait expired");
  const int its = host_[1];
  *state = host_[0];
  if (prof_on_) {
    unsigned long long h[8];
    TN_CHECK_CUDA(cudaMemcpy(h, tprof_, 8 * sizeof(unsigned long long), cudaMemcpyDeviceToHost));
    for (int i = 0; i < 7; ++i) prof_cycles_[i] += (double)h[i] / std::max(1, pl.ncta);
    prof_passes_ += (double)h[7] / std::max(1, pl.ncta);
  }
  // algorithmic work: its + 1 local matvecs and block-Jacobi applies
  const double mm = (double)r0 * n;
  const double fmv = 2.0 * n * r0 * r1 * ((double)r0 * a0 + (double)n * a0 * a1 + (double)r1 * a1);
  const double fbj = Pinv ? 2.0 * r1 * mm * mm : 0.0;
  prof_set_work(ctx, pidx, (its + 1) * (fmv + fbj), 0.0);
  return its;
}

#define TN_INST_FCG(U)                                                                                          \
  template FcgPlan FusedCg::plan<U>(tnfem_ctx*, int, int, int, int, int, bool);                                 \
  template int FusedCg::run<U>(tnfem_ctx*, const FcgPlan&, int, int, int, int, int, const U*, const U*, const U*, \
                               const float*, const U*, U*, double, int, int*);
TN_INST_FCG(float)
TN_INST_FCG(double)

}  // namespace tnfem
