// The local matvec (step a4) of the binary32 local solves on the tcgen05 tensor cores, fed by
// bulk TMA copies of pre-packed operands.
//
//   stage 1  T1[(a',beta)][(j,b)] = PhiL[(a',beta)][a] . x[a][(j,b)]          K = r0
//   stage 2  T2[(a',b)][(i,g)]    = T1[(a',b)][(beta,j)] . Ap[(beta,j)][(i,g)]  K = a0 n
//   stage 3  y[(a',i)][b']        = T2[(a',i)][(g,b)] . PhiR[b'][(g,b)]       K = a1 r1
//
// Every operand lives in HBM in the "packed" layout the MMAs read: tiles of RB rows x 32 K of TF32
// words, three planes hi = tf32(v), mid = tf32(v - hi), lo = tf32(v - hi - mid) (33 significant
// bits, more than binary32's 24), each plane in the canonical no-swizzle K-major core-matrix layout
// (8 rows x 16 bytes per core matrix).  A whole tile is one
// contiguous block, so a CTA stages it with a single cp.async.bulk into shared memory and the
// tensor cores read it from there unchanged.  The constant operands (PhiL, the operator core,
// PhiR) are packed once per local solve; x is packed once per matvec; stages 1 and 2 write their
// products straight into the packed layout of the next stage's A operand (the stage maps below),
// so no intermediate is ever re-read in plain form.  Six MMAs per K step (hi.hi, hi.mid, mid.hi,
// hi.lo, mid.mid, lo.hi: every product down to 2^-33 relative) leave binary32 accumulation in
// tensor memory as the only rounding, i.e. the accuracy of a binary32 CUDA-core contraction.
//
// Stage 3 has a long K (a1 r1); its K range is split over CTAs whose partial products are summed in
// split order by a small reduction kernel (deterministic, no atomics).  Every mbarrier wait is
// bounded; on expiry the CTA records an error, skips its output, frees its tensor memory and
// returns.
#include <atomic>
#include <algorithm>

#include "internal.h"
#include "tc_common.cuh"
#include "tc_matvec.h"

namespace tnfem {

namespace {

using namespace tc;

constexpr int KCH = 32;        // K words per tile
constexpr int TN = 64;         // N of every MMA here
constexpr int STAGES = 3;      // TMA pipeline depth
constexpr int NT = 128;        // threads per CTA
constexpr int NP = 3;          // TF32 planes per operand: hi, mid, lo
constexpr int kPlaneA = TM * KCH * 4;      // bytes of one TF32 plane of an A tile
constexpr int kPlaneB = TN * KCH * 4;      // ... of a B tile
constexpr int kTileA = NP * kPlaneA;
constexpr int kTileB = NP * kPlaneB;
constexpr int kStageBytes = kTileA + kTileB;

__device__ __forceinline__ uint32_t core_off(int row, int kg) {
  return (uint32_t)((row >> 3) * (KCH / 4) * 128 + kg * 128 + (row & 7) * 16);
}

// word offset of element (row, k) in plane 0 of a packed operand with tiles of TM rows
__device__ __forceinline__ long long packed_word_tm(int row, int k, int nkc) {
  const long long tile = (long long)(row >> 7) * nkc + (k >> 5);
  const int r = row & (TM - 1), kk = k & (KCH - 1);
  return tile * ((long long)NP * TM * KCH) + core_off(r, kk >> 2) / 4 + (kk & 3);
}

__device__ __forceinline__ void split3(float v, uint32_t& hi, uint32_t& mid, uint32_t& lo) {
  hi = to_tf32(v);
  const float r1 = v - __uint_as_float(hi);
  mid = to_tf32(r1);
  lo = to_tf32(r1 - __uint_as_float(mid));
}

// dst = packed(src): element (row, k) = src[row * sr + k * sk] for row < rows, k < K, zero beyond.
__global__ void pack_kernel(uint32_t* __restrict__ dst, const float* __restrict__ src, long long sr, long long sk,
                            int rows, int K, int rb, int nrb, int nkc) {
  const long long groups = (long long)nrb * rb * nkc * (KCH / 4);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < groups;
       t += (long long)gridDim.x * blockDim.x) {
    const int row = (int)(t / (nkc * (KCH / 4)));
    const int kg = (int)(t % (nkc * (KCH / 4)));
    uint32_t hi[4], mid[4], lo[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int k = kg * 4 + e;
      const float v = (row < rows && k < K) ? src[row * sr + k * sk] : 0.f;
      split3(v, hi[e], mid[e], lo[e]);
    }
    const long long tile = (long long)(row / rb) * nkc + (kg * 4) / KCH;
    const long long base = tile * ((long long)NP * rb * KCH) + core_off(row % rb, kg % (KCH / 4)) / 4;
    *reinterpret_cast<uint4*>(dst + base) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
    *reinterpret_cast<uint4*>(dst + base + rb * KCH) = make_uint4(mid[0], mid[1], mid[2], mid[3]);
    *reinterpret_cast<uint4*>(dst + base + 2 * rb * KCH) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
  }
}

enum Epi { EPI_STAGE1 = 1, EPI_STAGE2 = 2, EPI_PLAIN = 3 };

struct StageArgs {
  const uint32_t* A;  // packed, tiles of 128 rows
  const uint32_t* B;  // packed, tiles of TN rows
  int nkc;            // K tiles (same for A and B)
  int rows, N;        // valid output extent
  int splits, kc_per_split;
  // EPI_STAGE1 / 2: destination packed operand (tiles of 128 rows) and the stage map
  uint32_t* D;
  int d_nkc;
  int dm, dn, mr, mk;
  // EPI_PLAIN: y[m * N + n], or split-K partials work[split][m][n] when splits > 1
  float* Y;
  float* work;
  int* err;
  const int* skip;
};

template <int EPI>
__global__ void __launch_bounds__(NT) tc_stage_kernel(StageArgs g) {
  if (g.skip && *g.skip) return;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  __shared__ __align__(8) uint64_t full[STAGES], empty[STAGES], done;
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int rbA = blockIdx.x, rbB = blockIdx.y, sp = blockIdx.z;
  const int c0 = sp * g.kc_per_split;
  const int c1 = min(g.nkc, c0 + g.kc_per_split);
  const int nch = c1 - c0;

  if (warp == 0) tmem_alloc(smem_u32(&tmem_base), TN);
  if (tid == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), 1);
    }
    mbar_init(smem_u32(&done), 1);
    mbar_init_fence();
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_base;

  bool ok = true;
  if (tid == 0) {
    const uint32_t sbase = smem_u32(smem);
    auto load = [&](int i) {  // chunk c0 + i into stage i % STAGES
      const int s = i % STAGES;
      const uint32_t dst = sbase + s * kStageBytes;
      const int c = c0 + i;
      mbar_arrive_expect_tx(smem_u32(&full[s]), kStageBytes);
      tma_load_1d(dst, g.A + ((long long)rbA * g.nkc + c) * (kTileA / 4), kTileA, smem_u32(&full[s]));
      tma_load_1d(dst + kTileA, g.B + ((long long)rbB * g.nkc + c) * (kTileB / 4), kTileB, smem_u32(&full[s]));
    };
    uint32_t fph[STAGES] = {0u, 0u, 0u}, eph[STAGES] = {0u, 0u, 0u};
    for (int i = 0; i < min(STAGES, nch); ++i) load(i);
    constexpr uint32_t idesc = make_idesc(TN);
    constexpr uint32_t lbo = 128, sbo = (KCH / 4) * 128;
    for (int i = 0; i < nch && ok; ++i) {
      const int s = i % STAGES;
      if (!mbar_wait(smem_u32(&full[s]), fph[s])) { ok = false; break; }
      fph[s] ^= 1u;
      fence_after();
      const uint32_t a0p = sbase + s * kStageBytes;
      const uint32_t b0p = a0p + kTileA;
#pragma unroll
      for (int st = 0; st < KCH / 8; ++st) {
        const uint32_t ko = st * 256;
        const uint64_t da0 = make_desc(a0p + ko, lbo, sbo), da1 = make_desc(a0p + kPlaneA + ko, lbo, sbo),
                       da2 = make_desc(a0p + 2 * kPlaneA + ko, lbo, sbo);
        const uint64_t db0 = make_desc(b0p + ko, lbo, sbo), db1 = make_desc(b0p + kPlaneB + ko, lbo, sbo),
                       db2 = make_desc(b0p + 2 * kPlaneB + ko, lbo, sbo);
        // small terms first: hi.lo, mid.mid, lo.hi, hi.mid, mid.hi, hi.hi
        mma_tf32(tmem, da0, db2, idesc, (i > 0 || st > 0) ? 1u : 0u);
        mma_tf32(tmem, da1, db1, idesc, 1u);
        mma_tf32(tmem, da2, db0, idesc, 1u);
        mma_tf32(tmem, da0, db1, idesc, 1u);
        mma_tf32(tmem, da1, db0, idesc, 1u);
        mma_tf32(tmem, da0, db0, idesc, 1u);
      }
      mma_commit(smem_u32(&empty[s]));
      // refill the stage of the previous chunk once its MMAs (issued one step ago) are done
      if (i >= 1 && i - 1 + STAGES < nch) {
        const int sp_ = (i - 1) % STAGES;
        if (!mbar_wait(smem_u32(&empty[sp_]), eph[sp_])) { ok = false; break; }
        eph[sp_] ^= 1u;
        load(i - 1 + STAGES);
      }
    }
    if (ok) mma_commit(smem_u32(&done));
  }
  // everyone waits for the accumulator; the outcome is agreed by the whole CTA
  const bool w = (tid == 0 && !ok) ? false : mbar_wait(smem_u32(&done), 0u);
  ok = __syncthreads_and(w) != 0;
  fence_after();
  if (ok) {
    const int r = warp * 32 + lane;       // TMEM lane = row of the tile
    const int m = rbA * TM + r;
    const bool row_ok = m < g.rows;
    // per-row part of the stage map (one division per row, none per element)
    const int qa = row_ok && EPI != EPI_PLAIN ? m / g.dm : 0;
    const int ra = row_ok && EPI != EPI_PLAIN ? m - qa * g.dm : 0;
    float* part = (EPI == EPI_PLAIN && g.splits > 1) ? g.work + (long long)sp * g.rows * g.N : nullptr;
#pragma unroll 1
    for (int cc = 0; cc < TN; cc += 16) {
      uint32_t v[16];
      tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)cc, v);
      if (!row_ok) continue;
      const int nb = rbB * TN + cc;
      if (EPI == EPI_PLAIN) {
        float* dst = part ? part + (long long)m * g.N : g.Y + (long long)m * g.N;
#pragma unroll
        for (int e = 0; e < 16; ++e)
          if (nb + e < g.N) dst[nb + e] = __uint_as_float(v[e]);
      } else {
        int q = nb / g.dn, rr = nb - q * g.dn;  // n = q dn + rr, advanced incrementally
#pragma unroll
        for (int e = 0; e < 16; ++e) {
          if (nb + e < g.N) {
            // stage 1: m = a' dm + beta, n = j dn + b  ->  (a' mr + b, beta mk + j)
            // stage 2: m = a' dm + b,    n = i dn + g  ->  (a' mr + i, g mk + b)
            const int row2 = EPI == EPI_STAGE1 ? qa * g.mr + rr : qa * g.mr + q;
            const int k2 = EPI == EPI_STAGE1 ? ra * g.mk + q : rr * g.mk + ra;
            uint32_t hi, mid, lo;
            split3(__uint_as_float(v[e]), hi, mid, lo);
            const long long w = packed_word_tm(row2, k2, g.d_nkc);
            g.D[w] = hi;
            g.D[w + TM * KCH] = mid;
            g.D[w + 2 * TM * KCH] = lo;
          }
          if (++rr == g.dn) { rr = 0; ++q; }
        }
      }
    }
  } else if (tid == 0) {
    atomicExch(g.err, 1);
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0) tmem_dealloc(tmem, TN);
}

constexpr int kSmem = STAGES * kStageBytes + 1024;

template <int EPI>
void launch_stage(tnfem_ctx* ctx, const StageArgs& a, int nrbA, int nrbB, int splits, double flops, double bytes) {
  static std::atomic<unsigned long long> attr_set{0};
  const unsigned long long bit = 1ull << (ctx->device & 63);
  if (!(attr_set & bit)) {
    TN_CHECK_CUDA(cudaFuncSetAttribute(tc_stage_kernel<EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem));
    attr_set |= bit;
  }
  ProfScope ps(ctx, TNFEM_PROF_CONTRACT32, flops, bytes);
  tc_stage_kernel<EPI><<<dim3(nrbA, nrbB, splits), NT, kSmem, ctx->stream>>>(a);
  count_launch(ctx);
}

inline int cdiv(long long a, long long b) { return (int)((a + b - 1) / b); }

}  // namespace

void TcMatvec::plan(tnfem_ctx* ctx, int r0_, int n_, int r1_, int a0_, int a1_) {
  r0 = r0_; n = n_; r1 = r1_; a0 = a0_; a1 = a1_;
  auto dims = [](int rows, int K, int rb) { return PackDims{rows, K, rb, cdiv(rows, rb), cdiv(K, KCH)}; };
  pl = dims(r0 * a0, r0, TM);        // stage 1 A: rows (a',beta), K = a
  xp = dims(n * r1, r0, TN);         // stage 1 B: rows (j,b), K = a
  t1 = dims(r0 * r1, a0 * n, TM);    // stage 2 A: rows (a',b), K = (beta,j)
  ap = dims(n * a1, a0 * n, TN);     // stage 2 B: rows (i,g), K = (beta,j)
  t2 = dims(r0 * n, a1 * r1, TM);    // stage 3 A: rows (a',i), K = (g,b)
  pr = dims(r1, a1 * r1, TN);        // stage 3 B: rows b', K = (g,b)
  auto words = [](const PackDims& d) { return (size_t)d.nrb * d.nkc * NP * d.rb * KCH; };
  PL.ensure(ctx, words(pl));
  XP.ensure(ctx, words(xp));
  T1.ensure(ctx, words(t1));
  AP.ensure(ctx, words(ap));
  T2.ensure(ctx, words(t2));
  PR.ensure(ctx, words(pr));
  // stage 3 split over K: about four K tiles per CTA, at most ~one wave of CTAs
  const int tiles3 = t2.nrb * pr.nrb;
  splits3 = std::max(1, std::min(cdiv(t2.nkc, 4), std::max(1, 152 / tiles3)));
  kc3 = cdiv(t2.nkc, splits3);
  splits3 = cdiv(t2.nkc, kc3);
  work.ensure(ctx, (size_t)splits3 * r0 * n * r1);
  // padding of the packed intermediates must read as zero; the products rewrite the rest
  TN_CHECK_CUDA(cudaMemsetAsync(T1.p, 0, words(t1) * sizeof(uint32_t), ctx->stream));
  TN_CHECK_CUDA(cudaMemsetAsync(T2.p, 0, words(t2) * sizeof(uint32_t), ctx->stream));
}

void TcMatvec::pack(tnfem_ctx* ctx, uint32_t* dst, const PackDims& d, const float* src, long long sr, long long sk) {
  const long long groups = (long long)d.nrb * d.rb * d.nkc * (KCH / 4);
  ProfScope ps(ctx, TNFEM_PROF_OTHER, 0.0, (double)d.rows * d.K * 4 + groups * 32.0);
  pack_kernel<<<(int)std::min<long long>(152 * 8, (groups + 255) / 256), 256, 0, ctx->stream>>>(dst, src, sr, sk, d.rows,
                                                                                                d.K, d.rb, d.nrb, d.nkc);
  count_launch(ctx);
}

void TcMatvec::prepare(tnfem_ctx* ctx, const float* PhiL, const float* Ap, const float* PhiR) {
  // PhiL[a'][beta][a]: row (a',beta) stride r0, k = a stride 1
  pack(ctx, PL.p, pl, PhiL, r0, 1);
  // Ap[beta][j][i][g]: row (i,g) stride 1, k = (beta,j) stride n a1
  pack(ctx, AP.p, ap, Ap, 1, (long long)n * a1);
  // PhiR[b'][g][b]: row b' stride a1 r1, k = (g,b) stride 1
  pack(ctx, PR.p, pr, PhiR, (long long)a1 * r1, 1);
  check_launch(ctx, "tensor-core matvec prepare");
}

void TcMatvec::apply(tnfem_ctx* ctx, const float* x, float* y, const int* skip) {
  int* err = reinterpret_cast<int*>(ctx->scratch + kScratchDoubles - 8);
  // x[a][j][b]: row (j,b) stride 1, k = a stride n r1
  pack(ctx, XP.p, xp, x, 1, (long long)n * r1);
  const double f1 = 2.0 * r0 * a0 * r0 * n * r1, f2 = 2.0 * r0 * r1 * a0 * n * n * a1, f3 = 2.0 * r0 * n * a1 * r1 * r1;
  StageArgs s1{};
  s1.A = PL.p; s1.B = XP.p; s1.nkc = pl.nkc; s1.rows = r0 * a0; s1.N = n * r1;
  s1.splits = 1; s1.kc_per_split = pl.nkc;
  s1.D = T1.p; s1.d_nkc = t1.nkc; s1.dm = a0; s1.dn = r1; s1.mr = r1; s1.mk = n;
  s1.err = err; s1.skip = skip;
  launch_stage<EPI_STAGE1>(ctx, s1, pl.nrb, xp.nrb, 1, f1, 4.0 * (r0 * a0 * r0 + r0 * n * r1 + r0 * a0 * n * r1));
  StageArgs s2{};
  s2.A = T1.p; s2.B = AP.p; s2.nkc = t1.nkc; s2.rows = r0 * r1; s2.N = n * a1;
  s2.splits = 1; s2.kc_per_split = t1.nkc;
  s2.D = T2.p; s2.d_nkc = t2.nkc; s2.dm = r1; s2.dn = a1; s2.mr = n; s2.mk = r1;
  s2.err = err; s2.skip = skip;
  launch_stage<EPI_STAGE2>(ctx, s2, t1.nrb, ap.nrb, 1, f2, 4.0 * (2.0 * r0 * r1 * a0 * n + a0 * n * n * a1));
  StageArgs s3{};
  s3.A = T2.p; s3.B = PR.p; s3.nkc = t2.nkc; s3.rows = r0 * n; s3.N = r1;
  s3.splits = splits3; s3.kc_per_split = kc3;
  s3.Y = y; s3.work = work.p;
  s3.err = err; s3.skip = skip;
  launch_stage<EPI_PLAIN>(ctx, s3, t2.nrb, pr.nrb, splits3, f3, 4.0 * (r0 * n * a1 * r1 + r1 * a1 * r1 + r0 * n * r1));
  if (splits3 > 1) {
    GemmDesc gr{r0 * n, r1, 1, 1, 0, 0, 0, 0, 0, 0, r1, 1, 0};
    splitk_reduce<float>(ctx, gr, 1.0f, 0.0f, y, work.p, splits3, skip);
  }
  check_launch(ctx, "tensor-core matvec");
}

}  // namespace tnfem
