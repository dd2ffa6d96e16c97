// Batched binary32 GEMM on the sm_103a tensor cores (tcgen05, kind::tf32) with the three-term
// split that recovers binary32 accuracy from TF32 products:
//
//   a = a_hi + a_lo,  b = b_hi + b_lo  (a_hi = tf32(a), a_lo = tf32(a - a_hi), same for b)
//   a b ~= a_hi b_hi + a_hi b_lo + a_lo b_hi          (the a_lo b_lo term is below fp32 rounding)
//
// so every K step issues three 128 x TN x 8 MMAs accumulating in tensor memory (FP32).  This is
// the dense contraction of the binary32 local solves (the stages of the local matvec).
//
// Kernel structure (one CTA = one 128-row tile of C, 128 threads = 4 warps):
//  - rows of the tile are the flattened (batch, m) pairs when B is shared by all batches, else the
//    m rows of one batch (grid.z = batch); A, B and C may have any strides, so operands are staged
//    by ordinary loads (thread = row of A / column of B), split into hi / lo TF32 words and stored
//    in the canonical no-swizzle K-major core-matrix layout (8 rows x 16 bytes per core matrix);
//  - one elected thread issues tcgen05.mma for the chunk and commits to an mbarrier; the next
//    chunk is staged into the other buffer while the tensor cores work on this one;
//  - the accumulator (128 lanes x TN columns of TMEM) is read back with tcgen05.ld.32x32b (warp w
//    owns lanes 32w..32w+31 = rows) and written to C with alpha / beta.
// Every mbarrier wait is bounded: on expiry the kernel records an error, waits (bounded) for its
// own MMAs, frees its TMEM and returns.
#include <atomic>
#include <algorithm>

#include "internal.h"
#include "tc_common.cuh"
#include "tc_gemm.h"

namespace tnfem {

namespace {

using namespace tc;
constexpr int KC = 32;   // K elements per staged chunk (4 MMA K steps of 8)
constexpr int NT = 128;  // threads per CTA
constexpr int kTileABytes = TM * KC * 4;  // one TF32 plane of the A tile

// offset in bytes of element (row, k) of a rows x KC tile in the core-matrix K-major layout
__device__ __forceinline__ uint32_t tile_off(int row, int kg) {
  // kg = k / 4 (16-byte group); within a core matrix rows are 16 bytes apart
  return (uint32_t)((row >> 3) * (KC / 4) * 128 + kg * 128 + (row & 7) * 16);
}

struct TcArgs {
  int M, N, K, batch;
  long long sAm, sAk, sAb, sBk, sBn, sBb, sCm, sCn, sCb;
  int rows;    // rows covered by the grid's x dimension (M or M * batch when flattened)
  int flat;    // 1: rows are flattened (batch, m) pairs (B shared), 0: grid.z runs over batches
  int splits;  // K ranges; > 1 writes partial tiles to `work` ([split][batch][M][N]) instead of C
  int kchunk;  // K elements per split (multiple of KC)
};

template <int TN>
__global__ void __launch_bounds__(NT) tc_gemm_kernel(TcArgs g, float alpha, const float* __restrict__ A,
                                                     const float* __restrict__ B, float beta, float* __restrict__ C,
                                                     float* __restrict__ work, int* __restrict__ err,
                                                     const int* __restrict__ skip) {
  if (skip && *skip) return;
  constexpr int kTileBBytes = TN * KC * 4;
  constexpr int kStage = 2 * kTileABytes + 2 * kTileBBytes;  // A hi, A lo, B hi, B lo
  extern __shared__ unsigned char smem_raw[];
  // 1024-byte aligned start of the staging buffers (the launch reserves 1 KiB of slack)
  unsigned char* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int row0 = blockIdx.x * TM;
  const int n0 = blockIdx.y * TN;
  const int sp = blockIdx.z % g.splits;
  const int zb = g.flat ? 0 : blockIdx.z / g.splits;
  const int kbeg = sp * g.kchunk;
  const int kend = min(g.K, kbeg + g.kchunk);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(TN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[1])));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_base;

  // this thread's row of A (thread = row) and the A / C base of that row
  const int arow = row0 + tid;
  const bool arow_ok = arow < g.rows;
  long long a_base = 0;
  if (arow_ok) {
    const int b = g.flat ? arow / g.M : zb;
    const int m = g.flat ? arow % g.M : arow;
    a_base = (long long)b * g.sAb + (long long)m * g.sAm;
  }
  const long long b_base = (long long)zb * g.sBb;
  const int nchunks = (kend - kbeg + KC - 1) / KC;
  constexpr uint32_t idesc = make_idesc(TN);
  uint32_t phase[2] = {0u, 0u};
  bool ok = true;

  for (int c = 0; c < nchunks; ++c) {
    const int buf = c & 1;
    unsigned char* st = smem + buf * kStage;
    // the MMAs that last read this buffer (chunk c - 2) must be done before it is overwritten;
    // the outcome of the bounded wait is agreed by the whole CTA so that all threads leave together
    if (c >= 2) {
      const bool w = mbar_wait(smem_u32(&mbar[buf]), phase[buf]);
      if (!__syncthreads_and(w)) { ok = false; break; }
      phase[buf] ^= 1u;
    }
    const int k0 = kbeg + c * KC;
    // stage A: thread = row; 8 groups of 4 consecutive k
    {
      unsigned char* ahi = st;
      unsigned char* alo = st + kTileABytes;
#pragma unroll
      for (int kg = 0; kg < KC / 4; ++kg) {
        uint32_t hi[4], lo[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int k = k0 + kg * 4 + e;
          float v = 0.f;
          if (arow_ok && k < kend) v = A[a_base + (long long)k * g.sAk];
          hi[e] = to_tf32(v);
          lo[e] = to_tf32(v - __uint_as_float(hi[e]));
        }
        const uint32_t off = tile_off(tid, kg);
        *reinterpret_cast<uint4*>(ahi + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
        *reinterpret_cast<uint4*>(alo + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
      }
    }
    // stage B: thread = column n (TN / NT columns each)
    {
      unsigned char* bhi = st + 2 * kTileABytes;
      unsigned char* blo = bhi + kTileBBytes;
      for (int nl = tid; nl < TN; nl += NT) {
        const int n = n0 + nl;
        const bool n_ok = n < g.N;
#pragma unroll
        for (int kg = 0; kg < KC / 4; ++kg) {
          uint32_t hi[4], lo[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int k = k0 + kg * 4 + e;
            float v = 0.f;
            if (n_ok && k < kend) v = B[b_base + (long long)k * g.sBk + (long long)n * g.sBn];
            hi[e] = to_tf32(v);
            lo[e] = to_tf32(v - __uint_as_float(hi[e]));
          }
          const uint32_t off = tile_off(nl, kg);
          *reinterpret_cast<uint4*>(bhi + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
          *reinterpret_cast<uint4*>(blo + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
        }
      }
    }
    // make the generic-proxy stores visible to the tensor cores, then one thread issues
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    fence_before();
    __syncthreads();
    if (tid == 0) {
      fence_after();
      const uint32_t s_ahi = smem_u32(st), s_alo = s_ahi + kTileABytes;
      const uint32_t s_bhi = s_ahi + 2 * kTileABytes, s_blo = s_bhi + kTileBBytes;
      constexpr uint32_t lbo = 128, sbo = (KC / 4) * 128;
#pragma unroll
      for (int s = 0; s < KC / 8; ++s) {
        const uint32_t koff = s * 2 * 128;  // two 16-byte k groups per K step of 8
        const uint64_t dah = make_desc(s_ahi + koff, lbo, sbo), dal = make_desc(s_alo + koff, lbo, sbo);
        const uint64_t dbh = make_desc(s_bhi + koff, lbo, sbo), dbl = make_desc(s_blo + koff, lbo, sbo);
        mma_tf32(tmem, dah, dbh, idesc, (c > 0 || s > 0) ? 1u : 0u);
        mma_tf32(tmem, dah, dbl, idesc, 1u);
        mma_tf32(tmem, dal, dbh, idesc, 1u);
      }
      mma_commit(smem_u32(&mbar[buf]));
    }
  }
  // wait for the last commit of each buffer that is still outstanding
  if (ok) {
    for (int buf = 0; buf < 2; ++buf) {
      const int uses = (nchunks - buf + 1) / 2;  // chunks that used this buffer; all but the last waited
      if (uses >= 1) {
        const bool w = mbar_wait(smem_u32(&mbar[buf]), phase[buf]);
        if (!__syncthreads_and(w)) { ok = false; break; }
        phase[buf] ^= 1u;
      }
    }
  }
  fence_after();
  if (ok) {
    // epilogue: warp w reads TMEM lanes 32w..32w+31 (rows), 16 columns at a time
    const int row = row0 + warp * 32 + lane;
    const bool row_ok = row < g.rows;
    long long cb = 0, wb = 0;
    if (row_ok) {
      const int b = g.flat ? row / g.M : zb;
      const int m = g.flat ? row % g.M : row;
      cb = (long long)b * g.sCb + (long long)m * g.sCm;
      wb = (((long long)sp * g.batch + b) * g.M + m) * g.N;
    }
#pragma unroll 1
    for (int cc = 0; cc < TN; cc += 16) {
      uint32_t v[16];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)cc;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (row_ok) {
#pragma unroll
        for (int e = 0; e < 16; ++e) {
          const int n = n0 + cc + e;
          if (n < g.N) {
            if (g.splits > 1) {
              work[wb + n] = __uint_as_float(v[e]);
            } else {
              float* cp = C + cb + (long long)n * g.sCn;
              float r = alpha * __uint_as_float(v[e]);
              if (beta != 0.f) r += beta * (*cp);
              *cp = r;
            }
          }
        }
      }
    }
  } else if (tid == 0) {
    atomicExch(err, 1);
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TN));
}

template <int TN>
constexpr int stage_bytes() {
  return 2 * kTileABytes + 2 * TN * KC * 4;
}

template <int TN>
void launch_tc(tnfem_ctx* ctx, const TcArgs& a, float alpha, const float* A, const float* B, float beta, float* C,
               float* work, int* err, const int* skip) {
  const int smem = 2 * stage_bytes<TN>() + 1024;
  static std::atomic<unsigned long long> attr_set{0};  // one bit per device: the attribute is per device
  const unsigned long long bit = 1ull << (ctx->device & 63);
  if (!(attr_set & bit)) {
    TN_CHECK_CUDA(cudaFuncSetAttribute(tc_gemm_kernel<TN>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    attr_set |= bit;
  }
  dim3 grid((a.rows + TM - 1) / TM, (a.N + TN - 1) / TN, (a.flat ? 1 : a.batch) * a.splits);
  tc_gemm_kernel<TN><<<grid, NT, smem, ctx->stream>>>(a, alpha, A, B, beta, C, work, err, skip);
  count_launch(ctx);
}

}  // namespace

bool tc_gemm_supported(const GemmDesc& g) {
  if (g.M <= 0 || g.N <= 0 || g.K <= 0 || g.batch <= 0) return false;
  const long long rows = g.sBb == 0 ? (long long)g.M * g.batch : g.M;
  if (rows >= (1ll << 31) || g.batch >= 65536) return false;
  return true;
}

void tc_gemm(tnfem_ctx* ctx, const GemmDesc& g, float alpha, const float* A, const float* B, float beta, float* C,
             float* work, size_t work_elems, const int* skip) {
  TN_REQUIRE(tc_gemm_supported(g), "tensor-core GEMM: unsupported shape");
  TcArgs a{g.M, g.N, g.K, g.batch, g.sAm, g.sAk, g.sAb, g.sBk, g.sBn, g.sBb, g.sCm, g.sCn, g.sCb, 0, 0, 1, 0};
  a.flat = g.sBb == 0 ? 1 : 0;
  a.rows = a.flat ? g.M * g.batch : g.M;
  const int tn = g.N <= 64 ? 64 : 128;
  const long long tiles = (long long)((a.rows + TM - 1) / TM) * ((g.N + tn - 1) / tn) * (a.flat ? 1 : g.batch);
  // split K when the tiles alone leave most SMs idle and K is long
  const int kchunks = (g.K + KC - 1) / KC;
  int splits = 1;
  if (work && tiles < 152 && kchunks >= 4) {
    long long want = (152 + tiles - 1) / tiles;
    long long fit = (long long)(work_elems / ((size_t)g.batch * g.M * g.N));
    splits = (int)std::max<long long>(1, std::min(std::min(want, (long long)kchunks / 2), std::min(fit, 64ll)));
  }
  int kc = ((kchunks + splits - 1) / splits) * KC;
  splits = (g.K + kc - 1) / kc;
  a.splits = splits;
  a.kchunk = kc;
  TN_REQUIRE((long long)(a.flat ? 1 : g.batch) * splits < 65536, "tensor-core GEMM: grid too large");
  int* err = reinterpret_cast<int*>(ctx->scratch + kScratchDoubles - 8);
  const double mnk = (double)g.M * g.N * g.K * g.batch;
  const double words = ((double)g.M * g.K + (double)g.K * g.N + (double)g.M * g.N) * g.batch;
  {
    ProfScope ps(ctx, TNFEM_PROF_CONTRACT32, 2.0 * mnk, words * sizeof(float));
    if (tn == 64) launch_tc<64>(ctx, a, alpha, A, B, beta, C, work, err, skip);
    else launch_tc<128>(ctx, a, alpha, A, B, beta, C, work, err, skip);
  }
  if (splits > 1) splitk_reduce<float>(ctx, g, alpha, beta, C, work, splits, skip);
  check_launch(ctx, "tensor-core gemm");
}

int tc_gemm_error(tnfem_ctx* ctx) {
  int h = 0;
  int* err = reinterpret_cast<int*>(ctx->scratch + kScratchDoubles - 8);
  TN_CHECK_CUDA(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  sync(ctx);
  return h;
}

}  // namespace tnfem
