// Local matvec of the binary32 local solves on the tcgen05 tensor cores with TMA-fed packed
// operands (see tc_matvec.cu).
#pragma once

#include <cstdint>

#include "internal.h"

namespace tnfem {

// A matrix of `rows` x `K` packed into tiles of `rb` rows x 32 K (TF32 hi, mid and lo planes).
struct PackDims {
  int rows = 0, K = 0, rb = 0, nrb = 0, nkc = 0;
};

struct TcMatvec {
  int r0 = 0, n = 0, r1 = 0, a0 = 0, a1 = 0;
  PackDims pl, xp, t1, ap, t2, pr;
  DArr<uint32_t> PL, XP, T1, AP, T2, PR;  // packed operands and intermediates
  DArr<float> work;                       // split-K partial products of stage 3 [split][m][n]
  int splits3 = 1, kc3 = 1;
  // size the buffers for one local system (zeroes the padding of the intermediates)
  void plan(tnfem_ctx* ctx, int r0, int n, int r1, int a0, int a1);
  // pack the constant operands: PhiL [r0][a0][r0], the operator core with swapped mode indices
  // Ap [a0][j][i][a1], PhiR [r1][a1][r1] (binary32)
  void prepare(tnfem_ctx* ctx, const float* PhiL, const float* Ap, const float* PhiR);
  // y = B x for x, y [r0][n][r1]; launches are skipped while *skip != 0 (skip nullable)
  void apply(tnfem_ctx* ctx, const float* x, float* y, const int* skip);

 private:
  void pack(tnfem_ctx* ctx, uint32_t* dst, const PackDims& d, const float* src, long long sr, long long sk);
};

}  // namespace tnfem
