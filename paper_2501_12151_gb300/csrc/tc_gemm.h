// Binary32 GEMM on the tcgen05 tensor cores with a three-term TF32 split (see tc_gemm.cu).
#pragma once

#include "internal.h"

namespace tnfem {

bool tc_gemm_supported(const GemmDesc& g);
// C = alpha A B + beta C on the tensor cores; `work` (nullable) allows split-K partials of
// splits*batch*M*N elements; launches are skipped when *skip != 0.
void tc_gemm(tnfem_ctx* ctx, const GemmDesc& g, float alpha, const float* A, const float* B, float beta, float* C,
             float* work, size_t work_elems, const int* skip);
// Device error flag of the tensor-core kernels (1: a bounded wait ran out); synchronises.
int tc_gemm_error(tnfem_ctx* ctx);

}  // namespace tnfem
