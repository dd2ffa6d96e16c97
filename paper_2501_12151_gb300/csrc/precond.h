// Block-Jacobi preconditioner of the sweep's local systems (see precond.cu).
#pragma once

#include "internal.h"

namespace tnfem {

// Largest block order r0*n and largest total block storage (binary32 elements) for which the
// preconditioner is built; beyond them the local solve runs unpreconditioned.
constexpr long long kBlockJacobiMaxM = 1024;
constexpr long long kBlockJacobiMaxElems = 64ll << 20;

bool bj_fits(int r0, int n, int r1);
// Whether the sweep preconditions a local system with blocks of m = r0 n rows: always when a block
// is inverted in one CTA's shared memory (m up to ~234), and from global memory up to m = 512.
// Beyond (the 3D configuration: m = 768) the set-up cost more than the iterations it saved (2^7
// cube, rank cap 96: 15.2 s with the preconditioner, 11.9 s with plain CG, measured).
bool bj_worth_it(int r0, int n);
// Workspace (precision T elements) of bj_setup.
size_t bj_work_elems(int r0, int n, int r1, int a0, int a1);
// Build the inverses of the r1 diagonal blocks into Pinv ([r1][r0 n][r0 n] binary32).  Ap is the
// operator core with its mode indices swapped ([a0][j][i][a1]).  Returns false (preconditioner
// unusable) when a block is too large or a pivot was not positive.  Synchronises the stream.
template <typename T>
bool bj_setup(tnfem_ctx* ctx, int r0, int n, int r1, int a0, int a1, const T* PhiL, const T* Ap, const T* PhiR,
              float* Pinv, T* work, size_t work_elems, int* flag);
// z = M^{-1} r on a core [r0][n][r1] with `nblocks` CTAs (nblocks / r1 CTAs share each block b
// when nblocks >= r1, else each CTA takes blocks in turn); part[0..nblocks) receives partial
// sums of r.z; p_out (nullable) receives a copy of z.  Skipped
// when ctl[0] != 0 (ctl nullable).
template <typename T>
void bj_apply(tnfem_ctx* ctx, int r0, int n, int r1, const float* Pinv, const T* r, T* z, T* p_out, double* part,
              const int* ctl, int nblocks);

}  // namespace tnfem
