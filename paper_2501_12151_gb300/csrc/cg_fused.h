// Preconditioned conjugate gradients on one local system of the sweep as a single persistent
// cooperative kernel (see cg_fused.cu).
#pragma once

#include "internal.h"

namespace tnfem {

// Decomposition of one pass of the fused loop over the CTAs of a cooperative launch.
struct FcgPlan {
  bool ok = false;
  int ncta = 0;          // CTAs of the launch (all co-resident)
  size_t smem = 0;       // dynamic shared memory per CTA (bytes)
  int tr1 = 0, tc1 = 0;  // phase 1: output tile rows (a', beta) / columns (j, b)
  int n1 = 0;            // phase 1 tiles
  int S = 0, gw = 0;     // phase 2: slices of the right operator rank g, slice width
  int n2 = 0;            // phase 2 items (a', slice)
  int split = 0;         // phase 3: row slices per preconditioner block
  int n3 = 0;            // phase 3 items (b, row slice)
  size_t ws_bytes = 0;   // device workspace: repacked operators and the iteration's vectors
};

class FusedCg {
 public:
  FusedCg() = default;
  FusedCg(const FusedCg&) = delete;
  FusedCg& operator=(const FusedCg&) = delete;
  ~FusedCg();
  // Decomposition for the local system r0 x n x r1 with operator ranks a0, a1 in precision U
  // (float or double); plan.ok is false when the shape is outside the kernel's limits (mode size
  // above 8) or the CTAs cannot all be resident, and the caller keeps its launch-per-step loop.
  template <typename U>
  FcgPlan plan(tnfem_ctx* ctx, int r0, int n, int r1, int a0, int a1, bool pre);
  // Preconditioned CG on B x = g from the given x until r.r <= stop2 or maxit iterations.
  // PL [r0][a0][r0], Ap [a0][n][n][a1] (the operator core with its mode indices swapped),
  // PR [r1][a1][r1]; Pinv [r1][r0 n][r0 n] block inverses (nullptr: no preconditioner); g and x
  // [r0][n][r1].  The operators are repacked into a workspace the object owns (grown on demand).
  // Returns the iterations done; *state: 0 iteration limit, 1 converged, 2 loss of positive
  // curvature (x holds the last completed iterate).  Throws TNFEM_E_TIMEOUT when a grid
  // barrier wait expired.  Synchronises the stream.
  template <typename U>
  int run(tnfem_ctx* ctx, const FcgPlan& pl, int r0, int n, int r1, int a0, int a1, const U* PL, const U* Ap,
          const U* PR, const float* Pinv, const U* g, U* x, double stop2, int maxit, int* state);

 private:
  void ensure(tnfem_ctx* ctx, size_t parts, size_t ws_bytes);
  void* ws_ = nullptr;       // repacked operators and vectors
  size_t ws_bytes_ = 0;
  double* parts_ = nullptr;  // partial sums
  size_t parts_n_ = 0;
  int* ctl_ = nullptr;       // [0] state [1] iterations [4..7] grid barrier
  int* host_ = nullptr;      // pinned copy of ctl
  tnfem_ctx* ctx_ = nullptr;
  // TNFEM_FCG_PROF set: SM cycles per phase of every launch, summed and reported at destruction
  bool prof_on_ = false;
  unsigned long long* tprof_ = nullptr;
  double prof_cycles_[7] = {};
  double prof_passes_ = 0.0;
};

}  // namespace tnfem
