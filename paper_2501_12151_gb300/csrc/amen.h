// AMEn solve on the device (see amen.cu).
#pragma once

#include <chrono>
#include <vector>

#include "internal.h"

namespace tnfem {

// One term of the right-hand side b = sum_s coef * S: a train v (is_op == false) or the
// operator applied to a train, A v (is_op == true, same operator as the system).
struct AmenSource {
  const tnfem_tt* v = nullptr;
  bool is_op = false;
  double coef = 1.0;
};

// Default fraction of a local system's starting residual to which it is solved (see AmenParams)
constexpr double kLocalRtolDefault = 0.1;

struct AmenParams {
  double tol = 1e-10;       // stop when the largest local residual or local update is <= tol
  int rmax = 64;            // rank cap
  int kick = 4;             // enrichment rank
  int max_sweeps = 40;
  int local_maxit = 500;    // conjugate-gradient iterations per local solve
  double resid_damp = 2.0;  // local solves stop at tol / resid_damp ...
  double local_rtol = kLocalRtolDefault;  // ... or at local_rtol times their starting residual, whichever is larger
  bool precond = true;      // block-Jacobi preconditioned conjugate gradients for the local solves
  bool local_mixed = false; // binary64 sweep with binary32 local solves refined in binary64
  bool graphs = true;       // replay the conjugate-gradient chunks as CUDA graphs
  bool fused_cg = true;     // local CG as one persistent cooperative kernel where the shape fits
  double stall_dx = 4.0;    // stop when updates are within stall_dx * tol and residuals stagnate
  uint64_t seed = 0;
  bool verbose = false;
  // wall-clock limit of the solve (tnfem_solve_opts.timeout_us): checked after every core step
  bool has_deadline = false;
  std::chrono::steady_clock::time_point deadline;
};

// Phases of a core step timed when TNFEM_TRACE is set (see tnfem_solve_info.t_phase_ms).
enum {
  kPhaseRhs = 0,       // projection of the right-hand side onto the interfaces
  kPhaseResidual = 1,  // local residual before the solve
  kPhaseSolve = 2,     // local solve (preconditioner set-up, conjugate gradients, refinement)
  kPhaseSvd = 3,       // truncated SVD
  kPhaseEnrich = 4,    // residual projections, z update, QR of the enriched basis
  kPhaseEnv = 5,       // next-core update and environment contractions
  kPhaseOther = 6,     // orientation flips and bookkeeping
  kPhases = 7
};

struct AmenStats {
  int sweeps = 0;
  int max_rank = 0;
  int last_rank_trunc = 0;
  long long local_iters = 0;
  double max_res = 0, max_dx = 0;
  double flops = 0;
  bool converged = false;
  bool timed_out = false;  // the deadline passed; the iterate of the last completed core step is kept
  double phase_ms[kPhases] = {};
};

// Solve A x = b; `single` selects binary32 for the sweep (sources stay binary64).
tnfem_tt* amen_solve(tnfem_ctx* ctx, const tnfem_mpo* A, const std::vector<AmenSource>& src,
                     const AmenParams& prm, const tnfem_tt* x0, bool single, AmenStats& st);

}  // namespace tnfem
