/*
 * tnfem.h -- C ABI of the GB300 tensor-network FEM solver for linear elasticity.
 *
 * The library solves the Galerkin system A u = f of isotropic linear elasticity discretised
 * with Q1 (2D) / trilinear (3D) elements on a tensor grid of 2^levels nodes per axis
 * (Section 3, Eq. femsys; Section 5), with A, f and u held in the quantized tensor-train
 * (QTT) layout of Section 5.2: a component core of mode D first, then one core per level of
 * mode 2^D that carries that level's bit of every axis, most significant level first
 * (Section 4).  The solve is the AMEn sweep named in Section 5.4 / Algorithm 2.
 *
 * Conventions shared by every entry point:
 *  - Status: every call returns a tnfem_status and never aborts, exits or traps.  On failure
 *    tnfem_last_error(ctx) holds a one-line message (per context).
 *  - Ownership: handles (tnfem_ctx, tnfem_mpo, tnfem_tt) are created by the library and freed
 *    by the caller with the matching tnfem_*_destroy / tnfem_free_* call.  Host buffers passed
 *    in belong to the caller and are never retained after the call returns.  Device pointers
 *    passed to the tnfem_op_* kernel entry points belong to the caller as well.
 *  - Threading: a context is used by one host thread at a time.
 *  - Units: SI.  The grid spans the box [lo, hi]; node index (i, j[, k]) in [0, 2^levels)^D.
 *  - Precision: unless a call says otherwise, data crossing the boundary is IEEE binary64.
 *  - Core layouts (all row-major, last index fastest, no padding):
 *      vector core  [r_{k-1}][n_k][r_k]
 *      operator core [a_{k-1}][n_k (row, test)][n_k (column, trial)][a_k]
 */
#ifndef TNFEM_H
#define TNFEM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TNFEM_OK = 0,
  TNFEM_E_INVALID = 1,        /* bad argument: null pointer, size out of range, shape mismatch */
  TNFEM_E_NOMEM = 2,          /* device or host allocation failed */
  TNFEM_E_CUDA = 3,           /* a CUDA runtime call failed (message holds the CUDA error) */
  TNFEM_E_NOT_CONVERGED = 4,  /* solve stopped at max_sweeps / max_refine; result still filled */
  TNFEM_E_TIMEOUT = 5,        /* a bounded device-side wait ran out, or a solve's timeout_us passed
                                 (then the solve's result is still filled) */
  TNFEM_E_BUDGET = 6,         /* an allocation would exceed the context's device-memory budget
                                 (tnfem_set_hbm_budget); the context stays usable */
  TNFEM_E_NUMERIC = 7         /* NaN/Inf detected: every core step of the sweep checks its local
                                 right-hand side, residual and solution, so a non-finite value in
                                 the operator, the load, the start or an environment ends the solve
                                 within one sweep (no result is returned) */
} tnfem_status;

typedef struct tnfem_ctx tnfem_ctx;
typedef struct tnfem_mpo tnfem_mpo;
typedef struct tnfem_tt tnfem_tt;

/* Faces: 0 -x, 1 +x, 2 -y, 3 +y, 4 -z, 5 +z. */
typedef struct {
  int dim;             /* 2 or 3 */
  int levels;          /* L >= 1: 2^L nodes per axis, boundary nodes included (Section 5) */
  double lo[3], hi[3]; /* box corners; only the first dim entries are read */
  int clamped[6];      /* 1: homogeneous Dirichlet on all components of that face, 0: traction face */
  int plane_stress;    /* 2D only: 1 uses the modified Lame parameter lambda* = 2 lambda mu/(lambda+2 mu) */
  int mapped;          /* 0: the box [lo, hi].  1: the parallelogram / parallelepiped
                          {lo + sum_d xi_d edges[d] : xi in [0,1]^dim} (affine element maps, J
                          constant, Section 5.1; hi unused); faces are the images of the unit box's
                          faces; the material must be homogeneous (no E split inside the domain)
                          and loads are gravity and uniform tractions only.
                          2 (2D only, levels <= 12): the convex quadrilateral
                          {lo + xi edges[0] + eta edges[1] + xi eta edges[2] : (xi, eta) in [0,1]^2}
                          (corners lo, lo + edges[0], lo + edges[1], lo + edges[0] + edges[1] +
                          edges[2]), every element's Jacobian frozen at its centre as in
                          Algorithm 1; faces 0-3 are the sides xi = 0, xi = 1, eta = 0, eta = 1;
                          two materials, gravity, tractions and Fourier loads are accepted.
                          A quadrilateral whose det J changes sign or vanishes (not convex,
                          degenerate) is refused with TNFEM_E_INVALID */
  double edges[3][3];  /* mapped 1: edges[d] is the image of reference axis d (the columns of J);
                          mapped 2: the bilinear map's coefficients as above (x, y entries) */
} tnfem_grid;

typedef struct {
  double E[2];    /* Young's modulus; E[0] for elements whose centroid has x < split_x, E[1] otherwise */
  double split_x; /* set to a value beyond hi[0] (e.g. 1e300) for a homogeneous material */
  double nu;      /* Poisson's ratio, 0 <= nu < 0.5 */
} tnfem_material;

typedef enum {
  TNFEM_LOAD_GRAVITY = 0,      /* body force (0, -rho g) in 2D, (0, 0, -rho g) in 3D */
  TNFEM_LOAD_TRACTION = 1,     /* uniform traction vector on face `face` */
  TNFEM_LOAD_FOURIER = 2,      /* f_c(x) = scale * sum_m amp[c*n_modes+m] sin(pi wave_m . x + phase_m) */
  TNFEM_LOAD_MANUFACTURED = 3, /* 2D unit square: body force and free-face tractions of
                                  u* = (sin(pi x) sin(pi y), x(1-x) y(1-y)) */
  TNFEM_LOAD_NODAL_TT = 4      /* the nodal values f0 of a body force given as a train (Section 5.3:
                                  f = M f0, the Lagrange basis making nodal values the expansion
                                  coefficients); device builder only */
} tnfem_load_kind;

typedef struct {
  int kind;             /* tnfem_load_kind */
  double rho, g;        /* GRAVITY */
  int face;             /* TRACTION */
  double traction[3];   /* TRACTION */
  int n_modes;          /* FOURIER: number of modes */
  const double* amp;    /* FOURIER: [dim][n_modes] host array */
  const int* wave;      /* FOURIER: [n_modes][dim] host array of integer wave numbers */
  const double* phase;  /* FOURIER: [n_modes] host array */
  double scale;         /* FOURIER */
  const tnfem_tt* nodal; /* NODAL_TT: f0 as a train of the same context, laid out like the solution
                            (component core of mode dim, then levels cores of mode 2^dim); read
                            during the call only, not retained */
} tnfem_load;

/* FP64: every step in binary64.
 * MIXED: binary32 AMEn solves of the correction equation A e = f - A u inside an outer iterative
 *   refinement whose residual projections and u + e rounding are binary64.  The refinement
 *   contracts only while cond(A) times the binary32 unit roundoff is well below 1: it converges
 *   on small grids and stalls near 4e-4 relative energy error on 2^10 x 2^10 nodes.
 * MIXED_LOCAL: binary64 sweep (environments, projections, QR, SVD) whose local systems are solved
 *   by binary32 preconditioned CG, refined against the binary64 local residual until it meets the
 *   same tolerance as FP64.
 * MIXED_TF32: MIXED_LOCAL with the binary32 local matvecs on the tcgen05 tensor cores (TF32
 *   products in the three-term split a b = a_hi b_hi + a_hi b_lo + a_lo b_hi, FP32 accumulation);
 *   the same as MIXED_LOCAL with tensor_cores = 1. */
typedef enum { TNFEM_FP64 = 0, TNFEM_MIXED = 1, TNFEM_MIXED_LOCAL = 2, TNFEM_MIXED_TF32 = 3 } tnfem_precision;

typedef struct {
  double tol;          /* sweep stop: largest local residual or local update <= tol; truncation
                          threshold tol/sqrt(ncores) (relative Frobenius) */
  int rank_cap;        /* maximum TT rank of the solution (before enrichment) */
  int kickrank;        /* rank of the residual enrichment (AMEn), >= 0 */
  int max_sweeps;      /* per (inner) solve */
  int precision;       /* tnfem_precision */
  double refine_tol;   /* MIXED: stop refinement when ||e||_A / ||u||_A <= refine_tol */
  int max_refine;      /* MIXED: maximum outer refinement steps */
  uint64_t seed;       /* seed of the counter-based generator for the start guess / enrichment */
  int local_maxit;     /* cap on conjugate-gradient iterations per local solve */
  int no_precond;      /* 0: block-Jacobi preconditioned local solves (default); 1: plain CG */
  int tensor_cores;    /* MIXED / MIXED_LOCAL: 1 runs the binary32 contractions on the tcgen05
                          tensor cores (TF32 split products), 0 on CUDA-core FMA */
  double local_rtol;   /* each local solve stops at max(tol / 2, local_rtol * its starting relative
                          residual); 0 solves every local system to tol / 2.  Default 0.1 when the
                          field is negative */
  int cg_engine;       /* local solves: 0 one persistent cooperative kernel per solve (default),
                          1 one launch per conjugate-gradient step (graph-replayed chunks) */
  int64_t timeout_us;  /* wall-clock limit of the solve in microseconds (0: none), checked after
                          every core step; on expiry the solve returns TNFEM_E_TIMEOUT with *u and
                          *info filled from the last completed core step */
} tnfem_solve_opts;

typedef struct {
  int sweeps;          /* total sweeps over all (inner) solves */
  int refines;         /* outer refinement steps (MIXED), 0 for FP64 */
  int max_rank;        /* largest bond rank of u */
  long long local_iters; /* conjugate-gradient iterations over the whole solve */
  double max_res;      /* largest local residual of the last sweep */
  double max_dx;       /* largest relative local update of the last sweep */
  double energy_err_est; /* MIXED: last ||e||_A / ||u||_A; FP64: 0 */
  double t_solve_ms;   /* wall time of the solve (device-synchronised) */
  double flops;        /* algorithmic flops counted by the sweep's contractions */
  size_t bytes_A, bytes_f, bytes_u; /* storage of the operator, load and solution cores */
  int converged;       /* 1 when the stopping rule fired */
  double t_phase_ms[7]; /* with the environment variable TNFEM_TRACE set: wall time per phase of
                           the core steps (device-synchronised at phase boundaries): right-hand
                           side projection, local residual, local solve, truncated SVD,
                           enrichment, environment update, other; zeros otherwise */
} tnfem_solve_info;

/* ---- context ------------------------------------------------------------------------------ */

/* Create a context on CUDA device `device`.  `stream` is a cudaStream_t; all device work of this
 * context is enqueued on it.  With NULL the context creates its own blocking stream (ordered
 * with the legacy default stream in both directions, like NULL itself, but capturable into the
 * CUDA graphs the sweep replays); tnfem_set_stream(ctx, NULL) returns to that stream.  The optional
 * allocator callbacks route every device allocation of the context (e.g. into a framework's
 * caching allocator); when alloc_fn is NULL the library calls cudaMalloc/cudaFree itself. */
typedef void* (*tnfem_alloc_fn)(size_t bytes, void* user);
typedef void (*tnfem_free_fn)(void* ptr, void* user);
tnfem_status tnfem_create(int device, void* stream, tnfem_alloc_fn alloc_fn, tnfem_free_fn free_fn,
                          void* user, tnfem_ctx** out);
void tnfem_destroy(tnfem_ctx* ctx);
const char* tnfem_last_error(const tnfem_ctx* ctx);
tnfem_status tnfem_set_stream(tnfem_ctx* ctx, void* stream);
/* Number of kernels this context has launched since creation (for accounting). */
long long tnfem_kernel_launches(const tnfem_ctx* ctx);
/* Device-memory budget of the context in bytes (0: none, the default).  Every device allocation
 * of the context (its own cudaMalloc or the allocator callback) is counted; one that would take
 * the bytes held above the budget fails with TNFEM_E_BUDGET, the call that needed it returns that
 * status and frees what it had taken, and the context stays usable.  Bytes already held are not
 * affected by a lower budget.  The serving loop admits requests against this figure. */
tnfem_status tnfem_set_hbm_budget(tnfem_ctx* ctx, size_t bytes);
/* Bytes of device memory the context holds now (in_use) and its high-water mark since creation or
 * the last reset (peak); reset_peak != 0 sets the mark to the current holding.  Either output
 * pointer may be NULL. */
tnfem_status tnfem_memory_stats(tnfem_ctx* ctx, size_t* in_use, size_t* peak, int reset_peak);

/* ---- sampled kernel timing (tracing; not part of the method) ------------------------------ *
 * Kernel classes: the sweep's dense contractions (local matvec, environments, projections) in
 * binary32 and in binary64, the Krylov vector kernels, Householder QR, Jacobi SVD, the rest, and
 * the fused conjugate-gradient kernel in binary32 and in binary64 (one launch per local solve;
 * its flops are the local matvecs and preconditioner applies of the iterations it ran).  */
#define TNFEM_PROF_CONTRACT32 0
#define TNFEM_PROF_CONTRACT64 1
#define TNFEM_PROF_KRYLOV 2
#define TNFEM_PROF_QR 3
#define TNFEM_PROF_SVD 4
#define TNFEM_PROF_OTHER 5
#define TNFEM_PROF_CG32 6
#define TNFEM_PROF_CG64 7
#define TNFEM_PROF_CLASSES 8
/* Start (or restart) sampling: from now on every `every`-th launch of each class is bracketed by
 * two CUDA events on the context's stream; every <= 0 stops sampling.  Counters are reset. */
tnfem_status tnfem_profile_start(tnfem_ctx* ctx, int every);
/* Synchronise the stream and report class `cls` since tnfem_profile_start: launches seen,
 * launches sampled, summed device milliseconds of the sampled launches and their summed
 * algorithmic flops and bytes (any output pointer may be NULL). */
tnfem_status tnfem_profile_read(tnfem_ctx* ctx, int cls, long long* launches, long long* sampled,
                                double* ms, double* flops, double* bytes);
/* Measured CUDA-core FMA rate of the context's device in TFLOP/s (precision 0: binary64,
 * 1: binary32): register-resident FMA chains on 8 CTAs of 256 threads per SM, timed with events
 * after one warm-up launch.  The denominator for the ALU-bound contraction kernels. */
tnfem_status tnfem_measure_fma_peak(tnfem_ctx* ctx, int precision, double* tflops);

/* ---- assembly (Algorithm 1, Section 5.2 / 5.3) ------------------------------------------- */

/* Stiffness TT-operator with boundary conditions applied (Algorithm 1): A = P A0 P + s (I - P),
 * P the projector onto unknowns off the clamped faces, s the mean over components of A0's
 * diagonal at grid node (1,...,1).  Box and affine grids: built on the host as exact Kronecker
 * sums of 1D QTT matrices (constant Jacobian, Section 5.1), then rounded on the device to
 * relative accuracy 1e-14.  General quadrilaterals (mapped 2): the operator's 9-point stencil
 * coefficients are formed densely on the host (O(4^levels) memory, 36 doubles per node), put in
 * TT form by a TT-SVD on the device, multiplied by the per-axis offset automata and rounded on
 * the device (relative accuracy ~1e-14).  Errors: TNFEM_E_INVALID for dim not in {2,3}, levels < 1
 * or > 20 (> 12 for mapped 2), a degenerate box or quadrilateral, nu out of [0, 0.5). */
tnfem_status tnfem_build_stiffness(tnfem_ctx* ctx, const tnfem_grid* grid,
                                   const tnfem_material* mat, tnfem_mpo** out);

/* Mass TT-operator I_D (x) M_1D (x) ... (x) M_1D without boundary conditions (Section 5.3). */
tnfem_status tnfem_build_mass(tnfem_ctx* ctx, const tnfem_grid* grid, tnfem_mpo** out);

/* Load TT f = P (M f0 + sum_faces M_face t0) (Section 5.3), summed over n_loads loads and
 * rounded on the device to relative accuracy 1e-14.  A NODAL_TT load enters as P (M f0) with the
 * grid's mass operator applied to the given train on the device (each product rounded at 1e-14).
 * Errors: TNFEM_E_INVALID for a NODAL_TT load whose train is missing, belongs to another context or
 * does not match the grid. */
tnfem_status tnfem_build_load(tnfem_ctx* ctx, const tnfem_grid* grid, const tnfem_material* mat,
                              const tnfem_load* loads, int n_loads, tnfem_tt** out);

/* Host-only variants of the three builders above: they run the exact host construction
 * (Kronecker sums of 1D QTT matrices, Section 5.2 / 5.3; for general quadrilaterals a host
 * TT-SVD of the dense stencil coefficients, practical up to levels ~5) without device rounding
 * and without touching any GPU, and copy the train into caller memory.  Call with cores == NULL to get
 * ncores, ranks (ncores+1 entries, caller provides >= 64) and modes (>= 63) for sizing; then
 * again with `cores` holding sum_k ranks[k]*modes[k]*(modes[k] for operators)*ranks[k+1]
 * doubles, laid out as in tnfem_tt_export / tnfem_mpo_export.  `shift` (nullable) receives the
 * boundary-condition shift s of the stiffness operator. */
tnfem_status tnfem_host_stiffness(const tnfem_grid* grid, const tnfem_material* mat, int* ncores,
                                  int* ranks, int* modes, double* cores, double* shift);
tnfem_status tnfem_host_mass(const tnfem_grid* grid, int* ncores, int* ranks, int* modes,
                             double* cores);
tnfem_status tnfem_host_load(const tnfem_grid* grid, const tnfem_material* mat,
                             const tnfem_load* loads, int n_loads, int* ncores, int* ranks,
                             int* modes, double* cores);

/* ---- solve (Algorithm 2) ----------------------------------------------------------------- */

/* Solve A u = f by AMEn (Section 5.4).  x0 may be NULL (a seeded rank-2 start is used).
 * FP64: every contraction, local solve, QR and SVD in binary64.
 * MIXED: inner AMEn solves of the correction equation in binary32, outer iterative refinement
 * with binary64 residual projections and binary64 rounding of u + e.
 * On TNFEM_E_NOT_CONVERGED *u and *info are still filled with the last iterate. */
tnfem_status tnfem_solve(tnfem_ctx* ctx, const tnfem_mpo* A, const tnfem_tt* f,
                         const tnfem_solve_opts* opts, const tnfem_tt* x0, tnfem_tt** u,
                         tnfem_solve_info* info);

/* ---- evaluation -------------------------------------------------------------------------- */

/* Displacement at n grid nodes: nodes is a host array [n][dim] of node indices, out a host
 * array [n][dim].  Each value is the product of core slices along the train. */
tnfem_status tnfem_eval_displacement(tnfem_ctx* ctx, const tnfem_tt* u, const int64_t* nodes,
                                     int64_t n, double* out);

/* Small-strain tensor eps = sym(grad u) at the centres of n elements (element index = its
 * lowest-corner node, each index in [0, 2^levels - 1)), from the element's nodal values and the
 * Q1/trilinear shape gradients.  out: host [n][3] (xx, yy, xy) in 2D, [n][6] (xx,yy,zz,yz,xz,xy)
 * in 3D. */
tnfem_status tnfem_eval_strain(tnfem_ctx* ctx, const tnfem_tt* u, const tnfem_grid* grid,
                               const int64_t* elems, int64_t n, double* out);

/* Energy norm ||u - v||_A (v may be NULL for ||u||_A), computed on the explicitly formed and
 * orthogonalised difference so that the result does not cancel. */
tnfem_status tnfem_energy_norm(tnfem_ctx* ctx, const tnfem_mpo* A, const tnfem_tt* u,
                               const tnfem_tt* v, double* out);

/* a9's confirmation: the global relative residual ||f - A u||_2 / ||f||_2 in binary64, formed
 * explicitly so that it does not cancel.  Grids with at most 2^22 unknowns (2D up to 2^10 x 2^10,
 * 3D up to 2^6 per axis) whose dense expansion times the largest operator or train
 * rank fits 2^28 doubles: u and f are expanded to dense device vectors and A u is formed densely,
 * one operator core at a time (a batched GEMM per core; ~0.5 s at 2^10 x 2^10).  Larger grids: the
 * residual train (A u by the MPO-TT product, ranks a_k r_k, then f - A u by concatenation) is
 * orthogonalised and its norm read from the last core; its cost grows with (a r)^3 per core. */
tnfem_status tnfem_residual_norm(tnfem_ctx* ctx, const tnfem_mpo* A, const tnfem_tt* f, const tnfem_tt* u,
                                 double* out);
/* The same quantity always by the orthogonalised residual train (the route of the larger grids). */
tnfem_status tnfem_residual_norm_train(tnfem_ctx* ctx, const tnfem_mpo* A, const tnfem_tt* f, const tnfem_tt* u,
                                       double* out);

/* <x, y> and ||x|| (norm from the orthogonalised train). */
tnfem_status tnfem_tt_dot(tnfem_ctx* ctx, const tnfem_tt* x, const tnfem_tt* y, double* out);
tnfem_status tnfem_tt_norm(tnfem_ctx* ctx, const tnfem_tt* x, double* out);

/* ---- tensor-train algebra ---------------------------------------------------------------- */

/* TT rounding (a11): left-orthogonalise by Householder QR, then truncated SVDs right to left
 * with threshold eps/sqrt(ncores-1) * ||x|| per bond and rank cap rmax (Section 4, Eq. qr). */
tnfem_status tnfem_tt_round(tnfem_ctx* ctx, const tnfem_tt* x, double eps, int rmax, tnfem_tt** out);
/* z = x + beta * y (exact, ranks add). */
tnfem_status tnfem_tt_axpy(tnfem_ctx* ctx, const tnfem_tt* x, double beta, const tnfem_tt* y,
                           tnfem_tt** out);
/* y = A x exactly (ranks multiply). */
tnfem_status tnfem_mpo_apply(tnfem_ctx* ctx, const tnfem_mpo* A, const tnfem_tt* x, tnfem_tt** out);

/* Import / export of trains through host memory.  Export with cores == NULL fills ncores,
 * ranks (ncores+1 entries) and modes (ncores entries) so the caller can size `cores`;
 * ranks/modes must then hold at least 64 / 63 entries.  `cores` is the concatenation of the
 * cores in order, each in the layout given at the top of this file. */
tnfem_status tnfem_tt_export(tnfem_ctx* ctx, const tnfem_tt* x, int* ncores, int* ranks,
                             int* modes, double* cores);
tnfem_status tnfem_tt_import(tnfem_ctx* ctx, int ncores, const int* ranks, const int* modes,
                             const double* cores, tnfem_tt** out);
tnfem_status tnfem_mpo_export(tnfem_ctx* ctx, const tnfem_mpo* A, int* ncores, int* ranks,
                              int* modes, double* cores);
tnfem_status tnfem_mpo_import(tnfem_ctx* ctx, int ncores, const int* ranks, const int* modes,
                              const double* cores, tnfem_mpo** out);
void tnfem_free_tt(tnfem_tt* x);
void tnfem_free_mpo(tnfem_mpo* A);

/* ---- kernel-level entry points (device pointers, for parity tests of single sweep steps) ---- *
 * All pointers are device pointers to binary64 arrays in the layouts stated; the work is
 * enqueued on the context's stream and the call synchronises before returning.              */

/* a4: local matvec y[a',i,b'] = sum PhiL[a',beta,a] A[beta,i,j,g] PhiR[b',g,b] x[a,j,b].
 * PhiL [r0][a0][r0], A [a0][n][n][a1], PhiR [r1][a1][r1], x and y [r0][n][r1]. */
tnfem_status tnfem_op_local_matvec(tnfem_ctx* ctx, int r0, int n, int r1, int a0, int a1,
                                   const double* PhiL, const double* A, const double* PhiR,
                                   const double* x, double* y);
/* a2/a8: left environment Phi'[b',g,b] = sum y[a',i,b'] Phi[a',beta,a] A[beta,i,j,g] x[a,j,b].
 * Phi [ry0][a0][rx0], y [ry0][n][ry1], A [a0][n][n][a1], x [rx0][n][rx1], out [ry1][a1][rx1]. */
tnfem_status tnfem_op_env_left(tnfem_ctx* ctx, int ry0, int ry1, int rx0, int rx1, int n, int a0,
                               int a1, const double* Phi, const double* y, const double* A,
                               const double* x, double* out);
/* Local matvec of tnfem_op_local_matvec for callers that cannot allocate device memory (a
 * function running inside a CUDA stream capture that must not grow the memory pool, a host
 * framework that owns the device allocator, a real-time loop that must not block on cudaMalloc).
 * This entry point has no counterpart in the paper; it is the same contraction with its
 * intermediates taken from a static device array of TNFEM_NOALLOC_SCRATCH_DOUBLES binary64
 * elements (32 MiB), which every GPU that loads the library holds until the process exits.
 *  - stream: cudaStream_t (NULL: legacy default stream); the work is enqueued on it and the call
 *    returns without synchronising.  Device pointers and layouts as for tnfem_op_local_matvec; no
 *    context is needed, the current device is used.
 *  - Limit: a0*n*n*a1 + r0*a0*n*r1 + r0*n*a1*r1 + 1024 <= TNFEM_NOALLOC_SCRATCH_DOUBLES, else
 *    TNFEM_E_INVALID (as for null pointers or sizes < 1); TNFEM_E_CUDA if the device or the
 *    array's address cannot be obtained.
 *  - No cudaMalloc / cudaFree or other allocating routine is called.  The first call on each
 *    device looks up the array's device address (cudaGetSymbolAddress) with that device current;
 *    make that first call before any stream capture.  The address is kept for the life of the
 *    process: do not reset the device (cudaDeviceReset) between calls.
 *  - All calls share the array: calls that overlap on the GPU race and must be serialised by the
 *    caller.  The array keeps the last call's contents; nothing in it needs to start at zero. */
#define TNFEM_NOALLOC_SCRATCH_DOUBLES (1ll << 22)
tnfem_status tnfem_op_local_matvec_noalloc(void* stream, int r0, int n, int r1, int a0, int a1,
                                           const double* PhiL, const double* A, const double* PhiR,
                                           const double* x, double* y);
/* a5: preconditioned conjugate gradients on one local system B x = g, B the local matrix of
 * tnfem_op_local_matvec (symmetric positive definite for the sweep's systems), run as the solver
 * runs it: one persistent cooperative kernel for the whole iteration (three grid barriers per
 * step; the block-Jacobi preconditioner of precond.cu when precond = 1, plain CG when 0).
 *  - precision: TNFEM_FP64 for binary64 operands and vectors, any other value for binary32 (the
 *    local solves of MIXED / MIXED_LOCAL); every pointer is a device pointer to that type.
 *  - PhiL [r0][a0][r0], A [a0][n][n][a1], PhiR [r1][a1][r1], g and x [r0][n][r1]; x holds the
 *    start guess on entry and the last iterate on return.  Mode size n <= 8.
 *  - Stops when the recursively updated residual meets ||r|| <= rtol ||g|| or after maxit >= 0
 *    steps.  *iters: steps done; *state: 1 converged, 0 step limit, 2 loss of positive curvature
 *    (x holds the last completed iterate).
 *  - TNFEM_E_INVALID: null pointer, size < 1, n > 8, a shape whose CTAs cannot all be resident, or
 *    (precond = 1) a block of the preconditioner that is not positive definite; TNFEM_E_TIMEOUT:
 *    a grid barrier wait expired (2 s). */
tnfem_status tnfem_op_local_cg(tnfem_ctx* ctx, int precision, int precond, int r0, int n, int r1, int a0,
                               int a1, const void* PhiL, const void* A, const void* PhiR, const void* g,
                               void* x, double rtol, int maxit, int* iters, int* state);
/* Failure detection of the bounded device waits (no counterpart in the paper: the timeout path
 * of the grid barriers that the solver's cooperative kernels use, made to run out on purpose).
 * Launches `ctas` CTAs (1 <= ctas <= number of SMs) that pass three grid barriers whose waits are
 * bounded by limit_ms (0.01 .. 2000); CTA `late_cta` (-1: none) first sleeps late_ms (0 .. 1000,
 * bounded by the global timer) before its first arrival.  With late_ms beyond limit_ms the other
 * CTAs give up, flag the error and leave, the late CTA leaves on arrival, and the call returns
 * TNFEM_E_TIMEOUT; otherwise TNFEM_OK.  No wait is unbounded, and the context stays usable. */
tnfem_status tnfem_op_barrier_probe(tnfem_ctx* ctx, int ctas, int late_cta, double late_ms, double limit_ms);
/* Binary32 building blocks of the mixed-precision local solves (parity tests of both engines).
 * engine 0: CUDA-core FMA; engine 1: tcgen05 tensor cores, kind::tf32 with the three-term split
 * a b = a_hi b_hi + a_hi b_lo + a_lo b_hi (binary32-level accuracy from TF32 products), operands
 * staged by ordinary loads; engine 2 (local matvec only): the same arithmetic on operands packed
 * once into the tensor cores' tile layout and fed by bulk TMA copies, as the solver runs it.
 * tnfem_op_gemm_f32: C(b,m,n) = alpha sum_k A(b,m,k) B(b,k,n) + beta C(b,m,n) with element
 * (b,m,k) of A at A[b*sAb + m*sAm + k*sAk] (likewise B and C); every pointer is a device pointer to
 * binary32.  tnfem_op_local_matvec_f32: the contraction of tnfem_op_local_matvec in binary32. */
/* Binary64 GEMM of tnfem_op_gemm_f32's layout (every pointer a device pointer to binary64).
 * engine 0: binary64 FMA.  engine 1: double-binary32 arithmetic, the mixed-precision sweep's route
 * for large contractions on this part (binary64 issues at 1/64 of the binary32 rate): operands
 * split into (hi, lo) binary32 pairs, products carried with their exact rounding errors, sums as
 * binary32 pairs with two-sum error recovery; relative error about K * 2^-47 of the sum of |terms|
 * (binary64: K * 2^-53).  Engine 1 applies only to products of at least 2^20 multiply-adds
 * (smaller ones run in binary64) and returns TNFEM_E_INVALID if a value leaves the binary32 range.
 * The solve does not use engine 1: in the sweep its noise, amplified by the local systems'
 * conditioning, kept the relative core updates from falling below a 1e-9 tolerance. */
tnfem_status tnfem_op_gemm_f64(tnfem_ctx* ctx, int engine, int M, int N, int K, int batch, long long sAm,
                               long long sAk, long long sAb, long long sBk, long long sBn, long long sBb,
                               long long sCm, long long sCn, long long sCb, double alpha, const double* A,
                               const double* B, double beta, double* C);
tnfem_status tnfem_op_gemm_f32(tnfem_ctx* ctx, int engine, int M, int N, int K, int batch, long long sAm,
                               long long sAk, long long sAb, long long sBk, long long sBn, long long sBb,
                               long long sCm, long long sCn, long long sCb, float alpha, const float* A,
                               const float* B, float beta, float* C);
tnfem_status tnfem_op_local_matvec_f32(tnfem_ctx* ctx, int engine, int r0, int n, int r1, int a0, int a1,
                                       const float* PhiL, const float* A, const float* PhiR, const float* x,
                                       float* y);
/* Reduced Householder QR of an m x n row-major matrix: Q [m][k], R [k][n], k = min(m, n),
 * diag(R) >= 0 is not enforced (Householder signs). */
tnfem_status tnfem_op_qr(tnfem_ctx* ctx, int m, int n, const double* Ain, double* Q, double* R);
/* a7 (enrichment): Q, R of the m x (rk + w) row-major A = [U | W] whose first rk columns are
 * orthonormal (the left singular vectors of the truncation).  W is orthogonalised against U by
 * block Gram-Schmidt (twice) and its remainder by Householder QR, so A = [U | Q_w] [[I, C], [0,
 * R_w]]: Q [m][rk + w] has orthonormal columns, R [rk + w][rk + w] is upper triangular with
 * R[:, :rk] = [I; 0].  When W lies numerically inside span(U) the Householder QR of the whole
 * (projected) A is taken instead (Q R = A still holds; R[:, :rk] = Q^T U).  Requires m >= rk + w; A is
 * overwritten; binary64 device pointers.  Not a separate step of the paper: the same QR as
 * tnfem_op_qr of the enriched basis, exploiting U's orthonormality. */
tnfem_status tnfem_op_qr_ext(tnfem_ctx* ctx, int m, int rk, int w, double* A, double* Q, double* R);
/* Thin SVD by one-sided Jacobi of an m x n row-major matrix (m >= n): U [m][n] with unit
 * columns, S [n] descending, Vt [n][n].  Each column pair of U is signed so that its entry of
 * largest magnitude is positive. */
tnfem_status tnfem_op_svd(tnfem_ctx* ctx, int m, int n, const double* Ain, double* U, double* S,
                          double* Vt);

/* ---- serving (continuous batching of solve requests on one GPU) ------------------------- *
 * Not a step of the paper's method: a persistent request loop around tnfem_solve.  Requests of
 * different dimension, levels, material, load and rank cap are queued as they arrive and admitted,
 * in arrival order, when one of `workers` worker threads is idle and the sum of the memory
 * estimates (tnfem_serve_estimate) of the admitted requests stays within `hbm_budget` (0: 80% of
 * the device memory free at start); a request is always admitted when nothing else runs.  Each
 * worker owns a context on its own non-blocking stream and allocates stream-ordered from the
 * device's memory pool, so the admitted requests' kernels overlap on the device; each worker's
 * cooperative kernels take 1/workers of the SMs.  A worker builds the request's operator and load
 * (tnfem_build_stiffness / tnfem_build_load), solves (tnfem_solve) and copies the solution cores
 * to host memory.  A request's result does not depend on what else runs: the same request solved
 * alone or in the mix gives the same train up to rounding.
 * Threading: submit, wait and result_take may be called from any host threads. */
typedef struct tnfem_server tnfem_server;
typedef struct {
  tnfem_status status;        /* the request's own status (as tnfem_solve / the builders return) */
  char message[256];          /* its error message when status != TNFEM_OK */
  tnfem_solve_info info;
  double queued_us, run_us, latency_us;  /* submit -> start, start -> end, submit -> end */
  double start_us, end_us;    /* start and end relative to tnfem_server_start */
  int worker;                 /* worker that ran it */
  size_t est_bytes;           /* admission estimate */
  size_t peak_bytes;          /* device memory the worker's context held at the request's peak */
  int ncores;                 /* solution train: cores, ranks (ncores + 1), modes */
  int ranks[64];
  int modes[63];
  size_t result_doubles;      /* doubles that tnfem_result_take copies out */
} tnfem_request_info;
/* Start `workers` (1..64) worker threads on `device`. */
tnfem_status tnfem_server_start(int device, int workers, size_t hbm_budget, tnfem_server** out);
/* The budget in force (hbm_budget, or the default chosen at start). */
tnfem_status tnfem_server_budget(const tnfem_server* s, size_t* bytes);
/* Upper estimate of the device memory one request holds at its peak (operator with its derived
 * copies, environments, cores and local-solve workspace at the rank cap). */
tnfem_status tnfem_serve_estimate(const tnfem_grid* grid, const tnfem_solve_opts* opts, size_t* bytes);
/* Queue one request (arguments as for the builders and tnfem_solve; all host memory is copied,
 * Fourier arrays included).  *id identifies it.  TNFEM_E_INVALID after tnfem_server_stop began and
 * for a NODAL_TT load (its train lives in the caller's context, beyond the request's lifetime). */
tnfem_status tnfem_submit(tnfem_server* s, const tnfem_grid* grid, const tnfem_material* mat,
                          const tnfem_load* loads, int n_loads, const tnfem_solve_opts* opts, uint64_t* id);
/* Wait until request `id` is done (timeout_us < 0: no limit; TNFEM_E_TIMEOUT when it ran out) and
 * fill *out (nullable).  The request's own outcome is out->status. */
tnfem_status tnfem_wait(tnfem_server* s, uint64_t id, int64_t timeout_us, tnfem_request_info* out);
/* Copy a finished request's solution cores (out->result_doubles doubles, cores in train order,
 * layout of tnfem_tt_export; cores may be NULL to discard) and forget the request. */
tnfem_status tnfem_result_take(tnfem_server* s, uint64_t id, double* cores);
/* Cancel a request that is still queued: it ends at once with status TNFEM_E_INVALID ("cancelled
 * before admission"); TNFEM_E_INVALID when it is unknown, already running or done. */
tnfem_status tnfem_cancel(tnfem_server* s, uint64_t id);
/* Requests waiting for admission, requests running, and the sum of the running requests' memory
 * estimates (any output pointer may be NULL). */
tnfem_status tnfem_server_stats(tnfem_server* s, int* queued, int* running, size_t* admitted_bytes);
/* Stop: requests already admitted finish, queued ones end with TNFEM_E_INVALID; joins the workers
 * and frees the server. */
tnfem_status tnfem_server_stop(tnfem_server* s);

#ifdef __cplusplus
}
#endif
#endif /* TNFEM_H */
