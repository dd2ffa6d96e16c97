// Host-side exact construction of the stiffness TT-operator and load TT (see builder.cu).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "tnfem.h"

namespace tnfem {

// Host core [r0][N][r1] with a flattened mode N (N = n*n for operator cores).
struct HCore {
  int r0 = 1, N = 1, r1 = 1;
  std::vector<double> v;
};

struct HTrain {
  std::vector<HCore> c;
  // left-orthogonalise by Householder QR, then truncated SVDs right to left with threshold
  // eps / sqrt(d-1) * ||x|| per bond and rank cap rmax
  void round(double eps, int rmax);
};

// One separable term coef * E_{c c'} (x) op_0 (x) ... (x) op_{D-1} (vectors use c only).
struct SepTerm {
  int c = 0, c2 = 0;
  double coef = 1.0;
  std::vector<int> ops;
};

struct AxisOps {
  std::vector<std::string> names;
  std::vector<double> diag1;
  HTrain joint;  // modes [T, 4, 4, ...]: the stacked 1D operators of one axis
};

HTrain htt_from_vector(const std::vector<double>& v, int L);
// TT-SVD of a dense row-major array with the given modes (first mode slowest), relative accuracy eps
HTrain htt_svd(const std::vector<double>& v, const std::vector<int>& modes, double eps);
HTrain stack_trains(const std::vector<HTrain>& xs);
AxisOps axis_operators(int L, double lo, double hi, const std::vector<double>& w, bool clamp_lo,
                       bool clamp_hi, bool with_bc);
HTrain combine_axes(const std::vector<HTrain>& axes, const std::vector<SepTerm>& terms, int ncomp,
                    bool op);
// Lame parameters (Section 2); 2D plane stress takes the modified lambda* = 2 lambda mu / (lambda + 2 mu)
void lame(double E, double nu, int dim, bool plane_stress, double& lam, double& mu);
std::vector<SepTerm> stiffness_terms(int D, double lam, double mu);
HTrain stiffness_train(const tnfem_grid& g, const tnfem_material& mat, double* shift_out);
HTrain mass_train(const tnfem_grid& g);
// the Dirichlet projector P (diagonal: 0 on the clamped faces' unknowns, 1 elsewhere) as an operator train
HTrain projector_train(const tnfem_grid& g);
// J^{-1} (row p, column e: d xi_p / d x_e) and det J of a mapped grid (grid.mapped != 0)
void grid_affine_inverse(const tnfem_grid& g, double Jinv[3][3], double* det);
HTrain load_train(const tnfem_grid& g, const tnfem_material& mat, const tnfem_load* loads,
                  int n_loads);

// ---- general quadrilaterals (grid.mapped == 2, 2D; quad.cu) ---------------------------------
// x(xi, eta) = lo + xi edges[0] + eta edges[1] + xi eta edges[2] on the unit square; every element's
// Jacobian is frozen at its centre (Algorithm 1).

// Grid checks: dim 2, levels <= kQuadLevelsMax, det J of one sign on the closed unit square.
constexpr int kQuadLevelsMax = 12;
void check_quad(const tnfem_grid& g);
// Inverse of the frozen Jacobian of element (e0, e1): Jinv[p][e] = d xi_p / d x_e
void quad_element_inverse(const tnfem_grid& g, int64_t e0, int64_t e1, double Jinv[2][2]);
// Node-space stencil coefficients of the stiffness (mass == false: boundary conditions applied,
// `shift` receives s) or mass operator (mass == true, no boundary conditions): the dense array
// c[b][I][o], b = c*2 + c' the block, I the node's QTT (merged-bit) index, o = (o_0+1)*3 + (o_1+1)
// the column offset, so that block b's entry (i, i + o) is c[b][I(i)][o]; modes {4, 4^L.., 9}.
void quad_operator_coefficients(const tnfem_grid& g, const tnfem_material& mat, bool mass,
                                std::vector<double>& out, double* shift);
// The operator train from the coefficient train (modes {4, 4, ..., 4, 9}) in two stages.  Stage 1:
// per level the coefficient core (row bits i0, i1) times the axis-1 offset automaton, giving level
// modes (i0, i1, j1) = 8 and a trailing core over the axis-0 offset (mode 3).  Stage 2 (after a
// rounding): times the axis-0 automaton, level modes (i0 i1, j0 j1) = 16, the trailing offset
// contracted at the last level: the component core and L level cores of the operator.
HTrain quad_stage_axis1(const HTrain& coef);
HTrain quad_stage_axis0(const HTrain& B);
// Load values f[c][I] = P (M f0 + face tractions) on the quadrilateral, modes {2, 4^L..}.
void quad_load_values(const tnfem_grid& g, const tnfem_material& mat, const tnfem_load* loads,
                      int n_loads, std::vector<double>& out);

}  // namespace tnfem
