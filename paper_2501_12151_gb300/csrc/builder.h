// Host-side exact construction of the stiffness TT-operator and load TT (see builder.cu).
#pragma once

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
HTrain stack_trains(const std::vector<HTrain>& xs);
AxisOps axis_operators(int L, double lo, double hi, const std::vector<double>& w, bool clamp_lo,
                       bool clamp_hi, bool with_bc);
HTrain combine_axes(const std::vector<HTrain>& axes, const std::vector<SepTerm>& terms, int ncomp,
                    bool op);
std::vector<SepTerm> stiffness_terms(int D, double lam, double mu);
HTrain stiffness_train(const tnfem_grid& g, const tnfem_material& mat, double* shift_out);
HTrain mass_train(const tnfem_grid& g);
// J^{-1} (row p, column e: d xi_p / d x_e) and det J of a mapped grid (grid.mapped != 0)
void grid_affine_inverse(const tnfem_grid& g, double Jinv[3][3], double* det);
HTrain load_train(const tnfem_grid& g, const tnfem_material& mat, const tnfem_load* loads,
                  int n_loads);

}  // namespace tnfem
