// General quadrilateral domains in 2D (Algorithm 1, Section 5.1 / 5.2): the unit square's bilinear
// map x(xi, eta) = P0 + xi a + eta b + xi eta c onto the quadrilateral with corners P0, P0 + a,
// P0 + b, P0 + a + b + c, discretised on the tensor grid of 2^L x 2^L nodes.
//
// Every element's Jacobian J and det J are frozen at the element centre, as Algorithm 1 evaluates
// them at xi = 0 of the reference square.  At centre (xi, eta) the columns of J are a + eta c and
// b + xi c, so J and det J are affine in the element index (Section 5.1) while J^{-1} carries the
// non-separable 1 / det J; the element matrices follow from J^{-1} and |det J| as on a
// parallelogram (four derivative pairs (p, q) per block, each a product of 1D reference matrices).
//
// Tensorisation.  Where the paper forms TTs of the Jacobian entries, a TT-cross of 1 / det J and 64
// corner-pair operators, this builder works in node space: block b = (c, c') of the operator is a
// 9-point stencil, A_b = sum_o diag(coef_{b,o}) T_o with (T_o u)(i) = u(i + o), o in {-1,0,1}^2,
// whose coefficient at row node i gathers the corner pairs (alpha, beta = alpha + o) of the up to
// four elements i - alpha that hold node i:
//     coef_{b,o}(i) = p(i) p(i + o) sum_alpha K_e[b][alpha][alpha + o],   e = i - alpha,
// with the Dirichlet projector p folded in, plus s (1 - p(i)) on the diagonal blocks at o = 0.
// The coefficients are exact dense values (one pass over the elements, O(4^L)); their TT, with the
// block index first and the offset last, comes from a TT-SVD (on the device in production).  T_o
// is, per axis, the 3-state automaton of "j = i", "j = i + 1", "j = i - 1" read from the most
// significant bit; the operator train takes the axes one at a time: the coefficient train's level
// cores times the axis-1 automaton (rank 3 x the coefficient rank, the axis-0 offset left as a
// trailing index), rounded, then times the axis-0 automaton with that offset contracted at the
// last level, rounded again.  One 9-state product would carry rank 9 x the coefficient rank into a
// single rounding (~1100 at 2^10 x 2^10), whose cost grows with the cube of the rank.
#include <algorithm>
#include <cmath>
#include <thread>

#include "builder.h"
#include "internal.h"

namespace tnfem {

namespace {

struct QuadMap {
  double P0[2], a[2], b[2], c[2];
  int L = 1;
  int64_t n = 2;
  double h = 1.0;
};

QuadMap quad_map(const tnfem_grid& g) {
  QuadMap q;
  for (int x = 0; x < 2; ++x) {
    q.P0[x] = g.lo[x];
    q.a[x] = g.edges[0][x];
    q.b[x] = g.edges[1][x];
    q.c[x] = g.edges[2][x];
  }
  q.L = g.levels;
  q.n = (int64_t)1 << g.levels;
  q.h = 1.0 / (double)(q.n - 1);
  return q;
}

// J[x][d] = d x_x / d xi_d at unit-square point (xi, eta)
inline void jac(const QuadMap& q, double xi, double eta, double J[2][2]) {
  for (int x = 0; x < 2; ++x) {
    J[x][0] = q.a[x] + eta * q.c[x];
    J[x][1] = q.b[x] + xi * q.c[x];
  }
}

inline double det2(const double J[2][2]) { return J[0][0] * J[1][1] - J[0][1] * J[1][0]; }

inline void inv2(const double J[2][2], double det, double Jinv[2][2]) {
  Jinv[0][0] = J[1][1] / det;
  Jinv[0][1] = -J[0][1] / det;
  Jinv[1][0] = -J[1][0] / det;
  Jinv[1][1] = J[0][0] / det;
}

// node (i0, i1) -> QTT index: level k (most significant first) holds the bit pair (i0_k, i1_k)
inline size_t merged_index(int L, int64_t i0, int64_t i1) {
  size_t I = 0;
  for (int k = L - 1; k >= 0; --k) I = I * 4 + (size_t)((((i0 >> k) & 1) << 1) | ((i1 >> k) & 1));
  return I;
}

// 1D reference matrix on an element of length h for test corner al, trial corner be: K (both
// derivatives), G^T (test derivative), G (trial derivative) or M (none)
inline double ref1d(int d, int p, int q, int al, int be, double h) {
  if (p == d && q == d) return (al == be ? 1.0 : -1.0) / h;
  if (p == d) return al == 1 ? 0.5 : -0.5;
  if (q == d) return be == 1 ? 0.5 : -0.5;
  return h * (al == be ? 1.0 / 3.0 : 1.0 / 6.0);
}

// Element (e0, e1) with its Jacobian frozen at the centre: stiffness (mass == false) or mass
// entries K[b][alpha][beta], b = c*2 + c', alpha = alpha_0*2 + alpha_1 (corner bits per axis).
void element(const QuadMap& q, const tnfem_grid& g, const tnfem_material& mat, int64_t e0, int64_t e1,
             bool mass, double K[4][4][4]) {
  const double xi = (e0 + 0.5) * q.h, eta = (e1 + 0.5) * q.h;
  double J[2][2], Jinv[2][2];
  jac(q, xi, eta, J);
  const double det = det2(J), adet = std::fabs(det);
  for (int b = 0; b < 4; ++b)
    for (int al = 0; al < 4; ++al)
      for (int be = 0; be < 4; ++be) K[b][al][be] = 0.0;
  if (mass) {
    for (int al = 0; al < 4; ++al)
      for (int be = 0; be < 4; ++be) {
        const double v = adet * ref1d(0, -1, -1, al >> 1, be >> 1, q.h) * ref1d(1, -1, -1, al & 1, be & 1, q.h);
        K[0][al][be] = v;
        K[3][al][be] = v;
      }
    return;
  }
  inv2(J, det, Jinv);
  // material of the element: its centroid's x decides (two-material split)
  const double cx = q.P0[0] + xi * q.a[0] + eta * q.b[0] + xi * eta * q.c[0];
  double lam, mu;
  lame(cx < mat.split_x ? mat.E[0] : mat.E[1], mat.nu, 2, g.plane_stress != 0, lam, mu);
  for (int c = 0; c < 2; ++c)
    for (int c2 = 0; c2 < 2; ++c2)
      for (int p = 0; p < 2; ++p)
        for (int r = 0; r < 2; ++r) {
          // |det J| (lam d_c(test) d_c'(trial) + mu d_c'(test) d_c(trial) + mu [c = c'] grad . grad),
          // physical derivative d/dx_e = sum_p Jinv[p][e] d/dxi_p
          double k = lam * Jinv[p][c] * Jinv[r][c2] + mu * Jinv[p][c2] * Jinv[r][c];
          if (c == c2) k += mu * (Jinv[p][0] * Jinv[r][0] + Jinv[p][1] * Jinv[r][1]);
          k *= adet;
          for (int al = 0; al < 4; ++al)
            for (int be = 0; be < 4; ++be)
              K[c * 2 + c2][al][be] += k * ref1d(0, p, r, al >> 1, be >> 1, q.h) * ref1d(1, p, r, al & 1, be & 1, q.h);
        }
}

// Runs body(i0) for i0 in [0, n) on up to hardware_concurrency host threads.
template <typename F>
void parallel_rows(int64_t n, F body) {
  const int nt = (int)std::max<int64_t>(1, std::min<int64_t>({n, (int64_t)std::thread::hardware_concurrency(), 32}));
  if (nt == 1) {
    for (int64_t i = 0; i < n; ++i) body(i);
    return;
  }
  std::vector<std::thread> th;
  for (int t = 0; t < nt; ++t)
    th.emplace_back([=, &body] {
      for (int64_t i = t; i < n; i += nt) body(i);
    });
  for (auto& x : th) x.join();
}

}  // namespace

void check_quad(const tnfem_grid& g) {
  TN_REQUIRE(g.dim == 2, "a general quadrilateral grid (mapped = 2) is two-dimensional");
  TN_REQUIRE(g.levels >= 1 && g.levels <= kQuadLevelsMax, "a general quadrilateral grid takes levels in [1, 12]");
  for (int x = 0; x < 2; ++x) {
    TN_REQUIRE(std::isfinite(g.lo[x]), "quadrilateral corner is not finite");
    for (int d = 0; d < 3; ++d) TN_REQUIRE(std::isfinite(g.edges[d][x]), "quadrilateral edge is not finite");
  }
  // det J is affine on the unit square (the xi eta term cancels), so its sign at the four corners
  // decides: one strict sign means a convex, non-degenerate quadrilateral
  const QuadMap q = quad_map(g);
  double dmin = 1e300, dmax = -1e300, amax = 0;
  for (int k = 0; k < 4; ++k) {
    double J[2][2];
    jac(q, (double)(k >> 1), (double)(k & 1), J);
    const double det = det2(J);
    dmin = std::min(dmin, det);
    dmax = std::max(dmax, det);
    amax = std::max(amax, std::fabs(det));
  }
  TN_REQUIRE(amax > 0 && (dmin > 1e-12 * amax || dmax < -1e-12 * amax),
             "quadrilateral is not convex or is degenerate (det J changes sign or vanishes)");
}

void quad_element_inverse(const tnfem_grid& g, int64_t e0, int64_t e1, double Jinv[2][2]) {
  const QuadMap q = quad_map(g);
  double J[2][2];
  jac(q, (e0 + 0.5) * q.h, (e1 + 0.5) * q.h, J);
  inv2(J, det2(J), Jinv);
}

void quad_operator_coefficients(const tnfem_grid& g, const tnfem_material& mat, bool mass,
                                std::vector<double>& out, double* shift) {
  check_quad(g);
  const QuadMap q = quad_map(g);
  const int L = q.L;
  const int64_t n = q.n;
  const size_t N4 = (size_t)1 << (2 * L);
  out.assign((size_t)4 * N4 * 9, 0.0);
  auto pd = [&](int d, int64_t i) {
    if (mass) return 1.0;
    if (i == 0 && g.clamped[2 * d]) return 0.0;
    if (i == n - 1 && g.clamped[2 * d + 1]) return 0.0;
    return 1.0;
  };
  auto valid = [&](int64_t e) { return e >= 0 && e <= n - 2; };
  // s: mean over components of the unconstrained diagonal at node (1, 1)
  double s = 0.0;
  if (!mass) {
    for (int al = 0; al < 4; ++al) {
      const int64_t e0 = 1 - (al >> 1), e1 = 1 - (al & 1);
      if (!valid(e0) || !valid(e1)) continue;
      double K[4][4][4];
      element(q, g, mat, e0, e1, false, K);
      s += 0.5 * (K[0][al][al] + K[3][al][al]);
    }
  }
  if (shift) *shift = s;
  parallel_rows(n, [&](int64_t i0) {
    double K[4][4][4];
    for (int64_t i1 = 0; i1 < n; ++i1) {
      double acc[4][9] = {{0}};
      for (int al = 0; al < 4; ++al) {
        const int64_t e0 = i0 - (al >> 1), e1 = i1 - (al & 1);
        if (!valid(e0) || !valid(e1)) continue;
        element(q, g, mat, e0, e1, mass, K);
        for (int be = 0; be < 4; ++be) {
          const int o = ((be >> 1) - (al >> 1) + 1) * 3 + ((be & 1) - (al & 1) + 1);
          for (int b = 0; b < 4; ++b) acc[b][o] += K[b][al][be];
        }
      }
      if (!mass) {
        const double pi = pd(0, i0) * pd(1, i1);
        for (int o = 0; o < 9; ++o) {
          const int64_t j0 = i0 + o / 3 - 1, j1 = i1 + o % 3 - 1;
          const double pj = (j0 >= 0 && j0 < n && j1 >= 0 && j1 < n) ? pd(0, j0) * pd(1, j1) : 0.0;
          for (int b = 0; b < 4; ++b) acc[b][o] *= pi * pj;
        }
        acc[0][4] += s * (1.0 - pi);
        acc[3][4] += s * (1.0 - pi);
      }
      const size_t I = merged_index(L, i0, i1);
      for (int b = 0; b < 4; ++b)
        for (int o = 0; o < 9; ++o) out[((size_t)b * N4 + I) * 9 + o] = acc[b][o];
    }
  });
}

namespace {

// Offset automaton of one axis, most significant bit first: state 0 "j = i so far", 1 "j = i + 1"
// (i ends in 0 1..1, j in 1 0..0), 2 "j = i - 1"; step(state, i bit, j bit) is the next state or -1
// (no continuation: the pair can no longer end at that offset).
int step(int st, int bi, int bj) {
  if (st == 0) return bi == bj ? 0 : (bi == 0 ? 1 : 2);
  if (st == 1) return (bi == 1 && bj == 0) ? 1 : -1;
  return (bi == 0 && bj == 1) ? 2 : -1;
}
int offset_index(int st) { return st == 0 ? 1 : (st == 1 ? 2 : 0); }  // o + 1

}  // namespace

HTrain quad_stage_axis1(const HTrain& coef) {
  const int L = (int)coef.c.size() - 2;
  TN_REQUIRE(L >= 1 && coef.c.front().N == 4 && coef.c.back().N == 9, "quad_stage_axis1: coefficient train shape");
  HTrain out;
  out.c.push_back(coef.c[0]);  // block b = c*2 + c'
  for (int k = 1; k <= L; ++k) {
    const HCore& ck = coef.c[k];  // [rho0][row bits (i0, i1)][rho1]
    const int S0 = (k == 1) ? 1 : 3, R0 = ck.r0 * S0, R1 = ck.r1 * 3;
    HCore o{R0, 8, R1, std::vector<double>((size_t)R0 * 8 * R1, 0.0)};
    for (int a = 0; a < ck.r0; ++a)
      for (int st = 0; st < S0; ++st)
        for (int si = 0; si < 4; ++si)
          for (int bj = 0; bj < 2; ++bj) {
            const int t = step(st, si & 1, bj);
            if (t < 0) continue;
            double* dst = &o.v[((size_t)(a * S0 + st) * 8 + si * 2 + bj) * R1];
            const double* src = &ck.v[((size_t)a * 4 + si) * ck.r1];
            for (int b = 0; b < ck.r1; ++b) dst[(size_t)b * 3 + t] = src[b];
          }
    out.c.push_back(o);
  }
  // the axis-1 offset is fixed by the final state; o_0 stays as a trailing index
  const HCore& last = coef.c[L + 1];
  HCore sel{last.r0 * 3, 3, 1, std::vector<double>((size_t)last.r0 * 9, 0.0)};
  for (int b = 0; b < last.r0; ++b)
    for (int t = 0; t < 3; ++t)
      for (int x0 = 0; x0 < 3; ++x0) sel.v[(size_t)(b * 3 + t) * 3 + x0] = last.v[(size_t)b * 9 + x0 * 3 + offset_index(t)];
  out.c.push_back(sel);
  return out;
}

HTrain quad_stage_axis0(const HTrain& B) {
  const int L = (int)B.c.size() - 2;
  TN_REQUIRE(L >= 1 && B.c.front().N == 4 && B.c.back().N == 3, "quad_stage_axis0: train shape");
  HTrain out;
  out.c.push_back(B.c[0]);
  const HCore& sel = B.c[L + 1];
  for (int k = 1; k <= L; ++k) {
    const HCore& bk = B.c[k];  // [r0][(i0, i1, j1)][r1]
    const int S0 = (k == 1) ? 1 : 3;
    const bool fin = (k == L);
    const int R0 = bk.r0 * S0, R1 = fin ? 1 : bk.r1 * 3;
    HCore o{R0, 16, R1, std::vector<double>((size_t)R0 * 16 * R1, 0.0)};
    for (int a = 0; a < bk.r0; ++a)
      for (int st = 0; st < S0; ++st)
        for (int m8 = 0; m8 < 8; ++m8)
          for (int bj = 0; bj < 2; ++bj) {
            const int si = m8 >> 1, t = step(st, si >> 1, bj);
            if (t < 0) continue;
            const int mode = si * 4 + bj * 2 + (m8 & 1);  // row bits (i0, i1), column bits (j0, j1)
            double* dst = &o.v[((size_t)(a * S0 + st) * 16 + mode) * R1];
            const double* src = &bk.v[((size_t)a * 8 + m8) * bk.r1];
            if (!fin) {
              for (int b = 0; b < bk.r1; ++b) dst[(size_t)b * 3 + t] = src[b];
            } else {
              double v = 0.0;
              for (int b = 0; b < bk.r1; ++b) v += src[b] * sel.v[(size_t)b * 3 + offset_index(t)];
              dst[0] = v;
            }
          }
    out.c.push_back(o);
  }
  return out;
}

void quad_load_values(const tnfem_grid& g, const tnfem_material& mat, const tnfem_load* loads, int n_loads,
                      std::vector<double>& out) {
  (void)mat;
  check_quad(g);
  const QuadMap q = quad_map(g);
  const int L = q.L;
  const int64_t n = q.n;
  const size_t N4 = (size_t)1 << (2 * L);
  out.assign(2 * N4, 0.0);
  for (int li = 0; li < n_loads; ++li) {
    const tnfem_load& ld = loads[li];
    TN_REQUIRE(ld.kind == TNFEM_LOAD_GRAVITY || ld.kind == TNFEM_LOAD_TRACTION || ld.kind == TNFEM_LOAD_FOURIER,
               "general quadrilateral: loads must be gravity, tractions or Fourier body forces");
    if (ld.kind == TNFEM_LOAD_FOURIER)
      TN_REQUIRE(ld.n_modes >= 0 && (ld.n_modes == 0 || (ld.amp && ld.wave && ld.phase)), "fourier load arrays");
    if (ld.kind == TNFEM_LOAD_TRACTION) TN_REQUIRE(ld.face >= 0 && ld.face < 4, "traction face out of range");
  }
  auto pos = [&](int64_t i0, int64_t i1, double x[2]) {
    const double xi = i0 * q.h, eta = i1 * q.h;
    for (int d = 0; d < 2; ++d) x[d] = q.P0[d] + xi * q.a[d] + eta * q.b[d] + xi * eta * q.c[d];
  };
  // nodal body-force values f0 (Section 5.3: the Lagrange basis makes them the expansion coefficients)
  auto f0 = [&](int64_t i0, int64_t i1, double v[2]) {
    v[0] = v[1] = 0.0;
    double x[2];
    pos(i0, i1, x);
    for (int li = 0; li < n_loads; ++li) {
      const tnfem_load& ld = loads[li];
      if (ld.kind == TNFEM_LOAD_GRAVITY) {
        v[1] -= ld.rho * ld.g;
      } else if (ld.kind == TNFEM_LOAD_FOURIER) {
        for (int m = 0; m < ld.n_modes; ++m) {
          const double s = std::sin(M_PI * (ld.wave[m * 2] * x[0] + ld.wave[m * 2 + 1] * x[1]) + ld.phase[m]);
          for (int c = 0; c < 2; ++c) v[c] += ld.scale * ld.amp[c * ld.n_modes + m] * s;
        }
      }
    }
  };
  const tnfem_material any{{1.0, 1.0}, 1e300, 0.3};
  // f = M f0, element by element with the frozen |det J| (row node i gathers its elements i - alpha)
  parallel_rows(n, [&](int64_t i0) {
    double K[4][4][4];
    for (int64_t i1 = 0; i1 < n; ++i1) {
      double f[2] = {0.0, 0.0};
      for (int al = 0; al < 4; ++al) {
        const int64_t e0 = i0 - (al >> 1), e1 = i1 - (al & 1);
        if (e0 < 0 || e0 > n - 2 || e1 < 0 || e1 > n - 2) continue;
        element(q, g, any, e0, e1, true, K);
        for (int be = 0; be < 4; ++be) {
          double v[2];
          f0(e0 + (be >> 1), e1 + (be & 1), v);
          f[0] += K[0][al][be] * v[0];
          f[1] += K[3][al][be] * v[1];
        }
      }
      const size_t I = merged_index(L, i0, i1);
      out[I] = f[0];
      out[N4 + I] = f[1];
    }
  });
  // uniform tractions: the sides are straight, so each edge element on a side has length |side| h
  // and the face mass gives |side| h (1/2 at the side's ends, 1 inside) per node
  for (int li = 0; li < n_loads; ++li) {
    const tnfem_load& ld = loads[li];
    if (ld.kind != TNFEM_LOAD_TRACTION) continue;
    double side[2];
    for (int x = 0; x < 2; ++x) {
      const double sx[4] = {q.b[x], q.b[x] + q.c[x], q.a[x], q.a[x] + q.c[x]};
      side[x] = sx[ld.face];
    }
    const double len = std::sqrt(side[0] * side[0] + side[1] * side[1]);
    for (int64_t t = 0; t < n; ++t) {
      const double w = len * q.h * ((t == 0 || t == n - 1) ? 0.5 : 1.0);
      const int64_t i0 = ld.face < 2 ? (ld.face == 0 ? 0 : n - 1) : t;
      const int64_t i1 = ld.face < 2 ? t : (ld.face == 2 ? 0 : n - 1);
      const size_t I = merged_index(L, i0, i1);
      out[I] += ld.traction[0] * w;
      out[N4 + I] += ld.traction[1] * w;
    }
  }
  // f_bc = P f
  for (int64_t t = 0; t < n; ++t)
    for (int side = 0; side < 2; ++side) {
      const int64_t e = side ? n - 1 : 0;
      if (g.clamped[side]) {
        const size_t I = merged_index(L, e, t);
        out[I] = out[N4 + I] = 0.0;
      }
      if (g.clamped[2 + side]) {
        const size_t I = merged_index(L, t, e);
        out[I] = out[N4 + I] = 0.0;
      }
    }
}

}  // namespace tnfem
