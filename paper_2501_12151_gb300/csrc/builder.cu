// Assembly of the stiffness TT-operator and the load TT (Algorithm 1, Section 5.2 / 5.3) on the
// host, followed by rounding on the device.
//
// On an axis-aligned box the Jacobian of every element map is the same constant diagonal matrix
// (Section 5.1: J and det J are exact rank-1 tensors; no TT-cross is needed), and the Galerkin
// form separates axis by axis.  Each block A_{c c'} (test component c, trial component c') is a
// short sum of Kronecker products of 1D matrices per axis,
//     K = int phi_i' phi_j',  M = int phi_i phi_j,  G = int phi_i phi_j',  G^T,
// which is the tensorised form of the per-corner element terms of Algorithm 1.  Every 1D
// matrix is tridiagonal, X = diag(m) + diag(s) J + J^T diag(t) with J the unit superdiagonal,
// whose QTT cores are written down exactly (J has rank 2; the diagonals come from TT-SVDs of
// their coefficient vectors).  The 1D matrices of one axis are stacked into one train with a
// leading operator index and rounded on the host; the D-dimensional operator is then the
// component core, a first level core that contracts the block coefficients with the operator
// indices, and Kronecker products of the axis cores on the remaining levels (merged mode
// s = sum_d b_d 2^(D-1-d), x bit first).  The exact train is uploaded and rounded on the device.
//
// Dirichlet faces: A_bc = P A P + s (I - P), P = I_c (x) P_0 (x) ... (x) P_{D-1}; P_d zeroes the
// clamped end nodes of axis d, which only edits the diagonals of the 1D matrices.  Loads:
// f = P (M f0 + face tractions), every term separable.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <future>

#include "builder.h"
#include "internal.h"

namespace tnfem {

// ---- host linear algebra (small, exact sizes) ----------------------------------------------

namespace {

// Householder QR of row-major m x n: Q (m x k), R (k x n), k = min(m, n)
void hqr(int m, int n, const std::vector<double>& A, std::vector<double>& Q, std::vector<double>& R) {
  const int k = std::min(m, n);
  std::vector<double> W(A);
  std::vector<double> tau(k, 0.0);
  for (int j = 0; j < k; ++j) {
    double tail = 0;
    for (int i = j + 1; i < m; ++i) tail += W[(size_t)i * n + j] * W[(size_t)i * n + j];
    double alpha = W[(size_t)j * n + j];
    if (tail == 0.0) { tau[j] = 0.0; continue; }
    double nx = std::sqrt(alpha * alpha + tail);
    double beta = alpha >= 0 ? -nx : nx;
    tau[j] = (beta - alpha) / beta;
    double v0 = alpha - beta;
    for (int i = j + 1; i < m; ++i) W[(size_t)i * n + j] /= v0;
    W[(size_t)j * n + j] = beta;
    for (int c = j + 1; c < n; ++c) {
      double w = W[(size_t)j * n + c];
      for (int i = j + 1; i < m; ++i) w += W[(size_t)i * n + j] * W[(size_t)i * n + c];
      w *= tau[j];
      W[(size_t)j * n + c] -= w;
      for (int i = j + 1; i < m; ++i) W[(size_t)i * n + c] -= w * W[(size_t)i * n + j];
    }
  }
  R.assign((size_t)k * n, 0.0);
  for (int i = 0; i < k; ++i)
    for (int c = i; c < n; ++c) R[(size_t)i * n + c] = W[(size_t)i * n + c];
  Q.assign((size_t)m * k, 0.0);
  for (int i = 0; i < k; ++i) Q[(size_t)i * k + i] = 1.0;
  for (int j = k - 1; j >= 0; --j) {
    if (tau[j] == 0.0) continue;
    for (int c = j; c < k; ++c) {
      double w = Q[(size_t)j * k + c];
      for (int i = j + 1; i < m; ++i) w += W[(size_t)i * n + j] * Q[(size_t)i * k + c];
      w *= tau[j];
      Q[(size_t)j * k + c] -= w;
      for (int i = j + 1; i < m; ++i) Q[(size_t)i * k + c] -= w * W[(size_t)i * n + j];
    }
  }
}

// One-sided Jacobi SVD of row-major m x n (m >= n): U (m x n), S (n, descending), Vt (n x n)
void hsvd(int m, int n, const std::vector<double>& A, std::vector<double>& U, std::vector<double>& S,
          std::vector<double>& Vt) {
  std::vector<double> G((size_t)m * n), V((size_t)n * n, 0.0);
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < n; ++j) G[(size_t)j * m + i] = A[(size_t)i * n + j];
  for (int j = 0; j < n; ++j) V[(size_t)j * n + j] = 1.0;
  for (int sweep = 0; sweep < 60; ++sweep) {
    int rot = 0;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        double* gp = &G[(size_t)p * m];
        double* gq = &G[(size_t)q * m];
        double a = 0, b = 0, c = 0;
        for (int i = 0; i < m; ++i) { a += gp[i] * gp[i]; b += gq[i] * gq[i]; c += gp[i] * gq[i]; }
        if (c == 0.0 || a == 0.0 || b == 0.0 || std::fabs(c) <= 4e-16 * std::sqrt(a * b)) continue;
        double zeta = (b - a) / (2 * c);
        double t = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1 + zeta * zeta));
        double cs = 1 / std::sqrt(1 + t * t), sn = cs * t;
        for (int i = 0; i < m; ++i) { double x = gp[i], y = gq[i]; gp[i] = cs * x - sn * y; gq[i] = sn * x + cs * y; }
        double* vp = &V[(size_t)p * n];
        double* vq = &V[(size_t)q * n];
        for (int i = 0; i < n; ++i) { double x = vp[i], y = vq[i]; vp[i] = cs * x - sn * y; vq[i] = sn * x + cs * y; }
        ++rot;
      }
    if (!rot) break;
  }
  std::vector<double> sig(n);
  for (int j = 0; j < n; ++j) {
    double s = 0;
    for (int i = 0; i < m; ++i) s += G[(size_t)j * m + i] * G[(size_t)j * m + i];
    sig[j] = std::sqrt(s);
  }
  std::vector<int> ord(n);
  for (int j = 0; j < n; ++j) ord[j] = j;
  std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return sig[a] > sig[b]; });
  U.assign((size_t)m * n, 0.0);
  S.assign(n, 0.0);
  Vt.assign((size_t)n * n, 0.0);
  for (int pos = 0; pos < n; ++pos) {
    int j = ord[pos];
    S[pos] = sig[j];
    double inv = sig[j] > 0 ? 1.0 / sig[j] : 0.0;
    for (int i = 0; i < m; ++i) U[(size_t)i * n + pos] = G[(size_t)j * m + i] * inv;
    for (int i = 0; i < n; ++i) Vt[(size_t)pos * n + i] = V[(size_t)j * n + i];
  }
}

std::vector<double> htranspose(int m, int n, const std::vector<double>& A) {
  std::vector<double> B((size_t)m * n);
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < n; ++j) B[(size_t)j * m + i] = A[(size_t)i * n + j];
  return B;
}

// C (m x n) = A (m x k) B (k x n)
std::vector<double> hmm(int m, int k, int n, const double* A, const double* B) {
  std::vector<double> C((size_t)m * n, 0.0);
  for (int i = 0; i < m; ++i)
    for (int p = 0; p < k; ++p) {
      double a = A[(size_t)i * k + p];
      if (a == 0.0) continue;
      for (int j = 0; j < n; ++j) C[(size_t)i * n + j] += a * B[(size_t)p * n + j];
    }
  return C;
}

}  // namespace

// ---- host trains: cores [r0][N][r1] with a flattened mode N ----------------------------------

void HTrain::round(double eps, int rmax) {
  const int d = (int)c.size();
  if (d <= 1) return;
  // left-orthogonalise
  for (int k = 0; k < d - 1; ++k) {
    HCore& a = c[k];
    HCore& b = c[k + 1];
    int m = a.r0 * a.N, n = a.r1;
    std::vector<double> Q, R;
    hqr(m, n, a.v, Q, R);
    int kq = std::min(m, n);
    a.v = Q;
    a.r1 = kq;
    b.v = hmm(kq, n, b.N * b.r1, R.data(), b.v.data());
    b.r0 = kq;
  }
  double nrm = 0;
  for (double x : c[d - 1].v) nrm += x * x;
  nrm = std::sqrt(nrm);
  const double delta = eps / std::sqrt((double)(d - 1)) * nrm;
  for (int k = d - 1; k >= 1; --k) {
    HCore& a = c[k];
    HCore& p = c[k - 1];
    int r0 = a.r0, w = a.N * a.r1;
    std::vector<double> U, S, Vt, left, right;
    int q = std::min(r0, w);
    if (w >= r0) {
      hsvd(w, r0, htranspose(r0, w, a.v), U, S, Vt);  // M^T = U S Vt
      right = htranspose(w, q, U);                     // q x w
      left = htranspose(q, q, Vt);                     // r0 x q
    } else {
      hsvd(r0, w, a.v, U, S, Vt);
      right = Vt;
      left = U;
    }
    int rk = truncation_rank(S, delta, rmax);
    std::vector<double> LS((size_t)r0 * rk);
    for (int i = 0; i < r0; ++i)
      for (int j = 0; j < rk; ++j) LS[(size_t)i * rk + j] = left[(size_t)i * q + j] * S[j];
    a.v.assign(right.begin(), right.begin() + (size_t)rk * w);
    a.r0 = rk;
    p.v = hmm(p.r0 * p.N, r0, rk, p.v.data(), LS.data());
    p.r1 = rk;
  }
}

// TT-SVD of a vector of length 2^L into L cores of mode 2
HTrain htt_from_vector(const std::vector<double>& v, int L) {
  HTrain t;
  size_t n = v.size();
  std::vector<double> C(v);
  int r = 1;
  size_t rest = n;
  for (int k = 0; k < L - 1; ++k) {
    rest /= 2;
    int m = r * 2;
    // C is (m x rest) row-major; SVD through QR of its transpose
    std::vector<double> Ct = htranspose(m, (int)rest, C);  // rest x m
    std::vector<double> Q, R;
    hqr((int)rest, m, Ct, Q, R);                           // Ct = Q R, R: m' x m
    int mq = std::min((int)rest, m);
    // C = R^T Q^T; SVD of R^T (m x mq)
    std::vector<double> Rt = htranspose(mq, m, R);         // m x mq
    std::vector<double> U, S, Vt;
    int keep;
    if (m >= mq) {
      hsvd(m, mq, Rt, U, S, Vt);  // U: m x mq
      double tot = 0;
      for (double s : S) tot += s * s;
      keep = truncation_rank(S, 1e-15 * std::sqrt(tot), 1 << 20);
      HCore core{r, 2, keep, {}};
      core.v.assign((size_t)m * keep, 0.0);
      for (int i = 0; i < m; ++i)
        for (int j = 0; j < keep; ++j) core.v[(size_t)i * keep + j] = U[(size_t)i * mq + j];
      t.c.push_back(core);
      // next C = S Vt Q^T  (keep x rest)
      std::vector<double> SV((size_t)keep * mq);
      for (int i = 0; i < keep; ++i)
        for (int j = 0; j < mq; ++j) SV[(size_t)i * mq + j] = S[i] * Vt[(size_t)i * mq + j];
      std::vector<double> Qt = htranspose((int)rest, mq, Q);  // mq x rest
      C = hmm(keep, mq, (int)rest, SV.data(), Qt.data());
    } else {
      // m < mq cannot happen (mq = min(rest, m) <= m)
      throw Error(TNFEM_E_INVALID, "htt_from_vector: unexpected shape");
    }
    r = keep;
  }
  t.c.push_back(HCore{r, 2, 1, C});
  return t;
}

// TT-SVD of a dense array (row-major, modes[0] slowest), left to right: each unfolding C (m x rest)
// through the QR of its transpose and the SVD of the small factor, truncated to
// eps / sqrt(d-1) ||v|| per bond.
HTrain htt_svd(const std::vector<double>& v, const std::vector<int>& modes, double eps) {
  const int d = (int)modes.size();
  size_t total = 1;
  for (int m : modes) total *= (size_t)m;
  TN_REQUIRE(total == v.size(), "htt_svd: array size does not match the modes");
  double nrm = 0;
  for (double x : v) nrm += x * x;
  const double delta = eps / std::sqrt((double)std::max(1, d - 1)) * std::sqrt(nrm);
  HTrain t;
  std::vector<double> C(v);
  size_t rest = total;
  int r = 1;
  for (int k = 0; k < d - 1; ++k) {
    rest /= (size_t)modes[k];
    const int m = r * modes[k];
    std::vector<double> U, S, Vt, next;
    int keep, q;
    if ((size_t)m <= rest) {
      std::vector<double> Q, R;
      hqr((int)rest, m, htranspose(m, (int)rest, C), Q, R);  // C^T = Q R, R: m x m
      hsvd(m, m, htranspose(m, m, R), U, S, Vt);             // R^T = U S Vt, C = U S Vt Q^T
      keep = truncation_rank(S, delta, 1 << 20);
      q = m;
      std::vector<double> SV((size_t)keep * m);
      for (int i = 0; i < keep; ++i)
        for (int j = 0; j < m; ++j) SV[(size_t)i * m + j] = S[i] * Vt[(size_t)i * m + j];
      next = hmm(keep, m, (int)rest, SV.data(), htranspose((int)rest, m, Q).data());
    } else {
      hsvd(m, (int)rest, C, U, S, Vt);  // C = U S Vt directly (m > rest)
      keep = truncation_rank(S, delta, 1 << 20);
      q = (int)rest;
      next.assign((size_t)keep * rest, 0.0);
      for (int i = 0; i < keep; ++i)
        for (size_t j = 0; j < rest; ++j) next[(size_t)i * rest + j] = S[i] * Vt[(size_t)i * rest + j];
    }
    HCore core{r, modes[k], keep, std::vector<double>((size_t)m * keep)};
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < keep; ++j) core.v[(size_t)i * keep + j] = U[(size_t)i * q + j];
    t.c.push_back(core);
    C.swap(next);
    r = keep;
  }
  t.c.push_back(HCore{r, modes[d - 1], 1, C});
  return t;
}

// ---- 1D tridiagonal operators in QTT ----------------------------------------------------------

namespace {

// superdiagonal shift J (J[i][i+1] = 1), MSB first: rank 2 (no carry yet / carried)
HTrain shift_mpo(int L, bool transpose) {
  auto J2 = [&](int i, int j) { return transpose ? (i == 1 && j == 0) : (i == 0 && j == 1); };
  auto JT2 = [&](int i, int j) { return transpose ? (i == 0 && j == 1) : (i == 1 && j == 0); };
  HTrain t;
  if (L == 1) {
    HCore c{1, 4, 1, std::vector<double>(4, 0.0)};
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 2; ++j) c.v[i * 2 + j] = J2(i, j) ? 1.0 : 0.0;
    t.c.push_back(c);
    return t;
  }
  for (int k = 0; k < L; ++k) {
    int r0 = k == 0 ? 1 : 2, r1 = k == L - 1 ? 1 : 2;
    HCore c{r0, 4, r1, std::vector<double>((size_t)r0 * 4 * r1, 0.0)};
    auto set = [&](int a, int i, int j, int b, double v) { c.v[((size_t)a * 4 + i * 2 + j) * r1 + b] = v; };
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 2; ++j) {
        double I2 = (i == j) ? 1.0 : 0.0;
        double J = J2(i, j) ? 1.0 : 0.0, JT = JT2(i, j) ? 1.0 : 0.0;
        if (k == 0) { set(0, i, j, 0, I2); set(0, i, j, 1, J); }
        else if (k < L - 1) { set(0, i, j, 0, I2); set(0, i, j, 1, J); set(1, i, j, 1, JT); }
        else { set(0, i, j, 0, J); set(1, i, j, 0, JT); }
      }
    t.c.push_back(c);
  }
  return t;
}

// diag(v) as an operator train from the vector's QTT
HTrain diag_mpo(const std::vector<double>& v, int L) {
  HTrain x = htt_from_vector(v, L);
  HTrain t;
  for (auto& c : x.c) {
    HCore o{c.r0, 4, c.r1, std::vector<double>((size_t)c.r0 * 4 * c.r1, 0.0)};
    for (int a = 0; a < c.r0; ++a)
      for (int i = 0; i < 2; ++i)
        for (int b = 0; b < c.r1; ++b) o.v[((size_t)a * 4 + i * 3) * c.r1 + b] = c.v[((size_t)a * 2 + i) * c.r1 + b];
    t.c.push_back(o);
  }
  return t;
}

// product of operator trains (A B), modes 2x2 per core
HTrain mpo_mul(const HTrain& A, const HTrain& B) {
  HTrain t;
  for (size_t k = 0; k < A.c.size(); ++k) {
    const HCore& a = A.c[k];
    const HCore& b = B.c[k];
    int r0 = a.r0 * b.r0, r1 = a.r1 * b.r1;
    HCore o{r0, 4, r1, std::vector<double>((size_t)r0 * 4 * r1, 0.0)};
    for (int a0 = 0; a0 < a.r0; ++a0)
      for (int b0 = 0; b0 < b.r0; ++b0)
        for (int i = 0; i < 2; ++i)
          for (int j = 0; j < 2; ++j)
            for (int a1 = 0; a1 < a.r1; ++a1)
              for (int b1 = 0; b1 < b.r1; ++b1) {
                double s = 0;
                for (int l = 0; l < 2; ++l)
                  s += a.v[((size_t)a0 * 4 + i * 2 + l) * a.r1 + a1] * b.v[((size_t)b0 * 4 + l * 2 + j) * b.r1 + b1];
                o.v[((size_t)(a0 * b.r0 + b0) * 4 + i * 2 + j) * r1 + a1 * b.r1 + b1] = s;
              }
    t.c.push_back(o);
  }
  return t;
}

// block-diagonal sum of trains with identical modes
HTrain tt_sum(const std::vector<HTrain>& xs, const std::vector<double>& coef) {
  const int d = (int)xs[0].c.size();
  HTrain t;
  for (int k = 0; k < d; ++k) {
    int R0 = 0, R1 = 0;
    for (auto& x : xs) { R0 += x.c[k].r0; R1 += x.c[k].r1; }
    if (k == 0) R0 = 1;
    if (k == d - 1) R1 = 1;
    int N = xs[0].c[k].N;
    HCore o{R0, N, R1, std::vector<double>((size_t)R0 * N * R1, 0.0)};
    int o0 = 0, o1 = 0;
    for (size_t s = 0; s < xs.size(); ++s) {
      const HCore& c = xs[s].c[k];
      double f = (k == 0) ? coef[s] : 1.0;
      int q0 = (k == 0) ? 0 : o0, q1 = (k == d - 1) ? 0 : o1;
      if (d == 1) { q0 = 0; q1 = 0; }
      for (int a = 0; a < c.r0; ++a)
        for (int i = 0; i < N; ++i)
          for (int b = 0; b < c.r1; ++b) o.v[((size_t)(q0 + a) * N + i) * R1 + q1 + b] += f * c.v[((size_t)a * N + i) * c.r1 + b];
      o0 += c.r0;
      o1 += c.r1;
    }
    t.c.push_back(o);
  }
  return t;
}

// tridiagonal X = diag(m) + diag(s) J + J^T diag(t) (s[i] at (i, i+1), t[i] at (i+1, i))
HTrain tridiag_mpo(const std::vector<double>& m, const std::vector<double>& s, const std::vector<double>& t, int L) {
  std::vector<HTrain> parts;
  std::vector<double> coef;
  auto nz = [](const std::vector<double>& v) { for (double x : v) if (x != 0.0) return true; return false; };
  if (nz(m)) { parts.push_back(diag_mpo(m, L)); coef.push_back(1.0); }
  if (nz(s)) { parts.push_back(mpo_mul(diag_mpo(s, L), shift_mpo(L, false))); coef.push_back(1.0); }
  if (nz(t)) { parts.push_back(mpo_mul(shift_mpo(L, true), diag_mpo(t, L))); coef.push_back(1.0); }
  if (parts.empty()) {
    std::vector<double> z(m.size(), 0.0);
    parts.push_back(diag_mpo(z, L));
    coef.push_back(0.0);
  }
  HTrain x = tt_sum(parts, coef);
  x.round(1e-15, 1 << 20);
  return x;
}

}  // namespace

// ---- axis catalogues ---------------------------------------------------------------------------

AxisOps axis_operators(int L, double lo, double hi, const std::vector<double>& w, bool clamp_lo, bool clamp_hi,
                       bool with_bc) {
  const int n = 1 << L;
  const double h = (hi - lo) / (n - 1);
  std::vector<double> p(n, 1.0);
  if (with_bc && clamp_lo) p[0] = 0.0;
  if (with_bc && clamp_hi) p[n - 1] = 0.0;
  auto we = [&](int e) { return (e >= 0 && e < n - 1) ? w[e] : 0.0; };
  AxisOps ops;
  ops.names = {"K", "M", "G", "GT", "I", "P"};
  std::vector<HTrain> trains;
  std::vector<std::future<HTrain>> parts;
  for (const auto& name : ops.names) {
    std::vector<double> m(n, 0.0), s(n, 0.0), t(n, 0.0);
    for (int i = 0; i < n; ++i) {
      if (name == "K") {
        m[i] = (we(i - 1) + we(i)) / h;
        if (i < n - 1) { s[i] = -we(i) / h; t[i] = -we(i) / h; }
      } else if (name == "M") {
        m[i] = (we(i - 1) + we(i)) * h / 3.0;
        if (i < n - 1) { s[i] = we(i) * h / 6.0; t[i] = we(i) * h / 6.0; }
      } else if (name == "G") {  // int phi_i phi_j' (test i, trial j)
        m[i] = -0.5 * we(i) + 0.5 * we(i - 1);
        if (i < n - 1) { s[i] = 0.5 * we(i); t[i] = -0.5 * we(i); }
      } else if (name == "GT") {
        m[i] = -0.5 * we(i) + 0.5 * we(i - 1);
        if (i < n - 1) { s[i] = -0.5 * we(i); t[i] = 0.5 * we(i); }
      } else if (name == "I") {
        m[i] = 1.0;
      } else {  // P
        m[i] = p[i];
      }
      if (name != "I" && name != "P") {
        m[i] *= p[i] * p[i];
        if (i < n - 1) { s[i] *= p[i] * p[i + 1]; t[i] *= p[i + 1] * p[i]; }
      }
    }
    ops.diag1.push_back(m[std::min(1, n - 1)]);  // entry (1,1), used for the shift s
    // the six 1D operators are independent: their TT-SVDs and roundings run on host threads
    parts.push_back(std::async(std::launch::async, [m, s, t, L] { return tridiag_mpo(m, s, t, L); }));
  }
  for (auto& f : parts) trains.push_back(f.get());
  ops.joint = stack_trains(trains);
  ops.joint.round(1e-15, 1 << 20);
  return ops;
}

// Stack trains with identical modes under a leading index t: result has modes [T, N, N, ...]
HTrain stack_trains(const std::vector<HTrain>& xs) {
  const int T = (int)xs.size();
  const int d = (int)xs[0].c.size();
  HTrain out;
  HCore sel{1, T, T, std::vector<double>((size_t)T * T, 0.0)};
  for (int t = 0; t < T; ++t) sel.v[(size_t)t * T + t] = 1.0;
  out.c.push_back(sel);
  for (int k = 0; k < d; ++k) {
    int R0 = 0, R1 = 0;
    for (auto& x : xs) { R0 += (k == 0) ? 1 : x.c[k].r0; R1 += x.c[k].r1; }
    if (k == 0) R0 = T;
    if (k == d - 1) R1 = 1;
    int N = xs[0].c[k].N;
    HCore o{R0, N, R1, std::vector<double>((size_t)R0 * N * R1, 0.0)};
    int o0 = 0, o1 = 0;
    for (int s = 0; s < T; ++s) {
      const HCore& c = xs[s].c[k];
      int q0 = (k == 0) ? s : o0, q1 = (k == d - 1) ? 0 : o1;
      for (int a = 0; a < c.r0; ++a)
        for (int i = 0; i < N; ++i)
          for (int b = 0; b < c.r1; ++b) o.v[((size_t)(q0 + a) * N + i) * R1 + q1 + b] = c.v[((size_t)a * N + i) * c.r1 + b];
      o0 += c.r0;
      o1 += c.r1;
    }
    out.c.push_back(o);
  }
  return out;
}

// D-dimensional train from per-axis joint trains and a list of separable terms.
// Each axis train has modes [T_d, q, q, ...] (q = 4 for operators, 2 for vectors); the result
// has a component core of mode ncomp (vectors) or ncomp x ncomp (operators, `op` true) and
// level cores of mode q^D.
HTrain combine_axes(const std::vector<HTrain>& axes, const std::vector<SepTerm>& terms, int ncomp, bool op) {
  const int D = (int)axes.size();
  const int L = (int)axes[0].c.size() - 1;
  const int q = axes[0].c[1].N;  // 4 (operator bits i,j) or 2 (vector bit)
  const int qb = op ? 2 : 1;     // bits per mode side
  (void)qb;
  // blocks: operator -> p = c*ncomp + c'; vector -> p = c
  const int P = op ? ncomp * ncomp : ncomp;
  HTrain out;
  // component core
  {
    HCore c0{1, op ? ncomp * ncomp : ncomp, P, std::vector<double>((size_t)(op ? ncomp * ncomp : ncomp) * P, 0.0)};
    for (int p = 0; p < P; ++p) c0.v[(size_t)p * P + p] = 1.0;
    out.c.push_back(c0);
  }
  // first level core: merge operator index cores with the first bit cores
  std::vector<std::vector<double>> first(D);  // [T_d][q][rho_d]
  std::vector<int> Td(D), rho0(D);
  for (int d = 0; d < D; ++d) {
    const HCore& sel = axes[d].c[0];  // 1 x T x rA
    const HCore& b0 = axes[d].c[1];   // rA x q x rho
    Td[d] = sel.N;
    rho0[d] = b0.r1;
    first[d] = hmm(sel.N, sel.r1, q * b0.r1, sel.v.data(), b0.v.data());
  }
  const int Q = (int)std::lround(std::pow(q, D));
  auto merged = [&](const std::vector<int>& loc) {
    // loc[d] = local mode index of axis d (operator: i*2+j; vector: b). Merge bits across axes.
    if (!op) {
      int s = 0;
      for (int d = 0; d < D; ++d) s = s * 2 + loc[d];
      return s;
    }
    int si = 0, sj = 0;
    for (int d = 0; d < D; ++d) { si = si * 2 + loc[d] / 2; sj = sj * 2 + loc[d] % 2; }
    return si * (1 << D) + sj;
  };
  {
    int Rr = 1;
    for (int d = 0; d < D; ++d) Rr *= rho0[d];
    HCore c1{P, Q, Rr, std::vector<double>((size_t)P * Q * Rr, 0.0)};
    std::vector<int> loc(D), rr(D);
    for (const SepTerm& t : terms) {
      const int p = op ? t.c * ncomp + t.c2 : t.c;
      // iterate over local modes and right ranks of all axes
      long long total = 1;
      for (int d = 0; d < D; ++d) total *= (long long)q * rho0[d];
      for (long long idx = 0; idx < total; ++idx) {
        long long rem = idx;
        double v = t.coef;
        for (int d = D - 1; d >= 0; --d) {
          rr[d] = (int)(rem % rho0[d]);
          rem /= rho0[d];
          loc[d] = (int)(rem % q);
          rem /= q;
        }
        for (int d = 0; d < D && v != 0.0; ++d) v *= first[d][((size_t)t.ops[d] * q + loc[d]) * rho0[d] + rr[d]];
        if (v == 0.0) continue;
        int r = 0;
        for (int d = 0; d < D; ++d) r = r * rho0[d] + rr[d];
        c1.v[((size_t)p * Q + merged(loc)) * Rr + r] += v;
      }
    }
    out.c.push_back(c1);
  }
  // remaining level cores: Kronecker products of axis cores, formed axis by axis as
  // T <- T (x) c_d over (left rank, local mode, right rank) (axis 0 most significant in each),
  // then the local modes (loc_0, ..., loc_{D-1}) are merged into the level mode
  std::vector<int> mq(Q);
  {
    std::vector<int> loc(D);
    for (int lin = 0; lin < Q; ++lin) {
      int rm = lin;
      for (int d = D - 1; d >= 0; --d) { loc[d] = rm % q; rm /= q; }
      mq[lin] = merged(loc);
    }
  }
  for (int k = 2; k <= L; ++k) {
    const HCore& c0 = axes[0].c[k];
    int A0 = c0.r0, Qm = q, B0 = c0.r1;
    std::vector<double> T(c0.v);
    for (int d = 1; d < D; ++d) {
      const HCore& c = axes[d].c[k];
      const int A1 = A0 * c.r0, Q1 = Qm * q, B1 = B0 * c.r1;
      std::vector<double> T1((size_t)A1 * Q1 * B1);
      for (int a = 0; a < A0; ++a)
        for (int ad = 0; ad < c.r0; ++ad)
          for (int l = 0; l < Qm; ++l)
            for (int ld = 0; ld < q; ++ld) {
              double* o = &T1[(((size_t)a * c.r0 + ad) * Q1 + (size_t)l * q + ld) * B1];
              const double* t = &T[((size_t)a * Qm + l) * B0];
              const double* cc = &c.v[((size_t)ad * q + ld) * c.r1];
              for (int b = 0; b < B0; ++b)
                for (int bd = 0; bd < c.r1; ++bd) o[(size_t)b * c.r1 + bd] = t[b] * cc[bd];
            }
      T.swap(T1);
      A0 = A1;
      Qm = Q1;
      B0 = B1;
    }
    HCore ck{A0, Q, B0, std::vector<double>((size_t)A0 * Q * B0, 0.0)};
    for (int a = 0; a < A0; ++a)
      for (int lin = 0; lin < Q; ++lin) {
        const double* t = &T[((size_t)a * Q + lin) * B0];
        double* o = &ck.v[((size_t)a * Q + mq[lin]) * B0];
        for (int b = 0; b < B0; ++b) o[b] = (t[b] == 0.0) ? 0.0 : t[b];
      }
    out.c.push_back(ck);
  }
  return out;
}

// ---- elasticity operator terms -----------------------------------------------------------------

void lame(double E, double nu, int dim, bool plane_stress, double& lam, double& mu) {
  lam = E * nu / ((1 + nu) * (1 - 2 * nu));
  mu = E / (2 * (1 + nu));
  if (dim == 2 && plane_stress) lam = 2 * lam * mu / (lam + 2 * mu);
}

// op indices in AxisOps::names
enum { OP_K = 0, OP_M = 1, OP_G = 2, OP_GT = 3, OP_I = 4, OP_P = 5 };

std::vector<SepTerm> stiffness_terms(int D, double lam, double mu) {
  std::vector<SepTerm> out;
  for (int c = 0; c < D; ++c)
    for (int c2 = 0; c2 < D; ++c2) {
      SepTerm t1{c, c2, lam, std::vector<int>(D)};
      SepTerm t2{c, c2, mu, std::vector<int>(D)};
      for (int d = 0; d < D; ++d) {
        // lam d_c N_a d_c' N_b
        t1.ops[d] = (d == c && d == c2) ? OP_K : (d == c) ? OP_GT : (d == c2) ? OP_G : OP_M;
        // mu d_c' N_a d_c N_b
        t2.ops[d] = (d == c && d == c2) ? OP_K : (d == c2) ? OP_GT : (d == c) ? OP_G : OP_M;
      }
      out.push_back(t1);
      out.push_back(t2);
      if (c == c2)
        for (int e = 0; e < D; ++e) {
          SepTerm t{c, c, mu, std::vector<int>(D)};
          for (int d = 0; d < D; ++d) t.ops[d] = (d == e) ? OP_K : OP_M;
          out.push_back(t);
        }
    }
  return out;
}

// Affine grids (grid.mapped): x = lo + J xi on the unit box, J[e][d] = edges[d][e].  The builders
// run on the unit box and fold the map into the coefficients: physical derivatives are
// d/dx_e = sum_p Jinv[p][e] d/dxi_p, and every integral carries |det J|.
struct Affine {
  double J[3][3] = {{0}}, Jinv[3][3] = {{0}}, det = 1.0;
};

static Affine affine_of(const tnfem_grid& g) {
  Affine a;
  const int D = g.dim;
  for (int e = 0; e < D; ++e)
    for (int d = 0; d < D; ++d) a.J[e][d] = g.edges[d][e];
  if (D == 2) {
    a.det = a.J[0][0] * a.J[1][1] - a.J[0][1] * a.J[1][0];
    TN_REQUIRE(std::fabs(a.det) > 0, "mapped grid: the edges are linearly dependent");
    a.Jinv[0][0] = a.J[1][1] / a.det;
    a.Jinv[0][1] = -a.J[0][1] / a.det;
    a.Jinv[1][0] = -a.J[1][0] / a.det;
    a.Jinv[1][1] = a.J[0][0] / a.det;
  } else {
    const double(&m)[3][3] = a.J;
    a.det = m[0][0] * (m[1][1] * m[2][2] - m[1][2] * m[2][1]) - m[0][1] * (m[1][0] * m[2][2] - m[1][2] * m[2][0]) +
            m[0][2] * (m[1][0] * m[2][1] - m[1][1] * m[2][0]);
    TN_REQUIRE(std::fabs(a.det) > 0, "mapped grid: the edges are linearly dependent");
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        // cofactor of m[j][i] over det
        const int r0 = (j + 1) % 3, r1 = (j + 2) % 3, c0 = (i + 1) % 3, c1 = (i + 2) % 3;
        a.Jinv[i][j] = (m[r0][c0] * m[r1][c1] - m[r0][c1] * m[r1][c0]) / a.det;
      }
  }
  return a;
}

void grid_affine_inverse(const tnfem_grid& g, double Jinv[3][3], double* det) {
  const Affine a = affine_of(g);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) Jinv[i][j] = a.Jinv[i][j];
  if (det) *det = a.det;
}

static tnfem_grid unit_box(const tnfem_grid& g) {
  tnfem_grid u = g;
  u.mapped = 0;
  for (int d = 0; d < 3; ++d) {
    u.lo[d] = 0.0;
    u.hi[d] = 1.0;
  }
  return u;
}

// Stiffness terms of an affine grid on the unit box: block (c, c2) is
// sum_{p,q} K[p][q] int d_p(test) d_q(trial) dxi with
// K[p][q] = |det J| (lam Jinv[p][c] Jinv[q][c2] + mu Jinv[p][c2] Jinv[q][c] + mu [c = c2] sum_e Jinv[p][e] Jinv[q][e]);
// the reference integral factors per axis: K where p = q = d, G^T on the test-derivative axis,
// G on the trial-derivative axis, M elsewhere.
static std::vector<SepTerm> stiffness_terms_mapped(int D, double lam, double mu, const Affine& af) {
  std::vector<SepTerm> out;
  for (int c = 0; c < D; ++c)
    for (int c2 = 0; c2 < D; ++c2)
      for (int p = 0; p < D; ++p)
        for (int q = 0; q < D; ++q) {
          double k = lam * af.Jinv[p][c] * af.Jinv[q][c2] + mu * af.Jinv[p][c2] * af.Jinv[q][c];
          if (c == c2)
            for (int e = 0; e < D; ++e) k += mu * af.Jinv[p][e] * af.Jinv[q][e];
          k *= std::fabs(af.det);
          if (k == 0.0) continue;
          SepTerm t{c, c2, k, std::vector<int>(D)};
          for (int d = 0; d < D; ++d) t.ops[d] = (d == p && d == q) ? OP_K : (d == p) ? OP_GT : (d == q) ? OP_G : OP_M;
          out.push_back(t);
        }
  return out;
}

// dense quadrilateral arrays (quad.cu) -> trains by TT-SVD on the host
static std::vector<int> quad_modes(int L, int first, int last) {
  std::vector<int> m(1, first);
  m.insert(m.end(), L, 4);
  if (last) m.push_back(last);
  return m;
}

HTrain stiffness_train(const tnfem_grid& g_in, const tnfem_material& mat_in, double* shift_out) {
  if (g_in.mapped == 2) {
    std::vector<double> full;
    quad_operator_coefficients(g_in, mat_in, false, full, shift_out);
    HTrain B = quad_stage_axis1(htt_svd(full, quad_modes(g_in.levels, 4, 9), 1e-14));
    B.round(1e-14, 1 << 20);
    return quad_stage_axis0(B);
  }
  const bool mapped = g_in.mapped != 0;
  Affine af;
  tnfem_material mat = mat_in;
  if (mapped) {
    af = affine_of(g_in);
    // the element weights of a two-material split are not separable on a sheared grid: the whole
    // domain must lie on one side of the split (element centroids between xmin and xmax)
    double xmin = g_in.lo[0], xmax = g_in.lo[0];
    for (int d = 0; d < g_in.dim; ++d) (af.J[0][d] < 0 ? xmin : xmax) += af.J[0][d];
    TN_REQUIRE(mat_in.E[0] == mat_in.E[1] || !(mat_in.split_x > xmin && mat_in.split_x <= xmax),
               "mapped grid: the material must be homogeneous");
    const double E = (mat_in.split_x > xmax) ? mat_in.E[0] : mat_in.E[1];
    mat.E[0] = mat.E[1] = E;
    mat.split_x = 1e300;
  }
  const tnfem_grid g = mapped ? unit_box(g_in) : g_in;
  const int D = g.dim, L = g.levels, n = 1 << L;
  double lam, mu;
  lame(mat.E[0], mat.nu, D, g.plane_stress != 0, lam, mu);
  std::vector<HTrain> axes;
  std::vector<AxisOps> cats;
  std::vector<std::future<AxisOps>> cat_f;
  bool any_clamp = false;
  for (int f = 0; f < 2 * D; ++f) any_clamp |= g.clamped[f] != 0;
  for (int d = 0; d < D; ++d) {
    std::vector<double> w(n - 1, 1.0);
    if (d == 0) {
      const double h = (g.hi[0] - g.lo[0]) / (n - 1);
      for (int e = 0; e < n - 1; ++e) {
        double cx = g.lo[0] + (e + 0.5) * h;
        w[e] = (cx < mat.split_x ? mat.E[0] : mat.E[1]) / mat.E[0];
      }
    }
    cat_f.push_back(std::async(std::launch::async, [=, &g] {
      return axis_operators(L, g.lo[d], g.hi[d], w, g.clamped[2 * d] != 0, g.clamped[2 * d + 1] != 0, true);
    }));
  }
  for (auto& f : cat_f) {
    cats.push_back(f.get());
    axes.push_back(cats.back().joint);
  }
  std::vector<SepTerm> terms = mapped ? stiffness_terms_mapped(D, lam, mu, af) : stiffness_terms(D, lam, mu);
  // shift s: mean over components of the unconstrained diagonal at node (1,...,1); the
  // unconstrained entry (1,1) of each 1D matrix is kept in diag1 before projection for n > 2
  double s = 0;
  {
    // recompute unprojected (1,1) entries: projection only touches end nodes, node 1 is interior
    // for n >= 3; for n == 2 node 1 is an end node and may be clamped, so use the raw formula
    std::vector<std::vector<double>> e11(D, std::vector<double>(4));
    for (int d = 0; d < D; ++d) {
      const double h = (g.hi[d] - g.lo[d]) / (n - 1);
      double w0 = 1.0, w1 = 1.0;
      if (d == 0) {
        double c0 = g.lo[0] + 0.5 * h, c1 = g.lo[0] + 1.5 * h;
        w0 = (c0 < mat.split_x ? mat.E[0] : mat.E[1]) / mat.E[0];
        w1 = (n > 2) ? ((c1 < mat.split_x ? mat.E[0] : mat.E[1]) / mat.E[0]) : 0.0;
      } else if (n <= 2) {
        w1 = 0.0;
      }
      e11[d][OP_K] = (w0 + w1) / h;
      e11[d][OP_M] = (w0 + w1) * h / 3.0;
      e11[d][OP_G] = -0.5 * w1 + 0.5 * w0;
      e11[d][OP_GT] = e11[d][OP_G];
    }
    for (const SepTerm& t : terms) {
      if (t.c != t.c2) continue;
      double v = t.coef;
      for (int d = 0; d < D; ++d) v *= e11[d][t.ops[d]];
      s += v;
    }
    s /= D;
  }
  if (shift_out) *shift_out = s;
  if (any_clamp) {
    for (int c = 0; c < D; ++c) {
      terms.push_back(SepTerm{c, c, s, std::vector<int>(D, OP_I)});
      terms.push_back(SepTerm{c, c, -s, std::vector<int>(D, OP_P)});
    }
  }
  return combine_axes(axes, terms, D, true);
}

HTrain projector_train(const tnfem_grid& g) {
  // P = I_c (x) P_0 (x) ... (x) P_{D-1}: the faces are index-space boundaries on every grid kind
  const int D = g.dim, L = g.levels, n = 1 << L;
  std::vector<HTrain> axes;
  for (int d = 0; d < D; ++d)
    axes.push_back(axis_operators(L, 0.0, 1.0, std::vector<double>(n - 1, 1.0), g.clamped[2 * d] != 0,
                                  g.clamped[2 * d + 1] != 0, true).joint);
  std::vector<SepTerm> terms;
  for (int c = 0; c < D; ++c) terms.push_back(SepTerm{c, c, 1.0, std::vector<int>(D, OP_P)});
  return combine_axes(axes, terms, D, true);
}

HTrain mass_train(const tnfem_grid& g_in) {
  if (g_in.mapped == 2) {
    std::vector<double> full;
    const tnfem_material any{{1.0, 1.0}, 1e300, 0.3};
    quad_operator_coefficients(g_in, any, true, full, nullptr);
    HTrain B = quad_stage_axis1(htt_svd(full, quad_modes(g_in.levels, 4, 9), 1e-14));
    B.round(1e-14, 1 << 20);
    return quad_stage_axis0(B);
  }
  const double vol = g_in.mapped ? std::fabs(affine_of(g_in).det) : 1.0;
  const tnfem_grid g = g_in.mapped ? unit_box(g_in) : g_in;
  const int D = g.dim, L = g.levels, n = 1 << L;
  std::vector<std::future<AxisOps>> cat_f;
  for (int d = 0; d < D; ++d)
    cat_f.push_back(std::async(std::launch::async, [=, &g] {
      return axis_operators(L, g.lo[d], g.hi[d], std::vector<double>(n - 1, 1.0), false, false, false);
    }));
  std::vector<HTrain> axes;
  for (auto& f : cat_f) axes.push_back(f.get().joint);
  std::vector<SepTerm> terms;
  for (int c = 0; c < D; ++c) terms.push_back(SepTerm{c, c, vol, std::vector<int>(D, OP_M)});
  return combine_axes(axes, terms, D, true);
}

// ---- loads ---------------------------------------------------------------------------------------

namespace {

// y = M x for the 1D mass matrix on n nodes with spacing h
std::vector<double> mass_apply(const std::vector<double>& x, double h) {
  const int n = (int)x.size();
  std::vector<double> y(n, 0.0);
  for (int e = 0; e < n - 1; ++e) {
    y[e] += h / 3.0 * x[e] + h / 6.0 * x[e + 1];
    y[e + 1] += h / 6.0 * x[e] + h / 3.0 * x[e + 1];
  }
  return y;
}

struct VecCatalog {
  std::vector<std::vector<double>> v;
  int add(const std::vector<double>& x) { v.push_back(x); return (int)v.size() - 1; }
};

}  // namespace

HTrain load_train(const tnfem_grid& g_in, const tnfem_material& mat, const tnfem_load* loads, int n_loads) {
  if (g_in.mapped == 2) {
    std::vector<double> full;
    quad_load_values(g_in, mat, loads, n_loads, full);
    return htt_svd(full, quad_modes(g_in.levels, 2, 0), 1e-15);
  }
  // affine grid: body forces carry |det J|, a traction on a face the ratio of the face's measure
  // to the unit box face's (|J t| for the side along reference axis t in 2D, |J t1 x J t2| in 3D)
  const bool mapped = g_in.mapped != 0;
  Affine af;
  if (mapped) af = affine_of(g_in);
  auto face_scale = [&](int dn) {
    if (!mapped) return 1.0;
    double t[2][3] = {{0}};
    int k = 0;
    for (int d = 0; d < g_in.dim; ++d)
      if (d != dn) {
        for (int e = 0; e < 3; ++e) t[k][e] = e < g_in.dim ? af.J[e][d] : 0.0;
        ++k;
      }
    if (g_in.dim == 2) return std::sqrt(t[0][0] * t[0][0] + t[0][1] * t[0][1]);
    const double cx = t[0][1] * t[1][2] - t[0][2] * t[1][1], cy = t[0][2] * t[1][0] - t[0][0] * t[1][2],
                 cz = t[0][0] * t[1][1] - t[0][1] * t[1][0];
    return std::sqrt(cx * cx + cy * cy + cz * cz);
  };
  const tnfem_grid g = mapped ? unit_box(g_in) : g_in;
  const int D = g.dim, L = g.levels, n = 1 << L;
  std::vector<VecCatalog> cat(D);
  std::vector<std::vector<double>> X(D), P(D);
  std::vector<double> h(D);
  for (int d = 0; d < D; ++d) {
    h[d] = (g.hi[d] - g.lo[d]) / (n - 1);
    X[d].resize(n);
    P[d].assign(n, 1.0);
    for (int i = 0; i < n; ++i) X[d][i] = g.lo[d] + h[d] * i;
    if (g.clamped[2 * d]) P[d][0] = 0.0;
    if (g.clamped[2 * d + 1]) P[d][n - 1] = 0.0;
  }
  // projected mass-weighted function along axis d
  auto massfn = [&](int d, auto fn) {
    std::vector<double> x(n);
    for (int i = 0; i < n; ++i) x[i] = fn(X[d][i]);
    std::vector<double> y = mass_apply(x, h[d]);
    for (int i = 0; i < n; ++i) y[i] *= P[d][i];
    return cat[d].add(y);
  };
  auto endvec = [&](int d, int side) {
    std::vector<double> y(n, 0.0);
    y[side ? n - 1 : 0] = P[d][side ? n - 1 : 0];
    return cat[d].add(y);
  };
  std::vector<SepTerm> terms;
  auto add = [&](int c, double coef, std::vector<int> ops) { terms.push_back(SepTerm{c, c, coef, ops}); };
  for (int li = 0; li < n_loads; ++li) {
    const tnfem_load& ld = loads[li];
    if (ld.kind == TNFEM_LOAD_GRAVITY) {
      std::vector<int> ops(D);
      for (int d = 0; d < D; ++d) ops[d] = massfn(d, [](double) { return 1.0; });
      add(D - 1, -ld.rho * ld.g * (mapped ? std::fabs(af.det) : 1.0), ops);
    } else if (ld.kind == TNFEM_LOAD_TRACTION) {
      TN_REQUIRE(ld.face >= 0 && ld.face < 2 * D, "traction face out of range");
      const int dn = ld.face / 2, side = ld.face % 2;
      const double fs = face_scale(dn);
      for (int c = 0; c < D; ++c) {
        if (ld.traction[c] == 0.0) continue;
        std::vector<int> ops(D);
        for (int d = 0; d < D; ++d) ops[d] = (d == dn) ? endvec(d, side) : massfn(d, [](double) { return 1.0; });
        add(c, ld.traction[c] * fs, ops);
      }
    } else if (mapped) {
      TN_REQUIRE(false, "mapped grid: loads must be gravity or uniform tractions");
    } else if (ld.kind == TNFEM_LOAD_FOURIER) {
      TN_REQUIRE(ld.n_modes >= 0 && (ld.n_modes == 0 || (ld.amp && ld.wave && ld.phase)), "fourier load arrays");
      for (int m = 0; m < ld.n_modes; ++m) {
        std::vector<int> sinv(D), cosv(D);
        for (int d = 0; d < D; ++d) {
          const double kk = M_PI * ld.wave[m * D + d];
          sinv[d] = massfn(d, [kk](double x) { return std::sin(kk * x); });
          cosv[d] = massfn(d, [kk](double x) { return std::cos(kk * x); });
        }
        // sin(sum_d theta_d + phi) = sum_S sin(phi + |S| pi/2) prod_{d in S} sin theta_d prod_{d notin S} cos theta_d
        for (int S = 0; S < (1 << D); ++S) {
          int card = __builtin_popcount(S);
          double cf = std::sin(ld.phase[m] + card * M_PI / 2.0);
          if (std::fabs(cf) < 1e-300) continue;
          std::vector<int> ops(D);
          for (int d = 0; d < D; ++d) ops[d] = (S >> d & 1) ? sinv[d] : cosv[d];
          for (int c = 0; c < D; ++c) {
            double a = ld.scale * ld.amp[c * ld.n_modes + m] * cf;
            if (a != 0.0) add(c, a, ops);
          }
        }
      }
    } else if (ld.kind == TNFEM_LOAD_MANUFACTURED) {
      TN_REQUIRE(D == 2, "manufactured load is two-dimensional");
      double lam, mu;
      lame(mat.E[0], mat.nu, 2, g.plane_stress != 0, lam, mu);
      const double pi = M_PI;
      auto one = [](double) { return 1.0; };
      auto sinp = [pi](double x) { return std::sin(pi * x); };
      auto cosp = [pi](double x) { return std::cos(pi * x); };
      auto lin = [](double x) { return 1.0 - 2.0 * x; };
      auto quad = [](double x) { return x * (1.0 - x); };
      // body force -div sigma(u*), u* = (sin pi x sin pi y, x(1-x) y(1-y))
      add(0, (lam + 3 * mu) * pi * pi, {massfn(0, sinp), massfn(1, sinp)});
      add(0, -(lam + mu), {massfn(0, lin), massfn(1, lin)});
      add(1, 2 * mu, {massfn(0, one), massfn(1, quad)});
      add(1, 2 * (lam + 2 * mu), {massfn(0, quad), massfn(1, one)});
      add(1, -(lam + mu) * pi * pi, {massfn(0, cosp), massfn(1, cosp)});
      // tractions sigma(u*) n on every face that is not clamped (face mass along the face)
      for (int side = 0; side < 2; ++side) {
        if (!g.clamped[0 + side]) {  // x faces: g = (-(lam+2mu) pi sin pi y, -mu y(1-y))
          add(0, -(lam + 2 * mu) * pi, {endvec(0, side), massfn(1, sinp)});
          add(1, -mu, {endvec(0, side), massfn(1, quad)});
        }
        if (!g.clamped[2 + side]) {  // y faces: g = (-mu pi sin pi x, -(lam+2mu) x(1-x))
          add(0, -mu * pi, {massfn(0, sinp), endvec(1, side)});
          add(1, -(lam + 2 * mu), {massfn(0, quad), endvec(1, side)});
        }
      }
    } else if (ld.kind == TNFEM_LOAD_NODAL_TT) {
      throw Error(TNFEM_E_INVALID, "a nodal-train load is applied on the device (tnfem_build_load), not on the host");
    } else {
      throw Error(TNFEM_E_INVALID, "unknown load kind");
    }
  }
  if (terms.empty()) {
    std::vector<int> ops(D);
    for (int d = 0; d < D; ++d) ops[d] = cat[d].add(std::vector<double>(n, 0.0));
    add(0, 0.0, ops);
  }
  std::vector<HTrain> axes;
  for (int d = 0; d < D; ++d) {
    std::vector<HTrain> trains;
    for (auto& v : cat[d].v) trains.push_back(htt_from_vector(v, L));
    HTrain j = stack_trains(trains);
    j.round(1e-15, 1 << 20);
    axes.push_back(j);
  }
  return combine_axes(axes, terms, D, false);
}

}  // namespace tnfem
