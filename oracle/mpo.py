"""Oracle B, part 2: the elasticity stiffness TT-operator and load TT on the QTT layout.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

On an axis-aligned box the Q1 / trilinear Galerkin form (Section 3, Eq. elassembly) separates
axis by axis, so every block A_{c c'} of the stiffness operator (test component c, trial
component c') is a short sum of Kronecker products of three 1D matrices per axis:

  K[i,j] = int phi_i' phi_j',  M[i,j] = int phi_i phi_j,  G[i,j] = int phi_i phi_j'

Writing sigma(N_b e_c'):eps(N_a e_c) = lam d_c N_a d_c' N_b + mu delta_cc' grad N_a.grad N_b
+ mu d_c' N_a d_c N_b with N_a = prod_d phi_{a_d}(x_d), each product of derivatives integrates
to a product over axes of K (derivative on both), G^T (derivative on the test function only),
G (trial only) or M (neither).  This is the tensorised counterpart of Algorithm 1's per-corner
element terms (Section 5.2), specialised to rectangles where the Jacobian is constant
(Section 5.1: J and det J are then exact rank-1 tensors and no TT-cross is needed).

Each 1D matrix is assembled by a 1D element loop (element weights carry the piecewise constant
Young's modulus along x) and converted to QTT by TT-SVD; the D-dimensional level cores are the
interleaved Kronecker products (``oracle.tt.kron_levels``); the component core carries the
block index (Section 5.2: component core first, then level cores of mode 2^D).

Dirichlet faces: A_bc = P A P + s (I - P) with P = I_c (x) P_0 (x) ... (x) P_{D-1}, P_d the
diagonal projector that zeroes the clamped end nodes of axis d; s = mean over components of
A's diagonal at node (1,...,1).  The load is f_bc = P (M f0 + face tractions) (Section 5.3).
"""
from __future__ import annotations

import math
from typing import List, Sequence

import numpy as np

from paper_2501_12151_gb300.workloads import Grid, Material, Load
from . import tt


def lame(E: float, nu: float, dim: int, plane_stress: bool):
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = E / (2.0 * (1.0 + nu))
    if dim == 2 and plane_stress:
        lam = 2.0 * lam * mu / (lam + 2.0 * mu)
    return lam, mu


def matrices_1d(n: int, lo: float, hi: float, weights: np.ndarray = None):
    """Dense 1D K, M, G on n equidistant nodes by an element loop with element weights."""
    h = (hi - lo) / (n - 1)
    w = np.ones(n - 1) if weights is None else weights
    K = np.zeros((n, n))
    M = np.zeros((n, n))
    G = np.zeros((n, n))
    for e in range(n - 1):
        idx = [e, e + 1]
        Ke = w[e] / h * np.array([[1.0, -1.0], [-1.0, 1.0]])
        Me = w[e] * h / 6.0 * np.array([[2.0, 1.0], [1.0, 2.0]])
        # test i (row) without derivative, trial j (column) with derivative:
        # int phi_i phi_j' = (h/2) * (-1/h or +1/h)
        Ge = w[e] * np.array([[-0.5, 0.5], [-0.5, 0.5]])
        for a in range(2):
            for b in range(2):
                K[idx[a], idx[b]] += Ke[a, b]
                M[idx[a], idx[b]] += Me[a, b]
                G[idx[a], idx[b]] += Ge[a, b]
    return K, M, G


def axis_projector(n: int, clamp_lo: bool, clamp_hi: bool) -> np.ndarray:
    p = np.ones(n)
    if clamp_lo:
        p[0] = 0.0
    if clamp_hi:
        p[-1] = 0.0
    return np.diag(p)


def block_terms(dim: int, c: int, c2: int, lam: float, mu: float):
    """Kronecker terms of block (test c, trial c'): list of (coef, [op name per axis])."""
    terms = []
    # lam d_c N_a d_c' N_b
    ops = []
    for d in range(dim):
        if d == c and d == c2:
            ops.append("K")
        elif d == c:
            ops.append("GT")
        elif d == c2:
            ops.append("G")
        else:
            ops.append("M")
    terms.append((lam, ops))
    # mu d_c' N_a d_c N_b
    ops = []
    for d in range(dim):
        if d == c and d == c2:
            ops.append("K")
        elif d == c2:
            ops.append("GT")
        elif d == c:
            ops.append("G")
        else:
            ops.append("M")
    terms.append((mu, ops))
    # mu delta_cc' grad N_a . grad N_b
    if c == c2:
        for e in range(dim):
            terms.append((mu, ["K" if d == e else "M" for d in range(dim)]))
    return terms


def stiffness_mpo(grid: Grid, mat: Material, eps: float = 1e-13, with_bc: bool = True):
    """Boundary-condition-applied stiffness TT-operator on the QTT layout, and the shift s."""
    D, L, n = grid.dim, grid.levels, grid.n
    # element weights along x carry E(x)/E[0]
    xs = grid.lo[0] + (grid.hi[0] - grid.lo[0]) * np.arange(n) / (n - 1)
    cx = 0.5 * (xs[:-1] + xs[1:])
    wx = np.where(cx < mat.split_x, mat.E[0], mat.E[1]) / mat.E[0]
    lam, mu = lame(mat.E[0], mat.nu, D, grid.plane_stress)
    dense = []
    for d in range(D):
        K, M, G = matrices_1d(n, grid.lo[d], grid.hi[d], wx if d == 0 else None)
        P = axis_projector(n, grid.clamped[2 * d] and with_bc, grid.clamped[2 * d + 1] and with_bc)
        dense.append({"K": K, "M": M, "G": G, "GT": G.T.copy(), "P": P, "I": np.eye(n)})
    # shift s from the unconstrained diagonal at node (1,...,1)
    s = 0.0
    for c in range(D):
        for coef, ops in block_terms(D, c, c, lam, mu):
            s += coef * np.prod([dense[d][ops[d]][1, 1] for d in range(D)])
    s /= D
    modes2 = [2] * L
    qtt_cache = {}

    def q1d(d, name):
        key = (d, name)
        if key not in qtt_cache:
            X = dense[d][name]
            if with_bc and name in ("K", "M", "G", "GT"):
                X = dense[d]["P"] @ X @ dense[d]["P"]
            qtt_cache[key] = tt.mpo_from_dense(X, modes2, eps=1e-15)
        return qtt_cache[key]

    total = None
    for c in range(D):
        for c2 in range(D):
            E = np.zeros((1, D, D, 1))
            E[0, c, c2, 0] = 1.0
            for coef, ops in block_terms(D, c, c2, lam, mu):
                lev = tt.kron_levels([q1d(d, ops[d]) for d in range(D)])
                term = [E * coef] + lev
                total = term if total is None else tt.mpo_round(tt.mpo_add(total, term), eps)
    if with_bc and any(grid.clamped[: 2 * D]):
        Ic = np.eye(D).reshape(1, D, D, 1)
        ones = [Ic * s] + tt.kron_levels([q1d(d, "I") for d in range(D)])
        proj = [Ic * (-s)] + tt.kron_levels([q1d(d, "P") for d in range(D)])
        total = tt.mpo_round(tt.mpo_add(total, ones), eps)
        total = tt.mpo_round(tt.mpo_add(total, proj), eps)
    return total, s


def mass_mpo(grid: Grid):
    """Unconstrained mass TT-operator I_c (x) M_0 (x) ... (x) M_{D-1}."""
    D, L, n = grid.dim, grid.levels, grid.n
    ops = []
    for d in range(D):
        _, M, _ = matrices_1d(n, grid.lo[d], grid.hi[d])
        ops.append(tt.mpo_from_dense(M, [2] * L, eps=1e-15))
    return [np.eye(D).reshape(1, D, D, 1)] + tt.kron_levels(ops)


def load_tt_dense(f_natural: np.ndarray, grid: Grid, eps: float = 1e-14) -> List[np.ndarray]:
    """TT-SVD of a dense load vector given in natural order (for sizes that fit in memory)."""
    v = tt.to_qtt_order(f_natural, grid.dim, grid.levels)
    return tt.tt_svd(v, [grid.dim] + [1 << grid.dim] * grid.levels, eps)
