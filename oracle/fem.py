"""Oracle A: sparse Q1 / trilinear FEM for isotropic linear elasticity, FP64, CPU.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

What it computes, and where the paper defines it:

* Constitutive law sigma = lambda tr(eps) I + 2 mu eps and the equilibrium equation
  (Section 2, Eq. linelastic / diffeq).  The paper prints ``div sigma = f``; with the weak form
  a(u,v) = L(v) = int f.v and gravity f = (0, -rho g) this is read as ``-div sigma = f``.
* Plane strain Lame parameters, or the plane-stress "modified Lame parameters" of Section 2:
  lambda* = 2 lambda mu / (lambda + 2 mu).
* Galerkin system A u = f with A_ij = a(phi_j, phi_i) (Section 3, Eq. femsys), assembled element
  by element through the map from the reference element Q = [-1,1]^D with |det J| and the
  chain rule grad phi = J^{-T} grad_xi phi (Eq. elassembly, Eq. grads), 2-point Gauss rules per
  axis (exact for the bilinear/trilinear integrands on parallelepipeds).
* Grid: 2**levels equidistant nodes per axis including the boundary, (2**levels - 1)**D
  elements, D * 2**(D*levels) unknowns (Section 5).  The domain is a box, or the affine image of
  the unit box (a parallelogram / parallelepiped, grid.edges): node i at lo + sum_d i_d/(n-1)
  edges[d], every element the same parallelogram, the quadrature and the chain rule unchanged
  (Section 5.1: J constant per element, exact for such maps).  Or a general convex
  quadrilateral (2D, grid.quad: corners P0..P3, the bilinear map of the unit square): node
  (i, j) at the bilinear map of (i/(n-1), j/(n-1)); assembled either exactly (J at every
  quadrature point) or, as Algorithm 1 does, with each element's J and det J frozen at the
  element centre xi = 0 (``frozen_jacobian``).
* Load f = M f0 from nodal values f0 (Section 5.3); a traction t on a face enters the same way
  through the face mass matrix (the paper only names Neumann sides).
* Dirichlet faces: symmetric elimination A_bc = P A P + s (I - P), f_bc = P f, where P keeps the
  free unknowns and s is the mean over components of A's diagonal at grid node (1,...,1).  The
  solution does not depend on s (clamped unknowns solve to exactly zero).

Node ordering here is the natural one: unknown (c, i_0, ..., i_{D-1}) sits at
c * n**D + ravel(i_0, ..., i_{D-1}) with the x index most significant.  The QTT ordering of
Section 4 is a permutation of this (see ``oracle.tt.qtt_perm``).
"""
from __future__ import annotations

import itertools
import math
from typing import Dict, List, Sequence, Tuple

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from paper_2501_12151_gb300.workloads import Grid, Material, Load


# ---------------------------------------------------------------------------------------
# material
# ---------------------------------------------------------------------------------------

def lame(E: float, nu: float, dim: int, plane_stress: bool) -> Tuple[float, float]:
    """Lame parameters (Section 2); plane stress uses the modified lambda*."""
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = E / (2.0 * (1.0 + nu))
    if dim == 2 and plane_stress:
        lam = 2.0 * lam * mu / (lam + 2.0 * mu)
    return lam, mu


# ---------------------------------------------------------------------------------------
# reference element (Section 3)
# ---------------------------------------------------------------------------------------

def ref_corners(dim: int) -> np.ndarray:
    """Corner a of Q has bit pattern b (a = sum_d b_d 2^(dim-1-d)); xi_a = 2b - 1."""
    b = np.array(list(itertools.product((0, 1), repeat=dim)), dtype=np.int64)
    return b


def shape(dim: int, xi: np.ndarray):
    """Values N_a(xi) and reference gradients dN_a/dxi_e of the Q1 basis at one point."""
    b = ref_corners(dim)
    s = 2.0 * b - 1.0                       # (2^D, D)
    fac = 0.5 * (1.0 + s * xi[None, :])     # (2^D, D)
    N = np.prod(fac, axis=1)
    dN = np.zeros((1 << dim, dim))
    for e in range(dim):
        other = np.prod(np.delete(fac, e, axis=1), axis=1) if dim > 1 else np.ones(1 << dim)
        dN[:, e] = 0.5 * s[:, e] * other
    return N, dN


def gauss(dim: int):
    g = 1.0 / math.sqrt(3.0)
    pts = np.array(list(itertools.product((-g, g), repeat=dim)))
    w = np.ones(len(pts))
    return pts, w


def element_matrices(X: np.ndarray, lam: float, mu: float, frozen: bool = False):
    """Element stiffness and mass for corner coordinates X (2^D, D) (Eq. elassembly).

    Local unknown (a, c) sits at a*D + c.  Stiffness entry for test (a,c), trial (b,c'):
      int lam d_c N_a d_c' N_b + mu delta_cc' grad N_a . grad N_b + mu d_c' N_a d_c N_b
    which is sigma(N_b e_c') : eps(N_a e_c) written out.  With `frozen` the Jacobian is taken at
    the element centre xi = 0 for every quadrature point, as Algorithm 1 does (exact for
    parallelograms, an approximation on general quadrilaterals).
    """
    dim = X.shape[1]
    nb = 1 << dim
    K = np.zeros((nb * dim, nb * dim))
    M = np.zeros((nb * dim, nb * dim))
    pts, w = gauss(dim)
    J0 = X.T @ shape(dim, np.zeros(dim))[1]
    for q in range(len(pts)):
        N, dN = shape(dim, pts[q])
        J = J0 if frozen else X.T @ dN         # J[d, e] = dx_d / dxi_e
        detJ = np.linalg.det(J)
        G = dN @ np.linalg.inv(J)              # rows: grad_x N_a = J^{-T} grad_xi N_a
        wq = w[q] * abs(detJ)
        for a in range(nb):
            for bb in range(nb):
                gg = G[a] @ G[bb]
                nn = N[a] * N[bb]
                for c in range(dim):
                    for c2 in range(dim):
                        v = lam * G[a, c] * G[bb, c2] + mu * G[a, c2] * G[bb, c]
                        if c == c2:
                            v += mu * gg
                            M[a * dim + c, bb * dim + c2] += wq * nn
                        K[a * dim + c, bb * dim + c2] += wq * v
    return K, M


def facet_mass(X: np.ndarray, dim: int):
    """Mass matrix of a (dim-1)-dimensional facet with corner coordinates X (2^(dim-1), dim).

    Local unknown (a, c) at a*dim + c; entry delta_cc' int N_a N_b dS.
    """
    fd = dim - 1
    nb = 1 << fd
    Mf = np.zeros((nb * dim, nb * dim))
    pts, w = gauss(fd)
    for q in range(len(pts)):
        N, dN = shape(fd, pts[q])
        T = X.T @ dN                            # tangent vectors (dim, fd)
        dS = math.sqrt(abs(np.linalg.det(T.T @ T)))
        for a in range(nb):
            for bb in range(nb):
                for c in range(dim):
                    Mf[a * dim + c, bb * dim + c] += w[q] * dS * N[a] * N[bb]
    return Mf


# ---------------------------------------------------------------------------------------
# grid helpers
# ---------------------------------------------------------------------------------------

def axis_coords(grid: Grid) -> List[np.ndarray]:
    n = grid.n
    return [grid.lo[d] + (grid.hi[d] - grid.lo[d]) * np.arange(n) / (n - 1) for d in range(grid.dim)]


def node_lin(idx: Sequence[np.ndarray], n: int) -> np.ndarray:
    lin = np.zeros_like(np.asarray(idx[0]), dtype=np.int64)
    for a in idx:
        lin = lin * n + np.asarray(a, dtype=np.int64)
    return lin


def node_coords(grid: Grid, idx: Sequence[np.ndarray]) -> np.ndarray:
    """Physical coordinates (len, D) of the nodes with per-axis indices idx[d].  On a box the node
    sits at lo + i h per axis; on a parallelogram / parallelepiped (grid.edges) at
    lo + sum_d i_d / (n - 1) edges[d]."""
    D = grid.dim
    idx = [np.asarray(i).ravel() for i in idx]
    if getattr(grid, "quad", None) is not None:
        # bilinear map of the unit square onto the quadrilateral P0 P1 P2 P3 (Section 5.1)
        P = np.asarray(grid.quad, dtype=float)
        xi, eta = idx[0] / (grid.n - 1), idx[1] / (grid.n - 1)
        return (np.outer((1 - xi) * (1 - eta), P[0]) + np.outer(xi * (1 - eta), P[1]) +
                np.outer((1 - xi) * eta, P[2]) + np.outer(xi * eta, P[3]))
    if grid.edges is None:
        ax = axis_coords(grid)
        return np.stack([ax[d][idx[d]] for d in range(D)], axis=1)
    E = np.asarray(grid.edges, dtype=float)[:D, :D]
    xi = np.stack([i / (grid.n - 1) for i in idx], axis=1)
    return np.asarray(grid.lo[:D], dtype=float)[None, :] + xi @ E


def nodal_points(grid: Grid) -> np.ndarray:
    """Coordinates of all nodes in natural order, shape (n**D, D)."""
    idx = np.meshgrid(*[np.arange(grid.n)] * grid.dim, indexing="ij")
    return node_coords(grid, [m.ravel() for m in idx])


def constrained_nodes(grid: Grid) -> np.ndarray:
    """Boolean mask over nodes lying on a clamped face."""
    n = grid.n
    idx = np.meshgrid(*[np.arange(n)] * grid.dim, indexing="ij")
    mask = np.zeros(idx[0].shape, dtype=bool)
    for f in range(2 * grid.dim):
        if grid.clamped[f]:
            d, side = divmod(f, 2)
            mask |= idx[d] == (0 if side == 0 else n - 1)
    return mask.ravel()


# ---------------------------------------------------------------------------------------
# assembly (element loop, Section 3)
# ---------------------------------------------------------------------------------------

def assemble(grid: Grid, mat: Material, frozen_jacobian: bool = False):
    """Free-free stiffness A and mass M (CSR, natural ordering) by an element loop.

    Element matrices are computed per element from its corner coordinates; identical
    elements (same geometry and Young's modulus) reuse one computed matrix.  `frozen_jacobian`
    takes each element's Jacobian at its centre (Algorithm 1's assembly for general
    quadrilaterals).
    """
    D, n = grid.dim, grid.n
    N = n ** D
    ndof = D * N
    corners = ref_corners(D)
    ne = n - 1
    el = np.meshgrid(*[np.arange(ne)] * D, indexing="ij")
    el = [e.ravel() for e in el]
    n_el = len(el[0])
    # element corner coordinates relative to the element's first corner, and its centroid
    Xc = [node_coords(grid, [el[d] + corners[a, d] for d in range(D)]) for a in range(1 << D)]
    rel = np.stack([Xc[a] - Xc[0] for a in range(1 << D)], axis=1)      # (n_el, 2^D, D)
    cx = np.mean([Xc[a][:, 0] for a in range(1 << D)], axis=0)
    Es = np.where(cx < mat.split_x, mat.E[0], mat.E[1])
    geo = np.concatenate([np.round(rel.reshape(n_el, -1), 15), Es[:, None]], axis=1)
    uniq, inv = np.unique(geo, axis=0, return_inverse=True)
    inv = inv.ravel()
    Ks, Ms = [], []
    for u in uniq:
        X = u[:-1].reshape(1 << D, D)
        lam, mu = lame(u[-1], mat.nu, D, grid.plane_stress)
        K, M = element_matrices(X, lam, mu, frozen_jacobian)
        Ks.append(K)
        Ms.append(M)
    Ks = np.array(Ks)
    Ms = np.array(Ms)
    nb = 1 << D
    node_of = [node_lin([el[d] + corners[a, d] for d in range(D)], n) for a in range(nb)]
    rows, cols, kv, mv = [], [], [], []
    for a in range(nb):
        for c in range(D):
            r = c * N + node_of[a]
            for b in range(nb):
                for c2 in range(D):
                    col = c2 * N + node_of[b]
                    rows.append(r)
                    cols.append(col)
                    kv.append(Ks[inv, a * D + c, b * D + c2])
                    mv.append(Ms[inv, a * D + c, b * D + c2])
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    A = sp.csr_matrix((np.concatenate(kv), (rows, cols)), shape=(ndof, ndof))
    M = sp.csr_matrix((np.concatenate(mv), (rows, cols)), shape=(ndof, ndof))
    A.sum_duplicates()
    M.sum_duplicates()
    return A, M


def face_mass(grid: Grid, face: int) -> sp.csr_matrix:
    """Face mass matrix (natural ordering) of face ``face`` by a facet loop."""
    D, n = grid.dim, grid.n
    N = n ** D
    d, side = divmod(face, 2)
    fixed = 0 if side == 0 else n - 1
    tang = [e for e in range(D) if e != d]
    fc = ref_corners(D - 1)
    ne = n - 1
    el = np.meshgrid(*[np.arange(ne)] * (D - 1), indexing="ij")
    el = [e.ravel() for e in el]
    nb = 1 << (D - 1)
    rows, cols, vals = [], [], []
    # vectorised over facets with per-facet geometry
    Xs = np.zeros((len(el[0]), nb, D))
    node_idx = []
    for a in range(nb):
        full = [None] * D
        full[d] = np.full(len(el[0]), fixed)
        for t, e in enumerate(tang):
            full[e] = el[t] + fc[a, t]
        node_idx.append(node_lin(full, n))
        Xs[:, a, :] = node_coords(grid, full)
    # group identical facet geometry
    rel = np.round(Xs - Xs[:, :1, :], 15).reshape(len(el[0]), -1)
    uniq, inv = np.unique(rel, axis=0, return_inverse=True)
    inv = inv.ravel()
    mats = np.array([facet_mass(u.reshape(nb, D), D) for u in uniq])
    for a in range(nb):
        for b in range(nb):
            for c in range(D):
                rows.append(c * N + node_idx[a])
                cols.append(c * N + node_idx[b])
                vals.append(mats[inv, a * D + c, b * D + c])
    Mf = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                       shape=(D * N, D * N))
    Mf.sum_duplicates()
    return Mf


# ---------------------------------------------------------------------------------------
# manufactured field (2D, unit square)
# ---------------------------------------------------------------------------------------

def manufactured_u(x, y):
    """u* = (sin(pi x) sin(pi y), x(1-x) y(1-y))."""
    return np.sin(np.pi * x) * np.sin(np.pi * y), x * (1 - x) * y * (1 - y)


def manufactured_grad(x, y):
    """Gradient of u*: returns g[c][e] = d u*_c / d x_e."""
    p = np.pi
    u1x = p * np.cos(p * x) * np.sin(p * y)
    u1y = p * np.sin(p * x) * np.cos(p * y)
    u2x = (1 - 2 * x) * y * (1 - y)
    u2y = x * (1 - x) * (1 - 2 * y)
    return [[u1x, u1y], [u2x, u2y]]


def manufactured_stress(x, y, lam, mu):
    g = manufactured_grad(x, y)
    div = g[0][0] + g[1][1]
    sxx = lam * div + 2 * mu * g[0][0]
    syy = lam * div + 2 * mu * g[1][1]
    sxy = mu * (g[0][1] + g[1][0])
    return sxx, syy, sxy


def manufactured_force(x, y, lam, mu):
    """f = -div sigma(u*), written out from the second derivatives of u*."""
    p = np.pi
    u1xx = -p * p * np.sin(p * x) * np.sin(p * y)
    u1yy = u1xx
    u1xy = p * p * np.cos(p * x) * np.cos(p * y)
    u2xx = -2 * y * (1 - y)
    u2yy = -2 * x * (1 - x)
    u2xy = (1 - 2 * x) * (1 - 2 * y)
    f1 = -((lam + 2 * mu) * u1xx + mu * u1yy + (lam + mu) * u2xy)
    f2 = -(mu * u2xx + (lam + 2 * mu) * u2yy + (lam + mu) * u1xy)
    return f1, f2


# ---------------------------------------------------------------------------------------
# loads (Section 5.3)
# ---------------------------------------------------------------------------------------

def nodal_body_force(grid: Grid, mat: Material, load: Load) -> np.ndarray:
    """Nodal values f0 (natural ordering, component-major) of a body-force load."""
    D = grid.dim
    P = nodal_points(grid)
    N = P.shape[0]
    f0 = np.zeros((D, N))
    if load.kind == "gravity":
        f0[D - 1, :] = -load.rho * load.g
    elif load.kind == "fourier":
        for m in range(load.wave.shape[0]):
            arg = np.pi * (P @ load.wave[m].astype(float)) + load.phase[m]
            s = np.sin(arg)
            for c in range(D):
                f0[c] += load.scale * load.amp[c, m] * s
    elif load.kind == "manufactured":
        lam, mu = lame(mat.E[0], mat.nu, D, grid.plane_stress)
        f1, f2 = manufactured_force(P[:, 0], P[:, 1], lam, mu)
        f0[0], f0[1] = f1, f2
    elif load.kind == "nodal":
        f0[:] = np.asarray(load.values, dtype=float).reshape(D, N)   # given nodal values (Section 5.3)
    return f0.ravel()


def nodal_traction(grid: Grid, mat: Material, load: Load, face: int) -> np.ndarray:
    """Nodal traction values on a face (defined on all nodes; the face mass selects the face)."""
    D = grid.dim
    P = nodal_points(grid)
    N = P.shape[0]
    t0 = np.zeros((D, N))
    if load.kind == "traction":
        for c in range(D):
            t0[c, :] = load.traction[c]
    elif load.kind == "manufactured":
        lam, mu = lame(mat.E[0], mat.nu, D, grid.plane_stress)
        sxx, syy, sxy = manufactured_stress(P[:, 0], P[:, 1], lam, mu)
        nvec = np.zeros(D)
        d, side = divmod(face, 2)
        nvec[d] = -1.0 if side == 0 else 1.0
        t0[0] = sxx * nvec[0] + sxy * nvec[1]
        t0[1] = sxy * nvec[0] + syy * nvec[1]
    return t0.ravel()


def load_vector(grid: Grid, mat: Material, loads: Sequence[Load], M=None) -> np.ndarray:
    """f = M f0 plus face-mass tractions, before boundary conditions."""
    if M is None:
        _, M = assemble(grid, mat)
    f = np.zeros(M.shape[0])
    for ld in loads:
        if ld.kind in ("gravity", "fourier", "manufactured", "nodal"):
            f += M @ nodal_body_force(grid, mat, ld)
        if ld.kind == "traction":
            f += face_mass(grid, ld.face) @ nodal_traction(grid, mat, ld, ld.face)
        if ld.kind == "manufactured":
            for face in range(2 * grid.dim):
                if not grid.clamped[face]:
                    f += face_mass(grid, face) @ nodal_traction(grid, mat, ld, face)
    return f


# ---------------------------------------------------------------------------------------
# boundary conditions and solve
# ---------------------------------------------------------------------------------------

def bc_shift(grid: Grid, A: sp.csr_matrix) -> float:
    """s = mean over components of A's diagonal at grid node (1, ..., 1)."""
    D, n = grid.dim, grid.n
    N = n ** D
    node = node_lin([np.array(1 if n > 1 else 0)] * D, n)
    return float(np.mean([A[c * N + node, c * N + node] for c in range(D)]))


def apply_bc(grid: Grid, A: sp.csr_matrix, f: np.ndarray = None):
    """A_bc = P A P + s (I - P), f_bc = P f (symmetric elimination of clamped unknowns)."""
    D = grid.dim
    cn = constrained_nodes(grid)
    free = np.tile(~cn, D).astype(float)
    P = sp.diags(free)
    s = bc_shift(grid, A)
    Abc = (P @ A @ P + s * sp.diags(1.0 - free)).tocsr()
    Abc.eliminate_zeros()
    if f is None:
        return Abc
    return Abc, free * f


def system(grid: Grid, mat: Material, loads: Sequence[Load], frozen_jacobian: bool = False):
    """Boundary-condition-applied Galerkin system (A_bc, f_bc) in natural ordering."""
    A, M = assemble(grid, mat, frozen_jacobian)
    f = load_vector(grid, mat, loads, M)
    return apply_bc(grid, A, f)


def solve(A: sp.csr_matrix, f: np.ndarray, rtol: float = 1e-13, direct_max: int = 300_000):
    """u_h = A^{-1} f: sparse direct solve for small systems, Jacobi-preconditioned CG above."""
    if A.shape[0] <= direct_max:
        return spla.spsolve(A.tocsc(), f)
    d = A.diagonal()
    Minv = sp.diags(1.0 / d)
    u, info = spla.cg(A, f, rtol=rtol, atol=0.0, M=Minv, maxiter=200_000)
    if info != 0:
        raise RuntimeError(f"CG did not converge (info={info})")
    return u


def energy_norm(A: sp.csr_matrix, v: np.ndarray) -> float:
    return float(math.sqrt(max(v @ (A @ v), 0.0)))


# ---------------------------------------------------------------------------------------
# u_h at large sizes: conjugate gradients preconditioned by a geometric multigrid V-cycle
# ---------------------------------------------------------------------------------------
#
# The result is still the definition above, u_h = A^{-1} f (Section 3, Eq. femsys); the
# V-cycle only changes how fast CG gets there.  It is a textbook construction: linear
# interpolation between uniform grids of 2^l and 2^(l-1) nodes per axis (the grids are not
# nested: an odd number of intervals cannot be halved), Galerkin coarse operators P^T A P,
# Chebyshev smoothing on D^{-1} A (the same polynomial before and after the coarse correction,
# so the cycle is a symmetric operator), a sparse direct solve on the coarsest grid.

def interpolation_1d(n_fine: int, n_coarse: int) -> sp.csr_matrix:
    """Linear interpolation from n_coarse to n_fine equidistant nodes of the same interval."""
    t = np.arange(n_fine) * (n_coarse - 1) / (n_fine - 1)   # fine nodes in coarse index units
    j = np.minimum(np.floor(t).astype(np.int64), n_coarse - 2)
    w = t - j
    rows = np.concatenate([np.arange(n_fine), np.arange(n_fine)])
    cols = np.concatenate([j, j + 1])
    vals = np.concatenate([1.0 - w, w])
    P = sp.csr_matrix((vals, (rows, cols)), shape=(n_fine, n_coarse))
    P.eliminate_zeros()
    return P


def vector_interpolation(dim: int, n_fine: int, n_coarse: int) -> sp.csr_matrix:
    """I_D (x) P_1D (x) ... (x) P_1D in the natural ordering (component, then x, y[, z])."""
    P1 = interpolation_1d(n_fine, n_coarse)
    P = P1
    for _ in range(dim - 1):
        P = sp.kron(P, P1, format="csr")
    return sp.kron(sp.identity(dim, format="csr"), P, format="csr")


class MultigridV:
    """Symmetric V-cycle for the BC-applied elasticity matrix on a 2^levels tensor grid."""

    def __init__(self, dim: int, levels: int, A: sp.csr_matrix, coarsest_levels: int = 4, degree: int = 3):
        self.degree = degree
        self.As, self.Ps, self.dinv, self.lmax = [A.tocsr()], [], [], []
        l = levels
        while l > coarsest_levels:
            P = vector_interpolation(dim, 1 << l, 1 << (l - 1))
            self.Ps.append(P)
            self.As.append((P.T @ self.As[-1] @ P).tocsr())
            l -= 1
        for Al in self.As[:-1]:
            d = 1.0 / Al.diagonal()
            self.dinv.append(d)
            self.lmax.append(1.1 * self._power_max(Al, d))
        self.coarse = spla.splu(self.As[-1].tocsc())

    @staticmethod
    def _power_max(A, dinv, iters: int = 30) -> float:
        """Largest eigenvalue of D^{-1} A by power iteration (seeded start)."""
        v = np.random.Generator(np.random.Philox(key=17)).standard_normal(A.shape[0])
        lam = 0.0
        for _ in range(iters):
            w = dinv * (A @ v)
            lam = float(np.linalg.norm(w) / np.linalg.norm(v))
            v = w / np.linalg.norm(w)
        return lam

    def _smooth(self, l: int, x: np.ndarray, b: np.ndarray) -> np.ndarray:
        """Chebyshev iteration of the given degree on D^{-1} A over [lmax/30, lmax]."""
        A, dinv, hi = self.As[l], self.dinv[l], self.lmax[l]
        lo = hi / 30.0
        theta, delta = 0.5 * (hi + lo), 0.5 * (hi - lo)
        sigma = theta / delta
        rho = 1.0 / sigma
        r = dinv * (b - A @ x)
        d = r / theta
        for _ in range(self.degree):
            x = x + d
            r = r - dinv * (A @ d)
            rho_new = 1.0 / (2.0 * sigma - rho)
            d = rho_new * rho * d + 2.0 * rho_new / delta * r
            rho = rho_new
        return x

    def cycle(self, b: np.ndarray, l: int = 0) -> np.ndarray:
        if l == len(self.As) - 1:
            return self.coarse.solve(b)
        A, P = self.As[l], self.Ps[l]
        x = self._smooth(l, np.zeros_like(b), b)
        x = x + P @ self.cycle(P.T @ (b - A @ x), l + 1)
        return self._smooth(l, x, b)


def solve_mg(grid: Grid, A: sp.csr_matrix, f: np.ndarray, rtol: float = 1e-14, maxit: int = 500):
    """u_h = A^{-1} f by V-cycle preconditioned CG, for grids too large for a direct solve.

    Stops when the preconditioned residual r^T M r has fallen by rtol^2 (the recursive 2-norm
    residual can stall near eps * cond(A) before the error does).  Returns (u_h, info) with the
    iteration count and the true relative residual ||f - A u|| / ||f||.
    """
    mg = MultigridV(grid.dim, grid.levels, A)
    x = np.zeros_like(f)
    r = f.copy()
    z = mg.cycle(r)
    p = z.copy()
    rz = float(r @ z)
    rz0 = rz
    it = 0
    while it < maxit and rz > rtol * rtol * rz0:
        Ap = A @ p
        alpha = rz / float(p @ Ap)
        x += alpha * p
        r -= alpha * Ap
        z = mg.cycle(r)
        rz_new = float(r @ z)
        p = z + (rz_new / rz) * p
        rz = rz_new
        it += 1
    res = float(np.linalg.norm(f - A @ x) / np.linalg.norm(f))
    return x, {"iters": it, "rel_residual": res, "converged": rz <= rtol * rtol * rz0}


def manufactured_errors(grid: Grid, mat: Material, u: np.ndarray):
    """L2 and energy errors of u_h against u* (2D), by 2x2 Gauss quadrature per element.

    Returns (||u* - u_h||_L2, ||u* - u_h||_a) with a(v,v) = int lam (div v)^2 + 2 mu eps:eps.
    """
    assert grid.dim == 2
    n = grid.n
    N = n * n
    lam, mu = lame(mat.E[0], mat.nu, 2, grid.plane_stress)
    ax = axis_coords(grid)
    hx, hy = ax[0][1] - ax[0][0], ax[1][1] - ax[1][0]
    U = u.reshape(2, n, n)
    pts, w = gauss(2)
    l2 = 0.0
    en = 0.0
    ei, ej = np.meshgrid(np.arange(n - 1), np.arange(n - 1), indexing="ij")
    ei, ej = ei.ravel(), ej.ravel()
    corners = ref_corners(2)
    for q in range(len(pts)):
        Nq, dN = shape(2, pts[q])
        G = dN / np.array([hx / 2, hy / 2])[None, :]
        x = ax[0][ei] + 0.5 * hx * (1 + pts[q][0])
        y = ax[1][ej] + 0.5 * hy * (1 + pts[q][1])
        uh = np.zeros((2, len(ei)))
        gh = np.zeros((2, 2, len(ei)))
        for a in range(4):
            vals = U[:, ei + corners[a, 0], ej + corners[a, 1]]
            uh += Nq[a] * vals
            for e in range(2):
                gh[:, e] += G[a, e] * vals
        us = manufactured_u(x, y)
        gs = manufactured_grad(x, y)
        wq = w[q] * hx * hy / 4.0
        for c in range(2):
            l2 += wq * np.sum((us[c] - uh[c]) ** 2)
        ge = [[gs[c][e] - gh[c, e] for e in range(2)] for c in range(2)]
        div = ge[0][0] + ge[1][1]
        exy = 0.5 * (ge[0][1] + ge[1][0])
        epsd = ge[0][0] ** 2 + ge[1][1] ** 2 + 2 * exy ** 2
        en += wq * np.sum(lam * div ** 2 + 2 * mu * epsd)
    return math.sqrt(l2), math.sqrt(en)
