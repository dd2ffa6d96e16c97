"""Oracle B, part 1: a plain CPU tensor-train toolkit in FP64 (numpy).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

* Tensor trains / MPS and TT-operators / MPO (Section 4, Fig. TTdec): a vector core has shape
  ``[r_{k-1}, n_k, r_k]``, an operator core ``[a_{k-1}, n_k (row), n_k (column), a_k]``.
* QTT index (Section 4): a grid index i in {0..2^L-1} is split into bits, most significant
  first, i = sum_k i_k 2^(L-1-k).  The paper's layout for the elasticity unknowns (Section 5.2)
  puts the displacement component first (mode D) and then one core per level that carries the
  level's bit of every axis, merged as s = sum_d b_d 2^(D-1-d) (x bit most significant).
  ``qtt_perm`` maps this layout to the natural (component, x, y[, z]) ordering of ``oracle.fem``.
* TT-SVD and TT rounding with the Frobenius truncation rule of Oseledets (2011): drop the tail
  while its norm stays below delta ||T||, delta = eps / sqrt(d - 1).
* The reduced QR decomposition of Section 4 (Eq. qr) orthogonalises cores.

Every routine here is the textbook definition written out with numpy linear algebra
(``numpy.linalg.qr`` / ``svd``) as steps; nothing is blocked or fused.
"""
from __future__ import annotations

import math
from typing import List, Sequence

import numpy as np

Cores = List[np.ndarray]


# ---------------------------------------------------------------------------------------
# QTT index maps (Section 4, Section 5.2)
# ---------------------------------------------------------------------------------------

def qtt_perm(dim: int, levels: int) -> np.ndarray:
    """perm[q] = natural index of the unknown stored at QTT position q.

    q = ((c * 2^D + s_1) * 2^D + s_2) ... + s_L, s_k = sum_d bit_{k-1}(i_d) 2^(D-1-d),
    natural index = c * n^D + ravel(i_0, ..., i_{D-1}), n = 2^levels.
    """
    D, L = dim, levels
    n = 1 << L
    q = np.arange(D * (1 << (D * L)), dtype=np.int64)
    rest = q.copy()
    digits = []
    for _ in range(L):
        digits.append(rest % (1 << D))
        rest //= (1 << D)
    c = rest
    digits = digits[::-1]            # digits[k-1] = s_k
    idx = [np.zeros_like(q) for _ in range(D)]
    for k in range(L):
        s = digits[k]
        for d in range(D):
            bit = (s >> (D - 1 - d)) & 1
            idx[d] = idx[d] * 2 + bit
    lin = np.zeros_like(q)
    for d in range(D):
        lin = lin * n + idx[d]
    return c * (n ** D) + lin


def to_qtt_order(v_nat: np.ndarray, dim: int, levels: int) -> np.ndarray:
    return v_nat[qtt_perm(dim, levels)]


def to_natural_order(v_qtt: np.ndarray, dim: int, levels: int) -> np.ndarray:
    out = np.empty_like(v_qtt)
    out[qtt_perm(dim, levels)] = v_qtt
    return out


def matrix_to_qtt_order(A_nat, dim: int, levels: int) -> np.ndarray:
    """Dense matrix permuted to QTT order on rows and columns."""
    p = qtt_perm(dim, levels)
    A = A_nat.toarray() if hasattr(A_nat, "toarray") else np.asarray(A_nat)
    return A[np.ix_(p, p)]


# ---------------------------------------------------------------------------------------
# basic TT operations
# ---------------------------------------------------------------------------------------

def ranks(cores: Cores) -> List[int]:
    return [cores[0].shape[0]] + [c.shape[-1] for c in cores]


def modes(cores: Cores) -> List[int]:
    return [c.shape[1] for c in cores]


def tt_full(cores: Cores) -> np.ndarray:
    """Dense vector of a TT (first core's index most significant)."""
    t = cores[0].reshape(cores[0].shape[0] * cores[0].shape[1], cores[0].shape[2])
    for c in cores[1:]:
        t = t @ c.reshape(c.shape[0], -1)
        t = t.reshape(-1, c.shape[2])
    return t.reshape(-1)


def mpo_full(cores: Cores) -> np.ndarray:
    """Dense matrix of a TT-operator; row index = concatenated row modes."""
    d = len(cores)
    t = np.ones((1, 1, 1))          # (rows, cols, rank)
    for c in cores:
        a0, n, m, a1 = c.shape
        t = np.einsum("ija,abcd->ibjcd", t, c).reshape(t.shape[0] * n, t.shape[1] * m, a1)
    return t[:, :, 0]


def tt_svd(v: np.ndarray, mode_sizes: Sequence[int], eps: float = 1e-14, rmax: int = 1 << 30) -> Cores:
    """TT-SVD (Oseledets 2011, Algorithm 1) of a dense tensor given as a flat array."""
    d = len(mode_sizes)
    norm = np.linalg.norm(v)
    delta = eps / math.sqrt(max(d - 1, 1)) * norm
    cores = []
    C = np.asarray(v, dtype=float).reshape(1, -1)
    r = 1
    for k in range(d - 1):
        C = C.reshape(r * mode_sizes[k], -1)
        U, S, Vt = np.linalg.svd(C, full_matrices=False)
        rk = truncation_rank(S, delta, rmax)
        cores.append(U[:, :rk].reshape(r, mode_sizes[k], rk))
        C = S[:rk, None] * Vt[:rk]
        r = rk
    cores.append(C.reshape(r, mode_sizes[-1], 1))
    return cores


def truncation_rank(S: np.ndarray, delta: float, rmax: int) -> int:
    """Smallest rank whose discarded tail has Frobenius norm <= delta, capped at rmax.

    Singular values come sorted descending; on ties the lower index is kept first.
    """
    tail = np.sqrt(np.cumsum((S[::-1] ** 2)))[::-1]  # tail[i] = ||S[i:]||
    r = len(S)
    for i in range(len(S)):
        if tail[i] <= delta:
            r = i
            break
    return int(max(1, min(r, rmax)))


def mpo_from_dense(A: np.ndarray, mode_sizes: Sequence[int], eps: float = 1e-14,
                   rmax: int = 1 << 30) -> Cores:
    """TT-operator of a dense matrix by TT-SVD over merged (row_k, col_k) indices."""
    d = len(mode_sizes)
    shape = list(mode_sizes) + list(mode_sizes)
    T = A.reshape(shape)
    perm = []
    for k in range(d):
        perm += [k, d + k]
    T = T.transpose(perm).reshape(-1)
    merged = [n * n for n in mode_sizes]
    cores = tt_svd(T, merged, eps, rmax)
    return [c.reshape(c.shape[0], mode_sizes[k], mode_sizes[k], c.shape[2])
            for k, c in enumerate(cores)]


def tt_add(x: Cores, y: Cores, beta: float = 1.0) -> Cores:
    """x + beta*y by block-diagonal concatenation of cores (exact, ranks add)."""
    d = len(x)
    out = []
    for k in range(d):
        a, b = x[k], y[k]
        if k == 0:
            c = np.concatenate([a, beta * b], axis=-1)
        elif k == d - 1:
            c = np.concatenate([a, b], axis=0)
        else:
            sh = (a.shape[0] + b.shape[0],) + a.shape[1:-1] + (a.shape[-1] + b.shape[-1],)
            c = np.zeros(sh)
            c[: a.shape[0], ..., : a.shape[-1]] = a
            c[a.shape[0]:, ..., a.shape[-1]:] = b
        if d == 1:
            c = a + beta * b
        out.append(c)
    return out


def tt_dot(x: Cores, y: Cores) -> float:
    """<x, y> by left-to-right contraction of the Gram environments."""
    E = np.ones((1, 1))
    for a, b in zip(x, y):
        r0, n, r1 = b.shape
        T = (E @ b.reshape(r0, n * r1)).reshape(-1, r1)      # (i n), q
        E = a.reshape(-1, a.shape[2]).T @ T                  # p, q
    return float(E[0, 0])


def mpo_apply(A: Cores, x: Cores) -> Cores:
    """Exact TT-operator times TT: core[(a r), i, (a' r')] = sum_j A[a,i,j,a'] x[r,j,r']."""
    out = []
    for Ak, xk in zip(A, x):
        a0, n, _, a1 = Ak.shape
        r0, _, r1 = xk.shape
        c = np.einsum("aijb,rjs->aribs", Ak, xk)
        out.append(c.reshape(a0 * r0, n, a1 * r1))
    return out


def mpo_add(A: Cores, B: Cores, beta: float = 1.0) -> Cores:
    """A + beta*B for TT-operators (ranks add)."""
    xa = [c.reshape(c.shape[0], -1, c.shape[-1]) for c in A]
    xb = [c.reshape(c.shape[0], -1, c.shape[-1]) for c in B]
    s = tt_add(xa, xb, beta)
    return [c.reshape(c.shape[0], A[k].shape[1], A[k].shape[2], c.shape[-1]) for k, c in enumerate(s)]


# ---------------------------------------------------------------------------------------
# orthogonalisation and rounding (Section 4 Eq. qr; Oseledets 2011, Algorithm 2)
# ---------------------------------------------------------------------------------------

def orthogonalize_left(cores: Cores, upto: int = None) -> Cores:
    """Left-orthogonalise cores 0..upto-1 by reduced QR; the R factors move right."""
    x = [c.copy() for c in cores]
    d = len(x)
    upto = d - 1 if upto is None else upto
    for k in range(upto):
        r0, n, r1 = x[k].shape
        Q, R = np.linalg.qr(x[k].reshape(r0 * n, r1))
        x[k] = Q.reshape(r0, n, Q.shape[1])
        x[k + 1] = np.einsum("ab,bjc->ajc", R, x[k + 1])
    return x


def orthogonalize_right(cores: Cores, downto: int = 0) -> Cores:
    """Right-orthogonalise cores d-1..downto+1; the R factors move left."""
    x = [c.copy() for c in cores]
    d = len(x)
    for k in range(d - 1, downto, -1):
        r0, n, r1 = x[k].shape
        Q, R = np.linalg.qr(x[k].reshape(r0, n * r1).T)
        x[k] = Q.T.reshape(Q.shape[1], n, r1)
        x[k - 1] = np.einsum("ajb,cb->ajc", x[k - 1], R)
    return x


def tt_norm(cores: Cores) -> float:
    """||x|| from the last core after left orthogonalisation (no squared cancellation)."""
    x = orthogonalize_left(cores)
    return float(np.linalg.norm(x[-1]))


def tt_round(cores: Cores, eps: float = 1e-14, rmax: int = 1 << 30) -> Cores:
    """TT rounding: left-orthogonalise, then truncated SVDs right to left.

    The truncation threshold is delta = eps / sqrt(d-1) * ||x||, applied per bond.
    """
    d = len(cores)
    x = orthogonalize_left(cores)
    if d == 1:
        return x
    nrm = np.linalg.norm(x[-1])
    delta = eps / math.sqrt(d - 1) * nrm
    for k in range(d - 1, 0, -1):
        r0, n, r1 = x[k].shape
        U, S, Vt = np.linalg.svd(x[k].reshape(r0, n * r1), full_matrices=False)
        rk = truncation_rank(S, delta, rmax)
        x[k] = Vt[:rk].reshape(rk, n, r1)
        x[k - 1] = np.einsum("ajb,bc->ajc", x[k - 1], U[:, :rk] * S[:rk])
    return x


def mpo_round(cores: Cores, eps: float = 1e-14, rmax: int = 1 << 30) -> Cores:
    flat = [c.reshape(c.shape[0], -1, c.shape[-1]) for c in cores]
    r = tt_round(flat, eps, rmax)
    return [c.reshape(c.shape[0], cores[k].shape[1], cores[k].shape[2], c.shape[-1])
            for k, c in enumerate(r)]


# ---------------------------------------------------------------------------------------
# Kronecker structure on the QTT layout
# ---------------------------------------------------------------------------------------

def kron_levels(axis_ops: Sequence[Cores]) -> Cores:
    """Interleave per-axis 1D QTT operators (each ``levels`` cores [a,2,2,a']) into level
    cores with merged mode s = sum_d b_d 2^(D-1-d) (x bit most significant)."""
    D = len(axis_ops)
    L = len(axis_ops[0])
    out = []
    for k in range(L):
        c = axis_ops[0][k]
        for d in range(1, D):
            e = axis_ops[d][k]
            a0, n, m, a1 = c.shape
            b0, p, q, b1 = e.shape
            c = np.einsum("aijb,ckld->acikjlbd", c, e).reshape(a0 * b0, n * p, m * q, a1 * b1)
        out.append(c)
    return out
