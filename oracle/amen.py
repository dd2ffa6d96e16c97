"""Oracle B, part 3: the AMEn linear solver for A x = b in TT format, FP64, CPU.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper solves A u = M f0 with "the AMEn solver" (Section 5.4, Algorithm 2, citation key
``amen``: alternating minimal energy, Dolgov and Savostyanov).  The steps below follow that
method as published, core by core, with alternating sweep directions:

  for each core k of the sweep:
    1. project:  B_k = Phi_L (A_k) Phi_R  and  g_k = Psi_L b_k Psi_R  onto the current
       orthonormal interfaces of x (left of k and right of k);
    2. record the local residual ||g_k - B_k x_k|| / ||g_k|| (the sweep's convergence measure);
    3. solve B_k y = g_k (dense solve when small, conjugate gradients otherwise: B_k is
       symmetric positive definite because A is and the interfaces are orthonormal);
    4. truncate y by SVD with threshold delta = tol / sqrt(d) (relative Frobenius) and rank cap;
    5. enrich: project the residual onto the left interface of x and the right interface of the
       auxiliary TT z, append it to the kept singular vectors, re-orthogonalise by QR; update z
       from the residual projected onto z's own interfaces (top kickrank singular vectors);
    6. move the non-orthogonal factor into the next core and update the interface
       projections (environments) for x and z.

The sweep direction alternates; a backward sweep is a forward sweep over the reversed train
(cores flipped and transposed), which is the same computation written once.

Environments: Phi[a', beta, a] = sum over the contracted cores of conj(x) A x (bra index
first), Psi[a', c] for <x|b>, and the same with z as bra.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

from . import tt

Cores = List[np.ndarray]


@dataclass
class AmenInfo:
    sweeps: int = 0
    max_res: List[float] = field(default_factory=list)
    max_dx: List[float] = field(default_factory=list)
    ranks: List[int] = field(default_factory=list)
    local_iters: int = 0
    converged: bool = False


# ---------------------------------------------------------------------------------------
# environments and local operators
# ---------------------------------------------------------------------------------------

def _stage12(Phi, Ak, x):
    """T2[a',b,i,gamma] = sum_{beta,j} (sum_a Phi[a',beta,a] x[a,j,b]) A[beta,i,j,gamma]."""
    r0p, a0, r0 = Phi.shape
    _, n, _, a1 = Ak.shape
    r1 = x.shape[2]
    T1 = (Phi.reshape(r0p * a0, r0) @ x.reshape(r0, n * r1)).reshape(r0p, a0, n, r1)
    T1 = T1.transpose(0, 3, 1, 2).reshape(r0p * r1, a0 * n)            # (a' b), (beta j)
    T2 = T1 @ Ak.transpose(0, 2, 1, 3).reshape(a0 * n, n * a1)         # (a' b), (i gamma)
    return T2.reshape(r0p, r1, n, a1)


def env_left_op(Phi, y, Ak, x):
    """Phi'[b', gamma, b] = sum y[a',i,b'] Phi[a',beta,a] A[beta,i,j,gamma] x[a,j,b]."""
    T2 = _stage12(Phi, Ak, x)                                          # a', b, i, gamma
    r0p, r1, n, a1 = T2.shape
    T2 = T2.transpose(0, 2, 3, 1).reshape(r0p * n, a1 * r1)            # (a' i), (gamma b)
    out = y.reshape(r0p * n, -1).T @ T2                                # b', (gamma b)
    return out.reshape(-1, a1, r1)


def env_right_op(Phi, y, Ak, x):
    """Phi'[a', beta, a] = sum y[a',i,b'] A[beta,i,j,gamma] x[a,j,b] Phi[b',gamma,b]."""
    r0, n, r1 = x.shape
    r1p, a1, _ = Phi.shape
    a0 = Ak.shape[0]
    T1 = (x.reshape(r0 * n, r1) @ Phi.reshape(r1p * a1, r1).T).reshape(r0, n, r1p, a1)
    T1 = T1.transpose(0, 2, 1, 3).reshape(r0 * r1p, n * a1)            # (a b'), (j gamma)
    T2 = T1 @ Ak.transpose(2, 3, 0, 1).reshape(n * a1, a0 * n)         # (a b'), (beta i)
    T2 = T2.reshape(r0, r1p, a0, n).transpose(0, 2, 3, 1).reshape(r0 * a0, n * r1p)
    out = T2 @ y.reshape(y.shape[0], n * r1p).T                        # (a beta), a'
    return out.reshape(r0, a0, -1).transpose(2, 1, 0).copy()


def env_left_vec(Psi, y, fk):
    """Psi'[b', d] = sum y[a',i,b'] Psi[a',c] f[c,i,d]."""
    c, n, dd = fk.shape
    T = (Psi @ fk.reshape(c, n * dd)).reshape(-1, dd)                  # (a' i), d
    return y.reshape(-1, y.shape[2]).T @ T


def env_right_vec(Psi, y, fk):
    """Psi'[a', c] = sum y[a',i,b'] f[c,i,d] Psi[b',d]."""
    c, n, dd = fk.shape
    T = (fk.reshape(c * n, dd) @ Psi.T).reshape(c, n * Psi.shape[0])   # c, (i b')
    return y.reshape(y.shape[0], -1) @ T.T


def local_matvec(PhiL, Ak, PhiR, x):
    """y[a',i,b'] = sum PhiL[a',beta,a] A[beta,i,j,gamma] PhiR[b',gamma,b] x[a,j,b]."""
    T2 = _stage12(PhiL, Ak, x)                                         # a', b, i, gamma
    r0p, r1, n, a1 = T2.shape
    T2 = T2.transpose(0, 2, 3, 1).reshape(r0p * n, a1 * r1)            # (a' i), (gamma b)
    out = T2 @ PhiR.reshape(PhiR.shape[0], a1 * r1).T                  # (a' i), b'
    return out.reshape(r0p, n, -1)


def local_rhs(PsiL, fk, PsiR):
    c, n, dd = fk.shape
    T = (PsiL @ fk.reshape(c, n * dd)).reshape(-1, dd)
    return (T @ PsiR.T).reshape(PsiL.shape[0], n, PsiR.shape[0])


def local_dense(PhiL, Ak, PhiR):
    """Dense local matrix B[(a',i,b'), (a,j,b)] = sum PhiL[a',beta,a] A[beta,i,j,gamma] PhiR[b',gamma,b]."""
    r0p, a0, r0 = PhiL.shape
    _, n, _, a1 = Ak.shape
    r1p, _, r1 = PhiR.shape
    T = PhiL.transpose(0, 2, 1).reshape(r0p * r0, a0) @ Ak.reshape(a0, n * n * a1)
    B = T.reshape(r0p * r0 * n * n, a1) @ PhiR.transpose(1, 0, 2).reshape(a1, r1p * r1)
    B = B.reshape(r0p, r0, n, n, r1p, r1).transpose(0, 2, 4, 1, 3, 5)
    N = r0p * n * r1p
    return B.reshape(N, r0 * n * r1)


def cg(matvec, g, x0, rtol, maxit):
    """Plain conjugate gradients on an SPD operator, from x0, to ||g - Bx|| <= rtol ||g||."""
    x = x0.copy()
    r = g - matvec(x)
    gn = np.linalg.norm(g)
    if gn == 0.0:
        return np.zeros_like(g), 0
    p = r.copy()
    rr = r @ r
    it = 0
    while math.sqrt(rr) > rtol * gn and it < maxit:
        Bp = matvec(p)
        alpha = rr / (p @ Bp)
        x += alpha * p
        r -= alpha * Bp
        rr_new = r @ r
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
    return x, it


# ---------------------------------------------------------------------------------------
# the sweep
# ---------------------------------------------------------------------------------------

def _flip_tt(x: Cores) -> Cores:
    return [c.transpose(2, 1, 0).copy() for c in x[::-1]]


def _flip_mpo(A: Cores) -> Cores:
    return [c.transpose(3, 1, 2, 0).copy() for c in A[::-1]]


def amen_solve(A: Cores, b: Cores, x0: Cores, tol: float = 1e-10, rmax: int = 64,
               kickrank: int = 4, nswp: int = 40, z0: Optional[Cores] = None,
               dense_max: int = 4096, local_maxit: int = 2000, resid_damp: float = 2.0,
               seed: int = 0, verbose: bool = False):
    """Solve A x = b in TT format by AMEn; returns (x, info).

    tol: stop after a sweep whose largest local residual (step 2) or largest relative change
         of a core by its local solve is <= tol; also the truncation threshold
         delta = tol / sqrt(d).  (With a Frobenius truncation the local residual levels off near
         cond(B_k) * delta, while the solution change keeps tracking the accuracy.)
    rmax: rank cap; kickrank: rank of the residual enrichment.
    """
    d = len(A)
    info = AmenInfo()
    rng = np.random.default_rng(seed)
    x = tt.orthogonalize_right(x0)
    if z0 is None:
        zr = [1] + [max(kickrank, 1)] * (d - 1) + [1]
        z0 = [rng.standard_normal((zr[k], A[k].shape[1], zr[k + 1])) for k in range(d)]
    z = tt.orthogonalize_right(z0)
    delta = tol / math.sqrt(d)
    # right environments for the first forward sweep
    ra = [A[0].shape[0]] + [c.shape[3] for c in A]

    def right_envs(x, z, A, b):
        PhiR = [None] * d
        PsiR = [None] * d
        PhiZR = [None] * d
        PsiZR = [None] * d
        PhiR[d - 1] = np.ones((1, 1, 1))
        PsiR[d - 1] = np.ones((1, 1))
        PhiZR[d - 1] = np.ones((1, 1, 1))
        PsiZR[d - 1] = np.ones((1, 1))
        for k in range(d - 1, 0, -1):
            PhiR[k - 1] = env_right_op(PhiR[k], x[k], A[k], x[k])
            PsiR[k - 1] = env_right_vec(PsiR[k], x[k], b[k])
            if kickrank > 0:
                PhiZR[k - 1] = env_right_op(PhiZR[k], z[k], A[k], x[k])
                PsiZR[k - 1] = env_right_vec(PsiZR[k], z[k], b[k])
        return PhiR, PsiR, PhiZR, PsiZR

    PhiR, PsiR, PhiZR, PsiZR = right_envs(x, z, A, b)
    direction = 0
    for sweep in range(nswp):
        PhiL = [None] * d
        PsiL = [None] * d
        PhiZL = [None] * d
        PsiZL = [None] * d
        PhiL[0] = np.ones((1, 1, 1))
        PsiL[0] = np.ones((1, 1))
        PhiZL[0] = np.ones((1, 1, 1))
        PsiZL[0] = np.ones((1, 1))
        max_res = 0.0
        max_dx = 0.0
        for k in range(d):
            # 1. local system
            g = local_rhs(PsiL[k], b[k], PsiR[k])
            shp = g.shape
            N = g.size

            def mv(v, k=k):
                return local_matvec(PhiL[k], A[k], PhiR[k], v.reshape(shp)).reshape(-1)

            gn = np.linalg.norm(g)
            # 2. residual before the solve
            res = np.linalg.norm(g.reshape(-1) - mv(x[k].reshape(-1))) / max(gn, 1e-300)
            max_res = max(max_res, res)
            # 3. local solve
            if res > tol / resid_damp:
                if N <= dense_max:
                    B = local_dense(PhiL[k], A[k], PhiR[k])
                    y = np.linalg.solve(B, g.reshape(-1))
                else:
                    y, it = cg(mv, g.reshape(-1), x[k].reshape(-1), tol / resid_damp, local_maxit)
                    info.local_iters += it
                y = y.reshape(shp)
            else:
                y = x[k]
            max_dx = max(max_dx, np.linalg.norm(y - x[k]) / max(np.linalg.norm(y), 1e-300))
            if k == d - 1:
                x[k] = y
                if kickrank > 0:
                    # keep the z train's ranks consistent; this core is recomputed before use
                    z[k] = np.zeros((z[k - 1].shape[2] if k > 0 else 1, shp[1], 1))
                break
            # 4. truncation
            r0, n, r1 = shp
            U, S, Vt = np.linalg.svd(y.reshape(r0 * n, r1), full_matrices=False)
            rk = tt.truncation_rank(S, delta * np.linalg.norm(S), rmax)
            U = U[:, :rk]
            V = S[:rk, None] * Vt[:rk]          # rk x r1
            yt = (U @ V).reshape(shp)
            # 5. enrichment
            if kickrank > 0:
                # residual on z's interfaces -> new z core
                crz = local_matvec(PhiZL[k], A[k], PhiZR[k], yt) - local_rhs(PsiZL[k], b[k], PsiZR[k])
                rz0 = crz.shape[0]
                Uz, Sz, _ = np.linalg.svd(crz.reshape(rz0 * n, -1), full_matrices=False)
                kz = min(kickrank, Uz.shape[1])
                z[k] = Uz[:, :kz].reshape(rz0, n, kz)
                # residual on (x left, z right) interfaces -> enrichment block
                crs = local_matvec(PhiL[k], A[k], PhiZR[k], yt) - local_rhs(PsiL[k], b[k], PsiZR[k])
                Ue = np.concatenate([U, crs.reshape(r0 * n, -1)], axis=1)
                Q, R = np.linalg.qr(Ue)
                V = R[:, :rk] @ V
                U = Q
            rnew = U.shape[1]
            x[k] = U.reshape(r0, n, rnew)
            x[k + 1] = np.einsum("ab,bjc->ajc", V, x[k + 1])
            # 6. environments
            PhiL[k + 1] = env_left_op(PhiL[k], x[k], A[k], x[k])
            PsiL[k + 1] = env_left_vec(PsiL[k], x[k], b[k])
            if kickrank > 0:
                PhiZL[k + 1] = env_left_op(PhiZL[k], z[k], A[k], x[k])
                PsiZL[k + 1] = env_left_vec(PsiZL[k], z[k], b[k])
        info.sweeps = sweep + 1
        info.max_res.append(max_res)
        info.max_dx.append(max_dx)
        if verbose:
            print(f"sweep {sweep}: max local residual {max_res:.3e} ranks {tt.ranks(x)}")
        # reverse orientation: the left environments of this sweep are the right ones of the next
        x = _flip_tt(x)
        z = _flip_tt(z)
        A = _flip_mpo(A)
        b = _flip_tt(b)
        direction ^= 1
        # environments are (bra, [op,] ket) on both sides, so they carry over unchanged
        PhiR = PhiL[::-1]
        PsiR = PsiL[::-1]
        PhiZR = PhiZL[::-1]
        PsiZR = PsiZL[::-1]
        if max_res <= tol or max_dx <= tol:
            info.converged = True
            break
    if direction == 1:
        x = _flip_tt(x)
    info.ranks = tt.ranks(x)
    return x, info
