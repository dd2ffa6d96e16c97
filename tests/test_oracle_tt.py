"""Pins of oracle B (TT toolkit, elasticity TT-operator, AMEn) against facts fixed outside it:
dense linear algebra on tiny inputs, exact QTT ranks stated in the paper or derivable in closed
form, oracle A's element-loop matrix, and direct solves."""
import math

import numpy as np
import pytest

from oracle import amen, fem, mpo, tt
from paper_2501_12151_gb300 import workloads as W


def test_qtt_perm_hand_computed():
    # D=2, L=2: q = ((c*4 + s1)*4 + s2), s = 2*b_x + b_y, i = 2 b_x1 + b_x2, j = 2 b_y1 + b_y2,
    # natural = c*16 + 4 i + j.
    p = tt.qtt_perm(2, 2)
    assert list(p[:5]) == [0, 1, 4, 5, 2]
    assert p[16] == 16 and p[31] == 31
    assert sorted(p) == list(range(32))
    p3 = tt.qtt_perm(3, 1)
    assert list(p3) == list(range(24))      # one level: the merged mode is the natural order


def test_tt_svd_exact_and_truncation_bound():
    r = W.rng(3)
    T = r.standard_normal(2 * 4 * 4 * 4 * 4)
    cores = tt.tt_svd(T, [2, 4, 4, 4, 4], eps=1e-15)
    assert np.linalg.norm(tt.tt_full(cores) - T) <= 1e-13 * np.linalg.norm(T)
    # a tensor with decaying spectrum: truncation error below eps ||T||
    g = np.linspace(0, 1, 1024)
    T2 = np.exp(-3 * g) + 1e-4 * np.sin(40 * g) + 1e-9 * r.standard_normal(1024)
    for eps in (1e-3, 1e-6):
        c2 = tt.tt_svd(T2, [2] * 10, eps=eps)
        assert np.linalg.norm(tt.tt_full(c2) - T2) <= eps * np.linalg.norm(T2) * (1 + 1e-12)


def test_rounding_idempotent_and_sum():
    x = W.random_tt(5, [2, 4, 4, 4], [1, 2, 3, 3, 1])
    xr = tt.tt_round(x, 1e-14)
    assert np.linalg.norm(tt.tt_full(xr) - tt.tt_full(x)) <= 1e-13 * np.linalg.norm(tt.tt_full(x))
    s = tt.tt_round(tt.tt_add(x, x), 1e-13)
    assert tt.ranks(s) == tt.ranks(xr)
    np.testing.assert_allclose(tt.tt_full(s), 2 * tt.tt_full(x), atol=1e-12 * np.abs(tt.tt_full(x)).max())
    assert tt.tt_norm(x) == pytest.approx(np.linalg.norm(tt.tt_full(x)), rel=1e-13)
    assert tt.tt_dot(x, xr) == pytest.approx(np.linalg.norm(tt.tt_full(x)) ** 2, rel=1e-12)


def test_meshgrid_rank_two_section51():
    """Section 5.1: X(i, j) = i and Y(i, j) = j have TT rank at most 2 in the QTT layout."""
    L = 5
    n = 1 << L
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    for F in (i, j):
        v = tt.to_qtt_order(np.concatenate([F.ravel(), F.ravel()]).astype(float), 2, L)
        c = tt.tt_svd(v, [2] + [4] * L, eps=1e-14)
        assert max(tt.ranks(c)) <= 2


def test_sine_has_qtt_rank_two():
    L = 8
    xs = np.arange(1 << L) * 0.37 + 0.2
    for f in (np.sin(xs), np.cos(xs)):
        assert max(tt.ranks(tt.tt_svd(f, [2] * L, eps=1e-13))) == 2


def test_1d_matrix_qtt_ranks_independent_of_levels():
    """1D Q1 stiffness / mass / derivative-coupling matrices: Toeplitz tridiagonal plus corner
    corrections, so their QTT ranks stop growing once the train is long enough (Kazeev and
    Khoromskij: rank 3 for the Toeplitz part, one more per corner correction -> at most 5)."""
    ranks = {}
    for L in (4, 5, 6, 7, 8):
        K, M, G = mpo.matrices_1d(1 << L, 0.0, 1.0)
        ranks[L] = [max(tt.ranks(tt.mpo_from_dense(X, [2] * L, 1e-13))) for X in (K, M, G)]
    for L in (5, 6, 7, 8):
        assert ranks[L] == ranks[4]
    assert max(ranks[4]) <= 5


def test_mpo_apply_and_full_match_dense():
    A = W.random_mpo(7, [2, 4, 4], [1, 3, 2, 1])
    x = W.random_tt(8, [2, 4, 4], [1, 2, 3, 1])
    Ad = tt.mpo_full(A)
    xd = tt.tt_full(x)
    np.testing.assert_allclose(tt.tt_full(tt.mpo_apply(A, x)), Ad @ xd, rtol=1e-12, atol=1e-12)
    back = tt.mpo_from_dense(Ad, [2, 4, 4], 1e-15)
    np.testing.assert_allclose(tt.mpo_full(back), Ad, atol=1e-12 * np.abs(Ad).max())


@pytest.mark.parametrize("dim,levels,clamped,split", [
    (2, 3, (True, False, False, False, False, False), math.inf),
    (2, 4, (True, False, False, True, False, False), 0.5),
    (2, 4, (True, True, False, False, False, False), math.inf),
    (3, 2, (True, False, False, False, False, False), 0.5),
])
def test_stiffness_mpo_equals_element_loop_matrix(dim, levels, clamped, split):
    g = W.Grid(dim=dim, levels=levels, lo=(0.0, 0.5, -1.0), hi=(2.0, 1.5, 0.0), clamped=clamped)
    m = W.Material(E=(210.0, 70.0), nu=0.33, split_x=split)
    A, _ = fem.assemble(g, m)
    Abc = fem.apply_bc(g, A)
    Aq = tt.matrix_to_qtt_order(Abc, dim, levels)
    mp, s = mpo.stiffness_mpo(g, m)
    assert s == pytest.approx(fem.bc_shift(g, A), rel=1e-13)
    F = tt.mpo_full(mp)
    assert np.abs(F - Aq).max() <= 1e-12 * np.abs(Aq).max()


def test_mass_mpo_equals_element_loop_matrix():
    g = W.Grid(dim=2, levels=3, lo=(0.0, 0.0, 0.0), hi=(3.0, 1.0, 0.0))
    _, M = fem.assemble(g, W.Material())
    np.testing.assert_allclose(tt.mpo_full(mpo.mass_mpo(g)), tt.matrix_to_qtt_order(M, 2, 3),
                               atol=1e-15)


@pytest.mark.parametrize("problem", ["manufactured", "steel", "cube"])
def test_amen_matches_direct_solve(problem):
    if problem == "manufactured":
        pr = W.manufactured_2d(levels=4, rank_cap=64)
    elif problem == "steel":
        pr = W.steel_plate_2d(levels=4, rank_cap=64)
    else:
        pr = W.cantilever_3d(levels=2, rank_cap=64)
    D, L = pr.grid.dim, pr.grid.levels
    Abc, f = fem.system(pr.grid, pr.material, pr.loads)
    uh = fem.solve(Abc, f)
    A, _ = mpo.stiffness_mpo(pr.grid, pr.material)
    fq = mpo.load_tt_dense(f, pr.grid)
    x0 = W.random_tt(1, W.qtt_modes(D, L), [1] + [2] * L + [1])
    x, info = amen.amen_solve(A, fq, x0, tol=1e-11, rmax=64)
    assert info.converged
    u = tt.to_natural_order(tt.tt_full(x), D, L)
    rel = fem.energy_norm(Abc, u - uh) / fem.energy_norm(Abc, uh)
    assert rel < 1e-10, rel


def test_amen_respects_rank_cap():
    pr = W.manufactured_2d(levels=5, rank_cap=8)
    Abc, f = fem.system(pr.grid, pr.material, pr.loads)
    A, _ = mpo.stiffness_mpo(pr.grid, pr.material)
    fq = mpo.load_tt_dense(f, pr.grid)
    x0 = W.random_tt(1, W.qtt_modes(2, 5), [1] + [2] * 5 + [1])
    x, info = amen.amen_solve(A, fq, x0, tol=1e-10, rmax=8, kickrank=0, nswp=6)
    assert max(tt.ranks(x)) <= 8


def test_local_system_is_projection():
    """B_k from the environments equals V^T A V for the interface basis V (dense check)."""
    pr = W.steel_plate_2d(levels=2)
    A, _ = mpo.stiffness_mpo(pr.grid, pr.material)
    x = tt.orthogonalize_right(W.random_tt(2, [2, 4, 4], [1, 2, 3, 1]))
    x = tt.orthogonalize_left(x, upto=1)   # cores 0 left-orthogonal, core 2 right-orthogonal
    k = 1
    PhiL = amen.env_left_op(np.ones((1, 1, 1)), x[0], A[0], x[0])
    PhiR = amen.env_right_op(np.ones((1, 1, 1)), x[2], A[2], x[2])
    B = amen.local_dense(PhiL, A[k], PhiR)
    r0, n, r1 = x[1].shape
    # V maps the core's entries to the full vector
    V = np.zeros((32, r0 * n * r1))
    for col in range(r0 * n * r1):
        e = np.zeros(r0 * n * r1)
        e[col] = 1.0
        V[:, col] = tt.tt_full([x[0], e.reshape(r0, n, r1), x[2]])
    Ad = tt.mpo_full(A)
    np.testing.assert_allclose(B, V.T @ Ad @ V, atol=1e-12 * np.abs(Ad).max())
    assert np.allclose(V.T @ V, np.eye(V.shape[1]), atol=1e-12)


def _interface_basis(x):
    """V with V[:, c] = the full vector of the three-core train whose middle core is unit vector c."""
    r0, n, r1 = x[1].shape
    N = int(np.prod([c.shape[1] for c in x]))
    V = np.zeros((N, r0 * n * r1))
    for col in range(r0 * n * r1):
        e = np.zeros(r0 * n * r1)
        e[col] = 1.0
        V[:, col] = tt.tt_full([x[0], e.reshape(r0, n, r1), x[2]])
    return V


def _three_core_setup(seed):
    pr = W.steel_plate_2d(levels=2)
    A, _ = mpo.stiffness_mpo(pr.grid, pr.material)
    x = tt.orthogonalize_right(W.random_tt(seed, [2, 4, 4], [1, 2, 3, 1]))
    x = tt.orthogonalize_left(x, upto=1)
    return A, x


def test_local_matvec_is_projected_operator():
    """The structured local matvec (the contraction order the GPU kernels follow) applied to a
    core c equals V^T A V c with V the interface basis and A the full operator matrix."""
    A, x = _three_core_setup(3)
    PhiL = amen.env_left_op(np.ones((1, 1, 1)), x[0], A[0], x[0])
    PhiR = amen.env_right_op(np.ones((1, 1, 1)), x[2], A[2], x[2])
    V = _interface_basis(x)
    Ad = tt.mpo_full(A)
    c = W.rng(4).standard_normal(x[1].shape)
    got = amen.local_matvec(PhiL, A[1], PhiR, c).ravel()
    np.testing.assert_allclose(got, V.T @ (Ad @ (V @ c.ravel())), atol=1e-12 * np.abs(Ad).max() * np.abs(c).max())


def test_local_rhs_is_projected_load():
    """The local right-hand side from the load environments equals V^T f."""
    A, x = _three_core_setup(5)
    f = W.random_tt(6, [2, 4, 4], [1, 2, 2, 1])
    PsiL = amen.env_left_vec(np.ones((1, 1)), x[0], f[0])
    PsiR = amen.env_right_vec(np.ones((1, 1)), x[2], f[2])
    g = amen.local_rhs(PsiL, f[1], PsiR).ravel()
    np.testing.assert_allclose(g, _interface_basis(x).T @ tt.tt_full(f), atol=1e-12)


def test_environments_contract_to_bilinear_forms():
    """Sweeping the operator environments across two different trains y, x from either end gives
    y^T A x of the full matrix; the load environments give y^T f.  A is a random non-symmetric
    operator train, so that exchanging y and x (or the row and column index of A) is detected."""
    r = W.rng(12)
    modes = [2, 4, 4]
    a = [1, 3, 2, 1]
    A = [r.standard_normal((a[k], modes[k], modes[k], a[k + 1])) for k in range(3)]
    y = W.random_tt(7, modes, [1, 2, 3, 1])
    x = W.random_tt(8, modes, [1, 3, 2, 1])
    f = W.random_tt(9, modes, [1, 2, 2, 1])
    want = tt.tt_full(y) @ tt.mpo_full(A) @ tt.tt_full(x)
    Phi = np.ones((1, 1, 1))
    for k in range(len(A)):
        Phi = amen.env_left_op(Phi, y[k], A[k], x[k])
    assert Phi.shape == (1, 1, 1) and Phi[0, 0, 0] == pytest.approx(want, rel=1e-12)
    Phi = np.ones((1, 1, 1))
    for k in reversed(range(len(A))):
        Phi = amen.env_right_op(Phi, y[k], A[k], x[k])
    assert Phi[0, 0, 0] == pytest.approx(want, rel=1e-12)
    wantf = tt.tt_full(y) @ tt.tt_full(f)
    Psi = np.ones((1, 1))
    for k in range(len(f)):
        Psi = amen.env_left_vec(Psi, y[k], f[k])
    assert Psi[0, 0] == pytest.approx(wantf, rel=1e-12)
    Psi = np.ones((1, 1))
    for k in reversed(range(len(f))):
        Psi = amen.env_right_vec(Psi, y[k], f[k])
    assert Psi[0, 0] == pytest.approx(wantf, rel=1e-12)


def test_cg_solves_spd_system():
    """Plain CG on a random SPD matrix stops at the requested residual and approaches the direct
    solution; a zero right-hand side returns at once."""
    r = W.rng(10)
    M = r.standard_normal((40, 40))
    B = M @ M.T + 40 * np.eye(40)
    g = r.standard_normal(40)
    x, it = amen.cg(lambda v: B @ v, g, np.zeros(40), 1e-12, 500)
    assert 0 < it < 500
    # the recursive residual met 1e-12; the true one differs from it by rounding only
    assert np.linalg.norm(g - B @ x) <= 2e-12 * np.linalg.norm(g)
    np.testing.assert_allclose(x, np.linalg.solve(B, g), rtol=1e-9)
    z, it0 = amen.cg(lambda v: B @ v, np.zeros(40), np.ones(40), 1e-12, 500)
    assert it0 == 0 and not z.any()
