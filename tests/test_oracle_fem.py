"""Pins of oracle A (sparse Q1/trilinear FEM) against facts fixed outside the oracle.

Each test targets a plausible mistake: a wrong Lame formula, a transposed coupling block, a
dropped term in the element matrix, a sign error in the manufactured force, a wrong mass
scaling, a BC that leaks into the solution, or an assembly that breaks convergence rates.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import fem
from paper_2501_12151_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_lame_closed_forms():
    # plane strain: lambda = E nu / ((1+nu)(1-2nu)), mu = E / (2(1+nu)); E=1, nu=0.25 -> 0.4, 0.4
    lam, mu = fem.lame(1.0, 0.25, 2, False)
    assert lam == pytest.approx(0.4, rel=1e-15)
    assert mu == pytest.approx(0.4, rel=1e-15)
    # plane stress (Section 2, modified Lame parameter): lambda* = E nu / (1 - nu^2)
    lam_s, mu_s = fem.lame(1.0, 0.25, 2, True)
    assert lam_s == pytest.approx(0.25 / (1 - 0.0625), rel=1e-14)
    assert mu_s == pytest.approx(0.4, rel=1e-15)


def test_element_matrix_matches_published_plane_stress_square():
    """Unit-square Q1 plane-stress element stiffness against the closed form published with
    the 88-line topology-optimisation code (Andreassen et al., 2011), thickness 1."""
    E, nu = 1.0, 0.3
    lam, mu = fem.lame(E, nu, 2, True)
    X = fem.ref_corners(2).astype(float)          # corners (0,0),(0,1),(1,0),(1,1)
    K, _ = fem.element_matrices(X, lam, mu)
    k = [1 / 2 - nu / 6, 1 / 8 + nu / 8, -1 / 4 - nu / 12, -1 / 8 + 3 * nu / 8,
         -1 / 4 + nu / 12, -1 / 8 - nu / 8, nu / 6, 1 / 8 - 3 * nu / 8]
    idx = [[0, 1, 2, 3, 4, 5, 6, 7], [1, 0, 7, 6, 5, 4, 3, 2], [2, 7, 0, 5, 6, 3, 4, 1],
           [3, 6, 5, 0, 7, 2, 1, 4], [4, 5, 6, 7, 0, 1, 2, 3], [5, 4, 3, 2, 1, 0, 7, 6],
           [6, 3, 4, 1, 2, 7, 0, 5], [7, 2, 1, 4, 3, 6, 5, 0]]
    KE = E / (1 - nu * nu) * np.array([[k[j] for j in row] for row in idx])
    # published node order: lower-left, lower-right, upper-right, upper-left (x, y per node);
    # ours: corner a = 2*b_x + b_y -> (0,0)=0, (1,0)=2, (1,1)=3, (0,1)=1
    order = [0, 2, 3, 1]
    perm = [2 * a + c for a in order for c in range(2)]
    np.testing.assert_allclose(K[np.ix_(perm, perm)], KE, rtol=0, atol=1e-14)


@pytest.mark.parametrize("dim,levels", [(2, 3), (3, 2)])
def test_rigid_body_modes_in_kernel(dim, levels):
    g = W.Grid(dim=dim, levels=levels, lo=(0.1, -0.2, 0.3), hi=(1.3, 0.7, 1.1))
    A, _ = fem.assemble(g, W.Material(E=(3.0, 3.0), nu=0.3))
    P = fem.nodal_points(g)
    N = P.shape[0]
    modes = []
    for c in range(dim):
        v = np.zeros((dim, N))
        v[c] = 1.0
        modes.append(v.ravel())
    pairs = [(0, 1)] if dim == 2 else [(0, 1), (1, 2), (0, 2)]
    for a, b in pairs:
        v = np.zeros((dim, N))
        v[a] = -P[:, b]
        v[b] = P[:, a]
        modes.append(v.ravel())
    scale = abs(A).max()
    for v in modes:
        assert np.abs(A @ v).max() <= 1e-12 * scale * np.abs(v).max()
    assert np.abs(A - A.T).max() <= 1e-15 * scale


def test_patch_test_affine_field():
    """An affine displacement has constant strain: interior rows of A u vanish."""
    g = W.Grid(dim=2, levels=3)
    A, _ = fem.assemble(g, W.Material(E=(1.0, 1.0), nu=0.3))
    P = fem.nodal_points(g)
    u = np.concatenate([0.3 + 1.1 * P[:, 0] - 0.4 * P[:, 1], -0.2 + 0.7 * P[:, 0] + 0.5 * P[:, 1]])
    r = (A @ u).reshape(2, g.n, g.n)
    assert np.abs(r[:, 1:-1, 1:-1]).max() < 1e-13


@pytest.mark.parametrize("dim,levels", [(2, 3), (3, 2)])
def test_mass_matrix_integrates_constants(dim, levels):
    lo, hi = (0.0, -1.0, 2.0), (2.0, 0.5, 2.5)
    g = W.Grid(dim=dim, levels=levels, lo=lo, hi=hi)
    _, M = fem.assemble(g, W.Material())
    N = g.n ** dim
    vol = np.prod([hi[d] - lo[d] for d in range(dim)])
    for c in range(dim):
        e = np.zeros(dim * N)
        e[c * N:(c + 1) * N] = 1.0
        assert e @ (M @ e) == pytest.approx(vol, rel=1e-13)
    # face mass integrates the face area
    for face in range(2 * dim):
        Mf = fem.face_mass(g, face)
        d = face // 2
        area = np.prod([hi[e] - lo[e] for e in range(dim) if e != d])
        e = np.zeros(dim * N)
        e[:N] = 1.0
        assert e @ (Mf @ e) == pytest.approx(area, rel=1e-13)


def test_manufactured_force_is_minus_div_sigma():
    """The hand-derived body force equals -div sigma(u*) by central differences of sigma."""
    lam, mu = 1.7, 0.9
    x, y = np.array([0.23, 0.61, 0.87]), np.array([0.41, 0.13, 0.77])
    h = 1e-5
    sx1 = fem.manufactured_stress(x + h, y, lam, mu)
    sx0 = fem.manufactured_stress(x - h, y, lam, mu)
    sy1 = fem.manufactured_stress(x, y + h, lam, mu)
    sy0 = fem.manufactured_stress(x, y - h, lam, mu)
    div1 = (sx1[0] - sx0[0]) / (2 * h) + (sy1[2] - sy0[2]) / (2 * h)
    div2 = (sx1[2] - sx0[2]) / (2 * h) + (sy1[1] - sy0[1]) / (2 * h)
    f1, f2 = fem.manufactured_force(x, y, lam, mu)
    np.testing.assert_allclose(f1, -div1, rtol=1e-7)
    np.testing.assert_allclose(f2, -div2, rtol=1e-7)


def test_manufactured_convergence_rates():
    """Optimal rates: ||u* - u_h||_L2 = O(h^2), ||u* - u_h||_a = O(h)."""
    Ls = [3, 4, 5, 6, 7]
    l2, en, hs = [], [], []
    for L in Ls:
        pr = W.manufactured_2d(L)
        Abc, f = fem.system(pr.grid, pr.material, pr.loads)
        u = fem.solve(Abc, f)
        e_l2, e_en = fem.manufactured_errors(pr.grid, pr.material, u)
        l2.append(e_l2)
        en.append(e_en)
        hs.append(1.0 / (pr.grid.n - 1))
    s_l2 = np.polyfit(np.log(hs), np.log(l2), 1)[0]
    s_en = np.polyfit(np.log(hs), np.log(en), 1)[0]
    assert abs(s_l2 - 2.0) < 0.2, s_l2
    assert abs(s_en - 1.0) < 0.2, s_en


def test_dense_direct_solve_agrees_and_galerkin_identity():
    pr = W.steel_plate_2d(levels=4)
    Abc, f = fem.system(pr.grid, pr.material, pr.loads)
    u = fem.solve(Abc, f)
    ud = np.linalg.solve(Abc.toarray(), f)
    assert np.linalg.norm(u - ud) <= 1e-12 * np.linalg.norm(ud)
    # A u = f => u^T A u = f^T u
    assert u @ (Abc @ u) == pytest.approx(f @ u, rel=1e-12)
    # clamped unknowns solve to exactly zero
    cn = np.tile(fem.constrained_nodes(pr.grid), 2)
    assert np.all(u[cn] == 0.0)
    # positive definite after boundary conditions
    lmin = np.linalg.eigvalsh(Abc.toarray()).min()
    assert lmin > 0


def test_bc_shift_does_not_change_solution():
    pr = W.steel_plate_2d(levels=3)
    A, M = fem.assemble(pr.grid, pr.material)
    f = fem.load_vector(pr.grid, pr.material, pr.loads, M)
    Abc, fbc = fem.apply_bc(pr.grid, A, f)
    u1 = fem.solve(Abc, fbc)
    free = np.tile(~fem.constrained_nodes(pr.grid), 2).astype(float)
    Abc2 = (Abc + 7.5 * np.diag(1 - free))
    u2 = np.linalg.solve(np.asarray(Abc2), fbc)
    np.testing.assert_allclose(u1, u2, rtol=0, atol=1e-12 * np.abs(u1).max())


def test_grid_bookkeeping_golden():
    with open(os.path.join(GOLDEN, "section5_grid_counts.json")) as fh:
        gold = json.load(fh)
    for case in gold["cases"]:
        g = W.Grid(dim=2, levels=case["d"])
        assert g.n ** 2 == case["points"]
        assert g.dofs == case["dofs"]
        assert (g.n - 1) ** 2 == case["elements"]


def test_cantilever_tip_deflection_section6():
    """Section 6: the FE tip deflection of the 20 m x 1 m aluminium cantilever approaches the
    beam formula 3 rho g L^4 / (2 E H^2) (Euler-Bernoulli, so only to within a few percent)."""
    with open(os.path.join(GOLDEN, "section6_cantilever.json")) as fh:
        c = json.load(fh)
    ref = 3 * c["rho_kg_m3"] * c["g_m_s2"] * c["length_m"] ** 4 / (2 * c["E_pa"] * c["height_m"] ** 2)
    assert ref == pytest.approx(0.0935, rel=2e-3)
    defl = []
    for L in (6, 7):
        g = W.Grid(dim=2, levels=L, lo=(0.0, 0.0, 0.0), hi=(c["length_m"], c["height_m"], 0.0),
                   clamped=(True, False, False, False, False, False), plane_stress=True)
        mat = W.Material(E=(c["E_pa"], c["E_pa"]), nu=c["nu"])
        Abc, f = fem.system(g, mat, [W.Load(kind="gravity", rho=c["rho_kg_m3"], g=c["g_m_s2"])])
        u = fem.solve(Abc, f)
        uy = u[g.n ** 2:].reshape(g.n, g.n)
        defl.append(abs(uy[-1, g.n // 2]))
    # Q1 elements are too stiff in bending on 20:1 elements; refinement approaches the formula
    assert defl[1] > defl[0]
    assert abs(defl[1] - ref) / ref < 0.05, (defl, ref)


@pytest.mark.parametrize("dim,levels", [(2, 3), (3, 2)])
def test_load_resultants_equal_applied_forces(dim, levels):
    """Before boundary conditions the nodal load vector's components sum to the applied resultant:
    rho g |Omega| downward for gravity (the mass matrix integrates constants exactly) and t_c |F|
    for a uniform traction on face F.  A wrong mass scaling, a traction on the wrong face or
    component, or a dropped sign fails it."""
    g = W.Grid(dim=dim, levels=levels, lo=(0.0, 0.0, 0.0), hi=(2.0, 0.5, 0.25))
    m = W.Material()
    ext = [g.hi[d] - g.lo[d] for d in range(dim)]
    vol = float(np.prod(ext))
    N = g.n ** dim
    f = fem.load_vector(g, m, [W.Load(kind="gravity", rho=7850.0)])
    res = [f[c * N:(c + 1) * N].sum() for c in range(dim)]
    np.testing.assert_allclose(res[:-1], 0.0, atol=1e-9 * 7850.0 * W.GRAVITY * vol)
    assert res[-1] == pytest.approx(-7850.0 * W.GRAVITY * vol, rel=1e-12)
    for face in range(2 * dim):
        t = (3.0, -5.0, 7.0)[:dim] + (0.0,) * (3 - dim)
        f = fem.load_vector(g, m, [W.Load(kind="traction", face=face, traction=t)])
        area = vol / ext[face // 2]
        res = [f[c * N:(c + 1) * N].sum() for c in range(dim)]
        np.testing.assert_allclose(res, [t[c] * area for c in range(dim)], rtol=1e-12)
        # only the nodes of that face carry it
        coord = np.indices((g.n,) * dim).reshape(dim, -1)[face // 2]
        on_face = coord == (g.n - 1 if face % 2 else 0)
        for c in range(dim):
            assert not f[c * N:(c + 1) * N][~on_face].any()


def test_fourier_body_force_nodal_values_by_hand():
    """Fourier body force f_c(x) = scale * sum_m a[c,m] sin(pi k_m . x + phi_m) (the 3D
    cantilever's seeded load) at nodes chosen so that every sine has a value written by hand.

    Grid: 4 nodes per axis on [0, 1.5]^2, so coordinates are multiples of 1/2.  Two modes with
    k_0 = (1, 2), phi_0 = pi/6 and k_1 = (3, 1), phi_1 = pi/3; amplitudes a = [[2, -1], [0.5, 4]]
    (component-major), scale 0.5.  At x = (1/2, 1/2): pi k_0.x = 3pi/2 and pi k_1.x = 2pi, so
    sin(3pi/2 + pi/6) = -cos(pi/6) and sin(2pi + pi/3) = sin(pi/3).  At x = (1, 0): pi and 3pi,
    so both sines are -sin(phi_m).  A dropped pi, a transposed amplitude or wave-number index,
    or a phase added outside the sine fails one of the four values."""
    g = W.Grid(dim=2, levels=2, lo=(0.0, 0.0, 0.0), hi=(1.5, 1.5, 0.0))
    amp = np.array([[2.0, -1.0], [0.5, 4.0]])
    wave = np.array([[1, 2], [3, 1]])
    phase = np.array([np.pi / 6, np.pi / 3])
    ld = W.Load(kind="fourier", amp=amp, wave=wave, phase=phase, scale=0.5)
    f0 = fem.nodal_body_force(g, W.Material(), ld).reshape(2, 4, 4)
    c6, s3, s6 = math.sqrt(3) / 2, math.sqrt(3) / 2, 0.5   # cos(pi/6), sin(pi/3), sin(pi/6)
    # node (i, j) = (1, 1) is x = (1/2, 1/2); node (2, 0) is x = (1, 0)
    assert f0[0, 1, 1] == pytest.approx(0.5 * (2.0 * -c6 + -1.0 * s3), rel=1e-13)
    assert f0[1, 1, 1] == pytest.approx(0.5 * (0.5 * -c6 + 4.0 * s3), rel=1e-13)
    assert f0[0, 2, 0] == pytest.approx(0.5 * (2.0 * -s6 + -1.0 * -s3), rel=1e-13)
    assert f0[1, 2, 0] == pytest.approx(0.5 * (0.5 * -s6 + 4.0 * -s3), rel=1e-13)


@pytest.mark.parametrize("dim", [2, 3])
def test_fourier_load_integrates_to_closed_form(dim):
    """Summed over the nodes, M f0 of one Fourier mode is the integral of the nodal interpolant
    of f_c, which converges at O(h^2) to the closed-form integral of scale * a_c sin(pi k.x + phi)
    over the unit square / cube: Im(exp(i phi) prod_d (exp(i pi k_d) - 1) / (i pi k_d))."""
    k = np.array([1, 3, 1])[:dim]          # odd wave numbers: no factor of the integral vanishes
    phi = 0.7
    amp = np.array([[1.5], [-0.8], [2.5]])[:dim]
    ld = W.Load(kind="fourier", amp=amp, wave=k[None, :], phase=np.array([phi]), scale=3.0)
    exact_unit = (np.exp(1j * phi) * np.prod([(np.exp(1j * np.pi * kd) - 1) / (1j * np.pi * kd) for kd in k])).imag
    want = 3.0 * amp[:, 0] * exact_unit
    sums, hs = [], []
    for levels in ((5, 6) if dim == 2 else (3, 4)):
        g = W.Grid(dim=dim, levels=levels)
        N = g.n ** dim
        f = fem.load_vector(g, W.Material(), [ld])
        sums.append(np.array([f[c * N:(c + 1) * N].sum() for c in range(dim)]))
        hs.append(1.0 / (g.n - 1))
    errs = [np.abs(s - want).max() / np.abs(want).max() for s in sums]
    # second order: the error falls with h^2 ...
    assert errs[1] < 0.3 * errs[0], errs
    # ... and Richardson extrapolation in h^2 removes it to the next order
    (sc, sf), (hc, hf) = sums, hs
    extrap = (sf * hc * hc - sc * hf * hf) / (hc * hc - hf * hf)
    assert np.abs(extrap - want).max() < 0.05 * errs[1] * np.abs(want).max(), (extrap, want, errs)


def test_interpolation_reproduces_linear_fields():
    """The multigrid prolongation (linear interpolation between grids of 2^l and 2^(l-1) nodes)
    is exact on affine fields, per axis and for the vector field (rigid rotations included)."""
    P = fem.interpolation_1d(16, 8)
    xc, xf = np.linspace(0.0, 1.0, 8), np.linspace(0.0, 1.0, 16)
    np.testing.assert_allclose(P @ (2.0 - 3.0 * xc), 2.0 - 3.0 * xf, rtol=0, atol=1e-14)
    np.testing.assert_allclose(P.sum(axis=1), 1.0, rtol=0, atol=1e-15)
    Pv = fem.vector_interpolation(2, 16, 8)
    Xc, Yc = np.meshgrid(xc, xc, indexing="ij")
    Xf, Yf = np.meshgrid(xf, xf, indexing="ij")
    rot_c = np.concatenate([-Yc.ravel(), Xc.ravel()])
    rot_f = np.concatenate([-Yf.ravel(), Xf.ravel()])
    np.testing.assert_allclose(Pv @ rot_c, rot_f, rtol=0, atol=1e-14)


@pytest.mark.parametrize("problem", ["steel6", "steel7", "cube3"])
def test_multigrid_cg_matches_direct_solve(problem):
    """The V-cycle preconditioned CG used for u_h at large sizes reaches the sparse direct
    solution (the definition u_h = A^{-1} f) on grids small enough for a direct solve.  (Its
    isotropic coarsening suits square elements; it is not used for the 20:1 cantilever.)"""
    if problem == "steel6":
        pr = W.steel_plate_2d(levels=6)
    elif problem == "steel7":
        pr = W.steel_plate_2d(levels=7)
    else:
        pr = W.cantilever_3d(levels=3)
    Abc, f = fem.system(pr.grid, pr.material, pr.loads)
    u, info = fem.solve_mg(pr.grid, Abc, f)
    ud = spla.spsolve(Abc.tocsc(), f)
    assert info["converged"] and info["iters"] < 100, info
    assert fem.energy_norm(Abc, u - ud) <= 1e-10 * fem.energy_norm(Abc, ud)


SHEAR2 = ((1.5, 0.3), (0.6, 1.0))
SHEAR3 = ((1.2, 0.2, 0.1), (0.3, 0.9, 0.0), (0.1, 0.4, 0.8))


@pytest.mark.parametrize("dim,levels", [(2, 3), (3, 2)])
def test_mapped_domain_rigid_modes_area_and_patch(dim, levels):
    """Parallelogram / parallelepiped domains (the affine element maps of Section 5.1): the
    free-free operator annihilates the rigid-body modes evaluated at the mapped node positions,
    the mass matrix integrates 1 to |det J| (the domain's measure), and an affine displacement
    field leaves zero residual at every interior node (patch test)."""
    edges = SHEAR2 if dim == 2 else SHEAR3
    g = W.Grid(dim=dim, levels=levels, lo=(0.2, -0.1, 0.3), edges=edges)
    A, M = fem.assemble(g, W.Material(E=(2.0, 2.0), nu=0.3))
    P = fem.nodal_points(g)
    N = P.shape[0]
    vol = abs(np.linalg.det(np.asarray(edges)))
    e = np.zeros(dim * N)
    e[:N] = 1.0
    assert e @ (M @ e) == pytest.approx(vol, rel=1e-13)
    modes = [np.eye(dim)[c][:, None] * np.ones(N)[None, :] for c in range(dim)]
    for (a, b) in ([(0, 1)] if dim == 2 else [(0, 1), (0, 2), (1, 2)]):
        r = np.zeros((dim, N))
        r[a], r[b] = -P[:, b], P[:, a]
        modes.append(r)
    nA = abs(A).max()
    for m in modes:
        v = m.ravel()
        assert np.abs(A @ v).max() <= 1e-12 * nA * np.abs(v).max()
    # an affine field: only boundary rows feel it
    G = np.arange(1, dim * dim + 1, dtype=float).reshape(dim, dim) / 7.0
    v = (P @ G.T).T.ravel()
    interior = np.all((np.indices((g.n,) * dim).reshape(dim, -1) > 0) &
                      (np.indices((g.n,) * dim).reshape(dim, -1) < g.n - 1), axis=0)
    res = (A @ v).reshape(dim, N)
    assert np.abs(res[:, interior]).max() <= 1e-12 * nA * np.abs(v).max()


def test_mapped_domain_with_axis_edges_equals_box():
    """A parallelogram whose edges lie along the axes is the box: same matrices, same load."""
    g_box = W.Grid(dim=2, levels=3, lo=(0.1, 0.2, 0.0), hi=(1.6, 0.9, 0.0))
    g_map = W.Grid(dim=2, levels=3, lo=(0.1, 0.2, 0.0), edges=((1.5, 0.0), (0.0, 0.7)))
    m = W.Material(E=(3.0, 3.0), nu=0.25)
    loads = [W.Load(kind="gravity", rho=2.0), W.Load(kind="traction", face=1, traction=(0.5, -1.0, 0.0))]
    (A1, M1), (A2, M2) = fem.assemble(g_box, m), fem.assemble(g_map, m)
    assert abs(A1 - A2).max() <= 1e-13 * abs(A1).max()
    assert abs(M1 - M2).max() <= 1e-15
    np.testing.assert_allclose(fem.load_vector(g_box, m, loads), fem.load_vector(g_map, m, loads), rtol=0, atol=1e-14)


def test_mapped_traction_resultant():
    """A uniform traction on a side of a parallelogram sums to the traction times the side's length."""
    g = W.Grid(dim=2, levels=3, lo=(0.0, 0.0, 0.0), edges=SHEAR2)
    N = g.n ** 2
    for face in range(4):
        f = fem.load_vector(g, W.Material(), [W.Load(kind="traction", face=face, traction=(2.0, -3.0, 0.0))])
        length = np.linalg.norm(SHEAR2[1 - face // 2])       # the side runs along the other edge
        np.testing.assert_allclose([f[:N].sum(), f[N:].sum()], [2.0 * length, -3.0 * length], rtol=1e-12)


QUAD = ((0.0, 0.0), (1.0, 0.1), (0.2, 0.9), (1.3, 1.4))   # convex, not a parallelogram


def _shoelace(P):
    ring = [P[0], P[1], P[3], P[2]]
    return 0.5 * abs(sum(ring[i][0] * ring[i - 3][1] - ring[i - 3][0] * ring[i][1] for i in range(4)))


def test_quad_grid_on_a_parallelogram_is_the_affine_grid():
    """Corners with P3 = P1 + P2 - P0 make the bilinear map affine: the frozen-Jacobian assembly
    (Algorithm 1) then coincides with the exact affine assembly, node positions, matrices and
    loads alike."""
    P0, e0, e1 = np.array([0.2, -0.1]), np.array([1.5, 0.3]), np.array([0.6, 1.0])
    quad = (P0, P0 + e0, P0 + e1, P0 + e0 + e1)
    g_aff = W.Grid(dim=2, levels=3, lo=(0.2, -0.1, 0.0), edges=(e0, e1), clamped=(False, False, True, False))
    g_quad = W.Grid(dim=2, levels=3, quad=quad, clamped=(False, False, True, False))
    m = W.Material(E=(3.0, 3.0), nu=0.25)
    loads = [W.Load(kind="gravity", rho=2.0), W.Load(kind="traction", face=1, traction=(0.5, -1.0, 0.0))]
    np.testing.assert_allclose(fem.nodal_points(g_quad), fem.nodal_points(g_aff), rtol=0, atol=1e-15)
    (A1, M1), (A2, M2) = fem.assemble(g_aff, m), fem.assemble(g_quad, m, frozen_jacobian=True)
    assert abs(A1 - A2).max() <= 1e-13 * abs(A1).max()
    assert abs(M1 - M2).max() <= 1e-15
    A1b, f1 = fem.system(g_aff, m, loads)
    A2b, f2 = fem.system(g_quad, m, loads, frozen_jacobian=True)
    assert abs(A1b - A2b).max() <= 1e-13 * abs(A1b).max()
    np.testing.assert_allclose(f1, f2, rtol=0, atol=1e-14)


def test_frozen_element_matrix_is_that_of_the_centre_parallelogram():
    """Freezing the Jacobian at the element centre (Algorithm 1 evaluates J at xi = 0 of
    Q = [-1,1]^2) gives the exact matrices of the parallelogram x = x_c + J(0) xi spanned by the
    centre Jacobian: built here from the exact path on that other geometry."""
    R = 2.0 * fem.ref_corners(2) - 1.0                             # corner signs in [-1,1]^2
    at = {(-1, -1): (0.0, 0.0), (1, -1): (1.1, 0.2), (-1, 1): (0.3, 0.8), (1, 1): (1.6, 1.5)}
    X = np.array([at[(int(r[0]), int(r[1]))] for r in R])
    xc = X.mean(axis=0)
    J0 = X.T @ R / 4.0                                             # dx_d / dxi_e at xi = 0
    Xp = xc[None, :] + R @ J0.T
    Kf, Mf = fem.element_matrices(X, 1.7, 0.9, frozen=True)
    Kp, Mp = fem.element_matrices(Xp, 1.7, 0.9)
    np.testing.assert_allclose(Kf, Kp, rtol=0, atol=1e-14 * abs(Kp).max())
    np.testing.assert_allclose(Mf, Mp, rtol=0, atol=1e-15)
    Ke, _ = fem.element_matrices(X, 1.7, 0.9)
    assert abs(Ke - Kf).max() > 1e-3 * abs(Ke).max()             # the quadrilateral is not affine


def test_quad_frozen_assembly_area_translations_and_convergence():
    """General quadrilateral, Jacobian frozen per element: the mass integrates 1 to the exact area
    (det J is affine in xi, so the centre value is its element mean), translations are in the
    kernel, the rotation's energy and the distance to the exactly assembled Galerkin solution
    fall like h^2 (the frozen Jacobian is an O(h) relative perturbation of the element map's)."""
    m = W.Material(E=(2.0, 2.0), nu=0.3)
    loads = [W.Load(kind="gravity", rho=1.0), W.Load(kind="traction", face=1, traction=(0.0, -0.5, 0.0))]
    rot_energy, sol_diff = [], []
    for levels in (3, 4, 5):
        g = W.Grid(dim=2, levels=levels, quad=QUAD, clamped=(True, False, False, False))
        A, M = fem.assemble(g, m, frozen_jacobian=True)
        N = g.n ** 2
        P = fem.nodal_points(g)
        one = np.concatenate([np.ones(N), np.zeros(N)])
        assert one @ (M @ one) == pytest.approx(_shoelace(QUAD), rel=1e-13)
        nA = abs(A).max()
        for c in range(2):
            t = np.zeros(2 * N)
            t[c * N:(c + 1) * N] = 1.0
            assert np.abs(A @ t).max() <= 1e-12 * nA
        r = np.concatenate([-P[:, 1], P[:, 0]])
        rot_energy.append(r @ (A @ r))
        A_ex, _ = fem.assemble(g, m)
        assert abs(A_ex @ r).max() <= 1e-12 * abs(A_ex).max() * np.abs(r).max()
        Af, ff = fem.system(g, m, loads, frozen_jacobian=True)
        Ae, fe = fem.system(g, m, loads)
        uf, ue = spla.spsolve(Af.tocsc(), ff), spla.spsolve(Ae.tocsc(), fe)
        sol_diff.append(fem.energy_norm(Ae, uf - ue) / fem.energy_norm(Ae, ue))
    for k in range(2):
        assert 3.0 <= rot_energy[k] / rot_energy[k + 1] <= 5.0, rot_energy
        assert 3.0 <= sol_diff[k] / sol_diff[k + 1] <= 5.0, sol_diff
    assert sol_diff[-1] < 4e-3


def test_nodal_load_integrates_affine_fields():
    """f = M f0 from given nodal values (Section 5.3): for an affine f0 the component sums of f are
    the exact integrals of f0, area times its value at the centroid, on a box, a parallelogram and
    a general quadrilateral (exact assembly: det J is affine in xi, and the 2-point rule integrates
    its product with the bilinear interpolant exactly) whose centroid is computed independently."""
    a, b = np.array([0.7, -1.2]), np.array([[0.3, -0.5], [1.1, 0.4]])    # f0_c(x) = a_c + b_c . x
    grids = [(W.Grid(dim=2, levels=4, lo=(0.2, -0.3, 0.0), hi=(1.7, 0.9, 0.0)), False),
             (W.Grid(dim=2, levels=4, lo=(0.2, -0.3, 0.0), edges=SHEAR2), False),
             (W.Grid(dim=2, levels=5, quad=QUAD), False)]
    for g, frozen in grids:
        P = fem.nodal_points(g)
        vals = np.stack([a[c] + P @ b[c] for c in range(2)]).ravel()
        _, M = fem.assemble(g, W.Material(), frozen_jacobian=frozen)
        f = fem.load_vector(g, W.Material(), [W.Load(kind="nodal", values=vals)], M)
        if g.quad is not None:
            ring = [np.array(QUAD[i]) for i in (0, 1, 3, 2)]
            cross = [ring[i][0] * ring[i - 3][1] - ring[i - 3][0] * ring[i][1] for i in range(4)]
            area = 0.5 * sum(cross)
            cen = sum((ring[i] + ring[i - 3]) * cross[i] for i in range(4)) / (6.0 * area)
            area = abs(area)
        elif g.edges is not None:
            E = np.asarray(SHEAR2)
            area, cen = abs(np.linalg.det(E)), np.array(g.lo[:2]) + 0.5 * (E[0] + E[1])
        else:
            area = (g.hi[0] - g.lo[0]) * (g.hi[1] - g.lo[1])
            cen = 0.5 * (np.array(g.lo[:2]) + np.array(g.hi[:2]))
        N = g.n ** 2
        for c in range(2):
            assert f[c * N:(c + 1) * N].sum() == pytest.approx(area * (a[c] + b[c] @ cen), rel=1e-12)
