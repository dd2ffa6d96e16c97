"""Edge cases and degenerate inputs of the solve and of the C ABI, on the GPU: a zero load, the
smallest grid (one level), a rank cap of one, the plane-stress and two-material variants against
the Galerkin solution, a small 3D grid with a Fourier load, invalid arguments, out-of-range
evaluation points, train import/export round trips and an operator at the largest level count."""
import numpy as np
import pytest

from oracle import fem, tt
from paper_2501_12151_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_12151_gb300 import tnfem
    return tnfem


@pytest.fixture(scope="module")
def ctx(lib):
    return lib.Context(0)


def _solve_err(ctx, pr):
    Abc, f = fem.system(pr.grid, pr.material, pr.loads)
    uh = fem.solve(Abc, f)
    A = ctx.stiffness(pr.grid, pr.material)
    fv = ctx.load(pr.grid, pr.material, pr.loads)
    u, info = ctx.solve(A, fv, pr.opts)
    ud = tt.to_natural_order(tt.tt_full(u.cores()), pr.grid.dim, pr.grid.levels)
    return fem.energy_norm(Abc, ud - uh) / max(fem.energy_norm(Abc, uh), 1e-300), info, u


def test_zero_load_gives_zero_displacement(ctx):
    pr = W.steel_plate_2d(levels=4, rank_cap=16, tol=1e-10)
    pr.loads = [W.Load(kind="gravity", rho=0.0)]
    A = ctx.stiffness(pr.grid, pr.material)
    f = ctx.load(pr.grid, pr.material, pr.loads)
    for prec in ("fp64", "mixed-local"):
        pr.opts.precision = prec
        u, info = ctx.solve(A, f, pr.opts)
        assert np.abs(tt.tt_full(u.cores())).max() == 0.0, (prec, info)


@pytest.mark.parametrize("precision", ["fp64", "mixed-local"])
def test_single_level_grid(ctx, precision):
    pr = W.manufactured_2d(levels=1, rank_cap=8, tol=1e-12)
    pr.opts.precision = precision
    err, info, _ = _solve_err(ctx, pr)
    assert err <= 1e-8, (err, info)


def test_rank_cap_one_returns_a_rank_one_train(ctx):
    pr = W.manufactured_2d(levels=4, rank_cap=1, tol=1e-10)
    pr.opts.kickrank = 0
    pr.opts.max_sweeps = 4
    A = ctx.stiffness(pr.grid, pr.material)
    f = ctx.load(pr.grid, pr.material, pr.loads)
    u, info = ctx.solve(A, f, pr.opts)
    assert max(u.ranks()) == 1
    assert np.all(np.isfinite(tt.tt_full(u.cores())))


def test_plane_stress_and_two_materials(ctx):
    pr = W.steel_plate_2d(levels=5, rank_cap=64, tol=1e-11)
    pr.grid.plane_stress = True
    pr.material = W.Material(E=(210e9, 70e9), nu=0.33, split_x=0.5)
    err, info, _ = _solve_err(ctx, pr)
    assert err <= 1e-8, (err, info)


def test_small_3d_fourier_load_mixed_local(ctx):
    pr = W.cantilever_3d(levels=2, rank_cap=64, tol=1e-11)
    pr.opts.precision = "mixed-local"
    err, info, _ = _solve_err(ctx, pr)
    assert err <= 1e-8, (err, info)


def test_invalid_arguments_are_reported(ctx, lib):
    pr = W.manufactured_2d(levels=3, rank_cap=8, tol=1e-8)
    A = ctx.stiffness(pr.grid, pr.material)
    f = ctx.load(pr.grid, pr.material, pr.loads)
    bad = [("tol", 0.0), ("rank_cap", 0), ("kickrank", -1), ("max_sweeps", 0)]
    for field, value in bad:
        o = W.SolveOpts(**{**pr.opts.__dict__, field: value})
        with pytest.raises(lib.TnfemError) as ei:
            ctx.solve(A, f, o)
        assert ei.value.status == 1, field
    # operator and load on different grids
    g4 = W.Grid(dim=2, levels=4)
    f4 = ctx.load(g4, pr.material, pr.loads)
    with pytest.raises(lib.TnfemError):
        ctx.solve(A, f4, pr.opts)
    # evaluation outside the grid
    u, _ = ctx.solve(A, f, pr.opts)
    with pytest.raises(lib.TnfemError):
        u.displacement(np.array([[0, 8]]))
    with pytest.raises(lib.TnfemError):
        u.strain(pr.grid, np.array([[7, 0]]))


def test_export_import_round_trip(ctx):
    pr = W.manufactured_2d(levels=4, rank_cap=16, tol=1e-10)
    A = ctx.stiffness(pr.grid, pr.material)
    f = ctx.load(pr.grid, pr.material, pr.loads)
    u, _ = ctx.solve(A, f, pr.opts)
    cu = u.cores()
    u2 = ctx.tt_import(cu)
    for a, b in zip(cu, u2.cores()):
        np.testing.assert_array_equal(a, b)
    ca = A.cores()
    A2 = ctx.mpo_import(ca)
    for a, b in zip(ca, A2.cores()):
        np.testing.assert_array_equal(a, b)
    # the imported train as a start guess: already converged, so the sweep stops at once
    u3, info = ctx.solve(A, f, pr.opts, x0=u2)
    assert info["sweeps"] <= 3, info


def test_operator_at_the_largest_level_count(ctx, lib):
    """2^20 x 2^20 nodes (2.2e12 unknowns, never formed): the operator builds in QTT form with
    ranks bounded independently of the grid size (the device rounding never exceeds the host
    construction's ranks), and the operator applied to a constant field is finite."""
    g = W.Grid(dim=2, levels=20)
    mat = W.Material(E=(210e9, 210e9), nu=0.3)
    A = ctx.stiffness(g, mat)
    r = [1] + [c.shape[3] for c in A.cores()]
    host, _ = lib.host_stiffness(g, mat)
    rh = [1] + [c.shape[3] for c in host]
    assert len(r) == 22 and all(a <= b for a, b in zip(r, rh)), (r, rh)
    assert max(r) <= 128, r
    ones = ctx.tt_import([np.ones((1, 2, 1))] + [np.ones((1, 4, 1))] * 20)
    assert np.isfinite(A.apply(ones).norm())
