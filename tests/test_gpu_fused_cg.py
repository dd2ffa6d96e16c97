"""The local solves (step a5) as one persistent cooperative kernel: preconditioned CG on single
local systems through tnfem_op_local_cg, checked by the binary64 residual of the returned iterate
(computed with the oracle's local matvec), its edge cases, and whole solves with the fused kernel
against solves with one launch per CG step.

Local systems: B = sum_beta PhiL_beta (x) M_beta (x) PhiR_beta with every factor symmetric
positive semidefinite and the beta = 0 factors shifted by the identity, so B is symmetric positive
definite with the (PhiL, A, PhiR) structure of the sweep's systems and a spread spectrum.

Tolerances: binary64 runs stop on the recursively updated residual at rtol; the true residual of
the iterate differs from it by rounding only (a few 1e-16 relative per step), so 1.5 rtol bounds
it.  Binary32 runs use binary32 operands (the reference system is built from the same rounded
values) and rtol = 1e-4; the true residual then sits within a small multiple of eps32 * cond(B)
of the recursive one, and 2 rtol bounds it for these systems."""
import numpy as np
import pytest

from oracle import amen, tt
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


def spd_system(seed, r0, n, r1, a0, a1):
    r = W.rng(seed)
    PhiL = np.zeros((r0, a0, r0))
    PhiR = np.zeros((r1, a1, r1))
    A = np.zeros((a0, n, n, a1))
    for b in range(min(a0, a1)):
        L = r.standard_normal((r0, r0))
        R = r.standard_normal((r1, r1))
        M = r.standard_normal((n, n))
        s = 1.0 if b == 0 else 0.0
        PhiL[:, b, :] = L @ L.T / r0 + s * np.eye(r0)
        PhiR[:, b, :] = R @ R.T / r1 + s * np.eye(r1)
        A[b, :, :, b] = M @ M.T / n + s * np.eye(n)
    g = r.standard_normal((r0, n, r1))
    return PhiL, A, PhiR, g


def _dev(a, dt):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).cuda()


def _run(ctx, prec, pre, sysm, x0, rtol, maxit):
    dt = np.float64 if prec == "fp64" else np.float32
    PhiL, A, PhiR, g = (np.asarray(v, dtype=dt) for v in sysm)
    t = [_dev(v, dt) for v in (PhiL, A, PhiR, g)]
    x = _dev(x0, dt)
    r0, n, r1 = g.shape
    its, st = ctx.op_local_cg(prec, pre, r0, n, r1, A.shape[0], A.shape[3], *[v.data_ptr() for v in t],
                              x.data_ptr(), rtol, maxit)
    xs = x.cpu().numpy().astype(np.float64)
    res = g.astype(np.float64) - amen.local_matvec(*(v.astype(np.float64) for v in (PhiL, A, PhiR)), xs)
    gn = np.linalg.norm(g.astype(np.float64))
    return its, st, xs, (np.linalg.norm(res) / gn if gn > 0 else np.linalg.norm(res))


SHAPES = [(5, 4, 7, 9, 11), (33, 8, 20, 23, 17), (1, 2, 4, 1, 43), (12, 4, 70, 6, 5), (2, 8, 3, 5, 20),
          (49, 4, 49, 51, 51)]


@pytest.mark.parametrize("pre", [1, 0])
@pytest.mark.parametrize("shape", SHAPES)
def test_fp64_local_cg_meets_tolerance(ctx, shape, pre):
    sysm = spd_system(sum(shape), *shape)
    x0 = np.zeros(sysm[3].shape)
    its, st, _, rel = _run(ctx, "fp64", pre, sysm, x0, 1e-10, 5000)
    assert st == 1 and 0 < its < 5000, (its, st)
    assert rel <= 1.5e-10, rel


@pytest.mark.parametrize("shape", SHAPES)
def test_fp32_local_cg_meets_tolerance(ctx, shape):
    sysm = spd_system(7 + sum(shape), *shape)
    x0 = W.rng(3).standard_normal(sysm[3].shape) * 0.1
    its, st, _, rel = _run(ctx, "fp32", 1, sysm, x0, 1e-4, 5000)
    assert st == 1 and its > 0, (its, st)
    assert rel <= 2e-4, rel


def test_preconditioner_reduces_iterations(ctx):
    sysm = spd_system(11, 49, 4, 49, 51, 51)
    x0 = np.zeros(sysm[3].shape)
    it_pre, _, _, _ = _run(ctx, "fp64", 1, sysm, x0, 1e-8, 5000)
    it_plain, _, _, _ = _run(ctx, "fp64", 0, sysm, x0, 1e-8, 5000)
    assert it_pre < it_plain, (it_pre, it_plain)


def test_step_limit_and_zero_steps(ctx):
    sysm = spd_system(5, 9, 4, 11, 7, 7)
    x0 = W.rng(8).standard_normal(sysm[3].shape)
    its, st, xs, _ = _run(ctx, "fp64", 1, sysm, x0, 1e-14, 0)
    assert (its, st) == (0, 0) and np.array_equal(xs, x0)
    its, st, xs, _ = _run(ctx, "fp64", 1, sysm, x0, 1e-14, 3)
    assert (its, st) == (3, 0)
    # three steps of CG from x0 reduce the energy-norm error (a property every CG step has)
    PhiL, A, PhiR, g = sysm
    B = lambda v: amen.local_matvec(PhiL, A, PhiR, v)

    def err_energy(x):
        # ||x - x*||_B^2 = x.Bx - 2 g.x + const
        return float(np.sum(x * B(x)) - 2 * np.sum(g * x))

    assert err_energy(xs) < err_energy(x0)


def test_zero_right_hand_side_converges_at_once(ctx):
    sysm = list(spd_system(6, 6, 4, 5, 3, 3))
    sysm[3] = np.zeros_like(sysm[3])
    its, st, xs, _ = _run(ctx, "fp32", 1, sysm, np.zeros(sysm[3].shape), 1e-6, 100)
    assert (its, st) == (0, 1) and not xs.any()


def test_negative_definite_system_reports_breakdown(ctx):
    PhiL, A, PhiR, g = spd_system(4, 6, 4, 5, 3, 3)
    x0 = W.rng(2).standard_normal(g.shape)
    its, st, xs, _ = _run(ctx, "fp64", 0, (PhiL, -A, PhiR, g), x0, 1e-10, 100)
    assert (its, st) == (0, 2) and np.array_equal(xs, x0)


def test_invalid_arguments(ctx, lib):
    t = torch.zeros(64, dtype=torch.float64, device="cuda")
    p = t.data_ptr()
    with pytest.raises(lib.TnfemError):
        ctx.op_local_cg("fp64", 0, 2, 9, 2, 1, 1, p, p, p, p, p, 1e-8, 10)  # mode size above 8
    with pytest.raises(lib.TnfemError):
        ctx.op_local_cg("fp64", 0, 2, 2, 2, 1, 1, p, p, p, p, p, 1e-8, -1)


@pytest.mark.parametrize("precision", ["fp64", "mixed-local"])
def test_fused_and_stepwise_solves_agree(ctx, precision):
    pr = W.steel_plate_2d(levels=6, rank_cap=64, tol=1e-10)
    pr.opts.precision = precision
    A = ctx.stiffness(pr.grid, pr.material)
    f = ctx.load(pr.grid, pr.material, pr.loads)
    sols = {}
    for fused in (True, False):
        pr.opts.fused_cg = fused
        ctx.profile_start(1)
        u, info = ctx.solve(A, f, pr.opts)
        launches = ctx.profile_read("cg32")["launches"] + ctx.profile_read("cg64")["launches"]
        assert info["converged"], info
        assert (launches > 0) == fused, (fused, launches)
        sols[fused] = u
    fa = tt.tt_full(sols[True].cores())
    fb = tt.tt_full(sols[False].cores())
    assert np.linalg.norm(fa - fb) <= 1e-6 * np.linalg.norm(fb)
