"""Failure detection and the boundary's error paths, without faulting the GPU.

Device side: a bounded grid-barrier wait is made to run out on purpose (one CTA arrives later
than the bound) and the call must come back with TNFEM_E_TIMEOUT, after which the same context
still solves.  Host side: an allocation callback that fails, a device-memory budget that is too
small, a NaN planted in an imported load core, and a solve time limit, each through the C ABI,
each followed by a successful call on the same context.
"""
import numpy as np
import pytest

from paper_2501_12151_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def tn():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_12151_gb300 import tnfem
    return tnfem


def _small(tn, ctx, levels=5):
    pr = W.steel_plate_2d(levels=levels, rank_cap=32, tol=1e-8, precision="fp64")
    return pr, ctx.stiffness(pr.grid, pr.material), ctx.load(pr.grid, pr.material, pr.loads)


def test_grid_barrier_timeout_is_reported_and_context_survives(tn):
    ctx = tn.Context(0)
    assert ctx.barrier_probe(8, -1, 0.0, 50.0) == 0           # nobody late: three barriers pass
    assert ctx.barrier_probe(8, 3, 60.0, 5.0) == 5            # CTA 3 is 60 ms late, bound 5 ms
    assert "barrier" in tn.lib.tnfem_last_error(ctx.h).decode()
    assert ctx.barrier_probe(16, 0, 1.0, 200.0) == 0          # late but within the bound
    pr, A, f = _small(tn, ctx)
    u, info = ctx.solve(A, f, pr.opts)
    assert info["converged"] == 1


def test_allocation_callback_failure_is_nomem(tn):
    state = {"left": 10 ** 9, "live": {}}

    def alloc(nbytes):
        if state["left"] <= 0:
            return 0
        state["left"] -= 1
        t = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        state["live"][t.data_ptr()] = t
        return t.data_ptr()

    def free(ptr):
        state["live"].pop(ptr, None)

    ctx = tn.Context(0, alloc_hook=alloc, free_hook=free)
    pr, A, f = _small(tn, ctx)
    u, info = ctx.solve(A, f, pr.opts)      # warm: the operator's derived copies are cached on A
    del u
    held, _ = ctx.memory_stats()
    state["left"] = 3                       # the solve needs many more buffers than this
    with pytest.raises(tn.TnfemError) as e:
        ctx.solve(A, f, pr.opts)
    assert e.value.status == 2              # TNFEM_E_NOMEM
    assert ctx.memory_stats()[0] == held    # the failed solve released what it had taken
    state["left"] = 10 ** 9
    u, info = ctx.solve(A, f, pr.opts)
    assert info["converged"] == 1


def test_hbm_budget_is_enforced_and_recoverable(tn):
    ctx = tn.Context(0)
    pr, A, f = _small(tn, ctx, levels=6)
    u, info = ctx.solve(A, f, pr.opts)      # warm: the operator's derived copies are cached on A
    del u
    held, _ = ctx.memory_stats(reset_peak=True)
    ctx.set_hbm_budget(held + (64 << 10))   # 64 KiB of headroom: far below what a solve needs
    with pytest.raises(tn.TnfemError) as e:
        ctx.solve(A, f, pr.opts)
    assert e.value.status == 6              # TNFEM_E_BUDGET
    assert ctx.memory_stats()[0] == held    # everything the failed solve took was returned
    ctx.set_hbm_budget(0)
    u, info = ctx.solve(A, f, pr.opts)
    assert info["converged"] == 1
    _, peak = ctx.memory_stats()
    assert peak > held
    # a budget at the measured peak admits the same solve again
    del u
    ctx.set_hbm_budget(peak)
    u, info = ctx.solve(A, f, pr.opts)
    assert info["converged"] == 1


@pytest.mark.parametrize("precision", ["fp64", "mixed-local", "mixed"])
def test_nan_in_imported_load_is_numeric(tn, precision):
    ctx = tn.Context(0)
    pr, A, f = _small(tn, ctx)
    cores = f.cores()
    cores[3] = cores[3].copy()
    cores[3].flat[cores[3].size // 2] = np.nan
    fbad = ctx.tt_import(cores)
    o = W.steel_plate_2d(levels=5, rank_cap=32, tol=1e-8, precision=precision).opts
    with pytest.raises(tn.TnfemError) as e:
        ctx.solve(A, fbad, o)
    assert e.value.status == 7              # TNFEM_E_NUMERIC
    u, info = ctx.solve(A, f, o)
    assert info["converged"] == 1


def test_solve_time_limit(tn):
    ctx = tn.Context(0)
    pr, A, f = _small(tn, ctx, levels=7)
    pr.opts.tol = 1e-12
    pr.opts.timeout_us = 1                  # expires after the first core step
    u, info = ctx.solve(A, f, pr.opts)
    assert info["status"] == "TIMEOUT" and info["sweeps"] == 1, info
    assert len(u.cores()) == 8              # the last iterate is a complete train
    pr.opts.timeout_us = 0                  # without the limit the same context sweeps on
    pr.opts.tol = 1e-8
    pr.opts.max_sweeps = 6
    u, info = ctx.solve(A, f, pr.opts)
    assert info["status"] in ("OK", "NOT_CONVERGED") and info["sweeps"] > 1, info


def test_mixed_tf32_precision_value(tn):
    """TNFEM_MIXED_TF32 is MIXED_LOCAL with the binary32 local matvecs on tcgen05."""
    from oracle import fem, tt
    ctx = tn.Context(0)
    pr = W.steel_plate_2d(levels=5, rank_cap=32, tol=1e-10, precision="mixed-tf32")
    pr.opts.fused_cg = False                # the tensor-core matvec runs in the launch-per-step engine
    A = ctx.stiffness(pr.grid, pr.material)
    f = ctx.load(pr.grid, pr.material, pr.loads)
    u, info = ctx.solve(A, f, pr.opts)
    Abc, fv = fem.system(pr.grid, pr.material, pr.loads)
    uh = fem.solve(Abc, fv)
    ud = tt.to_natural_order(tt.tt_full(u.cores()), 2, 5)
    err = fem.energy_norm(Abc, ud - uh) / fem.energy_norm(Abc, uh)
    assert info["converged"] == 1 and err <= 1e-6, (err, info)
