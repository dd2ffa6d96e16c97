"""The serving loop (continuous batching of solve requests on one GPU).

A mixed set of small requests (2D and 3D, box and general-quadrilateral domains, different levels,
materials, loads and rank caps) is served by three workers.  Each result must equal, to rounding,
the same request served alone by an otherwise idle server with the same worker count (so the same
kernels and grid sizes), and
must meet the solver's accuracy against the oracle's Galerkin solution.  Admission must keep the
admitted estimates within the budget, each request's measured peak memory must stay within its
estimate, and with room for several requests their runs must overlap in time.
"""
import numpy as np
import pytest

from oracle import fem, tt
from paper_2501_12151_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _requests():
    out = []
    p = W.steel_plate_2d(levels=5, rank_cap=32, tol=1e-8, precision="mixed-local")
    out.append(p)
    p = W.manufactured_2d(levels=6, rank_cap=32, tol=1e-9)
    p.opts.precision = "mixed-local"
    out.append(p)
    p = W.cantilever_3d(levels=3, rank_cap=64, tol=1e-8, precision="mixed-local")
    out.append(p)
    p = W.steel_plate_2d(levels=6, rank_cap=64, tol=1e-9, precision="fp64")
    p.material = W.Material(E=(3e9, 3e9), nu=0.42)
    out.append(p)
    p = W.cantilever_paper_2d(levels=5, rank_cap=32, tol=1e-9, precision="mixed-local")
    out.append(p)
    p = W.steel_plate_2d(levels=7, rank_cap=64, tol=1e-8, precision="mixed-local")
    p.loads = [W.Load(kind="traction", face=W.FACE_XHI, traction=(0.0, -2e6, 0.0))]
    out.append(p)
    out.append(W.quad_plate_2d(levels=6, rank_cap=64, tol=1e-9, precision="mixed-local"))
    return out


@pytest.fixture(scope="module")
def tn():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_12151_gb300 import tnfem
    return tnfem


def _dense(cores, pr):
    return tt.to_natural_order(tt.tt_full(cores), pr.grid.dim, pr.grid.levels)


def test_results_same_alone_and_in_the_mix(tn):
    reqs = _requests()
    srv = tn.Server(0, workers=3)
    alone = []
    for pr in reqs:
        rid = srv.submit(pr.grid, pr.material, pr.loads, pr.opts)
        alone.append(srv.wait(rid))
    ids = [srv.submit(pr.grid, pr.material, pr.loads, pr.opts) for pr in reqs]
    mix = [srv.wait(i) for i in ids]
    srv.stop()
    runs = sorted((m[1]["start_us"], m[1]["end_us"]) for m in mix)
    assert any(runs[i + 1][0] < runs[i][1] for i in range(len(runs) - 1)), runs   # they overlapped
    for pr, (ca, da), (cm, dm) in zip(reqs, alone, mix):
        assert da["status"] == dm["status"] and dm["status"] in ("OK", "NOT_CONVERGED"), (pr.name, da, dm)
        assert da["info"]["sweeps"] == dm["info"]["sweeps"], pr.name
        ua, um = _dense(ca, pr), _dense(cm, pr)
        assert np.linalg.norm(um - ua) <= 1e-12 * np.linalg.norm(ua), pr.name
        Abc, fv = fem.system(pr.grid, pr.material, pr.loads, frozen_jacobian=pr.grid.quad is not None)
        uh = fem.solve(Abc, fv)
        err = fem.energy_norm(Abc, um - uh) / fem.energy_norm(Abc, uh)
        bar = 1e-4 if "paper" in pr.name else 1e-6
        assert err <= bar, (pr.name, err, dm["info"])
        assert dm["peak_bytes"] <= dm["est_bytes"], (pr.name, dm["peak_bytes"], dm["est_bytes"])


def test_admission_keeps_estimates_within_budget(tn):
    reqs = [pr for pr in _requests() if pr.grid.dim == 2]
    est = [tn.serve_estimate(pr.grid, pr.opts) for pr in reqs]
    budget = max(est) + sorted(est)[0] // 2   # the largest fits, but never with the smallest beside it
    srv = tn.Server(0, workers=3, hbm_budget=budget)
    assert srv.budget == budget
    ids = [srv.submit(pr.grid, pr.material, pr.loads, pr.opts) for pr in reqs]
    res = [srv.wait(i, take=False)[1] for i in ids]
    srv.stop()
    for r, e in zip(res, est):
        assert r["status"] in ("OK", "NOT_CONVERGED"), r
        assert r["est_bytes"] == e
    # whenever a request started, the estimates of the requests then running fit the budget
    for r in res:
        t = r["start_us"]
        running = [q["est_bytes"] for q in res if q["start_us"] <= t < q["end_us"]]
        assert sum(running) <= budget or len(running) == 1, (running, budget)
    # admitted in arrival order
    starts = [r["start_us"] for r in res]
    assert starts == sorted(starts)


def test_cancel_queued_request_and_stats(tn):
    """A request still waiting for admission can be cancelled (a fault injected on the host: the
    client gives up on a queued request); the running one is not affected, and the queue
    statistics count what waits and what runs."""
    pr = W.steel_plate_2d(levels=8, rank_cap=64, tol=1e-9, precision="mixed-local")
    srv = tn.Server(0, workers=1)
    ids = [srv.submit(pr.grid, pr.material, pr.loads, pr.opts) for _ in range(3)]
    st = srv.stats()
    assert st["queued"] + st["running"] == 3 and st["running"] <= 1
    assert srv.cancel(ids[2])
    assert not srv.cancel(ids[2])                          # already done (cancelled)
    _, info = srv.wait(ids[2], take=False)
    assert info["status"] == "INVALID" and "cancelled" in info["message"]
    first = srv.wait(ids[0], take=False)[1]
    assert first["status"] in ("OK", "NOT_CONVERGED")
    assert not srv.cancel(ids[0])                          # finished: nothing to cancel
    srv.wait(ids[1], take=False)
    assert srv.stats() == {"queued": 0, "running": 0, "admitted_bytes": 0}
    srv.stop()


def test_wait_timeout_and_stop_with_queued_requests(tn):
    pr = W.steel_plate_2d(levels=8, rank_cap=64, tol=1e-9, precision="mixed-local")
    srv = tn.Server(0, workers=1)
    ids = [srv.submit(pr.grid, pr.material, pr.loads, pr.opts) for _ in range(3)]
    with pytest.raises(tn.TnfemError) as e:
        srv.wait(ids[2], timeout_us=1000, take=False)    # still queued after 1 ms
    assert e.value.status == 5
    first = srv.wait(ids[0], take=False)[1]
    assert first["status"] in ("OK", "NOT_CONVERGED") and first["info"]["sweeps"] > 0
    srv.stop()                                            # the rest finish or are refused


def test_nodal_train_loads_are_refused(tn):
    """A request cannot carry a nodal-train load: the train lives in the caller's context and could
    be freed before the request runs, so submit refuses it."""
    pr = W.steel_plate_2d(levels=4, rank_cap=16, tol=1e-8, precision="mixed-local")
    ctx = tn.Context(0)
    rng = np.random.default_rng(0)
    f0 = ctx.tt_import([rng.standard_normal((1, 2, 2))] + [rng.standard_normal((2, 4, 2)) for _ in range(3)] +
                       [rng.standard_normal((2, 4, 1))])
    srv = tn.Server(0, workers=1)
    try:
        with pytest.raises(tn.TnfemError):
            srv.submit(pr.grid, pr.material, [W.Load(kind="nodal", nodal=f0)], pr.opts)
    finally:
        srv.stop()
