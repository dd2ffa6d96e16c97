"""The allocation-free local matvec (tnfem_op_local_matvec_noalloc) against the regular entry
point, through the C ABI.

Some callers cannot call cudaMalloc: code running inside a CUDA stream capture that must not grow
the memory pool, a host framework that owns the device allocator, a real-time loop that must not
block on the driver.  The no-alloc variant serves them from the library's static device scratch
array; it must give the same contraction as tnfem_op_local_matvec, and a second call must not see
anything left over from the first (the array keeps the previous call's contents).

This file is named to be collected last, so a run that stops at the first failure has already run
every other test; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

from oracle import amen
from paper_2501_12151_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# binary64 contractions; the same bound as the regular entry point's parity test
RTOL = 1e-12


def _contract_abs(PhiL, A, PhiR, x):
    return amen.local_matvec(np.abs(PhiL), np.abs(A), np.abs(PhiR), np.abs(x))


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_12151_gb300 import tnfem
    return tnfem


def _inputs(seed, r0, n, r1, a0, a1):
    PhiL = W.rng(seed).standard_normal((r0, a0, r0))
    A = W.rng(seed + 1).standard_normal((a0, n, n, a1))
    PhiR = W.rng(seed + 2).standard_normal((r1, a1, r1))
    x = W.rng(seed + 3).standard_normal((r0, n, r1))
    return PhiL, A, PhiR, x


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def test_noalloc_matvec_matches_regular_entry_point_twice(lib):
    ctx = lib.Context(0)
    stream = torch.cuda.current_stream().cuda_stream
    # two calls in a row with different shapes and data: the second overwrites the shared scratch
    for seed, shape in ((11, (67, 4, 64, 51, 51)), (21, (13, 8, 29, 9, 17))):
        r0, n, r1, a0, a1 = shape
        PhiL, A, PhiR, x = _inputs(seed, *shape)
        t = [_dev(v) for v in (PhiL, A, PhiR, x)]
        y_ref = torch.zeros(r0 * n * r1, dtype=torch.float64, device="cuda")
        y_new = torch.full((r0 * n * r1,), np.nan, dtype=torch.float64, device="cuda")
        ctx.op_local_matvec(r0, n, r1, a0, a1, *[v.data_ptr() for v in t], y_ref.data_ptr())
        lib.op_local_matvec_noalloc(stream, r0, n, r1, a0, a1, *[v.data_ptr() for v in t], y_new.data_ptr())
        torch.cuda.synchronize()
        ref = y_ref.cpu().numpy()
        got = y_new.cpu().numpy()
        scale = _contract_abs(PhiL, A, PhiR, x).reshape(-1)
        assert np.all(np.isfinite(got))
        assert np.all(np.abs(got - ref) <= RTOL * scale + 1e-300)


def test_noalloc_rejects_sizes_beyond_the_scratch(lib):
    big = 1 << 12  # a0 * n * n * a1 alone exceeds the static array
    p = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(lib.TnfemError) as ei:
        lib.op_local_matvec_noalloc(0, 1, 8, 1, big, big, *([p.data_ptr()] * 5))
    assert ei.value.status == 1
