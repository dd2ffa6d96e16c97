"""Binary32 contraction engines of the mixed-precision local solves: CUDA-core FMA (engine 0), the
tcgen05 tensor cores with the three-term TF32 split on load-staged operands (engine 1) and on
packed, TMA-fed operands (engine 2, the solver's local matvec), against the binary64 definition on
the same binary32 inputs.

Tolerance: both engines accumulate binary32 products; the split recovers binary32 accuracy from
TF32 words (the dropped a_lo b_lo term is ~2^-22 of |a b|), so every element must agree with the
binary64 value to 2e-5 of the sum of |terms| (a K-term binary32 accumulation stays well inside it
for K up to a few thousand)."""
import numpy as np
import pytest

from oracle import amen
from paper_2501_12151_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

RTOL32 = 2e-5


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_12151_gb300 import tnfem
    return tnfem.Context(0)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


# (M, N, K, batch, A layout, B shared across batches): ragged tails, several 128-row tiles,
# N tiles of 64 and 128, a long K that takes the split-K path, M-major and K-major operands
CASES = [
    (1, 1, 1, 1, "k", False),
    (37, 20, 13, 1, "k", True),
    (300, 200, 70, 1, "m", True),
    (49, 204, 204, 49, "m", True),      # stage 2 of a rank-49 local matvec (rows span batches)
    (2499, 196, 49, 1, "k", True),      # stage 1
    (196, 49, 2499, 1, "k", True),      # stage 3 (split K)
    (64, 96, 40, 3, "k", False),        # per-batch B
]


@pytest.mark.parametrize("engine", [0, 1])
@pytest.mark.parametrize("M,N,K,batch,alay,shared", CASES)
def test_gemm_f32(ctx, engine, M, N, K, batch, alay, shared):
    r = W.rng(100 + M + N + K)
    A = _f32(r.standard_normal((batch, M, K)) if alay == "k" else r.standard_normal((batch, K, M)))
    Bb = 1 if shared else batch
    B = _f32(r.standard_normal((Bb, K, N)))
    C0 = _f32(r.standard_normal((batch, M, N)))
    alpha, beta = 0.75, (0.0 if M % 2 else -0.5)
    if alay == "k":
        sAm, sAk, sAb = K, 1, M * K
        A64 = A.astype(np.float64)
    else:
        sAm, sAk, sAb = 1, M, M * K
        A64 = A.astype(np.float64).transpose(0, 2, 1)
    sBk, sBn, sBb = N, 1, (0 if shared else K * N)
    strides = (sAm, sAk, sAb, sBk, sBn, sBb, N, 1, M * N)
    tA, tB, tC = (torch.from_numpy(v).cuda() for v in (A, B, C0))
    ctx.op_gemm_f32(engine, M, N, K, batch, strides, alpha, tA.data_ptr(), tB.data_ptr(), beta, tC.data_ptr())
    got = tC.cpu().numpy().astype(np.float64)
    B64 = np.broadcast_to(B.astype(np.float64), (batch, K, N))
    ref = alpha * np.matmul(A64, B64) + beta * C0.astype(np.float64)
    scale = abs(alpha) * np.matmul(np.abs(A64), np.abs(B64)) + abs(beta) * np.abs(C0.astype(np.float64))
    assert np.all(np.abs(got - ref) <= RTOL32 * scale + 1e-30)


@pytest.mark.parametrize("engine", [0, 1, 2])
@pytest.mark.parametrize("r0,n,r1,a0,a1", [(5, 4, 7, 9, 11), (49, 4, 49, 51, 51), (33, 8, 20, 23, 17),
                                           (64, 4, 66, 51, 51), (1, 2, 4, 1, 43), (70, 8, 96, 30, 9)])
def test_local_matvec_f32(ctx, engine, r0, n, r1, a0, a1):
    PhiL = _f32(W.rng(1).standard_normal((r0, a0, r0)))
    A = _f32(W.rng(2).standard_normal((a0, n, n, a1)))
    PhiR = _f32(W.rng(3).standard_normal((r1, a1, r1)))
    x = _f32(W.rng(4).standard_normal((r0, n, r1)))
    ref = amen.local_matvec(*(v.astype(np.float64) for v in (PhiL, A, PhiR, x)))
    scale = amen.local_matvec(*(np.abs(v).astype(np.float64) for v in (PhiL, A, PhiR, x)))
    t = [torch.from_numpy(v).cuda() for v in (PhiL, A, PhiR, x)]
    y = torch.zeros(r0 * n * r1, dtype=torch.float32, device="cuda")
    ctx.op_local_matvec_f32(engine, r0, n, r1, a0, a1, *[v.data_ptr() for v in t], y.data_ptr())
    got = y.cpu().numpy().astype(np.float64).reshape(ref.shape)
    # three chained binary32 stages: each rounds once more
    assert np.all(np.abs(got - ref) <= 3 * RTOL32 * scale + 1e-30)
