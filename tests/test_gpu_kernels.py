"""GPU parity of the single sweep steps against the CPU oracle, element by element, on seeded
inputs that span several GEMM tiles and ragged tails: local matvec (a4), environment update
(a2/a8), QR and SVD (a6/a7 building blocks), TT rounding (a11), operator-times-train, inner
products, norms and the energy norm of a difference (A13)."""
import numpy as np
import pytest

from oracle import amen, tt
from paper_2501_12151_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_12151_gb300 import tnfem
    return tnfem.Context(0)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


# binary64 contractions of length K: rounding error well below 1e-13 relative to |terms|
RTOL = 1e-12


def contract(spec, *ops):
    """numpy.einsum along a pairwise path chosen without a memory cap (the default cap can force a
    single loop over every index at once, which does not finish at these sizes)."""
    path = np.einsum_path(spec, *ops, optimize=("greedy", 1e13))[0]
    return np.einsum(spec, *ops, optimize=path)


@pytest.mark.parametrize("r0,n,r1,a0,a1", [(1, 2, 3, 1, 4), (5, 4, 7, 9, 11), (67, 4, 64, 51, 51),
                                           (70, 8, 33, 23, 17), (13, 4, 1, 5, 1)])
def test_local_matvec(ctx, r0, n, r1, a0, a1):
    PhiL = W.rng(1).standard_normal((r0, a0, r0))
    A = W.rng(2).standard_normal((a0, n, n, a1))
    PhiR = W.rng(3).standard_normal((r1, a1, r1))
    x = W.rng(4).standard_normal((r0, n, r1))
    ref = amen.local_matvec(PhiL, A, PhiR, x)
    y = torch.zeros(r0 * n * r1, dtype=torch.float64, device="cuda")
    tPL, tA, tPR, tx = dev(PhiL), dev(A), dev(PhiR), dev(x)
    ctx.op_local_matvec(r0, n, r1, a0, a1, tPL.data_ptr(), tA.data_ptr(), tPR.data_ptr(), tx.data_ptr(), y.data_ptr())
    got = y.cpu().numpy().reshape(ref.shape)
    scale = contract("pba,bijc,sct,ajt->pis", np.abs(PhiL), np.abs(A), np.abs(PhiR), np.abs(x))
    assert np.all(np.abs(got - ref) <= RTOL * scale + 1e-300)


@pytest.mark.parametrize("ry0,ry1,rx0,rx1,n,a0,a1", [(1, 2, 1, 2, 2, 1, 6), (4, 7, 5, 9, 4, 13, 11),
                                                     (64, 66, 64, 68, 4, 51, 51), (3, 4, 40, 70, 8, 9, 30)])
def test_env_left(ctx, ry0, ry1, rx0, rx1, n, a0, a1):
    Phi = W.rng(5).standard_normal((ry0, a0, rx0))
    y = W.rng(6).standard_normal((ry0, n, ry1))
    A = W.rng(7).standard_normal((a0, n, n, a1))
    x = W.rng(8).standard_normal((rx0, n, rx1))
    ref = contract("pba,pis,bijc,ajt->sct", Phi, y, A, x)
    out = torch.zeros(ry1 * a1 * rx1, dtype=torch.float64, device="cuda")
    t = [dev(v) for v in (Phi, y, A, x)]
    ctx.op_env_left(ry0, ry1, rx0, rx1, n, a0, a1, t[0].data_ptr(), t[1].data_ptr(), t[2].data_ptr(),
                    t[3].data_ptr(), out.data_ptr())
    got = out.cpu().numpy().reshape(ref.shape)
    scale = contract("pba,pis,bijc,ajt->sct", np.abs(Phi), np.abs(y), np.abs(A), np.abs(x))
    assert np.all(np.abs(got - ref) <= RTOL * scale)


# Paths: n >= 16 with the columns in a cluster's shared memory -> qr_cluster_kernel ((272, 68),
# (64, 64), (1056, 136), (1152, 72)); m >= 8n, n >= 16 and columns longer than 3200 -> the
# tall-skinny QR (blocks of 2n rows, one CTA each, recursively: (4608, 53), (9001, 150) with a
# ragged last block, (28224, 441) the 3D operator rounding's unfolding); other tall matrices ->
# the blocked one-CTA kernel ((16384, 4), (16385, 4)); small or wide ones -> the row-major kernel.
@pytest.mark.parametrize("m,n", [(1, 1), (7, 3), (3, 7), (272, 68), (64, 64), (1056, 136), (1152, 72),
                                 (4608, 53), (9001, 150), (28224, 441), (16384, 4), (16385, 4), (40, 100)])
def test_qr(ctx, m, n):
    A = W.random_matrix(9, m, n)
    k = min(m, n)
    Q = torch.zeros(m * k, dtype=torch.float64, device="cuda")
    R = torch.zeros(k * n, dtype=torch.float64, device="cuda")
    tA = dev(A)
    ctx.op_qr(m, n, tA.data_ptr(), Q.data_ptr(), R.data_ptr())
    Qh = Q.cpu().numpy().reshape(m, k)
    Rh = R.cpu().numpy().reshape(k, n)
    assert np.abs(Qh @ Rh - A).max() <= 1e-13 * np.abs(A).max() * max(m, n)
    assert np.abs(Qh.T @ Qh - np.eye(k)).max() <= 1e-13 * max(m, n)
    assert np.abs(np.tril(Rh, -1)).max() == 0.0
    # R agrees with numpy's up to the sign of each row (the factorisation is unique otherwise)
    Rn = np.linalg.qr(A)[1][:k]
    sgn = np.sign(np.diag(Rh)) * np.sign(np.diag(Rn))
    np.testing.assert_allclose(sgn[:, None] * Rh, Rn, atol=1e-12 * np.abs(A).max() * max(m, n))


@pytest.mark.parametrize("m,n", [(300, 40), (1152, 72), (30, 30), (6000, 120)])
def test_qr_rank_deficient(ctx, m, n):
    """Columns that repeat earlier ones, a zero column and a zero first column: Q keeps orthonormal
    columns and Q R reproduces A (the Householder steps with a vanishing tail take tau = 0)."""
    B = W.random_matrix(4, m, n // 2)
    A = np.concatenate([B, B[:, : n - n // 2]], axis=1)
    A[:, 0] = 0.0
    A[:, n // 3] = 0.0
    Q = torch.zeros(m * n, dtype=torch.float64, device="cuda")
    R = torch.zeros(n * n, dtype=torch.float64, device="cuda")
    ctx.op_qr(m, n, dev(A).data_ptr(), Q.data_ptr(), R.data_ptr())
    Qh = Q.cpu().numpy().reshape(m, n)
    Rh = R.cpu().numpy().reshape(n, n)
    assert np.abs(Qh @ Rh - A).max() <= 1e-13 * np.abs(A).max() * m
    assert np.abs(Qh.T @ Qh - np.eye(n)).max() <= 1e-13 * m
    assert np.abs(np.tril(Rh, -1)).max() == 0.0


# binary64 GEMM engines: 0 binary64 FMA, 1 double-binary32 (hi/lo binary32 pairs; the
# mixed-precision sweep's route for large contractions).  Error bounds relative to the sum of
# |terms|: binary64 K * 2^-52, double-binary32 K * 2^-45 (its products and sums keep ~47 bits).
GEMM64_CASES = [
    (49, 204, 204, 49, "m", True),     # stage 2 of the working-shape local matvec (rows span batches)
    (2499, 196, 49, 1, "k", True),     # stage 1
    (196, 49, 2499, 1, "k", True),     # stage 3 (split K)
    (300, 200, 70, 1, "m", True),
    (64, 96, 40, 3, "k", False),       # per-batch B (below the 2^20 threshold: binary64 either way)
    (130, 257, 260, 2, "k", False),
]


@pytest.mark.parametrize("engine", [0, 1])
@pytest.mark.parametrize("M,N,K,batch,alay,shared", GEMM64_CASES)
def test_gemm_f64_engines(ctx, engine, M, N, K, batch, alay, shared):
    r = W.rng(200 + M + N + K)
    A = r.standard_normal((batch, M, K)) if alay == "k" else r.standard_normal((batch, K, M))
    Bb = 1 if shared else batch
    # magnitudes of the sweep's operands (environments ~1e11, cores ~1), signed
    B = r.standard_normal((Bb, K, N)) * 1e5
    C0 = r.standard_normal((batch, M, N))
    alpha, beta = 1.25, (0.0 if M % 2 else -0.5)
    if alay == "k":
        sAm, sAk, sAb = K, 1, M * K
        Am = A
    else:
        sAm, sAk, sAb = 1, M, M * K
        Am = A.transpose(0, 2, 1)
    sBk, sBn, sBb = N, 1, (0 if shared else K * N)
    strides = (sAm, sAk, sAb, sBk, sBn, sBb, N, 1, M * N)
    tA, tB, tC = (dev(v) for v in (A, B, C0))
    ctx.op_gemm_f64(engine, M, N, K, batch, strides, alpha, tA.data_ptr(), tB.data_ptr(), beta, tC.data_ptr())
    got = tC.cpu().numpy()
    Bf = np.broadcast_to(B, (batch, K, N))
    ref = alpha * np.matmul(Am, Bf) + beta * C0
    scale = abs(alpha) * np.matmul(np.abs(Am), np.abs(Bf)) + abs(beta) * np.abs(C0)
    tol = K * (2.0 ** -52 if engine == 0 else 2.0 ** -45)
    assert np.all(np.abs(got - ref) <= tol * scale + 1e-300)


def test_gemm_f64_df_out_of_range(ctx):
    from paper_2501_12151_gb300 import tnfem
    # products beyond the binary32 range are reported, not returned as garbage
    M, N, K = 128, 128, 128
    A = np.full((M, K), 1e25)
    B = np.full((K, N), 1e25)
    Cm = torch.zeros(M * N, dtype=torch.float64, device="cuda")
    strides = (K, 1, M * K, N, 1, K * N, N, 1, M * N)
    with pytest.raises(tnfem.TnfemError):
        ctx.op_gemm_f64(1, M, N, K, 1, strides, 1.0, dev(A).data_ptr(), dev(B).data_ptr(), 0.0, Cm.data_ptr())
    ctx.op_gemm_f64(0, M, N, K, 1, strides, 1.0, dev(A).data_ptr(), dev(B).data_ptr(), 0.0, Cm.data_ptr())
    assert np.allclose(Cm.cpu().numpy(), 128e50)


def _qr_ext(ctx, A, rk, w):
    m = A.shape[0]
    ld = rk + w
    Q = torch.zeros(m * ld, dtype=torch.float64, device="cuda")
    R = torch.zeros(ld * ld, dtype=torch.float64, device="cuda")
    tA = dev(A)
    ctx.op_qr_ext(m, rk, w, tA.data_ptr(), Q.data_ptr(), R.data_ptr())
    return Q.cpu().numpy().reshape(m, ld), R.cpu().numpy().reshape(ld, ld)


# [U | W] with U orthonormal (the enrichment's basis): shapes of the sweep (m = r0 n, rk + kick)
# and ragged ones; W general, W inside span(U) (the Householder fallback) and W partly inside
@pytest.mark.parametrize("m,rk,w", [(196, 49, 4), (5, 1, 4), (36, 31, 4), (288, 72, 4), (64, 60, 4), (9, 2, 3)])
@pytest.mark.parametrize("kind", ["general", "in_span", "partly"])
def test_qr_ext(ctx, m, rk, w, kind):
    r = W.rng(31 + m + rk)
    U, _ = np.linalg.qr(r.standard_normal((m, rk)))
    Wm = r.standard_normal((m, w))
    if kind == "in_span":
        Wm = U @ r.standard_normal((rk, w))
    elif kind == "partly":
        Wm[:, 0] = U @ r.standard_normal(rk)
    A = np.hstack([U, Wm])
    Qh, Rh = _qr_ext(ctx, A, rk, w)
    ld = rk + w
    scale = np.abs(A).max() * m
    assert np.abs(Qh.T @ Qh - np.eye(ld)).max() <= 1e-12, kind
    assert np.abs(Qh @ Rh - A).max() <= 1e-13 * scale, kind
    assert np.abs(np.tril(Rh, -1)).max() <= 1e-13 * scale
    # the span of [U | W] is kept: every column of A lies in span(Q)
    assert np.abs(Qh @ (Qh.T @ A) - A).max() <= 1e-12 * scale


# (1, 1), (9, 4): one CTA; (196, 49), (100, 16), (64, 63), (300, 33), (49, 49): one thread-block
# cluster (16 <= n <= 64); (272, 68), (68, 68), (512, 128), (848, 72): the cooperative multi-CTA
# kernel; (5200, 40): columns too long for the cluster's shared memory, the cooperative kernel
@pytest.mark.parametrize("m,n", [(1, 1), (9, 4), (196, 49), (100, 16), (64, 63), (300, 33), (49, 49),
                                 (272, 68), (68, 68), (512, 128), (848, 72), (5200, 40)])
def test_svd(ctx, m, n):
    r = W.rng(11)
    # graded singular values down to 1e-12 to exercise the truncation range
    U0, _ = np.linalg.qr(r.standard_normal((m, n)))
    V0, _ = np.linalg.qr(r.standard_normal((n, n)))
    s0 = np.logspace(0, -12, n)
    A = (U0 * s0) @ V0.T
    U = torch.zeros(m * n, dtype=torch.float64, device="cuda")
    S = torch.zeros(n, dtype=torch.float64, device="cuda")
    Vt = torch.zeros(n * n, dtype=torch.float64, device="cuda")
    tA = dev(A)
    ctx.op_svd(m, n, tA.data_ptr(), U.data_ptr(), S.data_ptr(), Vt.data_ptr())
    Uh, Sh, Vh = U.cpu().numpy().reshape(m, n), S.cpu().numpy(), Vt.cpu().numpy().reshape(n, n)
    np.testing.assert_allclose(Sh, np.linalg.svd(A, compute_uv=False), rtol=1e-10, atol=1e-15)
    assert np.all(np.diff(Sh) <= 0)
    assert np.abs((Uh * Sh) @ Vh - A).max() <= 1e-13 * max(m, n)
    assert np.abs(Vh @ Vh.T - np.eye(n)).max() <= 1e-12
    # sign convention: the largest-magnitude entry of each left singular vector is positive
    for j in range(n):
        if Sh[j] > 1e-10:
            col = Uh[:, j]
            assert col[np.argmax(np.abs(col))] > 0


@pytest.mark.parametrize("modes,ranks,eps", [([2, 4, 4, 4, 4], [1, 2, 5, 7, 3, 1], 1e-14),
                                              ([3, 8, 8, 8], [1, 3, 11, 6, 1], 1e-6),
                                              ([2] + [4] * 7, [1, 2, 8, 16, 20, 16, 8, 4, 1], 1e-10)])
def test_tt_round_matches_oracle(ctx, modes, ranks, eps):
    x = W.random_tt(13, modes, ranks)
    # make it redundant: x + x*0.5 then round
    X = ctx.tt_import(tt.tt_add(x, x, 0.5))
    Y = X.round(eps)
    y = Y.cores()
    ref = tt.tt_round(tt.tt_add(x, x, 0.5), eps)
    full_ref = tt.tt_full(tt.tt_add(x, x, 0.5))
    assert tt.ranks(y) == tt.ranks(ref)
    err = np.linalg.norm(tt.tt_full(y) - full_ref)
    assert err <= max(eps, 1e-13) * np.linalg.norm(full_ref) * 1.0001
    np.testing.assert_allclose(tt.tt_full(y), tt.tt_full(ref), atol=1e-12 * np.abs(full_ref).max() + 2 * eps * np.linalg.norm(full_ref))


def test_axpy_dot_norm_apply(ctx):
    x = W.random_tt(21, [2, 4, 4, 4], [1, 2, 3, 2, 1])
    y = W.random_tt(22, [2, 4, 4, 4], [1, 2, 2, 3, 1])
    A = W.random_mpo(23, [2, 4, 4, 4], [1, 3, 4, 2, 1])
    X, Y, Am = ctx.tt_import(x), ctx.tt_import(y), ctx.mpo_import(A)
    np.testing.assert_allclose(tt.tt_full(X.axpy(-0.7, Y).cores()), tt.tt_full(x) - 0.7 * tt.tt_full(y), atol=1e-12)
    assert X.dot(Y) == pytest.approx(float(tt.tt_full(x) @ tt.tt_full(y)), rel=1e-12)
    assert X.norm() == pytest.approx(np.linalg.norm(tt.tt_full(x)), rel=1e-13)
    np.testing.assert_allclose(tt.tt_full(Am.apply(X).cores()), tt.mpo_full(A) @ tt.tt_full(x), rtol=1e-12, atol=1e-10)


def test_energy_norm_of_tiny_difference(ctx):
    """||u - v||_A for v = u + 1e-9 w must come out near 1e-9 ||w||_A (no squared cancellation)."""
    from oracle import mpo as ompo
    pr = W.steel_plate_2d(levels=3)
    A, _ = ompo.stiffness_mpo(pr.grid, pr.material)
    u = W.random_tt(31, W.qtt_modes(2, 3), [1, 2, 4, 3, 1])
    w = W.random_tt(32, W.qtt_modes(2, 3), [1, 2, 2, 2, 1])
    v = tt.tt_add(u, w, 1e-9)
    Ad = tt.mpo_full(A)
    wd = tt.tt_full(w)
    ref = 1e-9 * np.sqrt(wd @ Ad @ wd)
    Am, U, V = ctx.mpo_import(A), ctx.tt_import(u), ctx.tt_import(v)
    assert Am.energy_norm(U, V) == pytest.approx(ref, rel=1e-6)
    ud = tt.tt_full(u)
    assert Am.energy_norm(U) == pytest.approx(np.sqrt(ud @ Ad @ ud), rel=1e-12)
