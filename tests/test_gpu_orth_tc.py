"""Tensor-core orthonormalisation (rSVD steps 2 and 4, Sec. 2.1) of the mixed
mode: CholeskyQR2 with tcgen05 Gram products and triangular applies in
error-corrected TF32, and its fall-back to Gram-Schmidt applied twice for
ill-conditioned sketches.  Checked against the FP64 oracle's randomized SVD
(the coarse operators G_n' on probe vectors, as for the other mixed builds)
and against the same build with the tensor-core path switched off."""
import numpy as np
import pytest

from paper_2508_08873_gb300 import api, workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = api.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def orc():
    from oracle import oracle
    return oracle


def _operator(U, S, V):
    return U.T @ np.diag(S) @ V


def _build(ctx, op, P, tc):
    try:
        ctx.set_param("orth_tc", tc)
        return api.Coarse(ctx, op, P.dt, P.M, P.N, P.R, P.p, P.seed, prec="mixed")
    finally:
        ctx.set_param("orth_tc", 1)


@pytest.mark.parametrize("R,p,n,N,M", [(8, 4, 1023, 16, 64), (32, 10, 1023, 128, 8),
                                        (16, 8, 4095, 64, 256), (48, 16, 1023, 256, 4),
                                        (1, 1, 1023, 16, 64), (1, 0, 511, 8, 32)])
def test_tensor_core_orth_matches_oracle_and_cgs2(ctx, orc, R, p, n, N, M):
    """Sketch widths 12, 42 (two K blocks of the apply), 24 (the full
    advection-diffusion-reaction configuration), 64 (the widest: N = 64 of
    the MMAs, two K blocks) and the degenerate widths 2 and 1, with spectra
    that decay slowly enough for CholeskyQR2: every interval takes the
    tensor-core path, and on sampled intervals its coarse operators are
    within 1e-4 sigma_1 of the FP64 oracle's and within 2e-5 sigma_1 of the
    Gram-Schmidt build."""
    P = W.adr1d(n=n, N=N, M=M, R=R, p=p)
    op = api.Operator.tridiag(ctx, P.lo, P.di, P.up)
    co = _build(ctx, op, P, 1)
    ref = _build(ctx, op, P, 0)
    assert co.orth_method() == {"tc_w": P.N, "tc_v": P.N}
    assert ref.orth_method() == {"tc_w": 0, "tc_v": 0}
    inf, rinf = co.info(), ref.info()
    assert np.all(inf["rank_w"] == R + p) and np.all(inf["rank_v"] == R + p)
    oop = orc.Tridiag(P.lo, P.di, P.up)
    probes = np.random.default_rng(3).standard_normal((3, P.n))
    for i in sorted({0, 1, P.N // 2, P.N - 1}):
        oc = orc.rsvd_interval(oop, P.dt, P.M, i, P.R, P.p, P.seed)
        s1 = oc.sigma[0]
        G = _operator(*co.factors(i))
        Go = oc.U @ np.diag(oc.S) @ oc.V.T
        Gr = _operator(*ref.factors(i))
        for x in probes:
            assert np.linalg.norm((G - Go) @ x) <= 1e-4 * s1 * np.linalg.norm(x)
            assert np.linalg.norm((G - Gr) @ x) <= 2e-5 * s1 * np.linalg.norm(x)
        assert np.max(np.abs(inf["sigma"][i] - oc.sigma)) <= 1e-4 * s1
        assert np.max(np.abs(inf["sigma"][i] - rinf["sigma"][i])) <= 2e-5 * s1


def test_tensor_core_orth_falls_back_on_rank_deficient_sketches(ctx):
    """heat1d: sigma_9 / sigma_1 ~ 1e-16, so the sketches are numerically rank
    deficient; the conditioning test sends every interval to Gram-Schmidt
    with deflation and the build equals the one with the path switched off."""
    P = W.heat1d()
    op = api.Operator.tridiag(ctx, P.lo, P.di, P.up)
    co = _build(ctx, op, P, 1)
    ref = _build(ctx, op, P, 0)
    assert co.orth_method() == {"tc_w": 0, "tc_v": 0}
    a, b = co.info(), ref.info()
    assert np.array_equal(a["rank_w"], b["rank_w"]) and np.array_equal(a["rank_v"], b["rank_v"])
    np.testing.assert_array_equal(a["sigma"], b["sigma"])


def test_tensor_core_orth_parareal_to_tolerance(ctx, orc):
    """A mixed-mode Parareal solve on coarse solvers built on the tensor cores
    reaches the oracle's sequential FP64 fine solution to 1e-8."""
    P = W.adr1d(n=1023, N=16, M=64, R=8, p=4)
    op = api.Operator.tridiag(ctx, P.lo, P.di, P.up)
    co = _build(ctx, op, P, 1)
    assert co.orth_method()["tc_w"] == P.N
    u, info = api.parareal_solve(ctx, co, P.u0, K=P.N, tol=1e-9)
    ref = orc.sequential_fine(orc.Tridiag(P.lo, P.di, P.up), P.dt, P.M, P.N, P.u0)
    assert info["converged"]
    assert orc.rel_err(u, ref) <= 1e-8


def _adv2d_ops(ctx, Ps):
    ops = []
    for P in Ps:
        op = api.Operator.stencil5(ctx, P.mx, P.my, P.st)
        op.set_krylov(1e-14, 1e-6, 20000)
        ops.append(op)
    return ops


def test_tensor_core_orth_2d_mixed_matches_oracle(ctx, orc):
    """2D advection-diffusion (31^2 grid, dt = 1/2048, R = 8, p = 4, FP32
    Jacobi-BiCGStab sketches to rtol 1e-6): every interval's bases come from
    the tensor-core CholeskyQR2, and the coarse operators of sampled
    intervals are within 1e-4 sigma_1 of the FP64 oracle's."""
    P = W.adv2d(0, m=31, N=32, M=64, R=8, p=4)
    op, = _adv2d_ops(ctx, [P])
    co = api.Coarse(ctx, op, P.dt, P.M, P.N, P.R, P.p, P.seed, prec="mixed")
    assert co.orth_method() == {"tc_w": P.N, "tc_v": P.N}
    oop = orc.Stencil5(P.mx, P.my, P.st["C"], P.st["W"], P.st["E"], P.st["S"], P.st["N"])
    probes = np.random.default_rng(5).standard_normal((3, P.n))
    inf = co.info()
    for i in (0, 13, P.N - 1):
        oc = orc.rsvd_interval(oop, P.dt, P.M, i, P.R, P.p, P.seed)
        s1 = oc.sigma[0]
        G = _operator(*co.factors(i))
        Go = oc.U @ np.diag(oc.S) @ oc.V.T
        for x in probes:
            assert np.linalg.norm((G - Go) @ x) <= 1e-4 * s1 * np.linalg.norm(x)
        assert np.max(np.abs(inf["sigma"][i] - oc.sigma)) <= 1e-4 * s1


def test_tensor_core_orth_in_captured_batch_build(ctx):
    """The batched build of uneven 2D problems captures its whole build,
    tensor-core orthonormalisation and lift included, in one CUDA graph; each
    problem's coarse solver equals its separate mixed build to FP32 accuracy
    and used the tensor-core path for every interval."""
    grids = (31, 23, 31)
    Ps = [W.adv2d(i, m=m, N=32, M=64, R=8, p=4) for i, m in enumerate(grids)]
    ops = _adv2d_ops(ctx, Ps)
    P0 = Ps[0]
    cos = api.build_coarse_batch(ctx, ops, P0.dt, P0.M, P0.N, P0.R, P0.p, 0, prec="mixed")
    probes = np.random.default_rng(9).standard_normal((2, max(P.n for P in Ps)))
    for P, op, co in zip(Ps, ops, cos):
        single = api.Coarse(ctx, op, P.dt, P.M, P.N, P.R, P.p, 0, prec="mixed")
        assert co.orth_method() == {"tc_w": P.N, "tc_v": P.N}
        assert single.orth_method() == {"tc_w": P.N, "tc_v": P.N}
        a, b = co.info(), single.info()
        s1 = b["sigma"].max()
        np.testing.assert_allclose(a["sigma"], b["sigma"], rtol=0, atol=1e-5 * s1)
        for i in (0, P.N - 1):
            G, Gs = _operator(*co.factors(i)), _operator(*single.factors(i))
            for x in probes:
                xx = x[:P.n]
                assert np.linalg.norm((G - Gs) @ xx) <= 1e-5 * s1 * np.linalg.norm(xx)
