"""GPU parity of the 2D (5-point stencil) hot path against the FP64 oracle.

The per-step solves are Krylov (CG for the symmetric diffusion operator,
BiCGStab for the upwind advection-diffusion operator); the oracle solves every
step with a banded LU.  Parity tests tighten the Krylov tolerance to 1e-14 so
that the comparison is limited by rounding, and compare at 1e-10 relative L2
(FP64); the FP32 path is compared at the tolerance its rtol 1e-6 allows.
Grids: 15^2 .. 255^2, so that one-CTA and multi-CTA cluster systems are both
exercised.
"""
import numpy as np
import pytest

from paper_2508_08873_gb300 import _native, api, workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    return api.Context(0)


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _problem(kind, m):
    if kind == "diff":
        st = W.diff2d_op(m, 10 ** np.random.default_rng(0).uniform(0, 2, (8, 8)))
    else:
        st = W.adv2d_op(m, 0.01)
    return st


def _ops(ctx, orc, kind, m, rtol64=1e-14, rtol32=1e-6):
    st = _problem(kind, m)
    op = api.Operator.stencil5(ctx, m, m, st)
    op.set_krylov(rtol64, rtol32, 20000)
    oop = orc.Stencil5(m, m, st["C"], st["W"], st["E"], st["S"], st["N"])
    return op, oop


@pytest.mark.parametrize("kind", ["diff", "adv"])
@pytest.mark.parametrize("m", [15, 63, 127])
@pytest.mark.parametrize("adjoint", [False, True])
def test_stencil_propagate_f64_parity(ctx, orc, kind, m, adjoint):
    op, oop = _ops(ctx, orc, kind, m)
    dt, M = 1.0 / 2048, 4
    X = np.random.default_rng(m).standard_normal((3, m * m))
    got = api.propagate(ctx, op, dt, M, X, adjoint=adjoint)
    want = orc.propagate(oop, dt, M, X, adjoint=adjoint)
    for v in range(3):
        e = rel(got[v], want[v])
        assert e <= 1e-10, e
    assert op.krylov_iterations() > 0


def test_stencil_propagate_large_cluster(ctx, orc):
    """255^2 grid: the system spans an 8-CTA cluster."""
    op, oop = _ops(ctx, orc, "adv", 255, rtol64=1e-13)
    dt, M = 1.0 / 2048, 2
    X = np.random.default_rng(1).standard_normal((2, 255 * 255))
    got = api.propagate(ctx, op, dt, M, X)
    want = orc.propagate(oop, dt, M, X)
    for v in range(2):
        assert rel(got[v], want[v]) <= 1e-9


@pytest.mark.parametrize("kind", ["diff", "adv"])
def test_stencil_propagate_f32(ctx, orc, kind):
    op, oop = _ops(ctx, orc, kind, 63)
    dt, M = 1.0 / 4096, 8
    X = np.random.default_rng(2).standard_normal((4, 63 * 63))
    got = api.propagate(ctx, op, dt, M, X, prec="mixed")
    want = orc.propagate(oop, dt, M, X)
    for v in range(4):
        assert rel(got[v], want[v]) <= 5e-5


def test_stencil_source_and_batch(ctx, orc):
    m, dt, M = 31, 1.0 / 1024, 5
    op, oop = _ops(ctx, orc, "diff", m)
    g = np.random.default_rng(3).standard_normal((2, m * m))
    c = np.random.default_rng(4).standard_normal((7, M, 2))
    X = np.random.default_rng(5).standard_normal((7, m * m))
    got = api.propagate(ctx, op, dt, M, X, g=g, c=c)
    want = orc.propagate(oop, dt, M, X, g=g, cvals=c)
    for v in range(7):
        assert rel(got[v], want[v]) <= 1e-10


def test_stencil_iteration_cap_reports_notconv(ctx, orc):
    op, oop = _ops(ctx, orc, "diff", 31)
    op.set_krylov(1e-14, 1e-6, 2)
    X = np.random.default_rng(6).standard_normal((2, 31 * 31))
    with pytest.raises(_native.LrpError) as ei:
        api.propagate(ctx, op, 1.0 / 64, 3, X)
    assert ei.value.status == _native.LRP_ENOTCONV


@pytest.mark.parametrize("kind", ["diff", "adv"])
def test_stencil_build_and_parareal_f64(ctx, orc, kind):
    m = 31
    if kind == "diff":
        P = W.diff2d(m=m, N=4, M=8, R=5, p=3)
    else:
        P = W.adv2d(0, m=m, N=4, M=8, R=5, p=3)
    op = api.Operator.stencil5(ctx, m, m, P.st)
    op.set_krylov(1e-14, 1e-6, 20000)
    oop = orc.Stencil5(m, m, P.st["C"], P.st["W"], P.st["E"], P.st["S"], P.st["N"])
    co = api.Coarse(ctx, op, P.dt, P.M, P.N, P.R, P.p, P.seed, prec="f64")
    info = co.info()
    oco = orc.build_coarse(oop, P.dt, P.M, P.N, P.R, P.p, P.seed)
    probes = np.random.default_rng(7).standard_normal((3, P.n))
    for i in range(P.N):
        oc = oco.intervals[i]
        s1 = oc.sigma[0]
        assert info["R"][i] == oc.S.shape[0]
        assert np.max(np.abs(info["sigma"][i, :oc.S.shape[0]] - oc.S)) <= 1e-9 * s1
        U, S, V = co.factors(i)
        Go = oc.U @ np.diag(oc.S) @ oc.V.T
        Gg = U.T @ np.diag(S) @ V
        assert max(np.linalg.norm((Gg - Go) @ x) / np.linalg.norm(x) for x in probes) <= 1e-9 * s1
    u, pinfo = api.parareal_solve(ctx, co, P.u0, K=2)
    res = orc.parareal(oop, P.dt, P.M, P.N, oco, P.u0, K=2)
    assert rel(u, res.iterates[-1]) <= 1e-9
    u, pinfo = api.parareal_solve(ctx, co, P.u0, K=P.N)
    ref = orc.sequential_fine(oop, P.dt, P.M, P.N, P.u0)
    assert orc.rel_err(u, ref) <= 1e-10


def test_batched_uneven_build_and_solve(ctx, orc):
    """Several 2D advection-diffusion problems on different grids built in one
    graph-captured queue build and solved together: each matches its own
    separate build/solve (same sketches) and the oracle."""
    grids = (15, 31, 23, 31, 15)
    Ps = [W.adv2d(i, m=m, N=4, M=8, R=5, p=3) for i, m in enumerate(grids)]
    ops = []
    for P in Ps:
        op = api.Operator.stencil5(ctx, P.mx, P.my, P.st)
        op.set_krylov(1e-14, 1e-6, 20000)
        ops.append(op)
    P0 = Ps[0]
    cos = api.build_coarse_batch(ctx, ops, P0.dt, P0.M, P0.N, P0.R, P0.p, 0, prec="f64")
    outs, kd = api.parareal_solve_batch(ctx, cos, [P.u0 for P in Ps], K=P0.N)
    assert list(kd) == [P0.N] * len(Ps)
    for P, op, co, u in zip(Ps, ops, cos, outs):
        single = api.Coarse(ctx, op, P.dt, P.M, P.N, P.R, P.p, 0, prec="f64")
        a, b = co.info(), single.info()
        np.testing.assert_allclose(a["sigma"], b["sigma"], rtol=0, atol=1e-9 * b["sigma"].max())
        oop = orc.Stencil5(P.mx, P.my, P.st["C"], P.st["W"], P.st["E"], P.st["S"], P.st["N"])
        ref = orc.sequential_fine(oop, P.dt, P.M, P.N, P.u0)
        assert orc.rel_err(u, ref) <= 1e-10            # K = N: the fine solution
    outs2, kd2 = api.parareal_solve_batch(ctx, cos, [P.u0 for P in Ps], K=2)
    for P, op, co, u in zip(Ps, ops, cos, outs2):
        uu, info = api.parareal_solve(ctx, co, P.u0, K=2)
        assert rel(u, uu) <= 1e-10


def test_batched_uneven_at_config_sizes(ctx, orc):
    """The uneven batch at its own sizes: one advection-diffusion problem on
    each grid of {63^2, 127^2, 255^2, 511^2} (nu drawn as in the workload),
    N = 32, M = 64, R = 24, p = 8, built in one graph-captured queue build
    (mixed mode: FP32 sketches) and solved together with BiCGStab fine
    solves (rtol 1e-14) through the device-driven batched solve.  At tol 1e-8
    the 63^2 and 127^2 results are within 1e-7 of the oracle's sequential
    fine solution, and at K = N they equal it (finite termination) to 1e-10;
    every problem reports its own Krylov iteration count."""
    grids = (511, 63, 255, 127)
    Ps = [W.adv2d(i, N=32, M=64, R=24, p=8, m=m) for i, m in enumerate(grids)]
    ops = []
    for P in Ps:
        op = api.Operator.stencil5(ctx, P.mx, P.my, P.st)
        op.set_krylov(1e-14, 1e-6, 20000)
        ops.append(op)
    P0 = Ps[0]
    it0 = [op.krylov_iterations() for op in ops]
    cos = api.build_coarse_batch(ctx, ops, P0.dt, P0.M, P0.N, P0.R, P0.p, 0, prec="mixed")
    it1 = [op.krylov_iterations() for op in ops]
    assert all(b > a for a, b in zip(it0, it1))
    # larger grids need more Krylov iterations per system, so the counts differ
    assert len(set(b - a for a, b in zip(it0, it1))) == len(ops)
    refs = {}
    for P in Ps:
        if P.mx <= 127:
            oop = orc.Stencil5(P.mx, P.my, P.st["C"], P.st["W"], P.st["E"], P.st["S"], P.st["N"])
            refs[P.mx] = orc.sequential_fine(oop, P.dt, P.M, P.N, P.u0)
    outs, kd = api.parareal_solve_batch(ctx, cos, [P.u0 for P in Ps], K=P0.N, tol=1e-8)
    assert all(1 <= k <= P0.N for k in kd)
    for P, u in zip(Ps, outs):
        if P.mx in refs:
            assert orc.rel_err(u, refs[P.mx]) <= 1e-7, (P.mx, orc.rel_err(u, refs[P.mx]))
    outs, kd = api.parareal_solve_batch(ctx, cos, [P.u0 for P in Ps], K=P0.N)
    assert list(kd) == [P0.N] * len(Ps)
    for P, u in zip(Ps, outs):
        if P.mx in refs:
            assert orc.rel_err(u, refs[P.mx]) <= 1e-10, (P.mx, orc.rel_err(u, refs[P.mx]))


# ---------------------------------------------------------------------------
# SDIRK steppers on 5-point operators (two solves with I + gamma dt A per
# step on the Krylov kernel with its vectors in global memory; the source at
# the stage times)
# ---------------------------------------------------------------------------
def _stage_samples(orc, scheme, fun, dt, J0, M):
    cst, _, _ = orc.sdirk_tableau(scheme)
    t = dt * (J0 + np.arange(M))
    return np.stack([fun(t + cst[0] * dt), fun(t + cst[1] * dt)], axis=1)


@pytest.mark.parametrize("scheme", ["sdirk2", "sdirk2l"])
@pytest.mark.parametrize("kind,m", [("diff", 15), ("diff", 63), ("adv", 31), ("adv", 127)])
def test_sdirk_2d_propagate_parity(ctx, orc, scheme, kind, m):
    """CG (diffusion) and BiCGStab (advection-diffusion), one-CTA and cluster
    systems, with a two-term source at the stage times and the adjoint,
    FP64 at rtol 1e-14 within 1e-10 of the oracle; FP32 at the sketch
    tolerance."""
    op, oop = _ops(ctx, orc, kind, m)
    op.set_stepper(scheme)
    oop.stepper = scheme
    dt, M, Q = 1.0 / 1024, 3, 2
    rng = np.random.default_rng(3 * m + len(scheme))
    X = rng.standard_normal((3, m * m))
    g = rng.standard_normal((Q, m * m))
    c = np.stack([_stage_samples(orc, scheme, lambda t, k=k: np.stack(
        [np.sin((2 + k) * 9 * t), np.cos((1 + k) * 4 * t)], axis=-1), dt, 5 * k, M) for k in range(3)])
    got = api.propagate(ctx, op, dt, M, X, g=g, c=c)
    want = orc.propagate(oop, dt, M, X, g=g, cvals=c)
    for v in range(3):
        assert rel(got[v], want[v]) <= 1e-10, (v, rel(got[v], want[v]))
    gadj = api.propagate(ctx, op, dt, M, X, adjoint=True)
    wadj = orc.propagate(oop, dt, M, X, adjoint=True)
    for v in range(3):
        assert rel(gadj[v], wadj[v]) <= 1e-10
    g32 = api.propagate(ctx, op, dt, M, X[:2], g=g, c=c[:2], prec="mixed")
    for v in range(2):
        assert rel(g32[v], want[v]) <= 5e-4


@pytest.mark.parametrize("scheme", ["sdirk2", "sdirk2l"])
def test_sdirk_2d_build_and_parareal(ctx, orc, scheme):
    """Low-rank Parareal with an SDIRK fine solver on the checkerboard
    diffusion operator, with a source: the build matches the oracle's, K = 2
    the oracle's iterate, K = N the oracle's sequential solution."""
    P = W.diff2d(m=31, N=4, M=6, R=6, p=3)
    op = api.Operator.stencil5(ctx, P.mx, P.my, P.st)
    op.set_krylov(1e-14, 1e-6, 20000)
    op.set_stepper(scheme)
    oop = orc.Stencil5(P.mx, P.my, P.st["C"], P.st["W"], P.st["E"], P.st["S"], P.st["N"],
                       stepper=scheme)
    g = np.exp(-20 * np.linspace(-1, 1, P.n) ** 2)[None, :]
    c = _stage_samples(orc, scheme, lambda t: np.sin(5 * np.pi * t)[:, None], P.dt, 0, P.N * P.M)
    co = api.Coarse(ctx, op, P.dt, P.M, P.N, P.R, P.p, P.seed, prec="f64")
    oco = orc.build_coarse(oop, P.dt, P.M, P.N, P.R, P.p, P.seed)
    info = co.info()
    for i in range(P.N):
        oc = oco.intervals[i]
        assert np.max(np.abs(info["sigma"][i, :oc.S.shape[0]] - oc.S)) <= 1e-9 * oc.sigma[0]
    ref = orc.sequential_fine(oop, P.dt, P.M, P.N, P.u0, g, c)
    u, _ = api.parareal_solve(ctx, co, P.u0, g, c, K=P.N)
    assert orc.rel_err(u, ref) <= 1e-10
    res = orc.parareal(oop, P.dt, P.M, P.N, oco, P.u0, g, c, K=2)
    u2, _ = api.parareal_solve(ctx, co, P.u0, g, c, K=2)
    assert rel(u2, res.iterates[-1]) <= 1e-10
    # batched builds keep backward-Euler steps
    with pytest.raises(_native.LrpError) as ei:
        api.build_coarse_batch(ctx, [op], P.dt, P.M, P.N, P.R, P.p, 0, prec="f64")
    assert ei.value.status == _native.LRP_EINVAL


@pytest.mark.parametrize("kind,m", [("adv", 63), ("adv", 255), ("diff", 127), ("adv", 511)])
def test_staged_stencil_inputs_bitwise(ctx, orc, kind, m):
    """With krylov_stage = 1 the FP32 passes of the global-memory Krylov
    kernel read their stencil input from a shared-memory tile filled by one
    bulk copy per pass; the values are the ones in global memory, so the
    results equal those of the unstaged kernel (the default) bitwise, for
    BiCGStab and for CG (the on-chip CG switched off), and stay at the FP32
    tolerance of the oracle."""
    st = _problem(kind, m)
    op = api.Operator.stencil5(ctx, m, m, st)
    dt, M = 1.0 / 4096, 3
    X = np.random.default_rng(40 + m).standard_normal((5, m * m))
    ctx.set_param("krylov_onchip", 2)
    # the same CTAs per cluster in both runs (the partition of the grid, and
    # so the order of the reductions, follows it)
    ctx.set_param("krylov_cluster", {63: 1, 127: 2, 255: 8, 511: 16}[m])
    try:
        ctx.set_param("krylov_stage", 1)
        got = api.propagate(ctx, op, dt, M, X, prec="mixed")
        adj = api.propagate(ctx, op, dt, M, X, adjoint=True, prec="mixed")
        ctx.set_param("krylov_stage", 0)
        ref = api.propagate(ctx, op, dt, M, X, prec="mixed")
        radj = api.propagate(ctx, op, dt, M, X, adjoint=True, prec="mixed")
    finally:
        ctx.set_param("krylov_stage", 0)
        ctx.set_param("krylov_onchip", 0)
        ctx.set_param("krylov_cluster", 0)
    assert np.array_equal(got, ref) and np.array_equal(adj, radj)
    if m <= 127:
        oop = orc.Stencil5(m, m, st["C"], st["W"], st["E"], st["S"], st["N"])
        want = orc.propagate(oop, dt, M, X[:2])
        for v in range(2):
            assert rel(got[v], want[v]) <= 5e-4
