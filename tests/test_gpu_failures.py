"""Failure detection without faulting the GPU: every failure here is raised by
the host from a status word or an argument check (zero pivots flagged by the
factorisation kernels, the HBM budget of a context, iteration caps), and the
context stays usable afterwards."""
import numpy as np
import pytest

from paper_2508_08873_gb300 import _native, api, workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,nvec", [(63, 3), (4095, 3), (4095, 200)])
def test_zero_pivot_reports_breakdown(n, nvec):
    ctx = api.Context(0)
    dt = 0.5                                      # power of two: 1 + dt * (-1/dt) == 0 exactly
    lo, di, up = W.heat1d_op(n)
    di = di.copy()
    lo = np.zeros(n)
    up = np.zeros(n)
    di[n // 3] = -1.0 / dt                       # 1 + dt*A has a zero pivot there
    op = api.Operator.tridiag(ctx, lo, di, up)
    X = np.ones((nvec, n))
    with pytest.raises(_native.LrpError) as ei:
        api.propagate(ctx, op, dt, 2, X)
    assert ei.value.status == _native.LRP_EBREAKDOWN
    # the context still works
    ok = api.Operator.tridiag(ctx, *W.heat1d_op(n))
    y = api.propagate(ctx, ok, dt, 2, X[:1])
    assert np.all(np.isfinite(y))


def test_hbm_budget_reports_enomem():
    ctx = api.Context(0, hbm_budget=1 << 20)       # 1 MiB
    P = W.adr1d()
    op = api.Operator.tridiag(ctx, P.lo, P.di, P.up)
    with pytest.raises(_native.LrpError) as ei:
        api.Coarse(ctx, op, P.dt, P.M, P.N, P.R, P.p, 0, prec="mixed")
    assert ei.value.status == _native.LRP_ENOMEM
    assert ctx.bytes_in_use() <= 1 << 20


def test_notconv_status_with_outputs():
    """tol not reached within K_max: LRP_ENOTCONV, outputs written."""
    ctx = api.Context(0)
    P = W.adr1d(n=511, N=16, M=32, R=4, p=2)
    op = api.Operator.tridiag(ctx, P.lo, P.di, P.up)
    co = api.Coarse(ctx, op, P.dt, P.M, P.N, P.R, P.p, 0)
    u, info = api.parareal_solve(ctx, co, P.u0, K=1, tol=1e-14, allow_notconv=True)
    assert info["status"] == _native.LRP_ENOTCONV and not info["converged"]
    assert np.all(np.isfinite(u)) and info["k_done"] == 1


def test_autotune_picks_valid_parameters():
    from paper_2508_08873_gb300 import autotune
    ctx = api.Context(0)
    P = W.adr1d(n=4095, N=16, M=32, R=4, p=2)
    op = api.Operator.tridiag(ctx, P.lo, P.di, P.up)
    co = api.Coarse(ctx, op, P.dt, P.M, P.N, P.R, P.p, 0, prec="f64")
    ref, _ = api.parareal_solve(ctx, co, P.u0, K=3)
    best = autotune.tune_solve(ctx, co, P.u0, K=2)
    assert set(best) == {"tri_cluster", "tri_chunk", "tri_spt", "tri_wchunk", "sweep_rows"}
    for k, v in best.items():
        assert ctx.get_param(k) == v
    u, _ = api.parareal_solve(ctx, co, P.u0, K=3)
    # launch shapes change only the rounding (FP64 path)
    assert np.linalg.norm(u - ref) <= 1e-12 * np.linalg.norm(ref)


def test_autotune_krylov_picks_a_valid_cluster_size():
    """The 2D tuner times the Krylov propagator under each CTA count per
    cluster and leaves the fastest applied; every choice gives the same step
    to the Krylov tolerance."""
    from paper_2508_08873_gb300 import autotune
    ctx = api.Context(0)
    P = W.diff2d(m=63, N=4, M=4, R=4, p=2)
    op = api.Operator.stencil5(ctx, 63, 63, P.st)
    op.set_krylov(1e-12, 1e-6, 20000)
    X = np.random.default_rng(1).standard_normal((4, P.n))
    ref = api.propagate(ctx, op, P.dt, 2, X)
    best = autotune.tune_krylov(ctx, op, P.dt, nsys=8, prec="f64")
    assert set(best) == {"krylov_cluster"} and best["krylov_cluster"] in autotune.KRYLOV_CANDIDATES
    assert ctx.get_param("krylov_cluster") == best["krylov_cluster"]
    got = api.propagate(ctx, op, P.dt, 2, X)
    assert np.linalg.norm(got - ref) <= 1e-10 * np.linalg.norm(ref)
    ctx.set_param("krylov_cluster", 0)
