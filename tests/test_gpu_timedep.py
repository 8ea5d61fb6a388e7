"""GPU parity of the time-dependent tridiagonal path (Experiment 2 of Sec. 4:
conductivity 1 + 0.9 sin(7 pi t + 2 pi x), Neumann conditions) against the
FP64 oracle: every fine step has its own matrix, each interval runs its own
steps, and the adjoint sketch runs the transposed steps in reversed order.

FP64 results are compared at 1e-12 (propagation) and 1e-10 (Parareal
iterates); FP32 propagation at 5e-5 (log2(P) reduction levels times M steps
of FP32 rounding); the coarse factors as operators on probes at 1e-9 sigma_1
(FP64 build) and 1e-4 sigma_1 (mixed build, FP32 sketches).
"""
import numpy as np
import pytest

from paper_2508_08873_gb300 import _native, api, workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup(orc):
    ctx = api.Context(0)
    P = W.heat_td()                       # n = 100, N = 10, M = 10, R = 5, p = 1
    op = api.Operator.tridiag_td(ctx, P.lo, P.di, P.up)
    oop = orc.TridiagTD(P.lo, P.di, P.up)
    return ctx, P, op, oop


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("mixed", 5e-5)])
@pytest.mark.parametrize("adjoint", [False, True])
def test_td_propagate_matches_oracle(setup, orc, prec, tol, adjoint):
    ctx, P, op, oop = setup
    X = np.random.default_rng(1).standard_normal((7, P.n))
    got = api.propagate(ctx, op, P.dt, P.M, X, adjoint=adjoint, prec=prec)
    want = orc.propagate(oop, P.dt, P.M, X, adjoint=adjoint, intervals=0)
    for v in range(X.shape[0]):
        assert rel(got[v], want[v]) <= tol, (v, rel(got[v], want[v]))


def test_td_propagate_with_source(setup, orc):
    ctx, P, op, oop = setup
    rng = np.random.default_rng(2)
    X = rng.standard_normal((4, P.n))
    c = rng.standard_normal((4, P.M, 1))
    got = api.propagate(ctx, op, P.dt, P.M, X, g=P.g, c=c)
    want = orc.propagate(oop, P.dt, P.M, X, g=P.g, cvals=c, intervals=0)
    for v in range(4):
        assert rel(got[v], want[v]) <= 1e-12


@pytest.mark.parametrize("prec,tol", [("f64", 1e-9), ("mixed", 1e-4)])
def test_td_build_matches_oracle_per_interval(setup, orc, prec, tol):
    """G_i' of every interval as an operator (its own forward and adjoint
    sketches over its own steps) against the oracle's build."""
    ctx, P, op, oop = setup
    co = api.Coarse(ctx, op, P.dt, P.M, P.N, P.R, P.p, P.seed, prec=prec)
    info = co.info()
    oco = orc.build_coarse(oop, P.dt, P.M, P.N, P.R, P.p, P.seed)
    probes = np.random.default_rng(3).standard_normal((4, P.n))
    for i in range(P.N):
        oc = oco.intervals[i]
        s1 = oc.sigma[0]
        R = oc.S.shape[0]
        assert np.max(np.abs(info["sigma"][i, :R] - oc.S)) <= tol * s1
        U, S, V = co.factors(i)
        Go = oc.U @ np.diag(oc.S) @ oc.V.T
        Gg = U.T @ np.diag(S) @ V
        assert max(np.linalg.norm((Gg - Go) @ x) / np.linalg.norm(x) for x in probes) <= tol * s1
    # the intervals' operators differ: the conductivity changes in time
    assert np.abs(info["sigma"][0] - info["sigma"][3]).max() > 1e-6


def test_td_parareal_matches_oracle(setup, orc):
    ctx, P, op, oop = setup
    co = api.Coarse(ctx, op, P.dt, P.M, P.N, P.R, P.p, P.seed, prec="f64")
    oco = orc.build_coarse(oop, P.dt, P.M, P.N, P.R, P.p, P.seed)
    ref = orc.sequential_fine(oop, P.dt, P.M, P.N, P.u0, P.g, P.c)
    u, info = api.parareal_solve(ctx, co, P.u0, P.g, P.c, K=2)
    res = orc.parareal(oop, P.dt, P.M, P.N, oco, P.u0, P.g, P.c, K=2)
    assert rel(u, res.iterates[-1]) <= 1e-10
    u, info = api.parareal_solve(ctx, co, P.u0, P.g, P.c, K=P.N)
    assert orc.rel_err(u, ref) <= 1e-12
    uf = api.fine_solution(ctx, op, P.dt, P.M, P.N, P.u0, P.g, P.c)
    assert orc.rel_err(uf, ref) <= 1e-12
    u, info = api.parareal_solve(ctx, co, P.u0, P.g, P.c, K=P.N, tol=1e-10)
    assert info["converged"] and orc.rel_err(u, ref) <= 1e-9


def test_td_served_equals_direct(setup):
    ctx, P, op, oop = setup
    co = api.Coarse(ctx, op, P.dt, P.M, P.N, P.R, P.p, P.seed, prec="mixed")
    srv = api.Server(ctx, max_slots=4, max_terms=4)
    reqs = []
    for k in range(3):
        u0, g, c = W.serving_request(P.n, P.N, P.M, P.dt, 700 + k)
        reqs.append((srv.submit(co, u0, g, c, K=P.N, tol=1e-10), u0, g, c))
    for t, u0, g, c in reqs:
        u, info = srv.wait(t, timeout=120)
        direct, _ = api.parareal_solve(ctx, co, u0, g, c, K=P.N, tol=1e-10)
        assert np.linalg.norm(u - direct) <= 1e-12 * np.linalg.norm(direct)
    srv.close()


def test_td_rejects_beyond_time_grid_and_classical(setup):
    ctx, P, op, oop = setup
    with pytest.raises(_native.LrpError) as ei:
        api.Coarse(ctx, op, P.dt, P.M, P.N + 1, P.R, P.p, P.seed, prec="f64")
    assert ei.value.status == _native.LRP_EINVAL
    with pytest.raises(_native.LrpError) as ei:
        api.parareal_solve_classical(ctx, op, P.dt, P.M, P.N, P.u0, K=1)
    assert ei.value.status == _native.LRP_EINVAL
    lo = np.zeros((4, 1025))
    with pytest.raises(_native.LrpError) as ei:
        api.Operator.tridiag_td(ctx, lo, lo + 1.0, lo)
    assert ei.value.status == _native.LRP_EINVAL


# ---------------------------------------------------------------------------
# SDIRK steppers on the time-dependent operator: two coefficient rows per
# step (the stage times), the adjoint as the transposed step map
# ---------------------------------------------------------------------------
def _stage_times(orc, scheme, dt, nJ):
    c, _, _ = orc.sdirk_tableau(scheme)
    return np.array([[(J + c[s]) * dt for s in range(2)] for J in range(nJ)]).ravel()


@pytest.fixture(scope="module", params=["sdirk2", "sdirk2l"])
def sdirk_td(request, orc):
    scheme = request.param
    ctx = api.Context(0)
    P = W.heat_td(n=100, N=6, M=8, R=5, p=2)
    lo, di, up = W.heat_td_at(P.n, _stage_times(orc, scheme, P.dt, P.N * P.M))
    op = api.Operator.tridiag_td(ctx, lo, di, up, stepper=scheme)
    oop = orc.TridiagTD(lo, di, up, stepper=scheme)
    c = np.sin(2 * np.pi * _stage_times(orc, scheme, P.dt, P.N * P.M)).reshape(-1, 2, 1)
    return ctx, P, op, oop, c, scheme


def test_sdirk_td_propagate_matches_oracle(sdirk_td, orc):
    ctx, P, op, oop, c, scheme = sdirk_td
    rng = np.random.default_rng(11)
    X = rng.standard_normal((5, P.n))
    cv = rng.standard_normal((5, P.M, 2, 1))
    got = api.propagate(ctx, op, P.dt, P.M, X, g=P.g, c=cv)
    want = orc.propagate(oop, P.dt, P.M, X, g=P.g, cvals=cv, intervals=0)
    for v in range(5):
        assert rel(got[v], want[v]) <= 1e-12, (v, rel(got[v], want[v]))
    adj = api.propagate(ctx, op, P.dt, P.M, X, adjoint=True)
    wadj = orc.propagate(oop, P.dt, P.M, X, adjoint=True, intervals=0)
    for v in range(5):
        assert rel(adj[v], wadj[v]) <= 1e-12, (v, rel(adj[v], wadj[v]))
    g32 = api.propagate(ctx, op, P.dt, P.M, X, adjoint=True, prec="mixed")
    for v in range(5):
        assert rel(g32[v], wadj[v]) <= 5e-5


def test_sdirk_td_build_and_parareal_match_oracle(sdirk_td, orc):
    ctx, P, op, oop, c, scheme = sdirk_td
    co = api.Coarse(ctx, op, P.dt, P.M, P.N, P.R, P.p, P.seed, prec="f64")
    oco = orc.build_coarse(oop, P.dt, P.M, P.N, P.R, P.p, P.seed)
    info = co.info()
    probes = np.random.default_rng(12).standard_normal((3, P.n))
    for i in range(P.N):
        oc = oco.intervals[i]
        U, S, V = co.factors(i)
        Go = oc.U @ np.diag(oc.S) @ oc.V.T
        Gg = U.T @ np.diag(S) @ V
        assert max(np.linalg.norm((Gg - Go) @ x) / np.linalg.norm(x) for x in probes) <= 1e-9 * oc.sigma[0]
    ref = orc.sequential_fine(oop, P.dt, P.M, P.N, P.u0, P.g, c)
    u, _ = api.parareal_solve(ctx, co, P.u0, P.g, c, K=2)
    res = orc.parareal(oop, P.dt, P.M, P.N, oco, P.u0, P.g, c, K=2)
    assert rel(u, res.iterates[-1]) <= 1e-10
    uf = api.fine_solution(ctx, op, P.dt, P.M, P.N, P.u0, P.g, c)
    assert orc.rel_err(uf, ref) <= 1e-12
    u, info = api.parareal_solve(ctx, co, P.u0, P.g, c, K=P.N)
    assert orc.rel_err(u, ref) <= 1e-12
    # the operator keeps its stepper; backward Euler needs the other constructor
    with pytest.raises(_native.LrpError):
        op.set_stepper("be")
