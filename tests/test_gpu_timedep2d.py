"""GPU parity of the time-dependent 5-point path against the FP64 oracle.

Experiment 3 of Sec. 4 (2D heat equation whose conductivity oscillates in time
on two quarters of the unit square, with a source) makes every fine step's
matrix different, so the fine solvers F_n of the intervals differ and the
adjoint sketch runs the transposed steps in reversed order.  Each step is
solved by Jacobi-CG (symmetric stencils) or Jacobi-BiCGStab (a time-dependent
upwind advection-diffusion stencil); the oracle solves every step with a
banded LU.  As in the time-invariant 2D tests the Krylov tolerance is
tightened to 1e-14 so that FP64 results are compared at 1e-10 (propagation,
iterates) and the factors as operators on probes at 1e-9 sigma_1; FP32 at
the tolerance its rtol 1e-6 allows.
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


def _adv_td(m, nJ, dt):
    """Upwind advection-diffusion whose viscosity changes every step
    (nonsymmetric: BiCGStab)."""
    t = dt * np.arange(1, nJ + 1)
    per = [W.adv2d_op(m, 0.01 * (1.0 + 0.5 * np.sin(9.0 * tt))) for tt in t]
    return {k: np.array([d[k] for d in per]) for k in "CWESN"}


def _ops(ctx, orc, st, m, rtol64=1e-14):
    op = api.Operator.stencil5_td(ctx, m, m, st)
    op.set_krylov(rtol64, 1e-6, 20000)
    oop = orc.Stencil5TD(m, m, *(st[k] for k in "CWESN"))
    return op, oop


def _case(kind, m, M):
    if kind == "heat":
        P = W.heat2d_td(m=m, N=2, M=M, T=0.02 * M)     # dt = 0.01 as in Experiment 3
        return P.extra["st_t"], P.dt
    dt = 1.0 / 2048
    return _adv_td(m, 2 * M, dt), dt


@pytest.mark.parametrize("kind", ["heat", "adv"])
@pytest.mark.parametrize("m", [15, 63])
@pytest.mark.parametrize("adjoint", [False, True])
def test_td2d_propagate_f64_parity(ctx, orc, kind, m, adjoint):
    M = 4
    st, dt = _case(kind, m, M)
    op, oop = _ops(ctx, orc, st, m)
    X = np.random.default_rng(m + adjoint).standard_normal((3, m * m))
    got = api.propagate(ctx, op, dt, M, X, adjoint=adjoint)
    want = orc.propagate(oop, dt, M, X, adjoint=adjoint, intervals=0)
    for v in range(3):
        assert rel(got[v], want[v]) <= 1e-10, (v, rel(got[v], want[v]))
    assert op.krylov_iterations() > 0


@pytest.mark.parametrize("kind", ["heat", "adv"])
def test_td2d_propagate_source_and_f32(ctx, orc, kind):
    m, M = 31, 5
    st, dt = _case(kind, m, M)
    op, oop = _ops(ctx, orc, st, m)
    rng = np.random.default_rng(4)
    X = rng.standard_normal((3, m * m))
    g = rng.standard_normal((2, m * m))
    c = rng.standard_normal((3, M, 2))
    got = api.propagate(ctx, op, dt, M, X, g=g, c=c)
    want = orc.propagate(oop, dt, M, X, g=g, cvals=c, intervals=0)
    for v in range(3):
        assert rel(got[v], want[v]) <= 1e-10
    g32 = api.propagate(ctx, op, dt, M, X, g=g, c=c, prec="mixed")
    for v in range(3):
        assert rel(g32[v], want[v]) <= 5e-5


def test_td2d_propagate_cluster(ctx, orc):
    """127^2 grid: every system spans a multi-CTA cluster; the steps'
    plans and the rescaling of the CG iterate between steps cross CTAs."""
    m, M = 127, 3
    st, dt = _case("heat", m, M)
    op, oop = _ops(ctx, orc, st, m, rtol64=1e-13)
    X = np.random.default_rng(5).standard_normal((2, m * m))
    for adjoint in (False, True):
        got = api.propagate(ctx, op, dt, M, X, adjoint=adjoint)
        want = orc.propagate(oop, dt, M, X, adjoint=adjoint, intervals=0)
        for v in range(2):
            assert rel(got[v], want[v]) <= 1e-9


@pytest.fixture(scope="module")
def heat31(ctx, orc):
    P = W.heat2d_td(m=31)                 # N = 10, M = 10, R = 6, p = 1
    op, oop = _ops(ctx, orc, P.extra["st_t"], P.mx)
    return P, op, oop


@pytest.mark.parametrize("prec,tol", [("f64", 1e-9), ("mixed", 1e-4)])
def test_td2d_build_matches_oracle_per_interval(ctx, orc, heat31, prec, tol):
    """G_i' of every interval as an operator (its own forward sketch and its
    adjoint sketch over its own steps in reversed order) against the oracle."""
    P, op, oop = heat31
    co = api.Coarse(ctx, op, P.dt, P.M, P.N, P.R, P.p, P.seed, prec=prec)
    info = co.info()
    oco = orc.build_coarse(oop, P.dt, P.M, P.N, P.R, P.p, P.seed)
    probes = np.random.default_rng(6).standard_normal((4, P.n))
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
    assert np.abs(info["sigma"][0] - info["sigma"][1]).max() > 1e-3


def test_td2d_parareal_matches_oracle(ctx, orc, heat31):
    P, op, oop = heat31
    co = api.Coarse(ctx, op, P.dt, P.M, P.N, P.R, P.p, P.seed, prec="f64")
    oco = orc.build_coarse(oop, P.dt, P.M, P.N, P.R, P.p, P.seed)
    ref = orc.sequential_fine(oop, P.dt, P.M, P.N, P.u0, P.g, P.c)
    u, info = api.parareal_solve(ctx, co, P.u0, P.g, P.c, K=2)
    res = orc.parareal(oop, P.dt, P.M, P.N, oco, P.u0, P.g, P.c, K=2)
    assert rel(u, res.iterates[-1]) <= 1e-10
    u, info = api.parareal_solve(ctx, co, P.u0, P.g, P.c, K=P.N)
    assert orc.rel_err(u, ref) <= 1e-10
    uf = api.fine_solution(ctx, op, P.dt, P.M, P.N, P.u0, P.g, P.c)
    assert orc.rel_err(uf, ref) <= 1e-10
    u, info = api.parareal_solve(ctx, co, P.u0, P.g, P.c, K=P.N, tol=1e-8)
    assert info["converged"] and orc.rel_err(u, ref) <= 1e-7


def test_td2d_full_size_mixed_build_solve(ctx, orc):
    """The Experiment 3 stand-in at its own size (99^2 grid, N = 10, M = 10,
    R = 6, p = 1) at the default Krylov tolerances (1e-12 FP64, 1e-6 FP32):
    mixed build, Parareal to tol 1e-8, checked against the oracle's
    sequential fine solution."""
    P = W.heat2d_td()
    op = api.Operator.stencil5_td(ctx, P.mx, P.my, P.extra["st_t"])
    oop = orc.Stencil5TD(P.mx, P.my, *(P.extra["st_t"][k] for k in "CWESN"))
    ref = orc.sequential_fine(oop, P.dt, P.M, P.N, P.u0, P.g, P.c)
    uf = api.fine_solution(ctx, op, P.dt, P.M, P.N, P.u0, P.g, P.c)
    assert orc.rel_err(uf, ref) <= 1e-9
    co = api.Coarse(ctx, op, P.dt, P.M, P.N, P.R, P.p, P.seed, prec="mixed")
    u, info = api.parareal_solve(ctx, co, P.u0, P.g, P.c, K=P.N, tol=1e-8)
    assert info["converged"] and info["k_done"] < P.N
    assert orc.rel_err(u, ref) <= 1e-7


def test_td2d_served_equals_direct(ctx, heat31):
    P, op, oop = heat31
    co = api.Coarse(ctx, op, P.dt, P.M, P.N, P.R, P.p, P.seed, prec="mixed")
    srv = api.Server(ctx, max_slots=4, max_terms=4)
    reqs = []
    for k in range(3):
        u0, g, c = W.serving_request(P.n, P.N, P.M, P.dt, 710 + k)
        reqs.append((srv.submit(co, u0, g, c, K=P.N, tol=1e-8), u0, g, c))
    for t, u0, g, c in reqs:
        u, info = srv.wait(t, timeout=120)
        direct, _ = api.parareal_solve(ctx, co, u0, g, c, K=P.N, tol=1e-8)
        assert np.linalg.norm(u - direct) <= 1e-12 * np.linalg.norm(direct)
    srv.close()


def test_td2d_rejects(ctx, heat31):
    P, op, oop = heat31
    with pytest.raises(_native.LrpError) as ei:
        api.Coarse(ctx, op, P.dt, P.M, P.N + 1, P.R, P.p, P.seed, prec="f64")
    assert ei.value.status == _native.LRP_EINVAL
    with pytest.raises(_native.LrpError) as ei:
        api.parareal_solve_classical(ctx, op, P.dt, P.M, P.N, P.u0, K=1)
    assert ei.value.status == _native.LRP_EINVAL
    with pytest.raises(_native.LrpError) as ei:
        op.set_stepper("sdirk2")
    assert ei.value.status == _native.LRP_EINVAL
    with pytest.raises(_native.LrpError) as ei:
        api.propagate(ctx, op, P.dt, P.N * P.M + 1, np.zeros((1, P.n)))
    assert ei.value.status == _native.LRP_EINVAL
    with pytest.raises(ValueError):
        api.Operator.stencil5_td(ctx, P.mx, P.my, {k: np.zeros((3, P.n + 1)) for k in "CWESN"})


# ---------------------------------------------------------------------------
# SDIRK steppers on time-dependent 5-point operators (Sec. 4, effect of the
# time discretisation on Experiment 3): the operator at both stage times of
# every step, the adjoint as the transposed step map
# ---------------------------------------------------------------------------
def _stage_times(orc, scheme, dt, nJ):
    c, _, _ = orc.sdirk_tableau(scheme)
    return np.array([[(J + c[s]) * dt for s in range(2)] for J in range(nJ)]).ravel()


def _sdirk_case(orc, kind, scheme, m, nJ):
    if kind == "heat":
        dt = 0.01
        return W.heat2d_td_at(m, _stage_times(orc, scheme, dt, nJ)), dt
    dt = 1.0 / 2048
    per = [W.adv2d_op(m, 0.01 * (1.0 + 0.5 * np.sin(9.0 * t)))
           for t in _stage_times(orc, scheme, dt, nJ)]
    return {k: np.array([d[k] for d in per]) for k in "CWESN"}, dt


@pytest.mark.parametrize("scheme", ["sdirk2", "sdirk2l"])
@pytest.mark.parametrize("kind", ["heat", "adv"])
@pytest.mark.parametrize("m", [15, 63])
def test_td2d_sdirk_propagate_parity(ctx, orc, scheme, kind, m):
    M = 3
    st, dt = _sdirk_case(orc, kind, scheme, m, 2 * M)
    op = api.Operator.stencil5_td(ctx, m, m, st, stepper=scheme)
    op.set_krylov(1e-14, 1e-6, 20000)
    oop = orc.Stencil5TD(m, m, *(st[k] for k in "CWESN"), stepper=scheme)
    rng = np.random.default_rng(20 + m)
    X = rng.standard_normal((3, m * m))
    g = rng.standard_normal((2, m * m))
    cv = rng.standard_normal((3, M, 2, 2))
    got = api.propagate(ctx, op, dt, M, X, g=g, c=cv)
    want = orc.propagate(oop, dt, M, X, g=g, cvals=cv, intervals=0)
    for v in range(3):
        assert rel(got[v], want[v]) <= 1e-10, (v, rel(got[v], want[v]))
    adj = api.propagate(ctx, op, dt, M, X, adjoint=True)
    wadj = orc.propagate(oop, dt, M, X, adjoint=True, intervals=0)
    for v in range(3):
        assert rel(adj[v], wadj[v]) <= 1e-10, (v, rel(adj[v], wadj[v]))
    g32 = api.propagate(ctx, op, dt, M, X, g=g, c=cv, prec="mixed")
    for v in range(3):
        assert rel(g32[v], want[v]) <= 5e-4


@pytest.mark.parametrize("scheme", ["sdirk2", "sdirk2l"])
def test_td2d_sdirk_build_and_parareal(ctx, orc, scheme):
    """Experiment 3's operator and source on a 15^2 grid with the SDIRK
    stepper: the build matches the oracle's, K = 2 the oracle's iterate and
    K = N the oracle's sequential solution."""
    m, N, M, dt = 15, 4, 5, 0.01
    ts = _stage_times(orc, scheme, dt, N * M)
    st = W.heat2d_td_at(m, ts)
    op = api.Operator.stencil5_td(ctx, m, m, st, stepper=scheme)
    op.set_krylov(1e-14, 1e-6, 20000)
    oop = orc.Stencil5TD(m, m, *(st[k] for k in "CWESN"), stepper=scheme)
    P = W.heat2d_td(m=m, N=N, M=M, T=N * M * dt)
    c = np.sin(5 * np.pi * ts).reshape(N * M, 2, 1)
    co = api.Coarse(ctx, op, dt, M, N, 4, 2, 0, prec="f64")
    oco = orc.build_coarse(oop, dt, M, N, 4, 2, 0)
    info = co.info()
    for i in range(N):
        oc = oco.intervals[i]
        assert np.max(np.abs(info["sigma"][i, :oc.S.shape[0]] - oc.S)) <= 1e-9 * oc.sigma[0]
    ref = orc.sequential_fine(oop, dt, M, N, P.u0, P.g, c)
    u, _ = api.parareal_solve(ctx, co, P.u0, P.g, c, K=N)
    assert orc.rel_err(u, ref) <= 1e-10
    res = orc.parareal(oop, dt, M, N, oco, P.u0, P.g, c, K=2)
    u2, _ = api.parareal_solve(ctx, co, P.u0, P.g, c, K=2)
    assert rel(u2, res.iterates[-1]) <= 1e-10


@pytest.mark.parametrize("m", [31, 63, 127])
def test_td2d_onchip_f32(ctx, orc, m):
    """FP32 steps of a symmetric time-dependent operator run on the on-chip
    CG (every step its own couplings and scales, the iterate rescaled
    between steps), forward with a source and adjoint, within the FP32
    tolerance of the oracle and of the global-memory kernel."""
    M = 4
    st, dt = _case("heat", m, M)
    op, oop = _ops(ctx, orc, st, m)
    rng = np.random.default_rng(60 + m)
    X = rng.standard_normal((3, m * m))
    g = rng.standard_normal((1, m * m))
    c = rng.standard_normal((3, M, 1))
    got = api.propagate(ctx, op, dt, M, X, g=g, c=c, prec="mixed")
    assert ctx.get_param("krylov_onchip_rows") > 0
    adj = api.propagate(ctx, op, dt, M, X, adjoint=True, prec="mixed")
    ctx.set_param("krylov_onchip", 2)
    try:
        glob = api.propagate(ctx, op, dt, M, X, g=g, c=c, prec="mixed")
        assert ctx.get_param("krylov_onchip_rows") == 0
    finally:
        ctx.set_param("krylov_onchip", 0)
    want = orc.propagate(oop, dt, M, X, g=g, cvals=c, intervals=0)
    wadj = orc.propagate(oop, dt, M, X, adjoint=True, intervals=0)
    tol = 2e-4 if m <= 63 else 1e-3
    for v in range(3):
        assert rel(got[v], want[v]) <= tol, (v, rel(got[v], want[v]))
        assert rel(adj[v], wadj[v]) <= tol, (v, rel(adj[v], wadj[v]))
        assert rel(glob[v], want[v]) <= tol


@pytest.mark.parametrize("adjoint", [False, True])
def test_td2d_refine_f64(ctx, orc, adjoint):
    """FP64 steps of a symmetric time-dependent operator by iterative
    refinement (the default: FP64 residual on the step's own plan, FP32
    on-chip corrections with that step's couplings) and on the FP64 Krylov
    kernel (krylov_refine = 2), both against the oracle."""
    m, M = 63, 4
    st, dt = _case("heat", m, M)
    op, oop = _ops(ctx, orc, st, m)
    X = np.random.default_rng(70 + adjoint).standard_normal((3, m * m))
    got = api.propagate(ctx, op, dt, M, X, adjoint=adjoint)
    ctx.set_param("krylov_refine", 2)
    try:
        ref = api.propagate(ctx, op, dt, M, X, adjoint=adjoint)
    finally:
        ctx.set_param("krylov_refine", 0)
    want = orc.propagate(oop, dt, M, X, adjoint=adjoint, intervals=0)
    for v in range(3):
        assert rel(got[v], want[v]) <= 1e-10, (v, rel(got[v], want[v]))
        assert rel(ref[v], want[v]) <= 1e-10
