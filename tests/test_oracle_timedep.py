"""Oracle: time-dependent operators (Experiment 2 of Sec. 4: a conductivity
varying in space and time, so that every fine step has its own matrix and the
F_n' of the intervals differ).

Pins: constant rows reproduce the time-invariant propagator; F_n' and its
adjoint equal the dense products of the step inverses written out from their
definition (F_n' = B_{j1}^-1 ... B_{j0}^-1, F_n'^* = B_{j0}^-T ... B_{j1}^-T,
the transposed solves in reversed order), while the transposes taken in the
forward order give a different operator; K = N and full rank behave as in the
time-invariant case; errors stay below the a posteriori bound.
"""
import numpy as np
import pytest

from paper_2508_08873_gb300 import workloads as W


def _dense_B(lo, di, up, dt):
    n = di.shape[0]
    B = np.diag(1.0 + dt * di)
    B[np.arange(1, n), np.arange(n - 1)] = dt * lo[1:]
    B[np.arange(n - 1), np.arange(1, n)] = dt * up[:-1]
    return B


@pytest.fixture(scope="module")
def small(orc):
    P = W.heat_td(n=24, N=5, M=4, R=4, p=2)
    op = orc.TridiagTD(P.lo, P.di, P.up)
    return P, op


def test_constant_rows_equal_time_invariant_propagate(orc):
    n, N, M, dt = 30, 3, 5, 0.01
    lo, di, up = W.heat1d_op(n)
    rep = lambda a: np.repeat(a[None, :], N * M, axis=0)
    td = orc.TridiagTD(rep(lo), rep(di), rep(up))
    ti = orc.Tridiag(lo, di, up)
    X = np.random.default_rng(1).standard_normal((4, n))
    for adj in (False, True):
        a = orc.propagate(td, dt, M, X, adjoint=adj, intervals=[0, 1, 2, 2])
        b = orc.propagate(ti, dt, M, X, adjoint=adj)
        np.testing.assert_allclose(a, b, rtol=1e-15, atol=0)


def test_interval_operator_and_adjoint_match_dense_products(orc, small):
    P, op = small
    n = P.n
    X = np.random.default_rng(2).standard_normal((3, n))
    for i in range(P.N):
        Fd = np.eye(n)
        for J in range(i * P.M, i * P.M + P.M):          # B_{j1}^-1 ... B_{j0}^-1
            Fd = np.linalg.solve(_dense_B(P.lo[J], P.di[J], P.up[J], P.dt), Fd)
        np.testing.assert_allclose(orc.propagate(op, P.dt, P.M, X, intervals=i), X @ Fd.T,
                                   rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(orc.propagate(op, P.dt, P.M, X, adjoint=True, intervals=i),
                                   X @ Fd, rtol=1e-12, atol=1e-14)
        # the transposed solves applied in the forward step order,
        # Wd = B_{j1}^-T ... B_{j0}^-T, are a different operator (the steps do
        # not commute), so the order of the adjoint's solves is pinned
        Wd = np.eye(n)
        for J in range(i * P.M, i * P.M + P.M):
            Wd = np.linalg.solve(_dense_B(P.lo[J], P.di[J], P.up[J], P.dt).T, Wd)
        adj = orc.propagate(op, P.dt, P.M, X, adjoint=True, intervals=i)
        assert np.abs(adj - X @ Wd.T).max() > 1e-6 * np.abs(adj).max()


def test_intervals_differ_and_steps_are_bounded(orc, small):
    P, op = small
    x = np.random.default_rng(3).standard_normal(P.n)
    y0 = orc.propagate(op, P.dt, P.M, x, intervals=0)
    y1 = orc.propagate(op, P.dt, P.M, x, intervals=1)
    assert np.linalg.norm(y0 - y1) > 1e-6 * np.linalg.norm(y0)
    with pytest.raises(ValueError):
        orc.propagate(op, P.dt, P.M, x, intervals=P.N)


def test_parareal_time_dependent_K_N_full_rank_and_bounds(orc, small):
    P, op = small
    ref = orc.sequential_fine(op, P.dt, P.M, P.N, P.u0, P.g, P.c)
    co = orc.build_coarse(op, P.dt, P.M, P.N, P.R, P.p, 0)
    res = orc.parareal(op, P.dt, P.M, P.N, co, P.u0, P.g, P.c, K=P.N)
    scale = np.max(np.linalg.norm(ref, axis=1))
    for k, it in enumerate(res.iterates):
        assert np.all(np.linalg.norm(it - ref, axis=1)[:k + 1] <= 1e-13 * scale)
    # Neumann conditions: every B_J^-1 fixes the constants, sigma_1 = 1
    ex = orc.exact_coarse(op, P.dt, P.M, P.N, P.R)
    assert abs(ex.delta - 1.0) <= 1e-12
    resx = orc.parareal(op, P.dt, P.M, P.N, ex, P.u0, P.g, P.c, K=P.N)
    for k in range(1, resx.k_done + 1):
        err = np.linalg.norm(resx.iterates[k] - ref, axis=1)
        assert np.all(err <= resx.bounds[k - 1] + 1e-13 * scale)
    full = orc.exact_coarse(op, P.dt, P.M, P.N, P.n)
    r1 = orc.parareal(op, P.dt, P.M, P.N, full, P.u0, P.g, P.c, K=1)
    assert orc.rel_err(r1.iterates[1], ref) <= 1e-12


# ---------------------------------------------------------------------------
# Time-dependent 5-point operators (Experiment 3: the conductivity varies in time)
# ---------------------------------------------------------------------------
def _stencil_td(m, nJ, seed):
    """A diffusion stencil whose face conductances oscillate in time, each
    step its own coefficients (symmetric in space at every step)."""
    rng = np.random.default_rng(seed)
    table = 10.0 ** rng.uniform(0, 1, (8, 8))
    out = {k: [] for k in "CWESN"}
    for J in range(nJ):
        st = W.diff2d_op(m, table * (1.0 + 0.5 * np.sin(0.7 * J + np.arange(64).reshape(8, 8))))
        for k in "CWESN":
            out[k].append(st[k])
    return {k: np.array(v) for k, v in out.items()}


def test_stencil_td_constant_rows_equal_time_invariant(orc):
    m, N, M, dt = 5, 3, 2, 0.01
    st = W.diff2d_op(m, 10.0 ** np.random.default_rng(1).uniform(0, 2, (8, 8)))
    rep = lambda a: np.repeat(a[None, :], N * M, axis=0)
    td = orc.Stencil5TD(m, m, *(rep(st[k]) for k in "CWESN"))
    ti = orc.Stencil5(m, m, *(st[k] for k in "CWESN"))
    X = np.random.default_rng(2).standard_normal((3, m * m))
    for adj in (False, True):
        a = orc.propagate(td, dt, M, X, adjoint=adj, intervals=[0, 1, 2])
        b = orc.propagate(ti, dt, M, X, adjoint=adj)
        np.testing.assert_allclose(a, b, rtol=1e-15, atol=0)


def test_stencil_td_dense_products_and_reversed_adjoint(orc):
    """F_i' = B_{j1}^-1 ... B_{j0}^-1 and F_i'^* = B_{j0}^-T ... B_{j1}^-T, the
    transposed solves in reversed order (the forward order differs)."""
    m, N, M, dt = 4, 3, 3, 0.05
    c = _stencil_td(m, N * M, 3)
    op = orc.Stencil5TD(m, m, c["C"], c["W"], c["E"], c["S"], c["N"])
    n = m * m
    X = np.random.default_rng(4).standard_normal((2, n))
    for i in range(N):
        Fd = np.eye(n)
        Wd = np.eye(n)
        for J in range(i * M, i * M + M):
            B = op.step(J).dense_B(dt)
            Fd = np.linalg.solve(B, Fd)
            Wd = np.linalg.solve(B.T, Wd)
        np.testing.assert_allclose(orc.propagate(op, dt, M, X, intervals=i), X @ Fd.T,
                                   rtol=1e-12, atol=1e-14)
        adj = orc.propagate(op, dt, M, X, adjoint=True, intervals=i)
        np.testing.assert_allclose(adj, X @ Fd, rtol=1e-12, atol=1e-14)
        assert np.abs(adj - X @ Wd.T).max() > 1e-8 * np.abs(adj).max()
    with pytest.raises(ValueError):
        orc.propagate(op, dt, M, X, intervals=N)


def test_stencil_td_parareal_K_N_and_full_rank(orc):
    m, N, M, dt = 5, 4, 3, 0.02
    c = _stencil_td(m, N * M, 5)
    op = orc.Stencil5TD(m, m, c["C"], c["W"], c["E"], c["S"], c["N"])
    n = m * m
    u0 = np.random.default_rng(6).standard_normal(n)
    g = np.random.default_rng(7).standard_normal((1, n))
    cv = np.sin(np.arange(N * M))[:, None]
    ref = orc.sequential_fine(op, dt, M, N, u0, g, cv)
    co = orc.build_coarse(op, dt, M, N, 4, 2, 0)
    res = orc.parareal(op, dt, M, N, co, u0, g, cv, K=N)
    scale = np.max(np.linalg.norm(ref, axis=1))
    for k, it in enumerate(res.iterates):
        assert np.all(np.linalg.norm(it - ref, axis=1)[:k + 1] <= 1e-13 * scale)
    full = orc.exact_coarse(op, dt, M, N, n)
    r1 = orc.parareal(op, dt, M, N, full, u0, g, cv, K=1)
    assert orc.rel_err(r1.iterates[1], ref) <= 1e-12
