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


# ---------------------------------------------------------------------------
# SDIRK steppers on time-dependent operators (Sec. 4, effect of the time
# discretisation, on Experiment 3's time-dependent operator): stage s of step J
# uses A(t_J + c_s dt); the adjoint is the transposed step map, reversed order
# ---------------------------------------------------------------------------
SCHEMES = ["sdirk2", "sdirk2l"]


def _stage_rows(orc, scheme, dt, nJ, fn):
    """(2 nJ, ...) rows fn(t_J + c_s dt), row 2J + s."""
    c, _, _ = orc.sdirk_tableau(scheme)
    t = np.array([[J * dt + c[s] * dt for s in range(2)] for J in range(nJ)]).ravel()
    return np.array([fn(tt) for tt in t])


def _tri_td_rows(orc, scheme, n, dt, nJ, seed):
    """A diagonally dominant nonsymmetric tridiagonal A(t) sampled at the
    stage times."""
    rng = np.random.default_rng(seed)
    base = rng.uniform(0.5, 1.5, (3, n))
    w = rng.uniform(2.0, 9.0, (3, n))

    def at(t):
        lo = -base[0] * (1.0 + 0.5 * np.sin(w[0] * t))
        up = -base[2] * (1.0 + 0.5 * np.cos(w[2] * t))
        di = 3.0 * base[1] * (2.0 + np.sin(w[1] * t))
        return np.stack([lo, di, up])

    r = _stage_rows(orc, scheme, dt, nJ, at)
    return r[:, 0], r[:, 1], r[:, 2]


def _dense_step(At, b, dt, A1, A2, u, f1=None, f2=None):
    """One SDIRK step on the 2n x 2n stage system written as a block matrix:
    [[I + dt a11 A1, 0], [dt a21 A2, I + dt a22 A2]] [K1; K2] = -[A1 u; A2 u] + [f1; f2]."""
    n = A1.shape[0]
    I = np.eye(n)
    Big = np.block([[I + dt * At[0, 0] * A1, np.zeros((n, n))],
                    [dt * At[1, 0] * A2, I + dt * At[1, 1] * A2]])
    rhs = -np.concatenate([A1 @ u, A2 @ u])
    if f1 is not None:
        rhs = rhs + np.concatenate([f1, f2])
    K = np.linalg.solve(Big, rhs)
    return u + dt * (b[0] * K[:n] + b[1] * K[n:])


@pytest.mark.parametrize("scheme", SCHEMES)
def test_sdirk_td_constant_rows_equal_time_invariant(orc, scheme):
    n, M, dt = 20, 4, 0.02
    lo, di, up = W.adr1d_op(n)
    rep = lambda a: np.repeat(a[None, :], 2 * 2 * M, axis=0)
    td = orc.TridiagTD(rep(lo), rep(di), rep(up), stepper=scheme)
    ti = orc.Tridiag(lo, di, up, stepper=scheme)
    rng = np.random.default_rng(1)
    X = rng.standard_normal((3, n))
    g = rng.standard_normal((2, n))
    cv = rng.standard_normal((3, M, 2, 2))
    np.testing.assert_allclose(orc.propagate(td, dt, M, X, g=g, cvals=cv, intervals=1),
                               orc.propagate(ti, dt, M, X, g=g, cvals=cv), rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(orc.propagate(td, dt, M, X, adjoint=True, intervals=[0, 1, 0]),
                               orc.propagate(ti, dt, M, X, adjoint=True), rtol=1e-13, atol=1e-14)
    m = 4
    st = W.diff2d_op(m, 10.0 ** rng.uniform(0, 1, (8, 8)))
    rep2 = lambda a: np.repeat(a[None, :], 2 * M, axis=0)
    td2 = orc.Stencil5TD(m, m, *(rep2(st[k]) for k in "CWESN"), stepper=scheme)
    ti2 = orc.Stencil5(m, m, *(st[k] for k in "CWESN"), stepper=scheme)
    X2 = rng.standard_normal((2, m * m))
    for adj in (False, True):
        np.testing.assert_allclose(orc.propagate(td2, dt, M, X2, adjoint=adj),
                                   orc.propagate(ti2, dt, M, X2, adjoint=adj), rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("scheme", SCHEMES)
def test_sdirk_td_dense_block_steps_and_transposed_adjoint(orc, scheme):
    """F_i' = S_{j1} ... S_{j0} with every step matrix from the block stage
    system; the adjoint is (F_i')^T; with a source the affine steps match."""
    _, At, b = orc.sdirk_tableau(scheme)
    n, N, M, dt = 6, 3, 3, 0.05
    lo, di, up = _tri_td_rows(orc, scheme, n, dt, N * M, 2)
    op = orc.TridiagTD(lo, di, up, stepper=scheme)
    dense = lambda r: _dense_B(lo[r], di[r], up[r], 1.0) - np.eye(n)    # A itself
    rng = np.random.default_rng(3)
    X = rng.standard_normal((2, n))
    g = rng.standard_normal((1, n))
    cv = rng.standard_normal((M, 2, 1))
    for i in range(N):
        F = np.eye(n)
        for J in range(i * M, i * M + M):
            S = np.column_stack([_dense_step(At, b, dt, dense(2 * J), dense(2 * J + 1), e)
                                 for e in np.eye(n)])
            F = S @ F
        np.testing.assert_allclose(orc.propagate(op, dt, M, X, intervals=i), X @ F.T,
                                   rtol=1e-12, atol=1e-14)
        adj = orc.propagate(op, dt, M, X, adjoint=True, intervals=i)
        np.testing.assert_allclose(adj, X @ F, rtol=1e-12, atol=1e-14)
        # affine steps with the source at the stage times
        u = X[0].copy()
        for j, J in enumerate(range(i * M, i * M + M)):
            u = _dense_step(At, b, dt, dense(2 * J), dense(2 * J + 1), u,
                            cv[j, 0] @ g, cv[j, 1] @ g)
        np.testing.assert_allclose(orc.propagate(op, dt, M, X[:1], g=g, cvals=cv, intervals=i)[0],
                                   u, rtol=1e-12, atol=1e-14)
    # the stage operators of a step differ and their order matters: the
    # transposed stages taken in the forward order give another map
    with pytest.raises(ValueError):
        orc.propagate(op, dt, M, X, intervals=N)


@pytest.mark.parametrize("scheme", SCHEMES)
def test_sdirk_td_second_order_with_time_dependent_coefficient(orc, scheme):
    """u' = -(1 + t)(u - 1) on [0, 1]: u = 1 + (u0 - 1) exp(-(t + t^2/2)).
    Both schemes converge at order 2 only with the operator and the source at
    the stage times."""
    T, u0 = 1.0, np.array([3.0, -2.0])
    exact = 1.0 + (u0 - 1.0) * np.exp(-(T + T * T / 2))
    errs = []
    for nJ in (20, 40, 80):
        dt = T / nJ
        a = _stage_rows(orc, scheme, dt, nJ, lambda t: 1.0 + t)
        di = np.stack([a, a], axis=1)
        z = np.zeros_like(di)
        op = orc.TridiagTD(z, di, z, stepper=scheme)
        g = np.ones((1, 2))
        cv = a.reshape(nJ, 2, 1)          # f = (1 + t) at the stage times
        u = orc.propagate(op, dt, nJ, u0[None, :], g=g, cvals=cv)[0]
        errs.append(np.abs(u - exact).max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.6 < r1 < 4.4 and 3.6 < r2 < 4.4, errs


@pytest.mark.parametrize("scheme", SCHEMES)
def test_sdirk_td_parareal_K_N(orc, scheme):
    m, N, M, dt = 4, 3, 2, 0.02
    rng = np.random.default_rng(4)
    c, _, _ = orc.sdirk_tableau(scheme)
    rows = {k: [] for k in "CWESN"}
    for J in range(N * M):
        for s in range(2):
            t = (J + c[s]) * dt
            st = W.diff2d_op(m, 10.0 ** (0.5 + 0.5 * np.sin(3 * t + np.arange(64).reshape(8, 8))))
            for k in "CWESN":
                rows[k].append(st[k])
    op = orc.Stencil5TD(m, m, *(np.array(rows[k]) for k in "CWESN"), stepper=scheme)
    n = m * m
    u0 = rng.standard_normal(n)
    g = rng.standard_normal((1, n))
    cv = rng.standard_normal((N * M, 2, 1))
    ref = orc.sequential_fine(op, dt, M, N, u0, g, cv)
    co = orc.build_coarse(op, dt, M, N, 3, 2, 0)
    res = orc.parareal(op, dt, M, N, co, u0, g, cv, K=N)
    scale = np.max(np.linalg.norm(ref, axis=1))
    for k, it in enumerate(res.iterates):
        assert np.all(np.linalg.norm(it - ref, axis=1)[:k + 1] <= 1e-13 * scale)
