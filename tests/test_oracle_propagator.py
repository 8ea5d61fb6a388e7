"""Oracle: tridiagonal / banded direct solves and the backward-Euler fine
propagators F, F' and F'^* (Sec. 4: backward Euler; Eq. (F_n_affine)).

Pins: dense library solves, the closed-form DST spectrum of the 1D heat
operator, the closed-form geometric sum for a constant source, the adjoint
identity (F'^* w, v) = (w, F' v) (Sec. 2.1 step 3), and interval bookkeeping.
"""
import numpy as np
import pytest

from paper_2508_08873_gb300 import workloads as W


def _rand_tridiag(rng, n):
    lo = rng.uniform(-1, 0, n)
    up = rng.uniform(-1, 0, n)
    di = 2.5 + rng.uniform(0, 1, n)
    return lo, di, up


@pytest.mark.parametrize("n", [1, 2, 3, 17, 64])
def test_thomas_matches_dense_solve(orc, n):
    rng = np.random.default_rng(n)
    op = orc.Tridiag(*_rand_tridiag(rng, n))
    d = rng.standard_normal(n)
    x = np.zeros(n)
    work = np.zeros(n)
    rc = orc.lib().orc_thomas(n, orc._p(op.lo), orc._p(op.di), orc._p(op.up), orc._p(d),
                              orc._p(x), orc._p(work))
    assert rc == 0
    np.testing.assert_allclose(x, np.linalg.solve(op.dense(), d), rtol=1e-13, atol=1e-14)


def _heat_modes(n, dt, M):
    h = 1.0 / (n + 1)
    j = np.arange(1, n + 1)
    lam = 4.0 / h ** 2 * np.sin(j * np.pi * h / 2) ** 2
    sig = (1.0 + dt * lam) ** (-M)
    x = np.arange(1, n + 1) * h
    V = np.sqrt(2 * h) * np.sin(np.pi * np.outer(j, x))      # rows: orthonormal DST-I modes
    return sig, V


def test_heat_propagator_on_dst_modes(orc):
    """F' v_j = (1 + dt lam_j)^(-M) v_j for the DST-I eigenvectors."""
    P = W.heat1d()
    op = orc.Tridiag(P.lo, P.di, P.up)
    sig, V = _heat_modes(P.n, P.dt, P.M)
    for j in (0, 1, 4, 50, 254):
        out = orc.propagate(op, P.dt, P.M, V[j])
        # cond(I + dt A) ~ 260: rounding of 64 solves stays near 1e-12 relative
        np.testing.assert_allclose(out, sig[j] * V[j], rtol=0, atol=1e-12 * sig[0] * np.abs(V[j]).max())


def test_heat_dense_singular_values_closed_form(orc):
    """Singular values of the dense F' (255 propagations) = (1+dt lam_j)^-M."""
    P = W.heat1d()
    op = orc.Tridiag(P.lo, P.di, P.up)
    Fp = orc.propagate(op, P.dt, P.M, np.eye(P.n)).T
    s = np.linalg.svd(Fp, compute_uv=False)
    sig, _ = _heat_modes(P.n, P.dt, P.M)
    ref = np.sort(sig)[::-1]
    # 64 solves with cond ~260 and a dense SVD: ~1e-13 sigma_1 absolute
    np.testing.assert_allclose(s[:4], ref[:4], rtol=1e-12)
    assert np.max(np.abs(s - ref)) < 1e-12 * ref[0]
    # sigma_1..sigma_3 of the closed form (1 + dt 4 (n+1)^2 sin^2(j pi / (2(n+1))))^-M,
    # evaluated to five digits for n = 255, dt = 1/1024, M = 64
    np.testing.assert_allclose(s[:3], [5.4124e-1, 8.8841e-2, 4.8763e-3], rtol=1e-4)


@pytest.mark.parametrize("maker", ["adr", "heat"])
def test_adjoint_is_transpose(orc, maker):
    n, dt, M = 23, 1e-3, 7
    lo, di, up = W.adr1d_op(n) if maker == "adr" else W.heat1d_op(n)
    op = orc.Tridiag(lo, di, up)
    Fp = orc.propagate(op, dt, M, np.eye(n)).T
    Fa = orc.propagate(op, dt, M, np.eye(n), adjoint=True).T
    np.testing.assert_allclose(Fa, Fp.T, rtol=1e-13, atol=1e-16)
    B = np.eye(n) + dt * op.dense()
    np.testing.assert_allclose(Fp, np.linalg.matrix_power(np.linalg.inv(B), M),
                               rtol=1e-11, atol=1e-15)
    rng = np.random.default_rng(1)
    v, w = rng.standard_normal(n), rng.standard_normal(n)
    lhs = orc.propagate(op, dt, M, w, adjoint=True) @ v
    rhs = w @ orc.propagate(op, dt, M, v)
    assert abs(lhs - rhs) <= 1e-13 * abs(rhs) + 1e-15


def test_constant_source_closed_form(orc):
    """With c_q(t) = 1: F 0 = sum_{j=1}^M dt B^{-j} g = (I - B^{-M}) A^{-1} g."""
    n, dt, M = 31, 2e-3, 9
    lo, di, up = W.adr1d_op(n, nu=0.05)
    op = orc.Tridiag(lo, di, up)
    A = op.dense()
    B = np.eye(n) + dt * A
    g = np.exp(-((np.arange(1, n + 1) / (n + 1) - 0.4) / 0.2) ** 2)
    out = orc.propagate(op, dt, M, np.zeros(n), g=g[None], cvals=np.ones((M, 1)))
    expect = (np.eye(n) - np.linalg.matrix_power(np.linalg.inv(B), M)) @ np.linalg.solve(A, g)
    np.testing.assert_allclose(out, expect, rtol=1e-12, atol=1e-15)


def test_affine_split_and_interval_bookkeeping(orc):
    """F v = F' v + F 0 (Eq. (F_n_affine)); two intervals of M steps equal one
    propagation of 2M steps with the concatenated source samples."""
    P = W.heat1d(n=63, N=4, M=16)
    op = orc.Tridiag(P.lo, P.di, P.up)
    v = P.u0
    full = orc.fine_solve(op, P.dt, P.M, v, 1, P.g, P.c)
    lin = orc.propagate(op, P.dt, P.M, v)
    aff = orc.fine_solve(op, P.dt, P.M, np.zeros(P.n), 1, P.g, P.c)
    np.testing.assert_allclose(full, lin + aff, rtol=1e-13, atol=1e-15)
    two = orc.fine_solve(op, P.dt, P.M, orc.fine_solve(op, P.dt, P.M, v, 1, P.g, P.c), 2, P.g, P.c)
    one = orc.propagate(op, P.dt, 2 * P.M, v, g=P.g, cvals=P.c[P.M:3 * P.M])
    np.testing.assert_allclose(two, one, rtol=1e-14, atol=1e-16)
    seq = orc.sequential_fine(op, P.dt, P.M, P.N, v, P.g, P.c)
    direct = orc.propagate(op, P.dt, P.N * P.M, v, g=P.g, cvals=P.c)
    np.testing.assert_allclose(seq[-1], direct, rtol=1e-13, atol=1e-16)


@pytest.mark.parametrize("kind", ["diff", "adv"])
def test_band_solve_matches_dense(orc, kind):
    m = 6
    if kind == "diff":
        st = W.diff2d_op(m, 10 ** np.random.default_rng(0).uniform(0, 2, (8, 8)))
    else:
        st = W.adv2d_op(m, 0.01)
    op = orc.Stencil5(m, m, st["C"], st["W"], st["E"], st["S"], st["N"])
    dt, M = 1e-3, 3
    B = op.dense_B(dt)
    Fp = orc.propagate(op, dt, M, np.eye(m * m)).T
    np.testing.assert_allclose(Fp, np.linalg.matrix_power(np.linalg.inv(B), M), rtol=1e-11,
                               atol=1e-15)
    Fa = orc.propagate(op, dt, M, np.eye(m * m), adjoint=True).T
    np.testing.assert_allclose(Fa, Fp.T, rtol=1e-12, atol=1e-15)
    if kind == "diff":
        np.testing.assert_allclose(B, B.T, rtol=0, atol=1e-12 * np.abs(B).max())
    # stencil rows against the operator definition on an interior node
    A = (B - np.eye(m * m)) / dt
    p = 2 * m + 3
    assert np.isclose(A[p, p], st["C"][p]) and np.isclose(A[p, p - 1], st["W"][p])
    assert np.isclose(A[p, p + m], st["N"][p]) and np.isclose(A[p, p - m], st["S"][p])


def test_diff2d_constant_kappa_modes(orc):
    """Constant kappa: sin(kx pi x) sin(ky pi y) are eigenvectors of F' with
    eigenvalue (1 + dt (kappa 4/h^2 (sin^2(kx pi h/2) + sin^2(ky pi h/2)) + c))^-M."""
    m, dt, M, kappa = 15, 1e-3, 5, 3.0
    st = W.diff2d_op(m, np.full((8, 8), kappa), react=1.0)
    op = orc.Stencil5(m, m, st["C"], st["W"], st["E"], st["S"], st["N"])
    h = 1.0 / (m + 1)
    x = np.arange(1, m + 1) * h
    for kx, ky in ((1, 1), (2, 5), (15, 3)):
        v = np.outer(np.sin(ky * np.pi * x), np.sin(kx * np.pi * x)).ravel()
        lam = kappa * 4 / h ** 2 * (np.sin(kx * np.pi * h / 2) ** 2 + np.sin(ky * np.pi * h / 2) ** 2) + 1.0
        out = orc.propagate(op, dt, M, v)
        np.testing.assert_allclose(out, (1 + dt * lam) ** (-M) * v, rtol=0, atol=1e-13 * np.abs(v).max())


# ---------------------------------------------------------------------------
# SDIRK fine steppers (Sec. 4, effect of the time discretisation)
# ---------------------------------------------------------------------------
def _stability(scheme, z, orc):
    """R(z) = 1 + z b^T (I - z A)^-1 1 from the Butcher tableau."""
    _, A, b = orc.sdirk_tableau(scheme)
    return 1.0 + z * b @ np.linalg.solve(np.eye(2) - z * A, np.ones(2))


@pytest.mark.parametrize("scheme", ["sdirk2", "sdirk2l"])
def test_sdirk_step_is_the_stability_function(orc, scheme):
    """Scalar problem u' = -lam u: one step multiplies by R(-dt lam); the
    limits at infinite stiffness are -1/2 (SDIRK2, not L-stable) and 0
    (SDIRK2-L, L-stable)."""
    for lam in (0.3, 7.0, 250.0, 1e6):
        op = orc.Tridiag(np.zeros(1), np.array([lam]), np.zeros(1), stepper=scheme)
        for dt in (0.01, 0.2):
            got = orc.propagate(op, dt, 1, np.array([[1.0]]))[0, 0]
            want = _stability(scheme, -dt * lam, orc)
            assert abs(got - want) <= 1e-14 * max(1.0, abs(want))
    op = orc.Tridiag(np.zeros(1), np.array([1e12]), np.zeros(1), stepper=scheme)
    r_inf = orc.propagate(op, 1.0, 1, np.array([[1.0]]))[0, 0]
    assert abs(r_inf - (-0.5 if scheme == "sdirk2" else 0.0)) <= 1e-9


@pytest.mark.parametrize("scheme", ["sdirk2", "sdirk2l"])
def test_sdirk_second_order_on_heat(orc, scheme):
    """Heat equation, one DST mode: the error of M steps against the exact
    decay exp(-lam T) falls by ~4 when dt halves (second order), against ~2
    for backward Euler."""
    n = 63
    lo, di, up = W.heat1d_op(n)
    h = 1.0 / (n + 1)
    x = np.arange(1, n + 1) * h
    mode = np.sin(3 * np.pi * x)
    lam = 4.0 / h ** 2 * np.sin(3 * np.pi * h / 2) ** 2
    T = 0.01
    errs = []
    for M in (16, 32, 64):
        op = orc.Tridiag(lo, di, up, stepper=scheme)
        u = orc.propagate(op, T / M, M, mode)
        errs.append(np.linalg.norm(u - np.exp(-lam * T) * mode) / np.linalg.norm(mode))
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5, errs


@pytest.mark.parametrize("scheme", ["sdirk2", "sdirk2l"])
def test_sdirk_adjoint_is_transpose(orc, scheme):
    n, dt, M = 30, 0.01, 3
    op = orc.Tridiag(*W.adr1d_op(n, nu=0.05), stepper=scheme)
    F = orc.propagate(op, dt, M, np.eye(n)).T
    Ft = orc.propagate(op, dt, M, np.eye(n), adjoint=True).T
    np.testing.assert_allclose(Ft, F.T, atol=1e-14 * np.abs(F).max())


# ---------------------------------------------------------------------------
# SDIRK fine steppers with a source f(t) = sum_q c_q(t) g_q, sampled at the
# stage times t + c_i dt of every step
# ---------------------------------------------------------------------------
def _stage_samples(orc, scheme, fun, dt, M, t0=0.0):
    """(M, 2, 1) samples of fun at the stage times of M steps from t0."""
    c, _, _ = orc.sdirk_tableau(scheme)
    t = t0 + dt * np.arange(M)
    return np.stack([fun(t + c[0] * dt), fun(t + c[1] * dt)], axis=1)[:, :, None]


@pytest.mark.parametrize("scheme", ["sdirk2", "sdirk2l"])
def test_sdirk_source_is_exact_quadrature_for_linear_forcing(orc, scheme):
    """A = 0: u' = f(t) g, and a second-order Runge-Kutta step is a quadrature
    rule exact for f linear in t (sum b_i = 1, sum b_i c_i = 1/2), so M steps
    give u0 + g (alpha T + beta T^2 / 2) to rounding.  A wrong stage time or
    weight breaks the second condition."""
    n, M, T = 5, 7, 0.9
    dt = T / M
    z = np.zeros(n)
    op = orc.Tridiag(z, z, z, stepper=scheme)
    g = np.random.default_rng(1).standard_normal((1, n))
    u0 = np.random.default_rng(2).standard_normal(n)
    alpha, beta = 0.7, -2.3
    cv = _stage_samples(orc, scheme, lambda t: alpha + beta * t, dt, M)
    got = orc.propagate(op, dt, M, u0, g=g, cvals=cv)
    np.testing.assert_allclose(got, u0 + g[0] * (alpha * T + beta * T * T / 2), rtol=0, atol=1e-14)
    # a quadratic forcing is not integrated exactly (second order only)
    cv2 = _stage_samples(orc, scheme, lambda t: t * t, dt, M)
    got2 = orc.propagate(op, dt, M, u0, g=g, cvals=cv2)
    assert np.abs(got2 - (u0 + g[0] * T ** 3 / 3)).max() > 1e-6


@pytest.mark.parametrize("scheme", ["sdirk2", "sdirk2l"])
def test_sdirk_source_steady_state_is_a_fixed_point(orc, scheme):
    """A constant source: the steady state u* = A^-1 g makes every stage
    derivative vanish, so the step map leaves it unchanged."""
    n = 40
    op = orc.Tridiag(*W.heat1d_op(n), stepper=scheme)
    g = np.random.default_rng(3).standard_normal((1, n))
    u_star = np.linalg.solve(op.dense(), g[0])
    cv = np.ones((5, 2, 1))
    got = orc.propagate(op, 0.01, 5, u_star, g=g, cvals=cv)
    np.testing.assert_allclose(got, u_star, rtol=1e-12, atol=1e-12 * np.abs(u_star).max())


@pytest.mark.parametrize("scheme", ["sdirk2", "sdirk2l"])
def test_sdirk_source_second_order(orc, scheme):
    """Decoupled scalar problems u' = -lam u + sin(w t) (diagonal A): the error
    against the closed-form solution falls by ~4 when dt halves."""
    lam = np.array([0.5, 3.0, 20.0])
    w, T, u0 = 9.0, 1.0, np.array([1.0, -0.5, 2.0])
    z = np.zeros(3)
    op = orc.Tridiag(z, lam, z, stepper=scheme)

    def exact(t):
        return (np.exp(-lam * t) * u0
                + (lam * np.sin(w * t) - w * np.cos(w * t) + w * np.exp(-lam * t)) / (lam ** 2 + w ** 2))

    errs = []
    for M in (40, 80, 160):
        cv = _stage_samples(orc, scheme, lambda t: np.sin(w * t), T / M, M)
        got = orc.propagate(op, T / M, M, u0, g=np.ones((1, 3)), cvals=cv)
        errs.append(np.abs(got - exact(T)).max())
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5, errs


# ---------------------------------------------------------------------------
# SDIRK steppers on 5-point operators (2D)
# ---------------------------------------------------------------------------
def _stencil(orc, st, m, scheme):
    return orc.Stencil5(m, m, st["C"], st["W"], st["E"], st["S"], st["N"], stepper=scheme)


@pytest.mark.parametrize("scheme", ["sdirk2", "sdirk2l"])
def test_sdirk_2d_step_is_the_stability_function(orc, scheme):
    """Symmetric diffusion stencil A = V diag(lam) V^T: M steps apply
    V R(-dt lam)^M V^T, R from the Butcher tableau alone."""
    m, dt, M = 7, 0.02, 3
    st = W.diff2d_op(m, 10.0 ** np.random.default_rng(1).uniform(0, 2, (8, 8)))
    op = _stencil(orc, st, m, scheme)
    A = op.dense_B(1.0) - np.eye(m * m)
    lam, V = np.linalg.eigh(0.5 * (A + A.T))
    R = np.array([_stability(scheme, -dt * l, orc) for l in lam])
    F = (V * R ** M) @ V.T
    X = np.random.default_rng(2).standard_normal((3, m * m))
    np.testing.assert_allclose(orc.propagate(op, dt, M, X), X @ F.T, rtol=0, atol=1e-12)


@pytest.mark.parametrize("scheme", ["sdirk2", "sdirk2l"])
def test_sdirk_2d_adjoint_is_transpose(orc, scheme):
    """Nonsymmetric advection-diffusion stencil: F'^* = F'^T."""
    m, dt, M = 6, 0.01, 2
    op = _stencil(orc, W.adv2d_op(m, 0.01), m, scheme)
    n = m * m
    F = orc.propagate(op, dt, M, np.eye(n)).T
    Ft = orc.propagate(op, dt, M, np.eye(n), adjoint=True).T
    np.testing.assert_allclose(Ft, F.T, atol=1e-14 * np.abs(F).max())


@pytest.mark.parametrize("scheme", ["sdirk2", "sdirk2l"])
def test_sdirk_2d_source_steady_state_is_a_fixed_point(orc, scheme):
    m = 8
    op = _stencil(orc, W.adv2d_op(m, 0.02), m, scheme)
    g = np.random.default_rng(4).standard_normal((1, m * m))
    u_star = np.linalg.solve(op.dense_B(1.0) - np.eye(m * m), g[0])
    got = orc.propagate(op, 0.01, 4, u_star, g=g, cvals=np.ones((4, 2, 1)))
    np.testing.assert_allclose(got, u_star, rtol=1e-12, atol=1e-12 * np.abs(u_star).max())
