"""Oracle: the Parareal iteration (Eq. (def_Parareal)), its a priori bounds
(Theorem 1), the a posteriori bound (Eq. (apost_bound)), the exact error
representation for invariant projections (Theorem 2 and its self-adjoint
corollary), the cost count (Eq. (num_F_eval)) and Remark (rem:affine_g_n)."""
import math
import pathlib

import numpy as np
import pytest

from paper_2508_08873_gb300 import workloads as W


@pytest.fixture(scope="module")
def heat_small(orc):
    P = W.heat1d(n=31, N=8, M=8, R=3, p=2)
    op = orc.Tridiag(P.lo, P.di, P.up)
    ref = orc.sequential_fine(op, P.dt, P.M, P.N, P.u0, P.g, P.c)
    return P, op, ref


def _bnorms(P, res):
    bn = np.zeros(P.N)
    bn[0] = np.linalg.norm(P.u0)
    bn[1:] = np.linalg.norm(res.b[:-1], axis=1)
    return bn


def test_R0_is_plain_fine_iteration(orc, heat_small):
    """G_n = b_n (rank 0): u^{k+1}_{n+1} = F_{n+1} u^k_n (Sec. 4, G = 0 case)."""
    P, op, ref = heat_small
    coarse = orc.build_coarse(op, P.dt, P.M, P.N, 0, 2, 0)
    res = orc.parareal(op, P.dt, P.M, P.N, coarse, P.u0, P.g, P.c, K=3)
    for k in range(3):
        prev, new = res.iterates[k], res.iterates[k + 1]
        for i in range(P.N):
            np.testing.assert_allclose(new[i + 1], orc.fine_solve(op, P.dt, P.M, prev[i], i, P.g, P.c),
                                       rtol=1e-14, atol=1e-15)


def test_K_equals_N_gives_fine_solution_and_finite_termination(orc, heat_small):
    P, op, ref = heat_small
    coarse = orc.build_coarse(op, P.dt, P.M, P.N, P.R, P.p, 0)
    res = orc.parareal(op, P.dt, P.M, P.N, coarse, P.u0, P.g, P.c, K=P.N + 5)
    assert res.k_done == P.N
    scale = np.max(np.linalg.norm(ref, axis=1))
    for k, it in enumerate(res.iterates):
        err = np.linalg.norm(it - ref, axis=1)
        # u^k_n = u_n for n <= k (empty sum in Eq. (error_bound_eps_delta))
        assert np.all(err[:k + 1] <= 1e-13 * scale)
    assert orc.rel_err(res.iterates[-1], ref) <= 1e-13


def test_full_rank_converges_in_one_iteration(orc):
    P = W.heat1d(n=10, N=6, M=5, R=10, p=0)
    op = orc.Tridiag(P.lo, P.di, P.up)
    ref = orc.sequential_fine(op, P.dt, P.M, P.N, P.u0, P.g, P.c)
    coarse = orc.exact_coarse(op, P.dt, P.M, P.N, R=10)
    assert coarse.eps == 0.0
    res = orc.parareal(op, P.dt, P.M, P.N, coarse, P.u0, P.g, P.c, K=1)
    # eps = 0: G = F, so u^0 is already exact and u^1 as well
    assert orc.rel_err(res.iterates[1], ref) <= 1e-13
    assert orc.rel_err(res.iterates[0], ref) <= 1e-13
    # and with the randomized SVD (ell >= n) the same holds
    coarse = orc.build_coarse(op, P.dt, P.M, P.N, 10, 2, 0)
    res = orc.parareal(op, P.dt, P.M, P.N, coarse, P.u0, P.g, P.c, K=1)
    assert orc.rel_err(res.iterates[1], ref) <= 1e-13


@pytest.mark.parametrize("maker", ["heat", "adr"])
def test_bounds_hold(orc, maker):
    if maker == "heat":
        P = W.heat1d(n=31, N=8, M=8, R=2, p=2)
    else:
        P = W.adr1d(n=63, N=8, M=16, R=3, p=3)
    op = orc.Tridiag(P.lo, P.di, P.up)
    ref = orc.sequential_fine(op, P.dt, P.M, P.N, P.u0, P.g, P.c)
    coarse = orc.exact_coarse(op, P.dt, P.M, P.N, P.R)     # exact delta, eps
    res = orc.parareal(op, P.dt, P.M, P.N, coarse, P.u0, P.g, P.c, K=P.N)
    d, e = coarse.delta, coarse.eps
    assert d < 1.0                                            # Dirichlet: contraction
    bn = _bnorms(P, res)
    slack = 1e-13 * np.max(np.linalg.norm(ref, axis=1))
    err0 = np.linalg.norm(res.iterates[0] - ref, axis=1)
    assert np.all(err0 <= orc.apriori_initial(d, e, bn) + slack)
    for k in range(1, res.k_done + 1):
        err = np.linalg.norm(res.iterates[k] - ref, axis=1)
        assert np.all(err <= res.bounds[k - 1] + slack), k            # Eq. (apost_bound)
        du = np.linalg.norm(res.iterates[k] - res.iterates[k - 1], axis=1)
        assert err.max() <= e / (1 - d) * du.max() + slack            # Eq. (apost_bound_sup)
        assert np.all(err <= orc.apriori_from_e0(d, e, err0, k) + slack)
        assert np.all(err <= orc.apriori_k(d, e, bn, k) + slack)
        assert err[1:].max() <= math.comb(P.N, k) * e ** k * err0[1:P.N - k + 1].max() + slack \
            if k < P.N else True                                      # Eq. (error_bound_eps)
        assert err[1:].max() <= (e / (1 - d)) ** k * err0[1:P.N - k + 1].max() + slack \
            if k < P.N else True                                      # Eq. (error_bound_eps_inf_time)


def test_exact_error_identity_invariant_projection(orc):
    """Theorem 2: F' self-adjoint, G' its truncated eigen-decomposition:
    e^k_n = (F' - G')^k e^0_{n-k} for n > k, else 0; and the corollary
    max_n ||e^k_n|| <= sigma_{R+1}^k max_n ||e^0_n||."""
    P = W.heat1d(n=20, N=7, M=6, R=2, p=0)
    op = orc.Tridiag(P.lo, P.di, P.up)
    ref = orc.sequential_fine(op, P.dt, P.M, P.N, P.u0, P.g, P.c)
    coarse = orc.exact_coarse(op, P.dt, P.M, P.N, P.R)
    Fp = orc.propagate(op, P.dt, P.M, np.eye(P.n)).T
    np.testing.assert_allclose(Fp, Fp.T, atol=1e-15)
    c0 = coarse.intervals[0]
    D = Fp - c0.U @ np.diag(c0.S) @ c0.V.T
    res = orc.parareal(op, P.dt, P.M, P.N, coarse, P.u0, P.g, P.c, K=4)
    e0 = res.iterates[0] - ref
    scale = np.max(np.linalg.norm(ref, axis=1))
    for k in range(1, 5):
        ek = res.iterates[k] - ref
        for n in range(P.N + 1):
            want = np.linalg.matrix_power(D, k) @ e0[n - k] if n > k else np.zeros(P.n)
            np.testing.assert_allclose(ek[n], want, atol=1e-13 * scale)
        sig = coarse.intervals[0].sigma[P.R]
        assert np.linalg.norm(ek, axis=1).max() <= sig ** k * np.linalg.norm(e0[1:P.N - k + 1], axis=1).max() + 1e-13 * scale


def test_delta_form_equals_literal_form(orc, heat_small):
    """Remark (rem:affine_g_n): u^{k+1}_{n+1} = F u^k_n + G'(u^{k+1}_n - u^k_n)."""
    P, op, ref = heat_small
    coarse = orc.build_coarse(op, P.dt, P.M, P.N, P.R, P.p, 0)
    res = orc.parareal(op, P.dt, P.M, P.N, coarse, P.u0, P.g, P.c, K=3)
    for k in range(3):
        prev, new = res.iterates[k], res.iterates[k + 1]
        u = prev[0].copy()
        for i in range(P.N):
            Fi = orc.fine_solve(op, P.dt, P.M, prev[i], i, P.g, P.c)
            u = Fi + coarse.apply_lin(i, u - prev[i])
            np.testing.assert_allclose(u, new[i + 1], rtol=1e-13, atol=1e-15)


def test_cost_count(orc, heat_small):
    """Eq. (num_F_eval): K_{F,n} = 2(R_n + p) + k + 1 fine evaluations."""
    P, op, ref = heat_small
    coarse = orc.build_coarse(op, P.dt, P.M, P.N, P.R, P.p, 0)
    res = orc.parareal(op, P.dt, P.M, P.N, coarse, P.u0, P.g, P.c, K=2)
    for c in coarse.intervals:
        assert c.fine_evals + res.fine_evals == 2 * (P.R + P.p) + res.k_done + 1


def test_tol_stopping(orc, heat_small):
    P, op, ref = heat_small
    coarse = orc.build_coarse(op, P.dt, P.M, P.N, P.R, P.p, 0)
    res = orc.parareal(op, P.dt, P.M, P.N, coarse, P.u0, P.g, P.c, K=P.N, tol=1e-9)
    scale = np.max(np.linalg.norm(res.iterates[-1], axis=1))
    assert res.bounds[-1].max() <= 1e-9 * scale
    if res.k_done > 1:
        assert res.bounds[-2].max() > 1e-9 * np.max(np.linalg.norm(res.iterates[-2], axis=1))
    assert orc.rel_err(res.iterates[-1], ref) <= 1e-9 * 1.0001


def _exp4_table():
    rows = []
    path = pathlib.Path(__file__).parent / "golden" / "exp4_fine_evaluations.txt"
    for line in path.read_text().splitlines():
        if line.strip() and not line.startswith("#"):
            rows.append([int(v) for v in line.split()])
    return rows


def test_fine_evaluation_count_matches_experiment4_table(orc):
    """The oracle's evaluation counters (sketch propagations of the build,
    plus b_n and one fine solve per Parareal iteration) reproduce the counts
    printed in the paper's Experiment 4 table, K_{F,n} + 1 of Eq. num_F_eval,
    for every (p, r) and k = 0..4.  Tiny full-rank problem, so no sketch
    direction is deflated."""
    n, N, M, dt = 12, 5, 3, 0.05
    lo = np.full(n, -1.0); di = np.full(n, 2.5); up = np.full(n, -1.2)
    op = orc.Tridiag(lo, di, up)
    g = np.linspace(0.5, 1.5, n)[None, :]
    c = np.ones((N * M, 1))
    u0 = np.sin(np.arange(n))
    for p, r, setup, *per_k in _exp4_table():
        co = orc.build_coarse(op, dt, M, N, r, p, 0)
        build = co.intervals[0].fine_evals
        assert all(iv.fine_evals == build for iv in co.intervals)
        assert build + 1 == setup                       # sketches + b_n
        for k, want in enumerate(per_k):
            res = orc.parareal(op, dt, M, N, co, u0, g, c, K=k)
            assert res.k_done == k
            assert build + res.fine_evals + 1 == want, (p, r, k)


# ---------------------------------------------------------------------------
# classical Parareal (backward-Euler coarse solver), the comparison method
# ---------------------------------------------------------------------------
def test_classical_parareal_scalar_closed_form(orc):
    """For a scalar linear problem Parareal's iterates have the closed form
    u^k_n = sum_{j<=k} binom(n, j) (F - G)^j G^(n-j) u0 (Gander and Vandewalle,
    SIAM J. Sci. Comput. 29 (2007), the linear analysis of Parareal), with
    F = (1 + dt lam)^-M and G = (1 + M dt lam)^-1."""
    lam, dt, M, N = 3.0, 0.02, 5, 9
    op = orc.Tridiag(np.zeros(1), np.array([lam]), np.zeros(1))
    F = (1.0 + dt * lam) ** (-M)
    G = 1.0 / (1.0 + M * dt * lam)
    u0 = np.array([1.7])
    for K in range(0, N + 1):
        res = orc.parareal_classical(op, dt, M, N, u0, K=K)
        want = [sum(math.comb(nn, j) * (F - G) ** j * G ** (nn - j) for j in range(0, min(K, nn) + 1)) * u0[0]
                for nn in range(N + 1)]
        np.testing.assert_allclose(res.iterates[-1][:, 0], want, rtol=1e-13, atol=0)


def test_classical_parareal_K_equals_N_and_exact_coarse(orc):
    P = W.heat1d(n=63, N=6, M=8)
    op = orc.Tridiag(P.lo, P.di, P.up)
    ref = orc.sequential_fine(op, P.dt, P.M, P.N, P.u0, P.g, P.c)
    res = orc.parareal_classical(op, P.dt, P.M, P.N, P.u0, P.g, P.c, K=P.N)
    assert orc.rel_err(res.iterates[-1], ref) <= 1e-13
    for k, it in enumerate(res.iterates):              # u^k_n exact for n <= k
        assert orc.rel_err(it[:k + 1], ref[:k + 1]) <= 1e-13
    # M = 1: the coarse step is the fine step, so u^0 is already the fine solution
    ref1 = orc.sequential_fine(op, P.dt * P.M, 1, P.N, P.u0, P.g, P.c[P.M - 1::P.M])
    res1 = orc.parareal_classical(op, P.dt * P.M, 1, P.N, P.u0, P.g, P.c[P.M - 1::P.M], K=0)
    assert orc.rel_err(res1.iterates[0], ref1) <= 1e-14


def test_low_rank_coarse_beats_classical_on_heat(orc):
    """The paper's comparison (Experiment 1): with rank-R coarse solvers the
    error after k iterations is far below the classical one."""
    P = W.heat1d()
    op = orc.Tridiag(P.lo, P.di, P.up)
    ref = orc.sequential_fine(op, P.dt, P.M, P.N, P.u0, P.g, P.c)
    co = orc.build_coarse(op, P.dt, P.M, P.N, 4, 2, 0)
    lr = orc.parareal(op, P.dt, P.M, P.N, co, P.u0, P.g, P.c, K=2)
    cl = orc.parareal_classical(op, P.dt, P.M, P.N, P.u0, P.g, P.c, K=2)
    e_lr = orc.rel_err(lr.iterates[-1], ref)
    e_cl = orc.rel_err(cl.iterates[-1], ref)
    assert e_lr < 1e-3 * e_cl, (e_lr, e_cl)


# ---------------------------------------------------------------------------
# the bound functions pinned by value
# ---------------------------------------------------------------------------
def _hand_values():
    """Rows of tests/golden/bound_hand_values.txt: name -> list of Fractions."""
    from fractions import Fraction
    out = {}
    path = pathlib.Path(__file__).parent / "golden" / "bound_hand_values.txt"
    for line in path.read_text().splitlines():
        if not line.strip() or line.startswith("#"):
            continue
        name, _, vals = [s.strip() for s in line.split("|")]
        out[name] = [Fraction(v) for v in vals.split()]
    return out


def test_bound_functions_match_hand_evaluated_values(orc):
    """apriori_initial (Eq. error_bound_initial), apriori_k
    (Eq. error_bound_eps_delta2), apriori_from_e0 (Eq. error_bound_eps_delta),
    apost_bound (Eq. apost_bound) and efficiency (Eq. def_efficiency) on the
    hand-worked example of tests/golden/bound_hand_values.txt (delta = 1/2,
    eps = 3/8, exact rationals)."""
    hv = _hand_values()
    d, e = 0.5, 0.375
    b = np.array([1.0, 2.0, 4.0])
    e0 = np.array([0.0, 1.0, 3.0, 5.0])
    du = np.array([7.0, 1.0, 2.0, 4.0, 8.0])

    def chk(got, name):
        want = np.array([float(v) for v in hv[name]])
        np.testing.assert_allclose(got, want, rtol=1e-15, atol=0, err_msg=name)

    chk(orc.apriori_initial(d, e, b), "apriori_initial")
    for k in (1, 2, 3):
        chk(orc.apriori_k(d, e, b, k), "apriori_k k=%d" % k)
    for k in (1, 2):
        chk(orc.apriori_from_e0(d, e, e0, k), "apriori_from_e0 k=%d" % k)
    ab = orc.apost_bound(d, e, du)
    chk(ab, "apost_bound")
    assert orc.efficiency(0.5, ab) == pytest.approx(float(hv["efficiency"][0]), rel=1e-15)
    # the printed range 1 <= n < N gives the other value (reading G11 takes n <= N)
    assert 0.5 / ab[1:-1].max() == pytest.approx(float(hv["efficiency_printed_range"][0]), rel=1e-15)


def _scalar_problem(orc, N=7, M=3, dt=0.1, lam=2.0):
    """Scalar u' = -lam u + f(t) with f > 0 and u0 > 0 (one degree of freedom)."""
    op = orc.Tridiag(np.zeros(1), np.array([lam]), np.zeros(1))
    g = np.ones((1, 1))
    t = dt * np.arange(1, N * M + 1)
    c = (1.0 + 0.5 * np.sin(3.0 * t))[:, None]          # positive source values
    u0 = np.array([1.3])
    return op, g, c, u0


def test_apost_bound_is_exact_on_scalar_rank0(orc):
    """A case where the a posteriori bound is attained.  For one degree of
    freedom and rank R = 0, G_n' = 0 and delta = eps = f := (1 + dt lam)^-M
    (sigma_1 of the scalar F'); with u0 > 0 and b_n > 0 every Parareal
    increment u^k_m - u^{k-1}_m = f^k b_{m-k} is positive, so the triangle
    inequality in the proof of Eq. apost_bound holds with equality and the
    bound equals ||e^k_n|| for every n and k.  An off-by-one in the sum, a
    wrong power of delta or a missing factor eps fails this.  The efficiency
    of Eq. def_efficiency is then exactly 1."""
    N, M, dt, lam = 7, 3, 0.1, 2.0
    op, g, c, u0 = _scalar_problem(orc, N, M, dt, lam)
    f = (1.0 + dt * lam) ** (-M)
    co = orc.build_coarse(op, dt, M, N, 0, 1, 0)
    assert co.delta == pytest.approx(f, rel=1e-14) and co.eps == pytest.approx(f, rel=1e-14)
    ref = orc.sequential_fine(op, dt, M, N, u0, g, c)
    res = orc.parareal(op, dt, M, N, co, u0, g, c, K=N)
    assert np.all(res.b[:, 0] > 0)
    for k in range(1, N):
        err = np.abs(res.iterates[k][:, 0] - ref[:, 0])
        inc = res.iterates[k][:, 0] - res.iterates[k - 1][:, 0]
        assert np.all(inc[k:] > 0) and np.all(inc[:k] == 0)
        # n <= k: both vanish (the iterate is exact up to the rounding of
        # F u + b - b); n > k: the bound equals the error
        assert np.all(res.bounds[k - 1][:k + 1] == 0)
        assert np.all(err[:k + 1] <= 1e-15 * np.abs(ref).max())
        np.testing.assert_allclose(res.bounds[k - 1][k + 1:], err[k + 1:], rtol=1e-12, atol=0)
        assert np.all(err[k + 1:] > 0)
        assert orc.efficiency(err.max(), res.bounds[k - 1]) == pytest.approx(1.0, rel=1e-12)


def test_initial_and_apriori_bounds_on_scalar_rank0(orc):
    """Same scalar rank-0 problem: e^0_n = -sum_{m<n} f^{n-m} b_m and
    e^k_n = f^k e^0_{n-k} (the error identity with G' = 0), so the
    m = n-1 term of Eq. error_bound_initial (min = eps) is attained while
    the others take 2 delta: bound_n = 2 ||e^0_n|| - f ||b_{n-1}||.  In
    Eq. error_bound_eps_delta the m = n-k term, binom(k, k-1) = k, carries
    e^k_n itself: bound_n = k ||e^k_n|| + (terms m < n-k) for delta = eps."""
    N, M, dt, lam = 6, 4, 0.05, 3.0
    op, g, c, u0 = _scalar_problem(orc, N, M, dt, lam)
    f = (1.0 + dt * lam) ** (-M)
    co = orc.build_coarse(op, dt, M, N, 0, 1, 0)
    ref = orc.sequential_fine(op, dt, M, N, u0, g, c)
    res = orc.parareal(op, dt, M, N, co, u0, g, c, K=N)
    bn = np.concatenate([[abs(u0[0])], np.abs(res.b[:-1, 0])])
    e0 = np.abs(res.iterates[0][:, 0] - ref[:, 0])
    bnd0 = orc.apriori_initial(co.delta, co.eps, bn)
    for n in range(1, N + 1):
        assert bnd0[n] == pytest.approx(2 * e0[n] - f * bn[n - 1], rel=1e-12)
    for k in range(1, N):
        ek = np.abs(res.iterates[k][:, 0] - ref[:, 0])
        np.testing.assert_allclose(ek[k + 1:], f ** k * e0[1:N - k + 1], rtol=1e-12)
        bk = orc.apriori_from_e0(co.delta, co.eps, e0, k)
        tail = np.array([sum(math.comb(n - m, k - 1) * f ** (n - m) * e0[m] for m in range(1, n - k))
                         for n in range(N + 1)])
        np.testing.assert_allclose(bk[k + 1:], k * ek[k + 1:] + tail[k + 1:], rtol=1e-12)
