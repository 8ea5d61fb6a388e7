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
