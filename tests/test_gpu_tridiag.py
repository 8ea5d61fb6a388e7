"""GPU parity of the 1D (tridiagonal) hot path against the FP64 oracle.

Rows covered: sketch vectors (rSVD step 1), the batched fine propagator F, F'
and F'^* (forward and adjoint sketches, b_i, Parareal fine solves), the coarse
build (rSVD steps 2-6), and the Parareal solve with the fused coarse sweep and
the a posteriori bound.  Tolerances: 1e-10 relative L2 in the all-FP64 path;
the FP32 paths state theirs per test.
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


# ---------------------------------------------------------------------------
# sketch vectors
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("interval,ncol,n", [(0, 12, 255), (37, 3, 4095), (5, 1, 1)])
def test_gaussian_matches_oracle(ctx, orc, interval, ncol, n):
    got = api.gaussian(ctx, 0, interval, ncol, n)
    want = orc.gauss_block(0, interval, n, ncol)
    # same Philox words; libm vs CUDA log/cos differ by a few ulp
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-14)
    got32 = api.gaussian(ctx, 0, interval, ncol, n, prec="mixed")
    # FP32 deviate from 24-bit uniforms: agrees to FP32 accuracy except where
    # U1 is tiny (its 24-bit rounding then shows in log U1)
    close = np.abs(got32 - want) <= 2e-5 * (1 + np.abs(want))
    assert close.mean() >= 0.999 and np.max(np.abs(got32 - want)) < 0.05


# ---------------------------------------------------------------------------
# fine propagator
# ---------------------------------------------------------------------------
OPS = {
    "heat": lambda n: W.heat1d_op(n),
    "adr": lambda n: W.adr1d_op(n),
}


@pytest.mark.parametrize("kind", ["heat", "adr"])
@pytest.mark.parametrize("n", [2, 3, 17, 255, 1000, 4095])
@pytest.mark.parametrize("adjoint", [False, True])
def test_propagate_f64_parity(ctx, orc, kind, n, adjoint):
    lo, di, up = OPS[kind](n)
    dt, M = 1.0 / 16384, 9
    op = api.Operator.tridiag(ctx, lo, di, up)
    rng = np.random.default_rng(n)
    X = rng.standard_normal((5, n))
    got = api.propagate(ctx, op, dt, M, X, adjoint=adjoint)
    want = orc.propagate(orc.Tridiag(lo, di, up), dt, M, X, adjoint=adjoint)
    # rounding of two different elimination orders: ~ cond(I + dt A) u per step
    cond = 1 + 2 * dt * np.max(np.abs(lo) + np.abs(di) + np.abs(up))
    tol = max(1e-12, 4 * M * cond * 2.2e-16)
    for v in range(X.shape[0]):
        e = rel(got[v], want[v])
        assert e <= tol, (e, tol)


@pytest.mark.parametrize("n", [255, 4095])
def test_propagate_source_parity(ctx, orc, n):
    P = W.heat1d(n=n, N=4, M=16)
    op = api.Operator.tridiag(ctx, P.lo, P.di, P.up)
    X = np.stack([P.u0, np.zeros(n), P.u0 * 3])
    cs = np.stack([P.c[0:16], P.c[16:32], P.c[32:48]])
    got = api.propagate(ctx, op, P.dt, P.M, X, g=P.g, c=cs)
    want = orc.propagate(orc.Tridiag(P.lo, P.di, P.up), P.dt, P.M, X, g=P.g, cvals=cs)
    cond = 1 + 4 * P.dt * (P.n + 1) ** 2
    tol = max(1e-12, 4 * P.M * cond * 2.2e-16)
    for v in range(3):
        e = rel(got[v], want[v])
        assert e <= tol, (e, tol)


@pytest.mark.parametrize("adjoint", [False, True])
def test_propagate_f32_parity(ctx, orc, adjoint):
    P = W.adr1d(n=4095, N=64, M=256)
    op = api.Operator.tridiag(ctx, P.lo, P.di, P.up)
    X = np.random.default_rng(3).standard_normal((7, P.n))
    got = api.propagate(ctx, op, P.dt, P.M, X, adjoint=adjoint, prec="mixed")
    want = orc.propagate(orc.Tridiag(P.lo, P.di, P.up), P.dt, P.M, X, adjoint=adjoint)
    for v in range(X.shape[0]):
        assert rel(got[v], want[v]) <= 2e-5          # FP32 arithmetic, 256 steps


def test_propagate_many_systems_and_empty(ctx, orc):
    """A batch spanning several CTAs per SM and a ragged count of systems."""
    lo, di, up = W.adr1d_op(255)
    op = api.Operator.tridiag(ctx, lo, di, up)
    X = np.random.default_rng(5).standard_normal((1237, 255))
    got = api.propagate(ctx, op, 1e-3, 4, X)
    want = orc.propagate(orc.Tridiag(lo, di, up), 1e-3, 4, X)
    assert np.max(np.linalg.norm(got - want, axis=1) / np.linalg.norm(want, axis=1)) <= 1e-12
    empty = api.propagate(ctx, op, 1e-3, 4, np.zeros((0, 255)))
    assert empty.shape == (0, 255)
    same = api.propagate(ctx, op, 1e-3, 0, X[:3])
    np.testing.assert_array_equal(same, X[:3])


# ---------------------------------------------------------------------------
# coarse build (rSVD)
# ---------------------------------------------------------------------------
def _operator_diff(orc_c, U, S, V, probes):
    Go = orc_c.U @ np.diag(orc_c.S) @ orc_c.V.T
    Gg = U.T @ np.diag(S) @ V
    return max(np.linalg.norm((Gg - Go) @ x) / np.linalg.norm(x) for x in probes)


@pytest.mark.parametrize("which", ["heat1d", "adr1d_small"])
def test_build_coarse_f64_parity(ctx, orc, which):
    if which == "heat1d":
        P = W.heat1d()                     # n=255, N=16, M=64, R=8, p=4
        check = range(P.N)
    else:
        P = W.adr1d(n=511, N=8, M=32, R=6, p=4)
        check = range(P.N)
    op = api.Operator.tridiag(ctx, P.lo, P.di, P.up)
    co = api.Coarse(ctx, op, P.dt, P.M, P.N, P.R, P.p, P.seed, prec="f64")
    info = co.info()
    oop = orc.Tridiag(P.lo, P.di, P.up)
    probes = np.random.default_rng(9).standard_normal((4, P.n))
    for i in check:
        oc = orc.rsvd_interval(oop, P.dt, P.M, i, P.R, P.p, P.seed)
        assert info["R"][i] == oc.S.shape[0]
        s1 = oc.sigma[0]
        kk = min(info["rank_w"][i], info["rank_v"][i])
        m = min(kk, oc.sigma.shape[0])
        assert np.max(np.abs(info["sigma"][i, :m] - oc.sigma[:m])) <= 1e-10 * s1
        U, S, V = co.factors(i)
        assert _operator_diff(oc, U, S, V, probes) <= 1e-10 * s1
    assert abs(info["delta"] - max(orc.rsvd_interval(oop, P.dt, P.M, i, P.R, P.p, P.seed).sigma[0]
                                   for i in check)) <= 1e-10


def test_build_coarse_heat_closed_form(ctx):
    """sigma_j = (1 + dt lam_j)^-M for the 1D heat operator (both precisions)."""
    P = W.heat1d()
    op = api.Operator.tridiag(ctx, P.lo, P.di, P.up)
    h = 1.0 / (P.n + 1)
    j = np.arange(1, P.R + 1)
    sig = (1 + P.dt * 4 / h ** 2 * np.sin(j * np.pi * h / 2) ** 2) ** (-P.M)
    for prec, tol in (("f64", 1e-12), ("mixed", 1e-5)):
        co = api.Coarse(ctx, op, P.dt, P.M, P.N, P.R, P.p, P.seed, prec=prec)
        info = co.info()
        R = info["R"].min()
        assert R >= (P.R if prec == "f64" else 4)
        assert np.max(np.abs(info["sigma"][:, :R] - sig[None, :R])) <= tol * sig[0]


def test_build_coarse_mixed_operator_error(ctx, orc):
    """Mixed build: G' within 1e-4 sigma_1 of the FP64 oracle's on probes."""
    P = W.adr1d(n=1023, N=4, M=64, R=8, p=4)
    op = api.Operator.tridiag(ctx, P.lo, P.di, P.up)
    co = api.Coarse(ctx, op, P.dt, P.M, P.N, P.R, P.p, P.seed, prec="mixed")
    oop = orc.Tridiag(P.lo, P.di, P.up)
    probes = np.random.default_rng(1).standard_normal((3, P.n))
    for i in range(P.N):
        oc = orc.rsvd_interval(oop, P.dt, P.M, i, P.R, P.p, P.seed)
        U, S, V = co.factors(i)
        assert _operator_diff(oc, U, S, V, probes) <= 1e-4 * oc.sigma[0]


# ---------------------------------------------------------------------------
# Parareal
# ---------------------------------------------------------------------------
def _run_both(ctx, orc, P, K=None, tol=0.0, prec="f64"):
    op = api.Operator.tridiag(ctx, P.lo, P.di, P.up)
    co = api.Coarse(ctx, op, P.dt, P.M, P.N, P.R, P.p, P.seed, prec=prec)
    u, info = api.parareal_solve(ctx, co, P.u0, P.g, P.c, K=K, tol=tol)
    return op, co, u, info


@pytest.mark.parametrize("K", [0, 1, 3])
def test_parareal_f64_iterates_match_oracle(ctx, orc, K):
    P = W.adr1d(n=511, N=8, M=32, R=4, p=2)
    P.g, P.c = W.heat1d(n=511, N=8, M=32).g, W.heat1d(n=511, N=8, M=32).c
    op, co, u, info = _run_both(ctx, orc, P, K=K)
    oop = orc.Tridiag(P.lo, P.di, P.up)
    oco = orc.build_coarse(oop, P.dt, P.M, P.N, P.R, P.p, P.seed)
    res = orc.parareal(oop, P.dt, P.M, P.N, oco, P.u0, P.g, P.c, K=K)
    assert info["k_done"] == res.k_done == K
    assert rel(u, res.iterates[-1]) <= 1e-10
    for k in range(1, K + 1):
        np.testing.assert_allclose(info["bounds"][k - 1], res.bounds[k - 1], rtol=1e-8, atol=1e-14)


@pytest.mark.parametrize("R,p", [(20, 4), (16, 4), (5, 2)])
def test_parareal_sweep_ranks_match_oracle(ctx, orc, R, p):
    """The sweep's R x R recurrence runs on one warp for R <= 16 and on the
    whole CTA above; both, and a rank that is not a power of two, give the
    oracle's iterates and bounds."""
    P = W.adr1d(n=511, N=8, M=32, R=R, p=p)
    op, co, u, info = _run_both(ctx, orc, P, K=3)
    oop = orc.Tridiag(P.lo, P.di, P.up)
    oco = orc.build_coarse(oop, P.dt, P.M, P.N, P.R, P.p, P.seed)
    res = orc.parareal(oop, P.dt, P.M, P.N, oco, P.u0, K=3)
    assert info["k_done"] == res.k_done == 3
    assert rel(u, res.iterates[-1]) <= 1e-10
    for k in range(1, 4):
        np.testing.assert_allclose(info["bounds"][k - 1], res.bounds[k - 1], rtol=1e-8, atol=1e-14)


@pytest.mark.parametrize("tol", [1e-2, 1e-4, 1e-6])
def test_parareal_device_stopping_matches_oracle(ctx, orc, tol):
    """The tolerance test runs on the device (the sweep sets a stop flag and
    the kernels of later iterations return at once) while the host enqueues
    iterations in batches of 1, 2, 4, 4, ...; the solve stops at the same
    iteration as the oracle's literal Parareal (here 6, 9 and 13: inside a
    batch), with the same iterate and the same a posteriori bounds."""
    P = W.adr1d(n=511, N=16, M=32, R=8, p=4)
    op = api.Operator.tridiag(ctx, P.lo, P.di, P.up)
    co = api.Coarse(ctx, op, P.dt, P.M, P.N, P.R, P.p, P.seed, prec="f64")
    u, info = api.parareal_solve(ctx, co, P.u0, K=P.N, tol=tol)
    oop = orc.Tridiag(P.lo, P.di, P.up)
    oco = orc.build_coarse(oop, P.dt, P.M, P.N, P.R, P.p, P.seed)
    res = orc.parareal(oop, P.dt, P.M, P.N, oco, P.u0, K=P.N, tol=tol)
    assert info["converged"] and info["k_done"] == res.k_done
    assert res.k_done not in (1, 3, 7, 11, 15)      # not at a batch end
    assert rel(u, res.iterates[-1]) <= 1e-10
    assert info["bounds"].shape[0] == res.k_done
    for k in range(res.k_done):
        np.testing.assert_allclose(info["bounds"][k], res.bounds[k], rtol=1e-8, atol=1e-14)


def test_parareal_heat1d_full_K_equals_N(ctx, orc):
    """Config: n=255, N=16, M=64, R=8, p=4, source sin(2 pi t) exp(-100(x-1/2)^2)."""
    P = W.heat1d()
    op, co, u, info = _run_both(ctx, orc, P, K=P.N)
    ref = orc.sequential_fine(orc.Tridiag(P.lo, P.di, P.up), P.dt, P.M, P.N, P.u0, P.g, P.c)
    assert info["k_done"] == P.N
    assert orc.rel_err(u, ref) <= 1e-10
    # and the device's own sequential sweep (same propagator) agrees to rounding
    fine = api.fine_solution(ctx, op, P.dt, P.M, P.N, P.u0, P.g, P.c)
    assert orc.rel_err(fine, ref) <= 1e-12
    assert np.max(np.abs(u - fine)) <= 1e-13 * np.abs(fine).max()


def test_parareal_heat1d_tol(ctx, orc):
    P = W.heat1d()
    op, co, u, info = _run_both(ctx, orc, P, K=P.N, tol=1e-10)
    ref = orc.sequential_fine(orc.Tridiag(P.lo, P.di, P.up), P.dt, P.M, P.N, P.u0, P.g, P.c)
    assert info["converged"]
    assert orc.rel_err(u, ref) <= 1e-10
    assert info["k_done"] <= 2


def test_parareal_finite_termination_and_R0(ctx, orc):
    P = W.adr1d(n=255, N=6, M=16, R=0, p=2)
    op, co, u, info = _run_both(ctx, orc, P, K=2)
    oop = orc.Tridiag(P.lo, P.di, P.up)
    ref = orc.sequential_fine(oop, P.dt, P.M, P.N, P.u0)
    err = np.linalg.norm(u - ref, axis=1)
    assert np.all(err[:3] <= 1e-13 * np.abs(ref).max())      # u^k_n exact for n <= k
    oco = orc.build_coarse(oop, P.dt, P.M, P.N, P.R, P.p, P.seed)
    res = orc.parareal(oop, P.dt, P.M, P.N, oco, P.u0, K=2)
    assert rel(u, res.iterates[-1]) <= 1e-10


@pytest.mark.parametrize("prec", ["f64", "mixed"])
def test_parareal_adr1d_full_size_to_1e8(ctx, orc, prec):
    """Full configuration n=4095, N=64, M=256, R=16, p=8 with tol 1e-8: the
    last iterate is within 1e-8 (relative, max over time) of the oracle's
    sequential FP64 fine solution, and the build's singular values match the
    oracle's randomized SVD on sampled intervals."""
    P = W.adr1d()
    op, co, u, info = _run_both(ctx, orc, P, K=P.N, tol=1e-8, prec=prec)
    oop = orc.Tridiag(P.lo, P.di, P.up)
    ref = orc.sequential_fine(oop, P.dt, P.M, P.N, P.u0)
    assert info["converged"]
    assert orc.rel_err(u, ref) <= 1e-8
    inf = co.info()
    for i in (0, 41):
        oc = orc.rsvd_interval(oop, P.dt, P.M, i, P.R, P.p, P.seed)
        tol = 1e-10 if prec == "f64" else 1e-4
        assert np.max(np.abs(inf["sigma"][i] - oc.sigma)) <= tol * oc.sigma[0]


def test_parareal_invalid_arguments(ctx):
    P = W.heat1d(n=31, N=2, M=4, R=2, p=1)
    op = api.Operator.tridiag(ctx, P.lo, P.di, P.up)
    from paper_2508_08873_gb300 import _native
    with pytest.raises(_native.LrpError):
        api.Coarse(ctx, op, P.dt, P.M, P.N, 40, 1, 0)       # rank + p > n
    with pytest.raises(_native.LrpError):
        api.Coarse(ctx, op, -1.0, P.M, P.N, 2, 1, 0)


@pytest.mark.parametrize("n,nvec", [(2048, 60), (4095, 5), (4095, 60), (7777, 3), (16384, 2)])
@pytest.mark.parametrize("adjoint", [False, True])
def test_propagate_cluster_paths_f64(ctx, orc, n, nvec, adjoint):
    """Batches small enough to spread each system over a 2- or 4-CTA cluster."""
    lo, di, up = W.adr1d_op(n)
    dt, M = 1.0 / 16384, 7
    op = api.Operator.tridiag(ctx, lo, di, up)
    X = np.random.default_rng(n + nvec).standard_normal((nvec, n))
    got = api.propagate(ctx, op, dt, M, X, adjoint=adjoint)
    want = orc.propagate(orc.Tridiag(lo, di, up), dt, M, X, adjoint=adjoint)
    cond = 1 + 2 * dt * np.max(np.abs(lo) + np.abs(di) + np.abs(up))
    tol = max(1e-12, 4 * M * cond * 2.2e-16)
    e = max(rel(got[v], want[v]) for v in range(nvec))
    assert e <= tol, (e, tol)
    got32 = api.propagate(ctx, op, dt, M, X[:2], adjoint=adjoint, prec="mixed")
    assert max(rel(got32[v], want[v]) for v in range(2)) <= 2e-5


def test_coarse_checkpoint_roundtrip(ctx, tmp_path):
    """A saved coarse handle reproduces the solves of the original bitwise."""
    P = W.heat1d(n=255, N=8, M=32, R=6, p=3)
    op = api.Operator.tridiag(ctx, P.lo, P.di, P.up)
    co = api.Coarse(ctx, op, P.dt, P.M, P.N, P.R, P.p, 0, prec="mixed")
    u1, i1 = api.parareal_solve(ctx, co, P.u0, P.g, P.c, K=3)
    path = str(tmp_path / "coarse.npz")
    co.save(path)
    co2 = api.Coarse.load(ctx, op, path)
    u2, i2 = api.parareal_solve(ctx, co2, P.u0, P.g, P.c, K=3)
    np.testing.assert_array_equal(u1, u2)
    a, b = co.info(), co2.info()
    np.testing.assert_array_equal(a["sigma"], b["sigma"])
    assert a["eps"] == b["eps"] and a["delta"] == b["delta"]


def test_sweep_slicing_does_not_change_the_iterates(ctx, orc):
    """The coarse sweep's partial sums per row slice are combined in a fixed
    order; several slices per vector give the iterates of one slice to
    rounding, and both match the oracle."""
    P = W.heat1d()
    op = api.Operator.tridiag(ctx, P.lo, P.di, P.up)
    co = api.Coarse(ctx, op, P.dt, P.M, P.N, P.R, P.p, P.seed, prec="f64")
    ref, _ = api.parareal_solve(ctx, co, P.u0, P.g, P.c, K=3)
    try:
        ctx.set_param("sweep_rows", 128)          # n = 255: two slices
        u, _ = api.parareal_solve(ctx, co, P.u0, P.g, P.c, K=3)
    finally:
        ctx.set_param("sweep_rows", 0)
    assert rel(u, ref) <= 1e-13
    oop = orc.Tridiag(P.lo, P.di, P.up)
    oco = orc.build_coarse(oop, P.dt, P.M, P.N, P.R, P.p, P.seed)
    res = orc.parareal(oop, P.dt, P.M, P.N, oco, P.u0, P.g, P.c, K=3)
    assert rel(u, res.iterates[-1]) <= 1e-10


@pytest.mark.parametrize("wchunk", [0, 9, 10, 11, 12, 13, 14, 15, 16])
@pytest.mark.parametrize("n,nvec,Q", [(3000, 7, 2), (1025, 9, 0), (4096, 40, 1), (200, 3, 1)])
def test_warp_cluster_kernel_matches_block_kernel_and_oracle(ctx, orc, n, nvec, Q, wchunk):
    """FP64 batches with n <= 4096 run on the one-warp-per-CTA cluster kernel
    (1..16 CTAs of 32 chunks of 8 to 16 rows); it agrees with the
    block kernel (tri_warp = 1) to rounding and with the oracle, with and
    without a source term, forward and adjoint."""
    lo, di, up = W.adr1d_op(n)
    dt, M = 1.0 / 16384, 9
    op = api.Operator.tridiag(ctx, lo, di, up)
    rng = np.random.default_rng(n)
    X = rng.standard_normal((nvec, n))
    g = rng.standard_normal((Q, n)) if Q else None
    c = rng.standard_normal((nvec, M, Q)) if Q else None
    oop = orc.Tridiag(lo, di, up)
    cond = 1 + 2 * dt * np.max(np.abs(lo) + np.abs(di) + np.abs(up))
    tol = max(1e-12, 4 * M * cond * 2.2e-16)
    for adjoint in (False, True):
        if adjoint and Q:
            continue
        try:
            ctx.set_param("tri_warp", 2)
            ctx.set_param("tri_wchunk", wchunk)
            got = api.propagate(ctx, op, dt, M, X, adjoint=adjoint, g=g, c=c)
        finally:
            ctx.set_param("tri_warp", 0)
            ctx.set_param("tri_wchunk", 0)
        try:
            ctx.set_param("tri_warp", 1)
            blk = api.propagate(ctx, op, dt, M, X, adjoint=adjoint, g=g, c=c)
        finally:
            ctx.set_param("tri_warp", 0)
        want = orc.propagate(oop, dt, M, X, adjoint=adjoint, g=g, cvals=c)
        for v in range(nvec):
            assert rel(got[v], want[v]) <= tol
            assert rel(got[v], blk[v]) <= tol


@pytest.mark.parametrize("M", [0, 1, 2, 3])
def test_warp_cluster_kernel_few_steps(ctx, orc, M):
    """The one-warp kernel defers each step's spike correction into the next
    step's interior solve and applies the last one with the spike vectors
    themselves: with 0 steps the input comes back unchanged, and 1, 2 and 3
    steps (no deferred correction, one, two) match the oracle, with a source
    term."""
    n, nvec, Q = 2049, 5, 2
    lo, di, up = W.adr1d_op(n)
    dt = 1.0 / 4096
    op = api.Operator.tridiag(ctx, lo, di, up)
    rng = np.random.default_rng(M)
    X = rng.standard_normal((nvec, n))
    g = rng.standard_normal((Q, n))
    c = rng.standard_normal((nvec, max(M, 1), Q))[:, :M, :]
    try:
        ctx.set_param("tri_warp", 2)
        if M == 0:
            got = api.propagate(ctx, op, dt, M, X)
        else:
            got = api.propagate(ctx, op, dt, M, X, g=g, c=np.ascontiguousarray(c))
    finally:
        ctx.set_param("tri_warp", 0)
    if M == 0:
        np.testing.assert_array_equal(got, X)
        return
    want = orc.propagate(orc.Tridiag(lo, di, up), dt, M, X, g=g, cvals=c)
    for v in range(nvec):
        assert rel(got[v], want[v]) <= 1e-12


@pytest.mark.parametrize("wsplit", [0, 1])
@pytest.mark.parametrize("wchunk", [8, 12, 16])
@pytest.mark.parametrize("n,nvec,Q,M", [(3000, 7, 2, 9), (1025, 9, 0, 9), (2049, 5, 2, 1),
                                        (2049, 5, 0, 2), (8192, 3, 1, 3)])
def test_warp_cluster_kernel_split_variants(ctx, orc, n, nvec, Q, M, wchunk, wsplit):
    """The split of the chunk-interior solve around the cluster barrier
    (tri_wsplit 0: all of it before the wait; 1, the default: its last
    backward rows after it) changes only the order of independent work: both
    variants match the oracle, with and without a source, for 1, 2 and 9
    steps."""
    lo, di, up = W.adr1d_op(n)
    dt = 1.0 / 16384
    op = api.Operator.tridiag(ctx, lo, di, up)
    rng = np.random.default_rng(n + M)
    X = rng.standard_normal((nvec, n))
    g = rng.standard_normal((Q, n)) if Q else None
    c = rng.standard_normal((nvec, M, Q)) if Q else None
    cond = 1 + 2 * dt * np.max(np.abs(lo) + np.abs(di) + np.abs(up))
    tol = max(1e-12, 4 * M * cond * 2.2e-16)
    try:
        ctx.set_param("tri_warp", 2)
        ctx.set_param("tri_wchunk", wchunk)
        ctx.set_param("tri_wsplit", wsplit)
        got = api.propagate(ctx, op, dt, M, X, g=g, c=c)
    finally:
        ctx.set_param("tri_warp", 0)
        ctx.set_param("tri_wchunk", 0)
        ctx.set_param("tri_wsplit", 1)
    want = orc.propagate(orc.Tridiag(lo, di, up), dt, M, X, g=g, cvals=c)
    for v in range(nvec):
        assert rel(got[v], want[v]) <= tol


@pytest.mark.parametrize("prec", ["mixed", "f64"])
@pytest.mark.parametrize("wchunk", [8, 12, 16])
@pytest.mark.parametrize("n,nvec,Q,M", [(4095, 200, 0, 37), (1000, 3, 2, 9), (255, 9, 1, 5),
                                        (100, 5, 0, 1), (2049, 4, 0, 0)])
def test_block_warp_kernel_matches_oracle(ctx, orc, n, nvec, Q, M, wchunk, prec):
    """One system per CTA of C warps (tri_wblock = 1; the FP32 sketches take
    it by default): forward and adjoint, with and without a source, against
    the oracle (FP32 to 2e-5, FP64 to rounding).  FP64 takes at most 8 warps
    per CTA: longer systems are refused with LRP_EINVAL."""
    lo, di, up = W.adr1d_op(n)
    dt = 1.0 / 16384
    op = api.Operator.tridiag(ctx, lo, di, up)
    rng = np.random.default_rng(n + nvec + M)
    X = rng.standard_normal((nvec, n))
    g = rng.standard_normal((Q, n)) if Q else None
    c = rng.standard_normal((nvec, M, Q)) if Q else None
    cond = 1 + 2 * dt * np.max(np.abs(lo) + np.abs(di) + np.abs(up))
    tol = 2e-5 if prec == "mixed" else max(1e-12, 4 * max(M, 1) * cond * 2.2e-16)
    units = ((n + wchunk - 1) // wchunk + 31) // 32
    oop = orc.Tridiag(lo, di, up)
    for adjoint in (False, True):
        if adjoint and Q:
            continue
        try:
            ctx.set_param("tri_wblock", 1)
            ctx.set_param("tri_wchunk", wchunk)
            if prec == "f64" and units > 8:
                with pytest.raises(_native.LrpError):
                    api.propagate(ctx, op, dt, M, X, adjoint=adjoint, g=g, c=c, prec=prec)
                continue
            got = api.propagate(ctx, op, dt, M, X, adjoint=adjoint, g=g, c=c, prec=prec)
        finally:
            ctx.set_param("tri_wblock", 0)
            ctx.set_param("tri_wchunk", 0)
        if M == 0:
            np.testing.assert_allclose(got, X, rtol=0, atol=1e-6 if prec == "mixed" else 0)
            continue
        want = orc.propagate(oop, dt, M, X, adjoint=adjoint, g=g, cvals=c)
        for v in range(nvec):
            assert rel(got[v], want[v]) <= tol


@pytest.mark.parametrize("n,wchunk", [(4095, 8), (4095, 9), (4095, 13), (4095, 15), (4095, 16),
                                      (3000, 12), (1023, 11), (2048, 16), (300, 10), (8191, 16),
                                      (8192, 16)])
@pytest.mark.parametrize("M", [1, 2, 3, 37, 700])
def test_toeplitz_warp_kernel_matches_oracle(ctx, orc, n, wchunk, M):
    """Constant-coefficient operators take the Toeplitz variant of the
    one-warp kernel (steady LU factors, a Sherman-Morrison term for the first
    row of each chunk, the state carried scaled by the steady pivot and
    rescaled every P steps: 700 steps cross several rescales).  Forward and
    adjoint against the oracle, for chunk lengths with n mod MM = 0 or MM - 1
    (padding rows only in chunks of their own)."""
    lo, di, up = W.adr1d_op(n)
    dt = 1.0 / 16384
    op = api.Operator.tridiag(ctx, lo, di, up)
    X = np.random.default_rng(n + M).standard_normal((6, n))
    oop = orc.Tridiag(lo, di, up)
    cond = 1 + 2 * dt * np.max(np.abs(lo) + np.abs(di) + np.abs(up))
    tol = max(1e-12, 4 * M * cond * 2.2e-16)
    for adjoint in (False, True):
        try:
            ctx.set_param("tri_warp", 2)
            ctx.set_param("tri_wchunk", wchunk)
            ctx.set_param("tri_wtoep", 1)
            got = api.propagate(ctx, op, dt, M, X, adjoint=adjoint)
        finally:
            ctx.set_param("tri_warp", 0)
            ctx.set_param("tri_wchunk", 0)
            ctx.set_param("tri_wtoep", 0)
        want = orc.propagate(oop, dt, M, X, adjoint=adjoint)
        for v in range(X.shape[0]):
            assert rel(got[v], want[v]) <= tol, (adjoint, v, rel(got[v], want[v]), tol)


@pytest.mark.parametrize("dt,M,nvec", [(1.0, 100, 4), (1e-9, 50, 4), (1.0 / 16384, 5, 200)])
def test_toeplitz_warp_kernel_stiff_mild_and_many(ctx, orc, dt, M, nvec):
    """The constant-coefficient kernel with a stiff step (steady pivot
    ~1.7e5: rescaled every 28 steps), an almost-identity step (pivot
    ~1 + 3.4e-4: no rescale) and more systems than resident clusters (each
    cluster loops over systems)."""
    n = 4095
    lo, di, up = W.adr1d_op(n)
    op = api.Operator.tridiag(ctx, lo, di, up)
    X = np.random.default_rng(nvec + M).standard_normal((nvec, n))
    cond = 1 + 2 * dt * np.max(np.abs(lo) + np.abs(di) + np.abs(up))
    tol = max(1e-12, 4 * M * min(cond, 1e4) * 2.2e-16)
    try:
        ctx.set_param("tri_warp", 2)
        ctx.set_param("tri_wchunk", 13)
        ctx.set_param("tri_wtoep", 1)
        got = api.propagate(ctx, op, dt, M, X)
    finally:
        ctx.set_param("tri_warp", 0)
        ctx.set_param("tri_wchunk", 0)
        ctx.set_param("tri_wtoep", 0)
    rows = list(range(0, nvec, max(1, nvec // 5)))
    want = orc.propagate(orc.Tridiag(lo, di, up), dt, M, X[rows])
    for k, v in enumerate(rows):
        assert rel(got[v], want[k]) <= tol, (v, rel(got[v], want[k]), tol)


@pytest.mark.parametrize("M", [1, 37, 300])
def test_toeplitz_block_kernel_f32(ctx, orc, M):
    """FP32 batches of a constant-coefficient operator (the sketches) run the
    FP32 block variant (S phi and S fq in shared memory, three CTAs per SM,
    rescaled every 13 steps): forward and adjoint against the oracle to FP32
    accuracy, and against the general FP32 block kernel."""
    n, nvec = 4095, 300
    lo, di, up = W.adr1d_op(n)
    dt = 1.0 / 16384
    op = api.Operator.tridiag(ctx, lo, di, up)
    X = np.random.default_rng(M).standard_normal((nvec, n))
    oop = orc.Tridiag(lo, di, up)
    for adjoint in (False, True):
        got = api.propagate(ctx, op, dt, M, X, adjoint=adjoint, prec="mixed")
        try:
            ctx.set_param("tri_wtoep", 2)
            gen = api.propagate(ctx, op, dt, M, X, adjoint=adjoint, prec="mixed")
        finally:
            ctx.set_param("tri_wtoep", 0)
        rows = list(range(0, nvec, 50))
        want = orc.propagate(oop, dt, M, X[rows], adjoint=adjoint)
        for k, v in enumerate(rows):
            assert rel(got[v], want[k]) <= 2e-5
        for v in range(nvec):
            assert rel(got[v], gen[v]) <= 4e-5


def test_toeplitz_warp_kernel_heat_and_eligibility(ctx, orc):
    """The heat operator (symmetric, diffusion only) on the Toeplitz variant
    matches the oracle; a variable-coefficient operator, a source term or a
    chunk length with n mod MM not in {0, MM - 1} are refused when the
    variant is forced, and fall back to the general kernel otherwise."""
    n, M, dt = 4095, 64, 1.0 / 1024
    lo, di, up = W.heat1d_op(n)
    X = np.random.default_rng(1).standard_normal((5, n))
    op = api.Operator.tridiag(ctx, lo, di, up)
    want = orc.propagate(orc.Tridiag(lo, di, up), dt, M, X)
    cond = 1 + 2 * dt * np.max(np.abs(lo) + np.abs(di) + np.abs(up))
    tol = max(1e-12, 4 * M * cond * 2.2e-16)
    try:
        ctx.set_param("tri_warp", 2)
        ctx.set_param("tri_wtoep", 1)
        got = api.propagate(ctx, op, dt, M, X)
        for v in range(5):
            assert rel(got[v], want[v]) <= tol
        g = np.ones((1, n))
        c = np.ones((M, 1))
        with pytest.raises(_native.LrpError):
            api.propagate(ctx, op, dt, M, X, g=g, c=c)
        ctx.set_param("tri_wchunk", 12)            # 4095 mod 12 = 3
        with pytest.raises(_native.LrpError):
            api.propagate(ctx, op, dt, M, X)
        ctx.set_param("tri_wchunk", 0)
        lo2 = lo * (1.0 + 0.01 * np.sin(np.arange(n)))
        op2 = api.Operator.tridiag(ctx, lo2, di, up)
        with pytest.raises(_native.LrpError):
            api.propagate(ctx, op2, dt, M, X)
        ctx.set_param("tri_wtoep", 0)
        got2 = api.propagate(ctx, op2, dt, M, X)
        want2 = orc.propagate(orc.Tridiag(lo2, di, up), dt, M, X)
        for v in range(5):
            assert rel(got2[v], want2[v]) <= tol
    finally:
        ctx.set_param("tri_warp", 0)
        ctx.set_param("tri_wchunk", 0)
        ctx.set_param("tri_wtoep", 0)


@pytest.mark.parametrize("n,nvec,M", [(4095, 300, 37), (511, 20, 700), (1023, 400, 3), (2048, 290, 1),
                                    (255, 9, 5)])
def test_toeplitz_block_kernel_matches_oracle(ctx, orc, n, nvec, M):
    """FP64 batches too large for the cluster kernels (or systems too short
    for them) with constant coefficients run the block variant of the
    constant-coefficient kernel (one system per CTA of 2 to 8 warps; n = 255
    stays on the general path): forward and adjoint against the oracle and
    against the general path (tri_wtoep = 2)."""
    lo, di, up = W.adr1d_op(n)
    dt = 1.0 / 16384
    op = api.Operator.tridiag(ctx, lo, di, up)
    X = np.random.default_rng(n + M).standard_normal((nvec, n))
    oop = orc.Tridiag(lo, di, up)
    cond = 1 + 2 * dt * np.max(np.abs(lo) + np.abs(di) + np.abs(up))
    tol = max(1e-12, 4 * M * cond * 2.2e-16)
    for adjoint in (False, True):
        try:
            ctx.set_param("tri_warp", 1)             # not the cluster kernels
            got = api.propagate(ctx, op, dt, M, X, adjoint=adjoint)
            ctx.set_param("tri_wtoep", 2)
            gen = api.propagate(ctx, op, dt, M, X, adjoint=adjoint)
        finally:
            ctx.set_param("tri_wtoep", 0)
            ctx.set_param("tri_warp", 0)
        rows = range(0, nvec, max(1, nvec // 7))
        want = orc.propagate(oop, dt, M, X[list(rows)], adjoint=adjoint)
        for k, v in enumerate(rows):
            assert rel(got[v], want[k]) <= tol
        for v in range(nvec):
            assert rel(got[v], gen[v]) <= tol


# ---------------------------------------------------------------------------
# classical Parareal (backward-Euler coarse step), the comparison method
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("K", [0, 1, 3])
def test_classical_parareal_matches_oracle(ctx, orc, K):
    P = W.heat1d(n=255, N=8, M=16)
    op = api.Operator.tridiag(ctx, P.lo, P.di, P.up)
    u, info = api.parareal_solve_classical(ctx, op, P.dt, P.M, P.N, P.u0, P.g, P.c, K=K)
    res = orc.parareal_classical(orc.Tridiag(P.lo, P.di, P.up), P.dt, P.M, P.N, P.u0, P.g, P.c, K=K)
    assert info["k_done"] == res.k_done == K
    assert rel(u, res.iterates[-1]) <= 1e-10
    for k in range(1, K + 1):
        d = res.bounds[k - 1]
        want = np.max(d) / np.max(np.linalg.norm(res.iterates[k], axis=1))
        assert abs(info["increments"][k - 1] - want) <= 1e-8 * want


def test_classical_parareal_adr1d_K_equals_N(ctx, orc):
    """Full adr1d size: K = N reproduces the sequential fine solution."""
    P = W.adr1d()
    op = api.Operator.tridiag(ctx, P.lo, P.di, P.up)
    oop = orc.Tridiag(P.lo, P.di, P.up)
    ref = orc.sequential_fine(oop, P.dt, P.M, P.N, P.u0)
    u, info = api.parareal_solve_classical(ctx, op, P.dt, P.M, P.N, P.u0, K=P.N)
    assert info["k_done"] == P.N
    assert orc.rel_err(u, ref) <= 1e-10


def test_low_rank_beats_classical_on_heat(ctx, orc):
    """Experiment 1's comparison on the heat configuration (n=255, N=16,
    M=64, R=8, p=4): after the same number of iterations the low-rank coarse
    solvers are far more accurate than one backward-Euler coarse step."""
    P = W.heat1d()
    op = api.Operator.tridiag(ctx, P.lo, P.di, P.up)
    ref = orc.sequential_fine(orc.Tridiag(P.lo, P.di, P.up), P.dt, P.M, P.N, P.u0, P.g, P.c)
    co = api.Coarse(ctx, op, P.dt, P.M, P.N, P.R, P.p, P.seed, prec="f64")
    for K in (1, 2):
        uc, _ = api.parareal_solve_classical(ctx, op, P.dt, P.M, P.N, P.u0, P.g, P.c, K=K)
        ul, _ = api.parareal_solve(ctx, co, P.u0, P.g, P.c, K=K)
        e_cl, e_lr = orc.rel_err(uc, ref), orc.rel_err(ul, ref)
        assert e_lr < 1e-3 * e_cl, (K, e_lr, e_cl)


# ---------------------------------------------------------------------------
# two-sided sketch variant (F'^* on independent random vectors, Sec. 2.2)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("which", ["heat", "adr"])
def test_build_two_sided_matches_oracle(ctx, orc, which):
    if which == "heat":
        P = W.heat1d(n=255, N=6, M=32, R=6, p=3)
    else:
        P = W.adr1d(n=1023, N=4, M=64, R=8, p=4)
    op = api.Operator.tridiag(ctx, P.lo, P.di, P.up)
    co = api.Coarse(ctx, op, P.dt, P.M, P.N, P.R, P.p, P.seed, prec="f64", independent_adjoint=True)
    info = co.info()
    oop = orc.Tridiag(P.lo, P.di, P.up)
    probes = np.random.default_rng(11).standard_normal((3, P.n))
    for i in range(P.N):
        oc = orc.rsvd_interval_indep(oop, P.dt, P.M, i, P.R, P.p, P.seed)
        s1 = oc.sigma[0]
        assert info["R"][i] == oc.S.shape[0]
        assert np.max(np.abs(info["sigma"][i, :oc.S.shape[0]] - oc.S)) <= 1e-9 * s1
        U, S, V = co.factors(i)
        assert _operator_diff(oc, U, S, V, probes) <= 1e-9 * s1
    # the coarse solvers drive Parareal to the fine solution
    u, pinfo = api.parareal_solve(ctx, co, P.u0, P.g, P.c, K=P.N)
    ref = orc.sequential_fine(oop, P.dt, P.M, P.N, P.u0, P.g, P.c)
    assert orc.rel_err(u, ref) <= 1e-10


def test_build_two_sided_mixed_close_to_two_pass(ctx, orc):
    """Mixed precision, heat: the two-sided coarse operators agree with the
    closed-form leading singular values to the FP32 sketch accuracy."""
    P = W.heat1d()
    op = api.Operator.tridiag(ctx, P.lo, P.di, P.up)
    co = api.Coarse(ctx, op, P.dt, P.M, P.N, P.R, P.p, P.seed, prec="mixed", independent_adjoint=True)
    info = co.info()
    h = 1.0 / (P.n + 1)
    lam = 4.0 / h ** 2 * np.sin(np.arange(1, P.n + 1) * np.pi * h / 2) ** 2
    sig = (1.0 + P.dt * lam) ** (-P.M)
    for i in range(P.N):
        assert np.max(np.abs(info["sigma"][i, :4] - sig[:4])) <= 1e-4 * sig[0]


# ---------------------------------------------------------------------------
# SDIRK fine steppers (Sec. 4, effect of the time discretisation)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("scheme", ["sdirk2", "sdirk2l"])
@pytest.mark.parametrize("n", [255, 4095])
def test_sdirk_propagate_parity(ctx, orc, scheme, n):
    lo, di, up = W.adr1d_op(n)
    dt, M = 1.0 / 16384, 9
    op = api.Operator.tridiag(ctx, lo, di, up)
    op.set_stepper(scheme)
    oop = orc.Tridiag(lo, di, up, stepper=scheme)
    X = np.random.default_rng(n).standard_normal((5, n))
    cond = 1 + 2 * dt * np.max(np.abs(lo) + np.abs(di) + np.abs(up))
    tol = max(1e-12, 8 * M * cond * 2.2e-16)
    for adjoint in (False, True):
        got = api.propagate(ctx, op, dt, M, X, adjoint=adjoint)
        want = orc.propagate(oop, dt, M, X, adjoint=adjoint)
        assert max(rel(got[v], want[v]) for v in range(5)) <= tol
        got32 = api.propagate(ctx, op, dt, M, X[:2], adjoint=adjoint, prec="mixed")
        assert max(rel(got32[v], want[v]) for v in range(2)) <= 5e-5
    # a source takes two samples per step with these steppers
    with pytest.raises(ValueError):
        api.propagate(ctx, op, dt, M, X[:1], g=np.ones((1, n)), c=np.ones((M, 1)))


def test_sdirk2l_build_and_parareal(ctx, orc):
    """Low-rank Parareal with an SDIRK2-L fine solver: the build matches the
    oracle's, and K = N reproduces the oracle's sequential SDIRK2-L solution."""
    P = W.heat1d(n=127, N=6, M=16, R=5, p=3)
    op = api.Operator.tridiag(ctx, P.lo, P.di, P.up)
    op.set_stepper("sdirk2l")
    oop = orc.Tridiag(P.lo, P.di, P.up, stepper="sdirk2l")
    co = api.Coarse(ctx, op, P.dt, P.M, P.N, P.R, P.p, P.seed, prec="f64")
    info = co.info()
    oco = orc.build_coarse(oop, P.dt, P.M, P.N, P.R, P.p, P.seed)
    for i in range(P.N):
        oc = oco.intervals[i]
        assert np.max(np.abs(info["sigma"][i, :oc.S.shape[0]] - oc.S)) <= 1e-9 * oc.sigma[0]
    u, _ = api.parareal_solve(ctx, co, P.u0, K=P.N)
    ref = orc.sequential_fine(oop, P.dt, P.M, P.N, P.u0)
    assert orc.rel_err(u, ref) <= 1e-10
    res = orc.parareal(oop, P.dt, P.M, P.N, oco, P.u0, K=2)
    u2, _ = api.parareal_solve(ctx, co, P.u0, K=2)
    assert rel(u2, res.iterates[-1]) <= 1e-10


def _stage_samples(orc, scheme, fun, dt, J0, M):
    """(M, 2, Q) samples of fun (returning Q values per time) at the stage times
    of fine steps J0 .. J0 + M - 1."""
    cst, _, _ = orc.sdirk_tableau(scheme)
    t = dt * (J0 + np.arange(M))
    return np.stack([fun(t + cst[0] * dt), fun(t + cst[1] * dt)], axis=1)


@pytest.mark.parametrize("scheme", ["sdirk2", "sdirk2l"])
@pytest.mark.parametrize("n", [200, 4095])
def test_sdirk_source_propagate_parity(ctx, orc, scheme, n):
    """SDIRK steps with a source sampled at the stage times, per-row samples,
    on the one-CTA-per-system kernel (n = 200) and the 4-CTA cluster kernel
    (n = 4095), FP64 and FP32."""
    lo, di, up = W.adr1d_op(n)
    dt, M, Q = 1.0 / 16384, 9, 2
    op = api.Operator.tridiag(ctx, lo, di, up)
    op.set_stepper(scheme)
    oop = orc.Tridiag(lo, di, up, stepper=scheme)
    rng = np.random.default_rng(n + 5)
    X = rng.standard_normal((4, n))
    g = rng.standard_normal((Q, n))
    c = np.stack([_stage_samples(orc, scheme, lambda t, k=k: np.stack(
        [np.sin((3 + k) * 7 * t), np.cos((2 + k) * 5 * t)], axis=-1), dt, 11 * k, M) for k in range(4)])
    cond = 1 + 2 * dt * np.max(np.abs(lo) + np.abs(di) + np.abs(up))
    tol = max(1e-12, 8 * M * cond * 2.2e-16)
    got = api.propagate(ctx, op, dt, M, X, g=g, c=c)
    want = orc.propagate(oop, dt, M, X, g=g, cvals=c)
    assert max(rel(got[v], want[v]) for v in range(4)) <= tol
    got32 = api.propagate(ctx, op, dt, M, X[:2], g=g, c=c[:2], prec="mixed")
    assert max(rel(got32[v], want[v]) for v in range(2)) <= 5e-5


@pytest.mark.parametrize("scheme", ["sdirk2", "sdirk2l"])
def test_sdirk_source_parareal_matches_oracle(ctx, orc, scheme):
    """Experiment 1's source on the heat1d operator with an SDIRK fine solver:
    K = N reproduces the oracle's sequential solution, K = 2 the oracle's
    Parareal iterate, and the fine solution equals the oracle's."""
    P = W.heat1d(n=127, N=6, M=16, R=5, p=3)
    op = api.Operator.tridiag(ctx, P.lo, P.di, P.up)
    op.set_stepper(scheme)
    oop = orc.Tridiag(P.lo, P.di, P.up, stepper=scheme)
    # f(t, x) = sin(2 pi t) g(x) (the heat1d source) at the stage times
    c = _stage_samples(orc, scheme, lambda t: np.sin(2 * np.pi * t)[:, None], P.dt, 0, P.N * P.M)
    co = api.Coarse(ctx, op, P.dt, P.M, P.N, P.R, P.p, P.seed, prec="f64")
    oco = orc.build_coarse(oop, P.dt, P.M, P.N, P.R, P.p, P.seed)
    ref = orc.sequential_fine(oop, P.dt, P.M, P.N, P.u0, P.g, c)
    u, _ = api.parareal_solve(ctx, co, P.u0, P.g, c, K=P.N)
    assert orc.rel_err(u, ref) <= 1e-10
    res = orc.parareal(oop, P.dt, P.M, P.N, oco, P.u0, P.g, c, K=2)
    u2, _ = api.parareal_solve(ctx, co, P.u0, P.g, c, K=2)
    assert rel(u2, res.iterates[-1]) <= 1e-10
    uf = api.fine_solution(ctx, op, P.dt, P.M, P.N, P.u0, P.g, c)
    assert orc.rel_err(uf, ref) <= 1e-11
    # the comparator and the server take sources with backward Euler only
    with pytest.raises(_native.LrpError) as ei:
        api.parareal_solve_classical(ctx, op, P.dt, P.M, P.N, P.u0, P.g, P.c, K=1)
    assert ei.value.status == _native.LRP_EINVAL
