"""GPU parity of the FP64 1D fine steps computed from FP32 solves refined by
residuals in pairs of FP32 numbers (tri_refine = 1) against the FP64 oracle
(banded LU per backward-Euler step) and against the FP64 kernels.

Bars: after M steps the refined state carries about M (u_32 kappa)^(R+1)
plus M 2^-48 relative error (R rounds per step; the pair form of B's FP64
entries keeps 48 bits, and its error enters every step alike: measured on
the adr1d operator, n = 4095, 256 steps, 2.7e-12 from the FP64 kernels for
one round and 1.4e-12 for two), so one round is held to 2e-11 and two
rounds to 5e-12; the FP64 kernels to 1e-12 on the same inputs.  Constant-
coefficient operators (adr1d, heat1d) run the register kernel -- on one
CTA per system or a cluster of one-warp CTAs per system, with 16-row chunks
and with 8-row chunks (up to 16 warps) -- the variable-coefficient one the
shared-memory kernel.
"""
import numpy as np
import pytest

from paper_2508_08873_gb300 import _native, api, workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = api.Context(0)
    yield c
    c.set_param("tri_refine", 0)
    c.set_param("tri_refine_rounds", 2)


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _case(name):
    if name == "adr4095":
        P = W.adr1d()
        return P.lo, P.di, P.up, P.dt, 256, P.u0
    if name == "adr1023":
        P = W.adr1d(n=1023, N=16, M=64)
        return P.lo, P.di, P.up, P.dt, 64, P.u0
    if name == "adr1500":
        P = W.adr1d(n=1500, N=8, M=32)
        return P.lo, P.di, P.up, P.dt, 32, P.u0
    if name == "heat255":
        P = W.heat1d()
        return P.lo, P.di, P.up, P.dt, 64, P.u0
    # variable, nonsymmetric coefficients on n = 700 (chunks with padding rows)
    n = 700
    rng = np.random.default_rng(70)
    h = 1.0 / (n + 1)
    lo = -rng.uniform(0.5, 1.5, n) / h ** 2
    up = -rng.uniform(0.5, 1.5, n) / h ** 2
    di = -(lo + up) + rng.uniform(0.0, 2.0, n)
    lo[0] = 0.0
    up[-1] = 0.0
    x = np.arange(1, n + 1) * h
    return lo, di, up, 1.0 / 4096, 40, np.sin(3 * np.pi * x)


@pytest.mark.parametrize("case", ["adr4095", "adr1023", "adr1500", "heat255", "var700"])
@pytest.mark.parametrize("rounds,tol", [(1, 2e-11), (2, 5e-12)])
@pytest.mark.parametrize("variant", ["cta", "cta8", "cluster", "cluster8"])
def test_tri_refine_matches_oracle(ctx, orc, case, rounds, tol, variant):
    lo, di, up, dt, M, u0 = _case(case)
    n = lo.shape[0]
    op = api.Operator.tridiag(ctx, lo, di, up)
    oop = orc.Tridiag(lo, di, up)
    rng = np.random.default_rng(rounds * 10 + n)
    X = np.vstack([u0[None, :], rng.standard_normal((4, n)), 1e-30 * rng.standard_normal((1, n))])
    f64 = api.propagate(ctx, op, dt, M, X)
    ctx.set_param("tri_refine", 1)
    ctx.set_param("tri_refine_rounds", rounds)
    ctx.set_param("tri_refine_cluster", 1 if variant.startswith("cluster") else 0)
    ctx.set_param("tri_wchunk", 8 if variant.endswith("8") else 0)
    try:
        got = api.propagate(ctx, op, dt, M, X)
    finally:
        ctx.set_param("tri_refine", 0)
        ctx.set_param("tri_refine_rounds", 2)
        ctx.set_param("tri_refine_cluster", 0)
        ctx.set_param("tri_wchunk", 0)
    want = orc.propagate(oop, dt, M, X)
    for v in range(X.shape[0]):
        assert rel(got[v], want[v]) <= tol, (v, rel(got[v], want[v]))
        assert rel(f64[v], want[v]) <= 1e-12
    # the refined path ran: its rounding differs from the FP64 kernels'
    assert not np.array_equal(got, f64)


def test_tri_refine_parareal(ctx, orc):
    """Low-rank Parareal on adr1d (n = 1023, N = 16, M = 64) with the fine
    solves refined: K = N equals the oracle's sequential fine solution, and
    the tolerance-driven solve stops within 1e-8 of it."""
    P = W.adr1d(n=1023, N=16, M=64, R=8, p=4)
    op = api.Operator.tridiag(ctx, P.lo, P.di, P.up)
    oop = orc.Tridiag(P.lo, P.di, P.up)
    ref = orc.sequential_fine(oop, P.dt, P.M, P.N, P.u0)
    ctx.set_param("tri_refine", 1)
    try:
        co = api.Coarse(ctx, op, P.dt, P.M, P.N, P.R, P.p, P.seed, prec="mixed")
        uN, _ = api.parareal_solve(ctx, co, P.u0, K=P.N)
        ut, info = api.parareal_solve(ctx, co, P.u0, K=P.N, tol=1e-8)
    finally:
        ctx.set_param("tri_refine", 0)
    assert orc.rel_err(uN, ref) <= 2e-12
    assert info["converged"] and orc.rel_err(ut, ref) <= 1e-8


def test_tri_refine_params(ctx):
    for name, bad in (("tri_refine", 2), ("tri_refine", -1), ("tri_refine_rounds", 0),
                      ("tri_refine_rounds", 4), ("tri_refine_cluster", 2)):
        with pytest.raises(_native.LrpError) as ei:
            ctx.set_param(name, bad)
        assert ei.value.status == _native.LRP_EINVAL
    assert ctx.get_param("tri_refine") == 0 and ctx.get_param("tri_refine_rounds") == 2
    assert ctx.get_param("tri_refine_cluster") == 0
