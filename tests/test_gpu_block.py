"""GPU parity of the block conjugate-gradient propagator (krylov_block = 4:
four systems that share the step matrix solved in one block Krylov space,
B^-orthonormal directions with a pivoted-Cholesky selection) against the
FP64 oracle (banded LU per backward-Euler step).

FP64 at rtol 1e-14 is compared at 1e-10 relative L2, as for the
single-system kernels: it runs the same kernel code and catches any error of
its logic (a wrong block coefficient, a missing halo row, a pivot dropped
wrongly).  FP32 (rtol 1e-6 per step and system, the sketch setting) is
compared at 2e-3 on grids above 128 rows and 5e-4 below: the error of a
step solved to a relative residual rtol is bounded by kappa(B) rtol, with
kappa(B) = 3e3 .. 5e4 for these operators at dt = 1/4096, and the block
iteration stops on the recursively updated residuals, which drift from the
true ones by a few FP32 roundings per iteration; an emulation of the same
arithmetic in numpy shows about twice the error of single-system CG.  The
cases cover blocks with fewer than four systems, several blocks per cluster,
zero and exactly dependent right-hand sides (the pivoting leaves them out),
the adjoint, the generated sketch input of a build, and the 511^2
checkerboard diffusion operator at its own size.
"""
import numpy as np
import pytest

from paper_2508_08873_gb300 import _native, api, workloads as W
from test_gpu_onchip import sym_stencil

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = api.Context(0)
    c.set_param("krylov_block", 4)
    c.set_param("krylov_refine", 2)      # single-system comparisons on the Krylov kernels themselves
    yield c
    c.set_param("krylov_refine", 0)
    c.set_param("krylov_block", 0)
    c.set_param("krylov_block_clusters", 0)


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _pair(ctx, orc, mx, my, seed=0, rtol64=1e-14, rtol32=1e-6):
    st = sym_stencil(mx, my, seed)
    op = api.Operator.stencil5(ctx, mx, my, st)
    op.set_krylov(rtol64, rtol32, 20000)
    oop = orc.Stencil5(mx, my, st["C"], st["W"], st["E"], st["S"], st["N"])
    return op, oop


def _used(ctx):
    return ctx.get_param("krylov_block_last_systems")


GRIDS = [(15, 15), (33, 47), (64, 64), (100, 130), (127, 127), (255, 200)]


@pytest.mark.parametrize("mx,my", [g for g in GRIDS if g[0] <= 256])
@pytest.mark.parametrize("adjoint", [False, True])
def test_block_f64_matches_oracle(ctx, orc, mx, my, adjoint):
    op, oop = _pair(ctx, orc, mx, my, seed=5 * mx + my)
    dt, M = 1.0 / 2048, 3
    X = np.random.default_rng(mx + 3 * my).standard_normal((7, mx * my))   # blocks of 4 and 3
    got = api.propagate(ctx, op, dt, M, X, adjoint=adjoint)
    assert _used(ctx) == 4
    want = orc.propagate(oop, dt, M, X, adjoint=adjoint)
    for v in range(X.shape[0]):
        assert rel(got[v], want[v]) <= 1e-10, (v, rel(got[v], want[v]))


@pytest.mark.parametrize("mx,my", GRIDS)
def test_block_f32_matches_oracle(ctx, orc, mx, my):
    op, oop = _pair(ctx, orc, mx, my, seed=mx + my)
    dt, M = 1.0 / 4096, 6
    X = np.random.default_rng(mx * my).standard_normal((6, mx * my))
    got = api.propagate(ctx, op, dt, M, X, prec="mixed")
    assert _used(ctx) == 4
    want = orc.propagate(oop, dt, M, X)
    tol = 2e-3 if my > 128 else 5e-4
    for v in range(X.shape[0]):
        assert rel(got[v], want[v]) <= tol, (v, rel(got[v], want[v]))


def test_block_fewer_iterations_than_single_systems(ctx, orc):
    """The same 8 systems: the block solver's iterations (counted per system)
    are below those of the single-system kernels, and both meet the oracle."""
    mx = my = 127
    op, oop = _pair(ctx, orc, mx, my, seed=77)
    dt, M = 1.0 / 4096, 4
    X = np.random.default_rng(78).standard_normal((8, mx * my))
    want = orc.propagate(oop, dt, M, X)
    before = op.krylov_iterations()
    got_b = api.propagate(ctx, op, dt, M, X)
    it_block = op.krylov_iterations() - before
    ctx.set_param("krylov_block", 0)
    try:
        before = op.krylov_iterations()
        got_s = api.propagate(ctx, op, dt, M, X)
        it_single = op.krylov_iterations() - before
    finally:
        ctx.set_param("krylov_block", 4)
    for v in range(8):
        assert rel(got_b[v], want[v]) <= 1e-10
        assert rel(got_s[v], want[v]) <= 1e-10
    assert 0 < it_block < 0.95 * it_single, (it_block, it_single)


def test_block_many_blocks_per_cluster(ctx, orc):
    """41 systems (ten full blocks and one of one system) on two clusters:
    every cluster runs several blocks in turn."""
    mx, my = 48, 70
    op, oop = _pair(ctx, orc, mx, my, seed=81)
    ctx.set_param("krylov_block_clusters", 2)
    try:
        X = np.random.default_rng(82).standard_normal((41, mx * my))
        got = api.propagate(ctx, op, 1.0 / 1024, 2, X)
        assert ctx.get_param("krylov_block_last_clusters") == 2
    finally:
        ctx.set_param("krylov_block_clusters", 0)
    want = orc.propagate(oop, 1.0 / 1024, 2, X)
    assert max(rel(got[v], want[v]) for v in range(41)) <= 1e-10


def test_block_zero_and_dependent_columns(ctx, orc):
    """A zero right-hand side and two equal ones in a block: the pivoted
    Cholesky leaves the dependent directions out; every result still
    matches the oracle (the zero one stays exactly 0)."""
    mx, my = 64, 64
    op, oop = _pair(ctx, orc, mx, my, seed=91)
    rng = np.random.default_rng(92)
    X = rng.standard_normal((8, mx * my))
    X[1] = 0.0
    X[2] = X[0]
    X[6] = 3.0 * X[5]
    for prec, tol in (("f64", 1e-10), ("mixed", 5e-4)):
        got = api.propagate(ctx, op, 1.0 / 4096, 5, X, prec=prec)
        want = orc.propagate(oop, 1.0 / 4096, 5, X)
        assert np.all(got[1] == 0.0)
        for v in (0, 2, 3, 4, 5, 6, 7):
            assert rel(got[v], want[v]) <= tol, (prec, v, rel(got[v], want[v]))


def test_block_cap_and_single_system(ctx, orc):
    mx, my = 40, 33
    op, oop = _pair(ctx, orc, mx, my, seed=31)
    X = np.random.default_rng(32).standard_normal((4, mx * my))
    # one system, or zero steps: the single-system kernels
    api.propagate(ctx, op, 1e-3, 1, X[:1])
    assert _used(ctx) == 0
    np.testing.assert_array_equal(api.propagate(ctx, op, 1e-3, 0, X), X)
    op.set_krylov(1e-14, 1e-6, 2)
    with pytest.raises(_native.LrpError) as ei:
        api.propagate(ctx, op, 1.0 / 64, 3, X)
    assert ei.value.status == _native.LRP_ENOTCONV
    assert _used(ctx) == 4


def test_block_mixed_build_matches_oracle(ctx, orc):
    """Mixed-mode coarse build of the checkerboard diffusion operator with the
    FP32 sketches (Omega generated in the kernel) on the block kernel: the
    singular values and G' as an operator agree with the oracle's FP64 build
    to the FP32 level."""
    P = W.diff2d(m=63, N=3, M=8, R=6, p=4)
    op = api.Operator.stencil5(ctx, P.mx, P.my, P.st)
    op.set_krylov(1e-14, 1e-6, 20000)
    oop = orc.Stencil5(P.mx, P.my, P.st["C"], P.st["W"], P.st["E"], P.st["S"], P.st["N"])
    co = api.Coarse(ctx, op, P.dt, P.M, P.N, P.R, P.p, P.seed, prec="mixed")
    info = co.info()
    oco = orc.build_coarse(oop, P.dt, P.M, P.N, P.R, P.p, P.seed)
    probes = np.random.default_rng(41).standard_normal((3, P.n))
    for i in range(P.N):
        oc = oco.intervals[i]
        s1 = oc.sigma[0]
        R = oc.S.shape[0]
        assert np.max(np.abs(info["sigma"][i, :R] - oc.S)) <= 1e-4 * s1
        U, S, V = co.factors(i)
        Go = oc.U @ np.diag(oc.S) @ oc.V.T
        Gg = U.T @ np.diag(S) @ V
        assert max(np.linalg.norm((Gg - Go) @ x) / np.linalg.norm(x) for x in probes) <= 1e-4 * s1


def test_block_full_size_511(ctx, orc):
    """The 511^2 checkerboard diffusion operator at its own size (dt = 1/4096,
    16-CTA clusters of 32 rows): FP32 at the sketch tolerance 1e-6 on five
    systems (a block of four and one of one), two steps, against the
    oracle's banded LU."""
    P = W.diff2d()
    op = api.Operator.stencil5(ctx, P.mx, P.my, P.st)
    op.set_krylov(1e-12, 1e-6, 20000)
    oop = orc.Stencil5(P.mx, P.my, P.st["C"], P.st["W"], P.st["E"], P.st["S"], P.st["N"])
    X = np.random.default_rng(51).standard_normal((5, P.n))
    X[1] = P.u0
    want = orc.propagate(oop, P.dt, 2, X)
    got = api.propagate(ctx, op, P.dt, 2, X, prec="mixed")
    assert _used(ctx) == 4 and ctx.get_param("krylov_block_last_cs") == 16
    for v in range(5):
        assert rel(got[v], want[v]) <= 2e-3, (v, rel(got[v], want[v]))
