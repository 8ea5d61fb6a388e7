"""GPU parity of the on-chip conjugate-gradient propagator (symmetric 5-point
operators, every Krylov vector in registers and shared memory of one
thread-block cluster per system) against the FP64 oracle (banded LU per
backward-Euler step).

Grids cover one-CTA and 16-CTA clusters, columns that fill whole warps and
columns that leave a partial last warp, CTAs with fewer rows than the others,
non-square grids, the row counts per CTA (8 and 16 in FP64, 16 and 32 in
FP32) and both precisions; the same cases through the kernel with the Krylov vectors in
global memory (krylov_onchip = 2) check that the two agree with the oracle
alike.  FP64 steps by iterative refinement (the library's default for these
grids) are switched off here (krylov_refine = 2) and tested in
test_gpu_refine.py.  FP64 at rtol 1e-14 is compared at 1e-10 relative L2: the FP64
cases run the same kernel code and catch any error of its logic.  FP32 (rtol
1e-6 per step, the sketch setting) is compared at 1e-3 on grids above 128
rows and 2e-4 below: the error of a step solved to a relative residual rtol
is bounded by kappa(B) rtol, with kappa(B) = 3e3 .. 5e4 for these operators
at dt = 1/4096 (Gershgorin), and both kernels show 1e-5 .. 4e-4 (the same
for the kernel with its vectors in global memory); a precision-specific
mistake (a coefficient rounded wrongly, a reduction in the wrong type)
shows at 1e-2 or above.
"""
import numpy as np
import pytest

from paper_2508_08873_gb300 import _native, api, workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = api.Context(0)
    c.set_param("krylov_refine", 2)      # FP64 steps on the FP64 Krylov kernels themselves
    yield c
    c.set_param("krylov_refine", 0)
    c.set_param("krylov_onchip", 0)
    c.set_param("krylov_cluster", 0)


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def sym_stencil(mx, my, seed, scale=None):
    """A symmetric 5-point operator -div(k grad u) + u on an mx x my grid
    with seeded positive face conductances (log-uniform over two decades):
    W_p = E_{p-1}, S_p = N_{p-mx}; couplings across the boundary are absent
    (Dirichlet), their faces still add to the diagonal."""
    rng = np.random.default_rng(seed)
    h2 = float(max(mx, my) + 1) ** 2 if scale is None else scale
    kx = 10 ** rng.uniform(0, 2, (my, mx + 1)) * h2      # face left of node ix: kx[:, ix]
    ky = 10 ** rng.uniform(0, 2, (my + 1, mx)) * h2      # face below node iy: ky[iy, :]
    C = kx[:, :-1] + kx[:, 1:] + ky[:-1, :] + ky[1:, :] + 1.0
    E = -kx[:, 1:].copy()
    E[:, -1] = 0.0
    Wc = -kx[:, :-1].copy()
    Wc[:, 0] = 0.0
    N = -ky[1:, :].copy()
    N[-1, :] = 0.0
    S = -ky[:-1, :].copy()
    S[0, :] = 0.0
    return {k: v.reshape(-1).copy() for k, v in (("C", C), ("W", Wc), ("E", E), ("S", S), ("N", N))}


def _pair(ctx, orc, mx, my, seed=0, rtol64=1e-14, rtol32=1e-6):
    st = sym_stencil(mx, my, seed)
    op = api.Operator.stencil5(ctx, mx, my, st)
    op.set_krylov(rtol64, rtol32, 20000)
    oop = orc.Stencil5(mx, my, st["C"], st["W"], st["E"], st["S"], st["N"])
    return op, oop


# (mx, my, CTAs per cluster or 0 for the automatic choice)
GRIDS = [
    (15, 15, 0),      # one CTA, a partial warp
    (33, 47, 0),      # two warps, the second almost empty
    (64, 64, 2),      # whole warps; 32 rows per CTA (FP32 32-row variant)
    (64, 64, 4),      # 16 rows per CTA (FP32 and FP64 16-row variants)
    (64, 64, 8),      # 8 rows per CTA (FP64 8-row variant)
    (100, 130, 0),    # last CTA padded with inert rows
    (127, 127, 0),
    (255, 200, 0),
]


@pytest.mark.parametrize("onchip", [0, 2])
@pytest.mark.parametrize("mx,my,cs", GRIDS)
def test_onchip_f32_matches_oracle(ctx, orc, mx, my, cs, onchip):
    ctx.set_param("krylov_onchip", onchip)
    ctx.set_param("krylov_cluster", cs if onchip == 0 else 0)
    try:
        op, oop = _pair(ctx, orc, mx, my, seed=mx + my)
        dt, M = 1.0 / 4096, 6
        X = np.random.default_rng(mx * my).standard_normal((5, mx * my))
        got = api.propagate(ctx, op, dt, M, X, prec="mixed")
        want = orc.propagate(oop, dt, M, X)
        tol = 1e-3 if my > 128 else 2e-4
        for v in range(X.shape[0]):
            assert rel(got[v], want[v]) <= tol, (v, rel(got[v], want[v]))
        assert op.krylov_iterations() > 0
    finally:
        ctx.set_param("krylov_onchip", 0)
        ctx.set_param("krylov_cluster", 0)


@pytest.mark.parametrize("mx,my,cs", [g for g in GRIDS if g[1] <= 256] + [(40, 255, 0)])
@pytest.mark.parametrize("adjoint", [False, True])
def test_onchip_f64_matches_oracle(ctx, orc, mx, my, cs, adjoint):
    ctx.set_param("krylov_cluster", cs)
    try:
        op, oop = _pair(ctx, orc, mx, my, seed=3 * mx + my)
        dt, M = 1.0 / 2048, 3
        X = np.random.default_rng(mx + 7 * my).standard_normal((3, mx * my))
        got = api.propagate(ctx, op, dt, M, X, adjoint=adjoint)
        want = orc.propagate(oop, dt, M, X, adjoint=adjoint)
        for v in range(X.shape[0]):
            assert rel(got[v], want[v]) <= 1e-10, (v, rel(got[v], want[v]))
    finally:
        ctx.set_param("krylov_cluster", 0)


@pytest.mark.parametrize("prec,tol", [("f64", 1e-10), ("mixed", 2e-4)])
def test_onchip_source_batch(ctx, orc, prec, tol):
    """Separable source f = sum_q c_q(t) g_q(x), per-system c, 9 systems."""
    mx, my, dt, M = 70, 45, 1.0 / 1024, 5
    op, oop = _pair(ctx, orc, mx, my, seed=11)
    rng = np.random.default_rng(12)
    g = rng.standard_normal((3, mx * my))
    c = rng.standard_normal((9, M, 3))
    X = rng.standard_normal((9, mx * my))
    got = api.propagate(ctx, op, dt, M, X, g=g, c=c, prec=prec)
    want = orc.propagate(oop, dt, M, X, g=g, cvals=c)
    for v in range(9):
        assert rel(got[v], want[v]) <= tol, (v, rel(got[v], want[v]))


def test_onchip_many_systems_per_cluster(ctx, orc):
    """More systems than clusters in flight: each cluster runs several systems
    in turn (the edge rows and reduction buffers are reused)."""
    mx, my, dt, M = 48, 30, 1.0 / 512, 2
    op, oop = _pair(ctx, orc, mx, my, seed=21)
    X = np.random.default_rng(22).standard_normal((600, mx * my))
    got = api.propagate(ctx, op, dt, M, X)
    want = orc.propagate(oop, dt, M, X)
    errs = [rel(got[v], want[v]) for v in range(X.shape[0])]
    assert max(errs) <= 1e-10


def test_onchip_iteration_cap_and_zero_steps(ctx, orc):
    mx, my = 40, 33
    op, oop = _pair(ctx, orc, mx, my, seed=31)
    X = np.random.default_rng(32).standard_normal((2, mx * my))
    np.testing.assert_array_equal(api.propagate(ctx, op, 1e-3, 0, X), X)
    op.set_krylov(1e-14, 1e-6, 2)
    with pytest.raises(_native.LrpError) as ei:
        api.propagate(ctx, op, 1.0 / 64, 3, X)
    assert ei.value.status == _native.LRP_ENOTCONV
    with pytest.raises(_native.LrpError) as ei:
        api.propagate(ctx, op, 1.0 / 64, 3, X, prec="mixed")
    assert ei.value.status == _native.LRP_ENOTCONV


def test_onchip_mixed_build_matches_oracle(ctx, orc):
    """Mixed-mode coarse build of the checkerboard diffusion operator: the FP32
    sketches (Omega generated in the kernel) run on the on-chip kernel; the
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


def test_onchip_full_size_511(ctx, orc):
    """The 511^2 checkerboard diffusion operator at its own size (dt = 1/4096):
    FP32 on the on-chip kernel (16-CTA clusters of 32 rows, q in shared
    memory) at the sketch tolerance 1e-6, and FP64 at 1e-12 (the fine-solve
    setting) and at 1e-14, two steps of two vectors each, against the
    oracle's banded LU."""
    P = W.diff2d()
    op = api.Operator.stencil5(ctx, P.mx, P.my, P.st)
    oop = orc.Stencil5(P.mx, P.my, P.st["C"], P.st["W"], P.st["E"], P.st["S"], P.st["N"])
    X = np.random.default_rng(51).standard_normal((2, P.n))
    X[1] = P.u0
    want = orc.propagate(oop, P.dt, 2, X)
    op.set_krylov(1e-12, 1e-6, 20000)
    got32 = api.propagate(ctx, op, P.dt, 2, X, prec="mixed")
    got12 = api.propagate(ctx, op, P.dt, 2, X)
    op.set_krylov(1e-14, 1e-6, 20000)
    got14 = api.propagate(ctx, op, P.dt, 2, X)
    for v in range(2):
        assert rel(got32[v], want[v]) <= 1e-3, rel(got32[v], want[v])
        assert rel(got12[v], want[v]) <= 1e-9, rel(got12[v], want[v])
        assert rel(got14[v], want[v]) <= 1e-10, rel(got14[v], want[v])
