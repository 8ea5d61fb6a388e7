"""Oracle: randomized SVD of the transfer operators (Sec. 2.1 steps 1-6).
Pins: the closed-form spectrum and DST-I singular vectors of the 1D heat
propagator; exactness of the rSVD when the sketch spans the whole space
(brute force against numpy's dense SVD); the orientation of the lifted
singular vectors, F' phi_r = sigma_r psi_r (Eq. (svd))."""
import numpy as np
import pytest

from paper_2508_08873_gb300 import workloads as W


def _heat_closed_form(n, dt, M):
    h = 1.0 / (n + 1)
    j = np.arange(1, n + 1)
    lam = 4.0 / h ** 2 * np.sin(j * np.pi * h / 2) ** 2
    x = np.arange(1, n + 1) * h
    return (1.0 + dt * lam) ** (-M), np.sqrt(2 * h) * np.sin(np.pi * np.outer(j, x))


@pytest.mark.parametrize("interval", [0, 9])
def test_rsvd_heat1d_closed_form(orc, interval):
    P = W.heat1d()                                   # n=255, M=64, dt=1/1024, R=8, p=4
    op = orc.Tridiag(P.lo, P.di, P.up)
    c = orc.rsvd_interval(op, P.dt, P.M, interval, P.R, P.p, P.seed)
    sig, modes = _heat_closed_form(P.n, P.dt, P.M)
    assert c.S.shape[0] == P.R
    # |sigma_hat_j - sigma_j| <= 1e-12 sigma_1 for j <= R
    assert np.max(np.abs(c.S - sig[:P.R])) <= 1e-12 * sig[0]
    # singular vectors = DST-I modes up to sign, for the well separated j <= 5
    for j in range(5):
        for vec in (c.U[:, j], c.V[:, j]):
            assert abs(abs(vec @ modes[j]) - 1.0) < 1e-10
    # the sketch of rank ~8 in 12 columns: deflation keeps the basis orthonormal
    assert c.rank_w <= P.R + P.p


@pytest.mark.parametrize("maker", ["heat", "adr"])
def test_rsvd_exact_when_sketch_spans_space(orc, maker):
    n, dt, M = 12, 1e-3, 5
    lo, di, up = W.heat1d_op(n) if maker == "heat" else W.adr1d_op(n, nu=0.05)
    op = orc.Tridiag(lo, di, up)
    Fp = orc.propagate(op, dt, M, np.eye(n)).T
    Uf, sf, Vft = np.linalg.svd(Fp)
    R = 5
    c = orc.rsvd_interval(op, dt, M, 0, R, n - R + 2, seed=3)   # ell = n + 2 >= n
    np.testing.assert_allclose(c.S, sf[:R], rtol=0, atol=1e-12 * sf[0])
    G = c.U @ np.diag(c.S) @ c.V.T
    Gex = Uf[:, :R] @ np.diag(sf[:R]) @ Vft[:R]
    np.testing.assert_allclose(G, Gex, atol=1e-11 * sf[0])
    # Eq. (truncation_error): ||F' - G'|| = sigma_{R+1}
    assert abs(np.linalg.norm(Fp - G, 2) - sf[R]) <= 1e-11 * sf[0]
    assert abs(c.sigma_next - sf[R]) <= 1e-12 * sf[0]


def test_rsvd_vector_orientation_nonsymmetric(orc):
    """F' phi_r = sigma_r psi_r and F'^* psi_r = sigma_r phi_r: the left vectors
    lie in the image of F' (basis w), the right ones in that of F'^*."""
    n, dt, M = 40, 1e-3, 6
    op = orc.Tridiag(*W.adr1d_op(n, nu=0.02))
    c = orc.rsvd_interval(op, dt, M, 2, 4, 40, seed=5)
    FV = orc.propagate(op, dt, M, c.V.T).T
    np.testing.assert_allclose(FV, c.U * c.S, atol=1e-11 * c.S[0])
    FtU = orc.propagate(op, dt, M, c.U.T, adjoint=True).T
    np.testing.assert_allclose(FtU, c.V * c.S, atol=1e-11 * c.S[0])


def test_rsvd_independent_intervals_and_seed(orc):
    P = W.heat1d(n=63, N=3, M=16, R=4, p=2)
    op = orc.Tridiag(P.lo, P.di, P.up)
    a = orc.rsvd_interval(op, P.dt, P.M, 0, P.R, P.p, 0)
    b = orc.rsvd_interval(op, P.dt, P.M, 1, P.R, P.p, 0)
    # different sketches, same operator: same leading singular values
    np.testing.assert_allclose(a.S[:3], b.S[:3], rtol=1e-9)
    assert a.fine_evals == 2 * (P.R + P.p)


# ---------------------------------------------------------------------------
# two-sided variant (F'^* on independent random vectors, Sec. 2.2)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("maker", ["heat", "adr"])
def test_rsvd_indep_exact_when_sketches_span_space(orc, maker):
    """With l >= n the forward sketch spans the space, Q is a complete basis
    and the least-squares core is exact: the two-sided rSVD equals the
    truncated dense SVD (brute force)."""
    n, dt, M = 12, 1e-3, 5
    lo, di, up = W.heat1d_op(n) if maker == "heat" else W.adr1d_op(n, nu=0.05)
    op = orc.Tridiag(lo, di, up)
    Fp = orc.propagate(op, dt, M, np.eye(n)).T
    Uf, sf, Vft = np.linalg.svd(Fp)
    R = 5
    c = orc.rsvd_interval_indep(op, dt, M, 0, R, n - R + 2, seed=3)
    np.testing.assert_allclose(c.S, sf[:R], rtol=0, atol=1e-11 * sf[0])
    G = c.U @ np.diag(c.S) @ c.V.T
    Gex = Uf[:, :R] @ np.diag(sf[:R]) @ Vft[:R]
    np.testing.assert_allclose(G, Gex, atol=1e-10 * sf[0])
    assert c.fine_evals == 3 * (n + 2)


def test_rsvd_indep_heat_spectrum_and_orientation(orc):
    """Heat configuration: the leading singular values follow the closed-form
    DST spectrum (to 1e-7 sigma_1: the two-sided core is a least-squares
    estimate), and F' phi_r ~ sigma_r psi_r."""
    P = W.heat1d()
    op = orc.Tridiag(P.lo, P.di, P.up)
    c = orc.rsvd_interval_indep(op, P.dt, P.M, 3, P.R, P.p, P.seed)
    sig, _ = _heat_closed_form(P.n, P.dt, P.M)
    assert np.max(np.abs(c.S[:6] - sig[:6])) <= 1e-7 * sig[0]
    FV = orc.propagate(op, P.dt, P.M, c.V[:, :4].T).T
    np.testing.assert_allclose(FV, c.U[:, :4] * c.S[:4], atol=1e-7 * c.S[0])


@pytest.mark.parametrize("maker", ["heat", "adr"])
def test_rsvd_indep_partial_sketch_equals_pseudoinverse_formula(orc, maker):
    """A partial sketch (l = R + p < n): the two-sided estimate of Sec. 2.2 is
    Q^T X with Q = orth(Y), X = (Psi^T Q^T)^+ Psi^T F' (the least-squares
    core), truncated to rank R.  Built here from the dense F', the same
    Gaussian vectors and numpy's pseudo-inverse and SVD: the oracle's Gram-
    Schmidt least squares and Jacobi SVD must give the same rank-R operator
    and singular values.  A transposed operand, the wrong sketch in the
    core or a dropped factor changes the result by O(sigma_1)."""
    n, dt, M, R, p, seed, i = 40, 2e-3, 6, 4, 3, 11, 2
    lo, di, up = W.heat1d_op(n) if maker == "heat" else W.adr1d_op(n, nu=0.05)
    op = orc.Tridiag(lo, di, up)
    Fp = orc.propagate(op, dt, M, np.eye(n)).T                 # F' column by column
    ell = R + p
    omega = orc.gauss_block(seed, i, n, ell)                   # rows omega_j
    psi = orc.gauss_block(seed, i, n, 2 * ell, stream=orc.STREAM_PSI)
    Qm, _ = np.linalg.qr((omega @ Fp.T).T)                     # n x l basis of range(F' Omega)
    X = np.linalg.pinv(psi @ Qm) @ (psi @ Fp)                  # l x n least-squares core
    Us, s, Vt = np.linalg.svd(Qm @ X)
    Gex = Us[:, :R] @ np.diag(s[:R]) @ Vt[:R]
    c = orc.rsvd_interval_indep(op, dt, M, i, R, p, seed)
    np.testing.assert_allclose(c.S, s[:R], rtol=0, atol=1e-9 * s[0])
    G = c.U @ np.diag(c.S) @ c.V.T
    np.testing.assert_allclose(G, Gex, rtol=0, atol=1e-9 * s[0])
    # not the exact truncated SVD: the partial sketch is an estimate
    sf = np.linalg.svd(Fp, compute_uv=False)
    assert np.abs(c.S - sf[:R]).max() > 1e-8 * sf[0]
