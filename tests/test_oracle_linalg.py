"""Oracle: modified Gram-Schmidt with re-orthogonalisation and deflation
(rSVD steps 2 and 4, Sec. 2.1) and the one-sided Jacobi SVD (step 5).
Pins: orthonormality and span (definition), known rank, numpy's LAPACK SVD."""
import numpy as np
import pytest


def test_mgs2_full_rank(orc):
    rng = np.random.default_rng(0)
    Y = rng.standard_normal((12, 300)) * np.logspace(0, -6, 12)[:, None]
    Q, keep = orc.mgs2(Y)
    assert Q.shape == (12, 300) and keep.all()
    np.testing.assert_allclose(Q @ Q.T, np.eye(12), atol=1e-14)
    # same span: Y = (Y Q^T) Q
    np.testing.assert_allclose((Y @ Q.T) @ Q, Y, atol=1e-13)
    # triangular structure: row j of Y lies in span(Q[:j+1])
    Rm = Y @ Q.T
    assert np.max(np.abs(np.triu(Rm, 1))) < 1e-13


def test_mgs2_deflates_known_rank(orc):
    rng = np.random.default_rng(1)
    base = rng.standard_normal((5, 200))
    mix = rng.standard_normal((9, 5))
    Y = mix @ base                                    # rank 5, 9 rows
    Y[3] = 0.0                                        # a zero row
    Q, keep = orc.mgs2(Y)
    assert Q.shape[0] == 5 and keep.sum() == 5 and not keep[3]
    np.testing.assert_allclose(Q @ Q.T, np.eye(5), atol=1e-14)
    np.testing.assert_allclose((Y @ Q.T) @ Q, Y, atol=1e-12)


def test_mgs2_empty(orc):
    Q, keep = orc.mgs2(np.zeros((0, 10)))
    assert Q.shape == (0, 10)


@pytest.mark.parametrize("shape", [(12, 12), (20, 7), (7, 20), (1, 1), (42, 42)])
def test_jacobi_svd_matches_lapack(orc, shape):
    rng = np.random.default_rng(sum(shape))
    A = rng.standard_normal(shape) @ np.diag(np.logspace(0, -10, shape[1]))
    U, s, V = orc.jacobi_svd(A)
    r = min(shape)
    assert U.shape == (shape[0], r) and V.shape == (shape[1], r)
    np.testing.assert_allclose(s, np.linalg.svd(A, compute_uv=False), rtol=1e-12, atol=1e-15 * s[0])
    np.testing.assert_allclose(U @ np.diag(s) @ V.T, A, atol=1e-14 * s[0])
    np.testing.assert_allclose(V.T @ V, np.eye(r), atol=1e-13)
    big = s > 1e-12 * s[0]
    np.testing.assert_allclose(U[:, big].T @ U[:, big], np.eye(big.sum()), atol=1e-12)
    assert np.all(np.diff(s) <= 0)


def test_jacobi_svd_degenerate(orc):
    A = np.diag([3.0, 3.0, 1.0, 0.0])
    U, s, V = orc.jacobi_svd(A)
    np.testing.assert_allclose(s, [3, 3, 1, 0], atol=1e-15)
    np.testing.assert_allclose(U @ np.diag(s) @ V.T, A, atol=1e-15)
    U, s, V = orc.jacobi_svd(np.zeros((3, 3)))
    assert np.all(s == 0)


def test_lstsq_mgs_normal_equations_and_consistent_systems(orc):
    """lstsq_mgs (the least-squares step of the two-sided sketch): on a
    consistent system B X0 = Z it returns X0; on an inconsistent one the
    residual is orthogonal to the range of B (the normal equations
    B^T (B X - Z) = 0 that define the least-squares solution); a rank-deficient
    B is refused."""
    rng = np.random.default_rng(5)
    for m, k, n in [(6, 3, 4), (48, 24, 100), (10, 10, 3), (2, 1, 5)]:
        B = rng.standard_normal((m, k))
        X0 = rng.standard_normal((k, n))
        np.testing.assert_allclose(orc.lstsq_mgs(B, B @ X0), X0, rtol=0, atol=1e-11)
        Z = rng.standard_normal((m, n))
        X = orc.lstsq_mgs(B, Z)
        res = B @ X - Z
        assert np.abs(B.T @ res).max() <= 1e-12 * np.abs(B).max() * np.abs(Z).max() * m
        # any other candidate has a residual at least as large
        Xp = X + 1e-3 * rng.standard_normal(X.shape)
        assert np.linalg.norm(B @ Xp - Z) >= np.linalg.norm(res)
    B = rng.standard_normal((8, 3))
    B[:, 2] = B[:, 0] - 2 * B[:, 1]
    with pytest.raises(RuntimeError):
        orc.lstsq_mgs(B, rng.standard_normal((8, 2)))
