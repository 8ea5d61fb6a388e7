"""FP64 CPU oracle for "A Parareal Algorithm with Low-Rank Coarse Solvers"
(Gander, Ohlberger, Rave; arXiv 2508.08873).

TEST INFRASTRUCTURE ONLY.  Only tests, the smoke check and the CPU-baseline leg
of the benchmark may import this module.  It shares no code with the CUDA
library: the numerics live in oracle/orc.c (loaded through ctypes) and the
method's steps are written out here in the paper's order and notation.

Conventions (0-based in code, 1-based in the paper):
  * interval i = 0..N-1 is the paper's interval n = i+1, [t_i, t_{i+1}];
  * vectors are rows of C-contiguous arrays: a batch of vectors is (nvec, n);
  * the fine solver F_i is M backward-Euler steps of u_t = -A u + f with the
    separable source f(t, x) = sum_q c_q(t) g_q(x) sampled at the end of each
    step; the coefficient array c has shape (N*M, Q), row J-1 holding the
    values at the fine time t = J*dt, J = 1..N*M.

Parity of each function is pinned by tests/test_oracle_*.py against closed
forms, library routines and the paper's theorems.  Functions whose results are
only checked through invariants say so in their docstring.
"""
from __future__ import annotations

import ctypes
import math
import os
import dataclasses
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

from . import build as _build

_lib = None


def lib():
    """Load (building on first use) the oracle's C primitives."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        d, i, u32, u64, L_ = (ctypes.c_double, ctypes.c_int, ctypes.c_uint32,
                              ctypes.c_uint64, ctypes.c_long)
        P = ctypes.c_void_p
        L.orc_gauss.restype = d
        L.orc_gauss.argtypes = [u64, u32, u32, u32, u32]
        L.orc_gauss_block.argtypes = [u64, u32, u32, i, i, P]
        L.orc_philox4x32_10.argtypes = [P, P, P]
        L.orc_philox_rows.argtypes = [u64, u32, u32, u32, i, P]
        L.orc_thomas.restype = i
        L.orc_thomas.argtypes = [i, P, P, P, P, P, P]
        L.orc_tridiag_propagate_many.restype = i
        L.orc_tridiag_propagate_many.argtypes = [i, P, P, P, d, i, i, i, P, P, L_, i, P]
        L.orc_tridiag_td_propagate_many.restype = i
        L.orc_tridiag_td_propagate_many.argtypes = [i, i, P, P, P, P, d, i, i, i, P, P, L_, i, P]
        L.orc_stencil_propagate_many.restype = i
        L.orc_stencil_propagate_many.argtypes = [i, i, P, P, P, P, P, d, i, i, i, P, P, L_, i, P]
        L.orc_stencil_dense.restype = i
        L.orc_stencil_dense.argtypes = [i, i, P, P, P, P, P, d, P]
        L.orc_band_lu.restype = i
        L.orc_band_lu.argtypes = [i, i, P]
        L.orc_mgs2.restype = i
        L.orc_mgs2.argtypes = [i, i, P, d, P, P]
        L.orc_jacobi_svd.restype = i
        L.orc_jacobi_svd.argtypes = [i, i, P, P, P, P]
        L.orc_num_threads.restype = i
        L.orc_set_num_threads.restype = None
        L.orc_set_num_threads.argtypes = [i]
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads() -> int:
    return lib().orc_num_threads()


def set_num_threads(n: int) -> None:
    """Threads of the C primitives' loops over independent vectors (n <= 0:
    all host cores).  Results do not depend on it."""
    lib().orc_set_num_threads(int(n))


# ----------------------------------------------------------------------------
# Operators (the semi-discretisation A of u_t = -A u + f is an input)
# ----------------------------------------------------------------------------
@dataclass
class Tridiag:
    """Tridiagonal A: row i is lo[i] x[i-1] + di[i] x[i] + up[i] x[i+1].
    stepper: the fine time stepper of `propagate` ("be" backward Euler,
    "sdirk2", "sdirk2l": the SDIRK methods of Sec. 4)."""
    lo: np.ndarray
    di: np.ndarray
    up: np.ndarray
    stepper: str = "be"

    def matvec(self, X: np.ndarray, adjoint: bool = False) -> np.ndarray:
        """A x (or A^T x) for every row x of X (nvec, n)."""
        lo, di, up = _f64(self.lo), _f64(self.di), _f64(self.up)
        Y = X * di
        if not adjoint:
            Y[:, 1:] += lo[1:] * X[:, :-1]
            Y[:, :-1] += up[:-1] * X[:, 1:]
        else:
            Y[:, 1:] += up[:-1] * X[:, :-1]
            Y[:, :-1] += lo[1:] * X[:, 1:]
        return Y

    @property
    def n(self) -> int:
        return self.di.shape[0]

    def dense(self) -> np.ndarray:
        n = self.n
        A = np.diag(self.di.astype(np.float64))
        A[np.arange(1, n), np.arange(0, n - 1)] = self.lo[1:]
        A[np.arange(0, n - 1), np.arange(1, n)] = self.up[:-1]
        return A


@dataclass
class TridiagTD:
    """Time-dependent tridiagonal A (Experiment 2 of Sec. 4): fine step J
    (0-based over the whole time grid) uses A_J = A(t_{J+1}) with row i
    lo_t[J, i] x[i-1] + di_t[J, i] x[i] + up_t[J, i] x[i+1].  The fine solver
    of interval i runs steps i*M .. i*M + M - 1.

    stepper "sdirk2" / "sdirk2l": the rows are the operator at the two stage
    times of every step, row 2J + s = A(t_J + c_s dt) (c from sdirk_tableau,
    t_J = J dt the start of step J)."""
    lo_t: np.ndarray
    di_t: np.ndarray
    up_t: np.ndarray
    stepper: str = "be"

    @property
    def n(self) -> int:
        return self.di_t.shape[1]

    @property
    def steps(self) -> int:
        return self.di_t.shape[0] // (1 if self.stepper == "be" else 2)

    def step(self, J: int) -> Tridiag:
        """The time-invariant operator A_J (backward Euler)."""
        return Tridiag(self.lo_t[J], self.di_t[J], self.up_t[J])

    def stage(self, J: int, s: int) -> Tridiag:
        """A at stage time s of step J (SDIRK steppers)."""
        r = 2 * J + s
        return Tridiag(self.lo_t[r], self.di_t[r], self.up_t[r])


@dataclass
class Stencil5:
    """5-point A on an mx x my grid, node p = iy*mx + ix:
    (A x)_p = C x_p + W x_{p-1} + E x_{p+1} + S x_{p-mx} + N x_{p+mx}, the
    neighbours outside the grid absent (homogeneous Dirichlet).
    stepper: the fine time stepper, as for Tridiag."""
    mx: int
    my: int
    C: np.ndarray
    W: np.ndarray
    E: np.ndarray
    S: np.ndarray
    N: np.ndarray
    stepper: str = "be"

    @property
    def n(self) -> int:
        return self.mx * self.my

    def matvec(self, X: np.ndarray, adjoint: bool = False) -> np.ndarray:
        """A x (or A^T x) for every row x of X (nvec, n), written out from the
        definition above on the (my, mx) grid."""
        mx, my = self.mx, self.my
        G = np.asarray(X, dtype=np.float64).reshape(-1, my, mx)
        C, W, E, S, N = (_f64(a).reshape(my, mx) for a in (self.C, self.W, self.E, self.S, self.N))
        Y = C * G
        if not adjoint:
            Y[:, :, 1:] += W[:, 1:] * G[:, :, :-1]      # west neighbour, ix > 0
            Y[:, :, :-1] += E[:, :-1] * G[:, :, 1:]     # east neighbour, ix < mx - 1
            Y[:, 1:, :] += S[1:, :] * G[:, :-1, :]      # south neighbour, iy > 0
            Y[:, :-1, :] += N[:-1, :] * G[:, 1:, :]     # north neighbour, iy < my - 1
        else:
            # (A^T x)_p = sum_q A_qp x_q: node q = p + 1 reaches p through its W, ...
            Y[:, :, :-1] += W[:, 1:] * G[:, :, 1:]
            Y[:, :, 1:] += E[:, :-1] * G[:, :, :-1]
            Y[:, :-1, :] += S[1:, :] * G[:, 1:, :]
            Y[:, 1:, :] += N[:-1, :] * G[:, :-1, :]
        return Y.reshape(np.asarray(X).shape)

    def dense_B(self, dt: float) -> np.ndarray:
        """Dense I + dt*A (tiny grids only)."""
        n = self.n
        out = np.zeros((n, n))
        rc = lib().orc_stencil_dense(self.mx, self.my, _p(_f64(self.C)), _p(_f64(self.W)),
                                     _p(_f64(self.E)), _p(_f64(self.S)), _p(_f64(self.N)),
                                     float(dt), _p(out))
        assert rc == 0
        return out


@dataclass
class Stencil5TD:
    """Time-dependent 5-point A (Experiment 3 of Sec. 4: a conductivity that
    varies in time): fine step J (0-based over the whole time grid) uses A_J
    with the coefficients C_t[J], W_t[J], E_t[J], S_t[J], N_t[J] (each
    mx*my values, as in Stencil5).  The fine solver of interval i runs steps
    i*M .. i*M + M - 1."""
    mx: int
    my: int
    C_t: np.ndarray
    W_t: np.ndarray
    E_t: np.ndarray
    S_t: np.ndarray
    N_t: np.ndarray
    stepper: str = "be"     # SDIRK: rows 2J + s = A(t_J + c_s dt), as for TridiagTD

    @property
    def n(self) -> int:
        return self.mx * self.my

    @property
    def steps(self) -> int:
        return self.C_t.shape[0] // (1 if self.stepper == "be" else 2)

    def step(self, J: int) -> Stencil5:
        """The time-invariant operator A_J (backward Euler)."""
        return Stencil5(self.mx, self.my, self.C_t[J], self.W_t[J], self.E_t[J], self.S_t[J],
                        self.N_t[J])

    def stage(self, J: int, s: int) -> Stencil5:
        """A at stage time s of step J (SDIRK steppers)."""
        r = 2 * J + s
        return Stencil5(self.mx, self.my, self.C_t[r], self.W_t[r], self.E_t[r], self.S_t[r],
                        self.N_t[r])


TIME_DEPENDENT = (TridiagTD, Stencil5TD)


def _propagate_stencil_td(op: Stencil5TD, dt, M, X, adjoint, g, cvals, intervals):
    """Backward-Euler steps with every step's own matrix, one banded solve per
    step; the adjoint runs the transposed steps in reversed order."""
    nvec = X.shape[0]
    j0s = np.broadcast_to(np.asarray(intervals) * M, (nvec,))
    if g is not None:
        cv = _f64(cvals)
        if cv.ndim == 2:
            cv = np.broadcast_to(cv, (nvec,) + cv.shape)
    for v in range(nvec):
        J0 = int(j0s[v])
        if J0 < 0 or J0 + M > op.steps:
            raise ValueError("time-dependent operator: steps beyond its time grid")
        order = range(M - 1, -1, -1) if adjoint else range(M)
        for j in order:
            A_J = op.step(J0 + j)
            if g is None:
                X[v] = propagate(A_J, dt, 1, X[v:v + 1], adjoint)[0]
            else:
                X[v] = propagate(A_J, dt, 1, X[v:v + 1], g=g, cvals=cv[v, j:j + 1])[0]
    return X


# ----------------------------------------------------------------------------
# Random sketch vectors (rSVD step 1; generator: Philox4x32-10 + Box-Muller)
# ----------------------------------------------------------------------------
STREAM_OMEGA = 0


def gauss_block(seed: int, interval: int, n: int, ncol: int, stream: int = STREAM_OMEGA):
    """(ncol, n) block of N(0,1) deviates omega_{interval, col}[row]."""
    out = np.empty((ncol, n))
    lib().orc_gauss_block(seed, stream, interval, n, ncol, _p(out))
    return out


def philox(ctr, key) -> np.ndarray:
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def philox_rows(seed: int, stream: int, interval: int, column: int, n: int) -> np.ndarray:
    out = np.zeros((n, 4), dtype=np.uint32)
    lib().orc_philox_rows(seed, stream, interval, column, n, _p(out))
    return out


# ----------------------------------------------------------------------------
# Fine propagators F_i, F_i' and F_i'^* (Sec. 4 backward Euler; Eq. (F_n_affine))
# ----------------------------------------------------------------------------
def propagate(op, dt: float, M: int, X: np.ndarray, adjoint: bool = False,
              g: Optional[np.ndarray] = None, cvals: Optional[np.ndarray] = None,
              intervals=0) -> np.ndarray:
    """Apply M backward-Euler steps to every row of X (nvec, n).

    g: (Q, n) spatial source profiles or None (linear part F').
    cvals: (M, Q) shared by all rows, or (nvec, M, Q) per row: c_q at the end
    of each step; for the SDIRK steppers (M, 2, Q) or (nvec, M, 2, Q): c_q at
    the two stage times of each step.  adjoint=True applies F'^* (no source
    allowed).
    intervals: for a time-dependent operator (TridiagTD, Stencil5TD), the interval of
    every row (a scalar or nvec values): row v runs steps intervals[v]*M ..
    intervals[v]*M + M - 1, and its adjoint the transposed solves of those
    steps in reversed order."""
    X = np.array(X, dtype=np.float64, order="C", copy=True)
    if X.ndim == 1:
        return propagate(op, dt, M, X[None, :], adjoint, g, cvals, intervals)[0]
    nvec, n = X.shape
    if nvec == 0:
        return X
    if isinstance(op, (Tridiag, Stencil5)) and op.stepper != "be":
        return propagate_sdirk(op, dt, M, X, op.stepper, adjoint, g, cvals)
    if isinstance(op, TIME_DEPENDENT) and op.stepper != "be":
        return propagate_sdirk_td(op, dt, M, X, adjoint, g, cvals, intervals)
    if isinstance(op, Stencil5TD):
        assert g is None or not adjoint, "the adjoint acts on the linear part only"
        return _propagate_stencil_td(op, dt, M, X, adjoint, g, cvals, intervals)
    Q = 0
    gp = cp = None
    cstride = 0
    if g is not None:
        assert not adjoint, "the adjoint acts on the linear part only"
        g = _f64(np.atleast_2d(g))
        Q = g.shape[0]
        cvals = _f64(cvals)
        if cvals.ndim == 2:
            assert cvals.shape == (M, Q)
        else:
            assert cvals.shape == (nvec, M, Q)
            cstride = M * Q
        gp, cp = _p(g), _p(cvals)
    L = lib()
    if isinstance(op, TridiagTD):
        j0s = np.ascontiguousarray(np.broadcast_to(np.asarray(intervals) * M, (nvec,)),
                                   dtype=np.int32)
        rc = L.orc_tridiag_td_propagate_many(n, op.steps, _p(_f64(op.lo_t)), _p(_f64(op.di_t)),
                                             _p(_f64(op.up_t)), _p(j0s), float(dt), int(M),
                                             int(adjoint), Q, gp, cp, cstride, nvec, _p(X))
        if rc == -3:
            raise ValueError("time-dependent operator: steps beyond its time grid")
    elif isinstance(op, Tridiag):
        rc = L.orc_tridiag_propagate_many(n, _p(_f64(op.lo)), _p(_f64(op.di)), _p(_f64(op.up)),
                                          float(dt), int(M), int(adjoint), Q, gp, cp, cstride,
                                          nvec, _p(X))
    else:
        rc = L.orc_stencil_propagate_many(op.mx, op.my, _p(_f64(op.C)), _p(_f64(op.W)),
                                          _p(_f64(op.E)), _p(_f64(op.S)), _p(_f64(op.N)),
                                          float(dt), int(M), int(adjoint), Q, gp, cp, cstride,
                                          nvec, _p(X))
    if rc != 0:
        raise RuntimeError("oracle propagation failed (zero pivot)")
    return X


def sdirk_tableau(scheme: str):
    """Butcher tableaus (c, A, b) of the two SDIRK methods of Sec. 4 (effect of
    the time discretisation)."""
    if scheme == "sdirk2":
        return np.array([1.0, 0.0]), np.array([[1.0, 0.0], [-1.0, 1.0]]), np.array([0.5, 0.5])
    if scheme == "sdirk2l":
        g = (2.0 - math.sqrt(2.0)) / 2.0
        return np.array([g, 1.0]), np.array([[g, 0.0], [1.0 - g, g]]), np.array([1.0 - g, g])
    raise ValueError(scheme)


def propagate_sdirk(op, dt: float, M: int, X: np.ndarray, scheme: str,
                    adjoint: bool = False, g: Optional[np.ndarray] = None,
                    cvals: Optional[np.ndarray] = None) -> np.ndarray:
    """M steps of a two-stage SDIRK method for u' = -A u + f(t) on every row of X:
    (I + a_ii dt A) K_i = -A (u + dt sum_{j<i} a_ij K_j) + f_i,
    u <- u + dt sum_i b_i K_i, with f_i = sum_q c_q(t + c_i dt) g_q the source
    at the stage time (cvals[..., step, i, q]).  Without a source the step map
    is R(-dt A) (R the stability function), so the adjoint is the same scheme
    with A^T."""
    _, At, b = sdirk_tableau(scheme)
    be = dataclasses.replace(op, stepper="be")   # the same A, backward-Euler solves
    U = np.array(X, dtype=np.float64, copy=True)
    nvec = U.shape[0]
    if g is not None:
        assert not adjoint, "the adjoint acts on the linear part"
        g = np.atleast_2d(np.asarray(g, dtype=np.float64))
        cv = np.asarray(cvals, dtype=np.float64)
        if cv.ndim == 3:
            cv = np.broadcast_to(cv, (nvec,) + cv.shape)
        assert cv.shape == (nvec, M, 2, g.shape[0]), "SDIRK sources take (M, 2, Q) stage samples"
    for step in range(M):
        K = []
        for i in range(2):
            arg = U + dt * sum(At[i, j] * K[j] for j in range(i))
            rhs = -op.matvec(arg, adjoint)
            if g is not None:
                rhs = rhs + cv[:, step, i, :] @ g
            K.append(propagate(be, At[i, i] * dt, 1, rhs, adjoint))
        U = U + dt * (b[0] * K[0] + b[1] * K[1])
    return U


def propagate_sdirk_td(op, dt: float, M: int, X: np.ndarray, adjoint: bool = False,
                       g: Optional[np.ndarray] = None, cvals: Optional[np.ndarray] = None,
                       intervals=0) -> np.ndarray:
    """Two-stage SDIRK steps for u' = -A(t) u + f(t) with a time-dependent A
    (TridiagTD / Stencil5TD with an SDIRK stepper): stage s of step J uses
    A_s = A(t_J + c_s dt) and the source at the same time,
      (I + a_ss dt A_s) K_s = -A_s (u + dt sum_{r<s} a_sr K_r) + f_s,
      u <- u + dt (b_1 K_1 + b_2 K_2).
    Row v runs steps intervals[v]*M .. intervals[v]*M + M - 1.  The adjoint
    applies the transpose of every step map, S_J^T, in reversed step order:
    with L_s = -(I + a_ss dt A_s)^-1 A_s (so that K_1 = L_1 u and
    K_2 = L_2 (u + dt a_21 K_1)),
      S_J^T v = v + dt b_2 w + L_1^T (dt b_1 v + dt^2 a_21 b_2 w),  w = L_2^T v,
    where L_s^T x = -A_s^T (I + a_ss dt A_s)^-T x."""
    _, At, b = sdirk_tableau(op.stepper)
    U = np.array(X, dtype=np.float64, copy=True)
    nvec = U.shape[0]
    j0s = np.broadcast_to(np.asarray(intervals) * M, (nvec,))
    if g is not None:
        assert not adjoint, "the adjoint acts on the linear part"
        g = np.atleast_2d(np.asarray(g, dtype=np.float64))
        cv = np.asarray(cvals, dtype=np.float64)
        if cv.ndim == 3:
            cv = np.broadcast_to(cv, (nvec,) + cv.shape)
        assert cv.shape == (nvec, M, 2, g.shape[0]), "SDIRK sources take (M, 2, Q) stage samples"

    def solve(A_s, a, x, transposed):
        return propagate(A_s, a * dt, 1, x[None, :], transposed)[0]

    for v in range(nvec):
        J0 = int(j0s[v])
        if J0 < 0 or J0 + M > op.steps:
            raise ValueError("time-dependent operator: steps beyond its time grid")
        u = U[v]
        for j in (range(M - 1, -1, -1) if adjoint else range(M)):
            A1, A2 = op.stage(J0 + j, 0), op.stage(J0 + j, 1)
            if not adjoint:
                r1 = -A1.matvec(u[None, :])[0]
                if g is not None:
                    r1 = r1 + cv[v, j, 0] @ g
                K1 = solve(A1, At[0, 0], r1, False)
                r2 = -A2.matvec((u + dt * At[1, 0] * K1)[None, :])[0]
                if g is not None:
                    r2 = r2 + cv[v, j, 1] @ g
                K2 = solve(A2, At[1, 1], r2, False)
                u = u + dt * (b[0] * K1 + b[1] * K2)
            else:
                w = -A2.matvec(solve(A2, At[1, 1], u, True)[None, :], adjoint=True)[0]
                z = dt * b[0] * u + dt * dt * At[1, 0] * b[1] * w
                u = u + dt * b[1] * w - A1.matvec(solve(A1, At[0, 0], z, True)[None, :],
                                                  adjoint=True)[0]
        U[v] = u
    return U


def interval_cvals(c: Optional[np.ndarray], i: int, M: int) -> Optional[np.ndarray]:
    """Source coefficients of interval i: rows i*M .. i*M+M-1 of c (N*M, Q), or
    of c (N*M, 2, Q) for the SDIRK steppers (the two stage samples of a step)."""
    if c is None:
        return None
    return c[i * M:(i + 1) * M]


def fine_solve(op, dt, M, v, i, g=None, c=None) -> np.ndarray:
    """F_i v: the full (affine) fine solver of interval i."""
    if g is None:
        return propagate(op, dt, M, v, intervals=i)
    return propagate(op, dt, M, v, g=g, cvals=interval_cvals(c, i, M), intervals=i)


def fine_solve_all(op, dt, M, V, g=None, c=None) -> np.ndarray:
    """F_i V[i] for every interval i = 0..N-1 at once (one call over the N
    independent propagations, which the C primitives run in parallel); row
    i is exactly fine_solve(op, dt, M, V[i], i, g, c)."""
    N = V.shape[0]
    iv = np.arange(N)
    if g is None:
        return propagate(op, dt, M, V, intervals=iv)
    return propagate(op, dt, M, V, g=g, cvals=np.stack([interval_cvals(c, i, M) for i in range(N)]),
                     intervals=iv)


def sequential_fine(op, dt, M, N, u0, g=None, c=None) -> np.ndarray:
    """u_{n+1} = F_{n+1} u_n (Sec. 2 problem statement): (N+1, n)."""
    u = np.zeros((N + 1, u0.shape[0]))
    u[0] = u0
    for i in range(N):
        u[i + 1] = fine_solve(op, dt, M, u[i], i, g, c)
    return u


# ----------------------------------------------------------------------------
# Randomized SVD (Sec. 2.1, steps 1-6)
# ----------------------------------------------------------------------------
MGS_TAU = 1e-13


def mgs2(Y: np.ndarray, tau: float = MGS_TAU):
    """Orthonormal basis of the span of the rows of Y (k, n): modified
    Gram-Schmidt applied twice with deflation (a row whose norm drops below
    tau times its original norm is discarded).  Returns (Q (r, n), keep)."""
    Y = _f64(Y)
    k, n = Y.shape
    Q = np.zeros((max(k, 1), n))
    keep = np.zeros(max(k, 1), dtype=np.int32)
    r = lib().orc_mgs2(n, k, _p(Y), float(tau), _p(Q), _p(keep))
    assert r >= 0
    return Q[:r].copy(), keep[:k].astype(bool)


def jacobi_svd(A: np.ndarray):
    """SVD of a small dense matrix A (m, k) by one-sided Jacobi.  Returns
    (U (m, r), s (r,), V (k, r)) with r = min(m, k), s descending."""
    A = np.asarray(A, dtype=np.float64)
    m, k = A.shape
    if m < k:
        V, s, U = jacobi_svd(A.T)
        return U, s, V
    Acm = np.asfortranarray(A)          # column-major m x k
    U = np.zeros((k, m))                 # rows = columns of U
    s = np.zeros(k)
    V = np.zeros((k, k))
    sweeps = lib().orc_jacobi_svd(m, k, Acm.ctypes.data_as(ctypes.c_void_p), _p(U), _p(s), _p(V))
    if sweeps < 0:
        raise RuntimeError("Jacobi SVD did not converge")
    return U.T.copy(), s, V.T.copy()


@dataclass
class CoarseInterval:
    """Factors of G_i' = U diag(S) V^T plus the data needed for the bounds."""
    U: np.ndarray            # (n, R_i)  left singular vectors psi
    S: np.ndarray            # (R_i,)    sigma_{i,1..R_i}
    V: np.ndarray            # (n, R_i)  right singular vectors phi
    sigma: np.ndarray        # all singular values of the small matrix (desc.)
    rank_w: int              # dim of span{F' omega}   after deflation
    rank_v: int              # dim of span{F'^* w}     after deflation
    sigma_next: float        # sigma_{i, R_i + 1} estimate (0 if unavailable)
    fine_evals: int          # forward + adjoint propagations spent


def rsvd_interval(op, dt, M, i, R, p, seed, tau=MGS_TAU) -> CoarseInterval:
    """Randomized SVD of F_i' in the steps of Sec. 2.1.

    The lifting in step 5 uses the left singular vectors of the small matrix
    with the basis w (image of F') and the right ones with the basis v
    (image of F'^*): with M_{ij} = (F'^* w_i, v_j) = (w_i, F' v_j) one has
    P_W F' = W M V^T, so the lifted SVD is (W Psi) Sigma (V Phi)^T.  (The
    paper's text pairs them the other way round; this follows its own formula
    for P_W F' in step 4.)"""
    n = op.n
    ell = R + p
    omega = gauss_block(seed, i, n, ell)                         # step 1
    Y = propagate(op, dt, M, omega, intervals=i)                 # F' omega
    W, _ = mgs2(Y, tau)                                          # step 2
    Z = propagate(op, dt, M, W, adjoint=True, intervals=i)       # step 3
    Vb, _ = mgs2(Z, tau)                                         # step 4
    Mm = Z @ Vb.T                                                # step 5: M_ij = (F'^*w_i, v_j)
    if Mm.size == 0:
        return CoarseInterval(np.zeros((n, 0)), np.zeros(0), np.zeros((n, 0)), np.zeros(0),
                              W.shape[0], Vb.shape[0], 0.0, ell + W.shape[0])
    Psi, s, Phi = jacobi_svd(Mm)
    Ri = min(R, s.shape[0])                                      # step 6
    U = W.T @ Psi[:, :Ri]
    V = Vb.T @ Phi[:, :Ri]
    # sigma_{R+1} from the oversampled small SVD; when deflation left no
    # (R+1)-th value, the directions dropped were below tau * sigma_1
    sig_next = float(s[Ri]) if s.shape[0] > Ri else tau * float(s[0])
    return CoarseInterval(U, s[:Ri].copy(), V, s, W.shape[0], Vb.shape[0], sig_next,
                          ell + W.shape[0])


@dataclass
class Coarse:
    intervals: List[CoarseInterval]
    R: int
    p: int

    @property
    def delta(self) -> float:
        """delta := max_n sigma_{n,1} (Eq. (bounds_delta_eps))."""
        return max((float(c.sigma[0]) if c.sigma.size else 0.0) for c in self.intervals)

    @property
    def eps(self) -> float:
        """eps := max_n sigma_{n,R_n+1} (Eq. (bounds_delta_eps)), estimated
        from the oversampled small SVD as in Sec. 4.5."""
        return max(c.sigma_next for c in self.intervals)

    def apply_lin(self, i: int, v: np.ndarray) -> np.ndarray:
        """G_i' v = sum_r psi_r sigma_r (phi_r, v) (Eq. (spectral_G) without b)."""
        c = self.intervals[i]
        return c.U @ (c.S * (c.V.T @ v))


def build_coarse(op, dt, M, N, R, p, seed) -> Coarse:
    """Coarse solvers of all N intervals (each an independent rSVD)."""
    return Coarse([rsvd_interval(op, dt, M, i, R, p, seed) for i in range(N)], R, p)


# ----------------------------------------------------------------------------
# Variant of Sec. 2.2: F'^* evaluated on an independent set of random vectors
# (a two-sided sketch) instead of on the basis w, so that both sketches are
# independent and run in one round, at some cost in accuracy.
# ----------------------------------------------------------------------------
STREAM_PSI = 3


def rsvd_interval_indep(op, dt, M, i, R, p, seed, tau=MGS_TAU) -> CoarseInterval:
    """Two-sided randomized SVD of F_i': Y = F' Omega (l = R + p columns),
    Z = F'^* Psi (2 l independent columns, Philox stream 3), Q = orth(Y),
    X = argmin ||(Psi^T Q) X - Psi^T F'|| (least squares, Psi^T F' = Z^T), so
    F' ~ Q X; the SVD of X (its row space orthonormalised, then the small
    SVD) gives U = Q^T Psi_s, S, V = Vh^T Phi_s.  Accuracy: exact when the
    sketches span the whole space (checked by brute force); otherwise below
    the two-pass variant.  Pinned also for partial sketches, against the
    same estimate formed from the dense F' with a library pseudo-inverse and
    SVD, and by the closed-form heat spectrum at a loose tolerance.  The
    least-squares step is lstsq_mgs (Gram-Schmidt QR and back substitution,
    no LAPACK)."""
    n = op.n
    ell = R + p
    ell2 = 2 * ell
    omega = gauss_block(seed, i, n, ell)
    psi = gauss_block(seed, i, n, ell2, stream=STREAM_PSI)
    Y = propagate(op, dt, M, omega, intervals=i)                 # rows F' omega_j
    Z = propagate(op, dt, M, psi, adjoint=True, intervals=i)     # rows F'^T psi_a
    Q, _ = mgs2(Y, tau)                                          # rows q_c
    k = Q.shape[0]
    if k == 0:
        return CoarseInterval(np.zeros((n, 0)), np.zeros(0), np.zeros((n, 0)), np.zeros(0),
                              0, 0, 0.0, ell + ell2)
    B = psi @ Q.T                                                # (2l, k): (psi_a, q_c)
    X = lstsq_mgs(B, Z, tau)                                     # (k, n): F' ~ Q^T X
    Vh, _ = mgs2(X, tau)                                         # row space of X
    Xs = X @ Vh.T                                                # (k, k'): X = Xs Vh
    Psi_s, s, Phi_s = jacobi_svd(Xs)
    Ri = min(R, s.shape[0])
    U = Q.T @ Psi_s[:, :Ri]
    V = Vh.T @ Phi_s[:, :Ri]
    sig_next = float(s[Ri]) if s.shape[0] > Ri else tau * float(s[0])
    return CoarseInterval(U, s[:Ri].copy(), V, s, k, Vh.shape[0], sig_next, ell + ell2)


def lstsq_mgs(B: np.ndarray, Z: np.ndarray, tau: float = MGS_TAU) -> np.ndarray:
    """Least-squares solution X of min ||B X - Z||_F for B (m, k) of full
    column rank k <= m, through a thin QR factorisation of B by the oracle's
    own Gram-Schmidt (mgs2 on the columns of B): B = Qb^T Rb with Qb (k, m)
    orthonormal rows and Rb = Qb B upper triangular, then Rb X = Qb Z by
    back substitution.  Raises when a column of B is deflated (B rank
    deficient), where the least-squares solution is not unique."""
    B = _f64(B)
    Z = _f64(Z)
    m, k = B.shape
    Qb, keep = mgs2(B.T, tau)
    if Qb.shape[0] != k:
        raise RuntimeError("lstsq_mgs: B is rank deficient (%d of %d columns kept)"
                           % (Qb.shape[0], k))
    Rb = Qb @ B                                                  # (k, k), upper triangular
    rhs = Qb @ Z                                                 # (k, n)
    X = np.zeros((k, Z.shape[1]))
    for j in range(k - 1, -1, -1):                               # back substitution
        X[j] = (rhs[j] - Rb[j, j + 1:] @ X[j + 1:]) / Rb[j, j]
    return X


def build_coarse_indep(op, dt, M, N, R, p, seed) -> Coarse:
    """Coarse solvers from the two-sided sketch (rsvd_interval_indep)."""
    return Coarse([rsvd_interval_indep(op, dt, M, i, R, p, seed) for i in range(N)], R, p)


def exact_coarse(op, dt, M, N, R) -> Coarse:
    """Truncated SVD of the dense F' (small n only): the exact G_n of
    Eq. (spectral_G), used by tests as a comparison coarse solver."""
    n = op.n

    def one(i):
        Fp = propagate(op, dt, M, np.eye(n), intervals=i).T      # column j = F_i' e_j
        Uf, s, Vf = jacobi_svd(Fp)
        return CoarseInterval(Uf[:, :R].copy(), s[:R].copy(), Vf[:, :R].copy(), s.copy(), n, n,
                              float(s[R]) if R < n else 0.0, 0)
    if isinstance(op, TIME_DEPENDENT):
        return Coarse([one(i) for i in range(N)], R, 0)
    return Coarse([one(0)] * N, R, 0)


# ----------------------------------------------------------------------------
# Parareal (Eq. (def_Parareal)) with the a posteriori bound (Eq. (apost_bound))
# ----------------------------------------------------------------------------
@dataclass
class PararealResult:
    iterates: List[np.ndarray]           # u^k, each (N+1, n), k = 0..k_done
    bounds: List[np.ndarray]             # a posteriori bound per k>=1, (N+1,), entry 0 = 0
    b: np.ndarray                        # affine parts b_i = F_i 0, (N, n)
    k_done: int
    fine_evals: int                      # fine evaluations per interval (Eq. (num_F_eval))


def apost_bound(delta: float, eps: float, du: np.ndarray) -> np.ndarray:
    """eps * sum_{m=1}^{n-1} delta^{n-m-1} ||u^k_m - u^{k-1}_m||  for n = 0..N
    (Eq. (apost_bound)); du[m] = ||u^k_m - u^{k-1}_m||, m = 0..N."""
    Np1 = du.shape[0]
    out = np.zeros(Np1)
    for n in range(1, Np1):
        out[n] = eps * sum(delta ** (n - m - 1) * du[m] for m in range(1, n))
    return out


def parareal(op, dt, M, N, coarse: Coarse, u0, g=None, c=None, K: Optional[int] = None,
             tol: Optional[float] = None) -> PararealResult:
    """Parareal with G_i v = G_i' v + b_i, literal form of Eq. (def_Parareal):

      u^0_0 = u0,  u^0_{i+1} = G_i u^0_i;
      u^{k+1}_0 = u0,  u^{k+1}_{i+1} = F_i u^k_i + G_i u^{k+1}_i - G_i u^k_i.

    Stops after K iterations (clamped to N, where the iterates equal the fine
    solution), or earlier at the first k >= 1 with
    max_n bound_n^k <= tol * max_n ||u^k_n|| when tol is given."""
    u0 = _f64(u0)
    n = u0.shape[0]
    Kmax = N if K is None else min(int(K), N)
    # affine parts b_i = F_i 0 (Eq. (F_n_affine)); one fine evaluation each
    if g is None:
        b = np.zeros((N, n))
    else:
        b = np.stack([fine_solve(op, dt, M, np.zeros(n), i, g, c) for i in range(N)])
    evals = 1

    def G(i, v):
        return coarse.apply_lin(i, v) + b[i]

    u = np.zeros((N + 1, n))
    u[0] = u0
    for i in range(N):
        u[i + 1] = G(i, u[i])
    iterates = [u]
    bounds = []
    delta, eps = coarse.delta, coarse.eps
    k = 0
    while k < Kmax:
        prev = iterates[-1]
        Fprev = fine_solve_all(op, dt, M, prev[:N], g, c)
        evals += 1
        new = np.zeros_like(prev)
        new[0] = u0
        for i in range(N):
            new[i + 1] = Fprev[i] + G(i, new[i]) - G(i, prev[i])
        k += 1
        iterates.append(new)
        du = np.linalg.norm(new - prev, axis=1)
        bounds.append(apost_bound(delta, eps, du))
        if tol is not None and tol > 0:
            scale = np.max(np.linalg.norm(new, axis=1))
            if np.max(bounds[-1]) <= tol * scale:
                break
    return PararealResult(iterates, bounds, b, k, evals)


# ----------------------------------------------------------------------------
# A priori bounds (Theorem 1)
# ----------------------------------------------------------------------------
def apriori_initial(delta: float, eps: float, bnorm: np.ndarray) -> np.ndarray:
    """Eq. (error_bound_initial): bound on ||e^0_n||, n = 0..N, where
    bnorm[m] = ||b_m|| with b_0 := u0 and b_m the affine part of the paper's
    F_m (m = 1..N-1)."""
    N = bnorm.shape[0]
    out = np.zeros(N + 1)
    for n in range(1, N + 1):
        out[n] = sum(min(2 * delta, (n - m) * eps) * delta ** (n - m - 1) * bnorm[m]
                     for m in range(0, n))
    return out


def apriori_k(delta: float, eps: float, bnorm: np.ndarray, k: int) -> np.ndarray:
    """Eq. (error_bound_eps_delta2): 2 eps^k sum_{m=0}^{n-k-1} C(n-m, k)
    delta^{n-m-k} ||b_m||, n = 0..N (k >= 1)."""
    N = bnorm.shape[0]
    out = np.zeros(N + 1)
    for n in range(1, N + 1):
        out[n] = 2 * eps ** k * sum(math.comb(n - m, k) * delta ** (n - m - k) * bnorm[m]
                                    for m in range(0, n - k))
    return out


def apriori_from_e0(delta: float, eps: float, e0: np.ndarray, k: int) -> np.ndarray:
    """Eq. (error_bound_eps_delta): eps^k sum_{m=1}^{n-k} C(n-m, k-1)
    delta^{n-m-k} ||e^0_m||, n = 0..N; e0[m] = ||e^0_m||."""
    Np1 = e0.shape[0]
    out = np.zeros(Np1)
    for n in range(1, Np1):
        out[n] = eps ** k * sum(math.comb(n - m, k - 1) * delta ** (n - m - k) * e0[m]
                                for m in range(1, n - k + 1))
    return out


def efficiency(err_max: float, bound: np.ndarray) -> float:
    """eta^k of Eq. (def_efficiency) with the bound maximised over 1 <= n <= N
    (the paper's n < N reads as a typo for n <= N; both are stated)."""
    b = float(np.max(bound[1:])) if bound.shape[0] > 1 else 0.0
    return err_max / b if b > 0 else math.inf


def rel_err(iterate: np.ndarray, ref: np.ndarray) -> float:
    """max_n ||u^k_n - u_n|| / max_n ||u_n|| (the paper's max-over-time l2 error,
    normalised)."""
    return float(np.max(np.linalg.norm(iterate - ref, axis=1)) /
                 np.max(np.linalg.norm(ref, axis=1)))


# ----------------------------------------------------------------------------
# Classical Parareal: a single backward-Euler step as coarse solver (the
# comparison method of Sec. 4, dashed lines of Experiments 1-4)
# ----------------------------------------------------------------------------
def coarse_be(op, dt, M, v, i, g=None, c=None) -> np.ndarray:
    """G_i v for the classical coarse solver: one backward-Euler step of size
    M*dt over interval i, the source sampled at the interval's end t_{i+1}
    (the step end, as in the fine solver)."""
    if isinstance(op, TIME_DEPENDENT):
        op = op.step(i * M + M - 1)          # A at the interval's end
    if g is None:
        return propagate(op, M * dt, 1, v)
    return propagate(op, M * dt, 1, v, g=g, cvals=interval_cvals(c, i, M)[-1:])


def parareal_classical(op, dt, M, N, u0, g=None, c=None, K: Optional[int] = None,
                       tol: Optional[float] = None) -> PararealResult:
    """Parareal (Eq. def_Parareal, literal form) with G_i = coarse_be.

    Stops after K iterations (clamped to N), or at the first k >= 1 with
    max_n ||u^k_n - u^{k-1}_n|| <= tol * max_n ||u^k_n|| (the classical
    coarse solver has no a posteriori bound of Eq. apost_bound).  `bounds`
    holds the increments ||u^k_n - u^{k-1}_n|| per iteration."""
    u0 = _f64(u0)
    n = u0.shape[0]
    Kmax = N if K is None else min(int(K), N)
    u = np.zeros((N + 1, n))
    u[0] = u0
    for i in range(N):
        u[i + 1] = coarse_be(op, dt, M, u[i], i, g, c)
    iterates = [u]
    incs = []
    k, evals = 0, 0
    while k < Kmax:
        prev = iterates[-1]
        Fprev = np.stack([fine_solve(op, dt, M, prev[i], i, g, c) for i in range(N)])
        evals += 1
        new = np.zeros_like(prev)
        new[0] = u0
        for i in range(N):
            new[i + 1] = Fprev[i] + coarse_be(op, dt, M, new[i], i, g, c) \
                - coarse_be(op, dt, M, prev[i], i, g, c)
        k += 1
        iterates.append(new)
        du = np.linalg.norm(new - prev, axis=1)
        incs.append(du)
        if tol is not None and tol > 0:
            if np.max(du) <= tol * np.max(np.linalg.norm(new, axis=1)):
                break
    return PararealResult(iterates, incs, np.zeros((N, n)), k, evals)
