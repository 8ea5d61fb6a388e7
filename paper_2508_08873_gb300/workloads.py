"""Seeded synthetic problem generators shared by the tests, the benchmark and
the oracle's callers.

This module only builds INPUTS: semi-discretised operators A of u_t = -A u + f
(finite differences, homogeneous Dirichlet, interior nodes only), initial values
u0 and separable sources f(t, x) = sum_q c_q(t) g_q(x).  It holds none of the
method's arithmetic (no time stepping, no randomized SVD, no Parareal), imports
neither the CUDA library nor the oracle, and is plain numpy.

The problems are finite-difference stand-ins for the paper's experiments
(Sec. 4: 1D heat equation, Experiment 1; 2D diffusion, Experiment 3):
  * heat1d      u_t = u_xx on (0,1), n interior nodes;
  * adr1d       u_t = 0.01 u_xx - u_x - 0.1 u, first-order upwind for u_x;
  * diff2d      u_t = div(kappa grad u) - u, kappa piecewise constant on an
                8x8 checkerboard with values 10^U(0,2), 5-point stencil,
                kappa evaluated at face midpoints;
  * adv2d       u_t = nu Lap u - b.grad u, b = (-(y-1/2), x-1/2), upwind;
  * heat_td     u_t = d/dx[(1 + 0.9 sin(7 pi t + 2 pi x)) u_x] + f with Neumann
                conditions (Experiment 2): a time-dependent tridiagonal A;
  * heat2d_td   u_t = div(d(x, y, t) grad u) + f on (0,1)^2 with Dirichlet
                conditions (Experiment 3): a time-dependent 5-point A.
Random problem data come from numpy's PCG64 seeded per problem; the Gaussian
sketch vectors of the method are NOT drawn here.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np


@dataclass
class Problem:
    """One Parareal problem: operator, time grid, data and rSVD parameters."""
    name: str
    kind: str                       # "tridiag" or "stencil5"
    n: int
    dt: float
    M: int                          # fine steps per coarse interval
    N: int                          # coarse intervals
    R: int                          # truncation rank
    p: int                          # oversampling
    seed: int                       # sketch seed
    u0: np.ndarray
    # tridiagonal A: row i = lo[i] x[i-1] + di[i] x[i] + up[i] x[i+1]
    lo: Optional[np.ndarray] = None
    di: Optional[np.ndarray] = None
    up: Optional[np.ndarray] = None
    # 5-point A on an mx x my grid (node p = iy*mx + ix)
    mx: int = 0
    my: int = 0
    st: Optional[dict] = None        # keys C, W, E, S, N -> (n,) arrays
    # separable source: g (Q, n), c (N*M, Q) at fine times J*dt, J = 1..N*M
    g: Optional[np.ndarray] = None
    c: Optional[np.ndarray] = None
    extra: dict = field(default_factory=dict)

    @property
    def T(self) -> float:
        return self.dt * self.M * self.N

    @property
    def Q(self) -> int:
        return 0 if self.g is None else self.g.shape[0]


def fine_times(N: int, M: int, dt: float) -> np.ndarray:
    """t_J = J*dt for J = 1..N*M (the step-end times where f is sampled)."""
    return dt * np.arange(1, N * M + 1, dtype=np.float64)


# ----------------------------------------------------------------------------
# 1D operators
# ----------------------------------------------------------------------------
def heat1d_op(n: int):
    """A = (1/h^2) tridiag(-1, 2, -1), h = 1/(n+1)."""
    h = 1.0 / (n + 1)
    lo = np.full(n, -1.0 / h ** 2)
    di = np.full(n, 2.0 / h ** 2)
    up = np.full(n, -1.0 / h ** 2)
    lo[0] = 0.0
    up[-1] = 0.0
    return lo, di, up


def adr1d_op(n: int, nu: float = 0.01, vel: float = 1.0, react: float = 0.1):
    """A u = -nu u_xx + vel u_x + react u, backward difference for u_x (vel > 0)."""
    h = 1.0 / (n + 1)
    lo = np.full(n, -nu / h ** 2 - vel / h)
    di = np.full(n, 2.0 * nu / h ** 2 + vel / h + react)
    up = np.full(n, -nu / h ** 2)
    lo[0] = 0.0
    up[-1] = 0.0
    return lo, di, up


def bumps1d(x: np.ndarray, rng: np.random.Generator, count: int = 5) -> np.ndarray:
    """sum_i exp(-((x - c_i)/w_i)^2), c_i ~ U(0.1, 0.9), w_i ~ U(0.02, 0.1)."""
    cs = rng.uniform(0.1, 0.9, count)
    ws = rng.uniform(0.02, 0.1, count)
    return sum(np.exp(-((x - c) / w) ** 2) for c, w in zip(cs, ws))


def heat1d(n: int = 255, N: int = 16, M: int = 64, R: int = 8, p: int = 4, seed: int = 0,
           T: float = 1.0, source: bool = True) -> Problem:
    """1D heat equation, u0 = x(1-x), f = sin(2 pi t) exp(-100 (x-1/2)^2)."""
    lo, di, up = heat1d_op(n)
    x = np.arange(1, n + 1) / (n + 1)
    dt = T / (N * M)
    g = c = None
    if source:
        g = np.exp(-100.0 * (x - 0.5) ** 2)[None, :]
        c = np.sin(2 * np.pi * fine_times(N, M, dt))[:, None]
    return Problem("heat1d", "tridiag", n, dt, M, N, R, p, seed, x * (1 - x),
                   lo=lo, di=di, up=up, g=g, c=c)


def adr1d(n: int = 4095, N: int = 64, M: int = 256, R: int = 16, p: int = 8, seed: int = 0,
          data_seed: int = 1, T: float = 1.0) -> Problem:
    """1D advection-diffusion-reaction, u0 = 5 seeded Gaussian bumps, f = 0."""
    lo, di, up = adr1d_op(n)
    x = np.arange(1, n + 1) / (n + 1)
    rng = np.random.default_rng(data_seed)
    return Problem("adr1d", "tridiag", n, T / (N * M), M, N, R, p, seed, bumps1d(x, rng),
                   lo=lo, di=di, up=up)


def heat_td_op(n: int, N: int, M: int, T: float = 1.0):
    """Experiment 2's operator, -d/dx[(1 + 0.9 sin(7 pi t + 2 pi x)) du/dx] with
    homogeneous Neumann conditions: n cells of width h = 1/n (unknowns at the
    cell centres), the conductivity at the interior faces x = (i+1) h and at
    the end t_{J+1} = (J+1) dt of every fine step J = 0..N*M-1 (fully implicit
    backward Euler), no flux through the boundary faces.  Returns lo_t, di_t,
    up_t, each (N*M, n): row J holds A(t_{J+1})."""
    return heat_td_at(n, fine_times(N, M, T / (N * M)))


def heat_td_at(n: int, times) -> tuple:
    """Experiment 2's operator (see heat_td_op) at the given times: lo, di,
    up, each (len(times), n), row r holding A(times[r])."""
    t = np.asarray(times, dtype=np.float64)
    h = 1.0 / n
    xf = h * np.arange(1, n)
    kap = (1.0 + 0.9 * np.sin(7 * np.pi * t[:, None] + 2 * np.pi * xf[None, :])) / h ** 2
    J = t.shape[0]
    di = np.zeros((J, n))
    di[:, :-1] += kap
    di[:, 1:] += kap
    lo = np.zeros((J, n))
    lo[:, 1:] = -kap
    up = np.zeros((J, n))
    up[:, :-1] = -kap
    return lo, di, up


def heat_td(n: int = 100, N: int = 10, M: int = 10, R: int = 5, p: int = 1, seed: int = 0,
            T: float = 1.0) -> Problem:
    """Experiment 2 stand-in: heat equation with the space- and time-dependent
    conductivity 1 + 0.9 sin(7 pi t + 2 pi x), Neumann conditions, n = 100
    cells, N = 10 intervals of M = 10 steps on [0, 1] (the paper's mesh and
    time grid), f = sin(2 pi t) exp(-100 (x-1/2)^2), u0 = x(1-x).  The
    operator arrays (N*M, n) are in lo, di, up (kind "tridiag_td")."""
    lo, di, up = heat_td_op(n, N, M, T)
    x = (np.arange(n) + 0.5) / n
    dt = T / (N * M)
    g = np.exp(-100.0 * (x - 0.5) ** 2)[None, :]
    c = np.sin(2 * np.pi * fine_times(N, M, dt))[:, None]
    return Problem("heat_td", "tridiag_td", n, dt, M, N, R, p, seed, x * (1 - x),
                   lo=lo, di=di, up=up, g=g, c=c)


# ----------------------------------------------------------------------------
# 2D operators (5-point stencils)
# ----------------------------------------------------------------------------
def _grid(m: int):
    h = 1.0 / (m + 1)
    coords = np.arange(1, m + 1) * h
    X, Y = np.meshgrid(coords, coords, indexing="xy")   # X[iy, ix] = x_ix
    return h, X.ravel(), Y.ravel()


def diff2d_op(m: int, kappa_table: np.ndarray, react: float = 1.0) -> dict:
    """A u = -div(kappa grad u) + react u; kappa sampled at face midpoints,
    block index floor(8 * coordinate) clamped to 0..7."""
    h = 1.0 / (m + 1)
    idx = np.arange(m)
    xn = (idx + 1) * h                       # node coordinates

    def kap(xx, yy):
        bx = np.clip(np.floor(8 * xx).astype(int), 0, 7)
        by = np.clip(np.floor(8 * yy).astype(int), 0, 7)
        return kappa_table[by, bx]

    XN, YN = np.meshgrid(xn, xn, indexing="xy")
    kE = kap(XN + 0.5 * h, YN)
    kW = kap(XN - 0.5 * h, YN)
    kN = kap(XN, YN + 0.5 * h)
    kS = kap(XN, YN - 0.5 * h)
    ih2 = 1.0 / h ** 2
    C = (kE + kW + kN + kS) * ih2 + react
    W = -kW * ih2
    E = -kE * ih2
    S = -kS * ih2
    Nn = -kN * ih2
    W[:, 0] = 0.0
    E[:, -1] = 0.0
    S[0, :] = 0.0
    Nn[-1, :] = 0.0
    return {k: v.ravel().astype(np.float64) for k, v in
            dict(C=C, W=W, E=E, S=S, N=Nn).items()}


def adv2d_op(m: int, nu: float) -> dict:
    """A u = -nu Lap u + b.grad u, b = (-(y-1/2), x-1/2) at the nodes; per node
    and component the backward difference when b_c >= 0, else forward."""
    h, X, Y = _grid(m)
    bx = -(Y - 0.5)
    by = X - 0.5
    ih2 = 1.0 / h ** 2
    C = 4 * nu * ih2 + (np.abs(bx) + np.abs(by)) / h
    W = -nu * ih2 - np.maximum(bx, 0) / h
    E = -nu * ih2 - np.maximum(-bx, 0) / h
    S = -nu * ih2 - np.maximum(by, 0) / h
    Nn = -nu * ih2 - np.maximum(-by, 0) / h
    ix = np.tile(np.arange(m), m)
    iy = np.repeat(np.arange(m), m)
    W[ix == 0] = 0.0
    E[ix == m - 1] = 0.0
    S[iy == 0] = 0.0
    Nn[iy == m - 1] = 0.0
    return dict(C=C, W=W, E=E, S=S, N=Nn)


def diff2d(m: int = 511, N: int = 128, M: int = 32, R: int = 32, p: int = 10, seed: int = 0,
           data_seed: int = 3, T: float = 1.0, modes: int = 32) -> Problem:
    """2D diffusion-reaction on a checkerboard conductivity; u0 = sum of
    modes^2 sine modes with N(0, 1/(kx^2+ky^2)) amplitudes; f = 0."""
    rng = np.random.default_rng(data_seed)
    table = 10.0 ** rng.uniform(0.0, 2.0, (8, 8))
    st = diff2d_op(m, table)
    h, X, Y = _grid(m)
    kk = np.arange(1, modes + 1)
    amp = rng.standard_normal((modes, modes)) / np.sqrt(kk[:, None] ** 2 + kk[None, :] ** 2)
    sx = np.sin(np.pi * np.outer(kk, X))      # (modes, n)
    sy = np.sin(np.pi * np.outer(kk, Y))
    u0 = np.einsum("ab,an,bn->n", amp, sx, sy)
    return Problem("diff2d", "stencil5", m * m, T / (N * M), M, N, R, p, seed, u0,
                   mx=m, my=m, st=st, extra=dict(kappa=table))


def bumps2d(X, Y, rng, count: int = 5):
    cx = rng.uniform(0.1, 0.9, count)
    cy = rng.uniform(0.1, 0.9, count)
    w = rng.uniform(0.02, 0.1, count)
    return sum(np.exp(-((X - a) ** 2 + (Y - b) ** 2) / ww ** 2) for a, b, ww in zip(cx, cy, w))


ADV2D_GRIDS = (63, 127, 255, 511)


def adv2d(index: int, grids=ADV2D_GRIDS, N: int = 32, M: int = 64, R: int = 24, p: int = 8,
          seed: int = 0, data_seed: int = 4, T: float = 1.0, m: Optional[int] = None) -> Problem:
    """Problem `index` of the uneven batch: grid drawn uniformly from `grids`,
    nu log-uniform in [0.002, 0.05], u0 = 5 seeded 2D bumps, f = 0."""
    rng = np.random.default_rng([data_seed, index])
    mm = int(rng.choice(np.asarray(grids))) if m is None else m
    nu = float(10.0 ** rng.uniform(np.log10(0.002), np.log10(0.05)))
    st = adv2d_op(mm, nu)
    h, X, Y = _grid(mm)
    return Problem("adv2d", "stencil5", mm * mm, T / (N * M), M, N, R, p, seed,
                   bumps2d(X, Y, rng), mx=mm, my=mm, st=st, extra=dict(nu=nu))


# ----------------------------------------------------------------------------
# Serving requests: new u0 and a new separable source on a resident operator
# ----------------------------------------------------------------------------
def serving_request(n: int, N: int, M: int, dt: float, index: int, data_seed: int = 2,
                    terms: int = 4):
    """f(t, x) = sum_{i<terms} a_i sin(w_i t) exp(-(x-c_i)^2 / w_i'^2), a_i ~ N(0,1),
    w_i ~ U(1, 20), c_i ~ U(0.1, 0.9), widths ~ U(0.02, 0.1); u0 = 5 bumps.
    Returns (u0, g (terms, n), c (N*M, terms))."""
    rng = np.random.default_rng([data_seed, index])
    x = np.arange(1, n + 1) / (n + 1)
    a = rng.standard_normal(terms)
    om = rng.uniform(1.0, 20.0, terms)
    cc = rng.uniform(0.1, 0.9, terms)
    ww = rng.uniform(0.02, 0.1, terms)
    g = np.stack([np.exp(-((x - cc[i]) / ww[i]) ** 2) for i in range(terms)])
    t = fine_times(N, M, dt)
    c = np.stack([a[i] * np.sin(om[i] * t) for i in range(terms)], axis=1)
    u0 = bumps1d(x, rng)
    return u0, g, c


def heat2d_td_op(m: int, N: int, M: int, T: float = 1.0) -> dict:
    """Experiment 3's operator, -div(d grad u) with d(x, y, t) = 1 + 0.9
    sin(7 pi t) on [0, 1/2]^2 + 0.9 cos(5 pi t) on [1/2, 1]^2 (closed
    squares; 1 elsewhere), homogeneous Dirichlet, m x m interior nodes of
    spacing h = 1/(m+1), d at the face midpoints and at the end t_{J+1} of
    every fine step J = 0..N*M-1.  Returns C, W, E, S, N, each (N*M, m*m):
    row J holds the stencil of A(t_{J+1})."""
    return heat2d_td_at(m, fine_times(N, M, T / (N * M)))


def heat2d_td_at(m: int, times) -> dict:
    """Experiment 3's operator (see heat2d_td_op) at the given times: C, W,
    E, S, N, each (len(times), m*m), row r the stencil of A(times[r])."""
    t = np.asarray(times, dtype=np.float64)
    h = 1.0 / (m + 1)
    xn = (np.arange(m) + 1) * h
    XN, YN = np.meshgrid(xn, xn, indexing="xy")
    sw = lambda xx, yy: ((xx <= 0.5) & (yy <= 0.5)).astype(np.float64)
    ne = lambda xx, yy: ((xx >= 0.5) & (yy >= 0.5)).astype(np.float64)
    faces = dict(E=(XN + 0.5 * h, YN), W=(XN - 0.5 * h, YN), N=(XN, YN + 0.5 * h),
                 S=(XN, YN - 0.5 * h))
    ih2 = 1.0 / h ** 2
    out = {}
    for k, (xx, yy) in faces.items():
        a = sw(xx, yy).ravel()
        b = ne(xx, yy).ravel()
        d = 1.0 + 0.9 * np.sin(7 * np.pi * t)[:, None] * a[None, :] + \
            0.9 * np.cos(5 * np.pi * t)[:, None] * b[None, :]
        out[k] = -d * ih2
    ix = np.tile(np.arange(m), m)
    iy = np.repeat(np.arange(m), m)
    C = -(out["E"] + out["W"] + out["N"] + out["S"])
    out["W"][:, ix == 0] = 0.0
    out["E"][:, ix == m - 1] = 0.0
    out["S"][:, iy == 0] = 0.0
    out["N"][:, iy == m - 1] = 0.0
    out["C"] = C
    return {k: np.ascontiguousarray(out[k]) for k in ("C", "W", "E", "S", "N")}


def heat2d_td(m: int = 99, N: int = 10, M: int = 10, R: int = 6, p: int = 1, seed: int = 0,
              T: float = 1.0) -> Problem:
    """Experiment 3 stand-in: 2D heat equation with the conductivity of
    heat2d_td_op, f = 100 sin(5 pi t)(1 + cos(3 pi x))(1 + sin(4 pi y)) (one
    separable term), u0 = 10 on [0.6, 0.8]^2 and 0 elsewhere; m = 99 (h =
    0.01, the paper's 100 x 100 mesh), N = 10 intervals of M = 10 steps on
    [0, 1], R = 6, p = 1.  The operator arrays (N*M, m*m) are in st_t
    (kind "stencil5_td")."""
    st_t = heat2d_td_op(m, N, M, T)
    h, X, Y = _grid(m)
    dt = T / (N * M)
    g = (100.0 * (1.0 + np.cos(3 * np.pi * X)) * (1.0 + np.sin(4 * np.pi * Y)))[None, :]
    c = np.sin(5 * np.pi * fine_times(N, M, dt))[:, None]
    u0 = 10.0 * ((X >= 0.6) & (X <= 0.8) & (Y >= 0.6) & (Y <= 0.8)).astype(np.float64)
    return Problem("heat2d_td", "stencil5_td", m * m, dt, M, N, R, p, seed, u0, mx=m, my=m,
                   g=g, c=c, extra=dict(st_t=st_t))
