"""Python wrappers over the C ABI of include/lrp.h (argument marshalling only).

Arrays: numpy (host) or torch tensors (host or CUDA), float64, C-contiguous.
Outputs are numpy arrays unless an `out` array is passed.
"""
from __future__ import annotations

import ctypes
from typing import Optional

import numpy as np

from . import _native as nat
from ._native import PREC_F64, PREC_MIXED, check, ptr


def _prec(p) -> int:
    if p in (PREC_F64, "f64", "fp64", None):
        return PREC_F64
    if p in (PREC_MIXED, "mixed", "f32", "fp32"):
        return PREC_MIXED
    raise ValueError("precision must be 'f64' or 'mixed'")


class Context:
    """A library context on one CUDA device (lrp_create)."""

    def __init__(self, device: int = 0, hbm_budget: int = 0):
        self.lib = nat.load()
        h = ctypes.c_void_p()
        st = self.lib.lrp_create(ctypes.byref(h), device, hbm_budget)
        if st != nat.LRP_OK:
            raise nat.LrpError(st, "lrp_create failed (is a CUDA device visible?)")
        self.h = h
        self.device = device

    def close(self):
        if getattr(self, "h", None) and not nat.exiting():
            self.lib.lrp_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def stream(self) -> int:
        return self.lib.lrp_get_stream(self.h) or 0

    def set_stream(self, stream_handle: Optional[int]):
        check(self.lib.lrp_set_stream(self.h, stream_handle), self.h)

    def synchronize(self):
        check(self.lib.lrp_synchronize(self.h), self.h)

    def bytes_in_use(self) -> int:
        return self.lib.lrp_bytes_in_use(self.h)

    def launch_count(self) -> int:
        return self.lib.lrp_launch_count(self.h)

    def set_param(self, name: str, value: int):
        check(self.lib.lrp_set_param(self.h, name.encode(), int(value)), self.h)

    def get_param(self, name: str) -> int:
        v = ctypes.c_int()
        check(self.lib.lrp_get_param(self.h, name.encode(), ctypes.byref(v)), self.h)
        return v.value

    def set_kernel_timing(self, on: bool):
        check(self.lib.lrp_set_kernel_timing(self.h, int(on)), self.h)

    def kernel_time(self, family: str):
        nl = ctypes.c_int()
        ms = ctypes.c_double()
        check(self.lib.lrp_kernel_time(self.h, family.encode(), ctypes.byref(nl), ctypes.byref(ms)),
              self.h)
        return nl.value, ms.value

    def reset_kernel_time(self):
        check(self.lib.lrp_reset_kernel_time(self.h), self.h)

    def last_error(self) -> str:
        return (self.lib.lrp_last_error(self.h) or b"").decode()


class Operator:
    """A semi-discretisation A of u_t = -A u + f held on the device."""

    def __init__(self, ctx: Context, handle, n: int, kind: str):
        self.ctx, self.h, self.n, self.kind = ctx, handle, n, kind

    @classmethod
    def tridiag(cls, ctx: Context, lo, di, up) -> "Operator":
        lo, di, up = (np.ascontiguousarray(a, dtype=np.float64) for a in (lo, di, up))
        h = ctypes.c_void_p()
        check(ctx.lib.lrp_operator_tridiag(ctx.h, di.shape[0], ptr(lo), ptr(di), ptr(up),
                                           ctypes.byref(h)), ctx.h)
        return cls(ctx, h, di.shape[0], "tridiag")

    @classmethod
    def tridiag_td(cls, ctx: Context, lo_t, di_t, up_t, stepper: str = "be") -> "Operator":
        """Time-dependent tridiagonal operator: (nJ, n) arrays, row J = A(t_{J+1});
        with an SDIRK stepper (2 nJ, n) arrays, row 2J + s = A(t_J + c_s dt)."""
        lo, di, up = (np.ascontiguousarray(a, dtype=np.float64) for a in (lo_t, di_t, up_t))
        h = ctypes.c_void_p()
        if stepper == "be":
            check(ctx.lib.lrp_operator_tridiag_td(ctx.h, di.shape[1], di.shape[0], ptr(lo),
                                                  ptr(di), ptr(up), ctypes.byref(h)), ctx.h)
        else:
            if di.shape[0] % 2:
                raise ValueError("SDIRK operators take two coefficient rows per fine step")
            check(ctx.lib.lrp_operator_tridiag_td_sdirk(ctx.h, di.shape[1], di.shape[0] // 2,
                                                        nat.STEPPERS[stepper], ptr(lo), ptr(di),
                                                        ptr(up), ctypes.byref(h)), ctx.h)
        op = cls(ctx, h, di.shape[1], "tridiag_td")
        op.stepper = stepper
        return op

    @classmethod
    def stencil5(cls, ctx: Context, mx: int, my: int, st: dict) -> "Operator":
        arr = [np.ascontiguousarray(st[k], dtype=np.float64) for k in ("C", "W", "E", "S", "N")]
        h = ctypes.c_void_p()
        check(ctx.lib.lrp_operator_stencil5(ctx.h, mx, my, *[ptr(a) for a in arr],
                                            ctypes.byref(h)), ctx.h)
        return cls(ctx, h, mx * my, "stencil5")

    @classmethod
    def stencil5_td(cls, ctx: Context, mx: int, my: int, st_t: dict,
                    stepper: str = "be") -> "Operator":
        """Time-dependent 5-point operator: st_t["C"], ... are (nJ, mx*my),
        row J the stencil of A(t_{J+1}); with an SDIRK stepper (2 nJ, mx*my),
        row 2J + s the stencil at stage time s of step J."""
        arr = [np.ascontiguousarray(st_t[k], dtype=np.float64) for k in ("C", "W", "E", "S", "N")]
        rows = arr[0].shape[0]
        if any(a.shape != (rows, mx * my) for a in arr):
            raise ValueError("stencil arrays must be (rows, mx*my)")
        h = ctypes.c_void_p()
        if stepper == "be":
            check(ctx.lib.lrp_operator_stencil5_td(ctx.h, mx, my, rows, *[ptr(a) for a in arr],
                                                   ctypes.byref(h)), ctx.h)
        else:
            if rows % 2:
                raise ValueError("SDIRK operators take two coefficient rows per fine step")
            check(ctx.lib.lrp_operator_stencil5_td_sdirk(ctx.h, mx, my, rows // 2,
                                                         nat.STEPPERS[stepper],
                                                         *[ptr(a) for a in arr],
                                                         ctypes.byref(h)), ctx.h)
        op = cls(ctx, h, mx * my, "stencil5_td")
        op.stepper = stepper
        return op

    @classmethod
    def from_problem(cls, ctx: Context, P) -> "Operator":
        if P.kind == "tridiag":
            return cls.tridiag(ctx, P.lo, P.di, P.up)
        return cls.stencil5(ctx, P.mx, P.my, P.st)

    def set_stepper(self, stepper: str = "be"):
        """Fine time stepper: "be" (backward Euler), "sdirk2", "sdirk2l".  With
        an SDIRK stepper a source takes two samples per fine step (its stage
        times): c arrays gain an axis of length 2 before the last."""
        check(self.ctx.lib.lrp_operator_set_stepper(self.h, nat.STEPPERS[stepper]), self.ctx.h)
        self.stepper = stepper

    def krylov_iterations(self) -> int:
        return int(self.ctx.lib.lrp_operator_krylov_iterations(self.h))

    def set_krylov(self, rtol_f64: float = 1e-12, rtol_f32: float = 1e-6, max_iter: int = 20000):
        check(self.ctx.lib.lrp_operator_set_krylov(self.h, rtol_f64, rtol_f32, max_iter), self.ctx.h)

    def close(self):
        if getattr(self, "h", None) and not nat.exiting():
            self.ctx.lib.lrp_operator_free(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _as_c(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return np.ascontiguousarray(a, dtype=np.float64)
    return a


def _source_samples(op) -> int:
    """Source samples per fine step: two for the SDIRK steppers."""
    return 1 if getattr(op, "stepper", "be") == "be" else 2


def _check_source(c, count: int):
    if isinstance(c, np.ndarray) and c.size != count:
        raise ValueError("source coefficients: %d values given, %d expected" % (c.size, count))


def propagate(ctx: Context, op: Operator, dt: float, M: int, X, adjoint: bool = False,
              g=None, c=None, prec="f64", out=None):
    """M fine steps on each row of X (nvec, n) (lrp_propagate).
    c: (nvec, M, Q) source samples per row, or (M, Q) shared; with an SDIRK
    stepper (nvec, M, 2, Q) or (M, 2, Q), the stage samples of every step."""
    X = _as_c(X)
    squeeze = False
    if isinstance(X, np.ndarray) and X.ndim == 1:
        X = X[None, :]
        squeeze = True
    nvec = X.shape[0]
    Q = 0
    if g is not None:
        g = np.ascontiguousarray(np.atleast_2d(g), dtype=np.float64) if isinstance(g, np.ndarray) else g
        Q = g.shape[0]
        c = _as_c(c)
        sps = _source_samples(op)
        if isinstance(c, np.ndarray) and c.ndim == (2 if sps == 1 else 3):
            c = np.ascontiguousarray(np.broadcast_to(c, (nvec,) + c.shape))
        _check_source(c, nvec * M * sps * Q)
    if out is None:
        out = np.empty((nvec, op.n))
    check(ctx.lib.lrp_propagate(ctx.h, op.h, float(dt), int(M), int(adjoint), nvec, ptr(X),
                                ptr(out), Q, ptr(g), ptr(c), _prec(prec)), ctx.h)
    return out[0] if squeeze else out


def gaussian(ctx: Context, seed: int, interval: int, ncol: int, n: int, prec="f64", out=None):
    """The sketch vectors omega_{interval, c}, c < ncol, as the build draws them."""
    if out is None:
        out = np.empty((ncol, n))
    check(ctx.lib.lrp_gaussian(ctx.h, int(seed), int(interval), int(ncol), int(n), _prec(prec),
                               ptr(out)), ctx.h)
    return out


class Coarse:
    """Low-rank coarse solvers G_i' = U_i diag(S_i) V_i^T of all intervals."""

    def __init__(self, ctx: Context, op: Operator, dt: float, M: int, N: int, rank: int,
                 oversample: int, seed: int = 0, prec="f64", independent_adjoint: bool = False):
        """independent_adjoint: the two-sided sketch variant (F'^* on independent
        random vectors; lrp_build_coarse_ex with LRP_BUILD_INDEPENDENT_ADJOINT)."""
        self.ctx, self.op = ctx, op
        self.dt, self.M, self.N, self.R, self.p = dt, M, N, rank, oversample
        self.prec = _prec(prec)
        h = ctypes.c_void_p()
        flags = nat.LRP_BUILD_INDEPENDENT_ADJOINT if independent_adjoint else 0
        check(ctx.lib.lrp_build_coarse_ex(ctx.h, op.h, float(dt), int(M), int(N), int(rank),
                                          int(oversample), int(seed), self.prec, flags,
                                          ctypes.byref(h)), ctx.h)
        self.h = h

    def info(self) -> dict:
        N, ell = self.N, self.R + self.p
        Ri = np.zeros(N, dtype=np.int32)
        rw = np.zeros(N, dtype=np.int32)
        rv = np.zeros(N, dtype=np.int32)
        sig = np.zeros((N, ell))
        d = ctypes.c_double()
        e = ctypes.c_double()
        check(self.ctx.lib.lrp_coarse_info(self.h, Ri.ctypes.data, rw.ctypes.data, rv.ctypes.data,
                                           sig.ctypes.data, ctypes.addressof(d),
                                           ctypes.addressof(e)), self.ctx.h)
        return dict(R=Ri, rank_w=rw, rank_v=rv, sigma=sig, delta=d.value, eps=e.value)

    def orth_method(self) -> dict:
        """Intervals whose bases (rSVD steps 2 and 4) came from CholeskyQR2
        on the tensor cores; the rest used Gram-Schmidt twice."""
        w = ctypes.c_int()
        v = ctypes.c_int()
        check(self.ctx.lib.lrp_coarse_orth_method(self.h, ctypes.addressof(w), ctypes.addressof(v)),
              self.ctx.h)
        return dict(tc_w=w.value, tc_v=v.value)

    def factors(self, i: int):
        Ri = int(self.info()["R"][i])
        U = np.zeros((Ri, self.op.n))
        V = np.zeros((Ri, self.op.n))
        S = np.zeros(Ri)
        check(self.ctx.lib.lrp_coarse_factors(self.h, i, U.ctypes.data, S.ctypes.data,
                                              V.ctypes.data), self.ctx.h)
        return U, S, V

    def save(self, path: str):
        """Checkpoint the factors and metadata to an .npz file."""
        N, n, ell = self.N, self.op.n, self.R + self.p
        Rm = max(self.R, 1)
        mi = np.zeros(6, dtype=np.int32)
        md = np.zeros(3)
        seed = ctypes.c_uint64()
        Ri, rw, rv = (np.zeros(N, dtype=np.int32) for _ in range(3))
        sig = np.zeros((N, ell))
        U = np.zeros((N, Rm, n))
        V = np.zeros((N, Rm, n))
        S = np.zeros((N, Rm))
        check(self.ctx.lib.lrp_coarse_export(self.h, mi.ctypes.data, md.ctypes.data, ctypes.byref(seed),
                                             Ri.ctypes.data, rw.ctypes.data, rv.ctypes.data,
                                             sig.ctypes.data, U.ctypes.data, S.ctypes.data,
                                             V.ctypes.data), self.ctx.h)
        np.savez(path, meta_i=mi, meta_d=md, seed=np.uint64(seed.value), Ri=Ri, rank_w=rw,
                 rank_v=rv, sigma=sig, U=U, S=S, V=V)

    @classmethod
    def load(cls, ctx: Context, op: Operator, path: str) -> "Coarse":
        z = np.load(path)
        mi = np.ascontiguousarray(z["meta_i"], dtype=np.int32)
        md = np.ascontiguousarray(z["meta_d"], dtype=np.float64)
        arrs = {k: np.ascontiguousarray(z[k]) for k in ("Ri", "rank_w", "rank_v", "sigma", "U", "S", "V")}
        h = ctypes.c_void_p()
        check(ctx.lib.lrp_coarse_import(ctx.h, op.h, mi.ctypes.data, md.ctypes.data, int(z["seed"]),
                                        arrs["Ri"].ctypes.data, arrs["rank_w"].ctypes.data,
                                        arrs["rank_v"].ctypes.data, arrs["sigma"].ctypes.data,
                                        arrs["U"].ctypes.data, arrs["S"].ctypes.data,
                                        arrs["V"].ctypes.data, ctypes.byref(h)), ctx.h)
        c = cls.__new__(cls)
        c.ctx, c.op = ctx, op
        c.M, c.N, c.R, c.p = int(mi[0]), int(mi[1]), int(mi[2]), int(mi[3])
        c.dt = float(md[0])
        c.prec = int(mi[5])
        c.h = h
        return c

    def close(self):
        if getattr(self, "h", None) and not nat.exiting():
            self.ctx.lib.lrp_coarse_free(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def build_coarse_batch(ctx: Context, ops, dt: float, M: int, N: int, rank: int, oversample: int,
                       seed: int = 0, prec="f64"):
    """Coarse solvers of many 2D operators in one graph-captured build
    (lrp_build_coarse_batch).  Returns a list of Coarse handles."""
    cnt = len(ops)
    harr = (ctypes.c_void_p * cnt)(*[o.h.value for o in ops])
    outs = (ctypes.c_void_p * cnt)()
    check(ctx.lib.lrp_build_coarse_batch(ctx.h, cnt, ctypes.cast(harr, ctypes.c_void_p), float(dt),
                                         int(M), int(N), int(rank), int(oversample), int(seed),
                                         _prec(prec), ctypes.cast(outs, ctypes.c_void_p)), ctx.h)
    res = []
    for i, o in enumerate(ops):
        c = Coarse.__new__(Coarse)
        c.ctx, c.op = ctx, o
        c.dt, c.M, c.N, c.R, c.p = dt, M, N, rank, oversample
        c.prec = _prec(prec)
        c.h = ctypes.c_void_p(outs[i])
        res.append(c)
    return res


def parareal_solve_batch(ctx: Context, cos, u0s, K: Optional[int] = None, tol: float = 0.0):
    """Parareal for many 2D problems at once (lrp_parareal_solve_batch)."""
    cnt = len(cos)
    u0s = [np.ascontiguousarray(u, dtype=np.float64) for u in u0s]
    outs = [np.empty((co.N + 1, co.op.n)) for co in cos]
    harr = (ctypes.c_void_p * cnt)(*[co.h.value for co in cos])
    uarr = (ctypes.c_void_p * cnt)(*[u.ctypes.data for u in u0s])
    oarr = (ctypes.c_void_p * cnt)(*[o.ctypes.data for o in outs])
    kd = np.zeros(cnt, dtype=np.int32)
    st = ctx.lib.lrp_parareal_solve_batch(ctx.h, cnt, ctypes.cast(harr, ctypes.c_void_p),
                                          ctypes.cast(uarr, ctypes.c_void_p),
                                          cos[0].N if K is None else int(K), float(tol),
                                          ctypes.cast(oarr, ctypes.c_void_p), kd.ctypes.data)
    check(st, ctx.h)
    return outs, kd


def parareal_solve(ctx: Context, co: Coarse, u0, g=None, c=None, K: Optional[int] = None,
                   tol: float = 0.0, out=None, bounds: bool = True, allow_notconv: bool = True):
    """Parareal iterations (lrp_parareal_solve).  Returns (u (N+1, n), info)."""
    N, n = co.N, co.op.n
    Kmax = N if K is None else int(K)
    u0 = _as_c(u0)
    Q = 0
    if g is not None:
        g = np.ascontiguousarray(np.atleast_2d(g), dtype=np.float64) if isinstance(g, np.ndarray) else g
        Q = g.shape[0]
        c = _as_c(c)
        _check_source(c, N * co.M * _source_samples(co.op) * Q)
    if out is None:
        out = np.empty((N + 1, n))
    bnd = np.zeros((max(Kmax, 1), N + 1)) if bounds else None
    kd = ctypes.c_int()
    stats = nat.SolveStats()
    ok = (nat.LRP_OK, nat.LRP_ENOTCONV) if allow_notconv else (nat.LRP_OK,)
    st = check(ctx.lib.lrp_parareal_solve(ctx.h, co.h, ptr(u0), Q, ptr(g), ptr(c), Kmax,
                                          float(tol), ptr(out),
                                          bnd.ctypes.data if bnd is not None else None,
                                          ctypes.byref(kd), ctypes.byref(stats)), ctx.h, ok)
    info = dict(k_done=kd.value, fine_evals=stats.fine_evals, converged=bool(stats.converged),
                final_bound=stats.final_bound, scale=stats.scale, device_ms=stats.device_ms,
                status=st, bounds=bnd[:kd.value] if bnd is not None else None)
    return out, info


def parareal_solve_classical(ctx: Context, op: Operator, dt: float, M: int, N: int, u0, g=None,
                             c=None, K: Optional[int] = None, tol: float = 0.0, out=None,
                             allow_notconv: bool = True):
    """Classical Parareal with one backward-Euler coarse step per interval
    (lrp_parareal_solve_classical).  Returns (u (N+1, n), info)."""
    n = op.n
    Kmax = N if K is None else int(K)
    u0 = _as_c(u0)
    Q = 0
    if g is not None:
        g = np.ascontiguousarray(np.atleast_2d(g), dtype=np.float64) if isinstance(g, np.ndarray) else g
        Q = g.shape[0]
        c = _as_c(c)
    if out is None:
        out = np.empty((N + 1, n))
    inc = np.zeros(max(Kmax, 1))
    kd = ctypes.c_int()
    stats = nat.SolveStats()
    ok = (nat.LRP_OK, nat.LRP_ENOTCONV) if allow_notconv else (nat.LRP_OK,)
    st = check(ctx.lib.lrp_parareal_solve_classical(ctx.h, op.h, float(dt), int(M), int(N), ptr(u0), Q,
                                                    ptr(g), ptr(c), Kmax, float(tol), ptr(out),
                                                    inc.ctypes.data, ctypes.byref(kd),
                                                    ctypes.byref(stats)), ctx.h, ok)
    info = dict(k_done=kd.value, fine_evals=stats.fine_evals, converged=bool(stats.converged),
                increments=inc[:kd.value], device_ms=stats.device_ms, status=st)
    return out, info


def fine_solution(ctx: Context, op: Operator, dt: float, M: int, N: int, u0, g=None, c=None,
                  out=None):
    """Sequential fine solution u_{i+1} = F_i u_i on the device, (N+1, n)."""
    u0 = _as_c(u0)
    Q = 0
    if g is not None:
        g = np.ascontiguousarray(np.atleast_2d(g), dtype=np.float64) if isinstance(g, np.ndarray) else g
        Q = g.shape[0]
        c = _as_c(c)
        _check_source(c, N * M * _source_samples(op) * Q)
    if out is None:
        out = np.empty((N + 1, op.n))
    check(ctx.lib.lrp_fine_solution(ctx.h, op.h, float(dt), int(M), int(N), ptr(u0), Q, ptr(g),
                                    ptr(c), ptr(out)), ctx.h)
    return out


class Server:
    """Continuous-batching server over resident coarse solvers (lrp_server_*)."""

    def __init__(self, ctx: Context, max_slots: int = 64, max_terms: int = 4, hbm_budget: int = 0):
        self.ctx = ctx
        self.lib = ctx.lib
        h = ctypes.c_void_p()
        check(self.lib.lrp_server_create(ctx.h, int(max_slots), int(max_terms), int(hbm_budget),
                                         ctypes.byref(h)), ctx.h)
        self.h = h
        self._shape = {}

    def submit(self, co: Coarse, u0, g=None, c=None, K: Optional[int] = None, tol: float = 1e-8) -> int:
        u0 = np.ascontiguousarray(u0, dtype=np.float64)
        Q = 0
        if g is not None:
            g = np.ascontiguousarray(np.atleast_2d(g), dtype=np.float64)
            c = np.ascontiguousarray(c, dtype=np.float64)
            Q = g.shape[0]
        t = ctypes.c_uint64()
        st = self.lib.lrp_server_submit(self.h, co.h, u0.ctypes.data, Q,
                                        g.ctypes.data if g is not None else None,
                                        c.ctypes.data if c is not None else None,
                                        co.N if K is None else int(K), float(tol), ctypes.byref(t))
        if st != nat.LRP_OK:
            raise nat.LrpError(st, "submit failed")
        self._shape[t.value] = (co.N + 1, co.op.n)
        return t.value

    def _info(self, inf: "nat.RequestInfo", st: int) -> dict:
        return dict(k_done=inf.k_done, status=inf.status, final_bound=inf.final_bound,
                    scale=inf.scale, queue_ms=inf.queue_ms, latency_ms=inf.latency_ms,
                    converged=(st == nat.LRP_OK))

    def poll(self, ticket: int):
        """(done, u, info); u is None while the request runs."""
        u = np.empty(self._shape[ticket])
        inf = nat.RequestInfo()
        st = self.lib.lrp_server_poll(self.h, ticket, u.ctypes.data, ctypes.byref(inf))
        if st == nat.LRP_PENDING:
            return False, None, None
        self._shape.pop(ticket, None)
        if st not in (nat.LRP_OK, nat.LRP_ENOTCONV):
            raise nat.LrpError(st, "served request failed")
        return True, u, self._info(inf, st)

    def wait(self, ticket: int, timeout: float = 0.0):
        u = np.empty(self._shape[ticket])
        inf = nat.RequestInfo()
        st = self.lib.lrp_server_wait(self.h, ticket, float(timeout), u.ctypes.data, ctypes.byref(inf))
        self._shape.pop(ticket, None)
        if st not in (nat.LRP_OK, nat.LRP_ENOTCONV):
            raise nat.LrpError(st, "served request failed")
        return u, self._info(inf, st)

    def set_latency_target(self, co: Coarse, target_ms: float):
        """Turn away (LrpError LRP_EBUSY at submit) requests on co whose estimated
        latency exceeds target_ms (0: no target)."""
        check(self.lib.lrp_server_set_latency_target(self.h, co.h, float(target_ms)))

    def estimate_ms(self, co: Coarse) -> float:
        v = ctypes.c_double()
        check(self.lib.lrp_server_estimate(self.h, co.h, ctypes.byref(v)))
        return v.value

    def stats(self) -> dict:
        s = nat.ServerStats()
        check(self.lib.lrp_server_stats_get(self.h, ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in s._fields_}

    def close(self):
        if getattr(self, "h", None) and not nat.exiting():
            self.lib.lrp_server_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
