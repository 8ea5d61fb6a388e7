"""Autotuner for the launch parameters of the library (lrp_set_param).

tune_solve: for a given coarse handle it times a short Parareal solve under each candidate
setting of the tridiagonal cluster split (CTAs per system, rows per chunk,
systems per thread, rows per chunk of the one-warp kernel) and of the
coarse-sweep slice (rows per CTA), using the library's
per-kernel CUDA-event timers, and leaves the fastest setting applied to the
context.  Results are cached in memory per (n, N, precision, device name).
tune_krylov: for a 2D (5-point stencil) operator it times one batched
backward-Euler step of the Krylov propagator under each CTA count per cluster
(the CG/BiCGStab block shape), in the precision the build will use.
Every candidate computes the same solution up to rounding; the tuner only
picks launch shapes.
"""
from __future__ import annotations

from typing import Dict, Iterable, Optional, Tuple

from . import api

_CACHE: Dict[Tuple, Dict[str, int]] = {}

# (tri_cluster, tri_chunk, tri_spt, tri_wchunk); all zeros = the library's own rule
TRI_CANDIDATES = ((0, 0, 0, 0), (0, 0, 0, 8), (0, 0, 0, 11), (0, 0, 0, 13), (0, 0, 0, 16),
                  (2, 16, 1, 0),
                  (2, 8, 2, 0), (4, 8, 2, 0), (4, 8, 1, 0), (1, 16, 1, 0))
SWEEP_CANDIDATES = (0, 256, 2048)


def _device_name(ctx: api.Context) -> str:
    try:
        import torch
        return torch.cuda.get_device_name(ctx.device)
    except Exception:
        return "cuda:%d" % ctx.device


def _apply(ctx: api.Context, params: Dict[str, int]):
    for k, v in params.items():
        ctx.set_param(k, v)


def tune_solve(ctx: api.Context, co: api.Coarse, u0, K: int = 6,
               tri: Iterable = TRI_CANDIDATES, sweep: Iterable = SWEEP_CANDIDATES,
               verbose: bool = False) -> Dict[str, int]:
    """Pick the launch parameters minimising the device time of K Parareal
    iterations (fine propagations + coarse sweeps) for this coarse handle."""
    key = (co.op.n, co.N, co.prec, _device_name(ctx))
    if key in _CACHE:
        _apply(ctx, _CACHE[key])
        return dict(_CACHE[key])
    best: Optional[Tuple[float, Dict[str, int]]] = None
    for (tc, m, spt, wm) in tri:
        for sc in sweep:
            params = {"tri_cluster": tc, "tri_chunk": m, "tri_spt": spt, "tri_wchunk": wm,
                      "sweep_rows": sc}
            try:
                _apply(ctx, params)
                api.parareal_solve(ctx, co, u0, K=2, bounds=False)        # plans, warm-up
                ctx.set_kernel_timing(True)
                ctx.reset_kernel_time()
                api.parareal_solve(ctx, co, u0, K=K, bounds=False)
                t = sum(ctx.kernel_time(f)[1] for f in ("propagate_f64", "propagate_f32", "sweep"))
            except Exception:
                continue
            finally:
                ctx.set_kernel_timing(False)
            if verbose:
                print("autotune", params, "%.3f ms" % t)
            if best is None or t < best[0]:
                best = (t, params)
    if best is None:
        params = {"tri_cluster": 0, "tri_chunk": 0, "tri_spt": 0, "tri_wchunk": 0, "sweep_rows": 0}
    else:
        params = best[1]
    _apply(ctx, params)
    _CACHE[key] = dict(params)
    return dict(params)


KRYLOV_CANDIDATES = (0, 16, 8, 4)


def tune_krylov(ctx: api.Context, op: api.Operator, dt: float, nsys: int = 32, prec: str = "mixed",
                candidates: Iterable = KRYLOV_CANDIDATES, verbose: bool = False) -> Dict[str, int]:
    """Pick the CTAs per cluster of the 2D Krylov propagator (krylov_cluster)
    minimising the device time per Krylov iteration of one backward-Euler
    step of nsys seeded vectors; leaves the choice applied to the context."""
    import numpy as np
    key = ("krylov", op.n, nsys, prec, _device_name(ctx))
    if key in _CACHE:
        _apply(ctx, _CACHE[key])
        return dict(_CACHE[key])
    X = np.random.default_rng(0).standard_normal((nsys, op.n))
    fam = "propagate_f64" if prec == "f64" else "propagate_f32"
    best: Optional[Tuple[float, Dict[str, int]]] = None
    for cs in candidates:
        params = {"krylov_cluster": cs}
        try:
            _apply(ctx, params)
            api.propagate(ctx, op, dt, 1, X, prec=prec)                   # plans, warm-up
            it0 = op.krylov_iterations()
            ctx.set_kernel_timing(True)
            ctx.reset_kernel_time()
            api.propagate(ctx, op, dt, 1, X, prec=prec)
            t = ctx.kernel_time(fam)[1] / max(1, op.krylov_iterations() - it0)
        except Exception:
            continue
        finally:
            ctx.set_kernel_timing(False)
        if verbose:
            print("autotune", params, "%.3f us per iteration" % (t * 1e3))
        if best is None or t < best[0]:
            best = (t, params)
    params = {"krylov_cluster": 0} if best is None else best[1]
    _apply(ctx, params)
    _CACHE[key] = dict(params)
    return dict(params)
