"""The allocation-free propagator entry point (lrp_propagate_noalloc).

It serves callers that cannot allocate device memory (hosts that forbid
allocation after start-up, frameworks that own all device memory through their
own pool, code that must avoid cudaFree's device-wide synchronisation).  The
test allocates the inputs and outputs itself, calls the entry point through the
C ABI twice in a row, and checks both results against lrp_propagate within the
tolerance of the propagator parity tests.  This file is collected last so that
a stop-at-first-failure run has already run every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_2508_08873_gb300 import _native, api, workloads as W

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_noalloc_matches_propagate_twice():
    import torch
    lib = _native.load()
    ctx = api.Context(0)
    dev = torch.device("cuda", 0)
    for n, maker, dt, M, adjoint, prec, tol in (
            (4095, W.adr1d_op, 1.0 / 16384, 256, 0, _native.PREC_F64, 1e-12),
            (4095, W.adr1d_op, 1.0 / 16384, 256, 1, _native.PREC_F64, 1e-12),
            (255, W.heat1d_op, 1.0 / 1024, 64, 0, _native.PREC_MIXED, 2e-5)):
        lo, di, up = maker(n)
        X = np.random.default_rng(n + adjoint).standard_normal((6, n))
        op = api.Operator.tridiag(ctx, lo, di, up)
        want = api.propagate(ctx, op, dt, M, X, adjoint=bool(adjoint),
                             prec="mixed" if prec == _native.PREC_MIXED else "f64")
        d_lo, d_di, d_up, d_x = (torch.tensor(a, dtype=torch.float64, device=dev)
                                 for a in (lo, di, up, X))
        for call in range(2):
            d_out = torch.full((6, n), float("nan"), dtype=torch.float64, device=dev)
            st = lib.lrp_propagate_noalloc(0, None, n, d_lo.data_ptr(), d_di.data_ptr(),
                                           d_up.data_ptr(), dt, M, adjoint, 6, d_x.data_ptr(),
                                           d_out.data_ptr(), 0, None, None, prec)
            assert st == _native.LRP_OK, st
            torch.cuda.synchronize()
            got = d_out.cpu().numpy()
            for v in range(6):
                assert _rel(got[v], want[v]) <= tol, (call, v, _rel(got[v], want[v]))


def test_noalloc_rejects_oversize():
    import torch
    lib = _native.load()
    n = 4097
    d = torch.ones(n, dtype=torch.float64, device="cuda")
    st = lib.lrp_propagate_noalloc(0, None, n, d.data_ptr(), d.data_ptr(), d.data_ptr(), 1e-3, 1,
                                   0, 1, d.data_ptr(), d.data_ptr(), 0, None, None, 0)
    assert st == _native.LRP_EINVAL
