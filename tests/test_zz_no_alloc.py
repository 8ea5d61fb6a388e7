"""The allocation-free propagator entry point (lrp_propagate_noalloc).

It serves callers that cannot allocate device memory (hosts that forbid
allocation after start-up, frameworks that own all device memory through their
own pool, code that must avoid cudaFree's device-wide synchronisation).  The
tests allocate the inputs and outputs themselves, call the entry point through
the C ABI twice in a row, and check the results against lrp_propagate and the
FP64 oracle within the tolerance of the propagator parity tests, with and
without a source term and initial values, at the largest size it takes, and
after a call that stopped on a zero pivot.  This file is collected last so that
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


def _dev(a, dev):
    import torch
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)


@pytest.mark.parametrize("n", [17, 511, 4096])
def test_noalloc_matches_oracle_with_source_and_zero_start(orc, n):
    """Against the FP64 oracle at the sizes that take different chunk lengths
    of the propagator (n = 17, 511, 4096 = the limit): a separable source
    (Q = 2, per-vector c) from zero initial values (x_in = NULL) and from
    given ones, twice in a row on the shared scratch."""
    import torch
    lib = _native.load()
    dev = torch.device("cuda", 0)
    lo, di, up = W.adr1d_op(n)
    dt, M, Q, nvec = 1.0 / 4096, 40, 2, 3
    rng = np.random.default_rng(n)
    g = rng.standard_normal((Q, n))
    c = rng.standard_normal((nvec, M, Q))
    X = rng.standard_normal((nvec, n))
    oop = orc.Tridiag(lo, di, up)
    want0 = orc.propagate(oop, dt, M, np.zeros((nvec, n)), g=g, cvals=c)
    wantx = orc.propagate(oop, dt, M, X, g=g, cvals=c)
    d_lo, d_di, d_up, d_x, d_g, d_c = (_dev(a, dev) for a in (lo, di, up, X, g, c))
    before = torch.cuda.current_device()
    for call in range(2):
        for x_ptr, want in ((None, want0), (d_x.data_ptr(), wantx)):
            d_out = torch.full((nvec, n), float("nan"), dtype=torch.float64, device=dev)
            st = lib.lrp_propagate_noalloc(0, None, n, d_lo.data_ptr(), d_di.data_ptr(),
                                           d_up.data_ptr(), dt, M, 0, nvec, x_ptr,
                                           d_out.data_ptr(), Q, d_g.data_ptr(), d_c.data_ptr(),
                                           _native.PREC_F64)
            assert st == _native.LRP_OK, st
            torch.cuda.synchronize()
            got = d_out.cpu().numpy()
            for v in range(nvec):
                assert _rel(got[v], want[v]) <= 1e-12, (call, v, _rel(got[v], want[v]))
    assert torch.cuda.current_device() == before


def test_noalloc_breakdown_then_good_call(orc):
    """A zero pivot (1 + dt a = 0 in one row) returns LRP_EBREAKDOWN; the next
    call on the same device, with a good operator, must not see the previous
    call's status word and matches the oracle."""
    import torch
    lib = _native.load()
    dev = torch.device("cuda", 0)
    n, dt = 300, 0.5
    lo, di, up = np.zeros(n), np.full(n, 3.0), np.zeros(n)
    di[n // 3] = -1.0 / dt
    X = np.ones((2, n))
    d_lo, d_di, d_up, d_x = (_dev(a, dev) for a in (lo, di, up, X))
    d_out = torch.zeros((2, n), dtype=torch.float64, device=dev)
    st = lib.lrp_propagate_noalloc(0, None, n, d_lo.data_ptr(), d_di.data_ptr(), d_up.data_ptr(),
                                   dt, 2, 0, 2, d_x.data_ptr(), d_out.data_ptr(), 0, None, None,
                                   _native.PREC_F64)
    assert st == _native.LRP_EBREAKDOWN
    lo, di, up = W.heat1d_op(n)
    d_lo, d_di, d_up = (_dev(a, dev) for a in (lo, di, up))
    st = lib.lrp_propagate_noalloc(0, None, n, d_lo.data_ptr(), d_di.data_ptr(), d_up.data_ptr(),
                                   1.0 / 1024, 8, 0, 2, d_x.data_ptr(), d_out.data_ptr(), 0, None,
                                   None, _native.PREC_F64)
    assert st == _native.LRP_OK
    torch.cuda.synchronize()
    want = orc.propagate(orc.Tridiag(lo, di, up), 1.0 / 1024, 8, X)
    got = d_out.cpu().numpy()
    assert max(_rel(got[v], want[v]) for v in range(2)) <= 1e-12
