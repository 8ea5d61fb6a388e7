"""Continuous-batching server: requests with new u0 and new sources on
resident coarse solvers of two operators (the 1D heat and 1D advection-
diffusion-reaction problems).  Each served result equals the direct solve of
the same request (alone) within 1e-12 relative, whatever else shares the
launches, and meets its tolerance against the oracle's fine solution."""
import threading
import time

import numpy as np
import pytest

from paper_2508_08873_gb300 import api, workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    ctx = api.Context(0)
    Ph = W.heat1d()
    Pa = W.adr1d(n=1023, N=16, M=64, R=8, p=4)
    oph = api.Operator.tridiag(ctx, Ph.lo, Ph.di, Ph.up)
    opa = api.Operator.tridiag(ctx, Pa.lo, Pa.di, Pa.up)
    coh = api.Coarse(ctx, oph, Ph.dt, Ph.M, Ph.N, Ph.R, Ph.p, 0, prec="mixed")
    coa = api.Coarse(ctx, opa, Pa.dt, Pa.M, Pa.N, Pa.R, Pa.p, 0, prec="mixed")
    return ctx, (Ph, oph, coh), (Pa, opa, coa)


def _request(P, k):
    u0, g, c = W.serving_request(P.n, P.N, P.M, P.dt, k)
    return u0, g, c


def test_served_equals_direct_alone_and_in_mix(setup, orc):
    ctx, H, A = setup
    srv = api.Server(ctx, max_slots=8, max_terms=4)
    reqs = []
    for k in range(10):
        P, op, co = (H, A)[k % 2]
        u0, g, c = _request(P, k)
        t = srv.submit(co, u0, g, c, K=P.N, tol=1e-10)
        reqs.append((t, P, op, co, u0, g, c))
    for t, P, op, co, u0, g, c in reqs:
        u, info = srv.wait(t, timeout=120)
        direct, dinfo = api.parareal_solve(ctx, co, u0, g, c, K=P.N, tol=1e-10)
        assert info["k_done"] == dinfo["k_done"]
        assert np.linalg.norm(u - direct) <= 1e-12 * np.linalg.norm(direct)
        ref = orc.sequential_fine(orc.Tridiag(P.lo, P.di, P.up), P.dt, P.M, P.N, u0, g, c)
        assert orc.rel_err(u, ref) <= 1e-9
        assert info["latency_ms"] >= info["queue_ms"] >= 0
    # the same request alone on a fresh server
    t0, P, op, co, u0, g, c = reqs[3]
    srv2 = api.Server(ctx, max_slots=8, max_terms=4)
    u_alone, _ = srv2.wait(srv2.submit(co, u0, g, c, K=P.N, tol=1e-10), timeout=60)
    direct, _ = api.parareal_solve(ctx, co, u0, g, c, K=P.N, tol=1e-10)
    assert np.linalg.norm(u_alone - direct) <= 1e-12 * np.linalg.norm(direct)
    st = srv.stats()
    assert st["completed"] == 10 and st["error"] == 0
    srv.close()
    srv2.close()


def test_admission_queue_and_poll(setup):
    """More requests than slots: the rest wait in the queue and are admitted
    as slots free up; poll is non-blocking."""
    ctx, H, A = setup
    P, op, co = A
    srv = api.Server(ctx, max_slots=2, max_terms=4)
    tickets = [srv.submit(co, *_request(P, 100 + k), K=3, tol=0.0) for k in range(7)]
    done = {}
    t_end = time.time() + 120
    while len(done) < len(tickets) and time.time() < t_end:
        for t in tickets:
            if t not in done:
                ok, u, info = srv.poll(t)
                if ok:
                    done[t] = info
        time.sleep(0.001)
    assert len(done) == 7
    assert all(d["k_done"] == 3 for d in done.values())
    assert max(d["queue_ms"] for d in done.values()) > 0
    srv.close()


def test_concurrent_submitters(setup):
    ctx, H, A = setup
    P, op, co = H
    srv = api.Server(ctx, max_slots=16, max_terms=4)
    out = {}

    def client(k):
        u0, g, c = _request(P, 200 + k)
        t = srv.submit(co, u0, g, c, K=P.N, tol=1e-10)
        out[k] = srv.wait(t, timeout=120)

    th = [threading.Thread(target=client, args=(k,)) for k in range(6)]
    for x in th:
        x.start()
    for x in th:
        x.join()
    assert len(out) == 6 and all(v[1]["converged"] for v in out.values())
    srv.close()


def test_latency_target_turns_requests_away(setup):
    """Admission control: with a latency target below the group's measured
    service time a new request is turned away with LRP_EBUSY; without a
    target (0) or with a generous one it is admitted."""
    from paper_2508_08873_gb300 import _native
    ctx, H, A = setup
    P, op, co = A
    srv = api.Server(ctx, max_slots=4, max_terms=4)
    assert srv.estimate_ms(co) == 0.0                      # no history: admit
    for k in range(3):
        srv.wait(srv.submit(co, *_request(P, 300 + k), K=3, tol=0.0), timeout=120)
    est = srv.estimate_ms(co)
    assert est > 0.0
    srv.set_latency_target(co, est * 1e-3)
    with pytest.raises(_native.LrpError) as ei:
        srv.submit(co, *_request(P, 310), K=3, tol=0.0)
    assert ei.value.status == _native.LRP_EBUSY
    srv.set_latency_target(co, 0.0)
    u, info = srv.wait(srv.submit(co, *_request(P, 311), K=3, tol=0.0), timeout=120)
    assert info["k_done"] == 3
    srv.set_latency_target(co, 1e9)
    u, info = srv.wait(srv.submit(co, *_request(P, 312), K=3, tol=0.0), timeout=120)
    assert info["k_done"] == 3
    srv.close()


def test_short_requests_not_held_behind_long_ones(setup, orc):
    """Each coarse handle is served by its own worker on its own stream (the
    cheaper handle's at a higher priority): heat1d requests submitted behind
    a burst of longer advection requests finish first and stay correct."""
    ctx, H, A = setup
    srv = api.Server(ctx, max_slots=64, max_terms=4)
    Pa, opa, coa = A
    Ph, oph, coh = H
    long_t = [srv.submit(coa, *_request(Pa, 400 + k), K=Pa.N, tol=1e-12) for k in range(24)]
    short = []
    for k in range(6):
        u0, g, c = _request(Ph, 500 + k)
        short.append((srv.submit(coh, u0, g, c, K=Ph.N, tol=1e-10), u0, g, c))
    short_lat = []
    for t, u0, g, c in short:
        u, info = srv.wait(t, timeout=120)
        short_lat.append(info["latency_ms"])
        direct, _ = api.parareal_solve(ctx, coh, u0, g, c, K=Ph.N, tol=1e-10)
        assert np.linalg.norm(u - direct) <= 1e-12 * np.linalg.norm(direct)
    long_lat = [srv.wait(t, timeout=300)[1]["latency_ms"] for t in long_t]
    assert max(short_lat) < np.median(long_lat), (short_lat, np.median(long_lat))
    srv.close()


def test_served_2d_with_concurrent_direct_solves():
    """2D handles (symmetric diffusion: FP64 steps by iterative refinement;
    upwind advection: FP32 BiCGStab corrections) served while the caller's
    context runs direct solves and propagations of other sizes with the same
    operators: the server's contexts and the caller's keep their own scratch,
    so every served result equals its direct solve."""
    ctx = api.Context(0)
    probs = [W.diff2d(m=31, N=6, M=4, R=5, p=3, T=6 * 4 / 2048), W.adv2d(0, m=31, N=6, M=4, R=5, p=3)]
    ops, cos = [], []
    for P in probs:
        op = api.Operator.stencil5(ctx, P.mx, P.my, P.st)
        ops.append(op)
        cos.append(api.Coarse(ctx, op, P.dt, P.M, P.N, P.R, P.p, P.seed, prec="mixed"))
    srv = api.Server(ctx, max_slots=8, max_terms=2)
    reqs = []
    for k in range(6):
        P, co = probs[k % 2], cos[k % 2]
        u0, g, c = W.serving_request(P.n, P.N, P.M, P.dt, 900 + k)
        reqs.append((srv.submit(co, u0, g[:2], c[:, :2], K=P.N, tol=1e-8), P, co, u0, g[:2], c[:, :2]))
    # meanwhile, direct work on the same operators with other batch sizes
    rng = np.random.default_rng(5)
    for P, op in zip(probs, ops):
        api.propagate(ctx, op, P.dt, 3, rng.standard_normal((17, P.n)))
    for t, P, co, u0, g, c in reqs:
        u, info = srv.wait(t, timeout=120)
        direct, _ = api.parareal_solve(ctx, co, u0, g, c, K=P.N, tol=1e-8)
        assert np.linalg.norm(u - direct) <= 1e-12 * np.linalg.norm(direct)
    srv.close()
