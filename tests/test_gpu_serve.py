"""Request server: continuous batching with admission by device memory.
Every request's result equals the same request solved alone with nls_solve."""
import threading
import time

import numpy as np
import pytest

from paper_2403_16341_gb300 import inputs as I
from tests.parity import gpu_solve

pytestmark = pytest.mark.gpu

LS, TR, MIXED = 1, 2, 1 << 8


def run_stream(server, payloads, alg, gap_s=0.0):
    import paper_2403_16341_gb300 as nls
    bufs = []
    for b in payloads:
        p = np.ascontiguousarray(b.params)
        u = np.ascontiguousarray(b.u0.copy())
        st = np.zeros(b.batch, dtype=np.int32)
        it = np.zeros(b.batch, dtype=np.int32)
        bufs.append((p, u, st, it))
    tickets, errors = [], []

    def producer():
        try:
            for b, (p, u, st, it) in zip(payloads, bufs):
                ptr = lambda a: a.ctypes.data if a.size else 0
                tickets.append(nls.nls_server_submit(server, b.family, ptr(p), ptr(u), b.n,
                                                     b.batch, alg, 1e-10, 50, ptr(st), ptr(it)))
                if gap_s:
                    time.sleep(gap_s)
        except Exception as e:  # surfaced in the test thread below
            errors.append(e)

    th = threading.Thread(target=producer)
    th.start()
    th.join()
    assert not errors, errors
    assert len(tickets) == len(payloads)
    res = [nls.nls_server_wait(server, t) for t in tickets]
    return bufs, res


def request_bytes(b):
    al = lambda x: (x + 255) // 256 * 256
    return al(b.params.size * 8) + al(b.u0.size * 8) + al(b.batch * 8) + 4 * al(b.batch * 4)


HALLEY, NW = 5, 1 << 13


# Halley runs on the thread tiling for n <= 8 and on warp segments for 16 and
# 32; the NocedalWright flag rides along with the trust region
@pytest.mark.parametrize("alg", [LS | MIXED, TR, HALLEY | MIXED, TR | NW])
def test_mix_equals_alone(alg):
    import paper_2403_16341_gb300 as nls
    payloads = I.serving_payloads(120, max_batch=1024)
    srv = nls.nls_server_create(0, 0, 4)
    try:
        bufs, res = run_stream(srv, payloads, alg, gap_s=0.0005)
        stats = nls.nls_server_stats(srv)
    finally:
        nls.nls_server_destroy(srv)
    solver = nls.Solver(0)
    for b, (p, u, st, it), (solved, ts, td) in zip(payloads, bufs, res):
        alone = gpu_solve(solver, b, alg)
        np.testing.assert_array_equal(u, alone["u"])
        np.testing.assert_array_equal(st, alone["status"])
        np.testing.assert_array_equal(it, alone["iters"])
        assert solved == alone["solved"] == b.batch
        assert td >= ts
    solver.close()
    assert stats["completed"] == len(payloads) and stats["admitted"] == len(payloads)


def test_small_arena_forces_queueing():
    import paper_2403_16341_gb300 as nls
    payloads = I.serving_payloads(60, max_batch=4096)
    # room for the largest request and a little more: most requests must wait
    budget = int(1.5 * max(request_bytes(b) for b in payloads))
    srv = nls.nls_server_create(0, budget, 2)
    try:
        bufs, res = run_stream(srv, payloads, LS | MIXED)
        stats = nls.nls_server_stats(srv)
    finally:
        nls.nls_server_destroy(srv)
    assert stats["max_queue"] > 1
    for b, (p, u, st, it), (solved, ts, td) in zip(payloads, bufs, res):
        assert solved == b.batch and (st == 0).all()


def test_oversize_request_rejected():
    import paper_2403_16341_gb300 as nls
    b = I.cubic_batch(32, 4096, config_id=3)
    srv = nls.nls_server_create(0, 1 << 20, 1)
    try:
        u = b.u0.copy()
        with pytest.raises(nls.NlsError) as e:
            nls.nls_server_submit(srv, 0, b.params.ctypes.data, u.ctypes.data, 32, 4096, LS,
                                  1e-10, 50)
        assert e.value.code == nls.NLS_E_NOMEM
    finally:
        nls.nls_server_destroy(srv)


def test_requests_overlap_on_the_device():
    import paper_2403_16341_gb300 as nls
    payloads = I.serving_payloads(200, max_batch=4096, seed=1)
    srv = nls.nls_server_create(0, 0, 4)
    try:
        run_stream(srv, payloads, TR)
        stats = nls.nls_server_stats(srv)
    finally:
        nls.nls_server_destroy(srv)
    assert stats["max_inflight"] > 1 and stats["completed"] == 200


def test_failed_request_reports_error_and_frees_its_space():
    # Halley with the analytic-Jacobian flag is admitted (the server does not
    # know every algorithm's limits) and then refused by nls_solve after its
    # inputs were copied: its wait reports the error, its arena space comes
    # back once the stream has passed those copies, and the requests around
    # it are solved as usual
    import paper_2403_16341_gb300 as nls
    payloads = I.serving_payloads(12, max_batch=512, seed=2)
    srv = nls.nls_server_create(0, 0, 2)
    try:
        bad = payloads[0]
        pb, ub = np.ascontiguousarray(bad.params), bad.u0.copy()
        ptr = lambda a: a.ctypes.data if a.size else 0
        t_bad = nls.nls_server_submit(srv, bad.family, ptr(pb), ptr(ub), bad.n, bad.batch,
                                      HALLEY | (1 << 9), 1e-10, 50)
        bufs, res = run_stream(srv, payloads[1:], LS | MIXED)
        with pytest.raises(nls.NlsError) as e:
            nls.nls_server_wait(srv, t_bad)
        assert e.value.code == nls.NLS_E_CUDA and "failed" in str(e.value)
        for b, (p, u, st, it), (solved, ts, td) in zip(payloads[1:], bufs, res):
            assert solved == b.batch and (st == 0).all()
        deadline = time.time() + 5.0
        while True:
            stats = nls.nls_server_stats(srv)
            if stats["inflight"] == 0 or time.time() > deadline:
                break
            time.sleep(0.01)
        assert stats["inflight"] == 0 and stats["largest_free"] == stats["arena_bytes"]
    finally:
        nls.nls_server_destroy(srv)


def test_stage_times_are_consistent():
    # the timed wait reports where each request's time went: host stages in
    # order, device stages non-negative and within the request's lifetime
    import paper_2403_16341_gb300 as nls
    payloads = I.serving_payloads(40, max_batch=2048, seed=4)
    srv = nls.nls_server_create(0, 0, 2)
    try:
        bufs, tickets = [], []
        for b in payloads:
            p, u = np.ascontiguousarray(b.params), b.u0.copy()
            bufs.append((p, u))
            tickets.append(nls.nls_server_submit(srv, b.family, p.ctypes.data if p.size else 0,
                                                 u.ctypes.data, b.n, b.batch, LS | MIXED, 1e-10, 50))
        res = [nls.nls_server_wait_timed(srv, t) for t in tickets]
    finally:
        nls.nls_server_destroy(srv)
    for b, (solved, t) in zip(payloads, res):
        assert solved == b.batch
        assert t["t_submit"] <= t["t_admit"] <= t["t_launch"] <= t["t_done"]
        assert t["h2d_ms"] >= 0 and t["solve_ms"] > 0 and t["d2h_ms"] >= 0
        assert t["wave_requests"] >= 1
        device_s = (t["h2d_ms"] + t["solve_ms"] + t["d2h_ms"]) / 1e3
        assert device_s <= t["t_done"] - t["t_admit"] + 1e-3
