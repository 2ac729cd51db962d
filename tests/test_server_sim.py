"""Admission and scheduling of the request loop (include/sparc_server.h), on the CPU.

The server runs in its simulated mode: the worker threads, the queue and the HBM budget
are the real ones, and a solve sleeps for the request's sim_seconds instead of running on
a GPU. Device memory estimates are the library's own (sparc_request_bytes)."""
import numpy as np
import pytest

from paper_1603_04334_gb300 import serve, sparc


def _spec(n, ns, sim, natoms=0, dtype="f32"):
    R = np.zeros((natoms, 3)) + 4.0
    return serve.Spec((n, n, n), 0.3, R, np.ones(natoms), np.zeros((natoms, 4)), ns,
                      sim_seconds=sim, dtype=dtype)


def test_estimate_grows_with_size_and_precision():
    a = serve.request_bytes(_spec(48, 32, 0))
    b = serve.request_bytes(_spec(96, 32, 0))
    c = serve.request_bytes(_spec(96, 256, 0))
    d = serve.request_bytes(_spec(96, 256, 0, dtype="f64"))
    assert 0 < a < b < c
    # the two orbital blocks alone
    assert c > 2 * 4 * 96 ** 3 * 256 and d > 2 * 8 * 96 ** 3 * 256
    # per-node projector and table memory is counted
    assert serve.request_bytes(_spec(48, 32, 0, natoms=20)) > a


def test_budget_and_slots_are_never_exceeded():
    specs = [_spec(n, ns, 0.02 + 0.03 * (i % 3)) for i, (n, ns) in
             enumerate([(48, 32), (64, 64), (96, 128), (48, 200), (80, 32), (64, 300),
                        (96, 64), (48, 32), (112, 32), (64, 128)])]
    est = [serve.request_bytes(s) for s in specs]
    budget = int(2.2 * max(est))
    srv = serve.Server(budget, slots=3, simulate=True)
    ids = [srv.submit(s) for s in specs]
    res = [srv.wait(i, timeout=30) for i in ids]
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(specs)
    assert st["peak_reserved"] <= budget
    assert 2 <= st["max_running"] <= 3
    for r, s, e in zip(res, specs, est):
        assert r["status"] == 0 and r["est_bytes"] == e
        assert r["t_submit"] <= r["t_admit"] <= r["t_done"]
        assert r["t_done"] - r["t_admit"] >= s.sim_seconds * 0.9
    # at no time do the requests admitted and not yet done exceed the budget or the slots
    events = sorted([(r["t_admit"], 1, r["est_bytes"]) for r in res] +
                    [(r["t_done"], 0, -r["est_bytes"]) for r in res])
    used = running = 0
    for _, kind, b in events:
        used += b
        running += 1 if kind else -1
        assert used <= budget and running <= 3


def test_small_request_joins_while_a_large_one_waits():
    big = _spec(128, 512, 0.4)
    small = _spec(48, 32, 0.05)
    eb, es = serve.request_bytes(big), serve.request_bytes(small)
    budget = eb + es  # room for one large and one small request at a time
    srv = serve.Server(budget, slots=4, simulate=True)
    b1 = srv.submit(big)
    b2 = srv.submit(big)       # cannot start before b1 finishes
    s1 = srv.submit(small)     # fits beside b1: admitted ahead of b2
    r1, r2, r3 = srv.wait(b1, 30), srv.wait(b2, 30), srv.wait(s1, 30)
    srv.close()
    assert r3["t_admit"] < r1["t_done"] <= r2["t_admit"]


def test_passed_over_request_eventually_blocks_later_arrivals():
    big = _spec(128, 512, 0.05)
    small = _spec(48, 32, 0.01)
    eb, es = serve.request_bytes(big), serve.request_bytes(small)
    budget = eb + es
    srv = serve.Server(budget, slots=2, simulate=True)
    first = srv.submit(_spec(48, 32, 0.3))   # holds part of the budget for a while
    bid = srv.submit(big)                    # does not fit until `first` is done
    smalls = [srv.submit(small) for _ in range(20)]
    rb = srv.wait(bid, 30)
    rs = [srv.wait(i, 30) for i in smalls]
    srv.wait(first, 30)
    srv.close()
    # at most 8 later requests overtook the large one
    assert sum(r["t_admit"] < rb["t_admit"] for r in rs) <= 8


def test_oversize_request_is_rejected_and_shutdown_cancels_queue():
    s = _spec(96, 256, 0.0)
    srv = serve.Server(serve.request_bytes(s) - 1, slots=1, simulate=True)
    with pytest.raises(sparc.SparcError) as ei:
        srv.submit(s)
    assert ei.value.status == sparc.SPARC_ERR_BUDGET
    srv.close()
    srv = serve.Server(10 * serve.request_bytes(s), slots=1, simulate=True)
    srv.submit(_spec(48, 32, 0.3))
    srv.submit(_spec(48, 32, 0.3))
    srv.close()  # returns after the running request; the queued one is cancelled


def test_fp64_estimate_caps_the_digit_workspace():
    # 160^3 x 1024 FP64: the whole block's 47-bit digits would be about 100 GB; the Gram and
    # rotation run in row slabs whose workspace stays within 24 GiB, so the estimate is the
    # request's blocks and FP64 work arrays plus at most that
    n, ns = 160, 1024
    block = 8 * n ** 3 * ns
    est = serve.request_bytes(_spec(n, ns, 0, dtype="f64"))
    assert 4 * block < est < 4 * block + 1.1 * (24 << 30) + (1 << 30) + 4 * block // 16
