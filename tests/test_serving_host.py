"""Host-side serving logic with fake bounds and executors (no GPU): budget
never exceeded, every request finishes, oversize requests are refused,
requests overlap when slots and budget allow."""
import threading
import time

from paper_2512_12036_gb300 import serving
from paper_2512_12036_gb300._lib import ERR_BUDGET


def test_admission_respects_budget_and_overlaps():
    in_flight = []
    peak = [0, 0]
    lock = threading.Lock()
    budget = 100

    def bound_fn(req):
        return req.A, 0

    def exec_fn(slot, req):
        with lock:
            in_flight.append(req.A)
            peak[0] = max(peak[0], sum(in_flight))
            peak[1] = max(peak[1], len(in_flight))
        time.sleep(0.01)
        with lock:
            in_flight.remove(req.A)
        return req.A * 2

    srv = serving.Server(bound_fn, exec_fn, slots=3, budget_bytes=budget)
    sizes = [30, 40, 50, 20, 10, 60, 35, 5, 99, 150, 25]
    reqs = [srv.submit(serving.Request(A=s, B=None)) for s in sizes]
    for r in reqs:
        assert r.event.wait(5)
    srv.close()
    assert peak[0] <= budget and srv.adm.peak <= budget
    assert peak[1] >= 2                          # requests overlapped
    for r, s in zip(reqs, sizes):
        if s > budget:
            assert r.error == ERR_BUDGET and r.result is None
        else:
            assert r.error == 0 and r.result == 2 * s
    assert srv.adm.used == 0 and sorted(srv.adm.free_slots) == [0, 1, 2]


def test_executor_failure_is_reported_and_releases_budget():
    class Boom(RuntimeError):
        code = 7

    def exec_fn(slot, req):
        if req.A == 2:
            raise Boom("device failure")
        return req.A

    srv = serving.Server(lambda r: (10, 0), exec_fn, slots=2, budget_bytes=20)
    reqs = [srv.submit(serving.Request(A=i, B=None)) for i in range(5)]
    for r in reqs:
        assert r.event.wait(5)
    srv.close()
    assert [r.error for r in reqs] == [0, 0, 7, 0, 0]
    assert srv.adm.used == 0


def test_latency_stats_and_arrivals():
    reqs = [serving.Request(A=None, B=None, arrival=0.0, done=0.001 * i) for i in range(1, 101)]
    st = serving.latency_stats(reqs)
    assert st["n"] == 100 and abs(st["p50_ms"] - 50.5) < 1.0 and st["p99_ms"] >= 98.0
    arr = serving.poisson_arrivals(20000, rate=100.0, seed=1)
    assert abs(arr[-1] / 20000 - 0.01) < 0.001 and (arr > 0).all()


def test_oversize_request_split_into_parts():
    def split_fn(req, budget):
        parts = []
        for q in range(4):
            p = serving.Request(A=req.A // 4, B=q)
            p.bound = req.A // 4
            parts.append(p)
        return parts

    srv = serving.Server(lambda r: (r.A, 0), lambda slot, r: (r.B, r.A), slots=2,
                         budget_bytes=50, split_fn=split_fn)
    big = srv.submit(serving.Request(A=160, B=None))
    small = srv.submit(serving.Request(A=10, B=None))
    huge = srv.submit(serving.Request(A=1000, B=None))
    for r in (big, small, huge):
        assert r.event.wait(5)
    srv.close()
    assert big.error == 0 and sorted(big.result) == [(q, 40) for q in range(4)]
    assert small.error == 0 and huge.error == ERR_BUDGET
    assert srv.adm.peak <= 50


def test_bound_or_split_failure_is_reported_and_dispatch_continues():
    """A bound or split function that raises fails that request only; the
    dispatcher keeps serving the requests after it."""
    class BoundError(RuntimeError):
        code = 4

    def bound_fn(req):
        if req.A == "bad-bound":
            raise BoundError("arena exhausted")
        if req.A == "bad-split":
            return 1000, 0
        return 10, 0

    def split_fn(req, limit):
        raise MemoryError("cannot split")

    srv = serving.Server(bound_fn, lambda slot, req: req.A, slots=2, budget_bytes=100,
                         split_fn=split_fn, request_limit=50)
    names = ["a", "bad-bound", "b", "bad-split", "c"]
    reqs = [srv.submit(serving.Request(A=n, B=None)) for n in names]
    for r in reqs:
        assert r.event.wait(5)
    srv.close()
    assert [r.error for r in reqs] == [0, 4, 0, -1, 0]
    assert [r.result for r in reqs if not r.error] == ["a", "b", "c"]
    assert srv.adm.used == 0


def test_run_served_marks_stuck_requests_instead_of_hanging():
    from paper_2512_12036_gb300._lib import ERR_TIMEOUT
    gate = threading.Event()

    def exec_fn(slot, req):
        gate.wait(10)
        return req.A

    srv = serving.Server(lambda r: (1, 0), exec_fn, slots=1, budget_bytes=10)
    reqs = [serving.Request(A=i, B=None) for i in range(2)]
    t0 = time.perf_counter()
    serving.run_served(srv, reqs, [0.0, 0.0], timeout_s=0.2)
    assert time.perf_counter() - t0 < 5
    assert all(r.error == ERR_TIMEOUT for r in reqs)
    gate.set()
    srv.close()
