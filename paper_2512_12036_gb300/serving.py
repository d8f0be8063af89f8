"""Continuous-batching SpGEMM service on one GPU.

Requests C = A*B arrive over time with device-resident operands. A
dispatcher takes them in arrival order, bounds each request's device memory
from its intermediate-product count (spgemm_count: nnz(C) <= IP, so C needs
at most 8*min(IP, rows*cols) bytes plus row pointers, on top of the
workspace and per-row scratch) and admits it as soon as a slot is free and
the bound fits the remaining budget. Each slot owns a plan and a CUDA
stream, so admitted requests overlap on the device while later ones keep
arriving. A request whose bound exceeds the whole budget is split into
blocks of consecutive rows that fit (each a zero-copy row view of A) and
completes when all its blocks have; one that cannot be split small enough
is refused (SPGEMM_ERR_BUDGET). Latency is completion minus arrival.

The admission logic takes the bound and executor as functions so it can be
exercised on the CPU with fakes.
"""
from __future__ import annotations

import queue
import statistics
import threading
import time
from dataclasses import dataclass, field

import numpy as np

from ._lib import ERR_BUDGET


@dataclass
class Request:
    A: object
    B: object
    tag: str = ""
    rid: int = -1
    arrival: float = 0.0
    admitted: float = 0.0
    done: float = 0.0
    bound: int = 0
    ip: int = 0
    result: object = None
    error: int = 0
    row_begin: int = 0
    parent: object = None
    parts: list = None
    pending: int = 0
    event: threading.Event = field(default_factory=threading.Event)

    @property
    def latency(self) -> float:
        return self.done - self.arrival


class Admission:
    """Budget accounting shared by the dispatcher and the slots."""

    def __init__(self, budget_bytes: int, slots: int):
        self.budget = int(budget_bytes)
        self.free_slots = list(range(slots))
        self.used = 0
        self.peak = 0
        self.cv = threading.Condition()

    def acquire(self, need: int) -> int:
        with self.cv:
            while not self.free_slots or self.used + need > self.budget:
                self.cv.wait()
            self.used += need
            self.peak = max(self.peak, self.used)
            return self.free_slots.pop(0)

    def release(self, slot: int, need: int) -> None:
        with self.cv:
            self.used -= need
            self.free_slots.append(slot)
            self.cv.notify_all()


class Server:
    """Dispatcher + slot workers. ``bound_fn(req) -> (bytes, ip)`` and
    ``exec_fn(slot, req) -> result`` do the device work (see gpu_server)."""

    def __init__(self, bound_fn, exec_fn, slots: int = 4, budget_bytes: int = 64 << 30,
                 split_fn=None):
        self.bound_fn, self.exec_fn, self.split_fn = bound_fn, exec_fn, split_fn
        self.adm = Admission(budget_bytes, slots)
        self.inbox: queue.Queue = queue.Queue()
        self.slot_q = [queue.Queue() for _ in range(slots)]
        self.requests: list[Request] = []
        self._ids = 0
        self._lock = threading.Lock()
        self.threads = [threading.Thread(target=self._dispatch, daemon=True)]
        self.threads += [threading.Thread(target=self._work, args=(s,), daemon=True)
                         for s in range(slots)]
        for t in self.threads:
            t.start()

    def submit(self, req: Request) -> Request:
        with self._lock:
            req.rid = self._ids
            self._ids += 1
            self.requests.append(req)
        req.arrival = time.perf_counter()
        self.inbox.put(req)
        return req

    def _dispatch(self) -> None:
        while True:
            req = self.inbox.get()
            if req is None:
                for q in self.slot_q:
                    q.put(None)
                return
            req.bound, req.ip = self.bound_fn(req)
            parts = [req]
            if req.bound > self.adm.budget:
                parts = self.split_fn(req, self.adm.budget) if self.split_fn else None
                if not parts or any(p.bound > self.adm.budget for p in parts):
                    req.error = ERR_BUDGET
                    req.done = time.perf_counter()
                    req.event.set()
                    continue
                req.parts = parts
                req.pending = len(parts)
                for p in parts:
                    p.parent = req
            for p in parts:
                slot = self.adm.acquire(p.bound)
                p.admitted = time.perf_counter()
                if p is not req and not req.admitted:
                    req.admitted = p.admitted
                self.slot_q[slot].put(p)

    def _work(self, slot: int) -> None:
        while True:
            req = self.slot_q[slot].get()
            if req is None:
                return
            try:
                req.result = self.exec_fn(slot, req)
            except Exception as exc:  # noqa: BLE001 - reported per request
                req.error = getattr(exc, "code", -1)
            req.done = time.perf_counter()
            self.adm.release(slot, req.bound)
            parent = req.parent
            if parent is None:
                req.event.set()
                continue
            with self._lock:
                parent.pending -= 1
                if req.error:
                    parent.error = req.error
                last = parent.pending == 0
            if last:
                parent.result = [p.result for p in parent.parts]
                parent.done = time.perf_counter()
                parent.event.set()

    def close(self) -> None:
        self.inbox.put(None)
        for t in self.threads:
            t.join()


def latency_stats(reqs) -> dict:
    lat = sorted(r.latency for r in reqs if not r.error)
    if not lat:
        return {"n": 0}
    q = lambda p: lat[min(len(lat) - 1, int(round(p * (len(lat) - 1))))]  # noqa: E731
    return {"n": len(lat), "p50_ms": 1e3 * q(0.50), "p99_ms": 1e3 * q(0.99),
            "mean_ms": 1e3 * statistics.fmean(lat), "max_ms": 1e3 * lat[-1]}


# ---------------------------------------------------------------------------
# GPU back end
# ---------------------------------------------------------------------------

def request_bound(plan, A, B, ws, ip_total: int) -> int:
    """Device bytes a request may need: workspace, IP/nnz scratch, row
    pointers and C (nnz(C) <= min(IP, rows*cols))."""
    nnz_bound = min(int(ip_total), int(A.rows) * int(B.cols))
    return (int(ws.numel()) + 12 * A.rows + 4 * (A.rows + 1) + 8 * nnz_bound)


def gpu_server(slots: int = 4, budget_bytes: int = 64 << 30, device: int = 0,
               max_block_nnz: int = 2**31 - 1, keep_results: bool = True) -> Server:
    """A Server whose slots each own a Plan and a CUDA stream. With
    keep_results=False a request's result is consumed on completion: only
    (rows, nnz, sum of values) is kept and C's memory returns to the pool."""
    import torch

    from .api import Plan

    torch.cuda.set_device(device)
    plans = [Plan(device=device) for _ in range(slots)]
    streams = [torch.cuda.Stream(device=device) for _ in range(slots)]
    count_plan = Plan(device=device)
    count_stream = torch.cuda.Stream(device=device)

    def bound_fn(req):
        torch.cuda.set_device(device)
        with torch.cuda.stream(count_stream):
            ws = count_plan.workspace(req.A, req.B)
            ip_row, ip_total = count_plan.count(req.A, req.B, ws)
        req.ip_row = ip_row
        return request_bound(count_plan, req.A, req.B, ws, ip_total), ip_total

    def split_fn(req, budget):
        """Blocks of consecutive rows whose bounds fit half the budget."""
        ip = req.ip_row.cpu().numpy()
        cols = int(req.B.cols)
        csum = np.cumsum(np.minimum(ip, cols) * 8 + 16)
        target = budget // 2
        parts, r0, base = [], 0, 0
        while r0 < ip.size:
            r1 = max(int(np.searchsorted(csum, base + target, side="right")), r0 + 1)
            parts.append((r0, r1))
            base = int(csum[r1 - 1])
            r0 = r1
        out = []
        for a, b in parts:
            sub = Request(A=req.A.view_rows(a, b), B=req.B, tag=req.tag, row_begin=a)
            sub.arrival = req.arrival
            with torch.cuda.stream(count_stream):
                ws = count_plan.workspace(sub.A, sub.B)
                _, ipt = count_plan.count(sub.A, sub.B, ws)
            sub.bound, sub.ip = request_bound(count_plan, sub.A, sub.B, ws, ipt), ipt
            out.append(sub)
        return out

    def exec_fn(slot, req):
        torch.cuda.set_device(device)
        plan = plans[slot]
        with torch.cuda.stream(streams[slot]):
            ws = plan.workspace(req.A, req.B)
            blocks, _, _ = plan.spgemm_blocks(req.A, req.B, max_block_nnz=max_block_nnz, ws=ws)
            if not keep_results:
                summary = (req.A.rows, sum(C.nnz for _, _, C in blocks),
                           float(sum(C.val.double().sum() for _, _, C in blocks)))
            streams[slot].synchronize()
            plan.check_status(ws, "served request")
        return blocks if keep_results else summary

    return Server(bound_fn, exec_fn, slots, budget_bytes, split_fn=split_fn)


def run_plain(reqs, arrivals, device: int = 0, max_block_nnz: int = 2**31 - 1):
    """The plain per-request path: one request at a time on one stream, in
    arrival order (a request waits for the ones before it)."""
    import torch

    from .api import Plan

    plan = Plan(device=device)
    t0 = time.perf_counter()
    for req, at in zip(reqs, arrivals):
        now = time.perf_counter() - t0
        if now < at:
            time.sleep(at - now)
        req.arrival = t0 + at
        ws = plan.workspace(req.A, req.B)
        blocks, req.ip, _ = plan.spgemm_blocks(req.A, req.B, max_block_nnz=max_block_nnz, ws=ws)
        torch.cuda.synchronize()
        req.result = blocks
        req.done = time.perf_counter()
    return reqs


def run_served(server: Server, reqs, arrivals):
    """Submit requests at the given arrival offsets (seconds) and wait."""
    t0 = time.perf_counter()
    for req, at in zip(reqs, arrivals):
        now = time.perf_counter() - t0
        if now < at:
            time.sleep(at - now)
        server.submit(req)
    for req in reqs:
        req.event.wait()
    return reqs


def poisson_arrivals(n: int, rate: float, seed: int) -> np.ndarray:
    """Arrival offsets (s) of a Poisson process of the given rate."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=n))
