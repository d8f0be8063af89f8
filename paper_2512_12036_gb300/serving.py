"""Continuous-batching SpGEMM service on one GPU.

Requests C = A*B arrive over time with device-resident operands. A
dispatcher takes them in arrival order, bounds each request's device memory
from its intermediate-product count (spgemm_count: nnz(C) <= IP, so C needs
at most 8*min(IP, rows*cols) bytes plus row pointers, on top of the
workspace and per-row scratch) and admits it as soon as a slot is free and
the bound fits the remaining budget. Each slot owns a plan and a CUDA
stream, so admitted requests overlap on the device while later ones keep
arriving. A request whose bound exceeds a slot's share is split into
blocks of consecutive rows that fit (each a zero-copy row view of A) and
completes when all its blocks have; one that cannot be split small enough
is refused (SPGEMM_ERR_BUDGET). The GPU back end preallocates every slot's
share once, so serving itself allocates no device memory. Latency is
completion minus arrival.

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

from ._lib import ERR_BUDGET, ERR_TIMEOUT


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
                 split_fn=None, request_limit: int | None = None):
        self.bound_fn, self.exec_fn, self.split_fn = bound_fn, exec_fn, split_fn
        self.adm = Admission(budget_bytes, slots)
        self.limit = int(request_limit) if request_limit is not None else int(budget_bytes)
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
            try:
                req.bound, req.ip = self.bound_fn(req)
                parts = [req]
                if req.bound > self.limit:
                    parts = self.split_fn(req, self.limit) if self.split_fn else None
                    if not parts or any(p.bound > self.limit for p in parts):
                        parts = None
                        req.error = ERR_BUDGET
            except Exception as exc:  # noqa: BLE001 - reported on the request
                parts = None
                req.error = getattr(exc, "code", -1) or -1
            if parts is None:
                req.done = time.perf_counter()
                req.event.set()
                continue
            if len(parts) > 1 or parts[0] is not req:
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

def request_bound(plan, A, B, ws_bytes: int, ip_total: int) -> int:
    """Device bytes a request may need: workspace, IP/nnz scratch, row
    pointers and C (nnz(C) <= min(IP, rows*cols)), with alignment slack."""
    nnz_bound = min(int(ip_total), int(A.rows) * int(B.cols))
    return (int(ws_bytes) + 12 * A.rows + 4 * (A.rows + 1) + 8 * nnz_bound + 8 * 256)


class Arena:
    """Views carved from one preallocated device buffer (no allocation while
    serving); every view starts on a 256-byte boundary."""

    def __init__(self, nbytes: int, device):
        import torch
        self.buf = torch.empty(int(nbytes) + 256, dtype=torch.uint8, device=device)
        self.base = (-self.buf.data_ptr()) % 256
        self.nbytes = int(nbytes)
        self.off = 0

    def reset(self) -> None:
        self.off = 0

    def take(self, nbytes: int, dtype):
        import torch
        nbytes = int(nbytes)
        start = self.base + self.off
        self.off += (nbytes + 255) // 256 * 256
        if self.off > self.nbytes:
            raise MemoryError("arena exhausted")
        view = self.buf[start:start + nbytes]
        return view.view(dtype) if dtype is not torch.uint8 else view

    def free(self) -> int:
        return self.nbytes - self.off


def gpu_server(slots: int = 4, budget_bytes: int = 64 << 30, device: int = 0,
               keep_results: bool = True, count_ws_bytes: int = 1 << 30,
               max_rows: int = 1 << 22) -> Server:
    """A Server whose slots each own a Plan, a CUDA stream and an arena of
    budget_bytes / slots preallocated device memory holding the request's
    workspace, per-row scratch and C, so serving allocates nothing. A
    request is admitted when a slot is free and its bound fits an arena;
    larger ones are split into row blocks that do. With keep_results=False
    a result is consumed on completion ((rows, nnz) is kept); otherwise C is
    copied out of the arena into its own tensors."""
    import torch

    from .api import DeviceCSR, Plan

    torch.cuda.set_device(device)
    dev = torch.device("cuda", device)
    per_slot = int(budget_bytes) // slots
    plans = [Plan(device=device) for _ in range(slots)]
    streams = [torch.cuda.Stream(device=device) for _ in range(slots)]
    arenas = [Arena(per_slot, dev) for _ in range(slots)]
    count_plan = Plan(device=device)
    count_stream = torch.cuda.Stream(device=device)
    count_arena = Arena(count_ws_bytes + 8 * max_rows, dev)

    def bound_fn(req):
        torch.cuda.set_device(device)
        count_arena.reset()
        nws = count_plan.workspace_bytes(req.A, req.B)
        with torch.cuda.stream(count_stream):
            ws = count_arena.take(nws, torch.uint8)
            count_plan.workspace_init(ws)
            ip_row = count_arena.take(8 * max(req.A.rows, 1), torch.int64)[:req.A.rows]
            ip_row, ip_total = count_plan.count(req.A, req.B, ws, ip_row=ip_row)
            bound = request_bound(count_plan, req.A, req.B, nws, ip_total)
            # the per-row counts are needed only to split a request that does
            # not fit a slot; they go to host memory (on the count stream,
            # before the next request reuses the arena), never to a new
            # device buffer
            req.ip_row = ip_row.cpu().numpy() if bound > per_slot else None
        return bound, ip_total

    def split_fn(req, budget):
        """Blocks of consecutive rows whose bounds fit half an arena."""
        ip = req.ip_row
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
            nws = count_plan.workspace_bytes(sub.A, sub.B)
            sub.ip = int(ip[a:b].sum())
            sub.bound = request_bound(count_plan, sub.A, sub.B, nws, sub.ip)
            out.append(sub)
        return out

    def exec_fn(slot, req):
        torch.cuda.set_device(device)
        plan, ar, st = plans[slot], arenas[slot], streams[slot]
        ar.reset()
        A, B = req.A, req.B
        with torch.cuda.stream(st):
            ws = ar.take(plan.workspace_bytes(A, B), torch.uint8)
            plan.workspace_init(ws)
            ip_row = ar.take(8 * max(A.rows, 1), torch.int64)[:A.rows]
            row_nnz = ar.take(4 * max(A.rows, 1), torch.int32)[:A.rows]
            row_ptr = ar.take(4 * (A.rows + 1), torch.int32)
            plan.count(A, B, ws, ip_row=ip_row, total=False)
            _, nnz = plan.symbolic(A, B, ip_row, ws, row_nnz=row_nnz)
            cap = ar.free() // 8 - 64
            if nnz > cap or nnz > 2**31 - 1:
                raise MemoryError("request exceeds its arena")
            col = ar.take(4 * max(nnz, 1), torch.int32)[:nnz]
            val = ar.take(4 * max(nnz, 1), torch.float32)[:nnz]
            plan.row_ptr(row_nnz, ws, out=row_ptr)
            plan.numeric(A, B, ip_row, row_ptr, ws, col, val)
            if keep_results:
                C = DeviceCSR(A.rows, B.cols, row_ptr.clone(), col.clone(), val.clone())
            st.synchronize()
            plan.check_status(ws, "served request", stream=st)
        return C if keep_results else (A.rows, nnz)

    return Server(bound_fn, exec_fn, slots, budget_bytes, split_fn=split_fn, request_limit=per_slot)


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


def run_served(server: Server, reqs, arrivals, timeout_s: float = 600.0):
    """Submit requests at the given arrival offsets (seconds) and wait, at
    most ``timeout_s`` after the last submission; a request still unfinished
    then is marked failed (ERR_TIMEOUT) instead of blocking the caller."""
    t0 = time.perf_counter()
    for req, at in zip(reqs, arrivals):
        now = time.perf_counter() - t0
        if now < at:
            time.sleep(at - now)
        server.submit(req)
    deadline = time.perf_counter() + timeout_s
    for req in reqs:
        if not req.event.wait(max(0.0, deadline - time.perf_counter())):
            req.error = ERR_TIMEOUT
            req.done = time.perf_counter()
    return reqs


def poisson_arrivals(n: int, rate: float, seed: int) -> np.ndarray:
    """Arrival offsets (s) of a Poisson process of the given rate."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=n))
