"""Batched products under a captured CUDA graph, and the autotuner that picks
the row-tier thresholds, hash-table load and narrow-tier shape for a batch.

Many small, uneven problems C_b = A_b * B_b are one product of the
block-diagonal stack of the A_b with the row stack of the B_b (the stacked
result is the stack of the C_b). ``BatchedSpGEMM`` keeps operands, scratch
and a capacity-sized output on the device, runs the product through
``spgemm_batched`` (no host synchronisation, no allocation) and captures it
once in a CUDA graph, so a batch is one graph launch.
"""
from __future__ import annotations

import ctypes
import statistics

import numpy as np
import torch

from . import _lib
from ._lib import check
from .api import DeviceCSR, Plan, _ptr
from .gen import HostCSR, csr_from_coo


def stack_problems(problems) -> tuple[HostCSR, HostCSR, np.ndarray, np.ndarray]:
    """Block-diagonal A and row-stacked B from [(A_b, B_b), ...] (host CSR).

    Returns (A, B, row_off, bcol) with row_off the first row of each problem
    in A (and in the stacked C). Every B_b must have the same column count."""
    cols = {Bb.cols for _, Bb in problems}
    if len(cols) > 1:
        raise ValueError("all B_b must share their column count")
    ncols = cols.pop() if cols else 0
    ra, ca, va, rb, cb, vb = [], [], [], [], [], []
    row_off = np.zeros(len(problems) + 1, dtype=np.int64)
    brow_off = np.zeros(len(problems) + 1, dtype=np.int64)
    for q, (Ab, Bb) in enumerate(problems):
        if Ab.cols != Bb.rows:
            raise ValueError("A_b.cols must equal B_b.rows")
        row_off[q + 1] = row_off[q] + Ab.rows
        brow_off[q + 1] = brow_off[q] + Bb.rows
        ra.append(np.repeat(np.arange(Ab.rows), np.diff(Ab.row_ptr.astype(np.int64))) + row_off[q])
        ca.append(Ab.col.astype(np.int64) + brow_off[q])
        va.append(Ab.val)
        rb.append(np.repeat(np.arange(Bb.rows), np.diff(Bb.row_ptr.astype(np.int64))) + brow_off[q])
        cb.append(Bb.col.astype(np.int64))
        vb.append(Bb.val)
    cat = lambda xs, dt: np.concatenate(xs).astype(dt) if xs else np.zeros(0, dt)  # noqa: E731
    A = csr_from_coo(int(row_off[-1]), int(brow_off[-1]), cat(ra, np.int64), cat(ca, np.int64),
                     cat(va, np.float32), sort=False)
    B = csr_from_coo(int(brow_off[-1]), ncols, cat(rb, np.int64), cat(cb, np.int64),
                     cat(vb, np.float32), sort=False)
    return A, B, row_off, brow_off


class BatchedSpGEMM:
    """Device-resident C = A*B for a fixed structure, replayable as a CUDA graph."""

    def __init__(self, A: DeviceCSR, B: DeviceCSR, plan: Plan | None = None,
                 capacity: int | None = None):
        self.plan = plan or Plan(device=A.device.index)
        self.A, self.B = A, B
        dev = A.device
        self.ws = self.plan.workspace(A, B)
        self.ip_row = torch.empty(A.rows, dtype=torch.int64, device=dev)
        self.row_nnz = torch.empty(A.rows, dtype=torch.int32, device=dev)
        self.row_ptr = torch.empty(A.rows + 1, dtype=torch.int32, device=dev)
        self.nnz_dev = torch.zeros(1, dtype=torch.int64, device=dev)
        if capacity is None:
            capacity = self.upper_bound()
        if capacity > 2**31 - 1:
            raise ValueError("capacity beyond int32 row pointers")
        self.capacity = int(capacity)
        self.col = torch.empty(self.capacity, dtype=torch.int32, device=dev)
        self.val = torch.empty(self.capacity, dtype=torch.float32, device=dev)
        self.graph = None
        self.stream = None

    def upper_bound(self) -> int:
        """sum_i min(IP_i, B.cols) >= nnz(C) (one synchronising count)."""
        ip, _ = self.plan.count(self.A, self.B, self.ws, ip_row=self.ip_row, total=False)
        torch.cuda.synchronize(self.A.device)
        return int(torch.clamp(ip, max=self.B.cols).sum().item())

    def enqueue(self, stream=None) -> None:
        s = (stream or torch.cuda.current_stream()).cuda_stream
        check(_lib.lib().spgemm_batched(self.plan.handle, ctypes.byref(self.A.struct()),
                                        ctypes.byref(self.B.struct()), _ptr(self.ws),
                                        self.ws.numel(), _ptr(self.ip_row), _ptr(self.row_nnz),
                                        _ptr(self.row_ptr), _ptr(self.col), _ptr(self.val),
                                        self.capacity, _ptr(self.nnz_dev), s),
              "spgemm_batched")

    def capture(self) -> None:
        """Run once (loads every kernel), then capture one run in a CUDA graph."""
        self.stream = torch.cuda.Stream(device=self.A.device)
        self.stream.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(self.stream):
            self.enqueue(self.stream)
        self.stream.synchronize()
        self.plan.check_status(self.ws, "batched warm-up", stream=self.stream)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=self.stream):
            self.enqueue(self.stream)
        self.graph = g

    def run(self) -> None:
        if self.graph is None:
            self.enqueue()
        else:
            self.graph.replay()

    def result(self) -> DeviceCSR:
        """Synchronise, check the status word and return C (views of the buffers)."""
        torch.cuda.synchronize(self.A.device)
        self.plan.check_status(self.ws, "spgemm_batched")
        n = int(self.nnz_dev.item())
        return DeviceCSR(self.A.rows, self.B.cols, self.row_ptr, self.col[:n], self.val[:n])


# ---------------------------------------------------------------------------
# Autotuner
# ---------------------------------------------------------------------------

# The autotuner's search space: the row-tier thresholds (the role of the
# paper's Table 1 group boundaries), the hash tables' target load (table
# sizes), and the narrow tiers' warps per block and row limit. The
# accumulation-precision rule (fp32_max_terms) is not a knob: every point
# meets the same tolerance.
BASE_OPTS = {"esc_max": 32, "warp_max_ip": 1024, "block_max_ip": 16384, "warp_max_nnz": 512,
             "block_max_nnz": 8192, "hash_load_pct": 50, "narrow_warps": 8,
             "narrow_max_ip": 32768}
SEARCH_SPACE = [
    ("narrow_warps", [{"narrow_warps": w} for w in (4, 8, 16)]),
    ("narrow_max_ip", [{"narrow_max_ip": v} for v in (4096, 32768, 131072)]),
    ("tiers", [{}, {"esc_max": 16},
               {"warp_max_ip": 256, "warp_max_nnz": 128},
               {"warp_max_ip": 512, "warp_max_nnz": 256},
               {"block_max_ip": 4096, "block_max_nnz": 2048},
               {"warp_max_nnz": 256, "block_max_nnz": 4096}]),
    ("hash_load_pct", [{"hash_load_pct": v} for v in (35, 50, 70)]),
]


def candidate_opts() -> list[dict]:
    """Every point the search can visit (each knob's values on the defaults)."""
    out, seen = [], set()
    for _, values in SEARCH_SPACE:
        for v in values:
            c = dict(BASE_OPTS, **v)
            key = tuple(sorted(c.items()))
            if key not in seen:
                seen.add(key)
                out.append(c)
    return out


def time_graph(bs: BatchedSpGEMM, reps: int = 5) -> float:
    """Median milliseconds of one graph replay (CUDA events on its stream)."""
    times = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(bs.stream)
        with torch.cuda.stream(bs.stream):
            bs.graph.replay()
        e1.record(bs.stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    return statistics.median(times)


def autotune(A: DeviceCSR, B: DeviceCSR, candidates: list[dict] | None = None, reps: int = 5,
             capacity: int | None = None):
    """Pick options for this batch by timing captured graphs. Without
    ``candidates``: coordinate descent over SEARCH_SPACE (one knob group at a
    time, each value tried on the best point so far, the fastest kept).
    Returns (best BatchedSpGEMM, best opts, {label: ms}) with every timed
    point in the dict."""
    timings = {}
    best = None

    def trial(label, opts):
        nonlocal best, capacity
        bs = BatchedSpGEMM(A, B, Plan(device=A.device.index, **opts), capacity=capacity)
        if capacity is None:
            capacity = bs.capacity
        bs.capture()
        ms = time_graph(bs, reps)
        timings[label] = ms
        if best is None or ms < best[0]:
            best = (ms, bs, dict(opts))
        else:
            del bs

    if candidates is not None:
        for q, opts in enumerate(candidates):
            trial(str(q), opts)
        return best[1], best[2], timings
    trial("default", dict(BASE_OPTS))
    for name, values in SEARCH_SPACE:
        base = dict(best[2])
        for v in values:
            opts = dict(base, **v)
            if opts == base:
                continue
            trial(f"{name}:{','.join(f'{k}={x}' for k, x in sorted(v.items())) or 'default'}", opts)
    return best[1], best[2], timings
