"""Markov clustering (Algorithm 6) on the GPU, held as M^T in CSR.

A column of M is a row of M^T, so the expansion M*M is computed as
E = M^T * M^T = (M*M)^T with the SpGEMM, and prune / top-k / inflate /
normalise run per row of E in the spgemm_mcl_step kernels.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib
from ._lib import check
from .api import DeviceCSR, Plan, _ptr, _stream


def mcl_step(plan: Plan, E: DeviceCSR, theta: float, k: int, r: float, order: int = 0,
             ws: torch.Tensor | None = None, stream=None) -> DeviceCSR:
    """Prune (< theta), keep the top k per row, inflate (^r), normalise rows."""
    if ws is None:
        ws = plan.workspace(E, DeviceCSR(0, 0, torch.zeros(1, dtype=torch.int32, device=E.device),
                                         torch.zeros(0, dtype=torch.int32, device=E.device), None))
    cap = E.nnz if k < 0 else min(E.nnz, E.rows * k)
    rp = torch.empty(E.rows + 1, dtype=torch.int32, device=E.device)
    col = torch.empty(max(cap, 1), dtype=torch.int32, device=E.device)
    val = torch.empty(max(cap, 1), dtype=torch.float32, device=E.device)
    nnz = ctypes.c_int64()
    check(_lib.lib().spgemm_mcl_step(plan.handle, ctypes.byref(E.struct()), float(theta), int(k),
                                     float(r), int(order), _ptr(ws), ws.numel(), _ptr(rp),
                                     _ptr(col), _ptr(val), ctypes.byref(nnz), _stream(stream)),
          "spgemm_mcl_step")
    n = int(nnz.value)
    return DeviceCSR(E.rows, E.cols, rp, col[:n], val[:n])


def normalise_rows(plan: Plan, M: DeviceCSR) -> DeviceCSR:
    """Column-stochastic start of Algorithm 6 on M^T: every row divided by its sum."""
    return mcl_step(plan, M, float("-inf"), -1, 1.0, 0)


@dataclass
class MCLResult:
    Mt: DeviceCSR
    iterations: int
    nnz_history: list
    ip_history: list


def markov_cluster(plan: Plan, Gt: DeviceCSR, iterations: int = 20, theta: float = 1e-4,
                   k: int = 32, r: float = 2.0, order: int = 0) -> MCLResult:
    """Gt: the graph with self-loops added, as M^T (rows = columns of M).
    A fixed number of iterations replaces the convergence test. Each
    expansion is one spgemm call (its own count, allocation and
    accumulation phases); the per-row product counts it writes are summed
    on the device and read once at the end."""
    M = normalise_rows(plan, Gt)
    nnz_hist, ip_sums = [M.nnz], []
    for _ in range(iterations):
        ip_row = torch.empty(M.rows, dtype=torch.int64, device=M.device)
        E = plan.spgemm(M, M, ip_row=ip_row)
        ip_sums.append(ip_row.sum())
        M = mcl_step(plan, E, theta, k, r, order)
        nnz_hist.append(M.nnz)
    ip_hist = [int(x) for x in torch.stack(ip_sums).cpu()] if ip_sums else []
    return MCLResult(M, iterations, nnz_hist, ip_hist)


def markov_cluster_served(server, plan: Plan, Gt: DeviceCSR, iterations: int = 20,
                          theta: float = 1e-4, k: int = 32, r: float = 2.0, order: int = 0,
                          tag: str = "mcl"):
    """markov_cluster with every expansion M*M submitted as a request to a
    continuous-batching server (serving.gpu_server with keep_results=True),
    so the expansions of several clustering jobs, or of other clients,
    share the device. Returns (MCLResult, the expansion requests)."""
    from .serving import Request

    M = normalise_rows(plan, Gt)
    nnz_hist, ip_hist, reqs = [M.nnz], [], []
    for it in range(iterations):
        req = server.submit(Request(A=M, B=M, tag=f"{tag}_expand{it}"))
        req.event.wait()
        if req.error:
            raise _lib.SpgemmError(req.error if req.error > 0 else _lib.ERR_INTERNAL,
                                   f"served MCL expansion {it}")
        E = req.result if not isinstance(req.result, list) else _stack_blocks(req.result, M)
        ip_hist.append(req.ip)
        reqs.append(req)
        M = mcl_step(plan, E, theta, k, r, order)
        nnz_hist.append(M.nnz)
    return MCLResult(M, iterations, nnz_hist, ip_hist), reqs


def _stack_blocks(parts, M: DeviceCSR) -> DeviceCSR:
    """One DeviceCSR from a split request's row blocks (in row order)."""
    rps, cols, vals, base = [], [], [], 0
    for q, C in enumerate(parts):
        rp = C.row_ptr.to(torch.int64) + base
        rps.append(rp if q == len(parts) - 1 else rp[:-1])
        cols.append(C.col)
        vals.append(C.val)
        base += C.nnz
    if base > 2**31 - 1:
        raise _lib.SpgemmError(_lib.ERR_OVERFLOW, "served MCL expansion")
    return DeviceCSR(M.rows, M.cols, torch.cat(rps).to(torch.int32), torch.cat(cols),
                     torch.cat(vals))


def interpret(Mt: DeviceCSR) -> np.ndarray:
    """InterpretMatrix: node j joins the attractor holding the largest value
    in column j of M (row j of M^T); ties go to the smaller index."""
    h = Mt.to_host()
    out = np.full(h.rows, -1, dtype=np.int64)
    for j in range(h.rows):
        c, v = h.row(j)
        if c.size:
            out[j] = int(c[np.argmax(v)])
    return out
