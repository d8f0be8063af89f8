"""Matrix-based bulk neighbourhood sampling on the SpGEMM (Section IV-C,
mini-batch GNN training).

For layer l (from L down to 1), with Q^l holding one row per frontier
vertex (value 1 at the vertex):
  P       = Q^l * A                       (the hash-based SpGEMM)
  Q^{l-1} = SAMPLE(P, s_l)                (spgemm_sample_rows; NORM is the
                                           division by the row total inside
                                           the inverse transform)
  S, F    = selector of Q^{l-1}'s vertices (spgemm_select_columns)
  A^l     = P * S = EXTRACT(A, Q^l, Q^{l-1})
and F (one row per selected vertex) is Q for the next layer. Several
minibatches are sampled in bulk by stacking their frontier rows in one Q.
The uniforms are an input (seeded, drawn on the device by the caller or by
``sample_layers``), so a run is reproducible and checkable.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import check
from .api import DeviceCSR, Plan, _ptr, _stream

UNIFORM, BY_VALUE, BY_SQUARE = 0, 1, 2


def _ws_rows(plan: Plan, rows: int, device) -> torch.Tensor:
    """Workspace for a matrix of ``rows`` rows (status word, scan scratch)."""
    empty = DeviceCSR(rows, 0, torch.zeros(rows + 1, dtype=torch.int32, device=device),
                      torch.zeros(0, dtype=torch.int32, device=device),
                      torch.zeros(0, dtype=torch.float32, device=device))
    return plan.workspace(empty, DeviceCSR(0, 0, torch.zeros(1, dtype=torch.int32, device=device),
                                           empty.col, empty.val))


def sample_rows(P: DeviceCSR, s: int, u: torch.Tensor, mode: int, plan: Plan,
                stream=None) -> DeviceCSR:
    """SAMPLE: up to s distinct columns per row of P drawn with uniforms u
    (P.rows x s, fp32 in [0, 1)); value 1 at every drawn column."""
    dev = P.device
    ws = _ws_rows(plan, P.rows, dev)
    rp = torch.empty(P.rows + 1, dtype=torch.int32, device=dev)
    col = torch.empty(P.rows * s, dtype=torch.int32, device=dev)
    val = torch.empty(P.rows * s, dtype=torch.float32, device=dev)
    nnz = ctypes.c_int64()
    check(_lib.lib().spgemm_sample_rows(plan.handle, ctypes.byref(P.struct()), s, _ptr(u), mode,
                                        _ptr(ws), ws.numel(), _ptr(rp), _ptr(col), _ptr(val),
                                        ctypes.byref(nnz), _stream(stream)),
          "spgemm_sample_rows")
    n = int(nnz.value)
    return DeviceCSR(P.rows, P.cols, rp, col[:n], val[:n])


def select_columns(Q: DeviceCSR, plan: Plan, stream=None) -> tuple[DeviceCSR, DeviceCSR]:
    """(S, F): S (Q.cols x m) selects Q's distinct columns, F = S^T (m x Q.cols)."""
    dev = Q.device
    n = Q.cols
    cap = max(1, min(n, Q.nnz))
    ws = _ws_rows(plan, n, dev)
    S_rp = torch.empty(n + 1, dtype=torch.int32, device=dev)
    F_rp = torch.empty(cap + 1, dtype=torch.int32, device=dev)
    S_col = torch.empty(cap, dtype=torch.int32, device=dev)
    S_val = torch.empty(cap, dtype=torch.float32, device=dev)
    F_col = torch.empty(cap, dtype=torch.int32, device=dev)
    F_val = torch.empty(cap, dtype=torch.float32, device=dev)
    m = ctypes.c_int64()
    check(_lib.lib().spgemm_select_columns(plan.handle, ctypes.byref(Q.struct()), _ptr(ws),
                                           ws.numel(), _ptr(S_rp), _ptr(S_col), _ptr(S_val),
                                           _ptr(F_rp), _ptr(F_col), _ptr(F_val), ctypes.byref(m),
                                           _stream(stream)),
          "spgemm_select_columns")
    m = int(m.value)
    S = DeviceCSR(n, m, S_rp, S_col[:m], S_val[:m])
    F = DeviceCSR(m, n, F_rp[:m + 1], F_col[:m], F_val[:m])
    return S, F


def frontier(vertices, n: int, device) -> DeviceCSR:
    """Q^L: one row per batch vertex (value 1), columns = the graph's vertices."""
    v = torch.as_tensor(np.asarray(vertices, dtype=np.int32), device=device)
    b = v.numel()
    return DeviceCSR(b, n, torch.arange(b + 1, dtype=torch.int32, device=device), v,
                     torch.ones(b, dtype=torch.float32, device=device))


def sample_layer(A: DeviceCSR, Q: DeviceCSR, s: int, u: torch.Tensor, mode: int, plan: Plan):
    """One layer: returns (F, A_l, P, Qs) with F the next frontier, A_l the
    sampled adjacency (Q's rows x F's vertices), P = Q*A, Qs = SAMPLE(P)."""
    P = plan.spgemm(Q, A)
    Qs = sample_rows(P, s, u, mode, plan)
    S, F = select_columns(Qs, plan)
    A_l = plan.spgemm(P, S)
    return F, A_l, P, Qs


def sample_layers(A: DeviceCSR, batch, fanouts, plan: Plan | None = None, mode: int = UNIFORM,
                  seed: int = 0):
    """Multi-layer sampling of the batch vertices with fanouts [s_L, ..., s_1]:
    returns ([A^L, ..., A^1], [Q^L, ..., Q^0], uniforms used)."""
    plan = plan or Plan(device=A.device.index)
    g = torch.Generator(device=A.device).manual_seed(seed)
    Q = frontier(batch, A.rows, A.device)
    adj, qs, us = [], [Q], []
    for s in fanouts:
        u = torch.rand(Q.rows, s, generator=g, device=A.device)
        Q, A_l, _, _ = sample_layer(A, Q, s, u, mode, plan)
        adj.append(A_l)
        qs.append(Q)
        us.append(u)
    return adj, qs, us
