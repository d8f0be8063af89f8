"""Thin Python binding over the C ABI (argument marshalling only).

PyTorch provides device memory and streams; every step of the SpGEMM runs
in the CUDA kernels of libspgemm.so. Names follow the paper: intermediate
products (IP, Algorithm 1), allocation phase (symbolic), accumulation phase
(numeric).
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib
from ._lib import CsrStruct, OptsStruct, check


def _ptr(t: torch.Tensor | None) -> int | None:
    if t is None:
        return None
    return t.data_ptr() if t.numel() > 0 else None


def _stream(stream) -> int | None:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


@dataclass
class DeviceCSR:
    """CSR matrix in device memory (int32 row_ptr/col, float32 val).

    ``row_ptr[0]`` need not be 0: ``view_rows`` returns a block of rows that
    shares the column and value arrays."""

    rows: int
    cols: int
    row_ptr: torch.Tensor
    col: torch.Tensor
    val: torch.Tensor | None

    @property
    def nnz(self) -> int:
        return int(self.col.numel())

    @property
    def device(self) -> torch.device:
        return self.row_ptr.device

    @staticmethod
    def from_host(A, device="cuda", non_blocking: bool = False) -> "DeviceCSR":
        def up(a, dt):
            t = torch.from_numpy(np.ascontiguousarray(a, dtype=dt))
            if non_blocking:
                t = t.pin_memory()
            return t.to(device, non_blocking=non_blocking)
        return DeviceCSR(A.rows, A.cols, up(A.row_ptr, np.int32), up(A.col, np.int32),
                         up(A.val, np.float32))

    def to_host(self):
        from .gen import HostCSR
        rp = self.row_ptr.cpu().numpy().astype(np.int64)
        base = int(rp[0]) if rp.size else 0
        end = int(rp[-1]) if rp.size else 0
        col = self.col[base:end].cpu().numpy()
        val = (self.val[base:end].detach().cpu().numpy() if self.val is not None
               else np.zeros(0, np.float32))
        return HostCSR(self.rows, self.cols, (rp - base).astype(np.int32), col, val)

    def view_rows(self, r0: int, r1: int) -> "DeviceCSR":
        return DeviceCSR(r1 - r0, self.cols, self.row_ptr[r0:r1 + 1], self.col, self.val)

    def struct(self) -> CsrStruct:
        return CsrStruct(self.rows, self.cols, self.nnz, _ptr(self.row_ptr), _ptr(self.col),
                         _ptr(self.val))


def default_opts() -> dict:
    o = OptsStruct()
    check(_lib.lib().spgemm_opts_default(ctypes.byref(o)), "spgemm_opts_default")
    return {n: getattr(o, n) for n in _lib.OPT_FIELDS}


class Plan:
    """An spgemm_plan on one device; stateless between calls."""

    def __init__(self, device: int | None = None, **opts):
        L = _lib.lib()
        o = OptsStruct()
        check(L.spgemm_opts_default(ctypes.byref(o)), "spgemm_opts_default")
        for k, v in opts.items():
            if k not in _lib.OPT_FIELDS:
                raise KeyError(k)
            setattr(o, k, int(v))
        self.opts = {n: getattr(o, n) for n in _lib.OPT_FIELDS}
        if device is None:
            device = torch.cuda.current_device()
        self.device = device
        h = ctypes.c_void_p()
        check(L.spgemm_plan_create(ctypes.byref(h), ctypes.byref(o), device), "spgemm_plan_create")
        self.handle = h

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            _lib.lib().spgemm_plan_destroy(h)
            self.handle = None

    # ----------------------------------------------------------------- helpers
    def workspace_bytes(self, A: DeviceCSR, B: DeviceCSR) -> int:
        n = ctypes.c_size_t()
        check(_lib.lib().spgemm_workspace_bytes(self.handle, ctypes.byref(A.struct()),
                                                ctypes.byref(B.struct()), ctypes.byref(n)),
              "spgemm_workspace_bytes")
        return int(n.value)

    def workspace(self, A: DeviceCSR, B: DeviceCSR, stream=None) -> torch.Tensor:
        """A 256-byte aligned, initialised workspace for operands of these shapes."""
        nbytes = self.workspace_bytes(A, B)
        ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=A.device)
        off = (-ws.data_ptr()) % 256
        ws = ws[off:off + nbytes]
        self.workspace_init(ws, stream)
        return ws

    def workspace_init(self, ws: torch.Tensor, stream=None) -> None:
        check(_lib.lib().spgemm_workspace_init(self.handle, _ptr(ws), ws.numel(), _stream(stream)),
              "spgemm_workspace_init")

    def row_cache_rows(self, A: DeviceCSR, B: DeviceCSR, ws: torch.Tensor) -> int:
        """Rows that hold a slot of the row bitmap cache after the last
        allocation phase on this workspace (0 without a cache)."""
        if self.opts.get("row_cache_mb", 0) <= 0:
            return 0
        wpr = (B.cols + 31) // 32
        if wpr == 0 or wpr > 48 * 1024:
            return 0
        # the workspace layout: per slot a bitmap and, when B's column panels
        # have a panel table (at most 1024 panels), one count per panel
        panels = -(-B.cols // self.opts["panel_cols"])
        counts = 0 < panels <= 1024
        slot_bytes = (4 * A.rows + 255) // 256 * 256 + (256 if counts else 0)
        row_bytes = 4 * wpr + (4 * panels if counts else 0)
        nslots = min(A.rows, max(0, ((self.opts["row_cache_mb"] << 20) - slot_bytes) // row_bytes))
        used = int(ws[:16].view(torch.int32)[2].item())     # slots asked for (control block)
        return min(used, nslots)

    # ------------------------------------------------------------------ phases
    def count(self, A: DeviceCSR, B: DeviceCSR, ws: torch.Tensor, ip_row: torch.Tensor | None = None,
              total: bool = True, stream=None):
        """Algorithm 1: int64 IP per row (device) and, if ``total``, the int64 sum."""
        if ip_row is None:
            ip_row = torch.empty(A.rows, dtype=torch.int64, device=A.device)
        t = ctypes.c_int64()
        check(_lib.lib().spgemm_count(self.handle, ctypes.byref(A.struct()), ctypes.byref(B.struct()),
                                      _ptr(ws), ws.numel(), _ptr(ip_row),
                                      ctypes.byref(t) if total else None, _stream(stream)),
              "spgemm_count")
        return ip_row, (int(t.value) if total else None)

    def group(self, key: torch.Tensor, thresholds, ws: torch.Tensor, stream=None):
        """Section III-B grouping of ``key`` (device int64) at ``thresholds``."""
        thr = torch.as_tensor(list(thresholds), dtype=torch.int64, device=key.device)
        n = key.numel()
        mp = torch.empty(n, dtype=torch.int32, device=key.device)
        off = torch.empty(thr.numel() + 2, dtype=torch.int32, device=key.device)
        check(_lib.lib().spgemm_group(self.handle, _ptr(key), n, _ptr(thr), thr.numel(), _ptr(ws),
                                      ws.numel(), _ptr(mp), _ptr(off), _stream(stream)),
              "spgemm_group")
        return mp, off

    def symbolic(self, A: DeviceCSR, B: DeviceCSR, ip_row: torch.Tensor, ws: torch.Tensor,
                 row_nnz: torch.Tensor | None = None, total: bool = True, stream=None):
        """Allocation phase: int32 nnz per row of C and (if ``total``) the int64 sum."""
        if row_nnz is None:
            row_nnz = torch.empty(A.rows, dtype=torch.int32, device=A.device)
        t = ctypes.c_int64()
        check(_lib.lib().spgemm_symbolic(self.handle, ctypes.byref(A.struct()),
                                         ctypes.byref(B.struct()), _ptr(ip_row), _ptr(ws),
                                         ws.numel(), _ptr(row_nnz),
                                         ctypes.byref(t) if total else None, _stream(stream)),
              "spgemm_symbolic")
        return row_nnz, (int(t.value) if total else None)

    def row_ptr(self, row_nnz: torch.Tensor, ws: torch.Tensor, out: torch.Tensor | None = None,
                total: bool = False, stream=None):
        n = row_nnz.numel()
        if out is None:
            out = torch.empty(n + 1, dtype=torch.int32, device=row_nnz.device)
        t = ctypes.c_int64()
        check(_lib.lib().spgemm_row_ptr(self.handle, _ptr(row_nnz), n, _ptr(ws), ws.numel(),
                                        _ptr(out), ctypes.byref(t) if total else None,
                                        _stream(stream)),
              "spgemm_row_ptr")
        return out, (int(t.value) if total else None)

    def row_ptr_static(self, row_nnz: torch.Tensor, out: torch.Tensor | None = None,
                       total: bool = False, stream=None):
        """Row pointers through the entry point that needs no workspace (its
        scratch is a fixed array inside the library; see spgemm_row_ptr_static)."""
        n = row_nnz.numel()
        if out is None:
            out = torch.empty(n + 1, dtype=torch.int32, device=row_nnz.device)
        t = ctypes.c_int64()
        check(_lib.lib().spgemm_row_ptr_static(self.handle, _ptr(row_nnz), n, _ptr(out),
                                               ctypes.byref(t) if total else None,
                                               _stream(stream)),
              "spgemm_row_ptr_static")
        return out, (int(t.value) if total else None)

    def numeric(self, A: DeviceCSR, B: DeviceCSR, ip_row: torch.Tensor, row_ptr_C: torch.Tensor,
                ws: torch.Tensor, col_C: torch.Tensor, val_C: torch.Tensor, row_begin: int = 0,
                row_end: int | None = None, stream=None) -> None:
        """Accumulation phase for rows [row_begin, row_end) into col_C/val_C."""
        if row_end is None:
            row_end = A.rows
        check(_lib.lib().spgemm_numeric(self.handle, ctypes.byref(A.struct()),
                                        ctypes.byref(B.struct()), _ptr(ip_row), row_begin, row_end,
                                        _ptr(row_ptr_C), _ptr(ws), ws.numel(), _ptr(col_C),
                                        _ptr(val_C), _stream(stream)),
              "spgemm_numeric")

    # ----------------------------------------------------------------- backward
    def backward_workspace(self, A: DeviceCSR, B: DeviceCSR) -> torch.Tensor:
        n = ctypes.c_size_t()
        check(_lib.lib().spgemm_backward_workspace_bytes(self.handle, ctypes.byref(A.struct()),
                                                         ctypes.byref(B.struct()), ctypes.byref(n)),
              "spgemm_backward_workspace_bytes")
        ws = torch.empty(int(n.value) + 256, dtype=torch.uint8, device=A.device)
        off = (-ws.data_ptr()) % 256
        ws = ws[off:off + int(n.value)]
        self.workspace_init(ws)
        return ws

    def backward(self, A: DeviceCSR, B: DeviceCSR, C: DeviceCSR, dC: torch.Tensor,
                 need_dA: bool = True, need_dB: bool = True, ws: torch.Tensor | None = None,
                 stream=None):
        """Gradients of sum(dC * C) with respect to A's and B's stored values
        (dA: SDDMM of dC*B^T at A's pattern; dB: A^T*dC at B's pattern)."""
        if ws is None:
            ws = self.backward_workspace(A, B)
        dA = torch.empty(A.nnz, dtype=torch.float32, device=A.device) if need_dA else None
        dB = torch.empty(B.nnz, dtype=torch.float32, device=A.device) if need_dB else None
        dC = dC.contiguous().to(torch.float32)
        check(_lib.lib().spgemm_backward(self.handle, ctypes.byref(A.struct()),
                                         ctypes.byref(B.struct()), _ptr(C.row_ptr), _ptr(C.col),
                                         C.nnz, _ptr(dC), _ptr(dA), _ptr(dB), _ptr(ws), ws.numel(),
                                         _stream(stream)),
              "spgemm_backward")
        return dA, dB

    # --------------------------------------------------------- diagnostics
    def launches(self) -> int:
        """Kernel launches this plan has made since creation."""
        return int(_lib.lib().spgemm_launch_total(self.handle))

    def profile(self, on: bool = True) -> None:
        check(_lib.lib().spgemm_profile_enable(self.handle, 1 if on else 0), "spgemm_profile_enable")

    def profile_read(self) -> dict:
        """{kernel name: (total ms, timed launches)} since the last read."""
        L = _lib.lib()
        n = L.spgemm_kernel_count()
        ms = (ctypes.c_double * n)()
        cnt = (ctypes.c_int64 * n)()
        check(L.spgemm_profile_read(self.handle, ms, cnt, n), "spgemm_profile_read")
        return {L.spgemm_kernel_name(k).decode(): (ms[k], int(cnt[k])) for k in range(n) if cnt[k]}

    def status(self, ws: torch.Tensor, stream=None) -> int:
        st = ctypes.c_int()
        check(_lib.lib().spgemm_status(self.handle, _ptr(ws), _stream(stream), ctypes.byref(st)),
              "spgemm_status")
        return int(st.value)

    def check_status(self, ws: torch.Tensor, where: str = "device", stream=None) -> None:
        check(self.status(ws, stream), where)

    # ------------------------------------------------------------ whole product
    def spgemm(self, A: DeviceCSR, B: DeviceCSR, ws: torch.Tensor | None = None,
               stream=None, ip_row: torch.Tensor | None = None) -> DeviceCSR:
        """C = A*B through the one-call entry point (C allocated by torch).
        ``ip_row`` (int64, A.rows, on the device) receives the per-row
        intermediate-product counts of the call (Algorithm 1) when given."""
        if ws is None:
            ws = self.workspace(A, B)
        dev = A.device
        if ip_row is None:
            ip_row = torch.empty(A.rows, dtype=torch.int64, device=dev)
        row_nnz = torch.empty(A.rows, dtype=torch.int32, device=dev)
        row_ptr = torch.empty(A.rows + 1, dtype=torch.int32, device=dev)
        keep = {}

        def alloc(ctx, nnz, colp, valp):
            keep["col"] = torch.empty(int(nnz), dtype=torch.int32, device=dev)
            keep["val"] = torch.empty(int(nnz), dtype=torch.float32, device=dev)
            colp[0] = _ptr(keep["col"])
            valp[0] = _ptr(keep["val"])
            return 0

        cb = _lib.ALLOC_FN(alloc)
        nnz = ctypes.c_int64()
        check(_lib.lib().spgemm(self.handle, ctypes.byref(A.struct()), ctypes.byref(B.struct()),
                                _ptr(ws), ws.numel(), _ptr(ip_row), _ptr(row_nnz), _ptr(row_ptr),
                                cb, None, ctypes.byref(nnz), _stream(stream)),
              "spgemm")
        return DeviceCSR(A.rows, B.cols, row_ptr, keep["col"], keep["val"])

    def spgemm_blocks(self, A: DeviceCSR, B: DeviceCSR, max_block_nnz: int = 2**31 - 1,
                      ws: torch.Tensor | None = None, stream=None, out=None):
        """C = A*B as blocks of consecutive rows, each with int32 row pointers and
        at most ``max_block_nnz`` entries (for results beyond 2^31-1 entries).

        Returns (blocks, ip_total, nnz_total) with blocks a list of
        (row_begin, row_end, DeviceCSR). ``out`` may give preallocated blocks
        from an earlier call with the same operands (the same structure): the
        call then reuses their row ranges and never waits for the device
        (ip_total and nnz_total come back as None)."""
        if ws is None:
            ws = self.workspace(A, B)
        fresh = out is None
        ip_row, ip_total = self.count(A, B, ws, total=fresh, stream=stream)
        row_nnz, nnz_total = self.symbolic(A, B, ip_row, ws, total=fresh, stream=stream)
        bounds = split_rows(row_nnz, max_block_nnz) if fresh else [(r0, r1) for r0, r1, _ in out]
        blocks = []
        for q, (r0, r1) in enumerate(bounds):
            if out is not None:
                _, _, Cq = out[q]
                rp = Cq.row_ptr
            else:
                rp = None
            rp, tot = self.row_ptr(row_nnz[r0:r1], ws, out=rp, total=out is None, stream=stream)
            if out is not None:
                col, val = Cq.col, Cq.val
            else:
                col = torch.empty(tot, dtype=torch.int32, device=A.device)
                val = torch.empty(tot, dtype=torch.float32, device=A.device)
            self.numeric(A, B, ip_row, rp, ws, col, val, r0, r1, stream=stream)
            blocks.append((r0, r1, DeviceCSR(r1 - r0, B.cols, rp, col, val)))
        return blocks, ip_total, nnz_total


def partition_rows(ip_row, parts: int):
    """Contiguous row ranges [(r0, r1), ...], one per part (a rank), that cut
    the prefix sums of the per-row intermediate products (Alg. 1) as evenly
    as contiguous ranges allow: part p ends at the first row where the
    prefix reaches (p+1)/parts of the total. Rows of C are independent, so
    each rank multiplies its range of A by the whole of B with no exchange."""
    ip = np.asarray(ip_row.cpu() if isinstance(ip_row, torch.Tensor) else ip_row,
                    dtype=np.int64)
    if parts < 1:
        raise ValueError("parts must be >= 1")
    n = ip.shape[0]
    csum = np.cumsum(ip)
    total = int(csum[-1]) if n else 0
    cuts = [0]
    for p in range(1, parts):
        target = (total * p + parts - 1) // parts
        r = int(np.searchsorted(csum, target, side="left")) + 1 if total else (n * p) // parts
        cuts.append(min(max(r, cuts[-1]), n))
    cuts.append(n)
    return [(cuts[p], cuts[p + 1]) for p in range(parts)]


def split_rows(row_nnz: torch.Tensor, max_block_nnz: int):
    """Consecutive row ranges whose nnz sums stay <= max_block_nnz (host-side
    planning from the per-row counts of the allocation phase). The fewest
    blocks the limit allows, cut at even shares of the total so that no block
    is a small remainder (a launch over a small block still waits for its
    heaviest row); greedy filling where even cuts would break the limit."""
    counts = row_nnz.to(torch.int64).cpu().numpy()
    n = counts.shape[0]
    if n == 0:
        return [(0, 0)]
    if counts.max(initial=0) > max_block_nnz:
        raise ValueError("a single row exceeds the block limit")
    csum = np.cumsum(counts)
    total = int(csum[-1])
    nb = max(1, -(-total // max_block_nnz))
    if nb > 1:
        cuts = [0]
        for q in range(1, nb):
            r = int(np.searchsorted(csum, total * q / nb, side="left")) + 1
            cuts.append(min(max(r, cuts[-1] + 1), n))
        cuts.append(n)
        bounds = [(a, b) for a, b in zip(cuts, cuts[1:]) if b > a]
        sums = [int(csum[b - 1] - (csum[a - 1] if a else 0)) for a, b in bounds]
        if max(sums) <= max_block_nnz:
            return bounds
    bounds = []
    r0 = 0
    base = 0
    while r0 < n:
        r1 = int(np.searchsorted(csum, base + max_block_nnz, side="right"))
        r1 = max(r1, r0 + 1)
        bounds.append((r0, r1))
        base = int(csum[r1 - 1])
        r0 = r1
    return bounds