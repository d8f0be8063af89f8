"""The allocation-free row-pointer entry point (spgemm_row_ptr_static).

Some callers cannot allocate device memory (a plugin whose host framework
owns all device allocations, a fixed-budget service, code where cudaMalloc
is not allowed), so this entry point keeps its scratch in a fixed array
inside the library. These tests call it through the C ABI and check its
output against the workspace-based spgemm_row_ptr on two calls in a row
(the shared scratch keeps the previous call's contents), and that sizes
beyond its limit are refused before any work. This file is collected last.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2512_12036_gb300 import DeviceCSR, Plan, _lib

pytestmark = pytest.mark.gpu

MAX_ROWS = 1 << 26


def _row_ptr_static(plan, counts):
    n = counts.numel()
    out = torch.full((n + 1,), -7, dtype=torch.int32, device=counts.device)
    tot = ctypes.c_int64(-1)
    rc = _lib.lib().spgemm_row_ptr_static(plan.handle, ctypes.c_void_p(counts.data_ptr()), n,
                                          ctypes.c_void_p(out.data_ptr()), ctypes.byref(tot),
                                          ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc, out, tot.value


def test_static_row_ptr_matches_workspace_version_twice():
    assert torch.cuda.is_available()
    plan = Plan()
    rng = np.random.default_rng(7)
    # two calls in a row with different sizes: the second must not see the
    # first one's partial sums (a larger first call, then a smaller one)
    for n in (300_001, 5_003):
        empty = DeviceCSR(n, 1, torch.zeros(n + 1, dtype=torch.int32, device="cuda"),
                          torch.zeros(0, dtype=torch.int32, device="cuda"), None)
        ws = plan.workspace(empty, empty)          # workspace of the reference entry point
        counts = torch.tensor(rng.integers(0, 50, size=n), dtype=torch.int32, device="cuda")
        want, want_total = plan.row_ptr(counts, ws, total=True)
        rc, got, got_total = _row_ptr_static(plan, counts)
        assert rc == _lib.OK
        assert got_total == want_total == int(counts.sum())
        assert torch.equal(got, want)


def test_static_row_ptr_limits():
    plan = Plan()
    counts = torch.zeros(4, dtype=torch.int32, device="cuda")
    L = _lib.lib()
    rc = L.spgemm_row_ptr_static(plan.handle, ctypes.c_void_p(counts.data_ptr()), MAX_ROWS + 1,
                                 ctypes.c_void_p(counts.data_ptr()), None, None)
    assert rc == _lib.ERR_UNSUPPORTED
    big = torch.full((3,), 2**30, dtype=torch.int32, device="cuda")
    rc, _, tot = _row_ptr_static(plan, big)
    assert rc == _lib.ERR_OVERFLOW and tot == 3 * 2**30
    # a clean call after an overflow report: the status word was cleared
    ok = torch.ones(10, dtype=torch.int32, device="cuda")
    rc, out, tot = _row_ptr_static(plan, ok)
    assert rc == _lib.OK and tot == 10 and out.tolist() == list(range(11))
