"""CPU-only checks of the C ABI: the library builds for sm_103a, loads, and
exports every function that include/spgemm.h declares."""
import ctypes

from paper_2512_12036_gb300 import _lib


def test_header_symbols_exported():
    L = _lib.lib()
    names = _lib.header_symbols()
    assert "spgemm_numeric" in names and "spgemm_count" in names
    for n in names:
        assert hasattr(L, n), n
        assert n in _lib.PROTOTYPES, f"{n} has no ctypes prototype"


def test_status_strings_and_defaults():
    L = _lib.lib()
    for code in range(0, 9):
        assert L.spgemm_status_string(code)
    o = _lib.OptsStruct()
    assert L.spgemm_opts_default(ctypes.byref(o)) == 0
    assert o.fp32_max_terms == 167 and o.esc_max == 32


def test_invalid_arguments_rejected_without_gpu():
    L = _lib.lib()
    assert L.spgemm_plan_create(None, None, 0) == _lib.ERR_INVALID
    n = ctypes.c_size_t()
    assert L.spgemm_workspace_bytes(None, None, None, ctypes.byref(n)) == _lib.ERR_INVALID


def test_every_entry_point_rejects_null_arguments():
    # NULL pointers and zero sizes everywhere: each status-returning call
    # reports ERR_INVALID before touching a device (destroying a NULL plan is
    # a no-op), so a caller's mistake never reaches a kernel
    L = _lib.lib()
    skip = {"spgemm_status_string", "spgemm_kernel_count", "spgemm_kernel_name",
            "spgemm_launch_total"}
    for name, (res, args) in _lib.PROTOTYPES.items():
        if name in skip:
            continue
        vals = []
        for a in args:
            if a in (ctypes.c_int, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t):
                vals.append(0)
            elif a is ctypes.c_float:
                vals.append(0.0)
            elif a is _lib.ALLOC_FN:
                vals.append(_lib.ALLOC_FN())
            else:
                vals.append(None)
        rc = getattr(L, name)(*vals)
        want = _lib.OK if name == "spgemm_plan_destroy" else _lib.ERR_INVALID
        assert rc == want, (name, rc)
    assert L.spgemm_launch_total(None) == 0
    assert L.spgemm_kernel_count() > 0 and L.spgemm_kernel_name(0)


def test_no_cpu_fallback_without_a_gpu():
    # the product path has no CPU fallback: without CUDA, making a plan or
    # moving a matrix to the device fails loudly
    import pytest
    import torch

    from paper_2512_12036_gb300 import DeviceCSR, Plan, gen
    if torch.cuda.is_available():
        pytest.skip("checks the behaviour of a machine without a GPU")
    with pytest.raises(Exception):
        Plan()
    with pytest.raises(Exception):
        DeviceCSR.from_host(gen.erdos_renyi(10, 2, seed=1))
