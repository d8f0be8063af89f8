"""Host logic of the benchmark (CPU): the clock summary (median and minimum
SM clock, power, and the throttle reasons active in any sample, from
nvidia-smi's CSV lines: index, sm, max sm, power, active mask, hw_slowdown,
hw_thermal_slowdown, sw_thermal_slowdown, sw_power_cap) and the per-tier
rows, products and compulsory bytes behind the roofline."""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def summary(lines):
    c = bench.ClockSampler(0)
    c.lines = lines
    return c.summary()


def test_clean_run():
    s = summary(["0, 2070, 2070, 489.8, 0x0, Not Active, Not Active, Not Active, Not Active",
                 "0, 2070, 2070, 501.2, 0x0, Not Active, Not Active, Not Active, Not Active",
                 "0, 2055, 2070, 510.0, 0x0, Not Active, Not Active, Not Active, Not Active"])
    assert s["sm_mhz"] == 2070 and s["sm_mhz_min"] == 2055 and s["sm_max_mhz"] == 2070
    assert s["power_w"] == 501.2 and s["reasons"] == [] and s["samples"] == 3


def test_reasons_from_any_sample():
    s = summary(["0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
                 "0, 1500, 2070, [N/A], 0x8, Active, Not Active, Active, Not Active",
                 "garbage line"])
    assert s["reasons"] == ["hw_slowdown", "sw_power_cap", "sw_thermal_slowdown"]
    assert s["samples"] == 2 and s["power_w"] == 1390.0 and s["sm_mhz_min"] == 1500


def test_unsampled():
    assert summary([])["reasons"] == ["unsampled"]


def test_tier_work_partitions_rows_and_products():
    # the per-tier rows, products and compulsory bytes behind the roofline:
    # each phase's tiers partition its rows, and the numeric bytes follow the
    # per-row formula 8 + 16|A_i| + 8 IP_i + 8 nnz_i
    import types

    import numpy as np

    import oracle
    from paper_2512_12036_gb300 import gen
    A = gen.rmat_symmetric(11, 16, seed=3)
    ip, _ = oracle.ip_count(A, A)
    ip = np.asarray(ip, dtype=np.int64)
    nnz = np.asarray(oracle.symbolic(A, A), dtype=np.int64)
    opts = {"esc_max": 32, "warp_max_ip": 1024, "block_max_ip": 4096, "warp_max_nnz": 128,
            "block_max_nnz": 1024, "fp32_max_terms": 40}
    w = bench.tier_work(types.SimpleNamespace(opts=opts), A, ip, nnz)
    na = np.diff(A.row_ptr.astype(np.int64))
    sym = [w[k] for k in ("sym_esc", "sym_warp", "sym_block", "sym_dense")]
    assert sum(t["rows"] for t in sym) == int((ip > 1).sum())
    assert sum(t["ip"] for t in sym) == int(ip[ip > 1].sum())
    num = [w[k] for k in w if k.startswith("num_")]
    assert sum(t["rows"] for t in num) == int((nnz > 0).sum())
    assert sum(t["nnz"] for t in num) == int(nnz.sum())
    assert sum(t["ip"] for t in num) == int(ip[nnz > 0].sum())
    for t in num:
        assert t["bytes"] == 8 * t["rows"] + 16 * t["a_entries"] + 8 * t["ip"] + 8 * t["nnz"]
    # both dense accumulation tiers are populated at these limits
    assert w["num_dense32"]["rows"] > 0 and w["num_dense64"]["rows"] > 0
    f64 = (na > 40) & (ip > 40)
    assert w["num_dense64"]["rows"] == int(((nnz > 1024) & f64 & ~((ip <= 32) & (na <= 32))).sum())
