"""Seeded random products and their backward against the oracle under random
plan options.

Small panels (1024 columns), low block-tier limits and low hash-tier limits
push small matrices through the multi-pass, multi-panel and word-range
paths of the dense tiers, the bucket sort and its fallback, and every
expansion form; shapes, densities, hub rows, repeated and unsorted columns
vary with the seed."""
import numpy as np
import pytest
import torch

import oracle
from paper_2512_12036_gb300 import DeviceCSR, Plan, gen
from parity import compare

pytestmark = pytest.mark.gpu

OPTION_SETS = [
    {},
    {"panel_cols": 1024, "block_max_nnz": 512, "block_max_ip": 1024},
    {"panel_cols": 2048, "block_max_nnz": 1024, "warp_max_nnz": 128, "warp_max_ip": 256},
    {"panel_cols": 1024, "block_max_nnz": 2048, "esc_max": 16, "fp32_max_terms": 40},
]


def random_problem(seed):
    rng = np.random.default_rng(seed)
    m = int(rng.integers(1, 400))
    k = int(rng.integers(1, 600))
    n = int(rng.choice([50, 3000, 20000, 70000]))
    hubs_a = set(rng.choice(m, size=min(m, int(rng.integers(0, 4))), replace=False).tolist())
    hubs_b = set(rng.choice(k, size=min(k, int(rng.integers(0, 30))), replace=False).tolist())

    def build(rows, cols, hubs, deg, heavy):
        r, c = [], []
        for i in range(rows):
            d = min(cols, heavy if i in hubs else int(rng.integers(0, deg + 1)))
            cc = rng.choice(cols, size=d, replace=False)
            r.append(np.full(d, i))
            c.append(cc)
        return np.concatenate(r), np.concatenate(c)

    ra, ca = build(m, k, hubs_a, 12, int(rng.integers(100, 600)))
    rb, cb = build(k, n, hubs_b, 30, int(rng.integers(200, 3000)))
    if rng.random() < 0.3:                                 # repeated columns
        extra = rng.integers(0, rb.size, size=rb.size // 20 + 1) if rb.size else np.zeros(0, int)
        rb, cb = np.concatenate([rb, rb[extra]]), np.concatenate([cb, cb[extra]])
    va = gen.uniform_open_closed(rng, ra.size)
    vb = gen.uniform_open_closed(rng, rb.size)
    if rng.random() < 0.3:
        va = va * np.where(rng.random(ra.size) < 0.5, -1, 1).astype(np.float32)
    A = gen.csr_from_coo(m, k, ra, ca, va)
    B = gen.csr_from_coo(k, n, rb, cb, vb)
    if rng.random() < 0.2:                                 # unsorted rows of B
        col = B.col.copy()
        val = B.val.copy()
        for i in range(k):
            s, e = B.row_ptr[i], B.row_ptr[i + 1]
            p = rng.permutation(e - s) + s
            col[s:e], val[s:e] = col[p], val[p]
        B = gen.HostCSR(k, n, B.row_ptr, col, val)
    return A, B


@pytest.mark.parametrize("seed", range(120))
def test_random_product(seed):
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    A, B = random_problem(seed)
    plan = Plan(**OPTION_SETS[seed % len(OPTION_SETS)])
    C = plan.spgemm(DeviceCSR.from_host(A), DeviceCSR.from_host(B))
    torch.cuda.synchronize()
    compare(C.to_host(), oracle.spgemm(A, B))


@pytest.mark.parametrize("seed", range(40))
def test_random_backward(seed):
    from test_gpu_backward import check_backward
    A, B = random_problem(1000 + seed)
    check_backward(Plan(**OPTION_SETS[seed % len(OPTION_SETS)]), A, B, seed=seed)
