"""Row routing between kernels of one tier, against the oracle:

- the block hash tiers run rows of at most a quarter of their limit with a
  quarter-size table, rows of at most half with a half-size table and the
  rest with the full table (allocation: by IP against block_max_ip;
  accumulation: by nnz against block_max_nnz, fp32 and fp64 alike);
- the fp32 dense tier's rank-compacted kernel takes rows of at most 256 A
  entries (its expansion tile), the fallback dense-array kernel the others,
  with and without the row bitmap cache (rows of more than 256 entries reach
  the fp32 tier only when fp32_max_terms is raised, so that test compares
  within the fp32 summation bound of its longest row)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2512_12036_gb300 import DeviceCSR, Plan, gen
from parity import compare

pytestmark = pytest.mark.gpu


def grouped_b(n_cols, lengths, rows_per_len, seed):
    """B whose row groups have the given lengths (random distinct columns
    below n_cols, sorted); returns B and the row range of each group."""
    rng = np.random.default_rng(seed)
    r, c, groups, k = [], [], [], 0
    for L in lengths:
        groups.append((k, k + rows_per_len))
        for _ in range(rows_per_len):
            r.append(np.full(L, k))
            c.append(rng.choice(n_cols, size=L, replace=False))
            k += 1
    r, c = np.concatenate(r), np.concatenate(c)
    return gen.csr_from_coo(k, n_cols, r, c, gen.uniform_open_closed(rng, r.size)), groups


def rows_from_groups(spec, groups, k_rows, seed):
    """A with one row per (na, group) of spec: na distinct rows of B drawn from
    that group (group None: from all of B)."""
    rng = np.random.default_rng(seed)
    r, c = [], []
    for i, (na, g) in enumerate(spec):
        lo, hi = groups[g] if g is not None else (0, k_rows)
        r.append(np.full(na, i))
        c.append(rng.choice(np.arange(lo, hi), size=na, replace=False))
    r, c = np.concatenate(r), np.concatenate(c)
    return gen.csr_from_coo(len(spec), k_rows, r, c, gen.uniform_open_closed(rng, r.size))


def test_block_tiers_all_table_sizes():
    # B groups: rows of 8, 30, 50 and 120 entries over 200,000 columns, and
    # rows of 40 entries over 3,000 columns (products that meet)
    B1, g1 = grouped_b(200_000, [8, 30, 50, 120], 400, seed=5)
    B2, _ = grouped_b(3_000, [40], 400, seed=6)
    k1 = B1.rows
    B = gen.csr_from_coo(k1 + B2.rows, 200_000,
                         np.concatenate([np.repeat(np.arange(k1), np.diff(B1.row_ptr)),
                                         k1 + np.repeat(np.arange(B2.rows), np.diff(B2.row_ptr))]),
                         np.concatenate([B1.col, B2.col]), np.concatenate([B1.val, B2.val]))
    groups = g1 + [(k1, k1 + B2.rows)]
    spec = []
    for rep in range(6):
        spec += [(40, 1),       # fp32, IP 1200: small accumulation table, light allocation bin
                 (100, 2),      # fp32, IP 5000: full tables
                 (60, 3),       # fp32, IP 7200
                 (60, 1),       # fp32, IP 1800
                 (200, 0),      # fp64 (> 167 entries), IP 1600: small table
                 (300, 1),      # fp64, IP 9000: full tables
                 (150, 4),      # fp32, IP 6000 into 3000 columns (many products meet)
                 (250, 4),      # fp64, IP 10000 into 3000 columns
                 (240, 1)]      # fp64, IP 7200
    A = rows_from_groups(spec, groups, B.rows, seed=7)
    plan = Plan()
    ip, _ = oracle.ip_count(A, B)
    nnz = oracle.symbolic(A, B)
    o = plan.opts
    na = np.diff(A.row_ptr)
    block = (nnz > o["warp_max_nnz"]) & (nnz <= o["block_max_nnz"])
    small = block & (nnz <= o["block_max_nnz"] // 4)
    mid = block & ~small & (nnz <= o["block_max_nnz"] // 2)
    large = block & ~small & ~mid
    f64 = (na > o["fp32_max_terms"]) & (ip > o["fp32_max_terms"])
    # every accumulation class is present, and every allocation table size
    for m in (small, mid, large):
        assert (m & ~f64).sum() >= 6 and (m & f64).sum() >= 6
    sym_block = (ip > o["warp_max_ip"]) & (ip <= o["block_max_ip"])
    assert (sym_block & (ip <= o["block_max_ip"] // 4)).sum() >= 6
    assert (sym_block & (ip > o["block_max_ip"] // 4) & (ip <= o["block_max_ip"] // 2)).sum() >= 6
    assert (sym_block & (ip > o["block_max_ip"] // 2)).sum() >= 6
    dA, dB = DeviceCSR.from_host(A), DeviceCSR.from_host(B)
    C = plan.spgemm(dA, dB)
    torch.cuda.synchronize()
    compare(C.to_host(), oracle.spgemm(A, B))


@pytest.mark.parametrize("cache_mb", [0, 64])
def test_fp32_dense_rows_beyond_the_rank_tile(cache_mb):
    terms = 1200
    B, g = grouped_b(300_000, [60, 100], 1500, seed=11)
    spec = [(na, 0) for na in (200, 240, 300, 700, 1000)] * 3 + [(180, 1), (1300, 1)] * 2
    A = rows_from_groups(spec, g, B.rows, seed=12)
    plan = Plan(fp32_max_terms=terms, row_cache_mb=cache_mb)
    nnz = oracle.symbolic(A, B)
    ip, _ = oracle.ip_count(A, B)
    na = np.diff(A.row_ptr)
    dense = nnz > plan.opts["block_max_nnz"]              # dense accumulation tiers
    bitmap = dense & (ip > plan.opts["block_max_ip"])     # ... with a bitmap from the allocation phase
    f32 = ~((na > terms) & (ip > terms))
    assert ((dense & f32) & (na <= 256)).sum() >= 6       # the rank-compacted kernel's rows
    assert ((dense & f32) & (na <= 256) & ~bitmap).sum() >= 4   # ... some never cached
    assert ((dense & f32) & (na > 256)).sum() >= 6        # the fallback kernel's rows
    assert (dense & ~f32).sum() >= 2                      # fp64-bound rows beside them
    dA, dB = DeviceCSR.from_host(A), DeviceCSR.from_host(B)
    ws = plan.workspace(dA, dB)
    C = plan.spgemm(dA, dB, ws=ws)
    torch.cuda.synchronize()
    plan.check_status(ws, "rank tile routing")
    if cache_mb:
        assert plan.row_cache_rows(dA, dB, ws) == int(bitmap.sum())
    # fp32 summation of up to `terms` products: (terms + 1) u of sum |a||b|
    compare(C.to_host(), oracle.spgemm(A, B), tol=max(1e-5, (terms + 1) * 2.0 ** -24 * 1.01))
