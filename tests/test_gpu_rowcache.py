"""The allocation phase's row bitmap cache (opts.row_cache_mb): products whose
dense rows read their columns from the cache match the oracle exactly as
without it, in both dense accumulation tiers (fp32 rank-compacted and the
fp64-bound tier with hot-column partial sums), with every dense row cached,
with only some rows cached (the rest recompute their occupancy), across
row blocks of the accumulation phase, and after a second allocation phase
on the same workspace (slots restart). A cache that no longer matches B is
reported on the status word."""
import numpy as np
import pytest
import torch

import oracle
from paper_2512_12036_gb300 import DeviceCSR, Plan, SpgemmError, gen
from parity import compare
from test_gpu_spgemm import hub_matrix

pytestmark = pytest.mark.gpu


def operands(bcols=70000):
    B = hub_matrix(3000, bcols, 15, heavy_rows=set(range(0, 3000, 11)), heavy_len=200,
                   light_deg=20)
    # dense rows with few A entries (fp32 tier: 150 entries on heavy rows of
    # B), with > 167 (fp64 tier: 400 entries), with more than one tile
    # (2500 entries, uncached-tile path), and light rows
    A = hub_matrix(300, 3000, 16, heavy_rows={1, 2, 100, 299}, heavy_len=2500, light_deg=30)
    rng = np.random.default_rng(17)
    heavy_b = np.arange(0, 3000, 11)
    r = [np.repeat(np.arange(A.rows), np.diff(A.row_ptr))]
    c = [A.col.astype(np.int64)]
    for i, n in [(i, 150) for i in range(10, 300, 13)] + [(i, 400) for i in range(5, 300, 29)]:
        if i in (1, 2, 100, 299):
            continue
        r.append(np.full(n, i))
        c.append(rng.choice(heavy_b, size=n, replace=False) if n <= heavy_b.size
                 else rng.choice(3000, size=n, replace=False))
    r, c = np.concatenate(r), np.concatenate(c)
    key = np.unique(r * 3000 + c)
    r, c = key // 3000, key % 3000
    A = gen.csr_from_coo(300, 3000, r, c, gen.uniform_open_closed(rng, r.size))
    return A, B


def dense_rows(A, B, plan):
    """(rows of C in a dense accumulation tier, rows of those that the
    allocation phase's bitmap tier handles (IP above the block tier), nnz)."""
    nnz = oracle.symbolic(A, B)
    ip, _ = oracle.ip_count(A, B)
    dense = nnz > plan.opts["block_max_nnz"]
    return int(dense.sum()), int((dense & (ip > plan.opts["block_max_ip"])).sum()), nnz


@pytest.mark.parametrize("bcols,cache_mb,splits,panel", [(70000, 64, 1, 16384),
                                                         (1_000_000, 1, 3, 16384),
                                                         (70000, 64, 4, 1024),
                                                         (70000, 64, 64, 1024),
                                                         (70000, 64, 0, 1024)])
def test_row_cache_parity(bcols, cache_mb, splits, panel):
    """splits > 1: each heavy row of the fp64-bound tier is cut into that
    many column ranges taken by different blocks (panel 1024: many passes
    per range); 0: ranges chosen per row by its product count."""
    A, B = operands(bcols)
    plan = Plan(row_cache_mb=cache_mb, dense_splits=splits, panel_cols=panel)
    ndense, nbitmap, nnz = dense_rows(A, B, plan)
    na = np.diff(A.row_ptr)
    assert ndense > 20 and (na[nnz > 8192] <= 167).any() and (na[nnz > 8192] > 1024).any()
    assert 0 < nbitmap < ndense        # dense rows with and without a bitmap from the allocation phase
    dA, dB = DeviceCSR.from_host(A), DeviceCSR.from_host(B)
    ws = plan.workspace(dA, dB)
    for rep in range(2):                      # a second allocation phase reuses the slots
        blocks, _, _ = plan.spgemm_blocks(dA, dB, ws=ws, max_block_nnz=int(nnz.sum()) // 3 + 1)
        torch.cuda.synchronize()
        plan.check_status(ws, "row cache")
        assert len(blocks) >= 3
        cached = plan.row_cache_rows(dA, dB, ws)
        slots_fit = (cache_mb << 20) // (4 * ((B.cols + 31) // 32))
        assert cached == min(nbitmap, slots_fit - 1) or cached == min(nbitmap, slots_fit)
        if bcols > 100000:
            assert 0 < cached < nbitmap         # the slots ran out
        else:
            assert cached == nbitmap
        rows = np.concatenate([np.diff(Cb.row_ptr.cpu().numpy()) for _, _, Cb in blocks])
        assert np.array_equal(rows, nnz)
        for r0, r1, Cb in blocks:
            compare(Cb.to_host(), oracle.spgemm(A, B, rows=np.arange(r0, r1)))


def test_row_cache_mismatch_reported():
    """Accumulation with a B whose columns differ from the allocation phase's:
    the cached bitmaps no longer match and the status word says so."""
    A, B = operands()
    rng = np.random.default_rng(3)
    B2 = gen.HostCSR(B.rows, B.cols, B.row_ptr.copy(),
                     np.sort(rng.integers(0, B.cols, size=B.nnz).astype(np.int32)),
                     B.val.copy())
    # keep every row sorted (the panel table of B stays usable)
    for i in range(B2.rows):
        s, e = B2.row_ptr[i], B2.row_ptr[i + 1]
        B2.col[s:e] = np.sort(rng.choice(B.cols, size=e - s, replace=False))
    plan = Plan(row_cache_mb=64)
    dA, dB, dB2 = DeviceCSR.from_host(A), DeviceCSR.from_host(B), DeviceCSR.from_host(B2)
    ws = plan.workspace(dA, dB)
    ip_row, _ = plan.count(dA, dB, ws)
    row_nnz, nnz = plan.symbolic(dA, dB, ip_row, ws)
    rp, _ = plan.row_ptr(row_nnz, ws)
    col = torch.empty(nnz, dtype=torch.int32, device="cuda")
    val = torch.empty(nnz, dtype=torch.float32, device="cuda")
    plan.numeric(dA, dB2, ip_row, rp, ws, col, val)
    torch.cuda.synchronize()
    with pytest.raises(SpgemmError):
        plan.check_status(ws, "stale row cache")


def test_row_cache_clustered_hot_columns():
    """More hot columns inside one table panel than the rank-compacted fp64
    tier has slots (2048): that pass is walked once per slot range."""
    rng = np.random.default_rng(41)
    rows, cols = 2000, 60000
    warm = rng.choice(16384, size=3000, replace=False)
    r, c = [], []
    for i in range(rows):
        cc = set(rng.choice(cols, size=rng.integers(5, 40), replace=False).tolist())
        cc |= set(warm[rng.random(warm.size) < 250 / rows].tolist())
        cc = np.array(sorted(cc))
        r.append(np.full(cc.size, i))
        c.append(cc)
    r, c = np.concatenate(r), np.concatenate(c)
    B = gen.csr_from_coo(rows, cols, r, c, gen.uniform_open_closed(rng, r.size))
    counts = np.bincount(B.col, minlength=cols)
    assert (counts[:16384] > 167).sum() > 2048
    A = hub_matrix(20, rows, 42, heavy_rows={0, 5, 19}, heavy_len=1200, light_deg=300)
    assert oracle.symbolic(A, B).max() > 8192
    for splits in (1, 2):
        plan = Plan(row_cache_mb=16, dense_splits=splits)
        dA, dB = DeviceCSR.from_host(A), DeviceCSR.from_host(B)
        ws = plan.workspace(dA, dB)
        C = plan.spgemm(dA, dB, ws=ws)
        torch.cuda.synchronize()
        plan.check_status(ws, "clustered hot columns")
        assert plan.row_cache_rows(dA, dB, ws) > 0
        compare(C.to_host(), oracle.spgemm(A, B))
