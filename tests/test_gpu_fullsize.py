"""GPU parity at the benchmark's full size: C = A*A for the R-MAT scale 20
matrix (ef 16, seed 2; nnz(C) = 2.38e10, produced in even row blocks of at
most 2^31-1 entries, as the benchmark runs it) and both products of the
contraction S^T*A*S (Algorithm 7).

Checked against the oracle: every row's entry count (the oracle's full
allocation phase, exact), and columns and values of sampled rows (the
heaviest rows by intermediate products, uniformly drawn rows and the first
rows; values within 1e-5 * sum|a||b|)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2512_12036_gb300 import DeviceCSR, Plan, gen
from contraction import assignment_labels, label_scatter
from parity import compare

pytestmark = pytest.mark.gpu


def rows_of_blocks(blocks, rows):
    """Host CSR of the given rows (ascending) of a list of (r0, r1, DeviceCSR)
    blocks; only those rows are copied off the device."""
    rows = np.asarray(rows, dtype=np.int64)
    cols, vals, counts = [], [], []
    for r0, r1, Cb in blocks:
        sel = rows[(rows >= r0) & (rows < r1)] - r0
        if sel.size == 0:
            continue
        sel_t = torch.from_numpy(sel).to(Cb.row_ptr.device)
        s = Cb.row_ptr[sel_t].long()
        e = Cb.row_ptr[sel_t + 1].long()
        n = e - s
        idx = torch.repeat_interleave(s, n) + (torch.arange(int(n.sum().item()), device=s.device)
                                              - torch.repeat_interleave(torch.cumsum(n, 0) - n, n))
        cols.append(Cb.col[idx].cpu().numpy())
        vals.append(Cb.val[idx].cpu().numpy())
        counts.append(n.cpu().numpy())
    counts = np.concatenate(counts)
    rp = np.concatenate([[0], np.cumsum(counts)]).astype(np.int32)
    return gen.HostCSR(rows.size, blocks[0][2].cols, rp, np.concatenate(cols),
                       np.concatenate(vals))


def sample_rows(ip, n, seed):
    rng = np.random.default_rng(seed)
    heavy = np.argsort(ip)[-300:]
    uniform = rng.choice(n, size=2000, replace=False)
    return np.unique(np.concatenate([heavy, uniform, np.arange(1000)]))


def test_rmat20_full_size_parity():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    A_h = gen.rmat_symmetric(20, 16, 0.57, 0.19, 0.19, seed=2)
    A = DeviceCSR.from_host(A_h)
    # the plan the benchmark times: the allocation phase's row bitmaps kept
    # for every dense row that fits beside the output
    import bench
    plan = Plan(row_cache_mb=bench.row_cache_size(Plan(), A, A, A.device))
    ws = plan.workspace(A, A)
    blocks, ip_total, nnz_total = plan.spgemm_blocks(A, A, ws=ws)
    torch.cuda.synchronize()
    plan.check_status(ws, "A*A")
    assert plan.row_cache_rows(A, A, ws) > 300000
    assert len(blocks) > 1                          # beyond int32 row pointers
    # every row's entry count against the oracle's allocation phase
    got_nnz = np.concatenate([np.diff(Cb.row_ptr.cpu().numpy().astype(np.int64))
                              for _, _, Cb in blocks])
    ref_nnz = oracle.symbolic(A_h, A_h).astype(np.int64)
    assert np.array_equal(got_nnz, ref_nnz)
    assert int(ref_nnz.sum()) == nnz_total
    ip, total = oracle.ip_count(A_h, A_h)
    assert int(total) == ip_total
    # columns and values of sampled rows
    rows = sample_rows(ip, A_h.rows, seed=1)
    got = rows_of_blocks(blocks, rows)
    ref = oracle.spgemm(A_h, A_h, rows=rows)
    compare(got, ref, rows=np.arange(rows.size))
    del blocks, ws
    torch.cuda.empty_cache()
    plan = Plan()

    # contraction S^T * A (the first factor of S^T A S)
    clusters = A_h.rows // 16
    S_h = gen.assignment_matrix(A_h.rows, clusters, seed=3)
    St_h = gen.transpose_structure(S_h)
    St = DeviceCSR.from_host(St_h)
    T_blocks, _, _ = plan.spgemm_blocks(St, A)
    torch.cuda.synchronize()
    ipt, _ = oracle.ip_count(St_h, A_h)
    rows = sample_rows(ipt, St_h.rows, seed=2)
    compare(rows_of_blocks(T_blocks, rows), oracle.spgemm(St_h, A_h, rows=rows),
            rows=np.arange(rows.size))

    # second product (S^T A) * S, as the benchmark runs it: sampled rows
    # against the oracle on the first product's actual output, and every
    # entry against A's entries scattered by cluster labels (fp64)
    assert len(T_blocks) == 1
    T = T_blocks[0][2]
    S = DeviceCSR.from_host(S_h)
    C2_blocks, _, nnz2 = plan.spgemm_blocks(T, S)
    torch.cuda.synchronize()
    assert len(C2_blocks) == 1
    T_h = T.to_host()
    C2_h = C2_blocks[0][2].to_host()
    ip2, _ = oracle.ip_count(T_h, S_h)
    rows = sample_rows(ip2, T_h.rows, seed=3)
    compare(rows_of_blocks(C2_blocks, rows), oracle.spgemm(T_h, S_h, rows=rows),
            rows=np.arange(rows.size))
    rp, col, val, absum = label_scatter(A_h, assignment_labels(S_h), clusters)
    assert nnz2 == col.size
    assert np.array_equal(C2_h.row_ptr.astype(np.int64), rp)
    assert np.array_equal(C2_h.col, col)
    assert (np.abs(C2_h.val.astype(np.float64) - val) <= 2e-5 * absum).all()
