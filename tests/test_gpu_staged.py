"""The staged block hash tier of the allocation phase (opts.stage_b: B-row
segments gathered by their row-pointer pairs and copied into shared memory
with cp.async before the inserts, a software form of the paper's range-2
near-memory access): the same structure and values as the oracle, on
inputs whose rows fill that tier, with rows spanning several tiles of A
entries, unsorted and repeated columns, and a malformed column reported."""
import numpy as np
import pytest
import torch

import oracle
from paper_2512_12036_gb300 import DeviceCSR, Plan, SpgemmError, gen
from parity import compare
from test_gpu_spgemm import hub_matrix

pytestmark = pytest.mark.gpu


def staged_rows(A, B, plan):
    ip, _ = oracle.ip_count(A, B)
    return int(((ip > plan.opts["warp_max_ip"]) & (ip <= 8192)).sum())


@pytest.mark.parametrize("case", ["rmat", "hubs", "long_a_rows", "unsorted_dups"])
def test_staged_block_tier_matches_oracle(case):
    plan = Plan(stage_b=1)
    if case == "rmat":
        A = gen.rmat_symmetric(12, 8, seed=3)
        B = A
    elif case == "hubs":
        B = hub_matrix(3000, 40000, 5, heavy_rows=set(range(0, 3000, 7)), heavy_len=300,
                       light_deg=12)
        A = hub_matrix(700, 3000, 6, heavy_rows={1, 50}, heavy_len=900, light_deg=60)
    elif case == "long_a_rows":
        # rows of A with more entries than one tile of the staging kernel (512)
        B = gen.random_csr(5000, 6000, 0.0008, seed=9)
        A = hub_matrix(200, 5000, 10, heavy_rows=set(range(0, 200, 3)), heavy_len=1500,
                       light_deg=5)
    else:
        B = gen.random_csr(2000, 3000, 0.004, seed=11, duplicates=True, unsorted=True)
        A = gen.random_csr(400, 2000, 0.05, seed=12, duplicates=True, unsorted=True)
    assert staged_rows(A, B, plan) > 10
    dA, dB = DeviceCSR.from_host(A), DeviceCSR.from_host(B)
    ws = plan.workspace(dA, dB)
    ip_row, _ = plan.count(dA, dB, ws)
    row_nnz, _ = plan.symbolic(dA, dB, ip_row, ws)
    torch.cuda.synchronize()
    assert np.array_equal(row_nnz.cpu().numpy().astype(np.int64), oracle.symbolic(A, B))
    C = plan.spgemm(dA, dB, ws=ws)
    torch.cuda.synchronize()
    compare(C.to_host(), oracle.spgemm(A, B))
    # the same structure as the unstaged allocation phase
    C0 = Plan().spgemm(dA, dB)
    assert torch.equal(C0.row_ptr, C.row_ptr) and torch.equal(C0.col, C.col)


def test_staged_block_tier_reports_bad_column():
    plan = Plan(stage_b=1)
    B = hub_matrix(3000, 40000, 5, heavy_rows=set(range(0, 3000, 7)), heavy_len=300,
                   light_deg=12)
    A = hub_matrix(300, 3000, 6, heavy_rows=set(), heavy_len=0, light_deg=60)
    assert staged_rows(A, B, plan) > 10
    col = B.col.copy()
    col[B.row_ptr[7] + 3] = 40000 + 5          # outside B's columns
    Bbad = gen.HostCSR(B.rows, B.cols, B.row_ptr, col, B.val)
    dA, dB = DeviceCSR.from_host(A), DeviceCSR.from_host(Bbad)
    ws = plan.workspace(dA, dB)
    ip_row, _ = plan.count(dA, dB, ws)
    with pytest.raises(SpgemmError):
        plan.symbolic(dA, dB, ip_row, ws)
