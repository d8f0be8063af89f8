"""GPU parity of spgemm_backward against the oracle's fp64 gradients, and of
the autograd wrapper against a dense torch reference.

Tolerance per gradient entry: 1e-5 * (sum of |terms|), where the sum of
|terms| is the oracle's backward applied to |A|, |B| and |dC|."""
import numpy as np
import pytest
import torch

import oracle
from paper_2512_12036_gb300 import DeviceCSR, Plan, gen
from paper_2512_12036_gb300.autograd import spgemm as spgemm_ag

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def plan():
    return Plan()


def _abs(M):
    return gen.HostCSR(M.rows, M.cols, M.row_ptr, M.col, np.abs(M.val))


def check_backward(plan, A, B, seed=0, need=(True, True)):
    dA_dev, dB_dev = DeviceCSR.from_host(A), DeviceCSR.from_host(B)
    C = plan.spgemm(dA_dev, dB_dev)
    Ch = C.to_host()
    ref = oracle.spgemm(A, B)
    assert np.array_equal(Ch.col, ref.col)
    dC = np.random.default_rng(seed).standard_normal(ref.nnz).astype(np.float32)
    ws = plan.backward_workspace(dA_dev, dB_dev)
    gA, gB = plan.backward(dA_dev, dB_dev, C, torch.from_numpy(dC).cuda(), *need, ws=ws)
    plan.check_status(ws, "backward")
    rA, rB = oracle.backward(A, B, ref, dC.astype(np.float64))
    bA, bB = oracle.backward(_abs(A), _abs(B), ref, np.abs(dC).astype(np.float64))
    if need[0]:
        err = np.abs(gA.cpu().numpy().astype(np.float64) - rA)
        assert np.all(err <= 1e-5 * bA + 1e-30), float((err - 1e-5 * bA).max())
    else:
        assert gA is None
    if need[1]:
        err = np.abs(gB.cpu().numpy().astype(np.float64) - rB)
        assert np.all(err <= 1e-5 * bB + 1e-30), float((err - 1e-5 * bB).max())
    else:
        assert gB is None


def test_backward_gnn_shaped(plan):
    batch = gen.gnn_batch(6, seed=3, n_min=64, n_max=300, features=256, k=32)
    check_backward(plan, batch.A, batch.X, seed=1)


def test_backward_dense_lookup_single_sided(plan):
    batch = gen.gnn_batch(3, seed=4, n_min=64, n_max=128)
    check_backward(plan, batch.A, batch.X, seed=2, need=(True, False))
    check_backward(plan, batch.A, batch.X, seed=3, need=(False, True))


def test_backward_hash_tiers(plan):
    # B with many columns: warp and block hash tiers
    A = gen.random_csr(400, 300, 0.05, 5, signed=True)
    B = gen.random_csr(300, 20000, 0.01, 6, signed=True, duplicates=True)
    check_backward(plan, A, B, seed=4)


def test_backward_panel_tier(plan):
    # rows of C with > 8192 entries: dense panels (sorted and unsorted B)
    A = gen.random_csr(20, 600, 0.5, 7)
    B = gen.random_csr(600, 70000, 0.004, 8)
    assert oracle.symbolic(A, B).max() > 8192
    check_backward(plan, A, B, seed=5)
    Bu = gen.random_csr(600, 70000, 0.004, 8, unsorted=True)
    check_backward(plan, A, Bu, seed=6)


def test_autograd_against_dense_torch(plan):
    A = gen.random_csr(50, 40, 0.1, 9, signed=True)
    B = gen.random_csr(40, 60, 0.1, 10, signed=True)
    dA_s, dB_s = DeviceCSR.from_host(A), DeviceCSR.from_host(B)
    a = dA_s.val.clone().requires_grad_(True)
    b = dB_s.val.clone().requires_grad_(True)
    C = spgemm_ag(a, b, dA_s, dB_s, plan)
    w = torch.randn(C.nnz, device="cuda")
    (C.val * w).sum().backward()
    # dense reference in fp64 (repeated entries summed, gradients per stored entry)
    ra = torch.repeat_interleave(torch.arange(A.rows), torch.from_numpy(np.diff(A.row_ptr)).long())
    rb = torch.repeat_interleave(torch.arange(B.rows), torch.from_numpy(np.diff(B.row_ptr)).long())
    av = a.detach().cpu().double().requires_grad_(True)
    bv = b.detach().cpu().double().requires_grad_(True)
    DA = torch.zeros(A.rows, A.cols, dtype=torch.float64).index_put((ra, torch.from_numpy(A.col).long()), av, accumulate=True)
    DB = torch.zeros(B.rows, B.cols, dtype=torch.float64).index_put((rb, torch.from_numpy(B.col).long()), bv, accumulate=True)
    Ch = C.to_host()
    rc = torch.repeat_interleave(torch.arange(Ch.rows), torch.from_numpy(np.diff(Ch.row_ptr)).long())
    Dc = (DA @ DB)[rc, torch.from_numpy(Ch.col).long()]
    (Dc * w.cpu().double()).sum().backward()
    assert torch.allclose(a.grad.cpu().double(), av.grad, rtol=1e-5, atol=1e-6)
    assert torch.allclose(b.grad.cpu().double(), bv.grad, rtol=1e-5, atol=1e-6)
