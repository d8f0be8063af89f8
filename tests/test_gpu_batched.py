"""Batched products: the graph-captured spgemm_batched path against the
plain path and the oracle, per problem and as one block-diagonal product;
capacity refusal; the autotuner's choice keeps exact structure."""
import numpy as np
import pytest
import torch

import oracle
from paper_2512_12036_gb300 import DeviceCSR, Plan, SpgemmError, gen, _lib
from paper_2512_12036_gb300.batched import BatchedSpGEMM, autotune, stack_problems
from parity import compare

pytestmark = pytest.mark.gpu


def problems(num, seed):
    batch = gen.gnn_batch(num, seed=seed, n_min=32, n_max=400, features=256, k=32)
    out = []
    for b in range(num):
        s, e = int(batch.node_off[b]), int(batch.node_off[b + 1])
        Ab = batch.A
        rp = Ab.row_ptr[s:e + 1].astype(np.int64)
        cols = Ab.col[rp[0]:rp[-1]] - s
        A_b = gen.HostCSR(e - s, e - s, (rp - rp[0]).astype(np.int32), cols.astype(np.int32),
                          Ab.val[rp[0]:rp[-1]].copy())
        xr = batch.X.row_ptr[s:e + 1].astype(np.int64)
        X_b = gen.HostCSR(e - s, 256, (xr - xr[0]).astype(np.int32), batch.X.col[xr[0]:xr[-1]].copy(),
                          batch.X.val[xr[0]:xr[-1]].copy())
        out.append((A_b, X_b))
    return out


def test_batched_graph_equals_plain_and_oracle():
    probs = problems(24, seed=1)
    A, B, row_off, _ = stack_problems(probs)
    dA, dB = DeviceCSR.from_host(A), DeviceCSR.from_host(B)
    bs = BatchedSpGEMM(dA, dB)
    bs.capture()
    for _ in range(2):                       # replays are repeatable
        bs.run()
        C = bs.result().to_host()
        compare(C, oracle.spgemm(A, B))
    plan = Plan()
    for q, (Ab, Xb) in enumerate(probs):     # each stacked block equals its own product
        Cq = plan.spgemm(DeviceCSR.from_host(Ab), DeviceCSR.from_host(Xb)).to_host()
        r0, r1 = int(row_off[q]), int(row_off[q + 1])
        s, e = C.row_ptr[r0], C.row_ptr[r1]
        assert np.array_equal(C.row_ptr[r0:r1 + 1] - s, Cq.row_ptr)
        assert np.array_equal(C.col[s:e], Cq.col)
        ref = oracle.spgemm(Ab, Xb)
        assert np.all(np.abs(C.val[s:e] - ref.val) <= 1e-5 * ref.bound)


def test_batched_capacity_refused():
    probs = problems(4, seed=2)
    A, B, _, _ = stack_problems(probs)
    dA, dB = DeviceCSR.from_host(A), DeviceCSR.from_host(B)
    need = oracle.spgemm(A, B).nnz
    bs = BatchedSpGEMM(dA, dB, capacity=need - 1)
    bs.col.fill_(-5)
    bs.enqueue()
    with pytest.raises(SpgemmError) as e:
        bs.result()
    assert e.value.code == _lib.ERR_BUDGET
    assert int(bs.nnz_dev.item()) == need
    assert bool((bs.col == -5).all())


def test_autotune_keeps_structure():
    probs = problems(16, seed=3)
    A, B, _, _ = stack_problems(probs)
    dA, dB = DeviceCSR.from_host(A), DeviceCSR.from_host(B)
    bs, opts, timings = autotune(dA, dB, reps=2)
    assert len(timings) >= 4 and all(t > 0 for t in timings.values())
    bs.run()
    compare(bs.result().to_host(), oracle.spgemm(A, B))
