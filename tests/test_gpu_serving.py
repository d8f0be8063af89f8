"""Served requests on the GPU: a mix of graph-contraction, MCL-expansion and
random A*B requests submitted concurrently into the continuous-batching
server; every result equals the same request computed alone (exact
structure) and both are within the SpGEMM tolerance of the oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_2512_12036_gb300 import DeviceCSR, gen, serving
from parity import compare

pytestmark = pytest.mark.gpu


def mixed_requests(seed):
    rng = np.random.default_rng(seed)
    out = []
    A = gen.rmat_symmetric(12, 8, seed=seed)
    S = gen.assignment_matrix(A.rows, 256, seed=seed + 1)
    out.append(("contract_StA", gen.transpose_structure(S), A))
    M = gen.rmat_symmetric(11, 8, seed=seed + 2, self_loops=True)
    out.append(("mcl_expand", M, M))
    for q in range(10):
        n = int(np.exp(rng.uniform(np.log(1000), np.log(20000))))
        d = rng.uniform(4, 32)
        if q % 2:
            Aq = gen.erdos_renyi(n, d, seed=seed + 10 + q)
            Bq = gen.erdos_renyi(n, d, seed=seed + 11 + q)
        else:
            sc = int(np.ceil(np.log2(n)))
            Aq = gen.rmat_symmetric(sc, max(1, int(d // 2)), seed=seed + 10 + q)
            Bq = gen.rmat_symmetric(sc, max(1, int(d // 2)), seed=seed + 11 + q)
        out.append((f"mixed{q}", Aq, Bq))
    return out


def test_results_same_alone_and_in_the_mix():
    reqs_h = mixed_requests(3)
    dev = [(t, DeviceCSR.from_host(A), DeviceCSR.from_host(B)) for t, A, B in reqs_h]
    alone = serving.run_plain([serving.Request(A=A, B=B, tag=t) for t, A, B in dev],
                              np.zeros(len(dev)))
    srv = serving.gpu_server(slots=4, budget_bytes=2 << 30)
    mixed = serving.run_served(srv, [serving.Request(A=A, B=B, tag=t) for t, A, B in dev],
                               np.zeros(len(dev)))
    srv.close()
    assert srv.adm.peak <= 2 << 30
    for (t, Ah, Bh), ra, rm in zip(reqs_h, alone, mixed):
        assert rm.error == 0, t
        ref = oracle.spgemm(Ah, Bh)
        (_, _, Ca), = ra.result
        Cm = rm.result
        ha, hm = Ca.to_host(), Cm.to_host()
        assert np.array_equal(ha.row_ptr, hm.row_ptr) and np.array_equal(ha.col, hm.col), t
        compare(ha, ref)
        compare(hm, ref)
    torch.cuda.synchronize()
