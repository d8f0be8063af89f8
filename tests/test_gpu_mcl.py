"""MCL on the GPU against the oracle, iteration by iteration: the expansion
against the oracle's product (exact structure, values within the SpGEMM
tolerance), then the prune/top-k/inflate/normalise step against the oracle's
step applied to the same fp32 expansion (decisions in fp32 on both sides:
exact structure; values within 4 fp32 ulps)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2512_12036_gb300 import DeviceCSR, Plan, gen
from paper_2512_12036_gb300.mcl import mcl_step, normalise_rows
from parity import compare

pytestmark = pytest.mark.gpu


def graph(scale, ef, seed):
    return gen.rmat_symmetric(scale, ef, seed=seed, self_loops=True)


def ulp_close(got, want, ulps=4):
    want32 = want.astype(np.float32)
    tol = ulps * np.spacing(np.abs(want32)).astype(np.float64)
    return np.all(np.abs(got.astype(np.float64) - want) <= tol + 1e-45)


@pytest.mark.parametrize("order", [0, 1])
def test_mcl_iterations_against_oracle(order):
    plan = Plan()
    G = graph(10, 8, seed=4)
    Gd = DeviceCSR.from_host(G)
    M = normalise_rows(plan, Gd)
    Mh = M.to_host()
    want = oracle.row_normalise(G)
    assert np.array_equal(Mh.col, G.col) and ulp_close(Mh.val, want)
    for it in range(4):
        E = plan.spgemm(M, M)
        Eh = E.to_host()
        compare(Eh, oracle.spgemm(Mh, Mh))
        M = mcl_step(plan, E, 1e-4, 32, 2.0, order)
        Mh = M.to_host()
        ref = oracle.mcl_step(Eh, 1e-4, 32, 2.0, order)
        assert np.array_equal(Mh.row_ptr.astype(np.int64), ref.row_ptr)
        assert np.array_equal(Mh.col, ref.col)
        assert ulp_close(Mh.val, ref.val)
        counts = np.diff(Mh.row_ptr)
        assert counts.max(initial=0) <= 32
        sums = np.add.reduceat(Mh.val.astype(np.float64), Mh.row_ptr[:-1][counts > 0]) if Mh.nnz else []
        assert np.allclose(sums, 1.0, atol=1e-5)


def test_mcl_step_long_rows_and_ties():
    plan = Plan()
    rng = np.random.default_rng(3)
    # rows longer than one warp's capacity (block kernel) and many equal values
    rows, cols = 6, 5000
    r = np.repeat(np.arange(rows), 3000)
    c = np.concatenate([rng.choice(cols, 3000, replace=False) for _ in range(rows)])
    v = rng.choice(np.array([1e-5, 2e-4, 5e-4, 5e-4, 1e-3], dtype=np.float32), size=r.size)
    E = gen.csr_from_coo(rows, cols, r, c, v)
    for order in (0, 1):
        got = mcl_step(plan, DeviceCSR.from_host(E), 1e-4, 32, 2.0, order).to_host()
        ref = oracle.mcl_step(E, 1e-4, 32, 2.0, order)
        assert np.array_equal(got.col, ref.col) and ulp_close(got.val, ref.val)


def test_mcl_expansions_served_match_plain_and_oracle():
    """Markov clustering with every expansion a request to the continuous-
    batching server: each served expansion against the oracle on its own
    input, and the clustering after three iterations against the plain
    (one spgemm call per expansion) run."""
    from paper_2512_12036_gb300 import serving
    from paper_2512_12036_gb300.mcl import markov_cluster, markov_cluster_served

    plan = Plan()
    G = graph(11, 8, seed=5)
    Gd = DeviceCSR.from_host(G)
    srv = serving.gpu_server(slots=2, budget_bytes=1 << 30, keep_results=True,
                             count_ws_bytes=64 << 20, max_rows=1 << 16)
    try:
        res_s, reqs = markov_cluster_served(srv, plan, Gd, iterations=3)
    finally:
        srv.close()
    assert len(reqs) == 3 and all(r.error == 0 for r in reqs)
    for req in reqs:
        Mh = req.A.to_host()
        compare(req.result.to_host(), oracle.spgemm(Mh, Mh))
    res_p = markov_cluster(plan, Gd, iterations=3)
    assert res_s.ip_history == res_p.ip_history
    assert res_s.nnz_history == res_p.nnz_history
    a, b = res_s.Mt.to_host(), res_p.Mt.to_host()
    assert np.array_equal(a.row_ptr, b.row_ptr) and np.array_equal(a.col, b.col)
    assert np.allclose(a.val, b.val, rtol=1e-4, atol=1e-7)
