"""GPU parity of bulk neighbourhood sampling (Section IV-C) against the CPU
oracle: SAMPLE bit-exact for the same uniforms (draws kept clear of
rounding ties, checked through the oracle's boundary gap), column selection
exact, and a two-layer pipeline whose products are single-term (so exact):
P = Q*A, SAMPLE, selection, EXTRACT = P*S."""
import numpy as np
import pytest
import torch

from oracle import sampling as osamp
from paper_2512_12036_gb300 import DeviceCSR, Plan, gen
from paper_2512_12036_gb300 import sampling

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def plan():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return Plan()


def random_P(n_rows, max_len, seed, ncols=5000, long_rows=()):
    rng = np.random.default_rng(seed)
    lens = rng.integers(0, max_len, size=n_rows)
    for r in long_rows:
        lens[r] = 3000
    rp = np.concatenate([[0], np.cumsum(lens)]).astype(np.int32)
    col = np.concatenate([np.sort(rng.choice(ncols, size=l, replace=False)) for l in lens])
    val = rng.uniform(0.01, 1.0, size=col.size).astype(np.float32)
    val[rng.random(col.size) < 0.05] = 0.0
    return gen.HostCSR(n_rows, ncols, rp, col.astype(np.int32), val)


@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("s", [1, 10, 32])
def test_sample_rows_matches_oracle(plan, mode, s):
    Ph = random_P(400, 200, seed=10 * mode + s, long_rows=(3, 77))
    u = np.random.default_rng(s + mode).random((400, s)).astype(np.float32)
    ref_rp, ref_col, _, gap = osamp.sample_rows(Ph.row_ptr, Ph.col, Ph.val, s, u, mode)
    assert gap > 1e-9                       # no draw within rounding of a boundary
    Q = sampling.sample_rows(DeviceCSR.from_host(Ph), s, torch.from_numpy(u).cuda(), mode, plan)
    Qh = Q.to_host()
    assert np.array_equal(Qh.row_ptr, ref_rp)
    assert np.array_equal(Qh.col, ref_col)
    assert (Qh.val == 1.0).all()


def test_sample_rows_edge_cases(plan):
    # empty matrix; rows of zero weight (uniform fallback); s outside 1..32
    P0 = DeviceCSR.from_host(gen.HostCSR(0, 10, np.zeros(1, np.int32), np.zeros(0, np.int32),
                                         np.zeros(0, np.float32)))
    Q0 = sampling.sample_rows(P0, 4, torch.zeros(0, 4, device="cuda"), 1, plan)
    assert Q0.rows == 0 and Q0.nnz == 0
    Ph = random_P(50, 100, seed=3)
    Ph.val[:] = 0.0
    u = np.random.default_rng(1).random((50, 6)).astype(np.float32)
    ref = osamp.sample_rows(Ph.row_ptr, Ph.col, Ph.val, 6, u, 1)
    Qh = sampling.sample_rows(DeviceCSR.from_host(Ph), 6, torch.from_numpy(u).cuda(), 1,
                              plan).to_host()
    assert np.array_equal(Qh.col, ref[1]) and np.array_equal(Qh.row_ptr, ref[0])
    from paper_2512_12036_gb300 import SpgemmError
    with pytest.raises(SpgemmError):
        sampling.sample_rows(DeviceCSR.from_host(Ph), 33, torch.zeros(50, 33, device="cuda"), 0,
                             plan)


def test_select_columns(plan):
    Qh = random_P(300, 40, seed=5, ncols=2000)
    S, F = sampling.select_columns(DeviceCSR.from_host(Qh), plan)
    vertices, rank = osamp.select_columns(Qh.col, 2000)
    Sh, Fh = S.to_host(), F.to_host()
    assert S.cols == vertices.size and F.rows == vertices.size
    assert np.array_equal(Sh.row_ptr, rank)
    assert np.array_equal(Sh.col, np.arange(vertices.size))
    assert np.array_equal(Fh.row_ptr, np.arange(vertices.size + 1))
    assert np.array_equal(Fh.col, vertices)


def dense_of(H):
    D = np.zeros((H.rows, H.cols))
    for i in range(H.rows):
        s, e = H.row_ptr[i], H.row_ptr[i + 1]
        np.add.at(D[i], H.col[s:e], H.val[s:e].astype(np.float64))
    return D


@pytest.mark.parametrize("mode", [0, 1])
def test_two_layer_pipeline(plan, mode):
    n = 4000
    Ah = gen.erdos_renyi(n, 12.0, seed=21)
    A = DeviceCSR.from_host(Ah)
    Ad = dense_of(Ah)
    batch = np.sort(np.random.default_rng(2).choice(n, size=256, replace=False))
    adj, qs, us = sampling.sample_layers(A, batch, [10, 5], plan, mode=mode, seed=3)
    rows = batch
    for l, (A_l, Qn, u) in enumerate(zip(adj, qs[1:], us)):
        # P = Q*A: the rows of A at the frontier (single-term products: exact)
        Ph = gen.HostCSR(len(rows), n,
                         np.concatenate([[0], np.cumsum(np.diff(Ah.row_ptr)[rows])]).astype(np.int32),
                         np.concatenate([Ah.col[Ah.row_ptr[r]:Ah.row_ptr[r + 1]] for r in rows]),
                         np.concatenate([Ah.val[Ah.row_ptr[r]:Ah.row_ptr[r + 1]] for r in rows]))
        s = u.shape[1]
        ref_rp, ref_col, _, gap = osamp.sample_rows(Ph.row_ptr, Ph.col, Ph.val, s,
                                                    u.cpu().numpy(), mode)
        assert gap > 1e-9
        vertices, _ = osamp.select_columns(ref_col, n)
        Fh = Qn.to_host()
        assert np.array_equal(Fh.col, vertices)
        # EXTRACT: A restricted to the frontier rows and the sampled vertices
        np.testing.assert_array_equal(dense_of(A_l.to_host()), osamp.extract(Ad, rows, vertices))
        rows = vertices
