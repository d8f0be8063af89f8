"""Host-side logic of the batched, autotuned and MCL drivers, on the CPU:
problem stacking for the batched product (block-diagonal A, row-stacked B),
the autotuner's candidate set, and MCL's cluster read-out."""
import numpy as np
import pytest
import torch

import oracle
from paper_2512_12036_gb300 import DeviceCSR, gen
from paper_2512_12036_gb300 import _lib
from paper_2512_12036_gb300.batched import candidate_opts, stack_problems
from paper_2512_12036_gb300.mcl import interpret


def problems(seed, count=5, n=24):
    rng = np.random.default_rng(seed)
    out = []
    for q in range(count):
        m, k = int(rng.integers(0, 12)), int(rng.integers(0, 10))
        out.append((gen.random_csr(m, k, 0.3, seed + 10 * q, unsorted=q % 2 == 1),
                    gen.random_csr(k, n, 0.2, seed + 10 * q + 5, duplicates=q % 3 == 0)))
    return out


def test_stacked_product_is_per_problem_products():
    # one product of the stack = the problems' products one under the other
    probs = problems(3)
    A, B, row_off, brow_off = stack_problems(probs)
    assert A.rows == row_off[-1] == sum(a.rows for a, _ in probs)
    assert B.rows == brow_off[-1] == A.cols
    C = oracle.spgemm(A, B)
    for q, (Ab, Bb) in enumerate(probs):
        Cb = oracle.spgemm(Ab, Bb)
        for i in range(Ab.rows):
            a = slice(C.row_ptr[row_off[q] + i], C.row_ptr[row_off[q] + i + 1])
            b = slice(Cb.row_ptr[i], Cb.row_ptr[i + 1])
            assert np.array_equal(C.col[a], Cb.col[b])
            assert np.array_equal(C.val[a], Cb.val[b])


def test_stack_rejects_mismatched_shapes():
    A1, B1 = gen.random_csr(3, 4, 0.5, 1), gen.random_csr(4, 6, 0.5, 2)
    with pytest.raises(ValueError):
        stack_problems([(A1, B1), (A1, gen.random_csr(4, 7, 0.5, 3))])
    with pytest.raises(ValueError):
        stack_problems([(A1, gen.random_csr(5, 6, 0.5, 4))])
    A, B, row_off, _ = stack_problems([])
    assert A.rows == 0 and B.rows == 0 and row_off.tolist() == [0]


def test_autotuner_candidates_are_valid_options():
    cands = candidate_opts()
    assert len(cands) >= 2 and len({tuple(sorted(c.items())) for c in cands}) == len(cands)
    for c in cands:
        assert set(c) <= set(_lib.OPT_FIELDS)
        assert 0 < c["esc_max"] <= c["warp_max_nnz"] <= c["block_max_nnz"]
        assert c["warp_max_ip"] <= c["block_max_ip"]
        assert 25 <= c["hash_load_pct"] <= 90 and 1 <= c["narrow_warps"] <= 16
        # the precision rule is not a tuning knob: every candidate keeps it
        assert "fp32_max_terms" not in c
    # every knob group varies something
    from paper_2512_12036_gb300.batched import SEARCH_SPACE
    assert {n for n, _ in SEARCH_SPACE} >= {"tiers", "hash_load_pct", "narrow_warps",
                                            "narrow_max_ip"}
    for _, values in SEARCH_SPACE:
        assert len(values) >= 2


def test_interpret_picks_largest_then_smaller_index():
    # rows of M^T: node j joins the column holding its row's largest value
    rp = torch.tensor([0, 3, 3, 5, 6], dtype=torch.int32)
    col = torch.tensor([0, 2, 3, 1, 3, 2], dtype=torch.int32)
    val = torch.tensor([0.2, 0.5, 0.3, 0.4, 0.4, 1.0])
    M = DeviceCSR(4, 4, rp, col, val)
    assert interpret(M).tolist() == [2, -1, 1, 2]
