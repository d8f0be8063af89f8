"""Pins of the bulk-sampling oracle (Section IV-C, mini-batch training)
against definitions computed another way: a hand-rolled inverse transform,
the equal-weight special case, empirical draw frequencies, np.unique and a
dense product for EXTRACT."""
import numpy as np
import pytest

from oracle import sampling


def brute_draw(weights, u):
    """First entry whose running weight exceeds u * total, by a plain loop."""
    total = 0.0
    for w in weights:
        total += w
    run = 0.0
    for i, w in enumerate(weights):
        run += w
        if run > u * total:
            return i
    return len(weights) - 1


def random_rows(n_rows, max_len, seed, ncols=1000):
    rng = np.random.default_rng(seed)
    lens = rng.integers(0, max_len, size=n_rows)
    rp = np.concatenate([[0], np.cumsum(lens)])
    col = np.concatenate([np.sort(rng.choice(ncols, size=l, replace=False)) for l in lens])
    val = rng.uniform(0.01, 1.0, size=col.size).astype(np.float32)
    return rp, col, val


@pytest.mark.parametrize("mode", [1, 2])
def test_weighted_draws_match_plain_loop(mode):
    rp, col, val = random_rows(60, 80, seed=mode)
    s = 7
    u = np.random.default_rng(9).random((60, s)).astype(np.float32)
    out_rp, out_col, _, _ = sampling.sample_rows(rp, col, val, s, u, mode)
    for i in range(60):
        a, b = rp[i], rp[i + 1]
        if b - a <= s:
            want = set(col[a:b].tolist())
        else:
            w = val[a:b].astype(np.float64)
            w = w * w if mode == 2 else w
            want = {int(col[a + brute_draw(w, float(u[i, t]))]) for t in range(s)}
        assert set(out_col[out_rp[i]:out_rp[i + 1]].tolist()) == want
        assert (np.diff(out_col[out_rp[i]:out_rp[i + 1]]) > 0).all()


def test_boundary_draws_skip_zero_and_negative_weights():
    # the draw is the first entry whose running weight exceeds u * total, so
    # a draw landing exactly on a boundary skips the zero-weight entries
    # there, and mode 1 weighs by max(value, 0): a negative value is never
    # drawn (mode 2 squares it: drawable). Values and uniforms are exact in
    # fp32 and fp64.
    rows = [([0.0, 0.0, 0.5, 0.0, 1.0], 0.0, 1, 2),     # u = 0: first positive weight
            ([1.0, 0.0, 1.0, 0.5], 0.4, 1, 2),          # target 1.0 = running weight of 0 and 1
            ([-1.0, 0.5, 0.5, 0.25], 0.0, 1, 1),        # negative weight clamped to 0
            ([-1.0, 0.5, 0.5, 0.25], 0.5, 2, 0)]        # mode 2: weights 1, .25, .25, .0625
    for w, u, mode, want in rows:
        val = np.array(w, np.float32)
        wt = val.astype(np.float64)
        wt = wt * wt if mode == 2 else np.maximum(wt, 0.0)
        assert brute_draw(wt, u) == want
        rp = np.array([0, val.size])
        col = np.arange(val.size)
        out_rp, out_col, _, _ = sampling.sample_rows(rp, col, val, 1, np.array([[u]], np.float32),
                                                     mode)
        assert out_col.tolist() == [want], (w, u, mode)


def test_equal_weights_reduce_to_uniform():
    rp, col, _ = random_rows(80, 60, seed=4)
    ones = np.ones(col.size, np.float32)
    u = np.random.default_rng(5).random((80, 5)).astype(np.float32)
    a = sampling.sample_rows(rp, col, ones, 5, u, 1)
    b = sampling.sample_rows(rp, col, ones, 5, u, 0)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_draw_frequencies_follow_weights():
    w = np.array([0.5, 0.1, 0.0, 0.25, 0.15, 1.0], dtype=np.float32)
    rows = 200_000
    rp = np.arange(rows + 1) * w.size
    col = np.tile(np.arange(w.size), rows)
    val = np.tile(w, rows)
    u = np.random.default_rng(6).random((rows, 1)).astype(np.float32)
    out_rp, out_col, _, _ = sampling.sample_rows(rp, col, val, 1, u, 1)
    freq = np.bincount(out_col, minlength=w.size) / rows
    p = w / w.sum()
    assert freq[2] == 0.0                         # a zero weight is never drawn
    assert (np.abs(freq - p) <= 4.5 * np.sqrt(p * (1 - p) / rows) + 1e-12).all()


def test_short_rows_kept_and_repeats_collapse():
    rp = np.array([0, 3, 3, 13])
    col = np.array([4, 9, 11] + list(range(10)))
    val = np.ones(13, np.float32)
    u = np.zeros((3, 4), np.float32)              # every draw of row 2 hits entry 0
    out_rp, out_col, out_val, _ = sampling.sample_rows(rp, col, val, 4, u, 0)
    assert out_rp.tolist() == [0, 3, 3, 4]
    assert out_col.tolist() == [4, 9, 11, 0] and (out_val == 1).all()


def test_select_columns_and_extract():
    rng = np.random.default_rng(7)
    n = 40
    A = (rng.random((n, n)) < 0.2) * rng.uniform(0.1, 1, (n, n))
    Qrows = np.array([3, 17, 21, 39])
    sampled = rng.choice(n, size=15)
    vertices, rank = sampling.select_columns(sampled, n)
    assert vertices.tolist() == sorted(set(sampled.tolist()))
    assert all(rank[v] == int((vertices < v).sum()) for v in range(n))
    assert rank[n] == vertices.size
    # EXTRACT = (Q A) S with Q selecting rows and S selecting columns
    Q = np.zeros((Qrows.size, n))
    Q[np.arange(Qrows.size), Qrows] = 1
    S = np.zeros((n, vertices.size))
    S[vertices, np.arange(vertices.size)] = 1
    np.testing.assert_array_equal(sampling.extract(A, Qrows, vertices), Q @ A @ S)
