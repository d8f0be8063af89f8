"""GPU parity: every phase of the CUDA path against the CPU oracle, through
the C ABI, on seeded inputs that reach every row tier (in-register, warp
hash, block hash, dense panels; fp32 and fp64 accumulation), several tiles
and ragged tails, plus empty and malformed inputs."""
import numpy as np
import pytest
import torch

import oracle
from paper_2512_12036_gb300 import DeviceCSR, Plan, SpgemmError, gen
from paper_2512_12036_gb300 import _lib
from contraction import assignment_labels, label_scatter
from parity import compare

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def plan():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return Plan()


def run(plan, A, B):
    dA, dB = DeviceCSR.from_host(A), DeviceCSR.from_host(B)
    C = plan.spgemm(dA, dB)
    torch.cuda.synchronize()
    return C.to_host()


def check_product(plan, A, B):
    got = run(plan, A, B)
    ref = oracle.spgemm(A, B)
    return compare(got, ref)


def hub_matrix(rows, cols, seed, heavy_rows, heavy_len, light_deg=4):
    """Rows with ``light_deg`` random columns, plus heavy rows of ``heavy_len``."""
    rng = np.random.default_rng(seed)
    r, c = [], []
    for i in range(rows):
        d = heavy_len if i in heavy_rows else rng.integers(0, light_deg + 1)
        cc = rng.choice(cols, size=min(d, cols), replace=False)
        r.append(np.full(cc.size, i))
        c.append(cc)
    r = np.concatenate(r)
    c = np.concatenate(c)
    return gen.csr_from_coo(rows, cols, r, c, gen.uniform_open_closed(rng, r.size))


def test_er4096_self_product(plan):
    A = gen.erdos_renyi(4096, 8, seed=1)
    check_product(plan, A, A)


@pytest.mark.parametrize("seed", [1, 2])
def test_rmat_small_skewed(plan, seed):
    A = gen.rmat_symmetric(12, 16, seed=seed)
    check_product(plan, A, A)


@pytest.mark.parametrize("kind", ["plain", "duplicates", "unsorted", "zeros_signed"])
def test_random_shapes(plan, kind):
    kw = {"plain": {}, "duplicates": {"duplicates": True}, "unsorted": {"unsorted": True},
          "zeros_signed": {"explicit_zeros": 0.3, "signed": True}}[kind]
    A = gen.random_csr(300, 200, 0.03, 11, **kw)
    B = gen.random_csr(200, 500, 0.05, 12, **kw)
    check_product(plan, A, B)


def test_every_tier(plan):
    # B: 40k columns (3 dense panels, ragged tail); rows of B of varied length
    B = hub_matrix(3000, 40000, 5, heavy_rows=set(range(0, 3000, 7)), heavy_len=300, light_deg=12)
    # A: light rows (in-register / warp), medium rows (block), heavy rows
    # (dense panels) incl. rows with > 167 entries (fp64 accumulation)
    A = hub_matrix(700, 3000, 6, heavy_rows={1, 50, 51, 300, 699}, heavy_len=900, light_deg=40)
    ip, _ = oracle.ip_count(A, B)
    nnz = oracle.symbolic(A, B)
    assert ip.max() > 16384 and (ip <= 32).sum() > 0 and ((ip > 1024) & (ip <= 16384)).sum() > 0
    assert nnz.max() > 8192 and ((nnz > 512) & (nnz <= 8192)).sum() > 0
    check_product(plan, A, B)


def test_dense_tier_long_a_rows(plan):
    # heavy rows with more A entries than one block tile (uncached dense path),
    # fp64 accumulation, ragged last panel
    B = hub_matrix(3000, 70000, 15, heavy_rows=set(range(0, 3000, 11)), heavy_len=200, light_deg=20)
    A = hub_matrix(40, 3000, 16, heavy_rows={0, 7, 39}, heavy_len=2500, light_deg=30)
    nnz = oracle.symbolic(A, B)
    assert nnz.max() > 8192 and np.diff(A.row_ptr).max() > 1024
    check_product(plan, A, B)


def test_dense_tier_hot_columns(plan):
    # B rows all hold a few hub columns, and 1400 columns of the first panel sit
    # in 300 rows each: hot columns (more than 167 entries) under contention,
    # and a pass with more hot columns than it has fp64 slots (1024)
    rng = np.random.default_rng(21)
    rows, cols = 2000, 40000
    hubs = np.array([5, 17, 9000, 30001])
    warm = rng.choice(16384, size=1400, replace=False)
    r, c = [], []
    for i in range(rows):
        cc = set(rng.choice(cols, size=rng.integers(5, 40), replace=False).tolist())
        cc |= set(hubs.tolist())
        cc |= set(warm[rng.random(warm.size) < 300 / rows].tolist())
        cc = np.array(sorted(cc))
        r.append(np.full(cc.size, i))
        c.append(cc)
    r, c = np.concatenate(r), np.concatenate(c)
    B = gen.csr_from_coo(rows, cols, r, c, gen.uniform_open_closed(rng, r.size))
    counts = np.bincount(B.col, minlength=cols)
    assert (counts[:16384] > 167).sum() > 1100
    A = hub_matrix(30, rows, 22, heavy_rows={0, 3, 9, 29}, heavy_len=1500, light_deg=400)
    assert np.diff(A.row_ptr).max() > 1024 and np.sort(np.diff(A.row_ptr))[-5] > 167
    assert oracle.symbolic(A, B).max() > 8192
    check_product(plan, A, B)


def test_dense_tier_repeated_columns_in_b(plan):
    # sorted B rows that repeat a column (hub columns twice): the fp64 tier's
    # per-copy term bound needs distinct columns, so these products take the
    # fp64 accumulator path
    rng = np.random.default_rng(31)
    rows, cols = 500, 50000
    r, c = [], []
    for i in range(rows):
        cc = list(rng.choice(cols, size=40, replace=False)) + [5, 77]
        if i % 2 == 0:
            cc += [5, 77, 77]
        r.append(np.full(len(cc), i))
        c.append(np.array(cc))
    r, c = np.concatenate(r), np.concatenate(c)
    B = gen.csr_from_coo(rows, cols, r, c, gen.uniform_open_closed(rng, r.size))
    assert (np.diff(B.col[B.row_ptr[0]:B.row_ptr[1]]) == 0).any()
    A = hub_matrix(50, rows, 32, heavy_rows={0, 10, 20}, heavy_len=300)
    assert oracle.symbolic(A, B).max() > 8192
    check_product(plan, A, B)


@pytest.mark.parametrize("cache", [0, 16])
def test_dense_tier_small_terms_after_large(plan, cache):
    # one row of 1024 ones against B rows that all hold column 0 (a hot
    # column): B[0,0] = 1 and B[k,0] = 2^-25 for k > 0. A single fp32 running
    # sum that takes the 1 first loses every small term (3e-5 of the sum);
    # the tier's partial sums must stay within the 1e-5 bound (cache: the
    # rank-compacted fp64 tier, whose slot sums are double-float pairs)
    if cache:
        plan = Plan(row_cache_mb=cache)
    rng = np.random.default_rng(41)
    na, cols = 1024, 40000
    r, c, v = [], [], []
    for k in range(na):
        cc = np.concatenate([[0], 1 + rng.choice(cols - 1, size=16, replace=False)])
        vv = gen.uniform_open_closed(rng, cc.size)
        vv[0] = 1.0 if k == 0 else 2.0 ** -25
        r.append(np.full(cc.size, k))
        c.append(cc)
        v.append(vv)
    B = gen.csr_from_coo(na, cols, np.concatenate(r), np.concatenate(c),
                         np.concatenate(v).astype(np.float32))
    A = gen.csr_from_coo(2, na, np.zeros(na, np.int64), np.arange(na),
                         np.ones(na, np.float32))
    assert oracle.symbolic(A, B).max() > 8192
    got = run(plan, A, B)
    ref = oracle.spgemm(A, B)
    compare(got, ref)
    assert got.col[0] == 0
    assert abs(float(got.val[0]) - (1.0 + 1023 * 2.0 ** -25)) <= 1e-5 * ref.bound[0]


def test_block_tier_clustered_columns(plan):
    # rows of C with 512..8192 entries (block hash tier, fp32 and fp64 rows)
    # whose columns crowd into [0, 3000) plus one far column: the bucket sort
    # sees buckets far above its limit and must fall back; other rows spread
    # their columns and take the bucket sort
    rng = np.random.default_rng(51)
    rows, cols = 2000, 1_000_000
    r, c = [], []
    for k in range(rows):
        if k < 1000:
            cc = rng.choice(3000, size=20, replace=False)
            if k == 0:
                cc = np.append(cc, cols - 1)
        else:
            cc = rng.choice(cols, size=20, replace=False)
        r.append(np.full(cc.size, k))
        c.append(cc)
    r, c = np.concatenate(r), np.concatenate(c)
    B = gen.csr_from_coo(rows, cols, r, c, gen.uniform_open_closed(rng, r.size))
    ra, ca = [], []
    for i, (lo, n) in enumerate([(0, 150), (0, 300), (1000, 150), (1000, 300), (0, 60)]):
        cc = lo + rng.choice(1000, size=n, replace=False)
        if i in (0, 1):
            cc = np.append(cc[cc != 0], 0)
        ra.append(np.full(cc.size, i))
        ca.append(cc)
    ra, ca = np.concatenate(ra), np.concatenate(ca)
    A = gen.csr_from_coo(5, rows, ra, ca, gen.uniform_open_closed(rng, ra.size))
    nnz = oracle.symbolic(A, B)
    assert ((nnz > 512) & (nnz <= 8192)).sum() >= 4
    check_product(plan, A, B)


def test_dense_tier_narrow_b_hot_columns():
    # a lower block-tier limit (2048) lets rows of a 5000-column B reach the
    # fp64 dense tier; its hot-column counts then come from the per-block
    # shared-memory histogram used for narrow B
    rng = np.random.default_rng(61)
    rows, cols = 1000, 5000
    r, c = [], []
    for k in range(rows):
        cc = np.unique(np.concatenate([rng.choice(cols, size=30, replace=False), [7, 4000]]))
        r.append(np.full(cc.size, k))
        c.append(cc)
    r, c = np.concatenate(r), np.concatenate(c)
    B = gen.csr_from_coo(rows, cols, r, c, gen.uniform_open_closed(rng, r.size))
    A = hub_matrix(20, rows, 62, heavy_rows={0, 5, 19}, heavy_len=400)
    nnz = oracle.symbolic(A, B)
    assert nnz.max() > 2048 and (np.bincount(B.col, minlength=cols) > 167).sum() >= 2
    check_product(Plan(block_max_nnz=2048), A, B)


def test_plans_with_different_tables_interleave(plan):
    # kernel shared-memory limits are process-wide: a plan with smaller
    # tables created later must not break the launches of an earlier plan
    A = gen.random_csr(200, 300, 0.1, seed=71)
    B = gen.random_csr(300, 100000, 0.002, seed=72)
    nnz = oracle.symbolic(A, B)
    assert nnz.max() > 4096 and nnz.max() <= 8192
    small = Plan(block_max_nnz=2048, block_max_ip=4096)
    check_product(plan, A, B)
    check_product(small, A, B)
    check_product(plan, A, B)
    del small
    check_product(plan, A, B)


def test_dense_tier_clustered_pass_overflow(plan):
    # a row of the fp32 dense tier (160 A entries) whose ~42k output columns
    # all sit in the first of 20 panels: sized for an even spread, its first
    # pass holds more entries than the compact value array and is
    # accumulated in word ranges
    rng = np.random.default_rng(81)
    cols, nb = 20 * 16384, 200
    r, c = [], []
    for k in range(nb):
        cc = rng.choice(50000, size=600, replace=False) if k < 160 else \
            rng.choice(cols, size=50, replace=False)
        r.append(np.full(cc.size, k))
        c.append(cc)
    r, c = np.concatenate(r), np.concatenate(c)
    B = gen.csr_from_coo(nb, cols, r, c, gen.uniform_open_closed(rng, r.size))
    A = gen.csr_from_coo(3, nb, np.concatenate([np.zeros(160), np.ones(40), np.full(30, 2)]),
                         np.concatenate([np.arange(160), np.arange(160, 200), np.arange(0, 30)]),
                         np.ones(230, np.float32))
    nnz = oracle.symbolic(A, B)
    assert nnz[0] > 40000 and np.diff(A.row_ptr)[0] <= 167
    check_product(plan, A, B)


def test_narrow_b_tiers(plan):
    # B with 700 columns: rows in the in-register tier, the narrow fp32 and
    # fp64 tiers (more than 167 A entries), and rows above the narrow tier's
    # product limit (block and dense tiers)
    rng = np.random.default_rng(91)
    k, n = 3000, 700
    B = gen.random_csr(k, n, 0.03, seed=92)                 # ~21 entries per row
    r, c = [], []
    for i, d in enumerate([3, 10, 60, 150, 170, 400, 900, 2500, 2999, 1, 0, 40]):
        cc = rng.choice(k, size=d, replace=False)
        r.append(np.full(d, i))
        c.append(cc)
    r, c = np.concatenate(r), np.concatenate(c)
    A = gen.csr_from_coo(12, k, r, c, gen.uniform_open_closed(rng, r.size))
    ip, _ = oracle.ip_count(A, B)
    assert ip.max() > 32768 and (ip[(np.diff(A.row_ptr) > 167)] <= 32768).any()
    check_product(plan, A, B)


def test_dense_tier_unsorted_b(plan):
    B = hub_matrix(500, 50000, 7, heavy_rows=set(range(0, 500, 3)), heavy_len=400)
    Bu = gen.random_csr(1, 1, 1.0, 0)  # placeholder for type
    rng = np.random.default_rng(1)
    col, val = B.col.copy(), B.val.copy()
    for i in range(B.rows):
        s, e = B.row_ptr[i], B.row_ptr[i + 1]
        p = rng.permutation(e - s) + s
        col[s:e], val[s:e] = col[p], val[p]
    Bu = gen.HostCSR(B.rows, B.cols, B.row_ptr, col, val)
    A = hub_matrix(50, 500, 8, heavy_rows={0, 10, 20}, heavy_len=300)
    assert oracle.symbolic(A, Bu).max() > 8192
    check_product(plan, A, Bu)


def test_all_products_one_column(plan):
    # every product of row 0 lands in column 3: nnz 1, IP 20000 (contended slot)
    k = 20000
    B = gen.HostCSR(k, 10, np.arange(k + 1, dtype=np.int32), np.full(k, 3, np.int32),
                    np.full(k, 0.5, np.float32))
    A = gen.HostCSR(2, k, np.array([0, k, k + 5], np.int32),
                    np.concatenate([np.arange(k), np.arange(5)]).astype(np.int32),
                    np.ones(k + 5, np.float32))
    check_product(plan, A, B)


def test_hash_collisions(plan):
    # columns that are multiples of 2^16 and consecutive runs
    cols = np.concatenate([np.arange(0, 2**16 * 30, 2**16), np.arange(100, 900)])
    n = cols.max() + 1
    B = gen.csr_from_coo(3, int(n), np.repeat(np.arange(3), cols.size), np.tile(cols, 3),
                         np.ones(3 * cols.size, np.float32))
    A = gen.HostCSR(1, 3, np.array([0, 3], np.int32), np.arange(3, dtype=np.int32),
                    np.array([1, 2, 3], np.float32))
    check_product(plan, A, B)


def test_empty_inputs(plan):
    B = gen.random_csr(5, 6, 0.5, seed=3)
    Z = gen.HostCSR(4, 5, np.zeros(5, np.int32), np.zeros(0, np.int32), np.zeros(0, np.float32))
    got = run(plan, Z, B)
    assert got.nnz == 0 and got.row_ptr.tolist() == [0] * 5
    E = gen.HostCSR(0, 5, np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(0, np.float32))
    got = run(plan, E, B)
    assert got.rows == 0 and got.nnz == 0
    one = gen.HostCSR(1, 1, np.array([0, 1], np.int32), np.array([0], np.int32),
                      np.array([2.0], np.float32))
    got = run(plan, one, one)
    assert got.col.tolist() == [0] and got.val.tolist() == [4.0]


def test_phases_individually(plan):
    A = gen.rmat_symmetric(11, 8, seed=5)
    dA = DeviceCSR.from_host(A)
    ws = plan.workspace(dA, dA)
    ip, total = plan.count(dA, dA, ws)
    ip_ref, total_ref = oracle.ip_count(A, A)
    assert total == total_ref and np.array_equal(ip.cpu().numpy(), ip_ref)
    nnz, nnz_total = plan.symbolic(dA, dA, ip, ws)
    nnz_ref = oracle.symbolic(A, A)
    assert np.array_equal(nnz.cpu().numpy(), nnz_ref) and nnz_total == int(nnz_ref.sum())
    rp, tot = plan.row_ptr(nnz, ws, total=True)
    assert tot == int(nnz_ref.sum())
    assert np.array_equal(rp.cpu().numpy()[1:], np.cumsum(nnz_ref)) and int(rp[0]) == 0
    mp, off = plan.group(ip, [32, 512, 8192], ws)
    mp_ref, off_ref = oracle.group_rows(ip_ref, [32, 512, 8192])
    assert np.array_equal(mp.cpu().numpy(), mp_ref) and np.array_equal(off.cpu().numpy(), off_ref)


def test_row_ptr_overflow_detected(plan):
    dA = DeviceCSR.from_host(gen.erdos_renyi(64, 4, seed=2))
    ws = plan.workspace(dA, dA)
    counts = torch.tensor([2**30, 2**30, 2**30], dtype=torch.int32, device="cuda")
    with pytest.raises(SpgemmError) as e:
        plan.row_ptr(counts, ws, total=True)
    assert e.value.code == _lib.ERR_OVERFLOW


def test_row_blocks_equal_whole(plan):
    A = gen.rmat_symmetric(11, 8, seed=6)
    dA = DeviceCSR.from_host(A)
    blocks, ip_total, nnz_total = plan.spgemm_blocks(dA, dA, max_block_nnz=20000)
    assert len(blocks) > 3
    ref = oracle.spgemm(A, A)
    assert nnz_total == ref.nnz and ip_total == oracle.ip_count(A, A)[1]
    for r0, r1, Cb in blocks:
        h = Cb.to_host()
        sub = oracle.OracleCSR(r1 - r0, A.cols, ref.row_ptr[r0:r1 + 1] - ref.row_ptr[r0],
                               ref.col[ref.row_ptr[r0]:ref.row_ptr[r1]],
                               ref.val[ref.row_ptr[r0]:ref.row_ptr[r1]],
                               ref.bound[ref.row_ptr[r0]:ref.row_ptr[r1]])
        compare(h, sub)


def test_row_view_input(plan):
    A = gen.erdos_renyi(1000, 10, seed=4)
    dA = DeviceCSR.from_host(A)
    V = dA.view_rows(300, 700)
    C = plan.spgemm(V, dA).to_host()
    ref = oracle.spgemm(A, A, rows=np.arange(300, 700, dtype=np.int32))
    compare(C, ref)


@pytest.mark.parametrize("bad", ["past_last_column", "negative"])
def test_malformed_column_in_dense_tiers(bad):
    # a column outside B on the hub rows of B, read by rows of both dense
    # accumulation tiers (the rank-compacted fp32 kernel and the fp64
    # hot-column kernel, through the panel table and the column words):
    # reported as ERR_INVALID, no fault, and the plan stays usable. The
    # corrupted entries keep their rows sorted, so the sorted-B paths run.
    opts = {"panel_cols": 1024, "block_max_nnz": 512, "block_max_ip": 1024,
            "fp32_max_terms": 40}
    A = gen.rmat_symmetric(12, 16, seed=5)
    na = np.diff(A.row_ptr.astype(np.int64))
    ip, _ = oracle.ip_count(A, A)
    nnz = oracle.symbolic(A, A)
    dense = (nnz > opts["block_max_nnz"]) & ~((ip <= 32) & (na <= 32))
    f64 = (na > opts["fp32_max_terms"]) & (ip > opts["fp32_max_terms"])
    hubs = np.argsort(na)[-5:]                       # the five hub rows
    reads_hub = np.zeros(A.rows, bool)
    reads_hub[np.repeat(np.arange(A.rows), na)[np.isin(A.col, hubs)]] = True
    assert (dense & f64 & reads_hub).sum() > 0 and (dense & ~f64 & reads_hub).sum() > 0
    B = gen.HostCSR(A.rows, A.cols, A.row_ptr, A.col.copy(), A.val)
    for k in hubs:
        s, e = int(A.row_ptr[k]), int(A.row_ptr[k + 1])
        if bad == "negative":
            B.col[s] = -1
        else:
            B.col[e - 1] = A.cols + 7
    plan = Plan(**opts)
    with pytest.raises(SpgemmError) as e:
        plan.spgemm(DeviceCSR.from_host(A), DeviceCSR.from_host(B))
    assert e.value.code == _lib.ERR_INVALID
    torch.cuda.synchronize()
    check_product(plan, A, A)


@pytest.mark.parametrize("unsorted", [False, True])
def test_dense_tiers_without_panel_table(unsorted):
    # B with 1.1M columns is wider than 1024 panels of 1024 columns, so there
    # is no panel table: heavy rows run the dense kernels that filter whole B
    # rows pass by pass (the fp32 dense-array kernel and the fp64 group
    # kernel), with sorted and with unsorted rows of B
    opts = {"panel_cols": 1024, "block_max_nnz": 512, "block_max_ip": 1024,
            "fp32_max_terms": 40}
    rng = np.random.default_rng(101)
    k, n, m = 2000, 1_100_000, 200
    r, c = [], []
    for i in range(k):
        cc = np.unique(rng.integers(0, n, size=int(rng.integers(0, 61))))
        r.append(np.full(cc.size, i))
        c.append(rng.permutation(cc) if unsorted else cc)
    B = gen.csr_from_coo(k, n, np.concatenate(r), np.concatenate(c),
                         gen.uniform_open_closed(rng, sum(x.size for x in c)))
    if unsorted:
        B = gen.HostCSR(k, n, B.row_ptr, np.concatenate(c).astype(np.int32), B.val)
    lens = [150] * 5 + [30] * 20 + [int(x) for x in rng.integers(0, 5, size=m - 25)]
    ra = np.concatenate([np.full(d, i) for i, d in enumerate(lens)])
    ca = np.concatenate([np.sort(rng.choice(k, size=d, replace=False)) for d in lens])
    A = gen.csr_from_coo(m, k, ra, ca, gen.uniform_open_closed(rng, ra.size))
    assert -(-n // opts["panel_cols"]) > 1024
    na = np.diff(A.row_ptr)
    ip, _ = oracle.ip_count(A, B)
    nnz = oracle.symbolic(A, B)
    dense = nnz > opts["block_max_nnz"]
    f64 = (na > opts["fp32_max_terms"]) & (ip > opts["fp32_max_terms"])
    assert (dense & f64).sum() == 5 and (dense & ~f64).sum() >= 15
    check_product(Plan(**opts), A, B)


def test_structure_deterministic(plan):
    A = gen.rmat_symmetric(12, 8, seed=8)
    c1 = run(plan, A, A)
    c2 = run(plan, A, A)
    assert np.array_equal(c1.row_ptr, c2.row_ptr) and np.array_equal(c1.col, c2.col)


@pytest.mark.parametrize("what", ["a_col", "b_col", "a_rowptr"])
def test_malformed_input_reported_not_faulted(plan, what):
    A = gen.erdos_renyi(100, 5, seed=1)
    B = gen.erdos_renyi(100, 5, seed=2)
    if what == "a_col":
        A.col = A.col.copy()
        A.col[7] = 100          # == B.rows: out of range
    elif what == "b_col":
        B.col = B.col.copy()
        B.col[3] = 1000         # >= B.cols
    else:
        A.row_ptr = A.row_ptr.copy()
        A.row_ptr[50] = A.row_ptr[49] - 1
    dA, dB = DeviceCSR.from_host(A), DeviceCSR.from_host(B)
    with pytest.raises(SpgemmError) as e:
        plan.spgemm(dA, dB)
    assert e.value.code == _lib.ERR_INVALID
    # the context is still usable afterwards
    torch.cuda.synchronize()
    C = plan.spgemm(DeviceCSR.from_host(gen.erdos_renyi(50, 3, seed=9)),
                    DeviceCSR.from_host(gen.erdos_renyi(50, 3, seed=9)))
    assert C.nnz > 0


@pytest.mark.parametrize("scale,clusters", [(12, 256), (14, 1024)])
def test_contraction_full_StAS(plan, scale, clusters):
    """Both products of the contraction S^T*A*S (Algorithm 7) on an R-MAT
    graph: each product against the oracle on the inputs it actually got
    (exact structure, 1e-5 * sum|a||b|), and the final result against A's
    entries scattered by cluster labels in fp64 (exact structure; values
    within 2e-5 * sum|a|, one 1e-5 share per product)."""
    A_h = gen.rmat_symmetric(scale, 16, 0.57, 0.19, 0.19, seed=2 + scale)
    S_h = gen.assignment_matrix(A_h.rows, clusters, seed=3)
    St_h = gen.transpose_structure(S_h)
    A, S, St = DeviceCSR.from_host(A_h), DeviceCSR.from_host(S_h), DeviceCSR.from_host(St_h)
    T = plan.spgemm(St, A)
    C2 = plan.spgemm(T, S)
    torch.cuda.synchronize()
    T_h, C2_h = T.to_host(), C2.to_host()
    compare(T_h, oracle.spgemm(St_h, A_h))
    compare(C2_h, oracle.spgemm(T_h, S_h))
    rp, col, val, absum = label_scatter(A_h, assignment_labels(S_h), clusters)
    assert np.array_equal(C2_h.row_ptr.astype(np.int64), rp)
    assert np.array_equal(C2_h.col, col)
    err = np.abs(C2_h.val.astype(np.float64) - val)
    assert (err <= 2e-5 * absum).all()
    # the contraction preserves the total weight of the graph
    assert abs(float(C2_h.val.astype(np.float64).sum()) - float(A_h.val.astype(np.float64).sum())) \
        <= 2e-5 * float(np.abs(A_h.val.astype(np.float64)).sum())


@pytest.mark.parametrize("opts", [{"narrow_warps": 4}, {"narrow_warps": 16},
                                  {"narrow_max_ip": 4096}, {"narrow_max_ip": 131072},
                                  {"hash_load_pct": 35}, {"hash_load_pct": 70},
                                  {"hash_load_pct": 90, "warp_max_nnz": 128}])
def test_tuning_knobs_keep_results(opts):
    """The autotuner's knobs (narrow-tier warps and row limit, hash-table
    load) change schedules and table sizes only: results match the oracle."""
    plan = Plan(**opts)
    # narrow B (the GNN feature shape) and a wide B that fills the hash tiers
    X = gen.topk_rows(np.random.default_rng(3).normal(size=(3000, 256)).astype(np.float32), 32)
    Ah = gen.sym_normalised_adjacency(3000, 24.0, np.random.default_rng(4))
    check_product(plan, Ah, X)
    A = gen.rmat_symmetric(12, 8, seed=6)
    check_product(plan, A, A)
