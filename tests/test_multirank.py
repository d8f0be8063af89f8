"""Rank-level host logic of the multi-GPU bench (replicas, max-over-ranks
time) and the IP-balanced row partition, as two gloo ranks on the CPU."""
import multiprocessing as mp
import socket

import numpy as np
import pytest

import multirank_worker
from paper_2512_12036_gb300.api import partition_rows


def free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks(tmp_path):
    out = tmp_path / "rank0.txt"
    ctx = mp.get_context("spawn")
    port = free_port()
    procs = [ctx.Process(target=multirank_worker.run, args=(r, 2, port, str(out)))
             for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
    codes = [p.exitcode for p in procs]
    for p in procs:
        if p.is_alive():
            p.kill()
    assert codes == [0, 0], codes
    assert out.read_text() == "ok"


@pytest.mark.parametrize("parts", [1, 2, 3, 8])
def test_partition_rows_balanced(parts):
    rng = np.random.default_rng(9)
    ip = rng.zipf(1.7, size=5000).clip(max=10**6).astype(np.int64)
    ip[rng.random(5000) < 0.1] = 0
    cuts = partition_rows(ip, parts)
    assert cuts[0][0] == 0 and cuts[-1][1] == ip.size and len(cuts) == parts
    for (a0, a1), (b0, b1) in zip(cuts, cuts[1:]):
        assert a1 == b0 and a0 <= a1
    loads = [int(ip[a:b].sum()) for a, b in cuts]
    assert sum(loads) == int(ip.sum())
    assert max(loads) <= ip.sum() / parts + ip.max()


def test_partition_rows_degenerate():
    assert partition_rows(np.zeros(10, np.int64), 3) == [(0, 3), (3, 6), (6, 10)]
    assert partition_rows(np.zeros(0, np.int64), 2) == [(0, 0), (0, 0)]
    with pytest.raises(ValueError):
        partition_rows(np.ones(4, np.int64), 0)
