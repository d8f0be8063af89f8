"""Worker for the two-rank gloo tests (imported by spawned processes)."""
import os

import numpy as np
import torch
import torch.distributed as dist


def run(rank: int, world: int, port: int, out: str) -> None:
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        import oracle
        from paper_2512_12036_gb300 import gen
        from paper_2512_12036_gb300.api import partition_rows

        # slowest rank's time
        t = bench.max_over_ranks(10.0 * rank + 1.5, torch.device("cpu"))
        assert t == 10.0 * (world - 1) + 1.5, t

        # IP-balanced row shards, each multiplied with the whole B, no exchange
        A = gen.rmat_symmetric(9, 8, seed=3)
        ip, total = oracle.ip_count(A, A)
        parts = partition_rows(ip, world)
        r0, r1 = parts[rank]
        rp = A.row_ptr.astype(np.int64)
        mine = gen.HostCSR(r1 - r0, A.cols, (rp[r0:r1 + 1] - rp[r0]).astype(np.int32),
                           A.col[rp[r0]:rp[r1]], A.val[rp[r0]:rp[r1]])
        C = oracle.spgemm(mine, A)
        got = [None] * world
        dist.all_gather_object(got, (r0, r1, int(ip[r0:r1].sum()), C.row_ptr, C.col, C.val))
        if rank == 0:
            full = oracle.spgemm(A, A)
            assert got[0][0] == 0 and got[-1][1] == A.rows
            for a, b in zip(got, got[1:]):
                assert a[1] == b[0]
            col = np.concatenate([g[4] for g in got])
            val = np.concatenate([g[5] for g in got])
            nnz = np.concatenate([np.diff(g[3]) for g in got])
            assert np.array_equal(nnz, np.diff(full.row_ptr))
            assert np.array_equal(col, full.col) and np.array_equal(val, full.val)
            # each shard within one row's IP of an even split
            assert max(g[2] for g in got) <= total / world + ip.max()
            with open(out, "w") as f:
                f.write("ok")
    finally:
        dist.destroy_process_group()
