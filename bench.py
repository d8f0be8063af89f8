#!/usr/bin/env python
"""SpGEMM throughput benchmark on one GB300 (or N replicas under torchrun).

Workload (one step = the whole hot path over one synthetic input):
  A = R-MAT scale 20, edge factor 16, (a,b,c,d) = (0.57,0.19,0.19,0.05),
      symmetrised, deduplicated, no self-loops, fp32 U(0,1] (seed 2);
  1. C = A*A, produced in blocks of consecutive rows with int32 row pointers
     (nnz(C) ~ 2.2e10 > 2^31-1): count, allocation phase, per-block row
     pointers and accumulation phase;
  2. graph contraction S^T * A * S with S a 2^20 x 65,536 assignment matrix
     (one 1.0 per row at a uniform cluster id, seed 3): two more products.
The metric is GFLOP/s = 2 * (intermediate products of the three products) /
step time. Inputs are resident in HBM before timing; they are larger than
L2 (A alone is 250 MB vs 129 MB of L2), so no flush is needed between steps.

`--impl reference` times the CPU oracle (plain C, fp64 dense accumulator) on
the host cores over a bounded sample of rows of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "spgemm_gflops"
UNIT = "GFLOP/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--scale", type=int, default=20, help="R-MAT scale (20 = the workload)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-patterns", action="store_true",
                    help="skip the batched / served / MCL pattern measurements")
    ap.add_argument("--gnn-graphs", type=int, default=8192)
    ap.add_argument("--panel-cols", type=int, default=None)
    ap.add_argument("--served-requests", type=int, default=2000)
    ap.add_argument("--dense-splits", type=int, default=None,
                    help="work items per heavy row in the fp64-bound dense tier")
    ap.add_argument("--only", choices=["batched", "served", "mcl", "er4096"], default=None,
                    help="run one pattern measurement alone (profiling); no benchmark line")
    ap.add_argument("--stage-b", action="store_true",
                    help="allocation block tier with B segments staged in shared memory")
    ap.add_argument("--no-row-cache", action="store_true",
                    help="accumulation phase without the allocation phase's row bitmaps")
    ap.add_argument("--row-stride", type=int, default=1,
                    help="left operand of A*A = every k-th row of A (a smaller case with the "
                         "same row mix and the full right operand, for profiling; not the "
                         "headline workload, no end-to-end leg)")
    return ap.parse_args()


def workload(scale: int):
    from paper_2512_12036_gb300 import gen
    A = gen.rmat_symmetric(scale, 16, 0.57, 0.19, 0.19, seed=2)
    clusters = max(1, (1 << scale) // 16)
    S = gen.assignment_matrix(A.rows, clusters, seed=3)
    St = gen.transpose_structure(S)
    return A, S, St, clusters


def workload_name(scale: int, row_stride: int = 1) -> str:
    if row_stride > 1:
        return f"rmat{scale}_ef16_AxA_rows1in{row_stride}_plus_StAS"
    return f"rmat{scale}_ef16_AxA_plus_StAS"


# ---------------------------------------------------------------------------
# CPU oracle baseline (rank 0 only): a bounded random sample of rows of A*A.
# ---------------------------------------------------------------------------

def host_threads() -> int:
    """Host cores this process may run on. The oracle is timed with all of
    them: rank 0 runs it alone (other ranks do no CPU work meanwhile), and
    torchrun's default OMP_NUM_THREADS=1 must not shrink it."""
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def cpu_baseline(A, seconds: float, seed: int = 0):
    import oracle
    rng = np.random.default_rng(seed)
    ip, _ = oracle.ip_count(A, A)
    cores = host_threads()
    # calibrate on a small sample, then size the main one to ~`seconds`
    order = rng.permutation(A.rows).astype(np.int32)
    csum = np.cumsum(ip[order])

    def take(products):
        k = int(np.searchsorted(csum, products)) + 1
        return order[:min(k, order.size)]

    cal = take(2e7)
    t0 = time.perf_counter()
    oracle.spgemm(A, A, rows=cal, nthreads=cores, with_bound=False)
    t_cal = max(time.perf_counter() - t0, 1e-3)
    rate = float(ip[cal].sum()) / t_cal
    rows = take(rate * seconds)
    prods = float(ip[rows].sum())
    t0 = time.perf_counter()
    oracle.spgemm(A, A, rows=rows, nthreads=cores, with_bound=False)
    t = time.perf_counter() - t0
    # the same oracle on one thread, over a sample 1/cores as large (about the
    # same wall time)
    rows1 = take(rate * seconds / max(cores, 1))
    prods1 = float(ip[rows1].sum())
    t0 = time.perf_counter()
    oracle.spgemm(A, A, rows=rows1, nthreads=1, with_bound=False)
    t1 = time.perf_counter() - t0
    return {"value": 2 * prods / t / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{rows.size} uniformly drawn rows of A*A ({prods:.3e} intermediate "
                      f"products, {t:.1f} s), fp64 dense accumulator, OpenMP over rows",
            "single_thread": {"value": 2 * prods1 / t1 / 1e9, "unit": UNIT, "cores": 1,
                              "sample": f"the first {rows1.size} of the same rows "
                                        f"({prods1:.3e} products, {t1:.1f} s)"}}


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, smax, reasons, power = [], None, set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            try:
                power.append(float(f[3].split()[0]))
            except (ValueError, IndexError):
                pass
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "sm_mhz_min": min(sm),
                "power_w": statistics.median(power) if power else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# our implementation
# ---------------------------------------------------------------------------

# DRAM bytes (read + write) per intermediate product of the dense accumulation
# kernels, from one ncu capture of the kernel as it stands (row sample 1 in
# 128 of the R-MAT scale 20 workload, right operand and L2 pressure as in the
# full case; the summary and its command are kept under profiles/).
# Scaled by the full workload's products of the tier to give the per-launch
# traffic; a kernel changed since its capture must drop out of this table.
DRAM_BYTES_PER_PRODUCT = {
    # k_num_dense_hotr (rank-compacted fp64-bound tier with the row bitmap cache)
    "num_dense64": (911.744000e6 + 341.544192e6) / 256228740,
    # k_num_dense_rank (rank-compacted fp32 tier with the row bitmap cache)
    "num_dense32": (1087.925e6 + 1067.939e6) / 257686006,
}


def max_over_ranks(x: float, device) -> float:
    """The largest x over the ranks of the default process group (the job's
    time is its slowest rank's)."""
    import torch
    import torch.distributed as dist
    if not dist.is_initialized() or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def tier_work(plan, A_host, ip, nnz):
    """Rows, products and compulsory bytes of each row tier of the allocation
    and accumulation phases of A*A, following the library's tier rules (used
    for the per-kernel roofline)."""
    o = plan.opts
    na = np.diff(A_host.row_ptr.astype(np.int64))
    small = (ip <= o["esc_max"]) & (na <= o["esc_max"])
    # allocation phase: tiers by IP
    live = ip > 1
    s_esc = live & small
    s_warp = live & ~small & (ip <= o["warp_max_ip"])
    s_block = live & ~small & ~s_warp & (ip <= o["block_max_ip"])
    s_dense = live & ~small & ~s_warp & ~s_block
    # accumulation phase: tiers by nnz, fp64 where > fp32_max_terms terms can meet
    f64 = (na > o["fp32_max_terms"]) & (ip > o["fp32_max_terms"])
    has = nnz > 0
    n_esc = has & small
    n_warp = has & ~small & (nnz <= o["warp_max_nnz"]) & (ip <= 16 * o["warp_max_nnz"])
    n_block = has & ~small & ~n_warp & (nnz <= o["block_max_nnz"])
    n_dense = has & ~small & ~n_warp & ~n_block
    tiers = {"sym_esc": (s_esc, 0), "sym_warp": (s_warp, 0), "sym_block": (s_block, 0),
             "sym_dense": (s_dense, 0),
             "num_esc": (n_esc, 1), "num_warp32": (n_warp & ~f64, 1), "num_warp64": (n_warp & f64, 1),
             "num_block32": (n_block & ~f64, 1), "num_block64": (n_block & f64, 1),
             "num_dense32": (n_dense & ~f64, 1), "num_dense64": (n_dense & f64, 1)}
    out = {}
    for k, (m, numeric) in tiers.items():
        rows, prods, ents, cn = int(m.sum()), int(ip[m].sum()), int(na[m].sum()), int(nnz[m].sum())
        if numeric:
            # A rows (row_ptr pair, col+val), gathered B row_ptr pairs, B col+val per
            # product, C col+val per entry
            byts = 8 * rows + 8 * ents + 8 * ents + 8 * prods + 8 * cn
        else:
            # A rows (row_ptr pair, col), gathered B row_ptr pairs, B col per product,
            # one count per row
            byts = 8 * rows + 4 * ents + 8 * ents + 4 * prods + 4 * rows
        out[k] = {"rows": rows, "ip": prods, "a_entries": ents, "nnz": cn, "bytes": byts}
    return out


# ---------------------------------------------------------------------------
# patterns beside the headline step: batched GNN aggregation (forward graph +
# backward), served requests (continuous batching vs plain per-request), MCL
# ---------------------------------------------------------------------------

def _pct(xs, p):
    xs = sorted(xs)
    return xs[min(len(xs) - 1, int(round(p * (len(xs) - 1))))] if xs else None


def pattern_batched(num_graphs: int, device):
    """8,192 subgraphs (n log-uniform [64, 2048], degree U[4,32], sym-normalised
    A_hat, X = per-row top-32 of N(0,1) over 256 features): C = A_hat X as one
    autotuned, graph-captured product, its backward, and the plain path (one
    spgemm call per subgraph, all arriving at t = 0)."""
    import torch

    from paper_2512_12036_gb300 import DeviceCSR, Plan, gen
    from paper_2512_12036_gb300.batched import SEARCH_SPACE, autotune, time_graph

    t0 = time.perf_counter()
    batch = gen.gnn_batch(num_graphs, seed=5)
    gen_s = time.perf_counter() - t0
    A = DeviceCSR.from_host(batch.A, device)
    X = DeviceCSR.from_host(batch.X, device)
    bs, opts, timings = autotune(A, X, reps=3)
    ms_fwd = time_graph(bs, reps=5)
    C = bs.result()
    ip_total = int(bs.ip_row.sum().item())
    plan = bs.plan
    dC = torch.randn(C.nnz, device=device)
    ws_b = plan.backward_workspace(A, X)
    plan.backward(A, X, C, dC, ws=ws_b)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(3):
        plan.backward(A, X, C, dC, ws=ws_b)
    e1.record()
    e1.synchronize()
    ms_bwd = e0.elapsed_time(e1) / 3
    plan.check_status(ws_b, "batched backward")
    layer = pattern_pruned_layer(A, plan, device)
    # plain per-request path over the same subgraphs (all arrive at t = 0)
    pplan = Plan(device=device.index)
    off = batch.node_off
    done_at = []
    max_rel = 0.0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for b in range(num_graphs):
        r0, r1 = int(off[b]), int(off[b + 1])
        Cb = pplan.spgemm(A.view_rows(r0, r1), X)
        done_at.append(time.perf_counter() - t0)
        if b % max(1, num_graphs // 16) == 0:      # same structure and values as the batch
            s, e = int(C.row_ptr[r0].item()), int(C.row_ptr[r1].item())
            assert torch.equal(C.col[s:e], Cb.col), "batched and plain structures differ"
            d = (C.val[s:e] - Cb.val).abs() / Cb.val.abs().clamp_min(1e-30)
            max_rel = max(max_rel, float(d.max().item()) if d.numel() else 0.0)
    plain_s = done_at[-1]
    gflop = 2.0 * ip_total / 1e9
    return {"workload": f"gnn{num_graphs}_n64-2048_deg4-32_X256_top32", "rows": A.rows,
            "nnz_A": A.nnz, "nnz_X": X.nnz, "ip": ip_total, "nnz_C": C.nnz,
            "generate_s": round(gen_s, 1),
            "batched": {"forward_ms": ms_fwd, "backward_ms": ms_bwd,
                        "forward_gflops": gflop / (ms_fwd / 1e3),
                        "p50_ms": ms_fwd, "p99_ms": ms_fwd, "launch": "one CUDA graph replay",
                        "autotuned_opts": opts, "candidates_ms": timings,
                        "search": "coordinate descent over " + ", ".join(
                            f"{n} ({len(v)} values)" for n, v in SEARCH_SPACE),
                        "default_ms": timings.get("default"),
                        "gain_vs_default": (timings["default"] / min(timings.values())
                                            if timings.get("default") else None)},
            "pruned_gcn_layer": layer,
            "plain": {"total_ms": 1e3 * plain_s, "gflops": gflop / plain_s,
                      "p50_ms": 1e3 * _pct(done_at, 0.5), "p99_ms": 1e3 * _pct(done_at, 0.99)},
            "max_rel_diff_batched_vs_plain": max_rel}


def pattern_pruned_layer(A, plan, device, d: int = 256, dout: int = 256, k: int = 32,
                         reps: int = 3):
    """One GCN layer with a top-k pruning layer (Eq. 1-3) on the batch graph:
    X dense N(0,1) n x d (seeded), W d x dout; forward A*TopK(X,k)*W and its
    backward (dX, dW), timed with CUDA events."""
    import torch

    from paper_2512_12036_gb300 import gnn

    torch.backends.cuda.matmul.allow_tf32 = False
    g = torch.Generator(device=device).manual_seed(7)
    X = torch.randn(A.rows, d, generator=g, device=device).requires_grad_(True)
    W = (torch.randn(d, dout, generator=g, device=device) / d ** 0.5).requires_grad_(True)
    dY = torch.randn(A.rows, dout, generator=g, device=device)

    def fwd():
        return gnn.pruned_aggregation(A, X, W, k, plan)

    Y = fwd()
    Y.backward(dY)
    torch.cuda.synchronize()
    tf, tb = [], []
    for _ in range(reps):
        X.grad = None
        W.grad = None
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record()
        Y = fwd()
        e1.record()
        Y.backward(dY)
        e2.record()
        e2.synchronize()
        tf.append(e0.elapsed_time(e1))
        tb.append(e1.elapsed_time(e2))
    ip = A.nnz * min(k, d)          # every row of TopK(X) holds min(k, d) entries
    fwd_ms, bwd_ms = statistics.median(tf), statistics.median(tb)
    dense_gflop = 2.0 * A.rows * d * dout / 1e9
    return {"n": A.rows, "d": d, "dout": dout, "k": k, "forward_ms": fwd_ms, "backward_ms": bwd_ms,
            "spgemm_products": int(ip),
            "forward_gflops_all": (2.0 * ip / 1e9 + dense_gflop) / (fwd_ms / 1e3),
            "note": "forward: TopK, A*TopK(X) (hash SpGEMM), dense C*W (spgemm_dense_gemm, "
                    "fp32 CUDA-core GEMM); backward: dY*W^T and C^T*dY (spgemm_dense_gemm, "
                    "split-K with fp64 partial sums), gather at C's pattern, spgemm_backward, "
                    "scatter into dX (M_k-masked)"}


def pattern_sampling(A, device, minibatches: int = 64, batch: int = 1024, fanouts=(25, 10),
                     reps: int = 3):
    """Bulk neighbourhood sampling (Section IV-C): `minibatches` minibatches of
    `batch` vertices of the R-MAT graph stacked in one Q, fanouts per layer;
    per layer P = Q*A, SAMPLE, column selection, EXTRACT = P*S. Uniform
    (GraphSAGE) and squared-weight (LADIES-style) draws. Wall time per bulk
    call (host syncs for the allocations included)."""
    import torch

    from paper_2512_12036_gb300 import Plan, sampling

    plan = Plan(device=device.index)
    rng = np.random.default_rng(12)
    verts = np.concatenate([np.sort(rng.choice(A.rows, size=batch, replace=False))
                            for _ in range(minibatches)])
    out = {"minibatches": minibatches, "batch": batch, "fanouts": list(fanouts)}
    for name, mode in (("uniform", sampling.UNIFORM), ("squared_weights", sampling.BY_SQUARE)):
        sampling.sample_layers(A, verts, fanouts, plan, mode=mode, seed=0)
        torch.cuda.synchronize()
        ts = []
        for r in range(reps):
            t0 = time.perf_counter()
            adj, qs, _ = sampling.sample_layers(A, verts, fanouts, plan, mode=mode, seed=r + 1)
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t0)
        edges = sum(a.nnz for a in adj)
        out[name] = {"ms": 1e3 * statistics.median(ts), "sampled_edges": int(edges),
                     "frontier_sizes": [q.rows for q in qs],
                     "edges_per_s": edges / statistics.median(ts)}
    return out


def served_pool(device, pairs: int, seed: int = 6):
    """Distinct request operands for the mixed-size serving pattern: n
    log-uniform in [1e3, 1e6], Erdos-Renyi or R-MAT (50/50), average degree
    U[4, 32], B independent of A (same n and generator, next seed)."""
    from paper_2512_12036_gb300 import DeviceCSR, gen
    rng = np.random.default_rng(seed)
    pool = []
    for q in range(pairs):
        n = int(np.exp(rng.uniform(np.log(1e3), np.log(1e6))))
        d = float(rng.uniform(4, 32))
        kind = "rmat" if rng.random() < 0.5 else "er"
        make = gen.rmat_graph if kind == "rmat" else gen.erdos_renyi
        Ah = make(n, d, seed=1000 + 2 * q)
        Bh = make(n, d, seed=1001 + 2 * q)
        pool.append((f"{kind}_n{n}_d{d:.0f}", DeviceCSR.from_host(Ah, device),
                     DeviceCSR.from_host(Bh, device), Ah, Bh))
    return pool


def pattern_served(n_requests: int, device, pairs: int = 24, loads=(0.5, 0.8)):
    """Mixed-size serving: `n_requests` A*B requests drawn from a pool of
    `pairs` distinct operand pairs (served_pool), arriving as a Poisson
    process at each load (a fraction of the plain path's measured
    capacity), then all at once (burst). The continuous-batching loop
    (4 slots, 64 GB budget, admission by the product-count bound) against
    the plain per-request path (one request at a time, C allocated per
    call) on the same arrivals; accuracy: one served result per pool pair
    against the oracle on sampled rows."""
    import torch

    import oracle
    from paper_2512_12036_gb300 import Plan, serving

    t0 = time.perf_counter()
    pool = served_pool(device, pairs)
    gen_s = time.perf_counter() - t0
    rng = np.random.default_rng(6)
    picks = rng.integers(0, len(pool), size=n_requests)

    def make():
        return [serving.Request(A=pool[i][1], B=pool[i][2], tag=pool[i][0]) for i in picks]

    plan = Plan(device=device.index)
    svc, ips = [], []
    for _, Ad, Bd, _, _ in pool:            # warm, then the service time of each pair
        plan.spgemm_blocks(Ad, Bd)
        torch.cuda.synchronize()
        ts = []
        for _ in range(3):
            t0 = time.perf_counter()
            blocks, ip_t, _ = plan.spgemm_blocks(Ad, Bd)
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t0)
            del blocks
        svc.append(min(ts))
        ips.append(ip_t)
    mean_svc = float(np.mean([svc[i] for i in picks]))
    gflop = 2.0 * sum(ips[i] for i in picks) / 1e9

    def run_plain(reqs, arrivals):
        t0 = time.perf_counter()
        for req, at in zip(reqs, arrivals):
            now = time.perf_counter() - t0
            if now < at:
                time.sleep(at - now)
            req.arrival = t0 + at
            blocks, req.ip, _ = plan.spgemm_blocks(req.A, req.B)
            torch.cuda.synchronize()
            del blocks
            req.done = time.perf_counter()
        return time.perf_counter() - t0

    srv = serving.gpu_server(slots=4, budget_bytes=64 << 30, device=device.index,
                             keep_results=False)
    out = {"requests": n_requests, "pool_pairs": len(pool), "pool": [p[0] for p in pool],
           "generate_s": round(gen_s, 1), "plain_capacity_rps": 1.0 / mean_svc,
           "gflop_total": gflop}
    try:
        for load in loads:
            rate = load / mean_svc
            arrivals = serving.poisson_arrivals(n_requests, rate, seed=7)
            plain = make()
            wall_p = run_plain(plain, arrivals)
            served = make()
            t0 = time.perf_counter()
            serving.run_served(srv, served, arrivals)
            wall_s = time.perf_counter() - t0
            out[f"load_{load}"] = {
                "arrival_rate_per_s": rate,
                "plain": {**serving.latency_stats(plain), "gflops": gflop / wall_p},
                "served": {**serving.latency_stats(served), "gflops": gflop / wall_s,
                           "errors": sum(1 for r in served if r.error)}}
        burst_p = make()
        wall_p = run_plain(burst_p, np.zeros(n_requests))
        burst_s = make()
        t0 = time.perf_counter()
        serving.run_served(srv, burst_s, np.zeros(n_requests))
        wall_s = time.perf_counter() - t0
        out["burst"] = {"plain": {**serving.latency_stats(burst_p), "gflops": gflop / wall_p},
                        "served": {**serving.latency_stats(burst_s), "gflops": gflop / wall_s,
                                   "errors": sum(1 for r in burst_s if r.error)}}
        out["served_peak_admitted_gb"] = srv.adm.peak / 2**30
    finally:
        srv.close()
    # accuracy: one served result per pool pair, sampled rows against the oracle
    vsrv = serving.gpu_server(slots=4, budget_bytes=64 << 30, device=device.index,
                              keep_results=True)
    worst, checked = 0.0, 0
    try:
        reqs = [serving.Request(A=p[1], B=p[2], tag=p[0]) for p in pool]
        serving.run_served(vsrv, reqs, np.zeros(len(reqs)))
        for req, (_, _, _, Ah, Bh) in zip(reqs, pool):
            if req.error:
                raise RuntimeError(f"served request {req.tag} failed ({req.error})")
            parts = req.result if isinstance(req.result, list) else [req.result]
            sub = req.parts if isinstance(req.result, list) else [req]
            rr = np.random.default_rng(checked)
            for part, C in zip(sub, parts):
                rows = np.unique(rr.integers(0, C.rows, size=min(C.rows, 500)))
                ref = oracle.spgemm(Ah, Bh, rows=rows + part.row_begin)
                rp = C.row_ptr.cpu().numpy().astype(np.int64)
                col, val = C.col.cpu().numpy(), C.val.cpu().numpy()
                gc = np.concatenate([col[rp[i]:rp[i + 1]] for i in rows])
                gv = np.concatenate([val[rp[i]:rp[i + 1]] for i in rows]).astype(np.float64)
                assert np.array_equal(np.diff(ref.row_ptr), rp[rows + 1] - rp[rows])
                assert np.array_equal(gc, ref.col)
                err = np.abs(gv - ref.val) / np.where(ref.bound > 0, ref.bound, 1.0)
                assert (err <= 1e-5).all(), f"served {req.tag}: value outside tolerance"
                worst = max(worst, float(err.max(initial=0.0)))
            checked += 1
    finally:
        vsrv.close()
    out["accuracy"] = {"pairs_checked": checked, "rows_per_pair": "<= 500 sampled",
                       "max_err_over_bound": worst, "tolerance": 1e-5}
    return out


def pattern_mcl(device, iterations: int = 20, jobs: int = 4):
    """Markov clustering on R-MAT scale 18, edge factor 8, symmetrised, with
    self-loops: 20 iterations of expansion, prune < 1e-4, top-32, inflation 2,
    renormalisation. Plain (one spgemm call per expansion) and served (every
    expansion a request to the continuous-batching server, the loop's
    operands staying on the device); the two must give the same clustering.
    Then `jobs` independent clusterings (seeds 4, 5, ...) back to back on
    the plain path against all of them at once through the server."""
    import threading

    import torch

    from paper_2512_12036_gb300 import DeviceCSR, Plan, gen, serving
    from paper_2512_12036_gb300.mcl import markov_cluster, markov_cluster_served

    graphs = [DeviceCSR.from_host(gen.rmat_symmetric(18, 8, seed=4 + j, self_loops=True), device)
              for j in range(jobs)]
    plan = Plan(device=device.index)
    markov_cluster(plan, graphs[0], iterations=1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res = markov_cluster(plan, graphs[0], iterations=iterations)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    ip = sum(res.ip_history)
    srv = serving.gpu_server(slots=4, budget_bytes=64 << 30, device=device.index,
                             keep_results=True)
    try:
        markov_cluster_served(srv, plan, graphs[0], iterations=1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res_s, reqs = markov_cluster_served(srv, plan, graphs[0], iterations=iterations)
        torch.cuda.synchronize()
        dt_s = time.perf_counter() - t0
        same = (res_s.ip_history == res.ip_history and res_s.nnz_history == res.nnz_history)
        a, b = res_s.Mt.to_host(), res.Mt.to_host()
        same = same and np.array_equal(a.col, b.col) and np.array_equal(a.row_ptr, b.row_ptr)
        # several independent clusterings: plain back to back vs all at once
        plans = [Plan(device=device.index) for _ in range(jobs)]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ip_jobs = 0
        for j in range(jobs):
            ip_jobs += sum(markov_cluster(plans[j], graphs[j], iterations=iterations).ip_history)
        torch.cuda.synchronize()
        dt_jobs_plain = time.perf_counter() - t0
        out = [None] * jobs

        def client(j):
            with torch.cuda.stream(torch.cuda.Stream(device=device)):
                out[j] = markov_cluster_served(srv, plans[j], graphs[j], iterations=iterations,
                                               tag=f"job{j}")

        ths = [threading.Thread(target=client, args=(j,)) for j in range(jobs)]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for t in ths:
            t.start()
        for t in ths:
            t.join()
        torch.cuda.synchronize()
        dt_jobs_served = time.perf_counter() - t0
        job_lat = [r.latency for o in out if o for r in o[1]]
    finally:
        srv.close()
    lat = [r.latency for r in reqs]
    return {"workload": "rmat18_ef8_selfloops_mcl", "iterations": iterations,
            "ip_first": res.ip_history[0], "nnz_final": res.nnz_history[-1],
            "plain": {"seconds": dt, "expansion_gflops": 2.0 * ip / dt / 1e9},
            "served": {"seconds": dt_s, "expansion_gflops": 2.0 * ip / dt_s / 1e9,
                       "expansion_p50_ms": 1e3 * _pct(lat, 0.5),
                       "expansion_p99_ms": 1e3 * _pct(lat, 0.99),
                       "same_clustering_as_plain": bool(same)},
            "concurrent_jobs": {"jobs": jobs, "plain_seconds": dt_jobs_plain,
                                "served_seconds": dt_jobs_served,
                                "plain_gflops": 2.0 * ip_jobs / dt_jobs_plain / 1e9,
                                "served_gflops": 2.0 * ip_jobs / dt_jobs_served / 1e9,
                                "served_expansion_p50_ms": 1e3 * _pct(job_lat, 0.5),
                                "served_expansion_p99_ms": 1e3 * _pct(job_lat, 0.99),
                                "all_ok": all(o is not None for o in out)}}


def pattern_er4096(device, reps: int = 50):
    """C = A*A for a 4096 x 4096 Erdos-Renyi adjacency (average degree 8,
    seed 1, fp32 U(0,1], no self-loops): latency of one plain call through
    the public API (C allocated by the call, the result's size read back)
    and of the device-resident form (buffers reused, no host sync inside),
    against the oracle on the host cores."""
    import torch

    import oracle
    from paper_2512_12036_gb300 import DeviceCSR, Plan, gen

    A_h = gen.erdos_renyi(4096, 8, seed=1)
    A = DeviceCSR.from_host(A_h, device)
    plan = Plan(device=device.index)
    ws = plan.workspace(A, A)
    C = plan.spgemm(A, A, ws=ws)
    blocks, ip, nnz = plan.spgemm_blocks(A, A, ws=ws)
    torch.cuda.synchronize()
    lat = []
    for _ in range(reps):
        t0 = time.perf_counter()
        C = plan.spgemm(A, A, ws=ws)
        torch.cuda.synchronize()
        lat.append(time.perf_counter() - t0)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        plan.spgemm_blocks(A, A, ws=ws, out=blocks)
    e1.record(stream)
    e1.synchronize()
    dev_ms = e0.elapsed_time(e1) / reps
    t0 = time.perf_counter()
    for _ in range(5):
        oracle.spgemm(A_h, A_h, nthreads=host_threads(), with_bound=False)
    cpu_ms = 1e3 * (time.perf_counter() - t0) / 5
    ref = oracle.spgemm(A_h, A_h)
    Ch = C.to_host()
    ok = (np.array_equal(Ch.row_ptr.astype(np.int64), ref.row_ptr) and np.array_equal(Ch.col, ref.col)
          and bool((np.abs(Ch.val.astype(np.float64) - ref.val) <= 1e-5 * ref.bound).all()))
    return {"workload": "er4096_deg8_AxA", "ip": int(ip), "nnz_C": int(nnz),
            "plain_call_p50_ms": 1e3 * _pct(lat, 0.5), "plain_call_p99_ms": 1e3 * _pct(lat, 0.99),
            "device_resident_ms": dev_ms, "device_resident_gflops": 2.0 * ip / (dev_ms / 1e3) / 1e9,
            "oracle_ms": cpu_ms, "oracle_cores": host_threads(), "matches_oracle": ok}


def row_cache_size(plan, L, A, device) -> int:
    """MiB of row bitmap cache that holds every row of L*A that reaches a
    dense accumulation tier (one B.cols-bit bitmap and one entry count per
    column panel per row, plus the slot index of every row), or as much of
    it as free device memory allows beside the output (8 bytes per entry of
    C) and 16 GiB of headroom."""
    import torch
    ws = plan.workspace(L, A)
    ip_row, _ = plan.count(L, A, ws)
    row_nnz, nnz = plan.symbolic(L, A, ip_row, ws)
    dense = int((row_nnz > plan.opts["block_max_nnz"]).sum().item())
    del ws, ip_row, row_nnz
    torch.cuda.empty_cache()
    panels = -(-A.cols // plan.opts["panel_cols"])
    need = dense * (((A.cols + 31) // 32) * 4 + 4 * panels) + 4 * L.rows + (1 << 20)
    free, _ = torch.cuda.mem_get_info(device)
    room = free - 8 * nnz - (16 << 30)
    return int(max(0, min(need, room)) >> 20)


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2512_12036_gb300 import DeviceCSR, Plan

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    A_h, S_h, St_h, clusters = workload(args.scale)
    dev = torch.device("cuda", local)
    A = DeviceCSR.from_host(A_h, dev)
    S = DeviceCSR.from_host(S_h, dev)
    St = DeviceCSR.from_host(St_h, dev)
    if args.row_stride > 1:
        from paper_2512_12036_gb300 import gen
        L_h = gen.sample_rows(A_h, args.row_stride)
        L = DeviceCSR.from_host(L_h, dev)
        args.no_e2e = True
    else:
        L_h, L = A_h, A
    opts = {}
    if args.panel_cols:
        opts["panel_cols"] = args.panel_cols
    # the contraction's products run on a plan without the row bitmap cache
    plan_c = Plan(device=local, **opts)
    cache_mb = 0 if args.no_row_cache else row_cache_size(plan_c, L, A, dev)
    if args.dense_splits:
        opts["dense_splits"] = args.dense_splits
    if args.stage_b:
        opts["stage_b"] = 1
    plan = Plan(device=local, row_cache_mb=cache_mb, **opts)
    ws_aa = plan.workspace(L, A)
    ws_sa = plan_c.workspace(St, A)

    # first pass: sizes and output buffers (untimed)
    blocks, ip_aa, nnz_aa = plan.spgemm_blocks(L, A, ws=ws_aa)
    T_blocks, ip_sa, _ = plan_c.spgemm_blocks(St, A, ws=ws_sa)
    T = T_blocks[0][2]
    ws_ts = plan_c.workspace(T, S)
    C2_blocks, ip_ts, nnz_ts = plan_c.spgemm_blocks(T, S, ws=ws_ts)
    plan.check_status(ws_aa, "first pass")
    for ws in (ws_sa, ws_ts):
        plan_c.check_status(ws, "first pass")
    ip_step = ip_aa + ip_sa + ip_ts
    n_blocks = len(blocks)
    stream = torch.cuda.current_stream()

    def step():
        plan.spgemm_blocks(L, A, ws=ws_aa, out=blocks)
        plan_c.spgemm_blocks(St, A, ws=ws_sa, out=T_blocks)
        plan_c.spgemm_blocks(T, S, ws=ws_ts, out=C2_blocks)

    def check_all(where):
        plan.check_status(ws_aa, where)
        for ws in (ws_sa, ws_ts):
            plan_c.check_status(ws, where)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    check_all("warm-up")

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # ---- timed region (device-resident inputs)
    plan.profile(True)
    plan_c.profile(True)
    launches0 = plan.launches() + plan_c.launches()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            step()
        ev1.record(stream)
        barrier()
    ms = ev0.elapsed_time(ev1)
    launches = plan.launches() + plan_c.launches() - launches0
    prof = plan.profile_read()
    for k, (t_ms, n) in plan_c.profile_read().items():
        a_ms, a_n = prof.get(k, (0.0, 0))
        prof[k] = (a_ms + t_ms, a_n + n)
    plan.profile(False)
    plan_c.profile(False)
    check_all("timed steps")
    ms = max_over_ranks(ms, dev)
    ms_step = ms / args.steps
    value = 2.0 * ip_step * world / (ms_step / 1e3) / 1e9

    # ---- per-kernel roofline for the dominant kernel
    ip_row = torch.empty(L.rows, dtype=torch.int64, device=dev)
    ip_row, _ = plan.count(L, A, ws_aa, ip_row=ip_row)
    nnz_row, _ = plan.symbolic(L, A, ip_row, ws_aa)
    work = tier_work(plan, L_h, ip_row.cpu().numpy(), nnz_row.to(torch.int64).cpu().numpy())
    rows_cached = plan.row_cache_rows(L, A, ws_aa)
    top = max(prof.items(), key=lambda kv: kv[1][0])
    top_name, (top_ms, top_n) = top
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    peak_gbs = float(peaks.get("hbm_gbs", 6800.0))
    roof = None
    if top_name in work and top_ms > 0:
        # algorithmic bytes the kernel moves per step (its tier's rows of A*A) over
        # its measured device time per step (= bytes per launch / mean launch time)
        bytes_step = work[top_name]["bytes"]
        achieved = bytes_step / (top_ms / args.steps / 1e3) / 1e9
        traffic = None
        if top_name in DRAM_BYTES_PER_PRODUCT and top_n > 0:
            traffic = int(DRAM_BYTES_PER_PRODUCT[top_name] * work[top_name]["ip"]
                          / (top_n / args.steps))
        roof = {"bound": "hbm", "kernel": top_name, "achieved": achieved, "peak": peak_gbs,
                "unit": "GB/s", "frac": achieved / peak_gbs, "traffic": traffic,
                "traffic_source": "ncu dram bytes per product (small case) x products"
                                  if traffic is not None else None,
                "peak_source": "measured" if "hbm_gbs" in peaks else "fallback",
                "launches_per_step": top_n / args.steps,
                "bytes_per_step": int(bytes_step),
                "share_of_step": top_ms / ms}
    compulsory = (4 * (L.rows + 1) + 8 * L.nnz) + (8 * ip_aa + 8 * L.nnz) + (8 * nnz_aa + 4 * (L.rows + 1))
    step_frac = compulsory / (ms_step / 1e3) / (peak_gbs * 1e9)

    # ---- end to end through the public API from pinned host buffers
    e2e = None
    if not args.no_e2e:
        pin = {k: torch.from_numpy(np.ascontiguousarray(v)).pin_memory() for k, v in
               {"rp": A_h.row_ptr, "col": A_h.col, "val": A_h.val, "srp": S_h.row_ptr,
                "scol": S_h.col, "sval": S_h.val, "trp": St_h.row_ptr, "tcol": St_h.col,
                "tval": St_h.val}.items()}
        h2d = sum(t.numel() * t.element_size() for t in pin.values())
        host_rp = [torch.empty(b[2].row_ptr.numel(), dtype=torch.int32).pin_memory() for b in blocks]
        host_c2 = [torch.empty(C2_blocks[0][2].row_ptr.numel(), dtype=torch.int32).pin_memory(),
                   torch.empty(C2_blocks[0][2].nnz, dtype=torch.int32).pin_memory(),
                   torch.empty(C2_blocks[0][2].nnz, dtype=torch.float32).pin_memory()]
        d2h = sum(t.numel() * t.element_size() for t in host_rp + host_c2)

        # two device copies of the operands: step i's inputs go into set i % 2
        # on a copy stream while step i - 1 computes on the other set; each
        # step's results are read back on the copy stream while the next step
        # runs (its outputs are overwritten only after that read-back ends)
        sets = [(A, S, St), (DeviceCSR.from_host(A_h, dev), DeviceCSR.from_host(S_h, dev),
                             DeviceCSR.from_host(St_h, dev))]
        copy_stream = torch.cuda.Stream(device=dev)
        h2d_done = [torch.cuda.Event(), torch.cuda.Event()]
        comp_done = [torch.cuda.Event(), torch.cuda.Event()]
        rp_done, c2_done = torch.cuda.Event(), torch.cuda.Event()

        def upload(k):
            Ad, Sd, Std = sets[k]
            with torch.cuda.stream(copy_stream):
                copy_stream.wait_event(comp_done[k])        # set k's previous step has ended
                for dst, src in ((Ad.row_ptr, "rp"), (Ad.col, "col"), (Ad.val, "val"),
                                 (Sd.row_ptr, "srp"), (Sd.col, "scol"), (Sd.val, "sval"),
                                 (Std.row_ptr, "trp"), (Std.col, "tcol"), (Std.val, "tval")):
                    dst.copy_(pin[src], non_blocking=True)
                h2d_done[k].record(copy_stream)

        def run(i):
            k = i % 2
            Ad, Sd, Std = sets[k]
            stream.wait_event(h2d_done[k])
            stream.wait_event(rp_done)                      # the last step's row pointers are read
            plan.spgemm_blocks(Ad, Ad, ws=ws_aa, out=blocks)
            stream.wait_event(c2_done)                      # the last step's C(S^T A S) is read
            plan_c.spgemm_blocks(Std, Ad, ws=ws_sa, out=T_blocks)
            plan_c.spgemm_blocks(T, Sd, ws=ws_ts, out=C2_blocks)
            comp_done[k].record(stream)
            with torch.cuda.stream(copy_stream):
                copy_stream.wait_event(comp_done[k])
                for hb, (_, _, Cb) in zip(host_rp, blocks):
                    hb.copy_(Cb.row_ptr, non_blocking=True)
                rp_done.record(copy_stream)
                C2 = C2_blocks[0][2]
                host_c2[0].copy_(C2.row_ptr, non_blocking=True)
                host_c2[1].copy_(C2.col, non_blocking=True)
                host_c2[2].copy_(C2.val, non_blocking=True)
                c2_done.record(copy_stream)

        def e2e_steps(n, start=None):
            if start is not None:
                copy_stream.wait_event(start)               # no copy before the timed region
            upload(0)
            for i in range(n):
                if i + 1 < n:
                    upload((i + 1) % 2)
                run(i)
            stream.wait_event(c2_done)                      # the last read-back is inside

        e2e_steps(2)
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(local) as clk_e2e:
            e0.record(stream)
            e2e_steps(args.steps, start=e0)
            e1.record(stream)
            barrier()
        ems = e0.elapsed_time(e1)
        ems = max_over_ranks(ems, dev)
        e2e = {"value": 2.0 * ip_step * world / (ems / args.steps / 1e3) / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "clocks": clk_e2e.summary(),
               "note": "inputs copied from pinned host memory each step (into one of two device "
                       "copies of the operands, overlapped with the previous step); C(S^T A S) "
                       "and the row pointers of every A*A block read back (the A*A values stay "
                       "in HBM)"}

    patterns = None
    if rank == 0 and world == 1 and not args.no_patterns:
        del blocks
        torch.cuda.empty_cache()
        patterns = {}
        patterns["served"] = pattern_served(args.served_requests, dev)
        torch.cuda.empty_cache()
        patterns["batched_gnn"] = pattern_batched(args.gnn_graphs, dev)
        torch.cuda.empty_cache()
        patterns["mcl"] = pattern_mcl(dev)
        torch.cuda.empty_cache()
        patterns["er4096"] = pattern_er4096(dev)
        torch.cuda.empty_cache()
        patterns["bulk_sampling"] = pattern_sampling(A, dev)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(A_h, args.cpu_seconds)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 (fp64 accumulation where "
            "more than 167 terms can meet)", "data": "synthetic",
            "row_cache": {"mib": cache_mb, "rows_with_slot": rows_cached},
            "config": {"workload": workload_name(args.scale, args.row_stride),
                       "rmat_scale": args.scale, "row_stride_AxA": args.row_stride,
                       "edge_factor": 16, "abcd": [0.57, 0.19, 0.19, 0.05],
                       "nnz_A": A.nnz, "clusters": clusters, "ip_step": ip_step,
                       "ip_AxA": ip_aa, "nnz_AxA": nnz_aa, "row_blocks_AxA": n_blocks,
                       "nnz_StAS": nnz_ts, "l2": "inputs larger than L2, no flush",
                       "plan_opts": plan.opts,
                       "parallelism": f"replicas{world}"},
            "roofline": roof,
            "step_hbm_fraction": {"compulsory_bytes_AxA": int(compulsory), "frac": step_frac,
                                  "peak_gbs": peak_gbs},
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
            "clocks": clk.summary(),
            "kernel_ms_per_step": {k: round(v[0] / args.steps, 3) for k, v in
                                   sorted(prof.items(), key=lambda kv: -kv[1][0])},
            "tiers_AxA": {k: {q: v[q] for q in ("rows", "ip", "nnz")} for k, v in work.items()},
            "patterns": patterns,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    A_h, _, _, _ = workload(args.scale)
    ip, _ = oracle.ip_count(A_h, A_h)
    cores = host_threads()
    rng = np.random.default_rng(1)
    # each step: a fresh uniformly drawn sample of ~1e8 intermediate products
    target = 1e8 if args.scale >= 18 else 1e7
    samples = []
    for _ in range(args.warmup + args.steps):
        order = rng.permutation(A_h.rows).astype(np.int32)
        k = int(np.searchsorted(np.cumsum(ip[order]), target)) + 1
        samples.append(order[:k])
    for r in samples[:args.warmup]:
        oracle.spgemm(A_h, A_h, rows=r, nthreads=cores, with_bound=False)
    prods = 0.0
    t0 = time.perf_counter()
    for r in samples[args.warmup:]:
        oracle.spgemm(A_h, A_h, rows=r, nthreads=cores, with_bound=False)
        prods += float(ip[r].sum())
    t = time.perf_counter() - t0
    value = 2 * prods / t / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": workload_name(args.scale), "rmat_scale": args.scale},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"per step ~{target:.0e} intermediate products of A*A "
                                       "from uniformly drawn rows"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_one_pattern(args):
    """One pattern measurement alone (for profiling a pattern's kernels);
    prints its record as one JSON line. Not the benchmark line."""
    import torch
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    if args.only == "batched":
        rec = pattern_batched(args.gnn_graphs, dev)
    elif args.only == "served":
        rec = pattern_served(args.served_requests, dev)
    elif args.only == "mcl":
        rec = pattern_mcl(dev)
    else:
        rec = pattern_er4096(dev)
    print(json.dumps({"pattern": args.only, **rec}), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.only:
        run_one_pattern(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
