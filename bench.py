#!/usr/bin/env python
"""Dynamic CSC throughput on one GB300 (or N independent replicas).

Headline workload (the large power-law configuration): Chung-Lu graph with
n = 8,000,000 nodes, power-law expected degrees (exponent 2.5, mean 25, about
1.9e8 stored entries), k = 64 planted communities with mixing 0.2; a sequence of
snapshots with 0.2% edge redrawing per step; d = 192 signals stored in bfloat16
(float32 recursion, float64 sums), Chebyshev order m = 80, reuse p = 0.8 (39 new
columns per snapshot), cutoff found by the eigencount dichotomy.  One bench step
is one snapshot through the whole hot path: set_graph, filter (signals,
recursion, moments, eigencount check and refinement, splice, row
normalisation) and k-means.

value = sum over timed snapshots of nnz * (columns filtered) * m / device time.
Reused columns and refinement passes are not credited.  Inputs (all snapshots'
CSR) are resident in HBM before the timed region; each snapshot reads a 0.8 GB
CSR and a 6 GB feature ring, so the inputs of every step exceed L2 (no flush).

Extra keys: the SBM sequence at n = 1e6 (d = 256, m = 100, p = 0.75, float32),
the batched-vs-plain comparison on 512 graphs, the differentiation timing and
the compressive k-means timing.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Chebyshev-filter nnz·d·m/s + HBM GB/s fraction; batched BF16 vs plain FP32 GPU"
UNIT = "nnz*col*order/s"
PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC = os.path.join(ROOT, "profiles", "cheb_step_traffic.json")

# the large power-law workload (headline)
CL = dict(name="chung_lu_8e6", n=8_000_000, exponent=2.5, deg=25.0, k=64, mixing=0.2, d=192, m=80,
          p=0.8, churn=0.002, precision=1)
# the dynamic SBM at scale (extra key)
SBM = dict(name="sbm_1e6", n=1_000_000, k=100, deg=30.0, ratio=10.0, zipf=0.8, d=256, m=100, p=0.75,
           churn=0.005, precision=0)
CPU_ORDER = 16   # Chebyshev steps per column in the bounded CPU samples
REF_ORDER = 4    # recursion order of one reference-arm step (a bounded sample of the m = 80 filter)
ORDERS = {0: "caller order", 1: "library order: degrees descending",
          2: "library order: degrees descending, regrouped by the first clustering"}


def args_parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--nodes", type=int, default=CL["n"],
                    help="nodes of the power-law workload (smaller values for profiling captures)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--tile", type=int, default=0, help="column-tile width (0 = library default)")
    ap.add_argument("--reorder", type=int, default=2,
                    help="node order of the library for the power-law workload (0 caller, 1 degrees, "
                         "2 degrees then grouped by the first clustering)")
    ap.add_argument("--no-sbm", action="store_true", help="skip the n = 1e6 SBM sequence")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-vs-plain comparison")
    ap.add_argument("--no-grad", action="store_true", help="skip the differentiation timing")
    ap.add_argument("--no-compressive", action="store_true", help="skip the compressive k-means timing")
    a = ap.parse_args()
    a.warmup = max(3, a.warmup)
    return a


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class Dist:
    """Barrier and max/sum reductions over ranks (gloo, host scalars only)."""

    def __init__(self, world):
        self.world = world
        if world > 1:
            import torch.distributed as dist
            dist.init_process_group("gloo")
            self.d = dist

    def barrier(self):
        if self.world > 1:
            self.d.barrier()

    def reduce(self, val, op):
        if self.world == 1:
            return val
        import torch
        t = torch.tensor([float(val)], dtype=torch.float64)
        self.d.all_reduce(t, op=self.d.ReduceOp.MAX if op == "max" else self.d.ReduceOp.SUM)
        return float(t.item())

    def close(self):
        if self.world > 1:
            self.d.destroy_process_group()


def cl_sequence(count, seed, n, device):
    """(row_ptr, col_idx) of `count` snapshots of the power-law workload, the nnz of each and
    the planted labels, generated on `device`."""
    import workloads as W
    g = W.chung_lu_graph_torch(n, CL["exponent"], CL["deg"], CL["k"], CL["mixing"], seed=seed, device=device)
    out, nnz = [(g.row_ptr, g.col_idx)], [g.nnz]
    for t in range(1, count):
        g = W.edge_redraw_torch(g, CL["churn"], seed=seed * 7919 + t)
        out.append((g.row_ptr, g.col_idx))
        nnz.append(g.nnz)
    return out, nnz, g.labels


def sbm_sequence(count, seed, device):
    import workloads as W
    sizes = W.zipf_block_sizes(SBM["n"], SBM["k"], SBM["zipf"])
    g = W.sbm_graph_torch(SBM["n"], sizes, SBM["deg"], SBM["ratio"], seed=seed, device=device)
    out, nnz = [(g.row_ptr, g.col_idx)], [g.nnz]
    for t in range(1, count):
        g = W.edge_redraw_torch(g, SBM["churn"], seed=seed * 7919 + t)
        out.append((g.row_ptr, g.col_idx))
        nnz.append(g.nnz)
    return out, nnz, g.labels


class Clocks:
    """nvidia-smi sampler running during a timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def peak_hbm():
    try:
        with open(PEAKS) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def kernel_sha():
    src = os.path.join(ROOT, "paper_1706_03591_gb300", "csrc", "cheb.cu")
    with open(src, "rb") as fh:
        return hashlib.sha256(fh.read()).hexdigest()[:16]


def ncu_traffic(workload, tile):
    """DRAM bytes per step launch from the committed ncu record of this workload and tile, if it
    was taken on the current step kernel."""
    try:
        with open(TRAFFIC) as fh:
            rec = json.load(fh)
    except (OSError, ValueError):
        return None
    for r in rec.get("records", []):
        if r.get("kernel_sha") == kernel_sha() and r.get("workload") == workload and int(r.get("tile", -1)) == tile:
            return r.get("dram_bytes_per_launch")
    return None


def _oracle_columns(lt, n, d, cols, order, threads, seed):
    """Runs the float64 oracle filter on `cols` independent signal columns over the shared CSR
    `lt`, one column per thread (scipy's sparse products release the GIL); returns seconds."""
    import numpy as np

    import workloads as W
    from oracle import chebyshev as cb
    blocks = [W.gaussian_block(n, 1, d, seed=seed + q).astype(np.float64) for q in range(cols)]
    lam = 0.1

    def work(q):
        cb.cheb_filter(lt, blocks[q], order, lam)

    t0 = time.perf_counter()
    for base in range(0, cols, threads):
        th = [threading.Thread(target=work, args=(q,)) for q in range(base, min(cols, base + threads))]
        for h in th:
            h.start()
        for h in th:
            h.join()
    return time.perf_counter() - t0


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_baseline(n, row_ptr, col_idx, d, label):
    """The float64 oracle as it stands, on a bounded sample of the workload's first snapshot:
    order-CPU_ORDER recursions of independent signal columns, first one column on one thread,
    then one column per thread on every host core."""
    from oracle import laplacian as lp
    lt = lp.shifted_laplacian(n, row_ptr, col_idx)
    nnz = int(col_idx.size)
    t1 = _oracle_columns(lt, n, d, 1, CPU_ORDER, 1, seed=5)
    cores = host_cores()
    tc = _oracle_columns(lt, n, d, cores, CPU_ORDER, cores, seed=5)
    single = nnz * CPU_ORDER / t1
    value = nnz * cores * CPU_ORDER / tc
    return {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
            "single_thread": single,
            "sample": f"oracle.chebyshev.cheb_filter (float64 scipy CSR) on {label}'s first snapshot "
                      f"(n={n}, nnz={nnz}): order {CPU_ORDER} on one column per thread, {cores} threads "
                      f"({tc:.1f} s); single thread one column {t1:.1f} s"}


def batched_comparison(seed=77, count=512, m=60):
    """Batched BF16 (one persistent graph-captured launch) vs plain FP32 (one graph at a time)
    on the many-graphs workload: 512 graphs alternating SBM / Chung-Lu, n log-uniform in
    [1e3, 2e5], k ~ U{5..50}, expected degree ~ U[10, 40], d = c = 4k, m = 60."""
    import numpy as np
    import torch

    import paper_1706_03591_gb300 as csc
    import workloads as W
    rng = np.random.default_rng(seed)
    graphs = []
    for i in range(count):
        n = int(np.exp(rng.uniform(np.log(1e3), np.log(2e5))))
        k = int(rng.integers(5, 51))
        deg = float(rng.uniform(10, 40))
        g = (W.sbm_graph_torch(n, k, deg, 10, seed=seed + i, device="cuda") if i % 2 == 0 else
             W.chung_lu_graph_torch(n, 2.5, deg, k, 0.2, seed=seed + i, device="cuda"))
        graphs.append(dict(n=g.n, row_ptr=g.row_ptr, col_idx=g.col_idx, vals=None, c=4 * k, d=4 * k,
                           lambda_c=float(rng.uniform(0.2, 1.0)), seed=seed * 1000 + i,
                           psi=torch.zeros((g.n, 4 * k), device="cuda")))
        del g
    units = float(sum(g["col_idx"].numel() * g["c"] * m for g in graphs))
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    reps = 3
    with csc.Context({"precision": 1}) as ctx:
        ctx.filter_batched(graphs, m)          # plan, autotune, capture
        ctx.stats(reset=True)
        torch.cuda.synchronize()
        ev[0].record(stream)
        for _ in range(reps):
            ctx.filter_batched(graphs, m)
        ev[1].record(stream)
        torch.cuda.synchronize()
        st = ctx.stats()
    t_batched = ev[0].elapsed_time(ev[1]) / reps
    # the same kernels one graph at a time, in the caller's node order like the batched launch
    with csc.Context({"precision": 0, "reorder": 0}) as ctx:
        rbuf = torch.zeros(max(g["n"] * g["c"] for g in graphs), device="cuda")

        def plain():
            for g in graphs:
                ctx.set_graph(g["n"], g["row_ptr"], g["col_idx"])
                r = rbuf[: g["n"] * g["c"]].view(g["n"], g["c"])
                ctx.signals(g["seed"], g["n"], 0, g["c"], g["d"], r)
                ctx.cheb_filter(m, g["lambda_c"], r, g["psi"], want_moments=True)
        plain()
        torch.cuda.synchronize()
        ev[2].record(stream)
        plain()
        ev[3].record(stream)
        torch.cuda.synchronize()
    t_plain = ev[2].elapsed_time(ev[3])
    sum_n = int(sum(g["n"] for g in graphs))
    sum_nnz = int(sum(g["col_idx"].numel() for g in graphs))
    return {"workload": f"{count} graphs (SBM / Chung-Lu alternating), n log-uniform [1e3, 2e5], "
                        f"k U[5,50], degree U[10,40], d=c=4k, m={m}; sum n={sum_n}, sum nnz={sum_nnz}",
            "graphs": count, "units_per_batch": units,
            "batched_bf16": {"value": units / (t_batched / 1e3), "ms": t_batched,
                             "graph_replays": st["graph_replays"], "launches": st["batched_launches"],
                             "waves": st["batched_waves"]},
            "plain_fp32": {"value": units / (t_plain / 1e3), "ms": t_plain},
            "speedup": t_plain / t_batched, "unit": UNIT}


def differentiation_timing(seed=4, reps=3):
    """Forward, loss gradient and vector-Jacobian product of the k-means loss of the filtered
    features, at the differentiation workload's size: SBM n = 2e5, k = 20, degree 25, d = 128,
    m = 60, unit weights, float32.  Two checkpoint plans: every step kept (stride 1, 6.1 GB at
    this size, nothing recomputed) and every ceil(sqrt m) = 8 steps (the backward pass
    recomputes each segment)."""
    import numpy as np
    import torch

    import paper_1706_03591_gb300 as csc
    import workloads as W
    n, k, c, m = 200_000, 20, 128, 60
    g = W.sbm_graph(n, k, 25, 10, seed=seed)
    gen = torch.Generator(device="cuda").manual_seed(seed)
    r = torch.randn((g.n, c), device="cuda", generator=gen) / float(np.sqrt(c))
    mu = torch.nn.functional.normalize(torch.randn((k, c), device="cuda", generator=gen), dim=1)
    assign = torch.randint(0, k, (g.n,), device="cuda", generator=gen, dtype=torch.int32)
    a = csc.csc_filter_coeffs(m, 0.3)
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    units = float(g.nnz) * c * m
    out = {"workload": f"SBM n={n}, k={k}, degree 25, d={c}, m={m}, unit weights, fp32", "nnz": int(g.nnz),
           "unit": UNIT}
    for name, stride in (("every_step_kept", 1), ("checkpoints_every_8", 0)):
        with csc.Context() as ctx:
            ctx.set_graph(g.n, torch.from_numpy(g.row_ptr).cuda(), torch.from_numpy(g.col_idx).cuda())
            psi = torch.zeros((g.n, c), device="cuda")
            gpsi = torch.zeros_like(psi)
            gw = torch.zeros(g.col_idx.size, device="cuda")
            t = [0.0, 0.0, 0.0]
            for rep in range(reps + 1):
                torch.cuda.synchronize()
                ev[0].record(stream)
                ctx.filter_forward(m, a, r, psi, stride)
                ev[1].record(stream)
                ctx.kmeans_loss_grad(psi, mu, assign, gpsi)
                ev[2].record(stream)
                ctx.filter_vjp(gpsi, gw)
                ev[3].record(stream)
                torch.cuda.synchronize()
                if rep > 0:
                    for i in range(3):
                        t[i] += ev[i].elapsed_time(ev[i + 1]) / reps
        out[name] = {"forward_ms": t[0], "loss_grad_ms": t[1], "vjp_ms": t[2],
                     "backward_over_forward": t[2] / t[0], "forward_rate": units / (t[0] / 1e3)}
    out["backward_over_forward"] = out["every_step_kept"]["backward_over_forward"]
    return out


def compressive_timing(ctx, full_assign, planted, k, n, seed=11, reps=3):
    """Compressive k-means (sampled k-means + k interpolating filterings) on the context's
    last snapshot, against the full k-means assignment of the same features and against the
    planted blocks of the generator."""
    import numpy as np
    import torch
    from scipy.optimize import linear_sum_assignment

    def agreement(a, b):
        c = np.zeros((k, k))
        np.add.at(c, (a, b), 1)
        ri, ci = linear_sum_assignment(-c)
        return float(c[ri, ci].sum() / a.size)

    full = full_assign.cpu().numpy()
    out = torch.zeros(n, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    res = {}
    for label, draws in (("default", 0), ("4x", int(np.ceil(8 * k * np.log(k))))):
        ctx.compressive_cluster(k, n_draws=draws, seed=seed, assign_out=out)  # warm-up
        st0 = ctx.stats()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        torch.cuda.synchronize()
        ev[0].record(stream)
        for _ in range(reps):
            r = ctx.compressive_cluster(k, n_draws=draws, seed=seed, assign_out=out)
        ev[1].record(stream)
        torch.cuda.synchronize()
        st1 = ctx.stats()
        got = out.cpu().numpy()
        res[label] = {"n_draws": draws or int(np.ceil(2 * k * np.log(k))),
                      "n_sampled": r["n_sampled"], "ms": ev[0].elapsed_time(ev[1]) / reps,
                      "interpolation_step_ms": (st1["step_ms"] - st0["step_ms"]) / reps,
                      "agreement_with_full_kmeans": agreement(got, full),
                      "agreement_with_planted": agreement(got, planted)}
    return {"workload": f"last timed snapshot of the SBM sequence: k={k} clusters, 10 restarts of the "
                        "reduced k-means, interpolation by the low pass of the features",
            "full_kmeans_agreement_with_planted": agreement(full, planted), **res}


def workload_config(cfg, n, tile):
    dq = cfg["d"] - int(cfg["p"] * cfg["d"])
    if cfg is CL:
        desc = (f"large power-law: Chung-Lu n={n}, degree exponent 2.5, mean degree 25, k=64 planted "
                f"communities (mixing 0.2), 0.2% edge churn per snapshot, d=192 bf16 signals with fp32 "
                f"recursion, m=80, p=0.8, cutoff by eigencount dichotomy")
    else:
        desc = ("dynamic CSC at scale: SBM n=1e6, k=100 Zipf(0.8) blocks, degree 30, p_in/p_out=10, "
                "0.5% edge churn per snapshot, d=256, m=100, p=0.75, fp32")
    out = {"workload": desc, "n": n, "k": cfg["k"], "avg_degree": cfg["deg"], "d": cfg["d"], "m": cfg["m"],
           "p": cfg["p"], "cols_filtered_per_step": dq, "churn": cfg["churn"],
           "signal_storage": "bf16" if cfg["precision"] == 1 else "fp32",
           "l2": "inputs larger than L2 (CSR + feature ring per snapshot exceed 129 MB; no flush)",
           "parallelism": "replicas (independent snapshot sequences per GPU)"}
    if tile is not None:
        out["col_tile"] = tile
    return out


def run_reference(a, rank, world):
    """The float64 oracle on the host cores: per step, one column per core through REF_ORDER
    recursions on the headline workload's first timed snapshot (warm-up steps: order 1).  The
    snapshots differ by 0.2 % of their edges, so one CSR stands for all of them, and building
    the oracle's 2e8-entry matrix once keeps the whole run within a few minutes."""
    if rank != 0:
        return 0
    import numpy as np
    import torch

    from oracle import laplacian as lp
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    seq, nnz, _ = cl_sequence(a.warmup + 1, seed=1000, n=a.nodes, device=dev)
    rp, ci = seq[a.warmup]
    rp_h, ci_h = rp.cpu().numpy(), ci.cpu().numpy()
    del seq
    lt = lp.shifted_laplacian(a.nodes, rp_h, ci_h)
    cores = host_cores()
    units, total = 0.0, 0.0
    for t in range(a.warmup + a.steps):
        order = REF_ORDER if t >= a.warmup else 1
        dt = _oracle_columns(lt, a.nodes, CL["d"], cores, order, cores, seed=t * 1000)
        if t >= a.warmup:
            units += nnz[a.warmup] * cores * order
            total += dt
    value = units / total
    sample = (f"per step: oracle.chebyshev.cheb_filter (float64 scipy CSR) on the first timed snapshot "
              f"(n={a.nodes}, nnz={nnz[a.warmup]}), one signal column per thread on {cores} threads, order "
              f"{REF_ORDER} of {CL['m']} (throughput per nnz*col*order is the same at every order); "
              f"warm-up steps at order 1")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": 1e3 * total / a.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference", "config": workload_config(CL, a.nodes, None),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_sequence(ctx, cfg, n, graphs, nnz, seed, inits, assign, timed_from, clocks, dist):
    """Runs Algorithm 1 over all snapshots; returns (device ms of the timed part, credited
    units, per-step details, clock record, mean phase times).

    Host graphs (the end-to-end run, pinned memory) are copied to the device on a second
    stream into two alternating buffers: the copy of snapshot t + 1 overlaps the filtering and
    clustering of snapshot t.  Every timed snapshot's copy lies inside the timed region: the
    first timed one is copied after the region opens, without overlap."""
    import torch
    stream = torch.cuda.current_stream()
    units = 0.0
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    marks, info = [], []
    host = graphs[0][0].device.type == "cpu"
    if host:
        copy_stream = torch.cuda.Stream()
        max_nnz = max(int(ci.numel()) for _, ci in graphs)
        bufs = [(torch.empty(n + 1, dtype=torch.int64, device="cuda"),
                 torch.empty(max_nnz, dtype=torch.int32, device="cuda")) for _ in range(2)]
        copied = [None] * len(graphs)
        freed = [None, None]

        def stage(t, on_side):
            rp_h, ci_h = graphs[t]
            drp, dci = bufs[t % 2]
            dci = dci[:ci_h.numel()]
            st = copy_stream if on_side else stream
            if on_side and freed[t % 2] is not None:
                copy_stream.wait_event(freed[t % 2])
            with torch.cuda.stream(st):
                drp.copy_(rp_h, non_blocking=True)
                dci.copy_(ci_h, non_blocking=True)
                ev = torch.cuda.Event()
                ev.record(st)
            copied[t] = (ev, drp, dci)
    for t in range(len(graphs)):
        if t == timed_from:
            ctx.stats(reset=True)
            dist.barrier()
            torch.cuda.synchronize()
            clocks.start()
            e0.record(stream)
        if host:
            if copied[t] is None:
                stage(t, on_side=False)
            ev, rp, ci = copied[t]
            stream.wait_event(ev)
        else:
            rp, ci = graphs[t]
        ev_t = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ev_t[0].record(stream)
        ctx.set_graph(n, rp, ci)
        ev_t[1].record(stream)
        if host:
            freed[t % 2] = torch.cuda.Event()
            freed[t % 2].record(stream)
            if t + 1 < len(graphs) and t + 1 != timed_from:
                stage(t + 1, on_side=True)
        lam, cnt, ev, cols = ctx.filter(cfg["m"], cfg["d"], cfg["p"], seed, cfg["k"])
        ev_t[2].record(stream)
        cost, iters = ctx.cluster(cfg["k"], seed, inits[t], assign)
        ev_t[3].record(stream)
        if t >= timed_from:
            marks.append(ev_t)
            units += nnz[t] * cols * cfg["m"]
            info.append(dict(lam=lam, count=cnt, evals=ev, cols=cols, iters=iters))
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    dist.barrier()
    phases = {name: sum(m[i].elapsed_time(m[i + 1]) for m in marks) / max(1, len(marks))
              for i, name in enumerate(("set_graph", "filter", "cluster"))}
    for i, ph in zip(info, marks):
        i["filter_ms"] = ph[1].elapsed_time(ph[2])
        i["cluster_ms"] = ph[2].elapsed_time(ph[3])
    return e0.elapsed_time(e1), units, info, clk, phases


def roofline(stats, n, nnz_mean, tile, workload):
    """The step kernel's algorithmic bytes (summed by the library over the timed launches, each
    counted for its own tile width) over its CUDA-event time."""
    peak, peak_kind = peak_hbm()
    launches = max(1, stats["step_launches"])
    avg_launch_s = stats["step_ms"] / launches / 1e3
    bytes_launch = stats["step_bytes"] / launches
    achieved = stats["step_bytes"] / (stats["step_ms"] / 1e3) / 1e9 if stats["step_ms"] > 0 else None
    return {"kernel": "cheb_rows_kernel (general step)", "bound": "hbm", "achieved": achieved, "peak": peak,
            "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak if achieved else None,
            "traffic": ncu_traffic(workload, tile), "avg_launch_us": avg_launch_s * 1e6,
            "launches_timed": stats["step_launches"], "bytes_per_launch": bytes_launch,
            "widest_tile": tile}


def sbm_extra(a, rank, dist, clocks_cls, local):
    """The n = 1e6 SBM sequence (20 snapshots: 4 warm-up, 16 timed) with its roofline and the
    compressive k-means timing on its last snapshot."""
    import numpy as np
    import torch

    import paper_1706_03591_gb300 as csc
    import workloads as W
    seed = 2000 + rank
    graphs, nnz, labels = sbm_sequence(20, seed, "cuda")
    inits = [W.forgy_indices(SBM["n"], SBM["k"], seed=seed + t) for t in range(len(graphs))]
    ctx = csc.Context({"timing": 1, "col_tile": a.tile, "precision": SBM["precision"]})
    assign = torch.zeros(SBM["n"], dtype=torch.int32, device="cuda")
    ms, units, info, clk, phases = run_sequence(ctx, SBM, SBM["n"], graphs, nnz, seed, inits, assign, 4,
                                                clocks_cls(local), dist)
    stats = ctx.stats()
    comp = None
    if not a.no_compressive:
        comp = compressive_timing(ctx, assign, labels.cpu().numpy(), SBM["k"], SBM["n"])
    ctx.close()
    nnz_mean = float(np.mean(nnz[4:]))
    return {"config": workload_config(SBM, SBM["n"], int(stats["tile"])), "value": units / (ms / 1e3),
            "unit": UNIT, "ms_per_step": ms / 16, "phase_ms": phases, "clocks": clk,
            "roofline": roofline(stats, SBM["n"], nnz_mean, int(stats["tile"]), SBM["name"]),
            "kmeans_iters": [i["iters"] for i in info],
            "kmeans": {"passes": stats["kmeans_passes"],
                       "near_ties_per_pass": stats["kmeans_near_ties"] / max(1, stats["kmeans_passes"]),
                       "rows_evaluated_fraction": stats["kmeans_rows"] / max(1, stats["kmeans_passes"] * SBM["n"])},
            "compressive_kmeans": comp}


def run_ours(a, rank, world, local):
    import numpy as np
    import torch

    import paper_1706_03591_gb300 as csc
    import workloads as W
    dist = Dist(world)
    torch.cuda.set_device(local)
    seed = 1000 + rank
    n = a.nodes
    count = a.warmup + a.steps
    graphs, nnz, labels = cl_sequence(count, seed, n, "cuda")
    inits = [W.forgy_indices(n, CL["k"], seed=seed + t) for t in range(count)]
    clocks = Clocks(local)
    opts = {"timing": 1, "col_tile": a.tile, "precision": CL["precision"], "reorder": a.reorder}
    ctx = csc.Context(opts)
    assign = torch.zeros(n, dtype=torch.int32, device="cuda")
    ms, units, info, clk, phases = run_sequence(ctx, CL, n, graphs, nnz, seed, inits, assign, a.warmup,
                                                clocks, dist)
    stats = ctx.stats()
    tile = int(stats["tile"])
    ctx.close()
    ms_max = dist.reduce(ms, "max")
    units_all = dist.reduce(units, "sum")
    value = units_all / (ms_max / 1e3)

    e2e = None
    if not a.no_e2e:
        host_graphs = [(rp.cpu().pin_memory(), ci.cpu().pin_memory()) for rp, ci in graphs]
        assign_h = torch.zeros(n, dtype=torch.int32).pin_memory()
        ctx2 = csc.Context(opts)
        ms2, units2, _, _, _ = run_sequence(ctx2, CL, n, host_graphs, nnz, seed, inits, assign_h, a.warmup,
                                            Clocks(local), dist)
        ctx2.close()
        del host_graphs
        ms2_max = dist.reduce(ms2, "max")
        units2_all = dist.reduce(units2, "sum")
        nnz_mean = float(np.mean(nnz[a.warmup:]))
        e2e = {"value": units2_all / (ms2_max / 1e3), "unit": UNIT,
               "h2d_bytes_per_step": int(8 * (n + 1) + 4 * nnz_mean), "d2h_bytes_per_step": 4 * n}

    base = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        rp, ci = graphs[0]
        base = cpu_baseline(n, rp.cpu().numpy(), ci.cpu().numpy(), CL["d"], "the power-law workload")
    del graphs
    torch.cuda.empty_cache()
    sbm = None
    if rank == 0 and not a.no_sbm:
        sbm = sbm_extra(a, rank, Dist(1), Clocks, local)
        torch.cuda.empty_cache()
    batched = None
    if rank == 0 and not a.no_batched:
        batched = batched_comparison()
        torch.cuda.empty_cache()
    grad = None
    if rank == 0 and not a.no_grad:
        grad = differentiation_timing()
    dist.close()
    if rank != 0:
        return 0
    nnz_timed = float(np.mean(nnz[a.warmup:]))
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": ms_max / a.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16 signals, f32 recursion, f64 sums",
        "data": "synthetic",
        "config": {**workload_config(CL, n, tile), "node_order": ORDERS[a.reorder]},
        "roofline": roofline(stats, n, nnz_timed, tile, CL["name"] if n == CL["n"] else f"chung_lu_{n}"),
        "cpu_baseline": base,
        "e2e": e2e,
        "clocks": clk,
        "gpu_launches": stats["launches"],
        "phase_ms": phases,
        "per_step": {"lambda": [i["lam"] for i in info], "count": [i["count"] for i in info],
                     "evals": [i["evals"] for i in info], "kmeans_iters": [i["iters"] for i in info],
                     "filter_ms": [i["filter_ms"] for i in info], "cluster_ms": [i["cluster_ms"] for i in info]},
        "kmeans": {"passes": stats["kmeans_passes"],
                   "near_ties_per_pass": stats["kmeans_near_ties"] / max(1, stats["kmeans_passes"]),
                   "rows_evaluated_fraction": stats["kmeans_rows"] / max(1, stats["kmeans_passes"] * n)},
        "nnz_mean": nnz_timed,
        "sbm_1e6": sbm,
        "batched_vs_plain": batched,
        "differentiation": grad,
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    a = args_parse()
    rank, world, local = dist_env()
    if a.impl == "reference":
        return run_reference(a, rank, world)
    return run_ours(a, rank, world, local)


if __name__ == "__main__":
    sys.exit(main())
