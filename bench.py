#!/usr/bin/env python
"""Dynamic CSC throughput on one GB300 (or N independent replicas).

Workload (the at-scale dynamic configuration): stochastic block model with
n = 1,000,000 nodes, k = 100 blocks of Zipf(0.8) sizes, expected degree 30,
p_in/p_out = 10, unit weights; a sequence of snapshots with 0.5% edge redrawing
per step; d = 256 signals, Chebyshev order m = 100, reuse p = 0.75 (64 new
columns per snapshot), float32.  One bench step is one snapshot through the
whole hot path: set_graph, filter (signals, recursion, moments, eigencount,
cutoff check/refinement, splice, row normalisation) and k-means.

value = sum over timed snapshots of nnz * (columns filtered) * m / device time.
Reused columns are not credited.  Inputs (all snapshots' CSR) are resident in
HBM before the timed region; each snapshot reads a 128 MB CSR and a 1 GB
feature ring, so the inputs of every step exceed L2.

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
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Chebyshev-filter nnz·d·m/s + HBM GB/s fraction; batched BF16 vs plain FP32 GPU"
UNIT = "nnz*col*order/s"
N_NODES, K_CLUST, DEG, RATIO, ZIPF = 1_000_000, 100, 30.0, 10.0, 0.8
D_SIG, M_ORDER, P_REUSE, CHURN = 256, 100, 0.75, 0.005
PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC = os.path.join(ROOT, "profiles", "cheb_step_traffic.json")


def args_parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=16)
    ap.add_argument("--warmup", type=int, default=4)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--tile", type=int, default=0, help="column-tile width (0 = library default)")
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


def make_snapshots(count, seed):
    import workloads as W
    sizes = W.zipf_block_sizes(N_NODES, K_CLUST, ZIPF)
    g = W.sbm_graph(N_NODES, sizes, DEG, RATIO, seed=seed)
    out = [g]
    for t in range(1, count):
        out.append(W.edge_redraw(out[-1], CHURN, seed=seed * 7919 + t))
    return out


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


def ncu_traffic(tile):
    """dram bytes per step launch from the committed ncu summary, if it matches this kernel."""
    try:
        with open(TRAFFIC) as fh:
            rec = json.load(fh)
    except (OSError, ValueError):
        return None
    if rec.get("kernel_sha") != kernel_sha() or int(rec.get("tile", -1)) != tile:
        return None
    return rec.get("dram_bytes_per_launch")


def step_bytes(n, nnz, tile):
    """Algorithmic bytes of one Chebyshev step launch over one column tile (forward form):
    col_idx 4 nnz + row_ptr 8(n+1) + D^-1/2 4n + T_{j-1}, T_j, T_{j+1} 3*4*n*w + Psi
    read+write 2*4*n*w."""
    return 4 * nnz + 8 * (n + 1) + 4 * n + 5 * 4 * n * tile


def cpu_baseline(graph, seconds_hint=True):
    """The FP64 oracle as it stands on a bounded sample: one signal column through the
    order-100 recursion on the full first snapshot, single thread."""
    import numpy as np

    import workloads as W
    from oracle import chebyshev as cb
    from oracle import laplacian as lp
    lt = lp.shifted_laplacian(graph.n, graph.row_ptr, graph.col_idx)
    r = W.gaussian_block(graph.n, 1, D_SIG, seed=5).astype(np.float64)
    t0 = time.perf_counter()
    cb.cheb_filter(lt, r, M_ORDER, 0.06)
    dt = time.perf_counter() - t0
    return {"value": graph.nnz * 1 * M_ORDER / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"oracle.chebyshev.cheb_filter, float64 scipy CSR, 1 of 64 columns, m={M_ORDER}, "
                      f"first snapshot (n={graph.n}, nnz={graph.nnz}), {dt:.1f} s"}


def batched_comparison(seed=77, count=128, m=60):
    """Batched BF16 (one persistent graph-captured launch) vs plain FP32 (one graph at a time)
    on a batch shaped like the many-graphs workload, scaled down to 128 graphs with n
    log-uniform in [1e3, 5e4], k ~ U{5..50}, degree ~ U[10, 40], d = 4k, m = 60."""
    import numpy as np
    import torch

    import paper_1706_03591_gb300 as csc
    import workloads as W
    rng = np.random.default_rng(seed)
    graphs = []
    for i in range(count):
        n = int(np.exp(rng.uniform(np.log(1e3), np.log(5e4))))
        k = int(rng.integers(5, 51))
        deg = float(rng.uniform(10, 40))
        g = (W.sbm_graph(n, k, deg, 10, seed=seed + i) if i % 2 == 0 else
             W.chung_lu_graph(n, 2.5, deg, k, 0.2, seed=seed + i))
        graphs.append(dict(n=g.n, row_ptr=torch.from_numpy(g.row_ptr).cuda(),
                           col_idx=torch.from_numpy(g.col_idx).cuda(), vals=None, c=4 * k, d=4 * k,
                           lambda_c=float(rng.uniform(0.2, 1.0)), seed=seed * 1000 + i,
                           psi=torch.zeros((g.n, 4 * k), device="cuda")))
    units = float(sum(g["col_idx"].numel() * g["c"] * m for g in graphs))
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    with csc.Context({"precision": 1}) as ctx:
        ctx.filter_batched(graphs, m)          # plan, autotune, capture
        ctx.stats(reset=True)
        torch.cuda.synchronize()
        ev[0].record(stream)
        reps = 3
        for _ in range(reps):
            ctx.filter_batched(graphs, m)
        ev[1].record(stream)
        torch.cuda.synchronize()
        st = ctx.stats()
    t_batched = ev[0].elapsed_time(ev[1]) / reps
    with csc.Context({"precision": 0}) as ctx:
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
    return {"workload": f"{count} graphs (SBM / Chung-Lu alternating), n log-uniform [1e3, 5e4], "
                        f"k U[5,50], degree U[10,40], d=4k, m={m}",
            "graphs": count, "units_per_batch": units,
            "batched_bf16": {"value": units / (t_batched / 1e3), "ms": t_batched,
                             "graph_replays": st["graph_replays"], "launches": st["batched_launches"],
                             "waves": st["batched_waves"]},
            "plain_fp32": {"value": units / (t_plain / 1e3), "ms": t_plain},
            "speedup": t_plain / t_batched, "unit": UNIT}


def differentiation_timing(seed=4, reps=3):
    """Forward (with checkpoints every ceil(sqrt m) steps), loss gradient and vector-Jacobian
    product of the k-means loss of the filtered features, at the differentiation workload's
    size: SBM n = 2e5, k = 20, degree 25, d = 128, m = 60, unit weights, float32."""
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
    with csc.Context() as ctx:
        ctx.set_graph(g.n, torch.from_numpy(g.row_ptr).cuda(), torch.from_numpy(g.col_idx).cuda())
        psi = torch.zeros((g.n, c), device="cuda")
        gpsi = torch.zeros_like(psi)
        gw = torch.zeros(g.col_idx.size, device="cuda")
        t = [0.0, 0.0, 0.0]
        for rep in range(reps + 1):
            torch.cuda.synchronize()
            ev[0].record(stream)
            ctx.filter_forward(m, a, r, psi, 0)
            ev[1].record(stream)
            ctx.kmeans_loss_grad(psi, mu, assign, gpsi)
            ev[2].record(stream)
            ctx.filter_vjp(gpsi, gw)
            ev[3].record(stream)
            torch.cuda.synchronize()
            if rep > 0:
                for i in range(3):
                    t[i] += ev[i].elapsed_time(ev[i + 1]) / reps
    units = float(g.nnz) * c * m
    return {"workload": f"SBM n={n}, k={k}, degree 25, d={c}, m={m}, unit weights, fp32, "
                        "checkpoints every 8 steps", "nnz": int(g.nnz),
            "forward_ms": t[0], "loss_grad_ms": t[1], "vjp_ms": t[2],
            "backward_over_forward": t[2] / t[0], "forward_rate": units / (t[0] / 1e3),
            "unit": UNIT}


def compressive_timing(ctx, full_assign, planted, seed=11, reps=3):
    """Compressive k-means (sampled k-means + k interpolating filterings) on the context's
    last snapshot, against the full k-means assignment of the same features and against the
    planted blocks of the generator."""
    import numpy as np
    import torch
    from scipy.optimize import linear_sum_assignment

    def agreement(a, b):
        c = np.zeros((K_CLUST, K_CLUST))
        np.add.at(c, (a, b), 1)
        ri, ci = linear_sum_assignment(-c)
        return float(c[ri, ci].sum() / a.size)

    full = full_assign.cpu().numpy()
    out = torch.zeros(N_NODES, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    res = {}
    for label, draws in (("default", 0), ("4x", int(np.ceil(8 * K_CLUST * np.log(K_CLUST))))):
        ctx.compressive_cluster(K_CLUST, n_draws=draws, seed=seed, assign_out=out)  # warm-up
        st0 = ctx.stats()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        torch.cuda.synchronize()
        ev[0].record(stream)
        for _ in range(reps):
            r = ctx.compressive_cluster(K_CLUST, n_draws=draws, seed=seed, assign_out=out)
        ev[1].record(stream)
        torch.cuda.synchronize()
        st1 = ctx.stats()
        got = out.cpu().numpy()
        res[label] = {"n_draws": draws or int(np.ceil(2 * K_CLUST * np.log(K_CLUST))),
                      "n_sampled": r["n_sampled"], "ms": ev[0].elapsed_time(ev[1]) / reps,
                      "interpolation_step_ms": (st1["step_ms"] - st0["step_ms"]) / reps,
                      "agreement_with_full_kmeans": agreement(got, full),
                      "agreement_with_planted": agreement(got, planted)}
    return {"workload": "last timed snapshot of the bench sequence: k=100 clusters, 10 restarts of the "
                        "reduced k-means, interpolation by the order-100 low pass of the features",
            "full_kmeans_agreement_with_planted": agreement(full, planted), **res}


def run_reference(a, rank, world):
    if rank != 0:
        return 0
    import numpy as np

    import workloads as W
    from oracle import chebyshev as cb
    from oracle import laplacian as lp
    m_ref = 25
    snaps = make_snapshots(a.warmup + a.steps, seed=1000)
    units, total = 0.0, 0.0
    for t, g in enumerate(snaps):
        lt = lp.shifted_laplacian(g.n, g.row_ptr, g.col_idx)
        r = W.gaussian_block(g.n, 1, D_SIG, seed=t).astype(np.float64)
        t0 = time.perf_counter()
        cb.cheb_filter(lt, r, m_ref, 0.06)
        dt = time.perf_counter() - t0
        if t >= a.warmup:
            units += g.nnz * m_ref
            total += dt
    value = units / total
    sample = (f"per step: oracle.chebyshev.cheb_filter on that snapshot, float64 scipy CSR, 1 of 64 "
              f"new columns, order {m_ref} (of {M_ORDER}); {a.steps} timed steps, single thread")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": 1e3 * total / a.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference", "config": workload_config(None),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def workload_config(tile):
    cfg = {"workload": "dynamic CSC at scale: SBM n=1e6, k=100 Zipf(0.8) blocks, degree 30, "
                       "p_in/p_out=10, 0.5% edge churn per snapshot, d=256, m=100, p=0.75, fp32",
           "n": N_NODES, "k": K_CLUST, "avg_degree": DEG, "d": D_SIG, "m": M_ORDER, "p": P_REUSE,
           "cols_filtered_per_step": D_SIG - int(P_REUSE * D_SIG), "churn": CHURN,
           "l2": "inputs larger than L2 (128 MB CSR + 1 GB feature ring per snapshot; no flush)",
           "parallelism": "replicas (independent snapshot sequences per GPU)"}
    if tile is not None:
        cfg["col_tile"] = tile
    return cfg


def run_ours(a, rank, world, local):
    import numpy as np
    import torch

    import paper_1706_03591_gb300 as csc
    import workloads as W
    dist = Dist(world)
    torch.cuda.set_device(local)
    seed = 1000 + rank
    snaps = make_snapshots(a.warmup + a.steps, seed=seed)
    dev_graphs = [(torch.from_numpy(g.row_ptr).cuda(), torch.from_numpy(g.col_idx).cuda()) for g in snaps]
    inits = [W.forgy_indices(N_NODES, K_CLUST, seed=seed + t) for t in range(len(snaps))]
    stream = torch.cuda.current_stream()

    def run_sequence(ctx, graphs, assign, timed_from):
        """Runs all snapshots; returns (device ms of the timed part, credited units, details)."""
        units = 0.0
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        marks = []
        info = []
        for t, (rp, ci) in enumerate(graphs):
            if t == timed_from:
                ctx.stats(reset=True)
                dist.barrier()
                torch.cuda.synchronize()
                clocks.start()
                e0.record(stream)
            ev_t = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            ev_t[0].record(stream)
            ctx.set_graph(N_NODES, rp, ci)
            ev_t[1].record(stream)
            lam, cnt, ev, cols = ctx.filter(M_ORDER, D_SIG, P_REUSE, seed, K_CLUST)
            ev_t[2].record(stream)
            cost, iters = ctx.cluster(K_CLUST, seed, inits[t], assign)
            ev_t[3].record(stream)
            if t >= timed_from:
                marks.append(ev_t)
                units += snaps[t].nnz * cols * M_ORDER
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

    clocks = Clocks(local)
    opts = {"timing": 1, "col_tile": a.tile}
    ctx = csc.Context(opts)
    assign = torch.zeros(N_NODES, dtype=torch.int32, device="cuda")
    ms, units, info, clk, phases = run_sequence(ctx, dev_graphs, assign, a.warmup)
    stats = ctx.stats()
    tile = int(stats["tile"])
    comp = None
    if rank == 0 and not a.no_compressive:
        comp = compressive_timing(ctx, assign, np.asarray(snaps[-1].labels))
    ctx.close()
    ms_max = dist.reduce(ms, "max")
    units_all = dist.reduce(units, "sum")
    value = units_all / (ms_max / 1e3)

    e2e = None
    if not a.no_e2e:
        host_graphs = [(torch.from_numpy(g.row_ptr).pin_memory(), torch.from_numpy(g.col_idx).pin_memory())
                       for g in snaps]
        assign_h = torch.zeros(N_NODES, dtype=torch.int32).pin_memory()
        ctx2 = csc.Context(opts)
        ms2, units2, _, _, _ = run_sequence(ctx2, host_graphs, assign_h, a.warmup)
        ctx2.close()
        ms2_max = dist.reduce(ms2, "max")
        units2_all = dist.reduce(units2, "sum")
        nnz_mean = float(np.mean([g.nnz for g in snaps[a.warmup:]]))
        e2e = {"value": units2_all / (ms2_max / 1e3), "unit": UNIT,
               "h2d_bytes_per_step": int(8 * (N_NODES + 1) + 4 * nnz_mean),
               "d2h_bytes_per_step": 4 * N_NODES}

    base = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        base = cpu_baseline(snaps[0])
    batched = None
    if rank == 0 and not a.no_batched:
        del dev_graphs
        torch.cuda.empty_cache()
        batched = batched_comparison()
    grad = None
    if rank == 0 and not a.no_grad:
        torch.cuda.empty_cache()
        grad = differentiation_timing()
    dist.close()
    if rank != 0:
        return 0
    peak, peak_kind = peak_hbm()
    avg_launch_s = stats["step_ms"] / max(1, stats["step_launches"]) / 1e3
    nnz_timed = float(np.mean([g.nnz for g in snaps[a.warmup:]]))
    bytes_launch = step_bytes(N_NODES, nnz_timed, tile)
    achieved = bytes_launch / avg_launch_s / 1e9 if avg_launch_s > 0 else None
    traffic = ncu_traffic(tile)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": ms_max / a.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload_config(tile),
        "roofline": {"kernel": "cheb_step", "bound": "hbm", "achieved": achieved, "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s",
                     "frac": achieved / peak if achieved else None, "traffic": traffic,
                     "avg_launch_us": avg_launch_s * 1e6, "launches_timed": stats["step_launches"],
                     "bytes_per_launch": bytes_launch},
        "cpu_baseline": base,
        "e2e": e2e,
        "clocks": clk,
        "gpu_launches": stats["launches"],
        "batched_vs_plain": batched,
        "differentiation": grad,
        "compressive_kmeans": comp,
        "phase_ms": phases,
        "per_step": {"lambda": [i["lam"] for i in info], "evals": [i["evals"] for i in info],
                     "kmeans_iters": [i["iters"] for i in info]},
        "kmeans": {"passes": stats["kmeans_passes"],
                   "near_ties_per_pass": stats["kmeans_near_ties"] / max(1, stats["kmeans_passes"])},
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
