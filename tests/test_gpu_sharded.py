"""The column-sharded driver with the library backend on the GPU: two ranks (processes) on one
GPU, host collectives over gloo.  Their kernels never wait on each other; only the host
collectives between the filtering passes cross ranks.  Every rank must end each snapshot with the
cutoff, dichotomy count, features and assignment of one process running csc_filter and
csc_cluster on all columns (Algorithm 1, Eq. 6).  A rank filters fewer columns in narrower tiles,
and a row's gather is split over a number of slots that depends on the tile width, so the
features agree to float32 rounding rather than bit for bit."""
import os
import socket

import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
mp = torch.multiprocessing
pytestmark = pytest.mark.gpu

N, K, D, M, SEED = 2000, 10, 64, 50, 17


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _graphs(count=4):
    g = W.sbm_graph(N, K, 20, 10, seed=2)
    out = [g]
    for t in range(1, count):
        out.append(W.sbm_perturb(out[-1], 0.01, 0.03, seed=300 + t))
    return out


def _inits(count=4):
    return [W.forgy_indices(N, K, seed=900 + t) for t in range(count)]


def _worker(rank, world, port, precision, p, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1706_03591_gb300.sharded import LibraryColumns, ShardedDynamicCSC
    be = LibraryColumns({"precision": precision})
    drv = ShardedDynamicCSC(be, N, K, D, p, M, SEED)
    res = []
    for g, idx in zip(_graphs(), _inits()):
        assign = torch.zeros(N, dtype=torch.int32, device="cuda")
        rec = drv.step(torch.from_numpy(g.row_ptr).cuda(), torch.from_numpy(g.col_idx).cuda(), idx, assign)
        theta = torch.zeros((N, D), device="cuda")
        be.ctx.get_features(theta)
        res.append((rec["lam"], rec["evals"], assign.cpu().numpy(), theta.cpu().numpy()))
    be.close()
    out[rank] = res
    dist.destroy_process_group()


@pytest.mark.parametrize("precision,p", [(0, 0.5), (1, 0.75)])
def test_two_ranks_equal_single_context(gpu_lib, precision, p):
    ref = []
    with gpu_lib.Context({"precision": precision}) as ctx:
        for g, idx in zip(_graphs(), _inits()):
            ctx.set_graph(N, torch.from_numpy(g.row_ptr).cuda(), torch.from_numpy(g.col_idx).cuda())
            lam, cnt, ev, cols = ctx.filter(M, D, p, SEED, K)
            assign = torch.zeros(N, dtype=torch.int32, device="cuda")
            ctx.cluster(K, SEED, idx, assign)
            theta = torch.zeros((N, D), device="cuda")
            ctx.get_features(theta)
            ref.append((lam, ev, assign.cpu().numpy(), theta.cpu().numpy()))
    ctx_mp = mp.get_context("spawn")
    with ctx_mp.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx_mp.Process(target=_worker, args=(r, 2, port, precision, p, out)) for r in range(2)]
        for pr in procs:
            pr.start()
        for pr in procs:
            pr.join(timeout=300)
            assert pr.exitcode == 0
        res = {r: out[r] for r in range(2)}
    for r in range(2):
        for t, ((lam, ev, assign, theta), (lam_r, ev_r, assign_r, theta_r)) in enumerate(zip(res[r], ref)):
            assert lam == lam_r and ev == ev_r, (r, t)
            err = np.linalg.norm(theta - theta_r) / np.linalg.norm(theta_r)
            assert err < 1e-6, (r, t, err)
            np.testing.assert_array_equal(assign, assign_r)
