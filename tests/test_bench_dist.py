"""bench.py's N>1 path on CPU: two gloo ranks, barrier, max of times and sum of units.

The GPU path runs independent replicas (no data-path collective); only the timing
aggregation crosses ranks, and that is what is checked here.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
mp = torch.multiprocessing


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    r, w, local = bench.dist_env()
    d = bench.Dist(w)
    d.barrier()
    t_max = d.reduce(10.0 + r, "max")
    u_sum = d.reduce(100.0 * (r + 1), "sum")
    d.close()
    out.put((r, w, local, t_max, u_sum))


def test_two_rank_aggregation():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[0] for r in res] == [0, 1]
    for r in res:
        assert r[1] == 2 and r[3] == 11.0 and r[4] == 300.0


def test_single_rank_defaults(monkeypatch):
    for key in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(key, raising=False)
    import bench
    assert bench.dist_env() == (0, 1, 0)
    d = bench.Dist(1)
    assert d.reduce(3.5, "max") == 3.5
