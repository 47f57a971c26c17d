"""Checkpoint / resume of the dynamic state (csc_save_state, csc_load_state).

Algorithm 1 carries the feature ring, the cutoff and the previous assignment from one
snapshot to the next.  A context resumed from a saved state must continue the snapshot
sequence bit for bit as the context that saved it does.
"""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _snapshot(ctx, g, t, n, k, d, m, p, seed):
    ctx.set_graph(n, _dev(g.row_ptr), _dev(g.col_idx))
    lam, cnt, ev, cols = ctx.filter(m, d, p, seed, k)
    assign = np.zeros(n, dtype=np.int32)
    ctx.cluster(k, seed, W.forgy_indices(n, k, seed=40 + t), assign)
    theta = np.zeros((n, d), dtype=np.float32)
    ctx.get_features(theta)
    return lam, cnt, assign, theta


@pytest.mark.parametrize("precision,reorder", [(0, 1), (1, 1), (0, 0), (0, 2)])
def test_resume_continues_the_sequence_exactly(gpu_lib, tmp_path, precision, reorder):
    n, k, d, m, p, seed = 2000, 10, 64, 50, 0.5, 11
    g0 = W.sbm_graph(n, k, 20, 10, seed=1)
    graphs = [g0]
    for t in range(1, 4):
        graphs.append(W.edge_redraw(graphs[-1], 0.01, seed=100 + t))
    path = tmp_path / "state.bin"
    with gpu_lib.Context({"precision": precision, "reorder": reorder}) as a:
        for t in range(2):
            _snapshot(a, graphs[t], t, n, k, d, m, p, seed)
        a.save_state(path)
        ref = [_snapshot(a, graphs[t], t, n, k, d, m, p, seed) for t in (2, 3)]
        mu_ref = gpu_lib.csc_get_moments(a.h, 2 * m + 1)
    with gpu_lib.Context({"precision": precision, "reorder": reorder}) as b:
        b.load_state(path)
        got = [_snapshot(b, graphs[t], t, n, k, d, m, p, seed) for t in (2, 3)]
        mu_got = gpu_lib.csc_get_moments(b.h, 2 * m + 1)
    for (lam_r, cnt_r, asg_r, th_r), (lam_g, cnt_g, asg_g, th_g) in zip(ref, got):
        assert lam_g == lam_r and cnt_g == cnt_r
        np.testing.assert_array_equal(th_g, th_r)
        np.testing.assert_array_equal(asg_g, asg_r)
    np.testing.assert_array_equal(mu_got, mu_ref)


def test_state_errors(gpu_lib, tmp_path):
    n, k, d, m = 600, 4, 16, 20
    g = W.sbm_graph(n, k, 12, 10, seed=3)
    path = tmp_path / "s.bin"
    with gpu_lib.Context() as ctx:
        with pytest.raises(gpu_lib.CscError):            # nothing filtered yet
            ctx.save_state(path)
        _snapshot(ctx, g, 0, n, k, d, m, 0.5, 5)
        ctx.save_state(path)
        with pytest.raises(gpu_lib.CscError):            # cannot open
            ctx.save_state(tmp_path / "missing_dir" / "s.bin")
    bogus = tmp_path / "bogus.bin"
    bogus.write_bytes(b"not a state file at all")
    truncated = tmp_path / "truncated.bin"
    truncated.write_bytes(path.read_bytes()[:-1000])
    with gpu_lib.Context() as ctx:
        with pytest.raises(gpu_lib.CscError, match="not a state file"):
            ctx.load_state(bogus)
        with pytest.raises(gpu_lib.CscError, match="truncated"):
            ctx.load_state(truncated)
        with pytest.raises(gpu_lib.CscError, match="cannot open"):
            ctx.load_state(tmp_path / "nothing_here.bin")
        ctx.load_state(path)
        g2 = W.sbm_graph(n + 1, k, 12, 10, seed=4)
        with pytest.raises(gpu_lib.CscError):            # the ring holds n = 600 rows
            ctx.set_graph(n + 1, _dev(g2.row_ptr), _dev(g2.col_idx))
        ctx.set_graph(n, _dev(g.row_ptr), _dev(g.col_idx))
        ctx.filter(m, d, 0.5, 5, k)                      # the resumed context keeps working
    with gpu_lib.Context({"precision": 1}) as ctx:
        with pytest.raises(gpu_lib.CscError, match="precision"):
            ctx.load_state(path)
    with gpu_lib.Context({"reorder": 0}) as ctx:
        with pytest.raises(gpu_lib.CscError, match="reorder"):
            ctx.load_state(path)
