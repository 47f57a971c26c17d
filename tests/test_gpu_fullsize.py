"""Parity at the full size of the large power-law workload: Chung-Lu n = 8e6 (degree exponent
2.5, mean degree 25, k = 64 planted communities, mixing 0.2; about 2e8 stored edges),
d = 192 signals stored in bfloat16, m = 80, cutoff by the eigencount dichotomy, node order
regrouped by the first clustering, as in the bench's timed snapshots.

The oracle cannot filter all columns at this size, so it recomputes sampled columns
(columns are independent: Section 3, Eq. 3 applies h(L) to each signal separately), one in
each column tile of the bench's 39/40-column pass (tiles of 32 and 8), and the dichotomy is
checked through properties that hold at any size.
"""
import threading

import numpy as np
import pytest

import workloads as W
from conftest import fp32_filter, rel
from oracle import chebyshev as cb
from oracle import laplacian as lp
from oracle.philox import gaussian_columns

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5
BF16_TOL = 3e-3


def test_full_size_power_law_bf16_sampled_columns(gpu_lib):
    """First snapshot through csc_filter (Philox signals, dichotomy, all d columns), one
    clustering, the node order regrouped by it, then a 40-column bfloat16 block filtered in
    tiles of 32 and 8 columns.  Checks:

    - the cutoff lies in (0, 2) and its eigencount is within tau = max(0.5, 2 sqrt(2k/d)) of k
      (or the dichotomy used all its evaluations);
    - that eigencount equals (d/c) ||Psi||_F^2 rebuilt from the pass's trace moments with the
      oracle's coefficients (the estimator of Section 3.2 with c = d); mu_0 equals ||R||_F^2
      of the same bfloat16 signals summed by torch, and no |mu_l| exceeds mu_0;
    - sampled columns 5 (32-column tile) and 35 (8-column tile) against the float64 oracle
      on the same bfloat16 signals, within max(1e-5, 2 x the float32 floor of the same
      recursion), and against the float64 oracle on the unrounded float64 signals within 3e-3
      (the bfloat16 rounding of the signals, about 2^-9 relative, carried through a linear
      filter)."""
    n, k, d, m, p, seed = 8_000_000, 64, 192, 80, 0.8, 1000
    g = W.chung_lu_graph_torch(n, 2.5, 25.0, k, 0.2, seed=seed, device="cuda")
    rp, ci = g.row_ptr, g.col_idx
    c, cols = 40, np.array([5, 35])
    with gpu_lib.Context({"precision": 1, "reorder": 2}) as ctx:
        ctx.set_graph(n, rp, ci)
        lam, cnt, evals, nc = ctx.filter(m, d, p, seed, k)
        mu = ctx.get_moments(2 * m + 1)
        r0 = torch.zeros((n, d), dtype=torch.bfloat16, device="cuda")
        ctx.signals(seed, n, 0, d, d, r0)  # the first snapshot's signal block
        mu0 = sum(float(r0[:, q:q + 32].double().pow(2).sum()) for q in range(0, d, 32))
        del r0
        assign = torch.empty(n, dtype=torch.int32, device="cuda")
        ctx.cluster(k, seed, W.forgy_indices(n, k, seed=seed), assign)
        ctx.set_graph(n, rp, ci)
        r = torch.zeros((n, c), dtype=torch.bfloat16, device="cuda")
        ctx.signals(seed + 1, n, 0, c, d, r)
        psi = torch.zeros((n, c), device="cuda")
        ctx.stats(reset=True)
        ctx.cheb_filter(m, lam, r, psi)
        st = ctx.stats()
        got = psi[:, cols].cpu().numpy()
        rb = r[:, cols].float().cpu().numpy().astype(np.float64)
    assert st["tile"] == 32 and st["filter_passes"] == 2  # tiles of 32 and 8 columns

    # the dichotomy's result
    assert nc == d and 0.0 < lam < 2.0
    assert abs(cnt - k) <= cb.count_tolerance(k, d) or evals >= 30
    a = cb.filter_coefficients(m, lam)
    i, j = np.meshgrid(np.arange(m + 1), np.arange(m + 1), indexing="ij")
    via = float(np.sum(a[i] * a[j] * (mu[i + j] + mu[np.abs(i - j)]) / 2.0))
    assert abs(via - cnt) <= 1e-5 * cnt
    # mu_0 = ||R||_F^2, and |mu_l| <= mu_0 since |T_l| <= 1 on the spectrum of L~ in [-1, 1]
    assert abs(mu[0] - mu0) <= 1e-6 * mu0
    assert np.all(np.abs(mu) <= mu0 * (1 + 1e-6))

    # sampled columns against the float64 oracle
    sig = gaussian_columns(seed + 1, n, cols, d)
    lt = lp.shifted_laplacian(n, rp.cpu().numpy(), ci.cpu().numpy())
    del g, rp, ci
    # one column per thread (scipy's sparse products release the GIL)
    blocks = [rb[:, :1], rb[:, 1:], sig[:, :1], sig[:, 1:]]
    out = [None] * 6

    def oracle64(q):
        out[q] = cb.cheb_filter(lt, blocks[q], m, lam)[:, 0]

    def float32_floor(q):
        out[4 + q] = fp32_filter(lt, blocks[q], a)[:, 0]

    th = [threading.Thread(target=oracle64, args=(q,)) for q in range(4)]
    th += [threading.Thread(target=float32_floor, args=(q,)) for q in range(2)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    ref_b, ref_s, f32 = np.stack(out[0:2], 1), np.stack(out[2:4], 1), np.stack(out[4:6], 1)
    for q in range(2):
        floor = rel(f32[:, q], ref_b[:, q])
        err_b = rel(got[:, q], ref_b[:, q])
        err_s = rel(got[:, q], ref_s[:, q])
        print(f"column {cols[q]}: error {err_b:.3e} (float32 floor {floor:.3e}), "
              f"against float64 signals {err_s:.3e}")
        assert err_b < max(FP32_TOL, 2.0 * floor)
        assert err_s < BF16_TOL
