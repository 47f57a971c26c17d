"""Algorithm 1 with the new signal columns of every snapshot split over the ranks of a process
group (one GPU per rank).

The filter of Sections 2.2 and 3.3 treats every signal column on its own: column g of R is the
Philox stream of global column id g, and Psi~ = h(L) R is computed column by column.  The only
quantities that mix columns are the trace moments mu_l = tr(R^T T_l(L~) R) behind the eigencount
(Section 3.3, Algorithm 1), which are sums over columns, and the k-means of Eq. 1, which needs
whole rows of Theta_t.  The split is therefore:

    quantity                                  owner                         exchange
    new columns of a snapshot, global ids     rank r: contiguous range      none (signals keyed
      next_id + [c0_r, c1_r)                    of column_ranges(c, G)        by global id)
    moments mu_0 .. mu_2m of a pass           partial sums on every rank    all-reduce (sum, fp64)
    cutoff decision (check, dichotomy)        rank 0, from the sums         broadcast (lambda,
                                                                            count, evaluations)
    filtered new columns Psi_t                rank r: n x (c1_r - c0_r)     all-gather, once per
                                                                            snapshot
    feature ring Theta_t, Y_t (Eq. 6)         replicated                    none
    k-means (Eq. 1)                           replicated (deterministic)    none

Every rank filters only its columns (the O(|E| d m) part), and the ring, the row normalisation and
the k-means repeat identically on every rank, so each rank ends the snapshot with the assignment.
Moment sums are all-reduced in float64; the cutoff values depend only on the sequence of
accept / bracket decisions of the dichotomy, and rank 0 makes them and broadcasts the result, so
every rank uses one cutoff by construction.

The compute of a rank goes through a backend object (`LibraryColumns` on a GPU: the library's
signal, filter, splice and k-means calls); collectives go through torch.distributed on the
group's device (NCCL for CUDA tensors, gloo for host tensors).  No device memory of another GPU is
read directly.
"""
from __future__ import annotations

import math

import numpy as np

from . import Context, csc_count_tolerance, csc_lambda_search_moments


def column_ranges(c: int, world: int) -> list[tuple[int, int]]:
    """Contiguous, balanced split of c columns over `world` ranks: rank r gets
    [r q + min(r, s), (r + 1) q + min(r + 1, s)) with q, s = divmod(c, world)."""
    q, s = divmod(c, world)
    return [(r * q + min(r, s), (r + 1) * q + min(r + 1, s)) for r in range(world)]


def new_column_count(t: int, d: int, p: float) -> int:
    """Columns filtered at snapshot t (0-based): d at the first snapshot or when p == 0, else
    d - floor(p d) (Eq. 6 with dp = floor(p d))."""
    return d if t == 0 or p <= 0.0 else d - int(math.floor(p * d))


class LibraryColumns:
    """Backend of one rank on its GPU: the library's calls on a context of its own."""

    def __init__(self, opts: dict | None = None):
        import torch
        self.torch = torch
        self.ctx = Context(opts)
        self.precision = (opts or {}).get("precision", 0)
        self.device = torch.device("cuda", torch.cuda.current_device())

    def set_graph(self, n, row_ptr, col_idx, vals=None):
        self.n = n
        self.ctx.set_graph(n, row_ptr, col_idx, vals)

    def filter(self, m, lam, seed, col0, c, d, want_psi):
        """(Psi of columns col0 .. col0 + c - 1 or None, their 2m + 1 moments)."""
        torch = self.torch
        if c == 0:
            psi = torch.zeros((self.n, 0), device=self.device) if want_psi else None
            return psi, np.zeros(2 * m + 1)
        dt = torch.bfloat16 if self.precision == 1 else torch.float32
        r = torch.empty((self.n, c), device=self.device, dtype=dt)
        self.ctx.signals(seed, self.n, col0, c, d, r)
        psi = torch.empty((self.n, c), device=self.device) if want_psi else None
        mu = self.ctx.cheb_filter(m, lam, r, psi, want_moments=True)
        return psi, mu

    def splice(self, n, d, p, psi_all, lam):
        self.ctx.splice(n, d, p, psi_all, lam)

    def cluster(self, k, seed, init_idx, assign_out):
        return self.ctx.cluster(k, seed, init_idx, assign_out)

    def close(self):
        self.ctx.close()


class ShardedDynamicCSC:
    """One rank's share of Algorithm 1 over a torch.distributed group.

    `step` takes the snapshot's graph (every rank holds it), filters this rank's columns,
    exchanges moments and features, and returns the assignment on every rank.  The eigencount
    is the ||Psi||^2 estimator with tolerance max(0.5, 2 sqrt(2k/c)) (or `tau`), and the
    dichotomy is the library's (csc_lambda_search_moments): the same rules as csc_filter."""

    def __init__(self, backend, n: int, k: int, d: int, p: float, m: int, seed: int,
                 group=None, tau: float | None = None, max_bisect: int = 30, device=None):
        """device: where the collectives run (a CUDA device for NCCL groups; the host, the
        default, for gloo groups)."""
        import torch
        import torch.distributed as dist
        self.torch, self.dist = torch, dist
        self.backend, self.group = backend, group
        self.n, self.k, self.d, self.p, self.m, self.seed = n, k, d, p, m, seed
        self.tau_fixed, self.max_bisect = tau, max_bisect
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)
        self.device = device if device is not None else torch.device("cpu")
        self.t = 0
        self.next_id = 0
        self.lam = None
        self.history: list[dict] = []

    # -- collectives -------------------------------------------------------------------------
    def _allreduce(self, mu: np.ndarray) -> np.ndarray:
        t = self.torch.as_tensor(np.ascontiguousarray(mu, dtype=np.float64), device=self.device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM, group=self.group)
        return t.cpu().numpy()

    def _broadcast(self, vals: list[float]) -> list[float]:
        t = self.torch.tensor(vals, dtype=self.torch.float64, device=self.device)
        self.dist.broadcast(t, src=self.dist.get_global_rank(self.group, 0) if self.group is not None else 0,
                            group=self.group)
        return [float(v) for v in t.cpu()]

    def _allgather_columns(self, psi, ranges):
        """n x c in global column order from every rank's n x (c1_r - c0_r) block."""
        torch = self.torch
        width = max(b - a for a, b in ranges)
        mine = torch.zeros((self.n, width), dtype=psi.dtype, device=self.device)
        mine[:, : psi.shape[1]] = psi.to(self.device)
        parts = [torch.empty_like(mine) for _ in range(self.world)]
        self.dist.all_gather(parts, mine, group=self.group)
        out = torch.cat([parts[r][:, : b - a] for r, (a, b) in enumerate(ranges)], dim=1)
        return out.to(psi.device).contiguous()

    # -- Algorithm 1 -------------------------------------------------------------------------
    def _decide(self, mu, c, lam_prev):
        """Rank 0's eigencount check and dichotomy on the summed moments, broadcast."""
        tau = self.tau_fixed if self.tau_fixed is not None else csc_count_tolerance(self.k, c)
        if self.rank == 0:
            lam, cnt, ev = csc_lambda_search_moments(self.m, mu, self.d, c, self.k, tau,
                                                     -1.0 if lam_prev is None else lam_prev,
                                                     self.max_bisect)
        else:
            lam, cnt, ev = 0.0, 0.0, 0
        lam, cnt, ev = self._broadcast([lam, cnt, float(ev)])
        return lam, cnt, int(ev)

    def step(self, row_ptr, col_idx, init_idx, assign_out, vals=None) -> dict:
        be, m, d = self.backend, self.m, self.d
        be.set_graph(self.n, row_ptr, col_idx, vals)
        c = new_column_count(self.t, d, self.p)
        ranges = column_ranges(c, self.world)
        a, b = ranges[self.rank]
        col0 = self.next_id + a
        if self.lam is None:
            # first cutoff: one moment pass (moments do not depend on the cutoff), dichotomy on [0, 2]
            _, mu_r = be.filter(m, 1.0, self.seed, col0, b - a, d, want_psi=False)
            mu = self._allreduce(mu_r)
            lam, cnt, evals = self._decide(mu, c, None)
            psi, _ = be.filter(m, lam, self.seed, col0, b - a, d, want_psi=True)
        else:
            lam = self.lam
            psi, mu_r = be.filter(m, lam, self.seed, col0, b - a, d, want_psi=True)
            mu = self._allreduce(mu_r)
            lam2, cnt, evals = self._decide(mu, c, lam)
            if lam2 != lam:
                psi, _ = be.filter(m, lam2, self.seed, col0, b - a, d, want_psi=True)
                lam = lam2
        psi_all = self._allgather_columns(psi, ranges)
        be.splice(self.n, d, self.p, psi_all, lam)
        cost, iters = be.cluster(self.k, self.seed, init_idx, assign_out)
        self.t += 1
        self.next_id += c
        self.lam = lam
        rec = dict(t=self.t, lam=lam, count=cnt, evals=evals, c=c, columns=(a, b), passes=iters, cost=cost)
        self.history.append(rec)
        return rec


__all__ = ["column_ranges", "new_column_count", "LibraryColumns", "ShardedDynamicCSC"]

