"""Seeded synthetic inputs for tests and benchmarks.

This module is shared by the FP64 oracle tests, the GPU parity tests and
``bench.py``.  It holds no arithmetic of the clustering method itself (no
Laplacian, no filter, no k-means): only random graphs, their edge churn,
Gaussian signal blocks handed to both sides as inputs, point clouds for
k-means tests and Forgy index draws.

Graph models follow the paper's experimental section (Section 5): stochastic
block models described by an average degree and an intra/inter probability
ratio, and "edge redrawing" churn that removes uniformly random edges and
redraws the same number from the model's probabilities.  Chung-Lu graphs with
a power-law expected degree sequence and planted communities stand in for the
large power-law workload.

Every generator is O(nnz): per-block-pair binomial edge counts with uniform
endpoint draws (SBM) or weight-proportional endpoint draws (Chung-Lu); no
O(n^2) loop.  Node ids are a random permutation of the planted structure.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Graph",
    "zipf_block_sizes",
    "sbm_graph",
    "chung_lu_graph",
    "edge_redraw",
    "gaussian_block",
    "clustered_points",
    "forgy_indices",
    "random_csr",
    "node_reassign",
    "sbm_perturb",
    "TorchGraph",
    "chung_lu_graph_torch",
    "edge_redraw_torch",
    "sbm_graph_torch",
]


@dataclass
class Graph:
    """Simple undirected graph stored as sorted symmetric edge keys.

    ``keys`` holds u*n+v for every stored (directed) entry, both directions,
    sorted ascending, no self-loops, no duplicates.  ``row_ptr``/``col_idx``
    are the matching CSR arrays (int64 / int32).  ``model`` keeps what the
    churn generator needs to redraw edges from the same model.
    """

    n: int
    keys: np.ndarray
    labels: np.ndarray | None = None
    model: dict = field(default_factory=dict)
    _csr: tuple | None = None

    @property
    def nnz(self) -> int:
        return int(self.keys.size)

    def csr(self) -> tuple[np.ndarray, np.ndarray]:
        if self._csr is None:
            rows = self.keys // self.n
            col_idx = (self.keys - rows * self.n).astype(np.int32)
            counts = np.bincount(rows, minlength=self.n).astype(np.int64)
            row_ptr = np.zeros(self.n + 1, dtype=np.int64)
            np.cumsum(counts, out=row_ptr[1:])
            self._csr = (row_ptr, col_idx)
        return self._csr

    @property
    def row_ptr(self) -> np.ndarray:
        return self.csr()[0]

    @property
    def col_idx(self) -> np.ndarray:
        return self.csr()[1]

    def upper_keys(self) -> np.ndarray:
        """Keys u*n+v with u < v (one per undirected edge), sorted."""
        rows = self.keys // self.n
        cols = self.keys - rows * self.n
        return self.keys[rows < cols]


def _symmetric_keys(n: int, upper: np.ndarray) -> np.ndarray:
    u = upper // n
    v = upper - u * n
    both = np.concatenate([upper, v * n + u])
    both.sort()
    return both


def _sorted_unique(x: np.ndarray) -> np.ndarray:
    x = np.sort(x)
    if x.size == 0:
        return x
    keep = np.empty(x.size, dtype=bool)
    keep[0] = True
    np.not_equal(x[1:], x[:-1], out=keep[1:])
    return x[keep]


def _in_sorted(x: np.ndarray, sorted_ref: np.ndarray) -> np.ndarray:
    """Membership of each x in a sorted unique array."""
    if sorted_ref.size == 0:
        return np.zeros(x.size, dtype=bool)
    pos = np.searchsorted(sorted_ref, x)
    pos = np.minimum(pos, sorted_ref.size - 1)
    return sorted_ref[pos] == x


def _canonical_upper(n: int, u: np.ndarray, v: np.ndarray) -> np.ndarray:
    """Unique u<v keys from endpoint arrays, self-loops dropped."""
    keep = u != v
    u = u[keep].astype(np.int64)
    v = v[keep].astype(np.int64)
    lo = np.minimum(u, v)
    hi = np.maximum(u, v)
    return _sorted_unique(lo * n + hi)


def zipf_block_sizes(n: int, k: int, exponent: float) -> np.ndarray:
    """Block sizes proportional to b^-exponent, b = 1..k, summing to n."""
    w = np.arange(1, k + 1, dtype=np.float64) ** (-exponent)
    sizes = np.floor(w / w.sum() * n).astype(np.int64)
    sizes = np.maximum(sizes, 1)
    # hand the rounding remainder to the largest blocks, one node each
    rem = n - int(sizes.sum())
    i = 0
    while rem != 0:
        step = 1 if rem > 0 else -1
        if sizes[i % k] + step >= 1:
            sizes[i % k] += step
            rem -= step
        i += 1
    return sizes


def _sbm_probs(sizes: np.ndarray, avg_degree: float, ratio: float) -> tuple[float, float]:
    """(p_in, p_out) with p_in = ratio*p_out and node-average expected degree avg_degree."""
    n = float(sizes.sum())
    s = sizes.astype(np.float64)
    denom = float(np.sum(s * (ratio * (s - 1.0) + (n - s))))
    p_out = avg_degree * n / denom
    return ratio * p_out, p_out


def _sbm_pair_table(sizes: np.ndarray, p_in: float, p_out: float):
    k = sizes.size
    a_idx, b_idx = np.triu_indices(k)
    sa = sizes[a_idx].astype(np.float64)
    sb = sizes[b_idx].astype(np.float64)
    same = a_idx == b_idx
    pairs = np.where(same, sa * (sa - 1.0) / 2.0, sa * sb)
    prob = np.where(same, p_in, p_out)
    return a_idx, b_idx, pairs, prob


def _sbm_draw_edges(rng, counts, a_idx, b_idx, offsets, sizes, members):
    a = np.repeat(a_idx, counts)
    b = np.repeat(b_idx, counts)
    ua = offsets[a] + np.floor(rng.random(a.size) * sizes[a]).astype(np.int64)
    vb = offsets[b] + np.floor(rng.random(b.size) * sizes[b]).astype(np.int64)
    return members[ua], members[vb]


def sbm_graph(n: int, sizes, avg_degree: float, ratio: float, seed: int) -> Graph:
    """Stochastic block model (Section 5): intra-block probability ratio times the inter-block one.

    ``sizes`` is an int array of block sizes or an int k for k equal blocks.
    Edges per block pair ~ Binomial(#pairs, p); endpoints uniform within the
    blocks; duplicates merged.  Node ids are randomly permuted.
    """
    rng = np.random.default_rng(seed)
    if np.isscalar(sizes):
        k = int(sizes)
        sizes = np.full(k, n // k, dtype=np.int64)
        sizes[: n - int(sizes.sum())] += 1
    sizes = np.asarray(sizes, dtype=np.int64)
    assert int(sizes.sum()) == n
    p_in, p_out = _sbm_probs(sizes, avg_degree, ratio)
    perm = rng.permutation(n).astype(np.int64)  # members[offsets[b] + i] = node id
    offsets = np.zeros(sizes.size, dtype=np.int64)
    np.cumsum(sizes[:-1], out=offsets[1:])
    labels = np.empty(n, dtype=np.int32)
    labels[perm] = np.repeat(np.arange(sizes.size, dtype=np.int32), sizes)
    a_idx, b_idx, pairs, prob = _sbm_pair_table(sizes, p_in, p_out)
    counts = rng.binomial(pairs.astype(np.int64), prob)
    u, v = _sbm_draw_edges(rng, counts, a_idx, b_idx, offsets, sizes, perm)
    upper = _canonical_upper(n, u, v)
    model = dict(kind="sbm", sizes=sizes, offsets=offsets, members=perm,
                 a_idx=a_idx, b_idx=b_idx, weight=pairs * prob, p_in=p_in, p_out=p_out)
    return Graph(n=n, keys=_symmetric_keys(n, upper), labels=labels, model=model)


def chung_lu_graph(n: int, exponent: float, avg_degree: float, k: int, mixing: float,
                   seed: int) -> Graph:
    """Chung-Lu graph with power-law expected degrees and k planted communities.

    Expected degrees w_i ~ i^(-1/(exponent-1)), rescaled to mean avg_degree and
    capped at sqrt(sum w).  Each of sum(w)/2 edges picks u ~ w; with
    probability 1-mixing v ~ w restricted to u's community, else v ~ w over all
    nodes.  Self-loops and duplicates are dropped; isolated nodes are kept.
    """
    rng = np.random.default_rng(seed)
    w = (np.arange(1, n + 1, dtype=np.float64)) ** (-1.0 / (exponent - 1.0))
    w *= avg_degree / w.mean()
    cap = np.sqrt(w.sum())
    w = np.minimum(w, cap)
    w *= avg_degree / w.mean()
    perm = rng.permutation(n).astype(np.int64)
    weight = np.empty(n)
    weight[perm] = w
    labels = rng.integers(0, k, size=n).astype(np.int32)
    model = _chung_lu_model(n, weight, labels, mixing)
    m_edges = int(round(weight.sum() / 2.0))
    u, v = _chung_lu_draw(rng, model, m_edges)
    upper = _canonical_upper(n, u, v)
    return Graph(n=n, keys=_symmetric_keys(n, upper), labels=labels, model=model)


def _chung_lu_model(n, weight, labels, mixing):
    order = np.argsort(labels, kind="stable")
    cw = np.cumsum(weight[order])
    k = int(labels.max()) + 1
    counts = np.bincount(labels, minlength=k)
    starts = np.zeros(k, dtype=np.int64)
    np.cumsum(counts[:-1], out=starts[1:])
    ends = starts + counts
    lo_w = np.where(starts > 0, cw[np.maximum(starts - 1, 0)], 0.0)
    hi_w = cw[np.maximum(ends - 1, 0)]
    return dict(kind="chung_lu", order=order, cw=cw, labels=labels, lo_w=lo_w,
                hi_w=hi_w, mixing=mixing, total=float(cw[-1]))


def _chung_lu_draw(rng, model, m_edges):
    order, cw, labels = model["order"], model["cw"], model["labels"]
    total = model["total"]
    u = order[np.minimum(np.searchsorted(cw, rng.random(m_edges) * total, side="right"),
                         cw.size - 1)]
    intra = rng.random(m_edges) >= model["mixing"]
    r = rng.random(m_edges)
    cu = labels[u]
    lo = np.where(intra, model["lo_w"][cu], 0.0)
    hi = np.where(intra, model["hi_w"][cu], total)
    v = order[np.minimum(np.searchsorted(cw, lo + r * (hi - lo), side="right"), cw.size - 1)]
    return u, v


def edge_redraw(g: Graph, frac: float, seed: int) -> Graph:
    """Edge redrawing churn (Section 5.1): remove round(frac*|E|) uniformly random
    edges, then add the same number drawn from the graph's own model
    probabilities (new edges only: no duplicates, no self-loops)."""
    rng = np.random.default_rng(seed)
    n = g.n
    upper = g.upper_keys()
    n_change = int(round(frac * upper.size))
    if n_change == 0:
        return Graph(n=n, keys=g.keys.copy(), labels=g.labels, model=g.model)
    drop = rng.choice(upper.size, size=n_change, replace=False)
    keep = np.ones(upper.size, dtype=bool)
    keep[drop] = False
    kept = upper[keep]
    added = np.empty(0, dtype=np.int64)
    while added.size < n_change:
        want = (n_change - added.size) * 2 + 16
        if g.model.get("kind") == "sbm":
            md = g.model
            pw = md["weight"] / md["weight"].sum()
            counts = rng.multinomial(want, pw)
            u, v = _sbm_draw_edges(rng, counts, md["a_idx"], md["b_idx"], md["offsets"],
                                   md["sizes"], md["members"])
        elif g.model.get("kind") == "chung_lu":
            u, v = _chung_lu_draw(rng, g.model, want)
        else:
            u = rng.integers(0, n, want)
            v = rng.integers(0, n, want)
        cand = _canonical_upper(n, u, v)
        # drop candidates already present (in the original graph or already added)
        present = _in_sorted(cand, upper) | _in_sorted(cand, np.sort(added))
        cand = cand[~present]
        cand = cand[rng.permutation(cand.size)]
        added = np.concatenate([added, cand[: n_change - added.size]])
    new_upper = _sorted_unique(np.concatenate([kept, added]))
    return Graph(n=n, keys=_symmetric_keys(n, new_upper), labels=g.labels, model=g.model)


def node_reassign(g: Graph, frac: float, seed: int) -> Graph:
    """Node reassignment churn of an SBM (Section 5.1): pick round(frac n) nodes uniformly, remove
    every edge with an end among them, move each to one of the other k - 1 blocks uniformly at
    random, and reconnect them by the model's probabilities (p_in inside the new block, p_out
    across): edges to the unpicked nodes are drawn per (picked node, block) as binomial counts
    with uniform endpoints, edges among the picked nodes as an SBM on the picked set.  The
    returned graph carries the new labels and the model of the new block sizes, so later churn
    draws from the perturbed model."""
    md = g.model
    if md.get("kind") != "sbm":
        raise ValueError("node_reassign: graph model must be sbm")
    rng = np.random.default_rng(seed)
    n = g.n
    k = int(md["sizes"].size)
    p_in, p_out = md["p_in"], md["p_out"]
    r = int(round(frac * n))
    picked = np.sort(rng.choice(n, size=r, replace=False)).astype(np.int64)
    is_picked = np.zeros(n, dtype=bool)
    is_picked[picked] = True
    labels = g.labels.astype(np.int64).copy()
    labels[picked] = (labels[picked] + rng.integers(1, k, size=r)) % k
    upper = g.upper_keys()
    kept = upper[~(is_picked[upper // n] | is_picked[upper % n])]
    # picked -> unpicked: per (picked node, block) binomial counts, uniform endpoints
    rest = np.flatnonzero(~is_picked)
    rest = rest[np.argsort(labels[rest], kind="stable")]
    rest_sizes = np.bincount(labels[rest], minlength=k)
    rest_off = np.concatenate([[0], np.cumsum(rest_sizes)[:-1]])
    prob = np.where(labels[picked][:, None] == np.arange(k)[None, :], p_in, p_out)
    cnt = rng.binomial(np.broadcast_to(rest_sizes, (r, k)), prob)
    src = np.repeat(np.repeat(picked, k), cnt.ravel())
    blk = np.repeat(np.tile(np.arange(k), r), cnt.ravel())
    dst = rest[rest_off[blk] + np.floor(rng.random(blk.size) * rest_sizes[blk]).astype(np.int64)]
    # picked <-> picked: the SBM restricted to the picked set
    pk = picked[np.argsort(labels[picked], kind="stable")]
    pk_sizes = np.bincount(labels[picked], minlength=k)
    pk_off = np.concatenate([[0], np.cumsum(pk_sizes)[:-1]])
    a_idx, b_idx, pairs, pprob = _sbm_pair_table(pk_sizes, p_in, p_out)
    pcnt = rng.binomial(pairs.astype(np.int64), pprob)
    pu, pv = _sbm_draw_edges(rng, pcnt, a_idx, b_idx, pk_off, np.maximum(pk_sizes, 1), pk)
    new = _canonical_upper(n, np.concatenate([src, pu]), np.concatenate([dst, pv]))
    sizes = np.bincount(labels, minlength=k).astype(np.int64)
    members = np.argsort(labels, kind="stable").astype(np.int64)
    offsets = np.zeros(k, dtype=np.int64)
    np.cumsum(sizes[:-1], out=offsets[1:])
    a_all, b_all, pairs_all, prob_all = _sbm_pair_table(sizes, p_in, p_out)
    model = dict(kind="sbm", sizes=sizes, offsets=offsets, members=members, a_idx=a_all,
                 b_idx=b_all, weight=pairs_all * prob_all, p_in=p_in, p_out=p_out)
    out = Graph(n=n, keys=_symmetric_keys(n, _sorted_unique(np.concatenate([kept, new]))),
                labels=labels.astype(np.int32), model=model)
    out.model["reassigned"] = picked
    return out


def sbm_perturb(g: Graph, node_frac: float, edge_frac: float, seed: int) -> Graph:
    """The combined perturbation of Section 5.2: node reassignment of node_frac of the nodes,
    then edge redrawing of edge_frac of the edges."""
    h = node_reassign(g, node_frac, seed)
    return edge_redraw(h, edge_frac, seed + 1)


def random_csr(n: int, avg_degree: float, seed: int, isolated: int = 0) -> Graph:
    """Erdos-Renyi-like graph (uniform endpoints), optionally with `isolated`
    nodes that receive no edges (for edge-case tests)."""
    rng = np.random.default_rng(seed)
    m_edges = int(round(n * avg_degree / 2.0))
    active = np.arange(isolated, n, dtype=np.int64)
    u = active[rng.integers(0, active.size, m_edges)]
    v = active[rng.integers(0, active.size, m_edges)]
    perm = rng.permutation(n).astype(np.int64)
    upper = _canonical_upper(n, perm[u], perm[v])
    return Graph(n=n, keys=_symmetric_keys(n, upper), model=dict(kind="er"))


def gaussian_block(n: int, c: int, d: int, seed: int, dtype=np.float32) -> np.ndarray:
    """n x c block of i.i.d. N(0, 1/d) entries (the paper's R, Section 2.2), row-major."""
    rng = np.random.default_rng(seed)
    r = rng.standard_normal((n, c)) / np.sqrt(d)
    return r.astype(dtype)


def clustered_points(n: int, d: int, k: int, seed: int, spread: float = 0.35,
                     normalize: bool = True) -> tuple[np.ndarray, np.ndarray]:
    """n points in R^d around k random centres (FP32), optionally unit-normalised rows."""
    rng = np.random.default_rng(seed)
    centres = rng.standard_normal((k, d))
    centres /= np.linalg.norm(centres, axis=1, keepdims=True)
    lab = rng.integers(0, k, n)
    x = centres[lab] + spread * rng.standard_normal((n, d)) / np.sqrt(d)
    if normalize:
        x /= np.maximum(np.linalg.norm(x, axis=1, keepdims=True), 1e-300)
    return x.astype(np.float32), lab.astype(np.int32)


def forgy_indices(n: int, k: int, seed: int) -> np.ndarray:
    """k distinct row indices drawn uniformly (Forgy initialisation input)."""
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(n, size=k, replace=False)).astype(np.int64)


# ------------------------------------------------------------------ large graphs on a torch device
#
# The power-law workload has n = 8e6 nodes and about 2e8 stored edges; the numpy generators
# above would spend minutes sorting 2e8 keys per snapshot.  The functions below draw the same
# models (Chung-Lu with planted communities, edge redrawing) with torch on any device (the GPU
# for full sizes, the CPU in tests), seeded by a torch.Generator, so the graph of a seed is
# fixed for a device type and torch's generator.  They hold no arithmetic of the method.

@dataclass
class TorchGraph:
    """Simple undirected graph on a torch device: sorted symmetric keys u*n+v (int64, both
    directions, no self-loops or duplicates), the matching CSR (row_ptr int64[n+1], col_idx
    int32[nnz]), planted labels and the model that edge redrawing samples from."""

    n: int
    keys: object
    row_ptr: object
    col_idx: object
    labels: object
    model: dict

    @property
    def nnz(self) -> int:
        return int(self.keys.numel())

    def to_numpy(self) -> Graph:
        """The same graph as a numpy Graph (for the oracle and small checks)."""
        g = Graph(n=self.n, keys=self.keys.cpu().numpy(),
                  labels=self.labels.cpu().numpy() if self.labels is not None else None)
        g._csr = (self.row_ptr.cpu().numpy(), self.col_idx.cpu().numpy())
        return g


def _t_upper_from_endpoints(torch, n, u, v):
    keep = u != v
    u, v = u[keep], v[keep]
    lo = torch.minimum(u, v)
    hi = torch.maximum(u, v)
    return torch.unique(lo * n + hi, sorted=True)


def _t_graph_from_upper(torch, n, upper, labels, model):
    u = upper // n
    v = upper - u * n
    keys = torch.cat([upper, v * n + u]).sort().values
    rows = keys // n
    col_idx = (keys - rows * n).to(torch.int32)
    counts = torch.bincount(rows, minlength=n)
    row_ptr = torch.zeros(n + 1, dtype=torch.int64, device=keys.device)
    torch.cumsum(counts, 0, out=row_ptr[1:])
    return TorchGraph(n=n, keys=keys, row_ptr=row_ptr, col_idx=col_idx, labels=labels, model=model)


def _t_chung_lu_draw(torch, gen, model, count):
    order, cw, labels = model["order"], model["cw"], model["labels"]
    total = model["total"]
    dev = cw.device
    top = cw.numel() - 1

    def pick(x):
        return order[torch.clamp(torch.searchsorted(cw, x, right=True), max=top)]

    u = pick(torch.rand(count, generator=gen, device=dev, dtype=torch.float64) * total)
    intra = torch.rand(count, generator=gen, device=dev, dtype=torch.float64) >= model["mixing"]
    r = torch.rand(count, generator=gen, device=dev, dtype=torch.float64)
    cu = labels[u].long()
    lo = torch.where(intra, model["lo_w"][cu], torch.zeros_like(r))
    hi = torch.where(intra, model["hi_w"][cu], torch.full_like(r, total))
    v = pick(lo + r * (hi - lo))
    return u, v


def _t_sbm_draw(torch, gen, model, count):
    """count endpoint pairs from the SBM: block pair ~ its expected edge share, endpoints
    uniform within the two blocks."""
    share = model["weight"]
    pair = torch.multinomial(share, count, replacement=True, generator=gen)
    a, b = model["a_idx"][pair], model["b_idx"][pair]
    sz, off, members = model["sizes_t"], model["offsets"], model["members"]
    dev = share.device
    ua = off[a] + torch.floor(torch.rand(count, generator=gen, device=dev, dtype=torch.float64)
                              * sz[a]).to(torch.int64)
    vb = off[b] + torch.floor(torch.rand(count, generator=gen, device=dev, dtype=torch.float64)
                              * sz[b]).to(torch.int64)
    return members[ua], members[vb]


def chung_lu_graph_torch(n: int, exponent: float, avg_degree: float, k: int, mixing: float,
                         seed: int, device="cpu") -> TorchGraph:
    """The Chung-Lu model of ``chung_lu_graph`` drawn with torch on ``device``.

    Expected degrees w_i ~ i^(-1/(exponent-1)), rescaled to mean avg_degree and capped at
    sqrt(sum w); nodes randomly permuted; k planted communities (uniform labels).  Each of
    round(sum(w)/2) edges picks u ~ w, then v ~ w within u's community with probability
    1 - mixing, else v ~ w over all nodes.  Self-loops and duplicates are dropped; isolated
    nodes are kept."""
    import torch
    dev = torch.device(device)
    gen = torch.Generator(device=dev).manual_seed(int(seed))
    w = torch.arange(1, n + 1, dtype=torch.float64, device=dev) ** (-1.0 / (exponent - 1.0))
    w *= avg_degree / w.mean()
    w = torch.minimum(w, torch.sqrt(w.sum()))
    w *= avg_degree / w.mean()
    perm = torch.randperm(n, generator=gen, device=dev)
    weight = torch.empty(n, dtype=torch.float64, device=dev)
    weight[perm] = w
    labels = torch.randint(0, k, (n,), generator=gen, device=dev, dtype=torch.int64).to(torch.int32)
    order = torch.sort(labels.long(), stable=True).indices
    cw = torch.cumsum(weight[order], 0)
    counts = torch.bincount(labels.long(), minlength=k)
    ends = torch.cumsum(counts, 0)
    starts = ends - counts
    zero = torch.zeros(k, dtype=torch.float64, device=dev)
    lo_w = torch.where(starts > 0, cw[torch.clamp(starts - 1, min=0)], zero)
    hi_w = torch.where(counts > 0, cw[torch.clamp(ends - 1, min=0)], lo_w)
    model = dict(kind="chung_lu", order=order, cw=cw, labels=labels, lo_w=lo_w, hi_w=hi_w,
                 mixing=float(mixing), total=float(cw[-1]))
    m_edges = int(round(float(weight.sum()) / 2.0))
    u, v = _t_chung_lu_draw(torch, gen, model, m_edges)
    upper = _t_upper_from_endpoints(torch, n, u, v)
    del u, v
    return _t_graph_from_upper(torch, n, upper, labels, model)


def edge_redraw_torch(g: TorchGraph, frac: float, seed: int) -> TorchGraph:
    """Edge redrawing (Section 5.1) of a TorchGraph: remove round(frac |E|) uniformly random
    edges, then add as many new edges (absent from the graph, no self-loops) drawn from the
    graph's own model."""
    import torch
    n = g.n
    dev = g.keys.device
    gen = torch.Generator(device=dev).manual_seed(int(seed))
    rows = g.keys // n
    upper = g.keys[rows < g.keys - rows * n]
    del rows
    n_change = int(round(frac * upper.numel()))
    if n_change == 0:
        return g
    drop = torch.randperm(upper.numel(), generator=gen, device=dev)[:n_change]
    keep = torch.ones(upper.numel(), dtype=torch.bool, device=dev)
    keep[drop] = False
    kept = upper[keep]
    added = torch.empty(0, dtype=torch.int64, device=dev)
    while added.numel() < n_change:
        want = (n_change - added.numel()) * 2 + 16
        if g.model.get("kind") == "chung_lu":
            u, v = _t_chung_lu_draw(torch, gen, g.model, want)
        elif g.model.get("kind") == "sbm":
            u, v = _t_sbm_draw(torch, gen, g.model, want)
        else:
            raise ValueError("edge_redraw_torch: graph model must be chung_lu or sbm")
        cand = _t_upper_from_endpoints(torch, n, u, v)
        pos = torch.clamp(torch.searchsorted(upper, cand), max=upper.numel() - 1)
        present = upper[pos] == cand
        if added.numel() > 0:
            sa = added.sort().values
            pa = torch.clamp(torch.searchsorted(sa, cand), max=sa.numel() - 1)
            present |= sa[pa] == cand
        cand = cand[~present]
        cand = cand[torch.randperm(cand.numel(), generator=gen, device=dev)]
        added = torch.cat([added, cand[: n_change - added.numel()]])
    new_upper = torch.cat([kept, added]).sort().values
    return _t_graph_from_upper(torch, n, new_upper, g.labels, g.model)


def sbm_graph_torch(n: int, sizes, avg_degree: float, ratio: float, seed: int,
                    device="cpu") -> TorchGraph:
    """The stochastic block model of ``sbm_graph`` drawn with torch on ``device``: edges per
    block pair ~ Binomial(#pairs, p) with p_in = ratio p_out solved for the node-average degree,
    endpoints uniform within the blocks, duplicates merged, node ids randomly permuted."""
    import torch
    dev = torch.device(device)
    gen = torch.Generator(device=dev).manual_seed(int(seed))
    if np.isscalar(sizes):
        k = int(sizes)
        sizes = np.full(k, n // k, dtype=np.int64)
        sizes[: n - int(sizes.sum())] += 1
    sizes = np.asarray(sizes, dtype=np.int64)
    assert int(sizes.sum()) == n
    p_in, p_out = _sbm_probs(sizes, avg_degree, ratio)
    a_idx, b_idx, pairs, prob = _sbm_pair_table(sizes, p_in, p_out)
    perm = torch.randperm(n, generator=gen, device=dev)
    sz = torch.as_tensor(sizes, device=dev)
    offsets = torch.cumsum(sz, 0) - sz
    labels = torch.empty(n, dtype=torch.int32, device=dev)
    labels[perm] = torch.repeat_interleave(torch.arange(sizes.size, dtype=torch.int32, device=dev), sz)
    counts = torch.binomial(torch.as_tensor(pairs, dtype=torch.float64, device=dev),
                            torch.as_tensor(prob, dtype=torch.float64, device=dev), generator=gen)
    counts = counts.to(torch.int64)
    a = torch.repeat_interleave(torch.as_tensor(a_idx, device=dev), counts)
    b = torch.repeat_interleave(torch.as_tensor(b_idx, device=dev), counts)
    ua = offsets[a] + torch.floor(torch.rand(a.numel(), generator=gen, device=dev, dtype=torch.float64)
                                  * sz[a]).to(torch.int64)
    vb = offsets[b] + torch.floor(torch.rand(b.numel(), generator=gen, device=dev, dtype=torch.float64)
                                  * sz[b]).to(torch.int64)
    upper = _t_upper_from_endpoints(torch, n, perm[ua], perm[vb])
    model = dict(kind="sbm", sizes=sizes, sizes_t=sz, offsets=offsets, members=perm,
                 a_idx=torch.as_tensor(a_idx, device=dev), b_idx=torch.as_tensor(b_idx, device=dev),
                 weight=torch.as_tensor(pairs * prob, dtype=torch.float64, device=dev))
    return _t_graph_from_upper(torch, n, upper, labels, model)
