import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long CPU-side oracle run")


def read_golden(name):
    """Non-comment lines of a golden fixture, split on whitespace."""
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def rel(a, b):
    """Relative Frobenius error ||a - b|| / ||b|| in float64."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def fp32_filter(lt, r, a):
    """A plain float32 evaluation of sum_j a_j T_j(L~) R by the three-term recursion."""
    lt32 = lt.astype(np.float32)
    a32 = np.asarray(a, dtype=np.float32)
    t_prev = np.asarray(r, dtype=np.float32)
    t_cur = lt32 @ t_prev
    out = a32[0] * t_prev + a32[1] * t_cur
    for j in range(2, a32.size):
        t_prev, t_cur = t_cur, 2.0 * (lt32 @ t_cur) - t_prev
        out += a32[j] * t_cur
    return out


def fp32_floor(lt, r, a, ref):
    """Error against ``ref`` of a plain float32 evaluation of sum_j a_j T_j(L~) R by the
    three-term recursion: the rounding floor that any float32 implementation of the filter
    meets at this size (large when the output cancels, e.g. h(1) on an edgeless graph)."""
    return rel(fp32_filter(lt, r, a), ref)


def graph_from_edges(n, edges):
    """CSR (row_ptr int64, col_idx int32) of an undirected edge list."""
    adj = [[] for _ in range(n)]
    for u, v in edges:
        adj[u].append(v)
        adj[v].append(u)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    cols = []
    for i in range(n):
        nb = sorted(adj[i])
        cols.extend(nb)
        row_ptr[i + 1] = row_ptr[i] + len(nb)
    return row_ptr, np.array(cols, dtype=np.int32)


@pytest.fixture(scope="session")
def gpu_lib():
    """The CUDA library binding on a GPU machine (fails loudly if it is missing)."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1706_03591_gb300 as csc
    return csc
