"""GB300-native dynamic compressive spectral clustering (arXiv:1706.03591).

Thin Python binding of libcsc's C ABI (include/csc.h): every function below
has the name of the C entry point it calls and only marshals arguments.
Arrays may be numpy arrays (host memory) or torch tensors (host or CUDA
memory); every step of the method runs in the CUDA library.  Importing this
package does not need a GPU; calling into the library does.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _abi
from ._abi import CSC_BF16, CSC_DEVICE, CSC_F32, CSC_HOST  # noqa: F401

__all__ = [
    "CscError", "Context", "csc_create", "csc_destroy", "csc_last_error", "csc_set_graph",
    "csc_filter_coeffs", "csc_count_tolerance", "csc_count_from_moments", "csc_trace_count_from_moments",
    "csc_lambda_search_moments", "csc_signals", "csc_cheb_filter", "csc_kmeans",
    "csc_estimate_lambda_k", "csc_filter", "csc_get_features", "csc_get_moments", "csc_cluster",
    "csc_abi_version", "csc_get_stats", "csc_cheb_filter_noalloc", "csc_filter_batched",
    "csc_filter_forward", "csc_filter_vjp", "csc_kmeans_loss_grad", "cheb_filter_layer",
    "csc_laplacian_distance", "csc_compressive_cluster", "csc_save_state", "csc_load_state",
    "csc_splice", "csc_reuse_policy", "csc_filter_adaptive", "csc_tile_plan", "csc_step_launch_bytes",
]


class CscError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"csc status {status}: {message}")
        self.status = status


def _lib():
    return _abi.load()


def _check(status: int, handle=None, what: str = ""):
    if status != _abi.CSC_OK:
        lib = _lib()
        msg = lib.csc_last_error(handle).decode() if handle else ""
        if not msg:
            msg = lib.csc_status_string(status).decode()
        raise CscError(status, f"{what}: {msg}" if what else msg)


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


# element types each array argument may have (numpy has no bfloat16: host features are float32)
_DTYPES = {
    "row_ptr": ("int64",), "col_idx": ("int32",), "vals": ("float32",),
    "assign_out": ("int32",), "prev_assign": ("int32",),
    "psi_out": ("float32",), "theta": ("float32",), "interp_out": ("float32",),
    "R": ("float32", "bfloat16"), "Y": ("float32", "bfloat16"),
    "out": ("float32", "bfloat16"), "dst": ("float32", "bfloat16"),
}


def _check_dtype(x, kind: str):
    want = _DTYPES.get(kind)
    if want is None:
        return
    name = str(x.dtype).replace("torch.", "")
    if name not in want:
        raise TypeError(f"{kind}: element type {name}, expected {' or '.join(want)}")


def _arr(x, kind: str):
    """(pointer, where, dtype-code, leading dimension) of a 1-D/2-D array argument."""
    if x is None:
        return None, _abi.CSC_HOST, _abi.CSC_F32, 0
    if _is_torch(x):
        import torch
        _check_dtype(x, kind)
        if x.numel() > 1 and (x.dim() == 2 and x.stride(1) != 1 or x.dim() == 1 and x.stride(0) != 1):
            raise ValueError(f"{kind}: innermost dimension must be contiguous")
        where = _abi.CSC_DEVICE if x.is_cuda else _abi.CSC_HOST
        code = _abi.CSC_BF16 if x.dtype == torch.bfloat16 else _abi.CSC_F32
        ld = x.stride(0) if x.dim() == 2 else 0
        return C.c_void_p(x.data_ptr()), where, code, ld
    a = np.asarray(x)
    _check_dtype(a, kind)
    if a.size > 1 and (a.ndim == 2 and a.strides[1] != a.itemsize
                       or a.ndim == 1 and a.strides[0] != a.itemsize):
        raise ValueError(f"{kind}: innermost dimension must be contiguous")
    ld = a.strides[0] // a.itemsize if a.ndim == 2 else 0
    return C.c_void_p(a.ctypes.data), _abi.CSC_HOST, _abi.CSC_F32, ld


def csc_abi_version() -> int:
    return _lib().csc_abi_version()


def csc_create(opts: dict | None = None, stream=None):
    """Creates a context; `stream` is a cudaStream_t integer (default: torch's current stream)."""
    lib = _lib()
    o = _abi.csc_opts()
    lib.csc_default_opts(C.byref(o))
    for key, val in (opts or {}).items():
        setattr(o, key, val)
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                stream = torch.cuda.current_stream().cuda_stream
        except ImportError:  # pragma: no cover
            stream = None
    h = C.c_void_p()
    _check(lib.csc_create(C.byref(h), C.byref(o), C.c_void_p(stream or 0)), None, "csc_create")
    return h


def csc_destroy(h) -> None:
    _lib().csc_destroy(h)


def csc_last_error(h) -> str:
    return _lib().csc_last_error(h).decode()


def csc_get_stats(h, reset: bool = False) -> dict:
    st = _abi.csc_stats()
    _check(_lib().csc_get_stats(h, C.byref(st), int(reset)), h, "csc_get_stats")
    return dict(launches=st.launches, step_launches=st.step_launches, step_ms=st.step_ms,
                filter_passes=st.filter_passes, tile=st.tile, batched_launches=st.batched_launches,
                graph_replays=st.graph_replays, autotune_trials=st.autotune_trials,
                batched_waves=st.batched_waves, kmeans_passes=st.kmeans_passes,
                kmeans_near_ties=st.kmeans_near_ties, step_bytes=st.step_bytes,
                kmeans_rows=st.kmeans_rows)


def csc_set_graph(h, n: int, row_ptr, col_idx, vals=None) -> None:
    rp, where, _, _ = _arr(row_ptr, "row_ptr")
    ci, where2, _, _ = _arr(col_idx, "col_idx")
    vv, where3, _, _ = _arr(vals, "vals")
    if where2 != where or (vals is not None and where3 != where):
        raise ValueError("row_ptr, col_idx and vals must live in the same memory")
    nnz = int(col_idx.numel() if _is_torch(col_idx) else np.asarray(col_idx).size)
    _check(_lib().csc_set_graph(h, n, nnz, rp, ci, vv, where), h, "csc_set_graph")


def csc_filter_coeffs(m: int, lambda_c: float) -> np.ndarray:
    a = np.zeros(m + 1)
    _check(_lib().csc_filter_coeffs(m, lambda_c, a.ctypes.data_as(C.POINTER(C.c_double))))
    return a


def csc_count_tolerance(k: int, c: int) -> float:
    return _lib().csc_count_tolerance(k, c)


def csc_tile_plan(c: int, col_tile: int = 0) -> list:
    """Widths of the column tiles of a filtering pass over c columns (host only)."""
    cap = max(1, c // 8 + 1)
    out = (C.c_int * cap)()
    t = _lib().csc_tile_plan(int(c), int(col_tile), out, cap)
    if t < 0:
        raise ValueError(f"csc_tile_plan: bad arguments (c={c}, col_tile={col_tile})")
    return [int(out[i]) for i in range(t)]


def csc_step_launch_bytes(n: int, nnz: int, weighted: bool, w: int, s_prev: int = 4) -> float:
    """Algorithmic bytes of one general step launch over a tile of width w (host only)."""
    return float(_lib().csc_step_launch_bytes(int(n), int(nnz), int(bool(weighted)), int(w), int(s_prev)))


def csc_count_from_moments(m: int, mu, lambda_c: float, d: int, c: int) -> float:
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    out = C.c_double()
    _check(_lib().csc_count_from_moments(m, mu.ctypes.data_as(C.POINTER(C.c_double)), lambda_c, d, c,
                                         C.byref(out)))
    return out.value


def csc_trace_count_from_moments(m: int, mu, lambda_c: float, d: int, c: int) -> float:
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    out = C.c_double()
    _check(_lib().csc_trace_count_from_moments(m, mu.ctypes.data_as(C.POINTER(C.c_double)), lambda_c, d, c,
                                               C.byref(out)))
    return out.value


def csc_lambda_search_moments(m, mu, d, c, k, tau, lambda_prev=-1.0, max_steps=30):
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    lam, cnt, ev = C.c_double(), C.c_double(), C.c_int()
    _check(_lib().csc_lambda_search_moments(m, mu.ctypes.data_as(C.POINTER(C.c_double)), d, c, k, tau,
                                            lambda_prev, max_steps, C.byref(lam), C.byref(cnt),
                                            C.byref(ev)))
    return lam.value, cnt.value, ev.value


def csc_signals(h, seed: int, n: int, col0: int, c: int, d: int, out) -> None:
    ptr, where, code, ld = _arr(out, "out")
    _check(_lib().csc_signals(h, seed, n, col0, c, d, ptr, code, ld or c, where), h, "csc_signals")


def csc_cheb_filter(h, m: int, lambda_c: float, R, psi_out=None, want_moments: bool = True):
    """Filters the caller's block R into psi_out; returns the 2m+1 trace moments (or None)."""
    rp, rw, rcode, ldr = _arr(R, "R")
    c = int(R.shape[1])
    pp, pw, _, ldp = _arr(psi_out, "psi_out")
    mu = np.zeros(2 * m + 1) if want_moments else None
    _check(_lib().csc_cheb_filter(h, m, lambda_c, rp, rcode, c, ldr or c, rw, pp, ldp or c, pw,
                                  mu.ctypes.data_as(C.POINTER(C.c_double)) if mu is not None else None),
           h, "csc_cheb_filter")
    return mu


def csc_kmeans(h, Y, k: int, init_idx, prev_assign=None, max_iter: int = 0, assign_out=None,
               want_centroids: bool = True):
    """Lloyd k-means of the rows of Y; returns dict(assign, centroids, inertia, iters)."""
    yp, yw, ycode, ldy = _arr(Y, "Y")
    n, d = int(Y.shape[0]), int(Y.shape[1])
    idx = np.ascontiguousarray(init_idx, dtype=np.int64)
    if assign_out is None:
        assign_out = np.zeros(n, dtype=np.int32)
    ap, aw, _, _ = _arr(assign_out, "assign_out")
    pv = None
    if prev_assign is not None:
        pv, pw, _, _ = _arr(prev_assign, "prev_assign")
        if pw != aw:
            raise ValueError("prev_assign must live where assign_out lives")
    cents = np.zeros((k, d)) if want_centroids else None
    inertia, iters = C.c_double(), C.c_int()
    _check(_lib().csc_kmeans(h, yp, ycode, n, d, ldy or d, yw, k, C.c_void_p(idx.ctypes.data), pv,
                             max_iter, ap, aw,
                             cents.ctypes.data_as(C.POINTER(C.c_double)) if cents is not None else None,
                             C.byref(inertia), C.byref(iters)), h, "csc_kmeans")
    return dict(assign=assign_out, centroids=cents, inertia=inertia.value, iters=iters.value)


def csc_estimate_lambda_k(h, k: int, m: int, d: int, seed: int):
    lam, cnt, ev = C.c_double(), C.c_double(), C.c_int()
    _check(_lib().csc_estimate_lambda_k(h, k, m, d, seed, C.byref(lam), C.byref(cnt), C.byref(ev)), h,
           "csc_estimate_lambda_k")
    return lam.value, cnt.value, ev.value


def csc_filter(h, m: int, d: int, p: float, seed: int, k: int = 0, lambda_c: float = -1.0):
    """Algorithm 1 (reuse, new filtering, eigencount check, refinement); returns (lambda_c, count, dichotomy evaluations, columns filtered)."""
    lam, cnt, ev, cols = C.c_double(), C.c_double(), C.c_int(), C.c_int()
    _check(_lib().csc_filter(h, m, d, p, seed, k, lambda_c, C.byref(lam), C.byref(cnt), C.byref(ev),
                             C.byref(cols)), h, "csc_filter")
    return lam.value, cnt.value, ev.value, cols.value


def _policy(alpha: float, budget: float, rho_skip: float):
    return _abi.csc_similarity_policy(float(alpha), float(budget), float(rho_skip))


def csc_reuse_policy(d: int, p_max: float, rho: float, alpha: float, budget: float, rho_skip: float,
                     rho_since: float = 0.0):
    """Host-only decision of the edge-similarity policy: (dp, check, rho summed since the check)."""
    pol = _policy(alpha, budget, rho_skip)
    dp, ck, acc = C.c_int(), C.c_int(), C.c_double()
    _check(_lib().csc_reuse_policy(d, p_max, rho, C.byref(pol), rho_since, C.byref(dp), C.byref(ck),
                                   C.byref(acc)))
    return dp.value, bool(ck.value), acc.value


def csc_filter_adaptive(h, m: int, d: int, p_max: float, seed: int, k: int, rho: float, alpha: float,
                        budget: float, rho_skip: float):
    """csc_filter under the edge-similarity policy; returns (lambda_c, count, evaluations,
    columns filtered, check ran)."""
    pol = _policy(alpha, budget, rho_skip)
    lam, cnt, ev, cols, ck = C.c_double(), C.c_double(), C.c_int(), C.c_int(), C.c_int()
    _check(_lib().csc_filter_adaptive(h, m, d, p_max, seed, k, rho, C.byref(pol), C.byref(lam), C.byref(cnt),
                                      C.byref(ev), C.byref(cols), C.byref(ck)), h, "csc_filter_adaptive")
    return lam.value, cnt.value, ev.value, cols.value, bool(ck.value)


def csc_splice(h, n: int, d: int, p: float, psi_new, lambda_c: float) -> None:
    """Eq. 6 splice of caller-filtered columns (n x c float32, host or device) into the ring."""
    ptr, where, _, ld = _arr(psi_new, "psi_out")
    c = int(psi_new.shape[1])
    _check(_lib().csc_splice(h, n, d, p, ptr, c, ld or c, where, lambda_c), h, "csc_splice")


def csc_get_features(h, dst, normalized: bool = False) -> None:
    ptr, where, code, ld = _arr(dst, "dst")
    _check(_lib().csc_get_features(h, ptr, code, ld or int(dst.shape[1]), int(normalized), where), h,
           "csc_get_features")


def csc_get_moments(h, length: int) -> np.ndarray:
    mu = np.zeros(length)
    _check(_lib().csc_get_moments(h, mu.ctypes.data_as(C.POINTER(C.c_double)), length), h,
           "csc_get_moments")
    return mu


def csc_cluster(h, k: int, seed: int, init_idx, assign_out):
    """Algorithm 1 (clustering of the combined features); writes assign_out and returns (cost C_Theta, Lloyd passes)."""
    idx = None if init_idx is None else np.ascontiguousarray(init_idx, dtype=np.int64)
    ap, aw, _, _ = _arr(assign_out, "assign_out")
    cost, iters = C.c_double(), C.c_int()
    _check(_lib().csc_cluster(h, k, seed, None if idx is None else C.c_void_p(idx.ctypes.data), ap, aw,
                              C.byref(cost), C.byref(iters)), h, "csc_cluster")
    return cost.value, iters.value


def csc_filter_batched(h, graphs, m: int, want_moments: bool = True):
    """Filters many graphs in one persistent launch.  ``graphs`` is a list of dicts with keys
    n, row_ptr, col_idx (device tensors), vals (device tensor or None), c, d, lambda_c, seed,
    psi (device float32 tensor n x c or None).  Returns the moments, shape (len(graphs), 2m+1)."""
    descs = (_abi.csc_graph_desc * len(graphs))()
    for i, g in enumerate(graphs):
        for key in ("row_ptr", "col_idx", "vals", "psi"):
            x = g.get(key)
            if x is not None:
                if not (_is_torch(x) and x.is_cuda):
                    raise ValueError(f"graph {i}: {key} must be a CUDA tensor")
                _check_dtype(x, "psi_out" if key == "psi" else key)
        dsc = descs[i]
        dsc.n = int(g["n"])
        dsc.nnz = int(g["col_idx"].numel())
        dsc.row_ptr = g["row_ptr"].data_ptr()
        dsc.col_idx = g["col_idx"].data_ptr() if g["col_idx"].numel() else None
        dsc.vals = g["vals"].data_ptr() if g.get("vals") is not None else None
        dsc.c = int(g["c"])
        dsc.d = int(g.get("d", g["c"]))
        dsc.lambda_c = float(g["lambda_c"])
        dsc.seed = int(g["seed"])
        psi = g.get("psi")
        dsc.psi = psi.data_ptr() if psi is not None else None
        dsc.ldp = int(psi.stride(0)) if psi is not None else int(g["c"])
    mu = np.zeros((len(graphs), 2 * m + 1)) if want_moments else None
    _check(_lib().csc_filter_batched(h, len(graphs), descs, m,
                                     mu.ctypes.data_as(C.POINTER(C.c_double)) if mu is not None else None),
           h, "csc_filter_batched")
    return mu


def _device_f32(x, kind: str):
    import torch
    if not (_is_torch(x) and x.is_cuda and x.dtype == torch.float32 and x.dim() == 2 and
            (x.numel() <= 1 or x.stride(1) == 1)):
        raise ValueError(f"{kind}: expected a CUDA float32 matrix with contiguous rows")
    return C.c_void_p(x.data_ptr()), int(x.stride(0))


def csc_filter_forward(h, m: int, coef, R, psi_out, stride: int = 0) -> None:
    """Psi = sum_j coef[j] T_j(L~) R into psi_out, keeping the recursion checkpoints for
    csc_filter_vjp (R and psi_out: CUDA float32, n x c)."""
    a = np.ascontiguousarray(coef, dtype=np.float64)
    if a.size != m + 1:
        raise ValueError("coef must have m + 1 entries")
    r, ldr = _device_f32(R, "R")
    p, ldp = _device_f32(psi_out, "psi_out")
    _check(_lib().csc_filter_forward(h, m, a.ctypes.data_as(C.POINTER(C.c_double)), r, int(R.shape[1]), ldr,
                                     p, ldp, stride), h, "csc_filter_forward")


def csc_filter_vjp(h, m: int, grad_psi, grad_w=None) -> np.ndarray:
    """dloss/dcoef (float64, m + 1) of the last csc_filter_forward (of order m); dloss/dw
    written to grad_w (CUDA float32, one entry per stored edge) when given."""
    g, ldg = _device_f32(grad_psi, "grad_psi")
    gw = None
    if grad_w is not None:
        import torch
        if not (grad_w.is_cuda and grad_w.dtype == torch.float32 and grad_w.is_contiguous()):
            raise ValueError("grad_w: expected a contiguous CUDA float32 vector")
        gw = C.c_void_p(grad_w.data_ptr())
    out = np.zeros(m + 1)
    _check(_lib().csc_filter_vjp(h, g, ldg, out.ctypes.data_as(C.POINTER(C.c_double)), gw), h, "csc_filter_vjp")
    return out


def csc_kmeans_loss_grad(h, psi, mu, assign, grad_out) -> float:
    """loss = sum_i ||psi_i/||psi_i|| - mu[assign[i]]||^2 and dloss/dPsi into grad_out
    (all CUDA tensors: psi, grad_out float32 n x c, mu float32 k x c, assign int32 n)."""
    import torch
    p, ldp = _device_f32(psi, "psi")
    go, ldg = _device_f32(grad_out, "grad_out")
    mu = mu.contiguous()
    if not (mu.is_cuda and mu.dtype == torch.float32 and assign.is_cuda and assign.dtype == torch.int32):
        raise ValueError("mu: CUDA float32 (k x c); assign: CUDA int32")
    loss = C.c_double()
    _check(_lib().csc_kmeans_loss_grad(h, p, ldp, int(psi.shape[0]), int(psi.shape[1]), C.c_void_p(mu.data_ptr()),
                                       int(mu.shape[0]), C.c_void_p(assign.contiguous().data_ptr()), go, ldg,
                                       C.byref(loss)), h, "csc_kmeans_loss_grad")
    return loss.value


def csc_laplacian_distance(h, n: int, graph_a, graph_b) -> float:
    """||L_b - L_a||_F (Definition 4.1); each graph is (row_ptr, col_idx, vals or None) of
    CUDA tensors."""
    ptrs = []
    for rp, ci, vv in (graph_a, graph_b):
        ptrs += [C.c_void_p(rp.data_ptr()), C.c_void_p(ci.data_ptr()) if ci.numel() else None,
                 None if vv is None else C.c_void_p(vv.data_ptr())]
    rho = C.c_double()
    _check(_lib().csc_laplacian_distance(h, n, *ptrs, C.byref(rho)), h, "csc_laplacian_distance")
    return rho.value


def csc_save_state(h, path: str) -> None:
    """Writes the context's dynamic state (feature ring, cutoff, previous assignment) to path."""
    _check(_lib().csc_save_state(h, str(path).encode()), h, "csc_save_state")


def csc_load_state(h, path: str) -> None:
    """Replaces the context's dynamic state with the one saved at path."""
    _check(_lib().csc_load_state(h, str(path).encode()), h, "csc_load_state")


def csc_compressive_cluster(h, k: int, theta=None, Y=None, n_draws: int = 0, n_init: int = 0,
                            lambda_c: float = -1.0, m: int = 0, seed: int = 0, max_iter: int = 0,
                            assign_out=None, want_sample: bool = False, interp_out=None):
    """Compressive k-means (see include/csc.h).  theta (float32) and Y (float32 or bfloat16),
    both n x d, or None for the context's current features.  Returns dict(assign, n_sampled,
    restart, sample, sample_labels); assign_out and interp_out (n x k float32) may be given
    as arrays or CUDA tensors, the sample arrays are host numpy arrays."""
    if (theta is None) != (Y is None):
        raise ValueError("give both theta and Y, or neither")
    tp, tw, _, ldt = _arr(theta, "theta")
    yp, yw, ycode, ldy = _arr(Y, "Y")
    d = 0
    if theta is not None:
        if tw != yw or ldt != ldy:
            raise ValueError("theta and Y must share memory kind and leading dimension")
        d = int(theta.shape[1])
    if assign_out is None:
        raise ValueError("assign_out (int32[n]) is required")
    ap, aw, _, _ = _arr(assign_out, "assign_out")
    xp, xw, _, ldx = _arr(interp_out, "interp_out")
    if interp_out is not None and xw != aw:
        raise ValueError("interp_out must live where assign_out lives")
    cap = int(n_draws) if n_draws > 0 else max(k, int(np.ceil(2.0 * k * np.log(max(k, 1)))))
    sample = np.zeros(cap, dtype=np.int32) if want_sample else None
    slabels = np.zeros(cap, dtype=np.int32) if want_sample else None
    if want_sample and aw != _abi.CSC_HOST:
        raise ValueError("want_sample needs host outputs (assign_out in host memory)")
    ns, rs = C.c_int64(), C.c_int()
    _check(_lib().csc_compressive_cluster(
        h, tp, yp, ycode, d, ldy or d, yw, k, n_draws, n_init, lambda_c, m, seed, max_iter, ap, aw,
        C.c_void_p(sample.ctypes.data) if sample is not None else None,
        C.c_void_p(slabels.ctypes.data) if slabels is not None else None,
        xp, ldx or k, C.byref(ns), C.byref(rs)), h, "csc_compressive_cluster")
    out = dict(assign=assign_out, n_sampled=ns.value, restart=rs.value, sample=None, sample_labels=None)
    if want_sample:
        out["sample"] = sample[: ns.value]
        out["sample_labels"] = slabels[: ns.value]
    return out


_FILTER_FN = None


def cheb_filter_layer(context, n: int, row_ptr, col_idx, weights, coef, R, stride: int = 0):
    """Differentiable Psi = sum_j coef[j] T_j(L~(weights)) R (torch.autograd): gradients flow to
    ``coef`` (float64 tensor, m + 1) and ``weights`` (CUDA float32, one per stored edge, the
    two copies of an edge holding the same value).  The graph of ``context`` is replaced by
    (row_ptr, col_idx, weights); one forward may be pending per context."""
    global _FILTER_FN
    if _FILTER_FN is None:
        import torch

        class ChebFilterFunction(torch.autograd.Function):
            @staticmethod
            def forward(fctx, coef_t, w_t, ctx_obj, n_, rp, ci, r_t, stride_):
                ctx_obj.set_graph(n_, rp, ci, w_t.detach().contiguous())
                psi = torch.empty((n_, r_t.shape[1]), device=r_t.device, dtype=torch.float32)
                csc_filter_forward(ctx_obj.h, coef_t.numel() - 1, coef_t.detach().cpu().numpy(), r_t, psi, stride_)
                fctx.ctx_obj, fctx.nnz, fctx.m = ctx_obj, int(ci.numel()), coef_t.numel() - 1
                fctx.coef_meta = (coef_t.dtype, coef_t.device)
                return psi

            @staticmethod
            def backward(fctx, grad_psi):
                gw = torch.empty(fctx.nnz, device=grad_psi.device, dtype=torch.float32)
                gc = csc_filter_vjp(fctx.ctx_obj.h, fctx.m, grad_psi.contiguous(), gw)
                gct = torch.from_numpy(gc).to(dtype=fctx.coef_meta[0], device=fctx.coef_meta[1])
                return gct, gw, None, None, None, None, None, None

        _FILTER_FN = ChebFilterFunction
    return _FILTER_FN.apply(coef, weights, context, n, row_ptr, col_idx, R, stride)


def csc_cheb_filter_noalloc(n: int, row_ptr, col_idx, vals, m: int, lambda_c: float, R,
                            psi_out=None, want_moments: bool = True, stream=None):
    """Allocation-free filter of a device signal block R over a device CSR graph (small
    graphs only; see include/csc.h).  Every array must be a CUDA torch tensor: row_ptr int64
    [n+1], col_idx int32 [nnz], vals float32 [nnz] or None, R float32 [n, c], psi_out float32
    [n, c] or None.  Returns the 2m+1 trace moments (or None)."""
    import torch
    n = int(n)
    named = (("row_ptr", row_ptr, torch.int64), ("col_idx", col_idx, torch.int32),
             ("vals", vals, torch.float32), ("R", R, torch.float32), ("psi_out", psi_out, torch.float32))
    for kind, x, dt in named:
        if x is None and kind in ("vals", "psi_out"):
            continue
        if not (_is_torch(x) and x.is_cuda):
            raise TypeError(f"csc_cheb_filter_noalloc: {kind} must be a CUDA tensor")
        if x.dtype != dt:
            raise TypeError(f"csc_cheb_filter_noalloc: {kind} must be {dt}, got {x.dtype}")
    if row_ptr.dim() != 1 or row_ptr.numel() != n + 1:
        raise ValueError("csc_cheb_filter_noalloc: row_ptr must hold n + 1 entries")
    if col_idx.dim() != 1 or not col_idx.is_contiguous():
        raise ValueError("csc_cheb_filter_noalloc: col_idx must be a contiguous vector")
    nnz = int(col_idx.numel())
    if vals is not None and (vals.dim() != 1 or vals.numel() != nnz or not vals.is_contiguous()):
        raise ValueError("csc_cheb_filter_noalloc: vals must hold one weight per stored edge")
    if R.dim() != 2 or R.shape[0] != n:
        raise ValueError("csc_cheb_filter_noalloc: R must be n x c")
    c = int(R.shape[1])
    if psi_out is not None and (psi_out.dim() != 2 or tuple(psi_out.shape) != (n, c)):
        raise ValueError("csc_cheb_filter_noalloc: psi_out must be n x c")
    rp, _, _, _ = _arr(row_ptr, "row_ptr")
    ci, _, _, _ = _arr(col_idx, "col_idx")
    vv, _, _, _ = _arr(vals, "vals")
    r, _, _, ldr = _arr(R, "R")
    pp, _, _, ldp = _arr(psi_out, "psi_out")
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    mu = np.zeros(2 * m + 1) if want_moments else None
    _check(_lib().csc_cheb_filter_noalloc(
        n, nnz, rp, ci, vv, m, lambda_c, r, c, ldr or c, pp, ldp or c,
        mu.ctypes.data_as(C.POINTER(C.c_double)) if mu is not None else None, C.c_void_p(stream or 0)),
        None, "csc_cheb_filter_noalloc")
    return mu


class Context:
    """Owns a csc context handle; methods forward to the csc_* functions above."""

    def __init__(self, opts: dict | None = None, stream=None):
        self.h = csc_create(opts, stream)

    def close(self):
        if self.h:
            csc_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def filter_batched(self, graphs, m, want_moments=True):
        return csc_filter_batched(self.h, graphs, m, want_moments)

    def stats(self, reset=False):
        return csc_get_stats(self.h, reset)

    def set_graph(self, n, row_ptr, col_idx, vals=None):
        csc_set_graph(self.h, n, row_ptr, col_idx, vals)

    def signals(self, seed, n, col0, c, d, out):
        csc_signals(self.h, seed, n, col0, c, d, out)

    def cheb_filter(self, m, lambda_c, R, psi_out=None, want_moments=True):
        return csc_cheb_filter(self.h, m, lambda_c, R, psi_out, want_moments)

    def kmeans(self, Y, k, init_idx, prev_assign=None, max_iter=0, assign_out=None, want_centroids=True):
        return csc_kmeans(self.h, Y, k, init_idx, prev_assign, max_iter, assign_out, want_centroids)

    def estimate_lambda_k(self, k, m, d, seed):
        return csc_estimate_lambda_k(self.h, k, m, d, seed)

    def filter(self, m, d, p, seed, k=0, lambda_c=-1.0):
        return csc_filter(self.h, m, d, p, seed, k, lambda_c)

    def filter_adaptive(self, m, d, p_max, seed, k, rho, alpha, budget, rho_skip=0.0):
        return csc_filter_adaptive(self.h, m, d, p_max, seed, k, rho, alpha, budget, rho_skip)

    def splice(self, n, d, p, psi_new, lambda_c):
        return csc_splice(self.h, n, d, p, psi_new, lambda_c)

    def get_features(self, dst, normalized=False):
        csc_get_features(self.h, dst, normalized)

    def save_state(self, path):
        csc_save_state(self.h, path)

    def load_state(self, path):
        csc_load_state(self.h, path)

    def compressive_cluster(self, k, theta=None, Y=None, **kw):
        return csc_compressive_cluster(self.h, k, theta, Y, **kw)

    def get_moments(self, length):
        return csc_get_moments(self.h, length)

    def cluster(self, k, seed, init_idx, assign_out):
        return csc_cluster(self.h, k, seed, init_idx, assign_out)

    def filter_forward(self, m, coef, R, psi_out, stride=0):
        csc_filter_forward(self.h, m, coef, R, psi_out, stride)
        self._grad_m = m

    def filter_vjp(self, grad_psi, grad_w=None):
        return csc_filter_vjp(self.h, getattr(self, "_grad_m", 0), grad_psi, grad_w)

    def kmeans_loss_grad(self, psi, mu, assign, grad_out):
        return csc_kmeans_loss_grad(self.h, psi, mu, assign, grad_out)

    def laplacian_distance(self, n, graph_a, graph_b):
        return csc_laplacian_distance(self.h, n, graph_a, graph_b)

    @property
    def last_error(self):
        return csc_last_error(self.h)
