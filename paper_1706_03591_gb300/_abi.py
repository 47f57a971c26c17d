"""ctypes declarations of libcsc's C ABI (include/csc.h).

Loading fails loudly when the shared library is missing: there is no CPU
fallback for any entry point.
"""
from __future__ import annotations

import ctypes as C
import os

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libcsc.so")

CSC_OK, CSC_EINVAL, CSC_ENOMEM, CSC_ECUDA, CSC_ETIMEOUT, CSC_ESTATE, CSC_ELIMIT = range(7)
CSC_HOST, CSC_DEVICE = 0, 1
CSC_F32, CSC_BF16 = 0, 1


class csc_opts(C.Structure):
    _fields_ = [
        ("precision", C.c_int),
        ("count_tol", C.c_double),
        ("max_bisect", C.c_int),
        ("max_iter", C.c_int),
        ("col_tile", C.c_int),
        ("checked", C.c_int),
        ("timing", C.c_int),
        ("estimator", C.c_int),
        ("reorder", C.c_int),
        ("wave_bytes", C.c_int64),
    ]


class csc_stats(C.Structure):
    _fields_ = [
        ("launches", C.c_int64),
        ("step_launches", C.c_int64),
        ("step_ms", C.c_double),
        ("filter_passes", C.c_int64),
        ("tile", C.c_int64),
        ("batched_launches", C.c_int64),
        ("graph_replays", C.c_int64),
        ("autotune_trials", C.c_int64),
        ("batched_waves", C.c_int64),
        ("kmeans_passes", C.c_int64),
        ("kmeans_near_ties", C.c_int64),
        ("step_bytes", C.c_double),
        ("kmeans_rows", C.c_int64),
    ]


class csc_similarity_policy(C.Structure):
    _fields_ = [("alpha", C.c_double), ("budget", C.c_double), ("rho_skip", C.c_double)]


class csc_graph_desc(C.Structure):
    _fields_ = [
        ("n", C.c_int64),
        ("nnz", C.c_int64),
        ("row_ptr", C.c_void_p),
        ("col_idx", C.c_void_p),
        ("vals", C.c_void_p),
        ("c", C.c_int),
        ("d", C.c_int),
        ("lambda_c", C.c_double),
        ("seed", C.c_uint64),
        ("psi", C.c_void_p),
        ("ldp", C.c_int64),
    ]


_p = C.c_void_p
_i32, _i64, _u64, _dbl = C.c_int, C.c_int64, C.c_uint64, C.c_double
_pd, _pi = C.POINTER(C.c_double), C.POINTER(C.c_int)

# name -> (restype, argtypes); the order matches include/csc.h
SIGNATURES = {
    "csc_default_opts": (None, [C.POINTER(csc_opts)]),
    "csc_status_string": (C.c_char_p, [_i32]),
    "csc_abi_version": (_i32, []),
    "csc_tile_plan": (_i32, [_i32, _i32, C.POINTER(C.c_int), _i32]),
    "csc_step_launch_bytes": (C.c_double, [C.c_int64, C.c_int64, _i32, _i32, _i32]),
    "csc_create": (_i32, [C.POINTER(_p), C.POINTER(csc_opts), _p]),
    "csc_destroy": (None, [_p]),
    "csc_last_error": (C.c_char_p, [_p]),
    "csc_get_stats": (_i32, [_p, C.POINTER(csc_stats), _i32]),
    "csc_set_graph": (_i32, [_p, _i64, _i64, _p, _p, _p, _i32]),
    "csc_filter_coeffs": (_i32, [_i32, _dbl, _pd]),
    "csc_count_tolerance": (_dbl, [_i32, _i32]),
    "csc_count_from_moments": (_i32, [_i32, _pd, _dbl, _i32, _i32, _pd]),
    "csc_trace_count_from_moments": (_i32, [_i32, _pd, _dbl, _i32, _i32, _pd]),
    "csc_lambda_search_moments": (_i32, [_i32, _pd, _i32, _i32, _i32, _dbl, _dbl, _i32, _pd, _pd, _pi]),
    "csc_signals": (_i32, [_p, _u64, _i64, _i64, _i32, _i32, _p, _i32, _i64, _i32]),
    "csc_cheb_filter": (_i32, [_p, _i32, _dbl, _p, _i32, _i32, _i64, _i32, _p, _i64, _i32, _pd]),
    "csc_kmeans": (_i32, [_p, _p, _i32, _i64, _i32, _i64, _i32, _i32, _p, _p, _i32, _p, _i32, _pd,
                          _pd, _pi]),
    "csc_estimate_lambda_k": (_i32, [_p, _i32, _i32, _i32, _u64, _pd, _pd, _pi]),
    "csc_filter": (_i32, [_p, _i32, _i32, _dbl, _u64, _i32, _dbl, _pd, _pd, _pi, _pi]),
    "csc_get_features": (_i32, [_p, _p, _i32, _i64, _i32, _i32]),
    "csc_get_moments": (_i32, [_p, _pd, _i32]),
    "csc_cluster": (_i32, [_p, _i32, _u64, _p, _p, _i32, _pd, _pi]),
    "csc_filter_batched": (_i32, [_p, _i32, _p, _i32, _pd]),
    "csc_reuse_policy": (_i32, [_i32, _dbl, _dbl, _p, _dbl, _pi, _pi, _pd]),
    "csc_filter_adaptive": (_i32, [_p, _i32, _i32, _dbl, _u64, _i32, _dbl, _p, _pd, _pd, _pi, _pi, _pi]),
    "csc_splice": (_i32, [_p, _i64, _i32, _dbl, _p, _i32, _i64, _i32, _dbl]),
    "csc_cheb_filter_noalloc": (_i32, [_i64, _i64, _p, _p, _p, _i32, _dbl, _p, _i32, _i64, _p, _i64,
                                       _pd, _p]),
    "csc_filter_forward": (_i32, [_p, _i32, _pd, _p, _i32, _i64, _p, _i64, _i32]),
    "csc_filter_vjp": (_i32, [_p, _p, _i64, _pd, _p]),
    "csc_kmeans_loss_grad": (_i32, [_p, _p, _i64, _i64, _i32, _p, _i32, _p, _p, _i64, _pd]),
    "csc_laplacian_distance": (_i32, [_p, _i64, _p, _p, _p, _p, _p, _p, _pd]),
    "csc_save_state": (_i32, [_p, C.c_char_p]),
    "csc_load_state": (_i32, [_p, C.c_char_p]),
    "csc_compressive_cluster": (_i32, [_p, _p, _p, _i32, _i32, _i64, _i32, _i32, _i64, _i32, _dbl, _i32, _u64,
                                       _i32, _p, _i32, _p, _p, _p, _i64, C.POINTER(C.c_int64), _pi]),
}

_lib = None


def load(path: str | None = None):
    """The loaded library with argtypes set (cached)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(
            f"libcsc.so not found at {path}: build it with "
            "`python -c 'import __graft_entry__ as g; g.build()'` (no CPU fallback exists)")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path == LIB_PATH:
        _lib = lib
    return lib
