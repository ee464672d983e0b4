"""ctypes binding of libcss (include/css.h).  Argument marshalling only.

The shared library is built in-tree (paper_1312_6838_gb300/libcss.so) by
``paper_1312_6838_gb300.build``.  Loading fails loudly when it is missing:
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcss.so")

CSS_OK = 0
CSS_RANK_EXHAUSTED = 1
CSS_ERR_INVALID_ARG = -1
CSS_ERR_CUDA = -2
CSS_ERR_NO_MEMORY = -3
CSS_ERR_WORKSPACE = -4
CSS_ERR_TIMEOUT = -5
CSS_ERR_NONFINITE = -6
CSS_ERR_UNSUPPORTED = -7
CSS_ERR_NOT_CONVERGED = -8

CSS_F64, CSS_F32, CSS_BF16 = 0, 1, 2
(CSS_OP_SELECT, CSS_OP_GCSS, CSS_OP_DISTRIBUTED, CSS_OP_PROJECT, CSS_OP_BACKWARD,
 CSS_OP_HOST_SELECT, CSS_OP_PROJECT_RANDOM, CSS_OP_RANDOMIZED, CSS_OP_EMBED,
 CSS_OP_LOWRANK) = range(10)
CSS_OMEGA_GAUSSIAN, CSS_OMEGA_SPARSE_SIGN = 0, 1
CSS_KNOB_TILE_COLS, CSS_KNOB_SPLIT_SHARE, CSS_KNOB_PIVOT_COST = 0, 1, 2


class css_opts(C.Structure):
    _fields_ = [
        ("tau_rel", C.c_double),
        ("forced", C.c_void_p),
        ("n_forced", C.c_int32),
        ("score_mode", C.c_int32),
        ("sync", C.c_int32),
        ("spin_budget_ns", C.c_uint64),
        ("grid_ctas", C.c_int32),
        ("tile_cols", C.c_int32),
        ("diag_argmax", C.c_void_p),
        ("timing_ms", C.c_void_p),
        ("diag_f", C.c_void_p),
        ("diag_g", C.c_void_p),
        ("init_path", C.c_int32),
        ("test_unmet_wait", C.c_int32),
        ("split_share", C.c_int32),
        ("pivot_cost", C.c_int32),
        ("reserved", C.c_int32 * 4),
        ("trace_ns", C.c_void_p),
        ("basis", C.c_void_p),
    ]


class css_problem(C.Structure):
    _fields_ = [
        ("A", C.c_void_p),
        ("m", C.c_int64),
        ("n", C.c_int64),
        ("lda", C.c_int64),
        ("k", C.c_int32),
        ("pad_", C.c_int32),
        ("sel", C.c_void_p),
        ("trace", C.c_void_p),
        ("n_sel", C.c_void_p),
        ("W", C.c_void_p),
    ]


P = C.c_void_p
I32 = C.c_int32
I64 = C.c_int64
SZ = C.c_size_t
DBL = C.c_double

class css_batched_plan(C.Structure):
    """Opaque host record of a prepared batch (css_select_batched_prepare)."""
    _fields_ = [("opaque", C.c_uint64 * 64)]


class css_distributed_plan(C.Structure):
    """Opaque host record of a prepared Algorithm 4 call (gcss_distributed_prepare)."""
    _fields_ = [("opaque", C.c_uint64 * 128)]


_SIGS = {
    "css_opts_default": (None, [C.POINTER(css_opts)]),
    "css_status_string": (C.c_char_p, [I32]),
    "css_version": (C.c_char_p, []),
    "css_workspace_size": (SZ, [I32, I32, I64, I64, I64, I32, I32, C.POINTER(css_opts)]),
    "css_select": (I32, [P, I32, I64, I64, I64, I32, P, P, P, P, P, SZ, C.POINTER(css_opts), P]),
    "gcss_select": (I32, [P, I32, I64, I64, I64, P, I64, I64, I32, P, P, P, P, P, SZ,
                          C.POINTER(css_opts), P]),
    "gcss_distributed_workspace_size": (SZ, [I32, I64, I64, I64, C.POINTER(I64), I32, I32, I32]),
    "gcss_distributed": (I32, [P, I32, I64, I64, I64, P, I64, I64, C.POINTER(I64), I32, I32, I32,
                               P, P, P, P, P, SZ, C.POINTER(css_opts), P]),
    "gcss_distributed_prepare": (I32, [P, I32, I64, I64, I64, P, I64, I64, C.POINTER(I64), I32, I32, I32,
                                       P, P, P, P, P, SZ, C.POINTER(css_opts),
                                       C.POINTER(css_distributed_plan), P]),
    "gcss_distributed_run": (I32, [C.POINTER(css_distributed_plan), P, P]),
    "css_project": (I32, [P, I32, I64, I64, I64, P, I64, I64, P, I64, P, SZ,
                          C.POINTER(css_opts), P]),
    "css_batched_workspace_size": (SZ, [C.POINTER(css_problem), I32, I32, C.POINTER(css_opts)]),
    "css_select_batched": (I32, [C.POINTER(css_problem), I32, I32, P, SZ, C.POINTER(css_opts), P]),
    "css_select_batched_prepare": (I32, [C.POINTER(css_problem), I32, I32, P, SZ, C.POINTER(css_opts),
                                         C.POINTER(css_batched_plan), P]),
    "css_select_batched_run": (I32, [C.POINTER(css_batched_plan), P, P]),
    "css_autotune_select": (I32, [P, I32, I64, I64, I64, I32, P, P, P, P, SZ, C.POINTER(C.c_int32),
                                  P, P]),
    "css_tile_record": (I32, [C.c_char_p, I32, I64, I64, I32]),
    "css_tile_lookup": (I32, [C.c_char_p, I32, I64, I64]),
    "css_tile_cache_save": (I32, [C.c_char_p]),
    "css_tile_cache_load": (I32, [C.c_char_p]),
    "css_tune_record": (I32, [C.c_char_p, I32, I64, I64, I32, I32]),
    "css_tune_lookup": (I32, [C.c_char_p, I32, I64, I64, I32]),
    "css_autotune_distributed": (I32, [P, I32, I64, I64, I64, P, I64, I64, C.POINTER(I64), I32, I32, I32,
                                       P, P, P, P, SZ, C.POINTER(C.c_int32), P, P]),
    "css_random_omega": (I32, [I64, I64, C.c_uint64, I32, I32, P, I64, P]),
    "css_project_random": (I32, [P, I32, I64, I64, I64, I64, C.c_uint64, I32, P, I64, P, SZ,
                                 C.POINTER(css_opts), P]),
    "css_select_randomized": (I32, [P, I32, I64, I64, I64, I32, C.c_uint64, I32, P, P, P, P, SZ,
                                    C.POINTER(css_opts), P]),
    "css_embed": (I32, [P, I32, I64, I64, I64, P, I32, P, I64, P, I64, P, SZ, C.POINTER(css_opts), P]),
    "css_lowrank": (I32, [P, I64, P, I64, I64, I64, I32, I32, P, P, I64, P, I64, P, P, P, SZ,
                          C.POINTER(css_opts), P]),
    "css_residual_backward": (I32, [P, I32, I64, I64, I64, P, I32, DBL, P, I64, P, P, SZ,
                                    C.POINTER(css_opts), P]),
    "css_select_host": (I32, [P, I32, I64, I64, I64, I32, P, P, P, P, P, SZ,
                              C.POINTER(css_opts), P]),
    "css_read_status": (I32, [P, P]),
    "css_select_noalloc": (I32, [P, I32, I64, I64, I64, I32, P, P, P, P, C.POINTER(css_opts), P]),
}

CSS_NOALLOC_SCRATCH_BYTES = 32 * 1024 * 1024

# every symbol include/css.h declares
EXPORTED = tuple(_SIGS)

_lib = None


class CssError(RuntimeError):
    def __init__(self, code, where=""):
        self.code = code
        super().__init__(f"{where}: {status_string(code)} ({code})")


def load(path: str | None = None):
    """Load libcss.so (once).  Raises if the library has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(
            f"libcss.so not found at {p}; build it with "
            "`python -m paper_1312_6838_gb300.build` (needs nvcc). There is no CPU fallback.")
    lib = C.CDLL(p)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def status_string(code: int) -> str:
    try:
        return load().css_status_string(int(code)).decode()
    except Exception:  # library missing
        return f"css_status {code}"


def default_opts() -> css_opts:
    o = css_opts()
    load().css_opts_default(C.byref(o))
    return o
