"""ctypes declarations of the C-ABI in include/trsgd.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os
import re

from . import build as _build

MAX_ORDER = 8

OK, EINVAL, ENOMEM, ECUDA, ENUMERIC, ETIMEOUT, EUNSUPPORTED, EBADINDEX = range(8)
DIST_UNIFORM, DIST_LEVERAGE, DIST_EUCLIDEAN, DIST_OPTIMAL = range(4)
PLAIN, SCALED = 0, 1
STEP_FIXED, STEP_ADAGRAD = 0, 1
FP64, FP32, BF16_MIXED = 0, 1, 2
DTYPE_F64, DTYPE_F32, DTYPE_BF16 = 0, 1, 2
PATH_AUTO, PATH_CLUSTER, PATH_GRID = 0, 1, 2
FP32_PIECES, FP32_FMA = 0, 1
DBG_MODE, DBG_IDX, DBG_PF, DBG_Z, DBG_E, DBG_G, DBG_P, DBG_H = range(8)


class Config(ctypes.Structure):
    _fields_ = [
        ("N", ctypes.c_int32),
        ("dist", ctypes.c_int32),
        ("I", ctypes.c_int64 * MAX_ORDER),
        ("R", ctypes.c_int64 * MAX_ORDER),
        ("J", ctypes.c_int64),
        ("J_H", ctypes.c_int64),
        ("variant", ctypes.c_int32),
        ("rule", ctypes.c_int32),
        ("prec", ctypes.c_int32),
        ("x_dtype", ctypes.c_int32),
        ("alpha", ctypes.c_double),
        ("eta", ctypes.c_double),
        ("b", ctypes.c_double),
        ("eps", ctypes.c_double),
        ("damping", ctypes.c_double),
        ("seed", ctypes.c_uint64),
        ("path", ctypes.c_int32),
        ("fp32_units", ctypes.c_int32),
    ]


class Shard(ctypes.Structure):
    _fields_ = [
        ("mode", ctypes.c_int32),
        ("j0", ctypes.c_int64), ("j1", ctypes.c_int64),
        ("h0", ctypes.c_int64), ("h1", ctypes.c_int64),
        ("gunit", ctypes.c_int64), ("hunit", ctypes.c_int64),
        ("gsplits", ctypes.c_int64), ("hsplits", ctypes.c_int64),
        ("gsplits_max", ctypes.c_int64), ("hsplits_max", ctypes.c_int64),
        ("gelems", ctypes.c_int64), ("helems", ctypes.c_int64),
    ]


class TrsgdError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {status_string(status)} (status {status})")


_lib = None

_SIGNATURES = {
    "trsgd_init": (ctypes.c_int, [ctypes.POINTER(Config), ctypes.c_int32, ctypes.POINTER(ctypes.c_void_p),
                                  ctypes.POINTER(ctypes.c_void_p), ctypes.c_void_p,
                                  ctypes.POINTER(ctypes.c_void_p)]),
    "trsgd_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64]),
    "trsgd_step_counter": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64]),
    "trsgd_set_counter": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64]),
    "trsgd_run": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                 ctypes.c_double, ctypes.c_double, ctypes.c_void_p,
                                 ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double)]),
    "trsgd_rel_error": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                       ctypes.POINTER(ctypes.c_double)]),
    "trsgd_rel_error_static": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(ctypes.c_int64),
                                              ctypes.POINTER(ctypes.c_int64), ctypes.c_int32,
                                              ctypes.POINTER(ctypes.c_void_p), ctypes.c_void_p, ctypes.c_void_p,
                                              ctypes.c_void_p]),
    "trsgd_reconstruct": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(ctypes.c_int64),
                                         ctypes.POINTER(ctypes.c_int64), ctypes.c_int32,
                                         ctypes.POINTER(ctypes.c_void_p), ctypes.c_void_p, ctypes.c_void_p]),
    "trsgd_sampled_loss_grad": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(ctypes.c_int64),
                                               ctypes.POINTER(ctypes.c_int64), ctypes.c_int32, ctypes.c_int64,
                                               ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                               ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p),
                                               ctypes.c_void_p, ctypes.c_void_p]),
    "trsgd_set_debug": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "trsgd_get_debug": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_size_t,
                                       ctypes.POINTER(ctypes.c_size_t)]),
    "trsgd_adagrad_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                           ctypes.c_size_t, ctypes.c_int32]),
    "trsgd_launch_shape": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                                          ctypes.POINTER(ctypes.c_int32)]),
    "trsgd_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "trsgd_launch_count": (ctypes.c_int64, [ctypes.c_void_p]),
    "trsgd_tensor_pieces": (ctypes.c_int32, [ctypes.c_void_p]),
    "trsgd_gd_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_double, ctypes.c_double]),
    "trsgd_shard_plan": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                        ctypes.POINTER(Shard)]),
    "trsgd_step_partial": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(Shard), ctypes.c_void_p,
                                          ctypes.c_void_p]),
    "trsgd_step_apply": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64,
                                        ctypes.c_void_p, ctypes.c_int64]),
    "trsgd_set_wait_limit": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64]),
    "trsgd_debug_index_bound": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64]),
    "trsgd_probe_peak": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p,
                                        ctypes.POINTER(ctypes.c_double)]),
    "trsgd_destroy": (None, [ctypes.c_void_p]),
    "trsgd_status_string": (ctypes.c_char_p, [ctypes.c_int]),
}


def header_symbols():
    """Function names declared in include/trsgd.h."""
    hdr = os.path.join(_build.ROOT, "include", "trsgd.h")
    text = open(hdr).read()
    return sorted(set(re.findall(r"\b(trsgd_[a-z_0-9]+)\s*\(", text)))


def library_path() -> str:
    """libtrsgd.so, or with TRSGD_DEBUG=1 in the environment the debug build
    (index checks compiled in)."""
    return _build.DEBUG_LIB if os.environ.get("TRSGD_DEBUG") == "1" else _build.LIB


def lib():
    """The loaded library; raises if it has not been built (there is no
    fallback)."""
    global _lib
    if _lib is None:
        path = library_path()
        if not os.path.exists(path):
            flag = " --debug" if path == _build.DEBUG_LIB else ""
            raise RuntimeError(f"{path} is missing: build the CUDA library first "
                               f"(python -m paper_2303_16492_gb300.build{flag})")
        L = ctypes.CDLL(path)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def status_string(s: int) -> str:
    return lib().trsgd_status_string(int(s)).decode()


def check(status: int, what: str):
    if status != OK:
        raise TrsgdError(status, what)
