"""ctypes binding of libgs (include/gs.h): argument marshalling only.

Every computation happens in the CUDA library; this module turns tensors or
numpy arrays into pointers and status codes into exceptions.  There is no
CPU fallback: if libgs.so is missing or no GPU is present, calls raise.
"""
from __future__ import annotations

import ctypes
import os
import re

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libgs.so")
HEADER = os.path.join(os.path.dirname(PKG), "include", "gs.h")

GS_OK, GS_ERR_INVALID_ARG, GS_ERR_CUDA, GS_ERR_OOM, GS_ERR_NONFINITE, GS_ERR_TIMEOUT, \
    GS_ERR_UNSUPPORTED = range(7)
STATUS_NAMES = {0: "GS_OK", 1: "GS_ERR_INVALID_ARG", 2: "GS_ERR_CUDA", 3: "GS_ERR_OOM",
                4: "GS_ERR_NONFINITE", 5: "GS_ERR_TIMEOUT", 6: "GS_ERR_UNSUPPORTED"}
GS_EXACT, GS_BH, GS_TRUNC = 0, 1, 2
RHS_NOALLOC_MAX_N = 16384  # GS_RHS_NOALLOC_MAX_N in include/gs.h
KERNEL_CLASSES = ("exact_fwd", "exact_adj", "tree_build", "bh_fwd", "bh_adj", "bh_walk")


class GSError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [("sigma", ctypes.c_double), ("lambda_", ctypes.c_double),
                ("thresh_sigmas", ctypes.c_double), ("T", ctypes.c_int32),
                ("mode", ctypes.c_int32), ("ckpt_every", ctypes.c_int32),
                ("flags", ctypes.c_uint32), ("leaf_size", ctypes.c_int32),
                ("criterion", ctypes.c_int32), ("sympl_iters", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


def make_params(sigma, T, mode=GS_EXACT, lam=1.0, thresh=3.0, ckpt_every=0, flags=0,
                leaf_size=1, criterion=0, sympl_iters=0) -> Params:
    if isinstance(mode, str):
        mode = {"exact": GS_EXACT, "bh": GS_BH, "trunc": GS_TRUNC}[mode.lower()]
    return Params(float(sigma), float(lam), float(thresh), int(T), int(mode), int(ckpt_every),
                  int(flags), int(leaf_size), int(criterion), int(sympl_iters), 0)


_lib = None
_vp, _i64, _i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
_SIGS = {
    "gs_create": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]),
    "gs_destroy": (None, [_vp]),
    "gs_last_error": (ctypes.c_char_p, [_vp]),
    "gs_sync": (ctypes.c_int, [_vp, _vp]),
    "gs_selftest_timeout": (ctypes.c_int, [_vp, _vp]),
    "gs_shoot": (ctypes.c_int, [_vp, _vp, _vp, _i64, ctypes.POINTER(Params), _vp, _vp, _vp, _vp]),
    "gs_shoot_grad": (ctypes.c_int, [_vp, _vp, _vp, _vp, _i64, ctypes.POINTER(Params), _vp, _vp,
                                     _vp, _vp]),
    "gs_shoot_batched": (ctypes.c_int, [_vp, _i32, _vp, _vp, _vp, _vp, ctypes.POINTER(Params),
                                        _vp, _vp, _vp]),
    "gs_descend_batched": (ctypes.c_int, [_vp, _i32, _vp, _vp, _vp, _vp, ctypes.POINTER(Params),
                                          ctypes.c_double, _i32, _vp, _vp]),
    "gs_lbfgs": (ctypes.c_int, [_vp, _vp, _vp, _vp, _i64, ctypes.POINTER(Params), _i32, _i32,
                                ctypes.c_double, _vp, _vp, _vp]),
    "gs_autotune": (ctypes.c_int, [_vp, _vp, _vp, _i64, ctypes.POINTER(Params), _vp, _i32, _vp,
                                   _vp, _vp]),
    "gs_autotune_exact": (ctypes.c_int, [_vp, _vp, _vp, _i64, ctypes.POINTER(Params), _vp, _i32,
                                         _vp, _vp, _vp]),
    "gs_flow": (ctypes.c_int, [_vp, _vp, _vp, _i64, _vp, _i64, ctypes.POINTER(Params), _vp, _vp,
                               _vp, _vp]),
    "gs_velocity": (ctypes.c_int, [_vp, _vp, _vp, _i64, _vp, _i64, ctypes.POINTER(Params), _vp,
                                   _vp]),
    "gs_rhs": (ctypes.c_int, [_vp, _vp, _vp, _i64, ctypes.POINTER(Params), _vp, _vp, _vp, _vp]),
    "gs_adj_rhs": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _i64, ctypes.POINTER(Params), _vp,
                                  _vp, _vp, _vp]),
    "gs_tree": (ctypes.c_int, [_vp, _vp, _i64, _vp, _vp, _vp, _vp, _i64, _vp, _vp]),
    "gs_alu_peaks": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
    "gs_timing": (ctypes.c_int, [_vp, ctypes.c_int]),
    "gs_set_option": (ctypes.c_int, [_vp, ctypes.c_char_p, _i64]),
    "gs_rhs_exact_noalloc": (ctypes.c_int, [_vp, _vp, _i64, ctypes.c_double, _vp, _vp, _vp]),
    "gs_timing_read": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "gs_shoot_traj": (ctypes.c_int, [_vp, _vp, _vp, _i64, ctypes.POINTER(Params), _vp, _vp, _vp]),
    "gs_bh_tally": (ctypes.c_int, [_vp, _vp, _i64, ctypes.POINTER(Params), _vp, _vp, _vp]),
    "gs_tree_sums": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _i64, _vp, _i64, _vp, _vp]),
}


def declared_symbols() -> list[str]:
    """Entry points declared in include/gs.h."""
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:gs_status|void|const char \*)\s*\*?\s*(gs_\w+)\s*\(",
                                 text, flags=re.M)))


def load():
    """Loads libgs.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libgs.so not built ({LIB_PATH}); run __graft_entry__.build()")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in _SIGS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib
