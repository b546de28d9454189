"""ctypes binding of libmuca.so: argument marshalling only, names as in include/muca.h.

Every compute step runs in the CUDA library; if the library cannot be loaded the
import fails loudly (there is no CPU fallback).
"""
from __future__ import annotations

import ctypes
import os

from . import _build

_lib = None

c_int, c_i64, c_u64, c_dbl, c_vp, c_sz = (ctypes.c_int, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double,
                                          ctypes.c_void_p, ctypes.c_size_t)
P = ctypes.POINTER

# name -> (restype, argtypes)
PROTOTYPES = {
    "muca_last_error": (ctypes.c_char_p, []),
    "muca_init": (c_int, [P(c_vp), c_int, c_int, c_int, c_int, c_u64]),
    "muca_workspace_size": (c_int, [c_int, c_int, c_int, c_int, P(c_sz)]),
    "muca_init_ex": (c_int, [P(c_vp), c_int, c_int, c_int, c_int, c_u64, c_vp, c_sz]),
    "muca_set_param": (c_int, [c_vp, ctypes.c_char_p, c_dbl]),
    "muca_set_stream": (c_int, [c_vp, c_vp]),
    "muca_iterate": (c_int, [c_vp, c_i64]),
    "muca_merge_and_update": (c_int, [c_vp, P(c_int)]),
    "muca_num_bins": (c_int, [c_vp, P(c_int)]),
    "muca_set_lnW": (c_int, [c_vp, c_vp, c_int]),
    "muca_poly_trace": (c_int, [c_vp, c_vp, c_i64]),
    "muca_get_lnW": (c_int, [c_vp, c_vp, c_int]),
    "muca_get_lnW_sampled": (c_int, [c_vp, c_vp, c_int]),
    "muca_get_histogram": (c_int, [c_vp, c_vp, c_int]),
    "muca_get_flatness": (c_int, [c_vp, c_vp]),
    "muca_get_reweight": (c_int, [c_vp, c_dbl, c_vp, c_vp]),
    "muca_get_observables": (c_int, [c_vp, c_dbl, c_vp, c_vp, c_int]),
    "muca_get_metrics": (c_int, [c_vp, c_vp]),
    "muca_merge_open": (c_int, [c_vp, c_vp]),
    "muca_update_with": (c_int, [c_vp, c_vp, c_vp]),
    "muca_get_state": (c_int, [c_vp, c_vp, P(c_sz)]),
    "muca_set_state": (c_int, [c_vp, c_vp, c_sz]),
    "muca_get_spins": (c_int, [c_vp, c_vp, c_i64]),
    "muca_get_walker_bins": (c_int, [c_vp, c_vp, c_int]),
    "muca_get_thresholds": (c_int, [c_vp, c_vp, c_i64]),
    "muca_get_sweep_counter": (c_int, [c_vp, P(c_i64)]),
    "muca_get_coords": (c_int, [c_vp, c_vp, c_i64, c_vp, c_int]),
    "muca_get_drift": (c_int, [c_vp, P(c_dbl)]),
    "muca_det_math": (c_int, [c_int, c_vp, c_vp, c_i64]),
    "muca_iterate_noalloc": (c_int, [c_vp, c_i64, c_vp]),
    "muca_batch_create": (c_int, [P(c_vp), c_int, P(c_vp)]),
    "muca_batch_run": (c_int, [c_vp, c_int, c_i64, c_int]),
    "muca_batch_free": (c_int, [c_vp]),
    "muca_batch_set_form": (c_int, [c_vp, c_int]),
    "muca_batch_set_sweeps": (c_int, [c_vp, c_vp, c_int]),
    "muca_synchronize": (c_int, [c_vp]),
    "muca_free": (c_int, [c_vp]),
}


def checked() -> bool:
    """MUCA_DEBUG=1 selects the checked build (bounds checks on the sweeps' table accesses)."""
    return os.environ.get("MUCA_DEBUG", "") == "1"


def library_path() -> str:
    return _build.LIB_CHECKED if checked() else _build.LIB


def load(build_if_missing: bool = True):
    """Load libmuca.so, or libmuca_checked.so under MUCA_DEBUG=1 (building it first if it is
    missing or stale)."""
    global _lib
    if _lib is None:
        path = library_path()
        if build_if_missing:
            _build.build(checked=checked())
        if not os.path.exists(path):
            raise ImportError("%s is not built; run __graft_entry__.build()" % os.path.basename(path))
        lib = ctypes.CDLL(path)
        for name, (res, args) in PROTOTYPES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


class MucaError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__("%s failed (%d): %s" % (where, code, msg))
        self.code = code


def check(rc: int, where: str):
    if rc != 0:
        raise MucaError(rc, where, (load().muca_last_error() or b"").decode(errors="replace"))
