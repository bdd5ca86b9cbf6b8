"""ctypes declarations of the C ABI in include/hacc_sr.h.

Only argument marshalling lives here.  The shared library is built in-tree by
``_build.build()``; if it is missing or cannot be loaded, every call raises.
"""

from __future__ import annotations

import ctypes
import os
import threading

from . import _build

HACC_OK = 0
HACC_ERR_INVALID = -1
HACC_ERR_CAPACITY = -2
HACC_ERR_CUDA = -3
HACC_ERR_TIMEOUT = -4
HACC_STATUS_CAPACITY = 1
HACC_STATUS_TIMEOUT = 2
HACC_STATUS_NONFINITE = 4
HACC_STATUS_SKIN = 8
HACC_STATUS_BOUNDS = 16

_ERRNAMES = {HACC_ERR_INVALID: "invalid argument", HACC_ERR_CAPACITY: "buffer or workspace too small",
             HACC_ERR_CUDA: "CUDA error", HACC_ERR_TIMEOUT: "timeout"}


class HaccError(RuntimeError):
    pass


class hacc_volume(ctypes.Structure):
    _fields_ = [("p_begin", ctypes.c_int64), ("p_end", ctypes.c_int64), ("cell_base", ctypes.c_int64),
                ("entry_base", ctypes.c_int64), ("n", ctypes.c_int32), ("R", ctypes.c_int32),
                ("S", ctypes.c_int32), ("L", ctypes.c_float), ("w", ctypes.c_float),
                ("inv_w", ctypes.c_float), ("rcut", ctypes.c_float), ("pad", ctypes.c_int32)]


class hacc_mesh(ctypes.Structure):
    _fields_ = [("vols", ctypes.c_void_p), ("V", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("N", ctypes.c_int64), ("n_cells", ctypes.c_int64), ("n_entries", ctypes.c_int64)]


class hacc_binned(ctypes.Structure):
    _fields_ = [("cell_of", ctypes.c_void_p), ("cell_start", ctypes.c_void_p), ("perm", ctypes.c_void_p),
                ("sorted4", ctypes.c_void_p), ("cell_origin", ctypes.c_void_p), ("mass_varies", ctypes.c_void_p)]


class hacc_lists(ctypes.Structure):
    _fields_ = [("nbr_off", ctypes.c_void_p), ("nbr_cell", ctypes.c_void_p), ("nbr_shift", ctypes.c_void_p),
                ("tasks", ctypes.c_void_p), ("n_tasks", ctypes.c_void_p), ("n_pairs", ctypes.c_void_p),
                ("task_order", ctypes.c_void_p), ("task_cap", ctypes.c_int64), ("split_T", ctypes.c_int32), ("pad", ctypes.c_int32)]


class hacc_tree(ctypes.Structure):
    _fields_ = [("leaf_max", ctypes.c_int32), ("max_depth", ctypes.c_int32), ("leaf_cap", ctypes.c_int64),
                ("n_leaves", ctypes.c_void_p), ("n_nodes", ctypes.c_void_p), ("leaf_start", ctypes.c_void_p),
                ("leaf_qbox", ctypes.c_void_p), ("leaf_origin", ctypes.c_void_p), ("node_qbox", ctypes.c_void_p),
                ("node_child", ctypes.c_void_p), ("root", ctypes.c_void_p)]


class hacc_sr_params(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_float), ("rcut", ctypes.c_float), ("c", ctypes.c_float * 6)]


class hacc_launch(ctypes.Structure):
    _fields_ = [("warps_per_cta", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("jtile", ctypes.c_int32), ("stages", ctypes.c_int32), ("wait_cycles", ctypes.c_int64)]


assert ctypes.sizeof(hacc_volume) == 64
assert ctypes.sizeof(hacc_mesh) == 40
assert ctypes.sizeof(hacc_launch) == 24

_P = ctypes.c_void_p
_PS = ctypes.POINTER
# name -> (restype, argtypes); the order of the header
SIGNATURES = {
    "hacc_version": (ctypes.c_char_p, []),
    "hacc_get_status": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_uint32), _P]),
    "hacc_kernel_launches": (ctypes.c_uint64, []),
    "hacc_mesh_plan": (ctypes.c_int, [ctypes.c_int32, _P, _P, ctypes.c_float, ctypes.c_float,
                                      _PS(hacc_volume), _PS(hacc_mesh)]),
    "hacc_bin_workspace_size": (ctypes.c_size_t, [_PS(hacc_mesh)]),
    "hacc_bin": (ctypes.c_int, [_PS(hacc_mesh), _P, _P, _P, _P, _P, _P, _P, _PS(hacc_binned), _P, ctypes.c_size_t,
                                _P, _P]),
    "hacc_bin_noalloc": (ctypes.c_int, [_PS(hacc_mesh), _P, _P, _P, _P, _PS(hacc_binned), _P, _P]),
    "hacc_task_capacity": (ctypes.c_int64, [_PS(hacc_mesh), ctypes.c_int32]),
    "hacc_lists_workspace_size": (ctypes.c_size_t, [_PS(hacc_mesh)]),
    "hacc_build_lists": (ctypes.c_int, [_PS(hacc_mesh), _PS(hacc_binned), _PS(hacc_lists), _P, ctypes.c_size_t,
                                        _P, _P]),
    "hacc_rcb_build_workspace_size": (ctypes.c_size_t, [_PS(hacc_mesh), ctypes.c_int32]),
    "hacc_rcb_build": (ctypes.c_int, [_PS(hacc_mesh), _P, _P, _P, _P, _PS(hacc_tree), _PS(hacc_binned), _P,
                                      ctypes.c_size_t, _P, _P]),
    "hacc_rcb_lists_workspace_size": (ctypes.c_size_t, [_PS(hacc_mesh), ctypes.c_int64, ctypes.c_int64]),
    "hacc_rcb_lists": (ctypes.c_int, [_PS(hacc_mesh), _PS(hacc_tree), _PS(hacc_lists), ctypes.c_int64, _P, _P,
                                      ctypes.c_size_t, _P, _P]),
    "hacc_force_workspace_size": (ctypes.c_size_t, [_PS(hacc_mesh)]),
    "hacc_sr_force": (ctypes.c_int, [_PS(hacc_mesh), _PS(hacc_binned), _PS(hacc_lists), _PS(hacc_sr_params),
                                     _P, _P, _P, _PS(hacc_launch), _P, ctypes.c_size_t, _P, _P]),
    "hacc_sr_force_symmetric": (ctypes.c_int, [_PS(hacc_mesh), _PS(hacc_binned), _PS(hacc_lists),
                                               _PS(hacc_sr_params), _P, _P, _P, _PS(hacc_launch), _P,
                                               ctypes.c_size_t, _P, _P]),
    "hacc_sr_force_adjoint_symmetric": (ctypes.c_int, [_PS(hacc_mesh), _PS(hacc_binned), _PS(hacc_lists),
                                                       _PS(hacc_sr_params), _P, _P, _P, _P, _P, _P, _P,
                                                       _PS(hacc_launch), _P, ctypes.c_size_t, _P, _P]),
    "hacc_sr_force_adjoint": (ctypes.c_int, [_PS(hacc_mesh), _PS(hacc_binned), _PS(hacc_lists),
                                             _PS(hacc_sr_params), _P, _P, _P, _P, _P, _P, _P, _PS(hacc_launch),
                                             _P, ctypes.c_size_t, _P, _P]),
    "hacc_count_pairs": (ctypes.c_int, [_PS(hacc_mesh), _PS(hacc_binned), _PS(hacc_lists), _PS(hacc_sr_params),
                                        _P, _P]),
    "hacc_kick": (ctypes.c_int, [_PS(hacc_mesh), ctypes.c_int64, _P, _P, _P, _P, _P, _P, ctypes.c_float,
                                 _P, _P, _P, ctypes.c_float, _P]),
    "hacc_drift_offsets": (ctypes.c_int, [_PS(hacc_mesh), _PS(hacc_binned), _P, _P, _P, ctypes.c_float,
                                          ctypes.c_float, _P, _P]),
    "hacc_moments_workspace_size": (ctypes.c_size_t, [ctypes.c_int64]),
    "hacc_moments": (ctypes.c_int, [ctypes.c_int64, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, ctypes.c_size_t, _P]),
    "hacc_sr_potential": (ctypes.c_int, [_PS(hacc_mesh), _PS(hacc_binned), _PS(hacc_lists), _PS(hacc_sr_params),
                                         _P, _PS(hacc_launch), _P, ctypes.c_size_t, _P, _P]),
}

_lock = threading.Lock()
_lib = None


def _open(path: str):
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


def load(build_if_missing: bool = True):
    """Load libhacc_sr.so (building it first if needed); raises if impossible."""
    global _lib
    with _lock:
        if _lib is None:
            if build_if_missing and not _build.up_to_date():
                _build.build(variants=("release",))
            if not os.path.exists(_build.LIB):
                raise HaccError(f"CUDA library missing: {_build.LIB} (run __graft_entry__.build())")
            _lib = _open(_build.LIB)
    return _lib


def use_library(debug: bool):
    """Route every later call through the debug build (bounds-checked pair
    kernels, libhacc_sr_debug.so) or back to the product build; returns the
    previously active library handle.  Device buffers are shared: both
    libraries run in the process's one CUDA context."""
    global _lib
    prev = load()
    path = _build.LIB_DEBUG if debug else _build.LIB
    if debug and not _build.up_to_date("debug"):
        _build.build(variants=("debug",))
    with _lock:
        _lib = _open(path)
    return prev


def check(rc: int, what: str) -> None:
    if rc != HACC_OK:
        raise HaccError(f"{what} failed: {rc} ({_ERRNAMES.get(rc, 'unknown')})")


def library_path() -> str:
    return _build.LIB
