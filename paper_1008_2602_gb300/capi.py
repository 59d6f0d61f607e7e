"""ctypes binding of libfdtd.so: the C-ABI of ``include/fdtd.h``, same names.

Argument marshalling only: every step of the solver runs in the CUDA kernels
of ``csrc/``.  Importing this module loads (building first if needed) the
in-tree ``_build/libfdtd.so``; if it cannot be built or loaded the import
fails loudly -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import re

from . import build as _build

c_int, c_double, c_void_p, c_longlong = ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_longlong

FDTD_OK, FDTD_EINVAL, FDTD_ENOMEM, FDTD_ECUDA, FDTD_EUNSTABLE, FDTD_ETIMEOUT, FDTD_ESTATE = 0, -1, -2, -3, -4, -5, -6
FDTD_FP32, FDTD_FP16_STORE = 0, 1
FDTD_WALL_PEC, FDTD_WALL_PMC = 0, 1
FDTD_X, FDTD_Y, FDTD_Z = 0, 1, 2
FDTD_EX, FDTD_EY, FDTD_EZ, FDTD_HX, FDTD_HY, FDTD_HZ = range(6)


class fdtd_grid(ctypes.Structure):
    _fields_ = [("nx", c_int), ("ny", c_int), ("nz", c_int), ("dx", c_double), ("dy", c_double),
                ("dz", c_double), ("courant", c_double), ("dt", c_double)]


class fdtd_boundary(ctypes.Structure):
    _fields_ = [("depth", c_int * 6), ("m", c_double), ("R0", c_double), ("kappa_max", c_double),
                ("wall", c_int * 6)]


class fdtd_box(ctypes.Structure):
    _fields_ = [("i0", c_int), ("i1", c_int), ("j0", c_int), ("j1", c_int), ("k0", c_int), ("k1", c_int)]


class fdtd_info_t(ctypes.Structure):
    _fields_ = [("nx", c_int), ("ny", c_int), ("nz", c_int), ("dt", c_double), ("step", c_longlong),
                ("n_sources", c_int), ("n_probes", c_int), ("n_total_steps", c_int), ("n_bins", c_int),
                ("precision", c_int), ("interior_nodes", c_longlong), ("fused_upml_nodes", c_longlong),
                ("slab_nodes", c_longlong),
                ("device_bytes", c_longlong), ("n_combo", c_int), ("slab_aux_values", c_longlong),
                ("pitch", c_int), ("depth", c_int)]


class fdtd_tuning(ctypes.Structure):
    _fields_ = [("tile_x", c_int), ("tile_y", c_int), ("zseg", c_int), ("graph_chunk", c_int),
                ("depth", c_int), ("pair_zseg", c_int)]


class FdtdError(RuntimeError):
    def __init__(self, code: int, func: str, msg: str):
        super().__init__(f"{func} failed: {msg or 'error'} (status {code})")
        self.code = code


P = ctypes.POINTER
_SIGS = {
    "fdtd_create": (c_int, [P(fdtd_grid), c_void_p, c_void_p, c_int, c_void_p, c_int, c_void_p, P(fdtd_boundary),
                            c_int, c_void_p, P(c_void_p)]),
    "fdtd_set_source": (c_int, [c_void_p, c_int, c_int, c_int, c_int, c_double, c_double, c_double, P(c_int)]),
    "fdtd_set_voltage_source": (c_int, [c_void_p, c_int, c_int, c_int, c_int, c_double, c_double, c_double,
                                        c_double, P(c_int)]),
    "fdtd_add_probe": (c_int, [c_void_p, c_int, c_int, c_int, c_int, P(c_int)]),
    "fdtd_get_plane": (c_int, [c_void_p, c_int, c_int, c_void_p]),
    "fdtd_set_spectrum": (c_int, [c_void_p, c_double, c_int]),
    "fdtd_step": (c_int, [c_void_p, c_int]),
    "fdtd_step_profiled": (c_int, [c_void_p, c_int, P(c_double)]),
    "fdtd_probe_spectra": (c_int, [c_void_p, c_void_p, c_int, P(c_int)]),
    "fdtd_probe_trace": (c_int, [c_void_p, c_int, c_void_p, c_int, P(c_int)]),
    "fdtd_get_field": (c_int, [c_void_p, c_int, c_void_p]),
    "fdtd_diagnostics": (c_int, [c_void_p, P(c_double), P(c_double)]),
    "fdtd_reset": (c_int, [c_void_p]),
    "fdtd_set_materials": (c_int, [c_void_p, c_void_p]),
    "fdtd_node_coefficients": (c_int, [P(fdtd_grid), c_void_p, c_void_p, c_int, c_void_p, c_int, c_void_p,
                                       P(fdtd_boundary), c_void_p, c_void_p, c_int, P(c_int)]),
    "fdtd_info": (c_int, [c_void_p, P(fdtd_info_t)]),
    "fdtd_device_bytes": (c_int, [P(fdtd_grid), P(fdtd_boundary), c_int, c_int, c_int, c_int, c_double,
                                  P(c_longlong)]),
    "fdtd_save": (c_int, [c_void_p, c_void_p, ctypes.c_size_t, P(ctypes.c_size_t)]),
    "fdtd_selftest_wait_timeout": (c_int, [c_void_p, ctypes.c_uint]),
    "fdtd_load": (c_int, [c_void_p, c_void_p, ctypes.c_size_t]),
    "fdtd_sync": (c_int, [c_void_p]),
    "fdtd_destroy": (None, [c_void_p]),
    "fdtd_strerror": (ctypes.c_char_p, [c_int]),
    "fdtd_last_error": (ctypes.c_char_p, []),
    "fdtd_energy_static": (c_int, [P(c_void_p), P(c_void_p), c_int, c_int, c_int, c_int, c_double, c_double,
                                   c_double, P(c_int), c_void_p, P(c_double), P(c_double)]),
    "fdtd_batch_create": (c_int, [c_void_p, P(c_void_p)]),
    "fdtd_batch_add": (c_int, [c_void_p, c_void_p, c_int]),
    "fdtd_batch_remove": (c_int, [c_void_p, c_void_p]),
    "fdtd_batch_step": (c_int, [c_void_p, c_int, P(c_int)]),
    "fdtd_batch_remaining": (c_int, [c_void_p, c_void_p, P(c_longlong)]),
    "fdtd_batch_sync": (c_int, [c_void_p]),
    "fdtd_batch_destroy": (None, [c_void_p]),
    "fdtd_set_tuning": (c_int, [c_void_p, P(fdtd_tuning)]),
    "fdtd_halo_pack": (c_int, [c_void_p, c_int, c_int, ctypes.c_uint, c_void_p]),
    "fdtd_halo_unpack": (c_int, [c_void_p, c_int, c_int, ctypes.c_uint, c_void_p]),
    "fdtd_halo_copy": (c_int, [c_void_p, c_int, c_void_p, c_int, c_int, ctypes.c_uint]),
    "fdtd_batch_set_tuning": (c_int, [c_void_p, P(fdtd_tuning)]),
}

LIB_PATH = _build.build()
lib = ctypes.CDLL(LIB_PATH)
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(lib, _name)
    _f.restype = _res
    _f.argtypes = _args


def header_functions() -> list:
    """Names of every function declared in include/fdtd.h."""
    hdr = os.path.join(_build.ROOT, "include", "fdtd.h")
    text = open(hdr).read()
    return sorted(set(re.findall(r"^\s*(?:int|void|const char \*)\s*(fdtd_\w+)\s*\(", text, re.M)))


def _check(func: str, code: int) -> int:
    if code != FDTD_OK:
        msg = lib.fdtd_last_error()
        raise FdtdError(code, func, msg.decode() if msg else lib.fdtd_strerror(code).decode())
    return code


def _wrap(name):
    f = getattr(lib, name)
    if f.restype is c_int:
        def call(*args):
            return _check(name, f(*args))
    else:
        def call(*args):
            return f(*args)
    call.__name__ = name
    call.__doc__ = f"ctypes call of {name} (include/fdtd.h); raises FdtdError on a non-zero status."
    return call


for _name in _SIGS:
    globals()[_name] = _wrap(_name)

__all__ = list(_SIGS) + ["fdtd_grid", "fdtd_boundary", "fdtd_box", "fdtd_info_t", "fdtd_tuning", "FdtdError",
                         "lib", "LIB_PATH", "header_functions"]
