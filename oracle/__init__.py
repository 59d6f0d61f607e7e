"""FP64 CPU FDTD oracle -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its
``cpu_baseline`` leg and ``--impl reference``) may import this package.  The
CUDA library never calls it; the two share no code, only the seeded
``Problem`` description from ``paper_1008_2602_gb300.workloads``.

``run(problem)`` executes ``oracle_run`` from ``fdtd_oracle.c`` (plain C,
FP64, full 3D D/B arrays everywhere, the paper's unified UPML treatment).
``cavity_fr`` is Eq. 9, ``cfl_dt`` is Eq. 7 with v = c, ``pulse`` is Eq. 8.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fdtd_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_libs = {}


class _Problem(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double),
        ("courant", ctypes.c_double), ("dt", ctypes.c_double),
        ("mat", ctypes.c_void_p), ("eps_r", ctypes.c_void_p), ("n_mat", ctypes.c_int),
        ("pec_boxes", ctypes.c_void_p), ("n_pec", ctypes.c_int),
        ("upml_depth", ctypes.c_int * 6),
        ("upml_m", ctypes.c_double), ("upml_R0", ctypes.c_double), ("upml_kappa_max", ctypes.c_double),
        ("walls", ctypes.c_int * 6),
        ("src", ctypes.c_void_p), ("src_prm", ctypes.c_void_p), ("n_src", ctypes.c_int),
        ("probe", ctypes.c_void_p), ("n_probe", ctypes.c_int),
        ("n_steps", ctypes.c_int), ("n_bins", ctypes.c_int), ("n_threads", ctypes.c_int),
        ("vsrc", ctypes.c_void_p), ("vsrc_prm", ctypes.c_void_p), ("n_vsrc", ctypes.c_int),
    ]


class _Outputs(ctypes.Structure):
    _fields_ = [
        ("dt", ctypes.c_double),
        ("trace", ctypes.c_void_p), ("dft", ctypes.c_void_p), ("energy", ctypes.c_void_p),
        ("divb", ctypes.c_void_p), ("src_wave", ctypes.c_void_p), ("fields", ctypes.c_void_p),
        ("vsrc_current", ctypes.c_void_p),
    ]


def build(force: bool = False) -> str:
    """Compile ``fdtd_oracle.c`` into ``oracle/_build/liboracle.so`` (gcc -O2, OpenMP)."""
    with _lock:
        if (not force and os.path.exists(_LIB_PATH)
                and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
            return _LIB_PATH
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def _load(lib_path: Optional[str] = None):
    """The oracle library (or, for the tests that plant a mistake in a copy of
    the oracle, the library built from that copy at ``lib_path``)."""
    path = lib_path or build()
    if path not in _libs:
        lib = ctypes.CDLL(path)
        lib.oracle_run.argtypes = [ctypes.POINTER(_Problem), ctypes.POINTER(_Outputs)]
        lib.oracle_run.restype = ctypes.c_int
        for name in ("oracle_cfl_dt",):
            getattr(lib, name).argtypes = [ctypes.c_double] * 3
            getattr(lib, name).restype = ctypes.c_double
        lib.oracle_cavity_fr.argtypes = [ctypes.c_int, ctypes.c_int] + [ctypes.c_double] * 4
        lib.oracle_cavity_fr.restype = ctypes.c_double
        lib.oracle_pulse.argtypes = [ctypes.c_double] * 4
        lib.oracle_pulse.restype = ctypes.c_double
        _libs[path] = lib
    return _libs[path]


def cavity_fr(m: int, n: int, Lx: float, Ly: float, Lz: float, eps_r: float) -> float:
    """Eq. 9 (fringing term L_z/2 included; pass Lz=0 for an ideal walled cavity)."""
    return _load().oracle_cavity_fr(m, n, Lx, Ly, Lz, eps_r)


def cfl_dt(dx: float, dy: float, dz: float) -> float:
    """Eq. 7 with v = c."""
    return _load().oracle_cfl_dt(dx, dy, dz)


def pulse(J0: float, t0: float, tau: float, t: float) -> float:
    """Eq. 8 with the square restored in the exponent."""
    return _load().oracle_pulse(J0, t0, tau, t)


def n_bins(prob, dt: float) -> int:
    """Number of DFT bins f_q = q / (N dt) with f_q <= f_max (all to Nyquist if None)."""
    N = prob.n_steps
    if prob.f_max is None:
        return N // 2 + 1
    return min(N // 2 + 1, int(np.floor(prob.f_max * N * dt + 1e-9)) + 1)


def run(prob, *, trace: bool = True, dft: bool = True, energy: bool = False, divb: bool = False,
        src_wave: bool = False, fields: bool = False, vsrc_current: bool = False,
        n_threads: Optional[int] = None, n_steps: Optional[int] = None,
        lib_path: Optional[str] = None) -> dict:
    """Run the oracle on a ``workloads.Problem``; returns a dict of numpy arrays."""
    lib = _load(lib_path)
    N = int(n_steps if n_steps is not None else prob.n_steps)
    mat = np.ascontiguousarray(prob.mat, dtype=np.uint8)
    eps = np.ascontiguousarray(prob.eps_r, dtype=np.float64)
    boxes = np.ascontiguousarray(prob.pec_boxes, dtype=np.int32).reshape(-1, 6)
    src = np.ascontiguousarray(prob.sources, dtype=np.int32).reshape(-1, 4)
    prm = np.ascontiguousarray(prob.source_params, dtype=np.float64).reshape(-1, 3)
    prb = np.ascontiguousarray(prob.probes, dtype=np.int32).reshape(-1, 4)
    assert mat.shape == (prob.nz, prob.ny, prob.nx)
    assert len(src) == len(prm)
    P = _Problem()
    P.nx, P.ny, P.nz = prob.nx, prob.ny, prob.nz
    P.dx, P.dy, P.dz = prob.dx, prob.dy, prob.dz
    P.courant, P.dt = prob.courant, prob.dt
    P.mat, P.eps_r, P.n_mat = mat.ctypes.data, eps.ctypes.data, len(eps)
    P.pec_boxes, P.n_pec = boxes.ctypes.data, len(boxes)
    P.upml_depth[:] = list(prob.upml_depth)
    P.upml_m, P.upml_R0, P.upml_kappa_max = prob.upml_m, prob.upml_R0, prob.upml_kappa_max
    P.walls[:] = list(prob.walls)
    P.src, P.src_prm, P.n_src = src.ctypes.data, prm.ctypes.data, len(src)
    P.probe, P.n_probe = prb.ctypes.data, len(prb)
    vs = np.ascontiguousarray(getattr(prob, "vsources", np.zeros((0, 4))), dtype=np.int32).reshape(-1, 4)
    vp = np.ascontiguousarray(getattr(prob, "vsource_params", np.zeros((0, 4))), dtype=np.float64).reshape(-1, 4)
    assert len(vs) == len(vp)
    P.vsrc, P.vsrc_prm, P.n_vsrc = vs.ctypes.data, vp.ctypes.data, len(vs)
    P.n_steps = N
    dt = prob.dt if prob.dt > 0 else prob.courant * cfl_dt(prob.dx, prob.dy, prob.dz)
    Q = n_bins(prob.replace(n_steps=N), dt) if dft else 0
    P.n_bins = Q
    P.n_threads = int(n_threads if n_threads is not None else 1)
    out = {}
    O = _Outputs()
    bufs = {
        "trace": (trace, (len(prb), N)), "dft": (dft, (len(prb), Q, 2)),
        "energy": (energy, (N,)), "divb": (divb, (N,)), "src_wave": (src_wave, (N,)),
        "fields": (fields, (6, prob.nz + 1, prob.ny + 1, prob.nx + 1)),
        "vsrc_current": (vsrc_current, (N,)),
    }
    for name, (want, shape) in bufs.items():
        if want:
            a = np.zeros(shape, dtype=np.float64)
            out[name] = a
            setattr(O, name, a.ctypes.data)
        else:
            setattr(O, name, None)
    rc = lib.oracle_run(ctypes.byref(P), ctypes.byref(O))
    if rc != 0:
        raise RuntimeError(f"oracle_run failed with code {rc}")
    out["dt"] = O.dt
    if "dft" in out:
        out["spectra"] = out["dft"][..., 0] + 1j * out["dft"][..., 1]
        out["freqs"] = np.arange(Q) / (N * O.dt)
    return out
