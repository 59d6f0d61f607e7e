"""Solver / Batch: a convenience layer over the C-ABI binding (``capi``).

``Solver(problem)`` creates a board from a ``workloads.Problem`` (material
volume, eps_r table, PEC boxes, UPML, walls, sources, probes, spectrum) and
exposes ``step``, ``spectra``, ``traces``, ``field``, ``diagnostics``.
``Batch`` steps many solvers with one launch per phase.  All arithmetic runs
in libfdtd.so's CUDA kernels; this module only marshals arguments.
"""
from __future__ import annotations

import ctypes
from typing import Iterable, List, Optional

import numpy as np

from . import capi as C

PRECISION = {"fp32": C.FDTD_FP32, "fp16": C.FDTD_FP16_STORE}


def _stream_ptr(stream) -> Optional[int]:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)   # a torch.cuda.Stream


def problem_structs(prob):
    """The fdtd_grid and fdtd_boundary of a workloads.Problem."""
    g = C.fdtd_grid(prob.nx, prob.ny, prob.nz, prob.dx, prob.dy, prob.dz, prob.courant, prob.dt)
    b = C.fdtd_boundary()
    b.depth[:] = list(prob.upml_depth)
    b.m, b.R0, b.kappa_max = prob.upml_m, prob.upml_R0, prob.upml_kappa_max
    b.wall[:] = list(prob.walls)
    return g, b


def device_bytes(prob, precision: str = "fp32") -> int:
    """Device memory the board needs (fdtd_device_bytes, asked of the library
    on the host, without a device)."""
    g, b = problem_structs(prob)
    n_src = len(np.asarray(prob.sources).reshape(-1, 4)) + len(np.asarray(prob.vsources).reshape(-1, 4))
    n_prb = len(np.asarray(prob.probes).reshape(-1, 4))
    out = ctypes.c_longlong()
    C.fdtd_device_bytes(ctypes.byref(g), ctypes.byref(b), PRECISION[precision], n_src, n_prb,
                        int(prob.n_steps) if n_prb else 0, float(prob.f_max) if prob.f_max else -1.0, ctypes.byref(out))
    return int(out.value)


class Solver:
    def __init__(self, prob, precision: str = "fp32", stream=None, tuning: Optional[dict] = None,
                 spectrum: bool = True):
        self.problem = prob
        self.precision = precision
        g, b = problem_structs(prob)
        self._mat = np.ascontiguousarray(prob.mat, dtype=np.uint8)
        self._eps = np.ascontiguousarray(prob.eps_r, dtype=np.float64)
        boxes = np.ascontiguousarray(prob.pec_boxes, dtype=np.int32).reshape(-1, 6)
        self._boxes = boxes
        ctx = ctypes.c_void_p()
        C.fdtd_create(ctypes.byref(g), self._mat.ctypes.data, self._eps.ctypes.data, len(self._eps),
                      boxes.ctypes.data if len(boxes) else None, len(boxes), None, ctypes.byref(b),
                      PRECISION[precision], _stream_ptr(stream), ctypes.byref(ctx))
        self.ctx = ctx
        try:
            for (i, j, k, comp), (J0, t0, tau) in zip(np.asarray(prob.sources).reshape(-1, 4),
                                                      np.asarray(prob.source_params).reshape(-1, 3)):
                C.fdtd_set_source(ctx, int(i), int(j), int(k), int(comp), float(J0), float(t0), float(tau), None)
            for (i, j, k, comp), (V0, t0, tau, Rs) in zip(np.asarray(prob.vsources).reshape(-1, 4),
                                                          np.asarray(prob.vsource_params).reshape(-1, 4)):
                C.fdtd_set_voltage_source(ctx, int(i), int(j), int(k), int(comp), float(V0), float(t0),
                                          float(tau), float(Rs), None)
            for (i, j, k, comp) in np.asarray(prob.probes).reshape(-1, 4):
                C.fdtd_add_probe(ctx, int(i), int(j), int(k), int(comp), None)
            if spectrum and prob.n_steps > 0 and len(prob.probes):
                C.fdtd_set_spectrum(ctx, float(prob.f_max) if prob.f_max else -1.0, int(prob.n_steps))
            if tuning:
                self.set_tuning(**tuning)
        except Exception:
            self.close()
            raise

    # -- stepping ------------------------------------------------------------
    def step(self, n: int) -> "Solver":
        C.fdtd_step(self.ctx, int(n))
        return self

    def step_profiled(self, n: int) -> np.ndarray:
        """n steps with per-phase CUDA-event timing: [slab H, fused z-UPML,
        fused interior, slab E, sources/probes, DFT] summed device
        milliseconds."""
        ms = (ctypes.c_double * 6)()
        C.fdtd_step_profiled(self.ctx, int(n), ms)
        return np.array(list(ms))

    def run(self) -> "Solver":
        return self.step(self.problem.n_steps)

    def sync(self):
        C.fdtd_sync(self.ctx)

    def reset(self):
        C.fdtd_reset(self.ctx)

    def set_materials(self, mat: np.ndarray):
        self._mat = np.ascontiguousarray(mat, dtype=np.uint8)
        C.fdtd_set_materials(self.ctx, self._mat.ctypes.data)

    def set_tuning(self, tile_x=0, tile_y=0, zseg=0, graph_chunk=0, depth=0, pair_zseg=0):
        """Kernel tuning (0 keeps a setting).  depth=2 advances the interior
        region two leapfrog steps per pass (time blocking; bit-identical
        results, one more field set in device memory)."""
        t = C.fdtd_tuning(tile_x, tile_y, zseg, graph_chunk, depth, pair_zseg)
        C.fdtd_set_tuning(self.ctx, ctypes.byref(t))

    # -- results ---------------------------------------------------------------
    def info(self) -> dict:
        inf = C.fdtd_info_t()
        C.fdtd_info(self.ctx, ctypes.byref(inf))
        return {name: getattr(inf, name) for name, _ in C.fdtd_info_t._fields_}

    @property
    def dt(self) -> float:
        return self.info()["dt"]

    def spectra(self) -> np.ndarray:
        """Complex [P, Q] running DFT (FP64)."""
        inf = self.info()
        P, Q = inf["n_probes"], inf["n_bins"]
        out = np.zeros((P, max(Q, 1), 2), dtype=np.float64)
        nb = ctypes.c_int()
        C.fdtd_probe_spectra(self.ctx, out.ctypes.data, max(Q, 1), ctypes.byref(nb))
        return (out[..., 0] + 1j * out[..., 1])[:, :Q]

    def spectra_into(self, out: np.ndarray) -> int:
        """Copy the raw [P, Q, 2] FP64 spectrum into a preallocated array."""
        nb = ctypes.c_int()
        C.fdtd_probe_spectra(self.ctx, out.ctypes.data, out.shape[1], ctypes.byref(nb))
        return nb.value

    def traces(self, max_len: Optional[int] = None) -> np.ndarray:
        inf = self.info()
        n = min(inf["step"], inf["n_total_steps"]) if max_len is None else max_len
        out = np.zeros((inf["n_probes"], n), dtype=np.float32)
        ln = ctypes.c_int()
        for p in range(inf["n_probes"]):
            C.fdtd_probe_trace(self.ctx, p, out[p].ctypes.data, n, ctypes.byref(ln))
        return out[:, : ln.value] if inf["n_probes"] else out

    def save(self) -> bytes:
        """Checkpoint of the whole solver state (fdtd_save)."""
        n = ctypes.c_size_t()
        C.fdtd_save(self.ctx, None, 0, ctypes.byref(n))
        buf = ctypes.create_string_buffer(n.value)
        C.fdtd_save(self.ctx, buf, n.value, ctypes.byref(n))
        return buf.raw

    def load(self, state: bytes) -> "Solver":
        """Restore a checkpoint taken from a solver of the same problem (fdtd_load)."""
        buf = ctypes.create_string_buffer(bytes(state), len(state))
        C.fdtd_load(self.ctx, buf, len(state))
        return self

    def field(self, comp: int) -> np.ndarray:
        p = self.problem
        out = np.zeros((p.nz + 1, p.ny + 1, p.nx + 1), dtype=np.float32)
        C.fdtd_get_field(self.ctx, int(comp), out.ctypes.data)
        return out

    def plane(self, comp: int, k: int) -> np.ndarray:
        """Node plane k of one component, [ny+1, nx+1] FP32 in SI units (fdtd_get_plane)."""
        p = self.problem
        out = np.zeros((p.ny + 1, p.nx + 1), dtype=np.float32)
        C.fdtd_get_plane(self.ctx, int(comp), int(k), out.ctypes.data)
        return out

    def diagnostics(self):
        e, d = ctypes.c_double(), ctypes.c_double()
        C.fdtd_diagnostics(self.ctx, ctypes.byref(e), ctypes.byref(d))
        return e.value, d.value

    def close(self):
        if getattr(self, "ctx", None):
            C.fdtd_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    def __init__(self, stream=None, tuning: Optional[dict] = None):
        b = ctypes.c_void_p()
        C.fdtd_batch_create(_stream_ptr(stream), ctypes.byref(b))
        self.b = b
        self.members: List[Solver] = []
        if tuning:
            self.set_tuning(**tuning)

    def set_tuning(self, tile_x=0, tile_y=0, zseg=0, graph_chunk=0, depth=0, pair_zseg=0):
        t = C.fdtd_tuning(tile_x, tile_y, zseg, graph_chunk, depth, pair_zseg)
        C.fdtd_batch_set_tuning(self.b, ctypes.byref(t))

    def add(self, s: Solver, n_steps: Optional[int] = None):
        C.fdtd_batch_add(self.b, s.ctx, int(s.problem.n_steps if n_steps is None else n_steps))
        self.members.append(s)

    def remove(self, s: Solver):
        C.fdtd_batch_remove(self.b, s.ctx)
        self.members.remove(s)

    def step(self, n: int) -> int:
        done = ctypes.c_int()
        C.fdtd_batch_step(self.b, int(n), ctypes.byref(done))
        return done.value

    def remaining(self, s: Solver) -> int:
        r = ctypes.c_longlong()
        C.fdtd_batch_remaining(self.b, s.ctx, ctypes.byref(r))
        return r.value

    def sync(self):
        C.fdtd_batch_sync(self.b)

    def close(self):
        if getattr(self, "b", None):
            C.fdtd_batch_destroy(self.b)
            self.b = None
            self.members = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
