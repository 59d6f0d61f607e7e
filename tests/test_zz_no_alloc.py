"""fdtd_energy_static: the energy / div B check for callers that cannot
allocate device memory (e.g. while capturing a CUDA graph or under a fixed
memory budget).  It works on caller-owned device buffers and keeps its
scratch in a fixed static device array, so it must agree with the context's
fdtd_diagnostics (which uses scratch allocated at fdtd_create) -- here on
two calls in a row, on two different field states, so that a call cannot
lean on what the previous one left in the shared array.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_1008_2602_gb300 import workloads as W

pytestmark = pytest.mark.gpu

MU0 = 4e-7 * np.pi


def _state(s, steps_before):
    """E^n, H^{n-1/2}, H^{n+1/2} (host copies) and the context's own
    diagnostics W^n, max|div B| after n + 1 = steps_before + 1 steps."""
    s.step(steps_before)
    e = [s.field(c) for c in range(3)]
    h0 = [s.field(c) for c in range(3, 6)]
    s.step(1)
    h1 = [s.field(c) for c in range(3, 6)]
    energy, divb = s.diagnostics()
    return e + h0 + h1, energy, divb


def test_energy_static_matches_context_diagnostics_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("a CUDA device is required for -m gpu tests")
    from paper_1008_2602_gb300 import capi, solver

    eps_r = 2.5
    p = W.box(30, 22, 14, d=(1e-3, 1.2e-3, 0.7e-3), eps_r=eps_r)
    p = W.add_ports(p, [(12, 9, 6, 2), (20, 14, 4, 0)], [(12, 9, 6, 2)], n_steps=400)
    s = solver.Solver(p)
    dev = torch.device("cuda", torch.cuda.current_device())
    eps = torch.full((p.nz + 1, p.ny + 1, p.nx + 1), eps_r, dtype=torch.float32, device=dev)
    eps_ptrs = (ctypes.c_void_p * 3)(*([eps.data_ptr()] * 3))
    depth = (ctypes.c_int * 6)(*([0] * 6))
    stream = torch.cuda.current_stream()

    # two states, each checked right after the other on the shared scratch
    states = [_state(s, 150), _state(s, 120)]
    results = []
    for fields, _, _ in states:
        bufs = [torch.from_numpy(np.ascontiguousarray(f)).to(dev) for f in fields]
        ptrs = (ctypes.c_void_p * 9)(*[b.data_ptr() for b in bufs])
        energy, divb = ctypes.c_double(), ctypes.c_double()
        capi.fdtd_energy_static(ptrs, eps_ptrs, p.nx, p.ny, p.nz, p.nx + 1, p.dx, p.dy, p.dz, depth,
                                ctypes.c_void_p(stream.cuda_stream), ctypes.byref(energy), ctypes.byref(divb))
        results.append((energy.value, divb.value, max(np.abs(f).max() for f in fields[6:])))
        del bufs
    for (e_static, d_static, hmax), (_, e_ctx, d_ctx) in zip(results, states):
        assert e_ctx > 0
        assert abs(e_static - e_ctx) <= 1e-6 * e_ctx, (e_static, e_ctx)
        bound = 1e-4 * MU0 * hmax / min(p.dx, p.dy, p.dz)   # same bound as the context's div B test
        assert d_static <= bound and d_ctx <= bound
        assert abs(d_static - d_ctx) <= bound
    assert results[0][0] != results[1][0]
    s.close()


def test_energy_static_rejects_oversized_grids():
    pytest.importorskip("torch")
    from paper_1008_2602_gb300 import capi
    ptrs = (ctypes.c_void_p * 9)(*([1] * 9))   # never dereferenced: the size check comes first
    with pytest.raises(capi.FdtdError) as ei:
        capi.fdtd_energy_static(ptrs, None, 1000, 1000, 100, 1001, 1e-3, 1e-3, 1e-3, None, None, None, None)
    assert ei.value.code == capi.FDTD_EINVAL
    assert "at most" in capi.lib.fdtd_last_error().decode()
