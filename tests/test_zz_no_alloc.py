"""fdtd_energy_static: the energy / div B check for callers that cannot
allocate device memory (code under a fixed memory budget or pool, real-time
loops that forbid allocator calls).  It works on caller-owned device buffers
and keeps its scratch in a fixed static device array, so it must agree with
the context's fdtd_diagnostics (which uses scratch allocated at fdtd_create)
-- here on two calls in a row, on two different field states, so that a call
cannot lean on what the previous one left in the shared array; once on a
board without UPML whose buffers are unpadded (pitch = nx + 1), once on a
board with a different UPML depth on every face whose buffers carry row
padding (pitch = nx + 8), where the div B window and the padded indexing are
what differ from the context's own kernel.

The argument checks (grid size limit, UPML depths) come before any device
work, so those tests run on the CPU.

This file is collected last on purpose: if its GPU test fails, a run that
stops at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_1008_2602_gb300 import workloads as W

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


def _padded(a, pitch):
    """[nz+1][ny+1][nx+1] host array -> [nz+1][ny+1][pitch] with zero padding."""
    out = np.zeros(a.shape[:2] + (pitch,), np.float32)
    out[..., : a.shape[2]] = a
    return out


@pytest.mark.gpu
@pytest.mark.parametrize("upml,pad", [((0,) * 6, 0), ((2, 3, 1, 4, 3, 2), 7)])
def test_energy_static_matches_context_diagnostics_twice(upml, pad):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("a CUDA device is required for -m gpu tests")
    from paper_1008_2602_gb300 import capi, solver

    eps_r = 2.5
    p = W.box(30, 22, 14, d=(1e-3, 1.2e-3, 0.7e-3), eps_r=eps_r, upml=upml)
    p = W.add_ports(p, [(12, 9, 6, 2), (20, 14, 4, 0)], [(12, 9, 6, 2)], n_steps=400)
    pitch = p.nx + 1 + pad
    s = solver.Solver(p)
    dev = torch.device("cuda", torch.cuda.current_device())
    eps = torch.full((p.nz + 1, p.ny + 1, pitch), eps_r, dtype=torch.float32, device=dev)
    eps_ptrs = (ctypes.c_void_p * 3)(*([eps.data_ptr()] * 3))
    depth = (ctypes.c_int * 6)(*upml)
    stream = torch.cuda.current_stream()

    # two states, each checked right after the other on the shared scratch
    states = [_state(s, 150), _state(s, 120)]
    results = []
    for fields, _, _ in states:
        bufs = [torch.from_numpy(_padded(f, pitch)).to(dev) for f in fields]
        ptrs = (ctypes.c_void_p * 9)(*[b.data_ptr() for b in bufs])
        energy, divb = ctypes.c_double(), ctypes.c_double()
        capi.fdtd_energy_static(ptrs, eps_ptrs, p.nx, p.ny, p.nz, pitch, p.dx, p.dy, p.dz, depth,
                                ctypes.c_void_p(stream.cuda_stream), ctypes.byref(energy), ctypes.byref(divb))
        results.append((energy.value, divb.value, max(np.abs(f).max() for f in fields[6:])))
        del bufs
    # div B outside the UPML is FP32 round-off accumulated over the run, so it
    # is bounded by the largest |H| the run has seen (with UPML the fields
    # later decay out of the board while that residue stays); a window one
    # cell into the UPML gives a value above this bound
    hmax_run = max(h for _, _, h in results)
    bound = 1e-4 * MU0 * hmax_run / min(p.dx, p.dy, p.dz)
    for (e_static, d_static, _), (_, e_ctx, d_ctx) in zip(results, states):
        assert e_ctx > 0
        assert abs(e_static - e_ctx) <= 1e-6 * e_ctx, (e_static, e_ctx)
        assert d_static <= bound and d_ctx <= bound, (d_static, d_ctx, bound)
        assert abs(d_static - d_ctx) <= bound
    assert results[0][0] != results[1][0]
    s.close()


def _call(capi, nx, ny, nz, pitch, depth):
    ptrs = (ctypes.c_void_p * 9)(*([1] * 9))   # never dereferenced: the argument checks come first
    d = (ctypes.c_int * 6)(*depth) if depth is not None else None
    with pytest.raises(capi.FdtdError) as ei:
        capi.fdtd_energy_static(ptrs, None, nx, ny, nz, pitch, 1e-3, 1e-3, 1e-3, d, None, None, None)
    assert ei.value.code == capi.FDTD_EINVAL
    return capi.lib.fdtd_last_error().decode()


def test_energy_static_rejects_oversized_grids():
    from paper_1008_2602_gb300 import capi
    assert "at most" in _call(capi, 1000, 1000, 100, 1001, None)


@pytest.mark.parametrize("depth", [(-1, 0, 0, 0, 0, 0), (0, 0, 0, -3, 0, 0), (6, 5, 0, 0, 0, 0), (0, 0, 0, 0, 9, 2)])
def test_energy_static_rejects_bad_upml_depths(depth):
    from paper_1008_2602_gb300 import capi
    assert "UPML" in _call(capi, 10, 12, 10, 11, depth)
