"""Parity at the benchmarked sizes, in the launch configuration bench.py times
(default tuning: 62x8 fused tiles, 10-plane z-segments, CUDA graphs of 16
steps), against the FP64 oracle:

* the full 880x680x100 multilayer board (60.6 M nodes) for 60 steps, with the
  pulse moved early and two extra sources in the air near opposite corners
  so the waves reach the UPML: every element of the six fields and the 64
  probe traces;
* its quarter-scale copy (280x230x100) for 400 steps, by which time the waves
  have entered the UPML on every face;
* the batched workload (64 uneven boards stepped together, one launch per
  phase): two sampled boards against the oracle after 300 steps, and every
  board finite.

Tolerances as in test_parity_gpu: FP32 relative L2 <= 1e-4 per field group
and every element within 1e-4 of the group's max |value|.
"""
import numpy as np
import pytest

import oracle
from paper_1008_2602_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fdtd():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("a CUDA device is required for -m gpu tests")
    from paper_1008_2602_gb300 import solver
    return solver


def rel_l2(a, b):
    """Relative L2 error of a against b (complex arrays compared as complex)."""
    a = np.asarray(a)
    b = np.asarray(b)
    dt = np.complex128 if np.iscomplexobj(a) or np.iscomplexobj(b) else np.float64
    a = a.astype(dt)
    b = b.astype(dt)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _fields_close(s, ref_fields, tol=1e-4):
    for comps in ((0, 1, 2), (3, 4, 5)):
        num = den = 0.0
        m = max(float(np.abs(ref_fields[c]).max()) for c in comps)
        for c in comps:
            g = s.field(c).astype(np.float64)
            r = ref_fields[c]
            d = g - r
            num += float(np.vdot(d, d))
            den += float(np.vdot(r, r))
            assert np.abs(d).max() <= tol * m, (c, np.abs(d).max() / m)
        assert m > 0
        assert np.sqrt(num / den) <= tol, (comps, np.sqrt(num / den))


def _early_pulse(p, steps, t0_steps=20, tau_steps=6):
    """Same board, sources and probes plus two E_z sources in the air gap near
    opposite corners (four cells from the x, y and z UPML), all with the
    Eq. 8 pulse centred t0_steps steps in and tau_steps steps wide, so a short
    run carries signal into the interior and into every UPML region."""
    dt = p.courant * oracle.cfl_dt(p.dx, p.dy, p.dz)
    d = p.upml_depth
    extra = np.array([[d[0] + 4, d[2] + 4, p.nz - d[5] - 4, 2],
                      [p.nx - d[1] - 5, p.ny - d[3] - 5, d[4] + 4, 2]], np.int32)
    src = np.vstack([np.asarray(p.sources, np.int32).reshape(-1, 4), extra])
    prm = np.tile(np.array([[float(np.asarray(p.source_params)[0, 0]), t0_steps * dt, tau_steps * dt]]),
                  (len(src), 1))
    return p.replace(sources=src, source_params=prm, n_steps=steps)


def test_full_size_multilayer_board(fdtd, ncpu):
    p = _early_pulse(W.multilayer_board(), 60)
    assert (p.nx, p.ny, p.nz) == (880, 680, 100)
    ref = oracle.run(p, n_threads=ncpu, fields=True, dft=False)
    s = fdtd.Solver(p)
    inf = s.info()
    assert inf["fused_upml_nodes"] > 0 and inf["slab_nodes"] > 0
    s.run()
    tr = s.traces()
    assert tr.shape == ref["trace"].shape
    assert np.abs(ref["trace"]).max() > 0
    assert rel_l2(tr, ref["trace"]) <= 1e-4
    # the UPML carries signal by now: the slab kernels and the fused z-UPML
    # launch are all exercised
    d = p.upml_depth
    ez = np.abs(ref["fields"][2])
    big = ez.max()
    assert ez[: d[4]].max() > 1e-6 * big and ez[-d[5]:].max() > 1e-6 * big
    assert ez[:, :, : d[0]].max() > 1e-6 * big and ez[:, :, -d[1]:].max() > 1e-6 * big
    _fields_close(s, ref["fields"])
    s.close()


def test_quarter_scale_multilayer_board(fdtd, ncpu):
    p = _early_pulse(W.multilayer_board(scale=4), 400)
    ref = oracle.run(p, n_threads=ncpu, fields=True, dft=False)
    s = fdtd.Solver(p)
    s.run()
    tr = s.traces()
    for q in range(len(tr)):
        if np.abs(ref["trace"][q]).max() > 0:
            assert rel_l2(tr[q], ref["trace"][q]) <= 1e-4, q
    # every UPML face has been reached (x, y slabs and z planes)
    d = p.upml_depth
    ez = np.abs(ref["fields"][2])
    big = ez.max()
    assert ez[:, :, : d[0]].max() > 1e-8 * big and ez[:, : d[2], :].max() > 1e-8 * big
    assert ez[: d[4]].max() > 1e-8 * big
    _fields_close(s, ref["fields"])
    s.close()


def test_batched_workload_sampled_boards(fdtd, ncpu):
    probs = W.batch_boards(seed=4, n_boards=64, n_steps=5000)
    b = fdtd.Batch()
    sols = [fdtd.Solver(p) for p in probs]
    for s in sols:
        b.add(s)
    steps = 300
    b.step(steps)
    b.sync()
    for s in sols:
        assert np.isfinite(s.traces()[:, :steps]).all()
    for q in (0, 37):
        p = probs[q]
        ref = oracle.run(p, n_threads=ncpu, fields=True, dft=False, n_steps=steps)
        tr = sols[q].traces()[:, :steps]
        assert rel_l2(tr, ref["trace"]) <= 1e-4, q
        _fields_close(sols[q], ref["fields"])
    b.close()
    for s in sols:
        s.close()
