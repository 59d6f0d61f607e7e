"""FP16 field storage (FP32 arithmetic) on the quarter-scale copy of
the 880x680x100 multilayer board (280x230x100, 1000 steps with the pulse
moved early so the run carries a full pulse), against the FP32 run and
against the FP64 oracle:

* probe traces: relative L2 over all probes, FP32 <= 1e-4 of the oracle,
  FP16 <= 1e-2 (the target for reduced storage);
* FP32 and FP16: the spectral peak of every probe with signal stays within
  one running-DFT bin of the oracle's (1000 steps give coarse bins, where a
  broad peak can sit between two nearly equal bins), or lands on a bin whose
  oracle magnitude ties the oracle's peak within the mode's spectral error
  (several probes of this board have two separate peaks within 1 % of each
  other, e.g. probe 51: bins 1 and 8 at a ratio of 0.996, which FP16
  rounding may order either way).
"""
import numpy as np
import pytest

import oracle
from paper_1008_2602_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-4, "fp16": 1e-2}
PEAK_TIE = {"fp32": 1e-3, "fp16": 2e-2}   # relative magnitude within which two peaks tie


@pytest.fixture(scope="module")
def quarter():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("a CUDA device is required for -m gpu tests")
    p = W.multilayer_board(scale=4, n_steps=1000)
    dt = p.courant * oracle.cfl_dt(p.dx, p.dy, p.dz)
    prm = np.array(p.source_params, np.float64).copy()
    prm[:, 1] = 60 * dt
    prm[:, 2] = 15 * dt
    return p.replace(source_params=prm, f_max=None)


@pytest.fixture(scope="module")
def runs(quarter, ncpu):
    from paper_1008_2602_gb300 import solver
    out = {"oracle": oracle.run(quarter, n_threads=ncpu)}
    for prec in ("fp32", "fp16"):
        s = solver.Solver(quarter, precision=prec)
        s.run()
        out[prec] = {"trace": s.traces().astype(np.float64), "spectra": s.spectra()}
        s.close()
    return out


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_storage_mode_error(runs, prec):
    ref = runs["oracle"]
    got = runs[prec]
    live = np.abs(ref["trace"]).max(axis=1) > 1e-3 * np.abs(ref["trace"]).max()
    assert live.sum() >= 4
    e_oracle = rel_l2(got["trace"][live], ref["trace"][live])
    e_fp32 = rel_l2(got["trace"][live], runs["fp32"]["trace"][live])
    assert e_oracle <= TOL[prec], (prec, e_oracle, e_fp32)
    assert e_fp32 <= TOL[prec] + 1e-4
    for q in np.nonzero(live)[0]:
        g = np.abs(got["spectra"][q][1:])
        r = np.abs(ref["spectra"][q][1:])
        i, j = int(np.argmax(g)), int(np.argmax(r))
        assert abs(i - j) <= 1 or r[i] >= (1 - PEAK_TIE[prec]) * r[j], (q, i, j, float(r[i] / r[j]))
