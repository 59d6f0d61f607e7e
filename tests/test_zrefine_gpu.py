"""The z-refinement study of the Results section (the 0.8 mm dielectric cut
into 1 to 15 cells) on the GPU.  The model and the compared quantity are a
reading (the paper gives neither): a 40 x 30 mm plane pair, a full-height
current filament at one corner, the voltage between the planes (sum of E_z dz)
at the opposite corner, air and z UPML of fixed thickness in mm, one common
dt (the finest grid's CFL limit) for all cuttings.

* parity: the 1- and 2-cell GPU runs match the FP64 oracle (relative L2 1e-4);
* convergence: the difference to the 15-cell run falls monotonically with
  refinement, by at least 2x per doubling of cells, and is below 0.1 % of
  the peak voltage from 4 cells on (the paper reports < 0.1 % over 1-15
  cells; this model gives about 1.7 % at 1 cell and 0.5 % at 2)."""
import numpy as np
import pytest

import oracle
from paper_1008_2602_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_z_refinement_sweep(ncpu):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("a CUDA device is required for -m gpu tests")
    from paper_1008_2602_gb300 import solver
    dt = 0.99 * oracle.cfl_dt(2e-3, 2e-3, 0.8e-3 / 15)
    n = int(1.5e-9 / dt)
    V = {}
    for nzd in (1, 2, 4, 8, 15):
        p = W.zrefine_board(nzd, dt, n)
        s = solver.Solver(p)
        s.run()
        V[nzd] = s.traces().astype(np.float64).sum(axis=0) * p.dz
        s.close()
        if nzd <= 2:
            ref = oracle.run(p, dft=False, n_threads=ncpu)["trace"].sum(axis=0) * p.dz
            assert np.linalg.norm(V[nzd] - ref) <= 1e-4 * np.linalg.norm(ref), nzd
    m = np.abs(V[15]).max()
    dev = [np.abs(V[k] - V[15]).max() / m for k in (1, 2, 4, 8)]
    for a, b in zip(dev, dev[1:]):
        assert b <= 0.5 * a, dev
    assert dev[2] < 1.5e-3 and dev[3] < 1e-3, dev
