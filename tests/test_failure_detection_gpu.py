"""Failure detection on the GPU without a fault: every device-side wait is
bounded and reports through a status word the host reads.  The self-test
waits on an mbarrier that nothing arrives at, with a short poll limit; it
must return FDTD_ETIMEOUT promptly, and the device must stay usable.
Non-finite fields (an unstable Courant number) are covered in
test_parity_gpu (FDTD_EUNSTABLE)."""
import time

import numpy as np
import pytest

from paper_1008_2602_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_device_stays_usable():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("a CUDA device is required for -m gpu tests")
    from paper_1008_2602_gb300 import capi, solver
    t0 = time.perf_counter()
    with pytest.raises(capi.FdtdError) as ei:
        capi.fdtd_selftest_wait_timeout(None, 4096)
    assert ei.value.code == capi.FDTD_ETIMEOUT
    assert time.perf_counter() - t0 < 30.0
    # the context and device are still usable afterwards
    p = W.random_problem(31, 20, 18, 12, upml=3, n_steps=50)
    s = solver.Solver(p)
    s.run()
    assert np.isfinite(s.traces()).all()
    s.close()
