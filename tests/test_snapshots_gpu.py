"""Headless snapshots of the ground-plane E_z (the data of the Results
section's Figs. 3-4) on the Fig. 3 board: the plane copied from the device
equals the oracle's field plane at the same step, and with the source at the
centre of a mirror-symmetric grid the snapshot is mirror-symmetric in x and y."""
import numpy as np
import pytest

import oracle
from paper_1008_2602_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_fig3_snapshot_matches_oracle_and_is_symmetric(ncpu, tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("a CUDA device is required for -m gpu tests")
    from paper_1008_2602_gb300 import snapshots
    p = W.fig3_board()
    snaps = snapshots.ez_snapshots(p, [150, 300])
    k = int(snaps["k"])
    ref = oracle.run(p.replace(n_steps=300), n_threads=ncpu, fields=True, dft=False)["fields"][2][k]
    ez = snaps["ez"][1].astype(np.float64)
    assert ez.shape == (p.ny + 1, p.nx + 1)
    m = np.abs(ref).max()
    assert m > 0 and np.abs(ez - ref).max() <= 1e-4 * m
    # mirror symmetry about the central source edge (i = nx/2, j = ny/2)
    live = ez[:, : p.nx + 1]
    assert np.abs(live - live[:, ::-1]).max() <= 1e-5 * m
    assert np.abs(live - live[::-1, :]).max() <= 1e-5 * m
    # the module's command line writes the same arrays
    snapshots.main(["--out", str(tmp_path), "--steps", "150"])
    saved = np.load(tmp_path / "ez_plane.npz")
    assert np.array_equal(saved["ez"][0], snaps["ez"][0])
