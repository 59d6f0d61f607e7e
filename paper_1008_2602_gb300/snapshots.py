"""Headless field snapshots: the data of the Results section's Figs. 3-4.

The paper shows the ground-plane E_z of its 100 x 60 x 0.8 mm board spreading
from a central current source and absorbed by the UPML at the board's edge.
There is no graphics stack here, so the figures are produced as arrays: the
E_z node plane through the dielectric, copied from the device at chosen steps
(fdtd_get_plane), saved with numpy.  Rendering them is left to the user.

    python -m paper_1008_2602_gb300.snapshots --out snaps --steps 100 200 400 800

writes snaps/ez_plane.npz with `steps`, `t` [s], `ez` [n, ny+1, nx+1] (V/m),
the plane index and the cell sizes.
"""
from __future__ import annotations

import argparse
import os
from typing import Dict, Sequence

import numpy as np

from . import solver as _solver
from . import workloads as W


def ez_snapshots(prob, steps: Sequence[int], k: int = None, precision: str = "fp32") -> Dict[str, np.ndarray]:
    """Advance a solver of ``prob`` and copy the E_z node plane ``k`` (default:
    the first dielectric layer) after each of ``steps`` leapfrog steps."""
    steps = sorted(int(s) for s in steps)
    if k is None:
        k = prob.dielectric_k[0][0] if prob.dielectric_k else prob.nz // 2
    s = _solver.Solver(prob.replace(n_steps=max(steps[-1], 1)), precision=precision)
    try:
        out, done = [], 0
        for n in steps:
            s.step(n - done)
            done = n
            out.append(s.plane(2, k))
        dt = s.dt
    finally:
        s.close()
    return {"steps": np.array(steps), "t": np.array(steps) * dt, "ez": np.stack(out), "k": np.array(k),
            "d": np.array([prob.dx, prob.dy, prob.dz])}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--out", default="snapshots")
    ap.add_argument("--steps", type=int, nargs="+", default=[100, 200, 300, 400, 600, 800])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp16"])
    a = ap.parse_args(argv)
    snaps = ez_snapshots(W.fig3_board(), a.steps, precision=a.precision)
    os.makedirs(a.out, exist_ok=True)
    path = os.path.join(a.out, "ez_plane.npz")
    np.savez(path, **snaps)
    print(path)


if __name__ == "__main__":
    main()
