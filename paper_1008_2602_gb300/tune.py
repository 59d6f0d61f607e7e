"""Autotuner for the launch configuration.

Times candidate configurations on a throwaway copy of the workload (the
real solvers are never advanced by tuning) and caches the fastest per
precision and grid class in a JSON file.  The search covers:
* the fused-tile shapes (tile_x x tile_y columns);
* the z-segment lengths;
* the CUDA-graph chunk sizes;
* for a single board, the blocking depth: one leapfrog step per interior
  sweep, or two (the two-step pass, with its z-segment length).  A batch
  advances one step per sweep.
"""
from __future__ import annotations

import json
import math
import os
import time
from typing import Dict, Iterable, List, Optional, Sequence

SHAPES = [(62, 4), (124, 4), (62, 8), (124, 8)]
ZSEGS = [8, 10, 16, 25]
CHUNKS = [16, 64]
PAIR_ZSEGS = [19, 38]   # two-step pass segments tried for a single board

CACHE = os.environ.get("FDTD_TUNE_CACHE",
                       os.path.join(os.path.expanduser("~"), ".cache", "paper_1008_2602_gb300", "tune.json"))


def grid_class(probs, precision: str) -> str:
    """Bucket of a workload: precision, board count, log2 of the mean cell
    count, and the z extent rounded to 16."""
    n = len(probs)
    cells = sum(p.cells for p in probs) / max(n, 1)
    nz = int(round(sum(p.nz for p in probs) / max(n, 1) / 16.0)) * 16
    return f"{precision}:n{n}:c{int(math.log2(max(cells, 1)))}:z{nz}"


def _load() -> Dict[str, dict]:
    try:
        with open(CACHE) as f:
            return json.load(f)
    except Exception:
        return {}


def _save(d: Dict[str, dict]) -> None:
    try:
        os.makedirs(os.path.dirname(CACHE), exist_ok=True)
        tmp = CACHE + f".{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(d, f, indent=1, sort_keys=True)
        os.replace(tmp, CACHE)
    except OSError:
        pass


def _time_batch(probs, precision: str, cfg: dict, steps: int) -> float:
    from . import solver
    b = solver.Batch(tuning=cfg)
    sols = []
    try:
        for p in probs:
            s = solver.Solver(p.replace(n_steps=max(steps * 3, 1)), precision=precision, spectrum=False)
            b.add(s, steps * 3)
            sols.append(s)
        b.step(steps)        # warm-up: plan, descriptors, graph capture
        b.sync()
        t0 = time.perf_counter()
        b.step(steps)
        b.sync()
        return time.perf_counter() - t0
    finally:
        b.close()
        for s in sols:
            s.close()


def _time_single(prob, precision: str, cfg: dict, steps: int) -> float:
    from . import solver
    s = solver.Solver(prob.replace(n_steps=max(steps * 3, 1)), precision=precision, spectrum=False, tuning=cfg)
    try:
        s.step(steps)        # warm-up: plan, descriptors, graph capture
        s.sync()
        t0 = time.perf_counter()
        s.step(steps)
        s.sync()
        return time.perf_counter() - t0
    finally:
        s.close()


def tune(probs: Sequence, precision: str = "fp32", steps: int = 32, shapes=SHAPES, zsegs=ZSEGS,
         chunks=CHUNKS, pair_zsegs=PAIR_ZSEGS, use_cache: bool = True, log=None) -> dict:
    """Best tuning dict (tile_x, tile_y, zseg, graph_chunk, depth, and for
    depth 2 pair_zseg) for stepping ``probs`` together (one board = a single
    solve, which also tries depth 2)."""
    key = grid_class(probs, precision)
    cache = _load() if use_cache else {}
    if use_cache and key in cache:
        return dict(cache[key]["tuning"])
    best, best_t = None, float("inf")
    trials = []
    for (tx, ty) in shapes:
        for zs in zsegs:
            cfg = dict(tile_x=tx, tile_y=ty, zseg=zs, graph_chunk=chunks[0])
            t = _time_batch(probs, precision, cfg, steps)
            trials.append((t, cfg))
            if log:
                log(f"tune {key} {cfg} {t * 1e3:.2f} ms")
            if t < best_t:
                best, best_t = cfg, t
    for ch in chunks[1:]:
        cfg = dict(best, graph_chunk=ch)
        t = _time_batch(probs, precision, cfg, steps)
        if log:
            log(f"tune {key} {cfg} {t * 1e3:.2f} ms")
        if t < best_t:
            best, best_t = cfg, t
    best = dict(best, depth=1)
    if len(probs) == 1 and pair_zsegs:
        # blocking depth, timed on the single-board path both depths run on
        best_t = _time_single(probs[0], precision, best, steps)
        trials.append((best_t, best))
        for pz in pair_zsegs:
            cfg = dict(best, depth=2, pair_zseg=pz)
            t = _time_single(probs[0], precision, cfg, steps)
            trials.append((t, cfg))
            if log:
                log(f"tune {key} {cfg} {t * 1e3:.2f} ms")
            if t < best_t:
                best, best_t = cfg, t
    if use_cache:
        cache = _load()
        cache[key] = {"tuning": best, "ms_per_step": best_t * 1e3 / steps,
                      "trials": [{"ms": t * 1e3, **c} for t, c in trials]}
        _save(cache)
    return dict(best)
