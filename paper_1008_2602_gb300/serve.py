"""Continuous-batching solve server (the served workload).

Requests are boards (``workloads.Request``: arrival time + ``Problem``).  The
server admits queued requests as soon as a batch slot and enough of the HBM
budget are free, keeps every admitted board's fields on the device, and
advances all admitted boards together with ``Batch.step`` in chunks of
leapfrog steps (one launch per phase for the whole mix, replayed as a CUDA
graph).  A board that reaches its step count retires at the next chunk
boundary: its spectra are copied back, its device memory released and its
latency (retire time - arrival time) recorded.  Requests that arrive while
others are on the GPU join at the next chunk boundary, so their work overlaps
on the device.  With a backend that can launch a chunk without waiting for
it (``launch`` / ``wait``), admission runs while the chunk executes: a new
board's host precompute and uploads (on its own stream) overlap the device
work of the boards already admitted, and it joins the mix at the next chunk.

The scheduling logic talks to a small backend interface so it can be
exercised without a GPU; ``CudaBackend`` is the real one (libfdtd.so).
"""
from __future__ import annotations

import dataclasses
import math
import time
from typing import Callable, Dict, List, Optional

import numpy as np


@dataclasses.dataclass
class Result:
    rid: int
    arrival: float
    admitted: float
    finished: float
    cells: int
    steps: int
    spectra: Optional[np.ndarray] = None

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


def estimate_bytes(prob, precision: str = "fp32") -> int:
    """Device bytes a board will hold, asked of the library before the board
    exists (fdtd_device_bytes: the library's own layout of fields, ids, UPML
    auxiliaries, traces and spectra; 16-bit ids assumed, so at most one byte
    per node and 1 MB above what the board then reports)."""
    from . import solver
    return solver.device_bytes(prob, precision)


class CudaBackend:
    """Backend over libfdtd.so: one Batch, one Solver per admitted request."""

    def __init__(self, precision: str = "fp32", tuning: Optional[dict] = None):
        from . import solver
        self._solver = solver
        self.precision = precision
        self.batch = solver.Batch(tuning=tuning)

    def admit(self, prob):
        s = self._solver.Solver(prob, precision=self.precision)
        self.batch.add(s, prob.n_steps)
        return s

    def device_bytes(self, handle) -> int:
        return handle.info()["device_bytes"]

    def step(self, n: int) -> None:
        self.batch.step(n)
        self.batch.sync()

    def launch(self, n: int) -> None:
        """Queue one chunk of n steps for every member; returns at once."""
        self.batch.step(n)

    def wait(self) -> None:
        """Wait for the queued chunk (and report device-side errors)."""
        self.batch.sync()

    def remaining(self, handle) -> int:
        return self.batch.remaining(handle)

    def retire(self, handle):
        self.batch.remove(handle)
        spectra = handle.spectra()
        handle.close()
        return spectra

    def close(self):
        self.batch.close()


class Server:
    """Admission by HBM budget and slot count, continuous batching in chunks."""

    def __init__(self, backend, hbm_budget: int, max_boards: int = 64, chunk: int = 250,
                 clock: Callable[[], float] = time.perf_counter, simulate_clock: bool = False):
        self.backend = backend
        self.budget = int(hbm_budget)
        self.max_boards = max_boards
        self.chunk = chunk
        self.clock = clock
        self.simulate = simulate_clock
        self.used = 0
        self.active: Dict[int, tuple] = {}     # rid -> (handle, bytes, Result)
        self.results: List[Result] = []
        self.rejected: List[int] = []

    def run(self, requests, time_scale: float = 1.0) -> List[Result]:
        """Serve ``requests`` (sorted by arrival, seconds * time_scale after
        the start).  Returns one Result per served request."""
        pending = sorted(requests, key=lambda r: r.arrival)
        queue: List = []
        t0 = self.clock()
        sim_now = 0.0
        i = 0
        overlap = not self.simulate and hasattr(self.backend, "launch") and hasattr(self.backend, "wait")

        def now_():
            return sim_now if self.simulate else self.clock() - t0

        def arrivals():
            nonlocal i
            while i < len(pending) and pending[i].arrival * time_scale <= now_():
                queue.append(pending[i])
                i += 1

        def admit():
            # admit in arrival order while a slot and the budget allow
            while queue and len(self.active) < self.max_boards:
                req = queue[0]
                need = estimate_bytes(req.problem, getattr(self.backend, "precision", "fp32"))
                if need > self.budget:
                    self.rejected.append(req.rid)     # can never fit
                    queue.pop(0)
                    continue
                if self.used + need > self.budget:
                    break
                queue.pop(0)
                h = self.backend.admit(req.problem)
                nb = max(need, self.backend.device_bytes(h))
                self.used += nb
                res = Result(rid=req.rid, arrival=req.arrival * time_scale, admitted=now_(), finished=math.nan,
                             cells=req.problem.cells, steps=req.problem.n_steps)
                self.active[req.rid] = (h, nb, res)

        while i < len(pending) or queue or self.active:
            arrivals()
            admit()
            if not self.active:
                if i < len(pending):          # idle until the next arrival
                    nxt = pending[i].arrival * time_scale
                    if self.simulate:
                        sim_now = max(sim_now, nxt)
                    else:
                        time.sleep(max(0.0, min(0.05, nxt - (self.clock() - t0))))
                continue
            # one chunk for every admitted board
            if self.simulate:
                sim_now += self.backend.step(self.chunk) or 0.0
            elif overlap:
                self.backend.launch(self.chunk)
                arrivals()                    # boards admitted now join at the next chunk
                admit()
                self.backend.wait()
            else:
                self.backend.step(self.chunk)
            now = now_()
            for rid in [r for r, (h, _, _) in self.active.items() if self.backend.remaining(h) == 0]:
                h, nb, res = self.active.pop(rid)
                res.spectra = self.backend.retire(h)
                res.finished = now
                self.used -= nb
                self.results.append(res)
        return self.results


def route(requests, n_ranks: int, rate_cells_per_s: float = 6e10) -> List[int]:
    """Rank for every request of one stream shared by n_ranks replicas (one
    GPU each): in arrival order, each request goes to the rank with the least
    estimated backlog (cell-updates still queued, drained at
    rate_cells_per_s per rank since the previous arrival).  Deterministic in
    its inputs, so every rank computes the same assignment and serves its own
    share with no exchange between ranks."""
    backlog = [0.0] * n_ranks
    t_prev = 0.0
    out = []
    for r in sorted(requests, key=lambda q: (q.arrival, q.rid)):
        drain = rate_cells_per_s * max(0.0, r.arrival - t_prev)
        t_prev = max(t_prev, r.arrival)
        backlog = [max(0.0, b - drain) for b in backlog]
        k = min(range(n_ranks), key=lambda i: (backlog[i], i))
        backlog[k] += float(r.problem.cells) * r.problem.n_steps
        out.append((r.rid, k))
    order = {rid: k for rid, k in out}
    return [order[r.rid] for r in requests]


def summarize(results: List[Result], wall: float) -> dict:
    lat = np.array([r.latency for r in results]) if results else np.zeros(1)
    cells_steps = float(sum(r.cells * r.steps for r in results))
    return {"solves": len(results), "solves_per_s": len(results) / wall if wall > 0 else 0.0,
            "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
            "mean_latency_s": float(lat.mean()), "gcell_updates_per_s": cells_steps / wall / 1e9 if wall > 0 else 0.0,
            "wall_s": wall}
