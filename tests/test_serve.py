"""Host-side logic of the continuous-batching server, with a fake backend
and a simulated clock (no GPU): admission by HBM budget and slot count,
arrival order, chunked progress, latency accounting, rejection of requests
that can never fit."""
import time

import numpy as np

from paper_1008_2602_gb300 import serve, workloads as W


class FakeBackend:
    precision = "fp32"

    def __init__(self, cells_per_s=1e10):
        self.rate = cells_per_s
        self.active = []
        self.max_active = 0
        self.order = []

    def admit(self, prob):
        h = {"prob": prob, "left": prob.n_steps}
        self.active.append(h)
        self.order.append(prob.name)
        self.max_active = max(self.max_active, len(self.active))
        self.max_bytes = max(getattr(self, "max_bytes", 0), sum(self.device_bytes(a) for a in self.active))
        return h

    def device_bytes(self, h):
        return serve.estimate_bytes(h["prob"])

    def step(self, n):
        work = 0.0
        for h in self.active:
            d = min(n, h["left"])
            h["left"] -= d
            work += d * h["prob"].cells
        return work / self.rate

    def remaining(self, h):
        return h["left"]

    def retire(self, h):
        self.active = [a for a in self.active if a is not h]   # by identity (boards hold numpy arrays)
        return np.zeros(1)


def _reqs(n=12, rate=20.0, seed=5):
    return W.request_stream(seed=seed, n_requests=n, rate=rate, step_scale=0.05, cell_scale=0.02)


def test_all_requests_served_in_arrival_order():
    reqs = _reqs()
    be = FakeBackend()
    srv = serve.Server(be, hbm_budget=1 << 40, chunk=50, simulate_clock=True)
    res = srv.run(reqs)
    assert sorted(r.rid for r in res) == [r.rid for r in reqs]
    assert be.order == [r.problem.name for r in reqs]
    for r in res:
        assert r.finished >= r.admitted >= r.arrival - 1e-12
        assert r.latency > 0


def test_budget_limits_concurrency():
    reqs = _reqs(n=10, rate=1e6)   # all arrive at once
    need = max(serve.estimate_bytes(r.problem) for r in reqs)
    be = FakeBackend()
    srv = serve.Server(be, hbm_budget=int(2.5 * need), chunk=50, simulate_clock=True)
    res = srv.run(reqs)
    assert len(res) == 10
    assert be.max_bytes <= int(2.5 * need)      # admitted bytes never exceed the budget
    assert 2 <= be.max_active < 10


def test_slot_limit_and_continuous_admission():
    reqs = _reqs(n=9, rate=1e6)
    be = FakeBackend()
    srv = serve.Server(be, hbm_budget=1 << 40, max_boards=3, chunk=25, simulate_clock=True)
    srv.run(reqs)
    assert be.max_active == 3


def test_oversized_request_is_rejected_not_hung():
    reqs = _reqs(n=4)
    be = FakeBackend()
    tiny = min(serve.estimate_bytes(r.problem) for r in reqs) - 1
    srv = serve.Server(be, hbm_budget=tiny, chunk=50, simulate_clock=True)
    res = srv.run(reqs)
    assert res == [] and sorted(srv.rejected) == [r.rid for r in reqs]


def test_summary_percentiles():
    rs = [serve.Result(rid=i, arrival=0.0, admitted=0.0, finished=float(i + 1), cells=10, steps=10) for i in range(100)]
    s = serve.summarize(rs, wall=100.0)
    assert abs(s["p50_latency_s"] - 50.5) < 1e-9 and s["p99_latency_s"] > 99.0
    assert abs(s["solves_per_s"] - 1.0) < 1e-12


class AsyncFakeBackend(FakeBackend):
    """A backend whose chunk is queued by launch() and finished by wait(),
    with real (short) durations, logging the order of calls."""

    def __init__(self):
        super().__init__()
        self.log = []

    def admit(self, prob):
        self.log.append(("admit", prob.name))
        return super().admit(prob)

    def launch(self, n):
        self.log.append(("launch", len(self.active)))
        self._n = n
        time.sleep(0.01)          # host time spent queueing the chunk

    def wait(self):
        time.sleep(0.01)          # device time of the chunk
        self.step(self._n)
        self.log.append(("wait", None))


def test_admission_overlaps_the_running_chunk():
    """Requests that arrive while a chunk is queued are admitted before the
    server waits for that chunk (their host set-up overlaps device work),
    join at the next chunk, and every request is served."""
    reqs = _reqs(n=6, rate=1e6)
    for k, r in enumerate(reqs):
        r.arrival = 0.0 if k == 0 else 0.005   # one board first, the rest during its first chunk
    be = AsyncFakeBackend()
    srv = serve.Server(be, hbm_budget=1 << 40, chunk=10, simulate_clock=False)
    res = srv.run(reqs)
    assert sorted(r.rid for r in res) == [r.rid for r in reqs]
    first_launch = be.log.index(("launch", 1))
    first_wait = be.log.index(("wait", None))
    admitted_between = [e for e in be.log[first_launch:first_wait] if e[0] == "admit"]
    assert len(admitted_between) == 5, be.log[:12]


def test_router_balances_one_stream_across_ranks():
    """route(): every request to exactly one rank, deterministic, and the
    cell-updates per rank balanced (largest share within 1.5x of the mean on
    a burst where all requests arrive at once)."""
    reqs = W.request_stream(seed=8, n_requests=40, rate=1e6, step_scale=0.05, cell_scale=0.02)
    ranks = serve.route(reqs, 4)
    assert ranks == serve.route(reqs, 4)
    assert set(ranks) <= {0, 1, 2, 3} and len(ranks) == len(reqs)
    work = [0.0] * 4
    for r, k in zip(reqs, ranks):
        work[k] += r.problem.cells * r.problem.n_steps
    assert max(work) <= 1.5 * (sum(work) / 4)
    assert serve.route(reqs, 1) == [0] * len(reqs)


def test_device_bytes_follows_the_library_layout():
    """fdtd_device_bytes (host only): a board without UPML or ports is its two
    field parities, 16-bit ids, the 65536-row table, the UPML factor tables
    and the fixed scratch, to the byte; UPML auxiliaries and probe traces add
    to it, and FP16 storage halves the fields."""
    from paper_1008_2602_gb300 import solver
    p = W.box(20, 10, 6)
    nodes = 32 * 11 * 7                 # rows of 21 nodes padded to a pitch of 32 (an odd multiple of 32)
    base = solver.device_bytes(p)
    fields = 12 * nodes * 4
    assert base > fields + 2 * nodes + 65536 * 16
    assert base < fields + 2 * nodes + 65536 * 16 + 64 * 1024
    assert solver.device_bytes(p, "fp16") == base - 6 * nodes * 4
    up = solver.device_bytes(p.replace(upml_depth=(3,) * 6))
    assert up > base + 8 * 1000                 # UPML auxiliaries (two or more per graded node)
    with_probes = solver.device_bytes(W.add_ports(p, [(5, 5, 3, 2)], [(6, 5, 3, 2)] * 3, n_steps=1000))
    assert with_probes >= base + 3 * 1000 * 4
