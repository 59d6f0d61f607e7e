"""One board split into sub-boards along y (slab decomposition).

The Yee curl of the Model section (Fig. 2) reaches one node plane, so a board
cut at node plane m can be stepped as two sub-boards that share the cell
layer [m, m+1]:

* part A holds cells [0, m+1) (node planes 0..m+1), part B cells [m, ny)
  (node planes m..ny); A owns node planes <= m, B owns planes >= m+1;
* each part runs the unchanged single-board step.  Its cut face has no UPML
  and a PEC wall, so the E components tangential to the cut (E_x, E_z) on
  its outer plane there come out wrong (zero), while every other sample it
  owns is exact: H on the shared layer is recomputed on both sides from E
  values both sides hold;
* after every step, A's plane m+1 receives B's E_x, E_z there, and B's plane
  m receives A's (``fdtd_halo_copy`` on one GPU or between peers,
  ``fdtd_halo_pack`` / ``fdtd_halo_unpack`` around a collective send/receive
  between ranks).  That is the whole exchange: 2 components x (nx+1)(nz+1)
  values each way per step.

Cuts must lie outside the y UPML (the shared cell is ungraded).  Several cuts
give several parts.  Sources sit in the part that owns their edge; an E_y
source on the shared cell layer is applied in both parts, since both update
that edge.  Probes are read from the owning part.

This module only partitions inputs and schedules copies; every update runs in
libfdtd.so's kernels.
"""
from __future__ import annotations

import dataclasses
from typing import Callable, List, Optional, Sequence, Tuple

import numpy as np

EX, EY, EZ = 0, 1, 2
TANGENTIAL_Y = (1 << EX) | (1 << EZ)     # E components tangential to a y = const cut


@dataclasses.dataclass
class Part:
    problem: object          # workloads.Problem of the sub-board
    lo: int                  # global node plane of local plane 0
    hi: int                  # global node plane of local plane ny_part
    own_lo: int              # first owned global node plane
    own_hi: int              # last owned global node plane
    probe_ids: List[int]     # indices into the global probe list, in local order


@dataclasses.dataclass
class Split:
    ny: int
    cuts: List[int]
    parts: List[Part]

    def exchanges(self) -> List[Tuple[int, int, int, int]]:
        """(dst part, dst local plane, src part, src local plane) per copy
        after every step: across cut c, the lower part's outer plane m+1
        from the upper part, the upper part's outer plane m from the lower."""
        out = []
        for c, m in enumerate(self.cuts):
            a, b = self.parts[c], self.parts[c + 1]
            out.append((c, (m + 1) - a.lo, c + 1, (m + 1) - b.lo))
            out.append((c + 1, m - b.lo, c, m - a.lo))
        return out


def _clip_boxes(boxes: np.ndarray, lo: int, hi: int) -> np.ndarray:
    """PEC boxes (cells [j0, j1), closed node box [j0, j1]) restricted to node
    planes [lo, hi] and shifted to local y."""
    out = []
    for i0, i1, j0, j1, k0, k1 in np.asarray(boxes).reshape(-1, 6):
        a, b = max(int(j0), lo), min(int(j1), hi)
        if a > b:
            continue
        out.append((i0, i1, a - lo, b - lo, k0, k1))
    return np.asarray(out, np.int32).reshape(-1, 6)


def split_y(prob, cuts: Sequence[int]) -> Split:
    """Partition `prob` at the given node planes (sorted, outside the y UPML,
    at least two cells apart)."""
    ny = prob.ny
    d = prob.upml_depth
    cuts = sorted(int(m) for m in cuts)
    prev = -2
    for m in cuts:
        if not (d[2] <= m and m + 1 <= ny - d[3]):
            raise ValueError(f"cut {m}: the shared cell [{m}, {m + 1}] must lie outside the y UPML")
        if m - prev < 2 or m < 1 or m > ny - 2:
            raise ValueError(f"cut {m}: every part needs at least two cells (cuts two or more planes apart)")
        prev = m
    bounds = [(0 if c == 0 else cuts[c - 1], ny if c == len(cuts) else cuts[c] + 1) for c in range(len(cuts) + 1)]
    parts = []
    srcs = np.asarray(prob.sources).reshape(-1, 4)
    prm = np.asarray(prob.source_params).reshape(-1, 3)
    vsrc = np.asarray(prob.vsources).reshape(-1, 4)
    vprm = np.asarray(prob.vsource_params).reshape(-1, 4)
    probes = np.asarray(prob.probes).reshape(-1, 4)
    last = len(bounds) - 1
    for p, (lo, hi) in enumerate(bounds):
        own_lo = lo if p == 0 else lo + 1
        own_hi = hi if p == last else hi - 1

        def owns(j, comp):
            # E_x, E_z on node plane j; E_y on the cell row j (both parts
            # holding the shared layer update it)
            if comp == EY:
                return lo <= j < hi
            return own_lo <= j <= own_hi

        def pick(rows, params):
            keep = [r for r, (i, j, k, comp) in enumerate(rows) if owns(int(j), int(comp))]
            loc = rows[keep].copy()
            loc[:, 1] -= lo
            return loc.astype(np.int32), params[keep].copy()

        s_loc, s_prm = pick(srcs, prm)
        v_loc, v_prm = pick(vsrc, vprm)
        # probes: the owner only (an E_y probe on the shared row m of a cut
        # belongs to the lower part, for which it is the top row)
        pid = [q for q, (i, j, k, comp) in enumerate(probes)
               if (own_lo <= int(j) <= own_hi if int(comp) != EY else
                   (lo <= int(j) < hi and (p == 0 or int(j) > lo)))]
        pr = probes[pid].copy()
        pr[:, 1] -= lo
        depth = list(d)
        walls = list(prob.walls)
        if p > 0:
            depth[2], walls[2] = 0, 0
        if p < last:
            depth[3], walls[3] = 0, 0
        sub = prob.replace(ny=hi - lo, mat=np.ascontiguousarray(prob.mat[:, lo:hi, :]),
                           pec_boxes=_clip_boxes(prob.pec_boxes, lo, hi), upml_depth=tuple(depth), walls=tuple(walls),
                           sources=s_loc, source_params=s_prm, vsources=v_loc, vsource_params=v_prm,
                           probes=pr.astype(np.int32), name=f"{prob.name}[y {lo}..{hi}]", board=None)
        parts.append(Part(sub, lo, hi, own_lo, own_hi, pid))
    return Split(ny, cuts, parts)


def even_cuts(prob, n_parts: int) -> List[int]:
    """Cut planes giving `n_parts` parts of about equal cell count."""
    ny, d = prob.ny, prob.upml_depth
    cuts = [int(round(ny * (p + 1) / n_parts)) - 1 for p in range(n_parts - 1)]
    return [min(max(m, d[2]), ny - d[3] - 1) for m in cuts]


def assemble(split: Split, per_part: Sequence[np.ndarray]) -> np.ndarray:
    """Global [nz+1][ny+1][nx+1] array from per-part node arrays (owned planes)."""
    a0 = per_part[0]
    out = np.zeros(a0.shape[:1] + (split.ny + 1,) + a0.shape[2:], a0.dtype)
    for part, a in zip(split.parts, per_part):
        out[:, part.own_lo:part.own_hi + 1] = a[:, part.own_lo - part.lo:part.own_hi - part.lo + 1]
    return out


def gather_probes(split: Split, per_part: Sequence[np.ndarray], n_probes: int) -> np.ndarray:
    """Per-probe rows (traces or spectra) back in the global probe order."""
    shape = next((a.shape[1:] for a in per_part if len(a)), (0,))
    dtype = next((a.dtype for a in per_part if len(a)), np.float64)
    out = np.zeros((n_probes,) + tuple(shape), dtype)
    for part, a in zip(split.parts, per_part):
        for row, q in enumerate(part.probe_ids):
            out[q] = a[row]
    return out


class SplitSolver:
    """The parts of one board on one or more devices of this process, with
    the halo copies between steps (``fdtd_halo_copy``).  Steps one leapfrog
    step at a time."""

    def __init__(self, prob, cuts: Sequence[int], precision: str = "fp32", devices: Optional[Sequence[int]] = None,
                 tuning: Optional[dict] = None):
        from . import solver
        import torch
        self.problem = prob
        self.split = split_y(prob, cuts)
        devices = list(devices) if devices is not None else [torch.cuda.current_device()] * len(self.split.parts)
        self.solvers = []
        for part, dev in zip(self.split.parts, devices):
            with torch.cuda.device(dev):
                self.solvers.append(solver.Solver(part.problem, precision=precision, tuning=tuning))
        self.steps = 0

    def step(self, n: int) -> "SplitSolver":
        from . import capi as C
        plan = self.split.exchanges()
        for _ in range(int(n)):
            for s in self.solvers:
                s.step(1)
            for dst, dplane, src, splane in plan:
                C.fdtd_halo_copy(self.solvers[dst].ctx, dplane, self.solvers[src].ctx, splane, 1, TANGENTIAL_Y)
            self.steps += 1
        return self

    def run(self) -> "SplitSolver":
        return self.step(self.problem.n_steps - self.steps)

    def sync(self):
        for s in self.solvers:
            s.sync()

    def field(self, comp: int) -> np.ndarray:
        return assemble(self.split, [s.field(comp) for s in self.solvers])

    def traces(self) -> np.ndarray:
        return gather_probes(self.split, [s.traces() for s in self.solvers], len(self.problem.probes))

    def spectra(self) -> np.ndarray:
        return gather_probes(self.split, [s.spectra() for s in self.solvers], len(self.problem.probes))

    def close(self):
        for s in self.solvers:
            s.close()
        self.solvers = []


def exchange_ranks(split: Split, rank: int, pack: Callable[[int], object], unpack: Callable[[int, object], None],
                   send: Callable[[object, int], object], recv: Callable[[int, int], object],
                   wait: Callable[[List[object]], None]) -> None:
    """One halo exchange of part `rank` with its neighbours, one part per
    rank.  pack(local_plane) -> buffer; unpack(local_plane, buffer);
    send(buffer, peer) / recv(like_plane, peer) start the transfers and
    return handles that wait() completes.  The schedule is
    split.exchanges() seen from this rank."""
    sends, recvs = [], []
    for dst, dplane, src, splane in split.exchanges():
        if src == rank:
            sends.append(send(pack(splane), dst))
        if dst == rank:
            recvs.append((dplane, recv(dplane, src)))
    wait(sends + [h for _, h in recvs])
    for dplane, h in recvs:
        unpack(dplane, h)


class DistributedSplitSolver:
    """Part `rank` of one board on this rank's GPU; the halo planes travel by
    torch.distributed point-to-point transfers (NCCL: device buffers packed
    and unpacked by the library on the solver's stream; gloo: staged through
    host memory)."""

    def __init__(self, prob, rank: int, world: int, precision: str = "fp32", tuning: Optional[dict] = None):
        import torch
        from . import solver
        self.torch = torch
        self.problem = prob
        self.rank = rank
        self.split = split_y(prob, even_cuts(prob, world))
        self.part = self.split.parts[rank]
        # one stream for the library's work and the torch copies and
        # transfers of the exchange, so that they are ordered
        self.stream = torch.cuda.Stream()
        self.s = solver.Solver(self.part.problem, precision=precision, stream=self.stream, tuning=tuning)
        self.es = 4 if precision == "fp32" else 2
        self.dtype = torch.float32 if precision == "fp32" else torch.float16
        self.count = 2 * (prob.nx + 1) * (prob.nz + 1)
        self.steps = 0

    def _exchange(self):
        import torch.distributed as dist
        from . import capi as C
        torch = self.torch
        nccl = dist.get_backend() == "nccl"
        dev = torch.device("cuda", torch.cuda.current_device())

        def pack(plane):
            buf = torch.empty(self.count, dtype=self.dtype, device=dev)
            C.fdtd_halo_pack(self.s.ctx, 1, plane, TANGENTIAL_Y, buf.data_ptr())
            return buf if nccl else buf.cpu()

        def unpack(plane, h):
            buf = h[1] if nccl else h[1].to(dev)
            C.fdtd_halo_unpack(self.s.ctx, 1, plane, TANGENTIAL_Y, buf.data_ptr())

        def send(buf, peer):
            return (dist.isend(buf, peer), buf)

        def recv(plane, peer):
            buf = torch.empty(self.count, dtype=self.dtype, device=dev if nccl else "cpu")
            return (dist.irecv(buf, peer), buf)

        def wait(handles):
            for w, _ in handles:
                w.wait()

        with torch.cuda.stream(self.stream):
            exchange_ranks(self.split, self.rank, pack, unpack, send, recv, wait)

    def step(self, n: int) -> "DistributedSplitSolver":
        for _ in range(int(n)):
            self.s.step(1)
            self._exchange()
            self.steps += 1
        return self

    def close(self):
        self.s.close()
