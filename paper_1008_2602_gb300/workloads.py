"""Seeded synthetic inputs: PCB stacks, test cavities, sources and probes.

This module only builds *inputs* (geometry, material ids, PEC boxes, source and
probe positions, run lengths).  It contains none of the method's arithmetic: no
time step, no UPML grading, no coefficients, no field update.  Both the FP64
oracle (``oracle/``) and the CUDA path consume the ``Problem`` it returns, so it
is the only code the two sides share.

Geometry follows the paper's model (Fig. 1 and the Model section): two (or more)
perfectly conducting power/ground sheets separated by a dielectric, the board
surrounded by an air gap, the whole domain terminated by a UPML backed by PEC.
Index conventions: cells ``(i, j, k)`` with ``0 <= i < nx`` etc.; the material
volume is stored ``[nz, ny, nx]`` with x fastest; a PEC box is a half-open cell
range ``(i0, i1, j0, j1, k0, k1)`` whose *closed* node box holds PEC edges (so
``k1 == k0`` describes a zero-thickness sheet on node plane ``k0``).
Component codes: 0 = x, 1 = y, 2 = z (an E edge starting at node ``(i, j, k)``).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

WALL_PEC = 0
WALL_PMC = 1

MM = 1e-3
PS = 1e-12


@dataclasses.dataclass
class Problem:
    """One board / test solve: everything both sides need, nothing computed."""

    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    dz: float
    courant: float
    mat: np.ndarray                  # uint8 [nz, ny, nx], x fastest
    eps_r: np.ndarray                # float64 [n_mat]
    pec_boxes: np.ndarray            # int32 [n_pec, 6]
    upml_depth: Tuple[int, ...]      # faces -x,+x,-y,+y,-z,+z
    walls: Tuple[int, ...]           # per face: WALL_PEC or WALL_PMC
    sources: np.ndarray              # int32 [n_src, 4]  (i, j, k, comp)
    source_params: np.ndarray        # float64 [n_src, 3] (J0 [A/m^2], t0 [s], tau [s])
    probes: np.ndarray               # int32 [n_probe, 4] (i, j, k, comp)
    n_steps: int
    f_max: Optional[float] = None    # spectrum up to f_max; None = up to Nyquist
    upml_m: float = 3.0
    upml_R0: float = 1e-6
    upml_kappa_max: float = 1.0
    dt: float = 0.0                  # > 0 overrides the Courant number
    name: str = ""
    board: Optional[Tuple[int, int, int, int]] = None   # (i0, i1, j0, j1) board cells
    dielectric_k: Optional[List[Tuple[int, int]]] = None  # per pair: (k0, k1) cell range
    # resistive voltage sources: int32 [n, 4] (i, j, k, comp) and float64 [n, 4]
    # (V0 [V], t0 [s], tau [s], Rs [ohm]), same pulse shape as Eq. 8
    vsources: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros((0, 4), np.int32))
    vsource_params: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros((0, 4), np.float64))

    @property
    def cells(self) -> int:
        return self.nx * self.ny * self.nz

    def replace(self, **kw) -> "Problem":
        return dataclasses.replace(self, **kw)


# ---------------------------------------------------------------------------
# PCB stack (Fig. 1): sheets / dielectric / air gap / UPML
# ---------------------------------------------------------------------------

def pcb_stack(*, board_cells: Tuple[int, int], layers: Sequence[Tuple[str, int, float]],
              air: Tuple[int, int, int], upml: Tuple[int, int, int],
              d: Tuple[float, float, float], courant: float = 0.99,
              sheet_thickness: int = 1) -> Tuple[Problem, dict]:
    """Build the material volume and PEC boxes of a board stack.

    ``layers`` is listed bottom to top; each entry is ``("pec", 0, 0)`` for a
    power/ground sheet or ``("diel", n_cells, eps_r)`` for a dielectric slab.
    Sheets are ``sheet_thickness`` cells thick (0 gives a zero-thickness sheet
    on a node plane).  ``air`` and ``upml`` give cells on each side per axis.
    Returns the problem (without sources/probes) and layout info.
    """
    bx, by = board_cells
    ax, ay, az = air
    px, py, pz = upml
    stack_h = sum((sheet_thickness if kind == "pec" else n) for kind, n, _ in layers)
    nx = 2 * px + 2 * ax + bx
    ny = 2 * py + 2 * ay + by
    nz = 2 * pz + 2 * az + stack_h
    i0, j0 = px + ax, py + ay
    i1, j1 = i0 + bx, j0 + by
    eps_list = [1.0]
    mat = np.zeros((nz, ny, nx), dtype=np.uint8)
    boxes = []
    diel = []
    k = pz + az
    pair_start = None
    for kind, n, eps in layers:
        if kind == "pec":
            boxes.append((i0, i1, j0, j1, k, k + sheet_thickness))
            k += sheet_thickness
            if pair_start is None:
                pair_start = k
            else:
                diel.append((pair_start, k - sheet_thickness))
                pair_start = None
        else:
            if float(eps) in eps_list:
                mid = eps_list.index(float(eps))
            else:
                eps_list.append(float(eps))
                mid = len(eps_list) - 1
            mat[k:k + n, j0:j1, i0:i1] = mid
            k += n
    prob = Problem(nx=nx, ny=ny, nz=nz, dx=d[0], dy=d[1], dz=d[2], courant=courant,
                   mat=mat, eps_r=np.asarray(eps_list, dtype=np.float64),
                   pec_boxes=np.asarray(boxes, dtype=np.int32).reshape(-1, 6),
                   upml_depth=(px, px, py, py, pz, pz), walls=(WALL_PEC,) * 6,
                   sources=np.zeros((0, 4), np.int32), source_params=np.zeros((0, 3)),
                   probes=np.zeros((0, 4), np.int32), n_steps=0,
                   board=(i0, i1, j0, j1), dielectric_k=diel)
    return prob, {"board": (i0, i1, j0, j1), "dielectric_k": diel}


def _pick_ez_edges(rng: np.random.Generator, prob: Problem, n: int,
                   pair: Optional[int] = None) -> np.ndarray:
    """Seeded z-edges strictly inside the board, inside a pair's dielectric."""
    i0, i1, j0, j1 = prob.board
    out = []
    for t in range(n):
        p = pair if pair is not None else int(rng.integers(len(prob.dielectric_k)))
        k0, k1 = prob.dielectric_k[p]
        i = int(rng.integers(i0 + 1, i1))
        j = int(rng.integers(j0 + 1, j1))
        k = int(rng.integers(k0, k1))
        out.append((i, j, k, 2))
    return np.asarray(out, dtype=np.int32).reshape(-1, 4)


def _with_ports(prob: Problem, rng: np.random.Generator, n_src: int, n_probe: int,
                t0: float, tau: float, J0: float = 1e6) -> Problem:
    src = _pick_ez_edges(rng, prob, n_src)
    prm = np.tile(np.array([[J0, t0, tau]], dtype=np.float64), (n_src, 1))
    prb = _pick_ez_edges(rng, prob, n_probe)
    return prob.replace(sources=src, source_params=prm, probes=prb)


# ---------------------------------------------------------------------------
# The five workloads
# ---------------------------------------------------------------------------

def small_pcb(seed: int = 1, n_steps: int = 2000) -> Problem:
    """Small PCB: 56x48x30, dx=dy=1 mm, dz=0.25 mm; 32x24 mm sheets, 4 cells of
    eps_r=4.4 between them, 4-cell air gap, 8-cell UPML (m=3, R0=1e-6); one
    z-directed Gaussian-derivative source (t0=40 ps, tau=15 ps) and 4 Ez probes
    between the planes, Courant 0.99, 2000 steps, spectra up to Nyquist."""
    rng = np.random.default_rng(seed)
    prob, _ = pcb_stack(board_cells=(32, 24), layers=[("pec", 0, 0), ("diel", 4, 4.4), ("pec", 0, 0)],
                        air=(4, 4, 4), upml=(8, 8, 8), d=(1 * MM, 1 * MM, 0.25 * MM))
    assert (prob.nx, prob.ny, prob.nz) == (56, 48, 30)
    prob = _with_ports(prob, rng, 1, 4, 40 * PS, 15 * PS)
    return prob.replace(n_steps=n_steps, f_max=None, name="small_pcb_56x48x30")


def realistic_board(seed: int = 2, n_steps: int = 20000) -> Problem:
    """Realistic board: 100x80 mm plane pair, dx=dy=0.5 mm, dz=0.2 mm, 5-cell
    FR4 (eps_r=4.4), 6-cell air gap, 10-cell UPML -> 232x192x39 cells; three
    seeded sources, 16 probes, 20000 steps, running DFT to 10 GHz."""
    rng = np.random.default_rng(seed)
    prob, _ = pcb_stack(board_cells=(200, 160), layers=[("pec", 0, 0), ("diel", 5, 4.4), ("pec", 0, 0)],
                        air=(6, 6, 6), upml=(10, 10, 10), d=(0.5 * MM, 0.5 * MM, 0.2 * MM))
    prob = _with_ports(prob, rng, 3, 16, 40 * PS, 15 * PS)
    return prob.replace(n_steps=n_steps, f_max=10e9, name="realistic_board_232x192x39")


def multilayer_board(seed: int = 3, n_steps: int = 50000, scale: int = 1,
                     n_src: int = 4, n_probe: int = 64) -> Problem:
    """Large multilayer board: 200x150 mm, four power/ground pairs with seeded
    eps_r in [3.5, 4.6] (6-cell dielectric per pair, 8-cell cores between
    pairs, also seeded), dx=dy=0.25 mm, dz=0.1 mm, 28-cell air gap in x/y and
    10 in z, 12-cell UPML -> 880x680x100 cells.  ``scale=4`` gives the
    quarter-scale copy (x and y board extent divided by 4, same stack)."""
    rng = np.random.default_rng(seed)
    eps = rng.uniform(3.5, 4.6, size=7)
    layers = []
    for p in range(4):
        layers += [("pec", 0, 0), ("diel", 6, float(eps[p])), ("pec", 0, 0)]
        if p < 3:
            layers.append(("diel", 8, float(eps[4 + p])))
    bx, by = 800 // scale, 600 // scale
    prob, _ = pcb_stack(board_cells=(bx, by), layers=layers, air=(28, 28, 10), upml=(12, 12, 12),
                        d=(0.25 * MM, 0.25 * MM, 0.1 * MM))
    prob = _with_ports(prob, rng, n_src, n_probe, 40 * PS, 15 * PS)
    tag = "" if scale == 1 else f"_scale1_{scale}"
    return prob.replace(n_steps=n_steps, f_max=10e9,
                        name=f"multilayer_board_{prob.nx}x{prob.ny}x{prob.nz}{tag}")


def batch_board(rng: np.random.Generator, *, dxy: float = 0.5 * MM, dz: float = 0.2 * MM,
                n_steps: int = 5000, n_probe: int = 4, size_mm=(20.0, 120.0),
                pairs=(1, 3), air=(6, 6, 6), upml=(10, 10, 10)) -> Problem:
    """One board of the batched workload: plane sides uniform in ``size_mm``,
    1-3 plane pairs (5-cell dielectric, 5-cell cores), eps_r uniform in
    [3.5, 4.6], one source and ``n_probe`` probes at seeded positions."""
    lx = rng.uniform(*size_mm)
    ly = rng.uniform(*size_mm)
    n_pairs = int(rng.integers(pairs[0], pairs[1] + 1))
    layers = []
    for p in range(n_pairs):
        layers += [("pec", 0, 0), ("diel", 5, float(rng.uniform(3.5, 4.6))), ("pec", 0, 0)]
        if p < n_pairs - 1:
            layers.append(("diel", 5, float(rng.uniform(3.5, 4.6))))
    bx = max(4, int(round(lx * MM / dxy)))
    by = max(4, int(round(ly * MM / dxy)))
    prob, _ = pcb_stack(board_cells=(bx, by), layers=layers, air=air, upml=upml, d=(dxy, dxy, dz))
    prob = _with_ports(prob, rng, 1, n_probe, 40 * PS, 15 * PS)
    return prob.replace(n_steps=n_steps, f_max=10e9, name=f"board_{prob.nx}x{prob.ny}x{prob.nz}")


def batch_boards(seed: int = 4, n_boards: int = 64, n_steps: int = 5000, **kw) -> List[Problem]:
    """Batched workload: ``n_boards`` uneven boards (plane sides 20-120 mm,
    1-3 pairs, dx=dy=0.5 mm, dz=0.2 mm, 6-cell air, 10-cell UPML), 5000 steps."""
    rng = np.random.default_rng(seed)
    return [batch_board(rng, n_steps=n_steps, **kw) for _ in range(n_boards)]


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float      # seconds from stream start
    problem: Problem


def request_stream(seed: int = 5, n_requests: int = 200, rate: float = 20.0,
                   median_cells: float = 2e6, max_cells: float = 40e6, sigma: float = 0.97,
                   steps=(2000, 20000), probes=(4, 32), step_scale: float = 1.0,
                   cell_scale: float = 1.0) -> List[Request]:
    """Served workload: Poisson arrivals (mean ``rate`` req/s); each request is
    a multilayer board (dx=dy=0.25 mm, dz=0.1 mm, 1-4 pairs, seeded eps_r)
    whose cell count is lognormal (median 2M, truncated at 40M), with 2000-20000
    steps and 4-32 probes.  ``step_scale``/``cell_scale`` shrink a stream
    uniformly for short runs (stated wherever used)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for r in range(n_requests):
        t += float(rng.exponential(1.0 / rate))
        cells = min(max_cells, float(np.exp(np.log(median_cells) + sigma * rng.standard_normal())))
        cells *= cell_scale
        n_pairs = int(rng.integers(1, 5))
        layers = []
        for p in range(n_pairs):
            layers += [("pec", 0, 0), ("diel", 6, float(rng.uniform(3.5, 4.6))), ("pec", 0, 0)]
            if p < n_pairs - 1:
                layers.append(("diel", 8, float(rng.uniform(3.5, 4.6))))
        stack = 8 * n_pairs + 8 * (n_pairs - 1)
        nz = 24 + 20 + stack
        aspect = float(rng.uniform(0.6, 1.0))
        plane = max(64.0, cells / nz)
        nxy_x = math.sqrt(plane / aspect)
        bx = max(8, int(nxy_x) - 80)
        by = max(8, int(nxy_x * aspect) - 80)
        prob, _ = pcb_stack(board_cells=(bx, by), layers=layers, air=(28, 28, 10), upml=(12, 12, 12),
                            d=(0.25 * MM, 0.25 * MM, 0.1 * MM))
        n_steps = int(max(16, round(rng.integers(steps[0], steps[1] + 1) * step_scale)))
        n_probe = int(rng.integers(probes[0], probes[1] + 1))
        prob = _with_ports(prob, rng, 1, n_probe, 40 * PS, 15 * PS)
        prob = prob.replace(n_steps=n_steps, f_max=10e9, name=f"req{r}_{prob.nx}x{prob.ny}x{prob.nz}")
        out.append(Request(rid=r, arrival=t, problem=prob))
    return out


# ---------------------------------------------------------------------------
# Test geometries used by the pins
# ---------------------------------------------------------------------------

def box(nx: int, ny: int, nz: int, d=(1 * MM, 1 * MM, 1 * MM), eps_r: float = 1.0,
        walls=(WALL_PEC,) * 6, upml=(0,) * 6, courant: float = 0.99) -> Problem:
    """Homogeneous box with the given walls and UPML depths, no sources."""
    mat = np.zeros((nz, ny, nx), np.uint8)
    eps = np.array([eps_r], np.float64)
    return Problem(nx=nx, ny=ny, nz=nz, dx=d[0], dy=d[1], dz=d[2], courant=courant, mat=mat,
                   eps_r=eps, pec_boxes=np.zeros((0, 6), np.int32), upml_depth=tuple(upml),
                   walls=tuple(walls), sources=np.zeros((0, 4), np.int32),
                   source_params=np.zeros((0, 3)), probes=np.zeros((0, 4), np.int32), n_steps=0,
                   name=f"box_{nx}x{ny}x{nz}")


def add_ports(prob: Problem, sources: Sequence[Tuple[int, int, int, int]],
              probes: Sequence[Tuple[int, int, int, int]], J0: float = 1e6,
              t0: float = 40 * PS, tau: float = 15 * PS, n_steps: int = 0,
              f_max: Optional[float] = None) -> Problem:
    src = np.asarray(sources, np.int32).reshape(-1, 4)
    prm = np.tile(np.array([[J0, t0, tau]], np.float64), (len(src), 1))
    return prob.replace(sources=src, source_params=prm,
                        probes=np.asarray(probes, np.int32).reshape(-1, 4),
                        n_steps=n_steps or prob.n_steps, f_max=f_max)


def add_voltage_sources(prob: Problem, edges: Sequence[Tuple[int, int, int, int]], V0: float = 5.0,
                        t0: float = 40 * PS, tau: float = 15 * PS, Rs: float = 10.0) -> Problem:
    """Append resistive voltage sources (amplitude V0, series resistance Rs)."""
    e = np.asarray(edges, np.int32).reshape(-1, 4)
    prm = np.tile(np.array([[V0, t0, tau, Rs]], np.float64), (len(e), 1))
    return prob.replace(vsources=np.vstack([np.asarray(prob.vsources, np.int32).reshape(-1, 4), e]),
                        vsource_params=np.vstack([np.asarray(prob.vsource_params, np.float64).reshape(-1, 4), prm]))


def table1_board(n_steps: int = 30000, air=(3, 3, 3), upml=(6, 6, 6)) -> Problem:
    """The Table 1 run of the Results section: a 40 x 30 x 0.8 mm board of
    eps_r = 4.0 (the value that reproduces the table's predicted column; the
    paper does not state it) between two zero-thickness PEC sheets, 2/2/0.4 mm
    cells, dt = 1 ps, a resistive voltage source (V0 = 5 V, Rs = 10 ohm, the
    Eq. 8 pulse shape with t0 = 100 ps, tau = 50 ps as stated for the current
    source) on the E_z edge at one corner of the board and the E_z probe at
    the opposite corner; air gap and UPML sizes are not given (defaults here)."""
    p, _ = pcb_stack(board_cells=(20, 15), layers=[("pec", 0, 0), ("diel", 2, 4.0), ("pec", 0, 0)],
                     air=air, upml=upml, d=(2 * MM, 2 * MM, 0.4 * MM), sheet_thickness=0)
    i0, i1, j0, j1 = p.board
    k0, _ = p.dielectric_k[0]
    p = add_ports(p, [], [(i1 - 1, j1 - 1, k0, 2)], n_steps=n_steps).replace(dt=1e-12, name="table1_board")
    return add_voltage_sources(p, [(i0 + 1, j0 + 1, k0, 2)], V0=5.0, t0=100 * PS, tau=50 * PS, Rs=10.0)


def fig3_board(n_steps: int = 1000, eps_r: float = 4.0, air=(3, 3, 3), upml=(8, 8, 6)) -> Problem:
    """The board of the Results section's Figs. 3-4: 100 x 60 x 0.8 mm, 2/2/0.4
    mm cells, dt = 1 ps, current source (Eq. 8, J0 = 1 A/mm^2, t0 = 100 ps,
    tau = 50 ps) on the E_z edge at the centre of the board, UPML around it.
    eps_r, the air gap and the UPML depth are not given (defaults here; eps_r
    as read for Table 1).  The grid is mirror-symmetric about the source."""
    p, _ = pcb_stack(board_cells=(50, 30), layers=[("pec", 0, 0), ("diel", 2, eps_r), ("pec", 0, 0)],
                     air=air, upml=upml, d=(2 * MM, 2 * MM, 0.4 * MM), sheet_thickness=0)
    k0, _ = p.dielectric_k[0]
    ic, jc = p.nx // 2, p.ny // 2
    return add_ports(p, [(ic, jc, k0, 2)], [(ic, jc, k0, 2)], J0=1e6, t0=100 * PS, tau=50 * PS,
                     n_steps=n_steps).replace(dt=1e-12, name="fig3_board")


def zrefine_board(nz_d: int, dt: float, n_steps: int, eps_r: float = 4.0, board_cells=(20, 15),
                  air_xy: int = 3, upml_xy: int = 6, air_z_mm: float = 2.4, upml_z_mm: float = 4.8) -> Problem:
    """The z-convergence model of the Results section: a 40 x 30 mm plane pair
    with a 0.8 mm dielectric cut into nz_d cells (2 mm cells in x and y); the
    air above and below and the z UPML keep their thickness in mm (rounded to
    whole cells), so only the board's z discretisation changes.
    The current source is a filament across the whole gap (every E_z edge of
    the dielectric at one corner carries J0 = 1 A/mm^2 with the Eq. 8 pulse,
    t0 = 100 ps, tau = 50 ps), so its total current does not depend on the
    cutting; the probes are every E_z edge of the column at the opposite corner,
    whose sum times dz is the voltage between the planes."""
    dz = 0.8 * MM / nz_d
    az, uz = int(round(air_z_mm * MM / dz)), int(round(upml_z_mm * MM / dz))
    p, _ = pcb_stack(board_cells=board_cells, layers=[("pec", 0, 0), ("diel", nz_d, eps_r), ("pec", 0, 0)],
                     air=(air_xy, air_xy, az), upml=(upml_xy, upml_xy, uz), d=(2 * MM, 2 * MM, dz),
                     sheet_thickness=0)
    i0, i1, j0, j1 = p.board
    k0, k1 = p.dielectric_k[0]
    src = [(i0 + 1, j0 + 1, k, 2) for k in range(k0, k1)]
    prb = [(i1 - 1, j1 - 1, k, 2) for k in range(k0, k1)]
    return add_ports(p, src, prb, J0=1e6, t0=100 * PS, tau=50 * PS, n_steps=n_steps).replace(
        dt=dt, name=f"zrefine_{nz_d}")


def random_problem(seed: int, nx: int, ny: int, nz: int, upml: int = 3, n_mat: int = 3,
                   n_src: int = 2, n_probe: int = 4, n_steps: int = 60,
                   d=(1 * MM, 1.5 * MM, 0.5 * MM)) -> Problem:
    """Small random-material grid (for parity at odd sizes): random eps_r per
    cell from ``n_mat`` materials, one random PEC box, UPML on all faces."""
    rng = np.random.default_rng(seed)
    mat = rng.integers(0, n_mat, size=(nz, ny, nx)).astype(np.uint8)
    eps = np.concatenate([[1.0], rng.uniform(2.0, 6.0, size=n_mat - 1)])
    # ports on edges whose every coordinate is outside the UPML: node index in
    # [upml, n - upml - 1] along each axis
    def port(n):
        m = max(upml, 1)   # also keep off the outer PEC walls
        return int(rng.integers(m, max(m + 1, n - m)))
    lo = upml + 1
    bi = sorted(rng.integers(lo, max(lo + 1, nx - upml - 1), size=2))
    bj = sorted(rng.integers(lo, max(lo + 1, ny - upml - 1), size=2))
    kk = int(rng.integers(lo, max(lo + 1, nz - upml - 1)))
    boxes = np.array([[bi[0], bi[1] + 1, bj[0], bj[1] + 1, kk, kk]], np.int32)
    src, prb = [], []
    ks = [k for k in range(max(upml, 1), nz - max(upml, 1)) if k != kk] or [max(upml, 1)]
    for _ in range(n_src):
        src.append((port(nx), port(ny), int(ks[int(rng.integers(len(ks)))]), int(rng.integers(0, 3))))
    for _ in range(n_probe):
        prb.append((int(rng.integers(1, nx)), int(rng.integers(1, ny)), int(rng.integers(1, nz)),
                    int(rng.integers(0, 3))))
    prob = Problem(nx=nx, ny=ny, nz=nz, dx=d[0], dy=d[1], dz=d[2], courant=0.95, mat=mat, eps_r=eps,
                   pec_boxes=boxes, upml_depth=(upml,) * 6, walls=(WALL_PEC,) * 6,
                   sources=np.asarray(src, np.int32), source_params=np.zeros((0, 3)),
                   probes=np.asarray(prb, np.int32), n_steps=n_steps, name=f"random_{nx}x{ny}x{nz}_s{seed}")
    prm = np.stack([rng.uniform(0.5e6, 2e6, n_src), np.full(n_src, 30 * PS), np.full(n_src, 10 * PS)], axis=1)
    return prob.replace(source_params=prm)
