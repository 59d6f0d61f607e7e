"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle (``oracle/fdtd_oracle.c``) against something other
than itself: printed values of the paper (Table 1, tests/golden/), closed forms
(Eq. 9 cavity, the Yee dispersion relation, the Fourier transform of the Eq. 8
pulse), exact discrete invariants (energy, energy balance with a source,
div B), the stability bound of Eq. 7, a large-domain reference for the UPML,
and symmetries (superposition, mirror).  A dropped term, wrong sign or index,
or transposed operand in the oracle breaks at least one of them.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1008_2602_gb300 import workloads as W

C0 = 299792458.0
PEC, PMC = W.WALL_PEC, W.WALL_PMC
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _table1():
    rows = []
    with open(os.path.join(GOLDEN, "table1_resonances.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            m, n, pred, label, model = line.split()
            rows.append((int(m), int(n), float(pred), label, float(model)))
    return rows


def _peak(x, dt, f_guess, pad=8, search=0.01):
    """Peak frequency near f_guess: Hann window, zero padding, log-parabola."""
    N = len(x)
    w = np.hanning(N)
    X = np.abs(np.fft.rfft(x * w, pad * N))
    f = np.fft.rfftfreq(pad * N, dt)
    lo, hi = np.searchsorted(f, f_guess * (1 - search)), np.searchsorted(f, f_guess * (1 + search))
    j = lo + int(np.argmax(X[lo:hi]))
    a, b, c = np.log(X[j - 1]), np.log(X[j]), np.log(X[j + 1])
    d = 0.5 * (a - c) / (a - 2 * b + c)
    return (j + d) / (pad * N * dt), X[j] / X.max()


# --------------------------------------------------------------------------
# Paper's printed numbers
# --------------------------------------------------------------------------

def test_eq9_reproduces_table1_predictions():
    """Eq. 9 with Lx=40, Ly=30, Lz=0.8 mm and eps_r=4.0 gives Table 1's
    'Predicted' column to its printed precision (0.01 GHz)."""
    for m, n, pred, _, _ in _table1():
        f = oracle.cavity_fr(m, n, 40e-3, 30e-3, 0.8e-3, 4.0) / 1e9
        assert abs(f - pred) <= 0.011, (m, n, f, pred)
    # eps_r = 4.4 (the FR4 value of the other runs) does not reproduce it
    worst = max(abs(oracle.cavity_fr(m, n, 40e-3, 30e-3, 0.8e-3, 4.4) / 1e9 - p) for m, n, p, _, _ in _table1())
    assert worst > 0.3


def test_cfl_dt_matches_eq7_and_paper_grid():
    """Eq. 7 at the paper's 2/2/0.4 mm grid: 1.284 ps (the text quotes 1.33 ps,
    which is dz/c alone); the 1 ps step used in the paper is below it."""
    dt = oracle.cfl_dt(2e-3, 2e-3, 0.4e-3)
    assert abs(dt - 1.2837e-12) < 1e-15
    assert abs(0.4e-3 / C0 - 1.334e-12) < 1e-15
    # cubic grid: dx / (c sqrt 3)
    assert abs(oracle.cfl_dt(1e-3, 1e-3, 1e-3) - 1e-3 / (C0 * np.sqrt(3))) < 1e-24


@pytest.mark.slow
def test_table1_board_run_lands_near_paper(ncpu):
    """Coarse reproduction of the Table 1 run (40x30x0.8 mm board, 2/2/0.4 mm
    cells, dt = 1 ps, 30000 steps, source at one corner, probe at the opposite
    one, air gap + UPML whose sizes the paper does not give).  The paper's own
    modelled peaks sit -3.6 %..+1.9 % from Eq. 9; for the five lowest isolated
    modes the nearest spectral peak of the oracle must sit in that band
    widened by 1 % on each side, and no peak may lie below the fundamental."""
    p, _ = W.pcb_stack(board_cells=(20, 15), layers=[("pec", 0, 0), ("diel", 2, 4.0), ("pec", 0, 0)],
                       air=(3, 3, 3), upml=(6, 6, 6), d=(2e-3, 2e-3, 0.4e-3), sheet_thickness=0)
    i0, i1, j0, j1 = p.board
    k0, _ = p.dielectric_k[0]
    p = W.add_ports(p, [(i0 + 1, j0 + 1, k0, 2)], [(i1 - 1, j1 - 1, k0, 2)], n_steps=30000).replace(dt=1e-12)
    r = oracle.run(p, dft=False, n_threads=ncpu)
    x, dt = r["trace"][0], r["dt"]
    pad = 4
    X = np.abs(np.fft.rfft(x * np.hanning(len(x)), pad * len(x)))
    f = np.fft.rfftfreq(pad * len(x), dt)
    peaks = np.array([f[j] for j in range(1, len(X) - 1)
                      if X[j] > X[j - 1] and X[j] > X[j + 1] and X[j] > 0.01 * X.max() and f[j] < 10.5e9])
    rows = {(m, n): pred * 1e9 for m, n, pred, _, _ in _table1()}
    for mode in [(1, 0), (0, 1), (2, 0), (0, 2), (3, 0)]:
        pred = rows[mode]
        near = peaks[np.argmin(np.abs(peaks - pred))]
        dev = (near - pred) / pred
        assert -0.046 <= dev <= 0.029, (mode, near, pred, dev)
    assert peaks.min() > 0.9 * rows[(1, 0)]


# --------------------------------------------------------------------------
# Closed forms
# --------------------------------------------------------------------------

def _cavity(nx, ny, nz, d, eps_r, n_steps, src, prb):
    p = W.box(nx, ny, nz, d=d, eps_r=eps_r, walls=(PMC, PMC, PMC, PMC, PEC, PEC))
    return W.add_ports(p, [src], [prb], n_steps=n_steps)


def test_cavity_resonances_match_eq9_closed_form(ncpu):
    """PEC top/bottom + four PMC walls (the paper's cavity model): TM_mn0 peaks
    within one FFT bin of f_mn = c/(2 sqrt(eps_r)) sqrt((m/a)^2 + (n/b)^2), and
    within 2e-4 of the exact Yee dispersion relation
    sin(w dt/2)/(v dt) = sqrt(sum_w sin^2(k_w d_w/2)/d_w^2), k = m pi / a."""
    nx, ny, nz, d, er = 40, 30, 2, (1e-3, 1e-3, 0.4e-3), 4.0
    r = oracle.run(_cavity(nx, ny, nz, d, er, 16000, (3, 4, 0, 2), (33, 23, 1, 2)), dft=False, n_threads=ncpu)
    x, dt = r["trace"][0], r["dt"]
    a, b = nx * d[0], ny * d[1]
    v = C0 / np.sqrt(er)
    bin_hz = 1.0 / (len(x) * dt)
    checked = 0
    for m, n in [(1, 0), (0, 1), (1, 1), (2, 0), (2, 1), (0, 2), (1, 2), (3, 0)]:
        fc = oracle.cavity_fr(m, n, a, b, 0.0, er)
        assert abs(fc - v / 2 * np.hypot(m / a, n / b)) < 1e-6 * fc
        s = np.sqrt((np.sin(m * np.pi / (2 * nx)) / d[0]) ** 2 + (np.sin(n * np.pi / (2 * ny)) / d[1]) ** 2)
        fd = np.arcsin(v * dt * s) / (np.pi * dt)
        f, amp = _peak(x, dt, fd)
        assert amp > 1e-3, (m, n)
        assert abs(f - fd) / fd < 2e-4, (m, n, f, fd)
        assert abs(f - fc) < bin_hz, (m, n, f, fc, bin_hz)
        checked += 1
    assert checked == 8


@pytest.mark.parametrize("layers", [[2.0, 8.0], [3.0, 3.0, 6.0, 9.0]])
def test_layered_cavity_series_permittivity(layers, ncpu):
    """Thin z-layered dielectric between PEC plates with PMC side walls: in the
    quasi-static limit the layers act as series capacitors, so the TM_mn0
    peaks follow Eq. 9 (no fringing) with 1/eps_eff = mean_k(1/eps_k), to 1 %.
    Pins the per-edge permittivity (E_z edges inside a layer, E_x/E_y edges on
    a layer interface)."""
    nz, nx, ny, d = len(layers), 40, 30, (1e-3, 1e-3, 0.1e-3)
    p = W.box(nx, ny, nz, d=d, walls=(PMC, PMC, PMC, PMC, PEC, PEC)).replace(eps_r=np.array(layers))
    for k in range(nz):
        p.mat[k] = k
    p = W.add_ports(p, [(3, 4, 0, 2)], [(33, 23, nz - 1, 2)], n_steps=16000)
    r = oracle.run(p, dft=False, n_threads=ncpu)
    eps_eff = 1.0 / np.mean(1.0 / np.asarray(layers))
    for m, n in [(1, 0), (0, 1), (1, 1), (2, 0)]:
        fq = oracle.cavity_fr(m, n, nx * d[0], ny * d[1], 0.0, eps_eff)
        f, amp = _peak(r["trace"][0], r["dt"], fq, search=0.05)
        assert amp > 1e-2
        assert abs(f - fq) / fq < 0.01, (m, n, f, fq)


def test_pulse_matches_its_fourier_transform():
    """The sampled Eq. 8 pulse J0 u exp(-u^2), u = (t - t0)/tau: its DFT equals
    the analytic transform -j J0 tau (sqrt(pi) w tau / 2) exp(-(w tau/2)^2)
    exp(-j w t0); it has zero mean and its peak J0 exp(-1/2)/sqrt(2) at
    u = 1/sqrt(2).  t0 = 6 tau so that the pulse is negligible at t = 0."""
    p = W.box(6, 6, 6)
    p = W.add_ports(p, [(3, 3, 3, 2)], [(3, 3, 3, 2)], J0=2.5e6, t0=300e-12, tau=50e-12, n_steps=1200)
    r = oracle.run(p, src_wave=True, dft=False)
    J, dt = r["src_wave"], r["dt"]
    t = (np.arange(len(J)) + 0.5) * dt
    J0, t0, tau = 2.5e6, 300e-12, 50e-12
    for f in [0.5e9, 2e9, 5e9, 9e9]:
        w = 2 * np.pi * f
        num = dt * np.sum(J * np.exp(-1j * w * t))
        ana = -1j * J0 * tau * (np.sqrt(np.pi) * w * tau / 2) * np.exp(-(w * tau / 2) ** 2) * np.exp(-1j * w * t0)
        assert abs(num - ana) < 1e-6 * J0 * tau, (f, num, ana)
    assert abs(J.sum()) < 1e-9 * np.abs(J).sum()
    assert abs(J.max() - J0 * np.exp(-0.5) / np.sqrt(2)) < 1e-3 * J0
    assert abs(t[np.argmax(J)] - (t0 + tau / np.sqrt(2))) < dt


def test_running_dft_equals_fft():
    """The FP64 running DFT equals dt * FFT of the stored trace (same bins)."""
    p = W.random_problem(7, 14, 12, 10, n_steps=300)
    r = oracle.run(p, trace=True, dft=True)
    ref = r["dt"] * np.fft.fft(r["trace"], axis=1)[:, : r["spectra"].shape[1]]
    assert np.abs(r["spectra"] - ref).max() <= 1e-12 * np.abs(ref).max()
    assert r["spectra"].shape[1] == 300 // 2 + 1


# --------------------------------------------------------------------------
# Exact discrete invariants
# --------------------------------------------------------------------------

def _pec_box_with_dielectric():
    p = W.box(12, 10, 8, d=(1e-3, 1.2e-3, 0.7e-3)).replace(eps_r=np.array([1.0, 3.0]))
    p.mat[3:6, 2:8, 3:9] = 1
    return W.add_ports(p, [(5, 5, 4, 2), (6, 3, 2, 0)], [(5, 5, 4, 2), (6, 3, 2, 0)], n_steps=3000)


def test_energy_conserved_in_lossless_pec_box():
    """Source-free lossless PEC box: W^n is constant to round-off once the
    pulse has died away (t > t0 + 8 tau)."""
    r = oracle.run(_pec_box_with_dielectric(), energy=True, dft=False)
    e = r["energy"][600:]
    assert e.mean() > 0
    assert (e.max() - e.min()) / e.mean() < 1e-12


def test_energy_balance_with_sources():
    """Discrete Poynting theorem of the Yee scheme with currents:
    W^{n+1} - W^n = -(dt/2) V sum_s J_s^{n+1/2} (E_s^n + E_s^{n+1})."""
    p = _pec_box_with_dielectric()
    r = oracle.run(p, energy=True, dft=False)
    dt, V = r["dt"], p.dx * p.dy * p.dz
    t = (np.arange(p.n_steps) + 0.5) * dt
    pred = 0.0
    for s in range(2):
        J0, t0, tau = p.source_params[s]
        u = (t - t0) / tau
        Js = J0 * u * np.exp(-u * u)
        e_new = r["trace"][s]
        e_old = np.concatenate([[0.0], e_new[:-1]])
        pred = pred - 0.5 * dt * V * Js * (e_old + e_new)
    dW = np.diff(r["energy"])
    assert np.abs(dW - pred[:-1]).max() < 1e-12 * np.abs(dW).max()


def test_energy_conserved_with_pmc_walls():
    """With PMC side walls (odd mirror of tangential H) W^n is conserved too,
    with half dual cells on the wall planes."""
    p = _cavity(16, 12, 3, (1e-3, 1e-3, 0.5e-3), 2.0, 1500, (3, 5, 1, 2), (10, 7, 1, 2))
    r = oracle.run(p, energy=True, dft=False)
    e = r["energy"][400:]
    assert (e.max() - e.min()) / e.mean() < 1e-12


def test_div_b_stays_zero_outside_upml(ncpu):
    """B is updated by a discrete curl, so div B stays at round-off in every
    cell outside the UPML (random materials, PEC sheet, several sources)."""
    p = W.random_problem(3, 20, 18, 16, upml=4, n_steps=200)
    r = oracle.run(p, divb=True, fields=True, dft=False, n_threads=ncpu)
    H = r["fields"][3:]
    mu0 = 4e-7 * np.pi
    scale = mu0 * np.abs(H).max() / min(p.dx, p.dy, p.dz)
    assert scale > 0
    assert r["divb"].max() < 1e-12 * scale


def test_courant_above_eq7_is_unstable():
    """Eq. 7 is the stability bound: Courant 0.99 stays bounded, 1.02 grows
    without bound from round-off."""
    base = W.add_ports(W.box(10, 9, 8), [(5, 4, 4, 2)], [(3, 3, 3, 2)], n_steps=1500)
    ok = oracle.run(base, energy=True, dft=False)
    bad = oracle.run(base.replace(courant=1.02), energy=True, dft=False)
    assert ok["energy"][-1] < 1.001 * ok["energy"][400]
    assert not np.isfinite(bad["energy"][-1]) or bad["energy"][-1] > 1e6 * bad["energy"][400]


# --------------------------------------------------------------------------
# UPML against a large-domain reference
# --------------------------------------------------------------------------

def _reflection(small, big, shift, srcs, prb, n_steps, ncpu):
    a = oracle.run(W.add_ports(small, srcs, [prb], n_steps=n_steps), dft=False, n_threads=ncpu)["trace"][0]
    mv = lambda q: (q[0] + shift[0], q[1] + shift[1], q[2] + shift[2], q[3])
    b = oracle.run(W.add_ports(big, [mv(s) for s in srcs], [mv(prb)], n_steps=n_steps),
                   dft=False, n_threads=ncpu)["trace"][0]
    return 20 * np.log10(np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_upml_plane_wave_reflection_below_40db(axis, ncpu):
    """Normal-incidence TEM plane wave (sheet current between PEC walls with
    PMC side walls) into a 10-cell UPML on each axis: reflection < -40 dB."""
    L, pad, depth = 60, 400, 10
    d = (1e-3, 1e-3, 1e-3)
    if axis == 0:    # E_z, travelling in x
        walls, comp = (PEC, PEC, PMC, PMC, PEC, PEC), 2
        size = lambda n: (n, 1, 1)
        srcs = [(20, j, 0, comp) for j in (0, 1)]
        prb = (45, 0, 0, comp)
    elif axis == 1:  # E_z, travelling in y
        walls, comp = (PMC, PMC, PEC, PEC, PEC, PEC), 2
        size = lambda n: (1, n, 1)
        srcs = [(i, 20, 0, comp) for i in (0, 1)]
        prb = (0, 45, 0, comp)
    else:            # E_x, travelling in z
        walls, comp = (PEC, PEC, PMC, PMC, PEC, PEC), 0
        size = lambda n: (1, 1, n)
        srcs = [(0, j, 20, comp) for j in (0, 1)]
        prb = (0, 0, 45, comp)
    up = [0] * 6
    up[2 * axis] = up[2 * axis + 1] = depth
    small = W.box(*size(L), d=d, walls=walls, upml=tuple(up))
    big = W.box(*size(L + 2 * pad), d=d, walls=walls)
    shift = [0, 0, 0]
    shift[axis] = pad
    db = _reflection(small, big, shift, srcs, prb, 400, ncpu)
    assert db < -40, db
    # sensitivity: with R0 = 1 the layer has sigma = 0 and the PEC wall reflects
    db0 = _reflection(small.replace(upml_R0=1.0), big, shift, srcs, prb, 400, ncpu)
    assert db0 > -10, db0


@pytest.mark.parametrize("plane", ["xy", "xz"])
def test_upml_line_source_reflection_below_40db(plane, ncpu):
    """2D cylindrical wave from a line current at all angles of incidence into
    a 10-cell UPML on four faces: reflection < -40 dB."""
    d = (1e-3, 1e-3, 1e-3)
    if plane == "xy":
        small = W.box(40, 40, 1, d=d, upml=(10, 10, 10, 10, 0, 0))
        big = W.box(300, 300, 1, d=d)
        shift, src, prb = (130, 130, 0), (20, 20, 0, 2), (27, 24, 0, 2)
    else:
        small = W.box(40, 1, 40, d=d, upml=(10, 10, 0, 0, 10, 10))
        big = W.box(300, 1, 300, d=d)
        shift, src, prb = (130, 0, 130), (20, 0, 20, 1), (27, 0, 24, 1)
    db = _reflection(small, big, shift, [src], prb, 300, ncpu)
    assert db < -40, db


@pytest.mark.slow
def test_upml_point_source_3d_reflection_below_40db(ncpu):
    """3D point current, 8-cell UPML on all six faces, against a 110^3 domain
    whose walls are too far to return a reflection within the window."""
    d = (1e-3, 1e-3, 1e-3)
    small = W.box(32, 32, 32, d=d, upml=(8,) * 6)
    big = W.box(110, 110, 110, d=d)
    db = _reflection(small, big, (39, 39, 39), [(16, 16, 16, 2)], (22, 17, 18, 2), 130, ncpu)
    assert db < -40, db


# --------------------------------------------------------------------------
# Symmetries
# --------------------------------------------------------------------------

def test_superposition_and_scaling():
    """The scheme is linear: two sources together = sum of each alone, and
    doubling J0 doubles every trace."""
    p = W.random_problem(11, 16, 14, 12, n_steps=150)
    both = oracle.run(p, dft=False)["trace"]
    one = oracle.run(p.replace(sources=p.sources[:1], source_params=p.source_params[:1]), dft=False)["trace"]
    two = oracle.run(p.replace(sources=p.sources[1:], source_params=p.source_params[1:]), dft=False)["trace"]
    assert np.abs(both - (one + two)).max() <= 1e-12 * np.abs(both).max()
    prm = p.source_params.copy()
    prm[:, 0] *= 2
    dbl = oracle.run(p.replace(source_params=prm), dft=False)["trace"]
    assert np.abs(dbl - 2 * both).max() <= 1e-12 * np.abs(dbl).max()


def test_mirror_symmetry():
    """Symmetric grid (UPML on all faces, z-layered dielectric), source on the
    central node column: E_z is even and E_x odd under x -> 20 - x."""
    p = W.box(20, 14, 10, d=(1e-3, 1e-3, 0.5e-3), upml=(4,) * 6).replace(eps_r=np.array([1.0, 4.4]))
    p.mat[4:6, :, :] = 1
    prb = [(7, 9, 4, 2), (13, 9, 4, 2), (6, 5, 5, 0), (13, 5, 5, 0)]
    p = W.add_ports(p, [(10, 7, 4, 2)], prb, n_steps=400)
    tr = oracle.run(p, dft=False)["trace"]
    amp = np.abs(tr).max()
    assert np.abs(tr[0]).max() > 1e-3 * amp and np.abs(tr[2]).max() > 1e-6 * amp
    assert np.abs(tr[0] - tr[1]).max() <= 1e-11 * amp
    assert np.abs(tr[2] + tr[3]).max() <= 1e-11 * amp
