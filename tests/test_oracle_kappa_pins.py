"""Pins of the oracle's kappa branch (Eq. 5's kappa grading inside the Eq. 4
recurrences), which the kappa_max = 1 workloads never exercise.

* A closed form.  A 1D cavity filled with one uniform stretched, lossy medium
  (grading order m = 0 makes sigma and kappa constant across a layer that
  spans the whole axis) has an exact discrete solution: with
  q = sigma dt / (2 eps0), every step multiplies each mode by
  (kappa - q) / (kappa + q), and mode m oscillates at
  f_m = asin((c dt / d) sin(m pi / (2 N)) / sqrt(kappa^2 - q^2)) / (pi dt).
  (Both the D and the H recurrence apply kappa (z - 1)/dt + q (z + 1)/dt to
  the sampled field; squaring and inserting the Yee curl-curl eigenvalue
  gives kappa sin(theta) - j q cos(theta) = (c dt / d) sin(m pi / (2N)) with
  theta = omega dt / 2, whose root has Im theta = atanh(q / kappa).)
* Reflection below -40 dB with kappa_max = 5 (m = 3, R0 = 1e-6): a plane wave,
  a 2D line source and a 3D point source against large-domain references.
* Sensitivity.  Four kappa mistakes planted in copies of the oracle (kappa
  dropped from the curl factor, kappa graded from the wrong end of the layer,
  kappa on the E/H recurrence axis instead of the D/B axis, kappa on the D->E
  axis) each break the closed form.  The reflection pins catch three of them;
  moving kappa between the two recurrence axes yields another valid stretched
  coordinate (on a face both E and H then see kappa (1 + sigma / (j omega
  eps0)) instead of kappa + sigma / (j omega eps0)), so only the closed form's
  decay rate exposes it.
"""
import os
import re
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from paper_1008_2602_gb300 import workloads as W

C0 = 299792458.0
MU0 = 4e-7 * np.pi
EPS0 = 1.0 / (MU0 * C0 * C0)
ETA0 = MU0 * C0
PEC, PMC = W.WALL_PEC, W.WALL_PMC
ORACLE_SRC = os.path.join(os.path.dirname(oracle.__file__), "fdtd_oracle.c")


def _stretched_cavity(axis, high_face, kappa, qk=4.3e-4, n=40, steps=12000):
    """1D cavity of n cells along `axis`, filled by a UPML layer on one face
    with m = 0 (uniform sigma, kappa).  sigma is set through R0 so that
    q / kappa = qk.  Returns (problem, q)."""
    d = (1e-3, 1e-3, 1e-3)
    if axis == 0:
        size, comp, walls = (n, 1, 1), 2, (PEC, PEC, PMC, PMC, PEC, PEC)
        srcs, prb = [(7, t, 0, comp) for t in (0, 1)], (29, 0, 0, comp)
    elif axis == 1:
        size, comp, walls = (1, n, 1), 2, (PMC, PMC, PEC, PEC, PEC, PEC)
        srcs, prb = [(t, 7, 0, comp) for t in (0, 1)], (0, 29, 0, comp)
    else:
        size, comp, walls = (1, 1, n), 0, (PEC, PEC, PMC, PMC, PEC, PEC)
        srcs, prb = [(0, t, 7, comp) for t in (0, 1)], (0, 0, 29, comp)
    up = [0] * 6
    up[2 * axis + (1 if high_face else 0)] = n
    p = W.box(*size, d=d, walls=walls, upml=tuple(up))
    dt = p.courant * oracle.cfl_dt(*d)
    q = qk * kappa
    sigma = 2 * EPS0 * q / dt
    # Eq. 5 with m = 0: sigma_max = -ln(R0) / (2 eta0 depth d)
    R0 = float(np.exp(-2 * ETA0 * n * d[axis] * sigma))
    p = p.replace(upml_m=0.0, upml_R0=R0, upml_kappa_max=kappa)
    return W.add_ports(p, srcs, [prb], n_steps=steps), q


def _peak(x, dt, f_guess, pad=8, search=0.05):
    """Peak frequency near f_guess: Hann window, zero padding, log-parabola."""
    N = len(x)
    X = np.abs(np.fft.rfft(x * np.hanning(N), pad * N))
    f = np.fft.rfftfreq(pad * N, dt)
    lo, hi = np.searchsorted(f, f_guess * (1 - search)), np.searchsorted(f, f_guess * (1 + search))
    j = lo + int(np.argmax(X[lo:hi]))
    a, b, c = np.log(X[j - 1]), np.log(X[j]), np.log(X[j + 1])
    return (j + 0.5 * (a - c) / (a - 2 * b + c)) / (pad * N * dt)


def _closed_form_errors(trace, dt, kappa, q, n=40, d=1e-3, start=600):
    """Per mode m = 1..3: relative frequency error of the decay-compensated
    trace's peak against f_m, and the ratio of the mode's amplitude in the
    second half of the compensated trace to the first (1 if the decay rate is
    (kappa - q) / (kappa + q) per step)."""
    rho = (kappa - q) / (kappa + q)
    y = trace[start:] * rho ** (-np.arange(start, len(trace), dtype=np.float64))
    h = len(y) // 2
    out = []
    for m in (1, 2, 3):
        beta = C0 * dt / d * np.sin(m * np.pi / (2 * n))
        fm = np.arcsin(beta / np.sqrt(kappa * kappa - q * q)) / (np.pi * dt)
        ferr = (_peak(y, dt, fm) - fm) / fm

        def amp(seg):
            t = np.arange(len(seg)) * dt
            return abs(np.sum(seg * np.hanning(len(seg)) * np.exp(-2j * np.pi * fm * t)))

        out.append((ferr, amp(y[h:2 * h]) / amp(y[:h])))
    return out


def _passes_closed_form(errs):
    return all(abs(f) <= 1e-4 and abs(a - 1.0) <= 1e-2 for f, a in errs)


@pytest.mark.parametrize("axis,high_face", [(0, False), (1, True), (2, False), (0, True)])
@pytest.mark.parametrize("kappa", [1.0, 2.5, 5.0])
def test_uniform_stretched_lossy_cavity_closed_form(axis, high_face, kappa, ncpu):
    p, q = _stretched_cavity(axis, high_face, kappa)
    r = oracle.run(p, dft=False, n_threads=ncpu)
    errs = _closed_form_errors(r["trace"][0], r["dt"], kappa, q)
    assert _passes_closed_form(errs), errs


def _reflection(small, big, shift, srcs, prb, n_steps, ncpu, lib_path=None):
    a = oracle.run(W.add_ports(small, srcs, [prb], n_steps=n_steps), dft=False, n_threads=ncpu,
                   lib_path=lib_path)["trace"][0]
    mv = lambda t: (t[0] + shift[0], t[1] + shift[1], t[2] + shift[2], t[3])
    b = oracle.run(W.add_ports(big, [mv(s) for s in srcs], [mv(prb)], n_steps=n_steps), dft=False,
                   n_threads=ncpu, lib_path=lib_path)["trace"][0]
    return 20 * np.log10(np.abs(a - b).max() / np.abs(b).max())


def _plane_wave_db(ncpu, kappa, lib_path=None):
    d, walls = (1e-3, 1e-3, 1e-3), (PEC, PEC, PMC, PMC, PEC, PEC)
    small = W.box(60, 1, 1, d=d, walls=walls, upml=(10, 10, 0, 0, 0, 0)).replace(upml_kappa_max=kappa)
    big = W.box(860, 1, 1, d=d, walls=walls)
    return _reflection(small, big, (400, 0, 0), [(20, j, 0, 2) for j in (0, 1)], (45, 0, 0, 2), 400, ncpu,
                       lib_path)


def _line_source_db(ncpu, kappa, lib_path=None):
    d = (1e-3, 1e-3, 1e-3)
    small = W.box(40, 40, 1, d=d, upml=(10, 10, 10, 10, 0, 0)).replace(upml_kappa_max=kappa)
    big = W.box(300, 300, 1, d=d)
    return _reflection(small, big, (130, 130, 0), [(20, 20, 0, 2)], (27, 24, 0, 2), 300, ncpu, lib_path)


def test_upml_with_kappa_plane_wave_and_line_source_below_40db(ncpu):
    """kappa_max = 5, m = 3, R0 = 1e-6: normal incidence (1D) and all angles
    of incidence (2D line current) reflect below -40 dB."""
    assert _plane_wave_db(ncpu, 5.0) < -40
    assert _line_source_db(ncpu, 5.0) < -40


@pytest.mark.slow
def test_upml_with_kappa_point_source_3d_below_40db(ncpu):
    """3D point current, 8-cell UPML with kappa_max = 5 on all six faces,
    against a 110^3 domain whose walls return nothing within the window."""
    d = (1e-3, 1e-3, 1e-3)
    small = W.box(32, 32, 32, d=d, upml=(8,) * 6).replace(upml_kappa_max=5.0)
    big = W.box(110, 110, 110, d=d)
    db = _reflection(small, big, (39, 39, 39), [(16, 16, 16, 2)], (22, 17, 18, 2), 130, ncpu)
    assert db < -40, db


# --------------------------------------------------------------------------
# Planted kappa mistakes (copies of the oracle, built on the CPU)
# --------------------------------------------------------------------------

_FACTOR_LINES = r"(tcoef a = (?:ci|chf)\[\d\]\[\w\], b = (?:ci|chf)\[\d\]\[\w\], c = (?:ci|chf)\[\d\]\[\w\];)"


def _planted_source(name):
    s = open(ORACLE_SRC).read()
    # let the per-position factors remember sigma and kappa, so a plant can
    # rebuild them with kappa moved to another axis
    keep = s.replace("typedef struct { double ca, cb, cp, cm; } tcoef;",
                     "typedef struct { double ca, cb, cp, cm, s, k; } tcoef;")
    keep = keep.replace("c.cm = q;", "c.cm = q; c.s = sigma; c.k = kappa;")
    if name == "kappa_dropped_from_curl_factor":
        out = s.replace("c.cb = 2.0 * EPS0 * dt / p;", "c.cb = 2.0 * EPS0 * dt / (2.0 * EPS0 + sigma * dt);")
    elif name == "kappa_graded_from_wrong_end":
        out = s.replace("*kappa = 1.0 + (kmax - 1.0) * r;", "*kappa = 1.0 + (kmax - 1.0) * (1.0 - r);")
    elif name == "kappa_on_field_axis_not_aux_axis":
        out, n = re.subn(_FACTOR_LINES, r"\1 { tcoef a2 = tc(a.s, b.k, dt), b2 = tc(b.s, a.k, dt); a = a2; b = b2; }",
                         keep)
        assert n == 6
    elif name == "kappa_on_conversion_axis":
        out, n = re.subn(_FACTOR_LINES, r"\1 { tcoef b2 = tc(b.s, c.k, dt), c2 = tc(c.s, b.k, dt); b = b2; c = c2; }",
                         keep)
        assert n == 6
    else:
        raise ValueError(name)
    assert out != s
    return out


PLANTS = ["kappa_dropped_from_curl_factor", "kappa_graded_from_wrong_end", "kappa_on_field_axis_not_aux_axis",
          "kappa_on_conversion_axis"]


@pytest.mark.parametrize("name", PLANTS)
def test_planted_kappa_mistakes_break_the_pins(name, tmp_path, ncpu):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc is needed to build a planted copy of the oracle")
    src = tmp_path / "planted.c"
    src.write_text(_planted_source(name))
    lib = str(tmp_path / "libplanted.so")
    subprocess.run([gcc, "-O2", "-fopenmp", "-shared", "-fPIC", "-o", lib, str(src), "-lm"], check=True)
    p, q = _stretched_cavity(0, False, 2.5)
    r = oracle.run(p, dft=False, n_threads=ncpu, lib_path=lib)
    assert not _passes_closed_form(_closed_form_errors(r["trace"][0], r["dt"], 2.5, q)), name
    # with kappa_max = 1 every plant is the correct oracle again
    p1, q1 = _stretched_cavity(0, False, 1.0)
    r1 = oracle.run(p1, dft=False, n_threads=ncpu, lib_path=lib)
    assert _passes_closed_form(_closed_form_errors(r1["trace"][0], r1["dt"], 1.0, q1)), name
    if name != "kappa_on_field_axis_not_aux_axis":
        assert max(_plane_wave_db(ncpu, 5.0, lib), _line_source_db(ncpu, 5.0, lib)) > -40, name
