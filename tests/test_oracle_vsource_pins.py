"""Pins of the oracle's resistive voltage source (Results section: V0 = 5 V,
Rs = 10 ohm on one E edge, the pulse shape of Eq. 8), each against something
other than the oracle itself:

* Rs -> infinity: the edge is open, the scheme is the plain one;
* Rs -> 0: an ideal voltage source, E = -Vs / l on its edge at every step;
* the discrete Poynting theorem of the Yee scheme with the lumped current
  I^{n+1/2} = (l E^{n+1/2} + Vs)/Rs:  W^{n+1} - W^n = -dt l I (E^n + E^{n+1})/2;
* the paper's own Table 1 run with this source: the lowest isolated modes of
  the 40 x 30 x 0.8 mm board sit in the band of the paper's modelled peaks;
* linearity in V0.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1008_2602_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _vs(t, V0, t0, tau):
    u = (t - t0) / tau
    return V0 * u * np.exp(-u * u)


def _box_with_dielectric(n_steps=2000):
    p = W.box(12, 10, 8, d=(1e-3, 1.2e-3, 0.7e-3)).replace(eps_r=np.array([1.0, 3.0]))
    p.mat[3:6, 2:8, 3:9] = 1
    return W.add_ports(p, [(6, 3, 2, 0)], [(5, 5, 4, 2), (6, 3, 2, 0)], n_steps=n_steps)


def test_infinite_resistance_is_the_plain_scheme():
    p = _box_with_dielectric(600)
    ref = oracle.run(p, dft=False)
    q = W.add_voltage_sources(p, [(5, 5, 4, 2)], V0=5.0, Rs=np.inf)
    got = oracle.run(q, dft=False)
    assert np.abs(got["trace"] - ref["trace"]).max() <= 1e-12 * np.abs(ref["trace"]).max()


def test_vanishing_resistance_is_an_ideal_voltage_source():
    p = _box_with_dielectric(600)
    V0, t0, tau = 5.0, 40e-12, 15e-12
    q = W.add_voltage_sources(p, [(5, 5, 4, 2)], V0=V0, t0=t0, tau=tau, Rs=1e-9)
    r = oracle.run(q, dft=False)
    t = (np.arange(q.n_steps) + 0.5) * r["dt"]
    # E^{n+1} on the edge against -Vs^{n+1/2}/l: with Rs -> 0 the edge voltage
    # is forced at the half step, so E^{n+1/2} = -Vs/l; compare the average
    e_new = r["trace"][0]
    e_old = np.concatenate([[0.0], e_new[:-1]])
    target = -_vs(t, V0, t0, tau) / q.dz
    assert np.abs(0.5 * (e_old + e_new) - target).max() <= 1e-6 * np.abs(target).max()


def test_discrete_energy_balance_with_the_lumped_current():
    p = _box_with_dielectric(3000)
    V0, t0, tau, Rs = 5.0, 40e-12, 15e-12, 10.0
    q = W.add_voltage_sources(p, [(5, 5, 4, 2)], V0=V0, t0=t0, tau=tau, Rs=Rs)
    r = oracle.run(q, energy=True, vsrc_current=True, dft=False)
    dt, V = r["dt"], q.dx * q.dy * q.dz
    t = (np.arange(q.n_steps) + 0.5) * dt
    # the probe on the voltage-source edge (E_z, l = dz) and the current source
    e_v = r["trace"][0]
    e_v_old = np.concatenate([[0.0], e_v[:-1]])
    I = r["vsrc_current"]
    # the lumped current follows its definition from the edge field
    assert np.allclose(I, (q.dz * 0.5 * (e_v_old + e_v) + _vs(t, V0, t0, tau)) / Rs, rtol=0,
                       atol=1e-12 * np.abs(I).max())
    J0, tj0, tjau = q.source_params[0]
    Js = J0 * ((t - tj0) / tjau) * np.exp(-((t - tj0) / tjau) ** 2)
    e_j = r["trace"][1]
    e_j_old = np.concatenate([[0.0], e_j[:-1]])
    pred = -0.5 * dt * V * Js * (e_j_old + e_j) - dt * q.dz * I * 0.5 * (e_v_old + e_v)
    dW = np.diff(r["energy"])
    assert np.abs(dW - pred[:-1]).max() < 1e-11 * np.abs(dW).max()
    # after the pulses the resistor only dissipates
    late = dW[int(8 * max(t0, tj0) / dt) + 400:]
    assert (late <= 1e-12 * np.abs(dW).max()).all()


def test_linear_in_v0():
    p = _box_with_dielectric(400).replace(source_params=np.array([[0.0, 40e-12, 15e-12]]))
    a = oracle.run(W.add_voltage_sources(p, [(5, 5, 4, 2)], V0=1.0), dft=False)["trace"]
    b = oracle.run(W.add_voltage_sources(p, [(5, 5, 4, 2)], V0=3.0), dft=False)["trace"]
    assert np.abs(b - 3.0 * a).max() <= 1e-12 * np.abs(b).max()


def _table1():
    rows = []
    with open(os.path.join(GOLDEN, "table1_resonances.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            m, n, pred, label, model = line.split()
            rows.append((int(m), int(n), float(pred), label, float(model)))
    return rows


def spectral_peaks(x, dt, f_top=10.5e9):
    pad = 4
    X = np.abs(np.fft.rfft(x * np.hanning(len(x)), pad * len(x)))
    f = np.fft.rfftfreq(pad * len(x), dt)
    return np.array([f[j] for j in range(1, len(X) - 1)
                     if X[j] > X[j - 1] and X[j] > X[j + 1] and X[j] > 0.01 * X.max() and f[j] < f_top])


def test_table1_run_with_the_resistive_source(ncpu):
    """The paper's modelled peaks sit -3.6 % .. +1.9 % from Eq. 9; the
    nearest oracle peak of each of the five lowest isolated modes must sit in
    that band widened by 1 % on each side, and no peak may lie below the
    fundamental."""
    p = W.table1_board()
    r = oracle.run(p, dft=False, n_threads=ncpu)
    peaks = spectral_peaks(r["trace"][0], r["dt"])
    rows = {(m, n): pred * 1e9 for m, n, pred, _, _ in _table1()}
    for mode in [(1, 0), (0, 1), (2, 0), (0, 2), (3, 0)]:
        pred = rows[mode]
        near = peaks[np.argmin(np.abs(peaks - pred))]
        dev = (near - pred) / pred
        assert -0.046 <= dev <= 0.029, (mode, near, pred, dev)
    assert peaks.min() > 0.9 * rows[(1, 0)]


def test_rejects_edges_in_the_upml_or_on_pec():
    p = W.add_ports(W.box(12, 10, 8, upml=(2,) * 6), [], [(6, 5, 4, 2)], n_steps=5)
    oracle.run(W.add_voltage_sources(p, [(6, 5, 4, 2)]), dft=False)          # interior edge: fine
    with pytest.raises(RuntimeError):
        oracle.run(W.add_voltage_sources(p, [(1, 5, 4, 2)]), dft=False)      # inside the x UPML
    with pytest.raises(RuntimeError):
        oracle.run(W.add_voltage_sources(p, [(6, 5, 6, 2)]), dft=False)      # E_z at z = 6.5 > 8 - 2: in the z UPML
    q = p.replace(pec_boxes=np.array([[3, 9, 2, 8, 4, 4]], np.int32))
    with pytest.raises(RuntimeError):
        oracle.run(W.add_voltage_sources(q, [(6, 5, 4, 0)]), dft=False)      # E_x on a PEC sheet
