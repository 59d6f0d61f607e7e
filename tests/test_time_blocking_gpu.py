"""Time blocking on the GPU: two leapfrog steps per interior pass (depth 2).

With FP32 storage the two-step pass must reproduce the one-step launches
bit for bit: it applies the same arithmetic to every element, and rounds
every intermediate value to the storage type exactly where the one-step path
stores it.

With FP16 storage one difference remains: the band's E.  The one-step kernel
updates E on the band nodes from the H~ it holds in registers.  The slab
kernels that finish the band read H~ back from memory, rounded to FP16.  So
FP16 runs are held to the FP16 storage bar instead (probe traces within 1e-2
of the FP64 oracle and of depth 1).

The checks:
* Random-material grids that span several 60 x 8 pass tiles and z segments,
  ragged in every axis.  They carry current and resistive voltage sources and
  probes both on the interior region's one-node outer layer (the band that
  the slab kernels finish) and inside it.
* FP32 and FP16 storage.
* The FP64 oracle.
* Depth switches in the middle of a run, checkpoints and diagnostics.
* The 880 x 680 x 100 multilayer board.
"""
import numpy as np
import pytest

import oracle
from paper_1008_2602_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fdtd():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("a CUDA device is required for -m gpu tests")
    from paper_1008_2602_gb300 import solver
    return solver


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def interior(p, prec="fp32"):
    """The interior region I the library lays out.

    The fused region has x bounds rounded inward to 32-byte sectors (8 FP32
    or 16 FP16 nodes), y in [max(d, 1), ny - d), z planes [max(d, 1),
    nz - d)."""
    xa = 8 if prec == "fp32" else 16
    d = p.upml_depth
    ix0, ix1 = max(d[0], 1), p.nx - d[1]
    ax0, ax1 = -(-ix0 // xa) * xa, ix1 // xa * xa
    if ax1 - ax0 >= xa:
        ix0, ix1 = ax0, ax1
    return ix0, ix1, max(d[2], 1), p.ny - d[3], max(d[4], 1), p.nz - d[5]


def band_problem(seed, shape, upml, prec, n_steps, **over):
    """A random problem plus sources and probes on the band and inside I.

    The band is the one-node outer layer of I.  The extra sources are E_z
    edges, which a PEC sheet never covers, plus an E_x and an E_y edge off
    the sheet's plane.  One resistive voltage source sits inside I and one
    on a band corner.  `over` replaces problem fields (UPML depths, walls,
    kappa_max) first; the random sources that then fall in a UPML are
    dropped."""
    p = W.random_problem(seed, *shape, upml=upml, n_steps=n_steps)
    if over:
        p = p.replace(**over)
    d, n = p.upml_depth, (p.nx, p.ny, p.nz)
    ix0, ix1, iy0, iy1, iz0, iz1 = interior(p, prec)
    kk = int(np.asarray(p.pec_boxes).reshape(-1, 6)[0][4])
    jm, km = (iy0 + iy1) // 2, (iz0 + iz1) // 2
    kx = km if km != kk else km + 1
    src = [tuple(int(v) for v in s) for s in np.asarray(p.sources).reshape(-1, 4)
           if all(d[2 * a] <= s[a] <= n[a] - d[2 * a + 1] - 1 for a in range(3))]
    src += [(ix0, jm, km, 2), (ix1 - 1, jm + 1, km, 2), (ix0 + 5, iy0, iz0, 2), (ix0 + 7, iy1 - 1, iz1 - 1, 2),
            (ix0 + 3, jm, iz0, 2), (ix0 + 2, jm, kx, 0), (ix1 - 2, jm - 1, kx, 1), (ix0 + 2, jm, kx, 0)]
    prb = [tuple(int(v) for v in q) for q in np.asarray(p.probes).reshape(-1, 4)]
    prb += [(ix0, jm, km, 1), (ix1 - 1, jm, km, 0), (ix0 + 10, iy0, iz0, 2), (ix0 + 11, iy1 - 1, iz1 - 1, 0),
            (ix0 + 20, jm + 2, km, 2), (ix1 - 1, iy1 - 1, iz1 - 1, 2)]
    p = W.add_ports(p, src, prb, n_steps=n_steps)
    return W.add_voltage_sources(p, [(ix0 + 9, jm - 1, km, 2), (ix1 - 1, iy0, iz0, 2)], V0=5.0, Rs=10.0)


def _run(fdtd, p, prec, steps, **tune):
    s = fdtd.Solver(p, precision=prec, tuning=tune or None)
    s.step(steps)
    out = [s.field(c) for c in range(6)], s.traces(), s.spectra(), s.info()["depth"], s.diagnostics()
    s.close()
    return out


@pytest.mark.parametrize("prec,seed,shape,upml,pair_zseg,steps", [
    ("fp32", 3, (150, 44, 30), 4, 5, 37),     # 3 x 5 tiles, five z segments (bottom, middle, top)
    ("fp16", 4, (170, 37, 27), 3, 38, 36),    # one z segment: the bottom and top at once; ragged tiles
    ("fp32", 5, (97, 30, 19), 0, 4, 23),      # PEC walls, no UPML: slab wall planes below and above I
    ("fp32", 6, (300, 20, 12), 4, 2, 41),     # shortest z segments, five tile columns, one tile row
])
def test_depth2_bitwise_equals_depth1(fdtd, ncpu, prec, seed, shape, upml, pair_zseg, steps):
    """FP32: every field element, probe sample and diagnostic bit-identical
    to the one-step launches after an odd and an even number of steps.
    FP16: probe traces within 1e-2 (relative L2) of the oracle and of depth 1."""
    p = band_problem(seed, shape, upml, prec, steps)
    f1, t1, sp1, d1, g1 = _run(fdtd, p, prec, steps)
    f2, t2, sp2, d2, g2 = _run(fdtd, p, prec, steps, depth=2, pair_zseg=pair_zseg, graph_chunk=8)
    assert d1 == 1 and d2 == 2
    if prec == "fp16":
        ref = oracle.run(p, n_threads=ncpu, fields=False, dft=False)["trace"]
        live = [k for k in range(len(ref)) if np.abs(ref[k]).max() > 0]
        assert rel_l2(t2[live], ref[live]) <= 1e-2
        assert rel_l2(t2[live], t1[live]) <= 1e-2
        return
    for c in range(6):
        assert np.array_equal(f1[c], f2[c]), c
    assert np.array_equal(t1, t2)
    assert np.allclose(sp1, sp2, rtol=0, atol=1e-12 * max(np.abs(sp1).max(), 1e-300))
    assert g1 == g2


def test_depth2_matches_oracle(fdtd, ncpu):
    """Depth 2 against the FP64 oracle: every field element (relative L2 and
    max error within 1e-4) and the probe traces (relative L2 1e-4)."""
    p = band_problem(7, (150, 44, 30), 4, "fp32", 120)
    ref = oracle.run(p, n_threads=ncpu, fields=True, dft=False)
    s = fdtd.Solver(p, tuning=dict(depth=2, pair_zseg=9))
    assert s.info()["depth"] == 2
    s.run()
    for name, comps in (("E", (0, 1, 2)), ("H", (3, 4, 5))):
        g = np.stack([s.field(c).astype(np.float64) for c in comps])
        r = np.stack([ref["fields"][c] for c in comps])
        m = np.abs(r).max()
        assert rel_l2(g, r) <= 1e-4, name
        assert np.abs(g - r).max() <= 1e-4 * m, name
    tr = s.traces()
    for k in range(len(tr)):
        if np.abs(ref["trace"][k]).max() > 0:
            assert rel_l2(tr[k], ref["trace"][k]) <= 1e-4, k
    s.close()


def test_depth_switch_checkpoint_and_diagnostics(fdtd):
    """Depth 1 for 7 steps, then depth 2: the diagnostics after step 27 and
    the fields after step 61 equal a depth-1 run.  A checkpoint taken at
    depth 2 (step 27, an odd state) resumes bit for bit in solvers of either
    depth."""
    p = band_problem(8, (150, 44, 30), 4, "fp32", 61)
    ref = fdtd.Solver(p)
    ref.step(7).step(20)
    g_ref = ref.diagnostics()
    ref.step(34)
    f_ref = [ref.field(c) for c in range(6)]
    a = fdtd.Solver(p)
    a.step(7)
    a.set_tuning(depth=2, pair_zseg=7)
    a.step(20)
    assert a.diagnostics() == g_ref
    state = a.save()
    a.step(34)
    for c in range(6):
        assert np.array_equal(a.field(c), f_ref[c]), c
    for depth in (1, 2):
        b = fdtd.Solver(p, tuning=dict(depth=depth))
        b.load(state)
        assert b.info()["step"] == 27
        b.step(34)
        for c in range(6):
            assert np.array_equal(b.field(c), f_ref[c]), (depth, c)
        b.close()
    a.set_tuning(depth=1)
    a.step(5)
    ref.step(5)
    for c in range(6):
        assert np.array_equal(a.field(c), ref.field(c)), c
    a.close()
    ref.close()


@pytest.mark.parametrize("variant", ["kappa5", "pmc_sides"])
def test_depth2_bitwise_with_stretched_upml_and_pmc_walls(fdtd, variant):
    """Depth 2 runs the slab and z-UPML launches of both steps through the
    three field sets; their auxiliaries keep the step parity.  Checked
    bitwise against depth 1 with kappa_max = 5 (m = 3) in an uneven UPML, and
    on a board with PMC x and y walls and no x/y UPML (z-UPML only)."""
    if variant == "kappa5":
        p = band_problem(13, (140, 41, 28), 4, "fp32", 45, upml_kappa_max=5.0, upml_depth=(4, 6, 5, 4, 4, 6))
    else:
        p = band_problem(14, (120, 37, 26), 4, "fp32", 45, upml_depth=(0, 0, 0, 0, 4, 4),
                         walls=(W.WALL_PMC,) * 4 + (W.WALL_PEC,) * 2)
    f1, t1, _, _, g1 = _run(fdtd, p, "fp32", 45)
    f2, t2, _, d2, g2 = _run(fdtd, p, "fp32", 45, depth=2, pair_zseg=6)
    assert d2 == 2
    for c in range(6):
        assert np.array_equal(f1[c], f2[c]), c
    assert np.array_equal(t1, t2)
    assert g1 == g2


def test_depth2_falls_back_where_the_pass_cannot_run(fdtd):
    """A PMC top wall without a z-UPML: the plane above I is a slab plane
    written after the pass would need it, so the board keeps one step per
    pass (depth 1 in effect) and its results are unchanged."""
    p = W.random_problem(9, 90, 30, 16, upml=3, n_steps=25)
    p = p.replace(upml_depth=(3, 3, 3, 3, 3, 0), walls=(W.WALL_PEC,) * 5 + (W.WALL_PMC,))
    f1, t1, _, d1, _ = _run(fdtd, p, "fp32", 25)
    f2, t2, _, d2, _ = _run(fdtd, p, "fp32", 25, depth=2)
    assert d1 == 1 and d2 == 1
    for c in range(6):
        assert np.array_equal(f1[c], f2[c]), c
    assert np.array_equal(t1, t2)


def test_full_board_depth2_bitwise(fdtd):
    """The 880 x 680 x 100 multilayer board (64 probes, 4 sources), 13 steps:
    eight planes of all six components (bottom wall, z-UPML, the band's
    bottom plane and the one above it, the middle, the top plane of I, the
    z-UPML above it, the top) and every probe trace equal to depth 1."""
    p = W.multilayer_board(n_steps=13)
    ix0, ix1, iy0, iy1, iz0, iz1 = interior(p)
    ks = [0, 5, iz0, iz0 + 1, (iz0 + iz1) // 2, iz1 - 1, iz1, p.nz - 1]
    planes, traces = [], []
    for tune in (None, dict(depth=2)):
        s = fdtd.Solver(p, tuning=tune)
        s.step(13)
        assert s.info()["depth"] == (2 if tune else 1)
        planes.append([[s.plane(c, k) for k in ks] for c in range(6)])
        traces.append(s.traces())
        s.close()
    for c in range(6):
        for i, k in enumerate(ks):
            assert np.array_equal(planes[0][c][i], planes[1][c][i]), (c, k)
    assert np.array_equal(traces[0], traces[1])


def test_tuner_searches_the_blocking_depth(fdtd, tmp_path, monkeypatch):
    """For a single board the tuner also times depth 2 (two pass segment
    lengths) and returns a configuration the library accepts.  The tuned run
    gives the same fields; a batch configuration keeps depth 1."""
    from paper_1008_2602_gb300 import tune
    monkeypatch.setattr(tune, "CACHE", str(tmp_path / "tune.json"))
    p = band_problem(10, (150, 44, 30), 4, "fp32", 40)
    cfg = tune.tune([p], steps=8, shapes=[(62, 8)], zsegs=[10], chunks=[16], pair_zsegs=[5, 19])
    assert cfg["depth"] in (1, 2)
    assert cfg["depth"] == 1 or cfg["pair_zseg"] in (5, 19)
    f_tuned, t_tuned, _, d, _ = _run(fdtd, p, "fp32", 40, **cfg)
    assert d == cfg["depth"]
    f_ref, t_ref, _, _, _ = _run(fdtd, p, "fp32", 40)
    for c in range(6):
        assert np.array_equal(f_tuned[c], f_ref[c]), c
    assert np.array_equal(t_tuned, t_ref)
    cfg2 = tune.tune([p, p], steps=4, shapes=[(62, 8)], zsegs=[10], chunks=[16])
    assert cfg2["depth"] == 1


def test_depth2_boards_in_a_batch_and_a_split(fdtd):
    """A depth-2 board stepped inside a batch runs single steps in the depth-2
    set order, and a board split along y whose parts are depth-2 contexts
    steps one step at a time with halo copies between the parts' current
    sets.  Both give the same bits as the boards alone at depth 1."""
    from paper_1008_2602_gb300 import decomp
    p = band_problem(11, (150, 44, 30), 4, "fp32", 77)
    q = band_problem(12, (97, 30, 19), 0, "fp32", 50)
    alone = []
    for prob in (p, q):
        f, t, _, _, _ = _run(fdtd, prob, "fp32", prob.n_steps)
        alone.append((f, t))
    b = fdtd.Batch()
    sol = [fdtd.Solver(p, tuning=dict(depth=2)), fdtd.Solver(q)]
    assert sol[0].info()["depth"] == 2
    sol[0].step(3)   # an odd step count on its own before joining
    b.add(sol[0], p.n_steps - 3)
    b.add(sol[1])
    done = 0
    while done < 2:
        done = b.step(16)
    b.sync()
    for s, (f, t) in zip(sol, alone):
        for c in range(6):
            assert np.array_equal(s.field(c), f[c]), c
        assert np.array_equal(s.traces(), t)
    b.close()
    for s in sol:
        s.close()
    sp = decomp.SplitSolver(p, [21], tuning=dict(depth=2))
    sp.step(p.n_steps)
    for c in range(6):
        assert np.array_equal(sp.field(c), alone[0][0][c]), c
    assert np.array_equal(sp.traces(), alone[0][1])
    sp.close()


def test_depth2_fp16_long_run_meets_the_storage_bar(fdtd, ncpu):
    """FP16 storage at depth 2 over the small PCB's 2000 steps: every probe
    trace within 1e-2 (relative L2) of the FP64 oracle and the spectral peaks
    in the oracle's bins, as for depth 1."""
    p = W.small_pcb()
    ref = oracle.run(p, n_threads=ncpu)
    s = fdtd.Solver(p, precision="fp16", tuning=dict(depth=2))
    assert s.info()["depth"] == 2
    s.run()
    tr = s.traces()
    errs = [rel_l2(tr[q], ref["trace"][q]) for q in range(len(tr))]
    assert max(errs) <= 1e-2, errs
    sp = s.spectra()
    for q in range(len(tr)):
        assert np.argmax(np.abs(sp[q][1:])) == np.argmax(np.abs(ref["spectra"][q][1:]))
    s.close()
