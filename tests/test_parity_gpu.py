"""Parity of the CUDA path (through the C-ABI) with the FP64 oracle.

Tolerances (FP32 arithmetic against FP64):
  * probe traces and spectra: relative L2 <= 1e-4 (the target stated for FP32);
  * whole fields, element by element: relative L2 <= 1e-4 per component and
    every element within 1e-4 of that component's max |value|;
  * FP16 storage (FP32 arithmetic): probe-trace relative L2 <= 1e-2;
  * resonant peaks of the spectra: the same FFT bin.
Sizes span several fused tiles (124 x 4 columns, z-segments of 50) with
ragged tails in every axis, the UPML on all faces, PEC sheets, PMC walls.
"""
import numpy as np
import pytest

import oracle
from paper_1008_2602_gb300 import workloads as W

pytestmark = pytest.mark.gpu

PEC, PMC = W.WALL_PEC, W.WALL_PMC


@pytest.fixture(scope="module")
def fdtd():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("a CUDA device is required for -m gpu tests")
    from paper_1008_2602_gb300 import solver
    return solver


def rel_l2(a, b):
    """Relative L2 error of a against b (complex arrays compared as complex)."""
    a = np.asarray(a)
    b = np.asarray(b)
    dt = np.complex128 if np.iscomplexobj(a) or np.iscomplexobj(b) else np.float64
    a = a.astype(dt)
    b = b.astype(dt)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _fields_close(gpu_solver, ref_fields, tol=1e-4):
    """Element-by-element comparison of the six final fields: for E (and for
    H) the relative L2 error over its three components together, and every
    element's error relative to the largest |value| of that field."""
    worst = {}
    for name, comps in (("E", (0, 1, 2)), ("H", (3, 4, 5))):
        g = np.stack([gpu_solver.field(c).astype(np.float64) for c in comps])
        r = np.stack([ref_fields[c] for c in comps])
        m = np.abs(r).max()
        if m == 0:
            assert np.abs(g).max() == 0, name
            continue
        worst[name] = (rel_l2(g, r), np.abs(g - r).max() / m)
        assert worst[name][0] <= tol, (name, worst[name])
        assert worst[name][1] <= tol, (name, worst[name])
    return worst


def test_small_pcb_traces_and_spectra(fdtd, ncpu):
    """Small PCB (56x48x30, 8-cell UPML, 2000 steps, 4 probes): FP32 traces
    and running-DFT spectra against the oracle; resonant peaks in the same bin."""
    p = W.small_pcb()
    ref = oracle.run(p, n_threads=ncpu, fields=True)
    s = fdtd.Solver(p)
    s.run()
    tr = s.traces()
    assert tr.shape == ref["trace"].shape
    for q in range(len(tr)):
        assert rel_l2(tr[q], ref["trace"][q]) <= 1e-4, q
    sp = s.spectra()
    assert sp.shape == ref["spectra"].shape
    assert rel_l2(np.abs(sp), np.abs(ref["spectra"])) <= 1e-4
    assert rel_l2(sp, ref["spectra"]) <= 1e-4
    for q in range(len(tr)):
        assert np.argmax(np.abs(sp[q][1:])) == np.argmax(np.abs(ref["spectra"][q][1:]))
    _fields_close(s, ref["fields"])
    s.close()


@pytest.mark.parametrize("seed,shape,upml", [
    (1, (37, 29, 23), 3),     # ragged in every axis, several tiles
    (2, (70, 13, 40), 4),     # > 2 tiles in x, thin y, 3 z segments
    (3, (9, 11, 8), 2),       # tiny interior
    (4, (33, 9, 18), 0),      # no UPML: PEC walls only
])
def test_random_grids_fields_match_oracle(fdtd, ncpu, seed, shape, upml):
    """Random materials, a PEC sheet, random sources (all three components)
    and probes; every field element after 80 steps against the oracle."""
    p = W.random_problem(seed, *shape, upml=max(upml, 0) if upml else 0, n_steps=80)
    if upml == 0:
        p = p.replace(upml_depth=(0,) * 6)
    ref = oracle.run(p, n_threads=ncpu, fields=True)
    s = fdtd.Solver(p)
    s.run()
    _fields_close(s, ref["fields"])
    tr = s.traces()
    for q in range(len(tr)):
        if np.abs(ref["trace"][q]).max() > 0:
            assert rel_l2(tr[q], ref["trace"][q]) <= 1e-4
    s.close()


@pytest.mark.parametrize("new_geometry", ["random", "uniform"])
def test_set_materials_equals_fresh_board(fdtd, ncpu, new_geometry):
    """fdtd_set_materials on a live board (same eps_r table, PEC and ports):
    the run that follows equals a board created with the new materials, bit
    for bit, and the oracle on them.  The random grid has about a thousand
    distinct edge coefficient triples (16-bit ids), the uniform one a handful
    (8-bit ids), so the "uniform" case also switches the id width."""
    a = W.random_problem(21, 31, 23, 17, upml=3, n_steps=60)
    rng = np.random.default_rng(22)
    if new_geometry == "random":
        mat = rng.integers(0, len(a.eps_r), size=a.mat.shape).astype(np.uint8)
    else:
        mat = np.full(a.mat.shape, 1, np.uint8)
    b = a.replace(mat=mat)
    s = fdtd.Solver(a)
    s.step(7)                       # the old geometry has run: set_materials also resets
    s.set_materials(b.mat)
    s.run()
    fresh = fdtd.Solver(b)
    fresh.run()
    for c in range(6):
        assert np.array_equal(s.field(c), fresh.field(c)), c
    assert np.array_equal(s.traces(), fresh.traces())
    ref = oracle.run(b, n_threads=ncpu, fields=True)
    _fields_close(s, ref["fields"])
    s.close()
    fresh.close()


def test_pmc_walls_match_oracle(fdtd, ncpu):
    """PEC top/bottom, PMC side walls (cavity model), anisotropic cells."""
    p = W.box(26, 19, 3, d=(1e-3, 1.3e-3, 0.4e-3), eps_r=4.4, walls=(PMC, PMC, PMC, PMC, PEC, PEC))
    p = W.add_ports(p, [(3, 4, 0, 2), (20, 2, 1, 2)], [(0, 0, 1, 2), (25, 18, 2, 2), (13, 9, 1, 2)], n_steps=600)
    ref = oracle.run(p, n_threads=ncpu, fields=True)
    s = fdtd.Solver(p)
    s.run()
    _fields_close(s, ref["fields"])
    tr = s.traces()
    for q in range(len(tr)):
        assert rel_l2(tr[q], ref["trace"][q]) <= 1e-4
    s.close()


@pytest.mark.parametrize("prec,m", [("fp32", 3.0), ("fp32", 2.0), ("fp16", 3.0)])
def test_kappa_upml_matches_oracle(fdtd, ncpu, prec, m):
    """kappa_max = 5 (Eq. 5's kappa grading) with a different UPML depth on
    every face and one face without UPML: every field element (FP32) or the
    probe traces (FP16 storage) against the oracle.  The grid has a fused
    region, so the kappa factors run through the z-UPML fused launch as well
    as the slab kernels."""
    p = W.random_problem(9, 31, 27, 21, upml=3, n_steps=100)
    p = p.replace(upml_depth=(2, 5, 0, 4, 3, 1), walls=(PEC, PEC, PMC, PEC, PEC, PEC), upml_kappa_max=5.0, upml_m=m)
    ref = oracle.run(p, n_threads=ncpu, fields=True)
    s = fdtd.Solver(p, precision=prec)
    s.run()
    if prec == "fp32":
        _fields_close(s, ref["fields"])
    tr = s.traces()
    for q in range(len(tr)):
        if np.abs(ref["trace"][q]).max() > 0:
            assert rel_l2(tr[q], ref["trace"][q]) <= (1e-4 if prec == "fp32" else 1e-2), q
    s.close()


def test_kappa_small_pcb_traces(fdtd, ncpu):
    """The small PCB (8-cell UPML on all faces) with kappa_max = 5: FP32
    traces and spectra against the oracle over its full 2000 steps."""
    p = W.small_pcb().replace(upml_kappa_max=5.0)
    ref = oracle.run(p, n_threads=ncpu)
    s = fdtd.Solver(p)
    s.run()
    tr = s.traces()
    for q in range(len(tr)):
        assert rel_l2(tr[q], ref["trace"][q]) <= 1e-4, q
    assert rel_l2(s.spectra(), ref["spectra"]) <= 1e-4
    s.close()


def test_mixed_walls_and_uneven_upml(fdtd, ncpu):
    """Different UPML depth on every face (one face without UPML, PMC)."""
    p = W.random_problem(9, 31, 27, 21, upml=3, n_steps=100)
    p = p.replace(upml_depth=(2, 5, 0, 4, 3, 1), walls=(PEC, PEC, PMC, PEC, PEC, PEC))
    ref = oracle.run(p, n_threads=ncpu, fields=True)
    s = fdtd.Solver(p)
    s.run()
    _fields_close(s, ref["fields"])
    s.close()


def test_reduced_storage_error_vs_oracle(fdtd, ncpu):
    """FP16 field storage with FP32 arithmetic against the FP64 oracle on the
    small PCB (2000 steps): every probe trace within the 1e-2 relative-L2
    target for reduced storage, spectral peaks in the same bin."""
    p = W.small_pcb()
    ref = oracle.run(p, n_threads=ncpu)
    s = fdtd.Solver(p, precision="fp16")
    s.run()
    tr = s.traces()
    errs = [rel_l2(tr[q], ref["trace"][q]) for q in range(len(tr))]
    assert max(errs) <= 1e-2, errs
    sp = s.spectra()
    for q in range(len(tr)):
        assert np.argmax(np.abs(sp[q][1:])) == np.argmax(np.abs(ref["spectra"][q][1:]))
    s.close()


def test_spectra_equal_fft_of_trace(fdtd):
    """GPU running DFT (FP64) equals dt * FFT of the GPU's own FP32 trace."""
    p = W.random_problem(5, 24, 20, 16, upml=3, n_steps=333)
    s = fdtd.Solver(p)
    s.step(100).step(1).step(232)
    tr = s.traces().astype(np.float64)
    sp = s.spectra()
    ref = s.dt * np.fft.fft(tr, axis=1)[:, : sp.shape[1]]
    assert np.abs(sp - ref).max() <= 1e-10 * np.abs(ref).max()
    s.close()


def test_row_bands_cover_every_tile(fdtd, ncpu):
    """The interior launch takes its items in bands of tile rows of about one
    wave of resident blocks.  A board one tile column wide and 624 tile rows
    tall (more than one wave of 62x8 tiles) is worked in two bands; every
    field element after 30 steps against the oracle."""
    p = W.random_problem(41, 70, 5000, 14, upml=4, n_steps=30)
    ref = oracle.run(p, n_threads=ncpu, fields=True)
    s = fdtd.Solver(p, tuning=dict(tile_x=62, tile_y=8, zseg=10, graph_chunk=16))
    s.run()
    _fields_close(s, ref["fields"])
    s.close()


def test_chunking_and_tiling_do_not_change_results(fdtd):
    """Bitwise identical fields for different graph chunks, tile shapes and
    z-segments (halo recomputation equals the owner's value)."""
    p = W.random_problem(6, 45, 38, 29, upml=4, n_steps=50)
    outs = []
    for tune in [dict(tile_x=124, tile_y=4, zseg=16, graph_chunk=16), dict(tile_x=62, tile_y=4, zseg=5, graph_chunk=1),
                 dict(tile_x=62, tile_y=8, zseg=64, graph_chunk=7), dict(tile_x=124, tile_y=8, zseg=3, graph_chunk=4),
                 dict(tile_x=124, tile_y=4, zseg=9, graph_chunk=16)]:
        s = fdtd.Solver(p, tuning=tune)
        s.run()
        outs.append([s.field(c) for c in range(6)])
        s.close()
    for o in outs[1:]:
        for c in range(6):
            assert np.array_equal(o[c], outs[0][c]), c


def test_energy_conserved_and_div_b_on_gpu(fdtd, ncpu):
    """Closed lossless PEC box: the GPU's FP64-reduced discrete energy matches
    the oracle's, stays constant after the pulse, and div B stays at FP32
    round-off."""
    p = W.box(24, 20, 16, d=(1e-3, 1.2e-3, 0.7e-3)).replace(eps_r=np.array([1.0, 3.0]))
    p.mat[4:9, 5:15, 3:20] = 1
    p = W.add_ports(p, [(10, 10, 6, 2), (7, 5, 3, 0)], [(10, 10, 6, 2)], n_steps=1200)
    ref = oracle.run(p, energy=True, divb=True, n_threads=ncpu)
    s = fdtd.Solver(p)
    s.step(700)
    e1, d1 = s.diagnostics()
    s.step(500)
    e2, d2 = s.diagnostics()
    assert abs(e1 - ref["energy"][699]) <= 1e-4 * ref["energy"][699]
    assert abs(e2 - ref["energy"][1199]) <= 1e-4 * ref["energy"][1199]
    assert abs(e2 - e1) <= 2e-5 * e1
    hmax = max(np.abs(s.field(c)).max() for c in (3, 4, 5))
    mu0 = 4e-7 * np.pi
    assert d2 <= 1e-4 * mu0 * hmax / 0.7e-3
    s.close()


def test_batch_equals_alone(fdtd):
    """Boards of different sizes and step counts stepped in one batch give
    bitwise the same traces, spectra and fields as each board alone."""
    rng = np.random.default_rng(12)
    probs = [W.batch_board(rng, n_steps=n, dxy=2e-3, dz=0.4e-3, upml=(6, 6, 6), size_mm=(20, 60))
             for n in (150, 90, 150, 40)]
    alone = []
    for p in probs:
        s = fdtd.Solver(p)
        s.run()
        alone.append((s.traces(), s.spectra(), s.field(2)))
        s.close()
    b = fdtd.Batch()
    sol = [fdtd.Solver(p) for p in probs]
    for s in sol:
        b.add(s)
    done = 0
    while done < len(sol):
        done = b.step(37)
    b.sync()
    for s, (tr, sp, ez) in zip(sol, alone):
        assert np.array_equal(s.traces(), tr)
        assert np.array_equal(s.field(2), ez)
        assert np.allclose(s.spectra(), sp, rtol=0, atol=1e-12 * np.abs(sp).max())
    b.close()
    for s in sol:
        s.close()


def test_errors_are_reported_not_raised_in_kernels(fdtd):
    """Invalid requests return an error status (raised as FdtdError)."""
    from paper_1008_2602_gb300 import capi
    p = W.small_pcb()
    with pytest.raises(capi.FdtdError):
        fdtd.Solver(p.replace(walls=(PMC,) * 6))          # PMC behind a UPML
    bad = p.replace(sources=np.array([[1, 1, 1, 2]], np.int32))
    with pytest.raises(capi.FdtdError):
        fdtd.Solver(bad)                                    # source inside the UPML
    s = fdtd.Solver(p)
    with pytest.raises(capi.FdtdError):
        s.diagnostics()                                     # no step yet
    s.step(3)
    with pytest.raises(capi.FdtdError):
        capi.fdtd_add_probe(s.ctx, 20, 20, 14, 2, None)    # after the first step
    s.close()


def test_unstable_courant_is_detected(fdtd):
    """Courant > 1 (beyond Eq. 7) blows up; the library reports EUNSTABLE."""
    from paper_1008_2602_gb300 import capi
    p = W.add_ports(W.box(12, 10, 8), [(5, 4, 4, 2)], [(3, 3, 3, 2)], n_steps=4000).replace(courant=1.05)
    s = fdtd.Solver(p)
    s.step(4000)
    with pytest.raises(capi.FdtdError) as ei:
        s.sync()
    assert ei.value.code == capi.FDTD_EUNSTABLE
    s.close()


def test_served_results_equal_alone(fdtd, ncpu):
    """Requests arriving at staggered times join a running mix (continuous
    batching); every request's spectrum equals the same board solved alone."""
    from paper_1008_2602_gb300 import serve
    reqs = W.request_stream(seed=21, n_requests=6, rate=400.0, step_scale=0.03, cell_scale=0.01)
    alone = {}
    for r in reqs:
        s = fdtd.Solver(r.problem)
        s.run()
        alone[r.rid] = s.spectra()
        s.close()
    be = serve.CudaBackend()
    srv = serve.Server(be, hbm_budget=8 << 30, chunk=37)
    res = srv.run(reqs)
    be.close()
    assert sorted(x.rid for x in res) == sorted(alone)
    for x in res:
        ref = alone[x.rid]
        assert x.spectra.shape == ref.shape
        assert np.abs(x.spectra - ref).max() <= 1e-12 * np.abs(ref).max(), x.rid
    assert max(x.latency for x in res) > 0
    # and every served spectrum against the FP64 oracle (FP32 target 1e-4)
    by_id = {r.rid: r for r in reqs}
    for x in res:
        ref = oracle.run(by_id[x.rid].problem, n_threads=ncpu)["spectra"]
        assert rel_l2(x.spectra, ref) <= 1e-4, x.rid


def test_autotuner_picks_a_valid_configuration(fdtd, tmp_path, monkeypatch):
    """The tuner times candidate launch shapes on throwaway copies and returns
    one the library accepts; the tuned run gives the same fields."""
    from paper_1008_2602_gb300 import tune
    monkeypatch.setattr(tune, "CACHE", str(tmp_path / "tune.json"))
    rng = np.random.default_rng(3)
    probs = [W.batch_board(rng, n_steps=60, dxy=2e-3, dz=0.4e-3, upml=(6, 6, 6), size_mm=(30, 60)) for _ in range(3)]
    cfg = tune.tune(probs, steps=6, zsegs=[16, 50], chunks=[16])
    assert (cfg["tile_x"], cfg["tile_y"]) in tune.SHAPES
    a = fdtd.Solver(probs[0], tuning=cfg)
    a.run()
    b = fdtd.Solver(probs[0])
    b.run()
    assert np.array_equal(a.field(2), b.field(2))
    assert tune.tune(probs, steps=6) == cfg   # cached
    a.close(); b.close()


def test_checkpoint_resume_is_bitwise(fdtd):
    """Run N steps = run k steps, save, load into a fresh solver of the same
    problem, run N - k: fields and traces bitwise equal, spectra equal to
    FP64 rounding (the running DFT folds samples at chunk boundaries, which
    differ between the two runs); a checkpoint of another board is refused
    and leaves the solver unchanged."""
    p = W.random_problem(21, 40, 30, 20, upml=4, n_steps=300)
    ref = fdtd.Solver(p)
    ref.run()
    a = fdtd.Solver(p)
    a.step(137)
    state = a.save()
    a.close()
    b = fdtd.Solver(p)
    b.load(state)
    assert b.info()["step"] == 137
    b.step(300 - 137)
    for c in range(6):
        assert np.array_equal(b.field(c), ref.field(c)), c
    assert np.array_equal(b.traces(), ref.traces())
    sp, sr = b.spectra(), ref.spectra()
    assert np.allclose(sp, sr, rtol=0, atol=1e-12 * np.abs(sr).max())
    assert b.diagnostics() == ref.diagnostics()
    other = fdtd.Solver(W.random_problem(22, 41, 30, 20, upml=4, n_steps=300))
    from paper_1008_2602_gb300 import capi
    with pytest.raises(capi.FdtdError) as ei:
        other.load(state)
    assert ei.value.code == capi.FDTD_EINVAL
    assert other.info()["step"] == 0
    for s in (ref, b, other):
        s.close()


def test_resistive_voltage_source_matches_oracle(fdtd, ncpu):
    """A resistive voltage source (V0, Rs in series on an E edge) next to a
    current source on a random-material grid: traces and fields against the
    oracle's semi-implicit lumped-element update; the open (Rs = inf) source
    leaves the run unchanged bit for bit."""
    p = W.random_problem(17, 30, 24, 18, upml=3, n_steps=400)
    s0 = p.sources[0]
    q = W.add_voltage_sources(p, [(int(s0[0]) + 2, int(s0[1]) + 1, int(s0[2]), 2)], V0=5.0, Rs=10.0)
    ref = oracle.run(q, n_threads=ncpu, fields=True, dft=False)
    s = fdtd.Solver(q)
    s.run()
    tr = s.traces()
    for k in range(len(tr)):
        assert rel_l2(tr[k], ref["trace"][k]) <= 1e-4, k
    _fields_close(s, ref["fields"])
    s.close()
    a = fdtd.Solver(p)
    a.run()
    b = fdtd.Solver(W.add_voltage_sources(p, [(int(s0[0]) + 2, int(s0[1]) + 1, int(s0[2]), 2)], Rs=np.inf))
    b.run()
    assert np.array_equal(a.traces(), b.traces())
    a.close()
    b.close()


@pytest.mark.parametrize("shape,upml,src", [
    ((1, 1, 1), (0,) * 6, (0, 0, 0, 2)),               # one cell: no fused region, every node a slab node
    ((6, 5, 1), (0,) * 6, (3, 2, 0, 2)),               # a single z cell (one-plane z-march slabs)
    ((1, 7, 6), (0,) * 6, (0, 3, 2, 2)),               # a single x cell
    ((12, 10, 8), (4,) * 6, (5, 5, 4, 0)),             # UPML on every face leaves no interior columns
    ((14, 12, 9), (6, 6, 6, 6, 4, 4), (7, 6, 4, 2)),   # UPML layers meeting in the middle of y
])
def test_degenerate_grids_match_oracle(fdtd, ncpu, shape, upml, src):
    """Grids at the edges of the decomposition: fields and traces against the
    oracle element by element (the source sits on an edge outside the UPML).
    Errors are measured against each field's natural scale, max |E| for E and
    max(|H|, |E|/eta0) for H (the kernels hold E and eta0 H at one scale): on
    these tiny grids a single H component can be a near-cancellation far below
    that scale."""
    nx, ny, nz = shape
    walls = (PMC, PMC, PMC, PMC, PEC, PEC) if not any(upml) else (PEC,) * 6
    p = W.box(nx, ny, nz, d=(1e-3, 1.1e-3, 0.6e-3), eps_r=2.0, walls=walls, upml=upml)
    p = W.add_ports(p, [src], [src], n_steps=80)
    ref = oracle.run(p, n_threads=ncpu, fields=True, dft=False)
    s = fdtd.Solver(p)
    s.run()
    assert np.abs(ref["trace"]).max() > 0
    assert rel_l2(s.traces(), ref["trace"]) <= 1e-4
    eta0 = 4e-7 * np.pi * 299792458.0
    me = max(np.abs(ref["fields"][c]).max() for c in range(3))
    mh = max(max(np.abs(ref["fields"][c]).max() for c in range(3, 6)), me / eta0)
    for c in range(6):
        g, r = s.field(c).astype(np.float64), ref["fields"][c]
        assert np.abs(g - r).max() <= 1e-4 * (me if c < 3 else mh), c
    s.close()


def test_no_sources_no_probes(fdtd):
    """A board with neither sources nor probes steps, stays at zero and
    reports empty spectra."""
    p = W.random_problem(41, 20, 16, 12, upml=3, n_steps=30).replace(
        sources=np.zeros((0, 4), np.int32), source_params=np.zeros((0, 3)), probes=np.zeros((0, 4), np.int32))
    s = fdtd.Solver(p)
    s.run()
    assert s.info()["step"] == 30
    for c in range(6):
        assert not np.any(s.field(c))
    s.close()


@pytest.mark.parametrize("prob", ["small", "random", "multilayer_q"])
def test_device_bytes_bounds_what_a_board_allocates(fdtd, prob):
    """fdtd_device_bytes (host only, used for admission) against the device
    memory the created board reports after its first step: never below it,
    and above it by exactly the id width saving (one byte per node and the
    table's 65536 - 256 rows) when the board's ids are 8-bit."""
    p = {"small": W.small_pcb(), "random": W.random_problem(61, 33, 25, 19, upml=3, n_steps=40),
         "multilayer_q": W.multilayer_board(scale=4, n_steps=50)}[prob]
    est = fdtd.device_bytes(p)
    s = fdtd.Solver(p)
    s.step(1)
    inf = s.info()
    s.close()
    nodes = inf["pitch"] * (p.ny + 1) * (p.nz + 1)
    slack = 0 if inf["n_combo"] > 256 else nodes + (65536 - 256) * 16
    assert est == inf["device_bytes"] + slack, (est, inf["device_bytes"], slack)
