"""A board split into sub-boards along y (decomp.py), stepped with the halo
exchange of fdtd_halo_copy / fdtd_halo_pack / fdtd_halo_unpack, against the
same board stepped whole: every owned field element and every probe trace
bitwise equal, spectra equal to FP64 rounding, and the FP64 oracle at the
FP32 target.  Two and three parts on one GPU through fdtd_halo_copy; two
ranks (processes) sharing the GPU through pack / gloo / unpack."""
import os
import socket

import numpy as np
import pytest

import oracle
from paper_1008_2602_gb300 import decomp, workloads as W

pytestmark = pytest.mark.gpu


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


def _problem():
    p = W.random_problem(51, 40, 44, 26, upml=4, n_steps=160)
    # ports on both sides of the cuts and on the shared rows (E_y on row 19 and 29)
    src = np.vstack([p.sources, [[20, 19, 12, 1], [9, 20, 10, 2], [30, 29, 14, 1]]]).astype(np.int32)
    prm = np.vstack([p.source_params, np.tile(p.source_params[:1], (3, 1))])
    prb = np.vstack([p.probes, [[20, 19, 12, 1], [9, 20, 10, 2], [12, 19, 9, 0], [30, 30, 14, 2]]]).astype(np.int32)
    return p.replace(sources=src, source_params=prm, probes=prb)


@pytest.mark.parametrize("cuts", [[19], [19, 29]])
def test_split_board_equals_whole_board(fdtd, ncpu, cuts):
    p = _problem()
    whole = fdtd.Solver(p)
    whole.run()
    sp = decomp.SplitSolver(p, cuts)
    sp.run()
    for c in range(6):
        assert np.array_equal(sp.field(c), whole.field(c)), c
    assert np.array_equal(sp.traces(), whole.traces())
    a, b = sp.spectra(), whole.spectra()
    assert np.allclose(a, b, rtol=0, atol=1e-12 * np.abs(b).max())
    ref = oracle.run(p, n_threads=ncpu)
    tr = sp.traces()
    for q in range(len(tr)):
        if np.abs(ref["trace"][q]).max() > 0:
            assert rel_l2(tr[q], ref["trace"][q]) <= 1e-4, q
    sp.close()
    whole.close()


def test_split_quarter_scale_multilayer_board(fdtd):
    """The quarter-scale multilayer board (280x230x100, 12-cell UPML, four
    plane pairs) cut in two: probe traces bitwise equal to the whole board."""
    p = W.multilayer_board(scale=4, n_steps=120)
    whole = fdtd.Solver(p)
    whole.run()
    sp = decomp.SplitSolver(p, decomp.even_cuts(p, 2))
    sp.run()
    assert np.array_equal(sp.traces(), whole.traces())
    assert np.array_equal(sp.field(2), whole.field(2))
    sp.close()
    whole.close()


def test_halo_calls_reject_bad_arguments(fdtd):
    from paper_1008_2602_gb300 import capi as C
    p = _problem()
    sp = decomp.SplitSolver(p, [19])
    a, b = sp.solvers
    with pytest.raises(C.FdtdError):
        C.fdtd_halo_copy(a.ctx, 0, b.ctx, 1, 3, decomp.TANGENTIAL_Y)      # bad axis
    with pytest.raises(C.FdtdError):
        C.fdtd_halo_copy(a.ctx, 0, b.ctx, 1, 1, 0)                        # empty mask
    with pytest.raises(C.FdtdError):
        C.fdtd_halo_copy(a.ctx, 0, b.ctx, 999, 1, decomp.TANGENTIAL_Y)    # plane out of range
    with pytest.raises(C.FdtdError):
        C.fdtd_halo_copy(a.ctx, 0, b.ctx, 1, 0, decomp.TANGENTIAL_Y)      # x planes differ in shape
    a.step(1)
    with pytest.raises(C.FdtdError) as ei:
        C.fdtd_halo_copy(a.ctx, 0, b.ctx, 1, 1, decomp.TANGENTIAL_Y)      # different step counts
    assert ei.value.code == C.FDTD_ESTATE
    sp.close()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p = _problem()
        d = decomp.DistributedSplitSolver(p, rank, world)
        d.step(p.n_steps)
        d.s.sync()
        q.put((rank, d.part.probe_ids, d.s.traces(), d.s.field(2), d.part.lo, d.part.own_lo, d.part.own_hi))
        d.close()
    finally:
        dist.destroy_process_group()


def test_two_ranks_with_pack_and_unpack(fdtd):
    """Two processes, one part each, sharing the GPU: the halo planes are
    packed by the library, sent through gloo (host memory) and unpacked.
    No kernel waits on another process; the exchange is host-side."""
    torch = pytest.importorskip("torch")
    p = _problem()
    whole = fdtd.Solver(p)
    whole.run()
    tr_w, ez_w = whole.traces(), whole.field(2)
    whole.close()
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    got = [q.get(timeout=600) for _ in range(2)]
    for pr in procs:
        pr.join(60)
    for rank, pids, tr, ez, lo, own_lo, own_hi in got:
        for row, g in enumerate(pids):
            assert np.array_equal(tr[row], tr_w[g]), (rank, g)
        assert np.array_equal(ez[:, own_lo - lo:own_hi - lo + 1], ez_w[:, own_lo:own_hi + 1]), rank
