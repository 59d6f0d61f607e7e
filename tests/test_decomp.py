"""Host-side logic of the single-board slab decomposition (decomp.py), on CPU:

* every part's per-node edge coefficients (fdtd_node_coefficients, host
  only) equal the undivided board's on the node planes the part owns, and on
  the shared cell row for E_y, so each part updates its nodes with the
  board's coefficients;
* sources and probes land where they belong (E_y sources on a shared row in
  both parts, every probe in exactly one part);
* the halo schedule, run between two gloo ranks on host arrays with the same
  exchange_ranks() the GPU path uses, leaves every part's outer cut planes
  equal to the neighbour's owned values; and on three parts in one process.
"""
import ctypes
import os
import socket

import numpy as np
import pytest

from paper_1008_2602_gb300 import decomp, workloads as W


def _node_coefs(prob):
    """[nz+1][ny+1][nx+1] x 3 edge coefficients (ce_x, ce_y, ce_z) of a problem."""
    from paper_1008_2602_gb300 import capi as C
    g = C.fdtd_grid(prob.nx, prob.ny, prob.nz, prob.dx, prob.dy, prob.dz, prob.courant, prob.dt)
    b = C.fdtd_boundary()
    b.depth[:] = list(prob.upml_depth)
    b.m, b.R0, b.kappa_max = prob.upml_m, prob.upml_R0, prob.upml_kappa_max
    b.wall[:] = list(prob.walls)
    mat = np.ascontiguousarray(prob.mat, np.uint8)
    eps = np.ascontiguousarray(prob.eps_r, np.float64)
    boxes = np.ascontiguousarray(prob.pec_boxes, np.int32).reshape(-1, 6)
    ids = np.zeros((prob.nz + 1, prob.ny + 1, prob.nx + 1), np.uint16)
    table = np.zeros((65536, 4), np.float32)
    n = ctypes.c_int()
    C.fdtd_node_coefficients(ctypes.byref(g), mat.ctypes.data, eps.ctypes.data, len(eps),
                             boxes.ctypes.data if len(boxes) else None, len(boxes), None, ctypes.byref(b),
                             ids.ctypes.data, table.ctypes.data, 65536, ctypes.byref(n))
    return table[ids][..., :3]


@pytest.mark.parametrize("cuts", [[9], [6, 14], [4, 8, 12]])
def test_parts_carry_the_boards_coefficients(cuts):
    p = W.random_problem(31, 17, 21, 11, upml=3, n_steps=20)
    # a PEC sheet crossing the cuts, and one ending exactly on a cut plane
    p = p.replace(pec_boxes=np.array([[4, 12, 2, 18, 5, 5], [6, 10, 1, cuts[0], 7, 8]], np.int32))
    whole = _node_coefs(p)
    sp = decomp.split_y(p, cuts)
    for part in sp.parts:
        c = _node_coefs(part.problem)
        lo = part.lo
        own = slice(part.own_lo - lo, part.own_hi - lo + 1)
        assert np.array_equal(c[:, own, :, 0], whole[:, part.own_lo:part.own_hi + 1, :, 0])
        assert np.array_equal(c[:, own, :, 2], whole[:, part.own_lo:part.own_hi + 1, :, 2])
        # E_y on every cell row of the part (shared rows included)
        assert np.array_equal(c[:, :-1, :, 1], whole[:, part.lo:part.hi, :, 1])


def test_ports_are_assigned_to_owners():
    p = W.random_problem(32, 15, 24, 10, upml=3, n_steps=20)
    cuts = [9, 15]
    extra_src = np.array([[5, 9, 4, 1], [6, 10, 5, 0], [7, 15, 3, 2], [8, 9, 2, 2]], np.int32)
    extra_prb = np.array([[5, 9, 4, 1], [6, 10, 5, 0], [7, 15, 3, 2], [7, 16, 3, 2], [3, 15, 2, 1]], np.int32)
    p = p.replace(sources=np.vstack([p.sources, extra_src]),
                  source_params=np.vstack([p.source_params, np.tile(p.source_params[:1], (4, 1))]),
                  probes=np.vstack([p.probes, extra_prb]))
    sp = decomp.split_y(p, cuts)
    # every probe in exactly one part, at the same global edge
    seen = sorted(q for part in sp.parts for q in part.probe_ids)
    assert seen == list(range(len(p.probes)))
    for part in sp.parts:
        for row, q in enumerate(part.probe_ids):
            g = p.probes[q]
            loc = part.problem.probes[row]
            assert (loc[0], loc[1] + part.lo, loc[2], loc[3]) == tuple(g)
    # sources: E_y on a shared row (9 and 15) in both parts holding it, others once
    count = {}
    for part in sp.parts:
        for s in part.problem.sources:
            key = (int(s[0]), int(s[1]) + part.lo, int(s[2]), int(s[3]))
            count[key] = count.get(key, 0) + 1
    for s in p.sources:
        key = tuple(int(x) for x in s)
        expect = 2 if key[3] == 1 and key[1] in cuts else 1
        assert count[key] == expect, key


def test_cuts_inside_the_upml_or_too_close_are_refused():
    p = W.random_problem(33, 12, 30, 10, upml=4, n_steps=10)
    for bad in ([2], [27], [10, 11], [0]):
        with pytest.raises(ValueError):
            decomp.split_y(p, bad)


def _parts_of(arr, sp):
    """Host copies of a global [nz+1][ny+1][nx+1] array per part, with the
    cut planes the part cannot compute replaced by NaN."""
    out = []
    for c, part in enumerate(sp.parts):
        a = arr[:, part.lo:part.hi + 1].copy()
        if c > 0:
            a[:, 0] = np.nan
        if c < len(sp.parts) - 1:
            a[:, -1] = np.nan
        out.append(a)
    return out


def test_three_parts_exchange_in_one_process():
    p = W.random_problem(34, 9, 26, 7, upml=2, n_steps=10)
    sp = decomp.split_y(p, [7, 16])
    rng = np.random.default_rng(0)
    glob = rng.standard_normal((p.nz + 1, p.ny + 1, p.nx + 1))
    parts = _parts_of(glob, sp)
    for dst, dplane, src, splane in sp.exchanges():
        parts[dst][:, dplane] = parts[src][:, splane]
    for part, a in zip(sp.parts, parts):
        assert np.array_equal(a, glob[:, part.lo:part.hi + 1])


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _gloo_rank(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p = W.random_problem(35, 8, 30, 6, upml=3, n_steps=10)
        sp = decomp.split_y(p, decomp.even_cuts(p, world))
        rng = np.random.default_rng(1)
        glob = rng.standard_normal((2, p.nz + 1, p.ny + 1, p.nx + 1)).astype(np.float32)   # E_x, E_z
        part = sp.parts[rank]
        mine = glob[:, :, part.lo:part.hi + 1].copy()
        if rank > 0:
            mine[:, :, 0] = 0
        if rank < world - 1:
            mine[:, :, -1] = 0

        def pack(plane):
            return torch.from_numpy(np.ascontiguousarray(mine[:, :, plane]).reshape(-1))

        def unpack(plane, h):
            mine[:, :, plane] = h[1].numpy().reshape(2, p.nz + 1, p.nx + 1)

        def send(buf, peer):
            return (dist.isend(buf, peer), buf)

        def recv(plane, peer):
            buf = torch.empty(2 * (p.nz + 1) * (p.nx + 1), dtype=torch.float32)
            return (dist.irecv(buf, peer), buf)

        def wait(handles):
            for w, _ in handles:
                w.wait()

        decomp.exchange_ranks(sp, rank, pack, unpack, send, recv, wait)
        q.put((rank, bool(np.array_equal(mine, glob[:, :, part.lo:part.hi + 1]))))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_exchange_the_cut_planes():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_gloo_rank, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    for pr in procs:
        pr.join(120)
    res = dict(q.get(timeout=5) for _ in range(2))
    assert res == {0: True, 1: True}
