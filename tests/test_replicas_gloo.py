"""Multi-GPU host logic on CPU: ``bench.py --gpus N`` runs N independent
replicas (one board or batch per rank, no data-path collective; the served
stream is one stream split across the ranks by ``serve.route``) and reports
the whole-job throughput over the slowest rank.  Here two gloo ranks on
127.0.0.1 check the cross-rank max, that the replicas draw different seeded
inputs of the same shape, and that the routed stream is served exactly once
across the ranks."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    try:
        dist.init_process_group("gloo", rank=rank, world_size=world)
        import bench
        from paper_1008_2602_gb300 import workloads as W
        # whole-job time is the slowest rank's
        t = bench._max_over_ranks(1.0 + 0.75 * rank)
        # replica inputs: same shapes, different seeded content per rank
        p = bench._workload("small", seed_offset=rank)
        probs = W.batch_boards(seed=4 + 100 * rank, n_boards=3, n_steps=10)
        sig = (p.mat.shape, int(p.mat.sum()), tuple(p.sources.ravel()), [b.cells for b in probs])
        out = [None] * world
        dist.all_gather_object(out, sig)
        dist.barrier()
        dist.destroy_process_group()
        q.put((rank, t, out))
    except Exception as e:   # report, never hang the parent
        q.put((rank, None, repr(e)))


def test_two_gloo_replicas_max_and_inputs():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = {}
    for _ in range(world):
        rank, t, out = q.get(timeout=240)
        res[rank] = (t, out)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank in range(world):
        t, out = res[rank]
        assert t is not None, out
        assert t == pytest.approx(1.75)
    sigs = res[0][1]
    assert sigs == res[1][1]                       # every rank saw the same gathered list
    (shape0, sum0, src0, cells0), (shape1, sum1, src1, cells1) = sigs
    assert shape0 == shape1                       # same workload shape on every replica
    assert (sum0, src0) != (sum1, src1) or cells0 != cells1   # different seeded content
    assert cells0 != cells1


def test_max_over_ranks_is_identity_without_a_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert not dist.is_initialized()
    assert bench._max_over_ranks(3.25) == 3.25


def _route_rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    try:
        dist.init_process_group("gloo", rank=rank, world_size=world)
        from paper_1008_2602_gb300 import serve, workloads as W
        from test_serve import FakeBackend
        reqs = W.request_stream(seed=5, n_requests=30, rate=40.0, step_scale=0.05, cell_scale=0.02)
        mine = [r for r, k in zip(reqs, serve.route(reqs, world)) if k == rank]
        res = serve.Server(FakeBackend(), hbm_budget=1 << 40, chunk=50, simulate_clock=True).run(mine)
        out = [None] * world
        dist.all_gather_object(out, sorted(x.rid for x in res))
        dist.barrier()
        dist.destroy_process_group()
        q.put((rank, out, [r.rid for r in reqs]))
    except Exception as e:
        q.put((rank, None, repr(e)))


def test_routed_stream_is_served_once_across_two_gloo_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_route_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict((rank, (out, all_ids)) for rank, out, all_ids in (q.get(timeout=240) for _ in range(world)))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out, all_ids = res[0]
    assert out is not None, all_ids
    assert res[1][0] == out                              # every rank gathered the same shares
    assert sorted(out[0] + out[1]) == sorted(all_ids)   # each request served exactly once
    assert out[0] and out[1]                             # both ranks got work
