"""Benchmark of the Yee + UPML FDTD hot path on GB300 (one JSON line).

Default workload: the large multilayer board (880 x 680 x 100 cells, four
power/ground pairs, 12-cell UPML, 4 sources, 64 probes, running DFT to
10 GHz over a 50000-step solve), FP32.  A bench "step" is a window of
``--window`` leapfrog steps of that solve, each doing the whole hot path
(UPML/boundary H, fused interior H+E, UPML/boundary E, sources, probes, and
the FP64 running-DFT update at the end of the window).  The fields (3 GB in
FP32) are far larger than L2, so no flush is needed between steps.

value  = cell-updates / s (Gcell-updates/s) with inputs resident in HBM.
e2e    = the same metric through the C-ABI with host buffers: every step
         re-uploads the material volume (fdtd_set_materials, host -> device),
         runs the window and copies the spectra back (device -> host).
roofline: the fused interior launch (the dominant kernel), algorithmic
         bytes per node-update (49 B in FP32: 6 fields read + written, 1 id
         byte; 25 B with 16-bit storage) over its mean launch time measured
         with CUDA events on its stream, against the measured HBM copy
         bandwidth; the z-UPML launch (+16 B of auxiliaries per node) is
         reported beside it.
cpu_baseline: the FP64 oracle on the same full-size grid for a few steps.
batched: the batched half of the metric, measured in the same run: 64 uneven
         boards x 5000 steps in one batch (one timed batched solve) against the
         same 64 boards solved one at a time (solves/s of each, their ratio,
         the largest trace difference, clocks).
served / served_fp16: a short Poisson stream (24 requests at 20 req/s,
         boards and steps scaled by 1/4) served by continuous batching
         (solves/s, p50/p99 latency) against the same requests served one at
         a time, in FP32 and FP16 storage.

Other workloads: --workload small | realistic | batched | served (full lines).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Yee+UPML Gcell-updates/s & % HBM roofline; batched/served solves/s, p50/p99 latency"
NOMINAL_HBM_GBS = 7900.0   # GB300 HBM3e nominal bandwidth (context beside the measured copy peak)


def _measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []
        self.thread = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _max_over_ranks(x: float) -> float:
    """Max of a per-rank float over all ranks (identity on one rank): the
    bench's whole-job time.  NCCL reduces a device tensor, gloo a host one."""
    import torch
    dist = torch.distributed
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return x
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _workload(name: str, seed_offset: int = 0):
    from paper_1008_2602_gb300 import workloads as W
    if name == "small":
        return W.small_pcb(seed=1 + seed_offset)
    if name == "realistic":
        return W.realistic_board(seed=2 + seed_offset)
    if name == "multilayer":
        return W.multilayer_board(seed=3 + seed_offset)
    if name == "multilayer_q":
        return W.multilayer_board(seed=3 + seed_offset, scale=4)
    if name == "multilayer_h":
        return W.multilayer_board(seed=3 + seed_offset, scale=2)
    raise ValueError(name)


def _describe(prob, name, window, prec):
    return {"workload": f"{prob.name} ({name}): {prob.nx}x{prob.ny}x{prob.nz} cells, "
                        f"{len(prob.sources)} sources, {len(prob.probes)} probes, UPML {prob.upml_depth[0]} cells, "
                        f"{prob.n_steps}-step solve, step = {window} leapfrog steps",
            "cells": prob.cells, "leapfrog_steps_per_step": window, "precision": prec,
            "l2": "inputs larger than L2 (no flush)" if prob.cells * 48 > 129e6 else
                  "working set fits in L2 (not flushed)"}


def _traffic_for(kernel_tag: str, nodes: int):
    """DRAM bytes per launch of a kernel from the committed ncu summary, if it
    was taken on the current kernel source (scaled to `nodes`)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)[kernel_tag]
        src = os.path.join(ROOT, "paper_1008_2602_gb300", "csrc", "fdtd_kernels.cu")
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        if d.get("kernel_sha") != sha:
            return None
        return d["bytes_per_node"] * nodes
    except Exception:
        return None


def run_single(args, world, rank, local):
    import numpy as np
    import torch
    from paper_1008_2602_gb300 import solver

    dev = local
    torch.cuda.set_device(dev)
    prob = _workload(args.workload, seed_offset=rank)
    window = args.window
    s = solver.Solver(prob, precision=args.precision)
    tune_kw = None
    if args.tile_x or args.tile_y or args.zseg or args.depth or args.pair_zseg:
        tune_kw = dict(tile_x=args.tile_x, tile_y=args.tile_y, zseg=args.zseg, depth=args.depth,
                       pair_zseg=args.pair_zseg)
        s.set_tuning(**tune_kw)
    inf = s.info()
    cells = prob.cells
    interior_nodes = inf["interior_nodes"]
    stream = None

    # warm-up
    for _ in range(args.warmup):
        s.step_profiled(window)
    s.sync()

    if world > 1:
        torch.distributed.barrier()
    phase = np.zeros(6)
    with ClockSampler(dev) as clk:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            phase += s.step_profiled(window)
        s.sync()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
    elapsed = t1 - t0
    elapsed = _max_over_ranks(elapsed)
    dev_ms = float(phase.sum())
    total_updates = float(cells) * window * args.steps * world
    value = total_updates / elapsed / 1e9

    # roofline of the dominant kernel, the fused interior launch: 12 field
    # values + 1 id byte per node.  The z-UPML launch also reads and writes
    # the B~z and D~z auxiliaries of each node (reported beside it).
    es = 4 if args.precision == "fp32" else 2
    bytes_per_node = 12 * es + (2 if inf["n_combo"] > 256 else 1)
    upml_nodes = inf["fused_upml_nodes"]
    int_nodes = interior_nodes - upml_nodes
    alg_bytes = bytes_per_node * int_nodes
    n_launch = window * args.steps
    depth = inf["depth"]
    # depth 2: a window of `window` steps from an even step runs (window - 1) // 2
    # two-step passes and one or two single steps (fdtd_step's split)
    pairs = (window - 1) // 2 if depth == 2 and window >= 3 else 0
    singles = window - 2 * pairs
    t_int = phase[2] / 1e3 / (n_launch if depth == 1 else pairs * args.steps)
    t_zp = phase[1] / 1e3 / n_launch
    achieved = alg_bytes / t_int / 1e9
    zp_bytes = (bytes_per_node + 16) * upml_nodes
    # the two slab launches together: each slab node's 12 field values + id
    # (H and E halves), and every slab auxiliary read and written once
    t_sl = (phase[0] + phase[3]) / 1e3 / n_launch
    sl_bytes = bytes_per_node * inf["slab_nodes"] + 8 * inf["slab_aux_values"]
    # whole leapfrog step: every node's 12 field values + id, the z-UPML
    # auxiliaries and the slab auxiliaries (each read and written once)
    step_bytes = bytes_per_node * (interior_nodes + inf["slab_nodes"]) + 16 * upml_nodes + 8 * inf["slab_aux_values"]
    t_leap = elapsed / (window * args.steps)
    peak, peak_kind = _measured_peaks()
    traffic = _traffic_for(f"{'k_fused_interior' if depth == 1 else 'k_pair'}_{args.precision}", int_nodes)

    # e2e: host buffers through the C-ABI
    e2e = None
    if not args.no_e2e:
        mat = np.ascontiguousarray(prob.mat)
        Q = inf["n_bins"]
        spec = np.zeros((inf["n_probes"], max(Q, 1), 2))
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        # two contexts of the board take the windows in turn: each window ingests its
        # board (host precompute of the node coefficient ids and their H2D from
        # page-locked memory; fdtd_set_materials also resets the context), steps,
        # and reads its spectra back.  A context is ingested for its next window
        # while the other one's window runs on the GPU, and only after its own
        # previous spectra have been read.
        other = solver.Solver(prob, precision=args.precision, tuning=tune_kw)
        ctxs = [s, other]
        specs = [spec, np.zeros_like(spec)]
        te0 = time.perf_counter()
        ctxs[0].set_materials(mat)
        ctxs[0].step(window)
        for w in range(args.e2e_steps):
            cur, nxt = ctxs[w % 2], ctxs[(w + 1) % 2]
            if w + 1 < args.e2e_steps:
                nxt.set_materials(mat)      # host work overlaps window w on the GPU
                nxt.step(window)
            cur.spectra_into(specs[w % 2])  # D2H of window w's FP64 spectra (waits for it)
        te1 = time.perf_counter()
        et = te1 - te0
        et = _max_over_ranks(et)
        h2d = inf["pitch"] * (prob.ny + 1) * (prob.nz + 1) + 256 * 16   # 8-bit ids and their table
        e2e = {"value": float(cells) * window * args.e2e_steps * world / et / 1e9, "unit": "Gcell-updates/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(spec.nbytes),
               "steps": args.e2e_steps,
               "includes": "per window: fdtd_set_materials (host precompute + H2D from page-locked memory), "
                           "fdtd_step, fdtd_probe_spectra (D2H); two contexts alternate windows, so one ingests "
                           "while the other steps"}
        other.close()
    s.close()

    out = {
        "metric": METRIC, "value": round(value, 3), "unit": "Gcell-updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(elapsed / args.steps * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if args.precision == "fp32" else f"{args.precision}-storage/f32-compute",
        "data": "synthetic (seeded board geometry, sources and probes)",
        "config": {**_describe(prob, args.workload, window, args.precision),
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "phase_ms_per_leapfrog_step": {k: round(v / n_launch, 5) for k, v in
                                       zip(["slab_h", "fused_zupml", "fused_interior", "slab_e", "post", "dft_total"],
                                           phase)},
        "roofline": {"bound": "hbm", "kernel": "k_fused interior launch (fused H+E, planes outside the z-UPML)"
                     if depth == 1 else "k_pair two-step interior pass (two leapfrog steps per launch; the phase "
                     "also holds the window's single-step interior launches)",
                     "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4),
                     "frac_of_nominal": round(achieved / NOMINAL_HBM_GBS, 4),
                     "traffic": traffic, "peak_source": peak_kind,
                     "bytes_per_unit": bytes_per_node, "units_per_launch": int_nodes,
                     "algorithmic_bytes_per_launch": alg_bytes, "mean_launch_ms": round(t_int * 1e3, 5)},
        "roofline_step": {"what": "whole leapfrog step (all kernels, wall time per step)",
                          "algorithmic_bytes_per_step": int(step_bytes),
                          "bytes_per_cell": round(step_bytes / cells, 2),
                          "achieved": round(step_bytes / t_leap / 1e9, 1), "peak": peak, "unit": "GB/s",
                          "frac": round(step_bytes / t_leap / 1e9 / peak, 4),
                          "frac_of_nominal": round(step_bytes / t_leap / 1e9 / NOMINAL_HBM_GBS, 4),
                          "roofline_gcell_updates_per_s": round(cells / (step_bytes / (peak * 1e9)) / 1e9, 2)},
        "roofline_zupml": {"kernel": "k_fused z-UPML launch", "bytes_per_unit": bytes_per_node + 16,
                           "units_per_launch": upml_nodes, "mean_launch_ms": round(t_zp * 1e3, 5),
                           "achieved": round(zp_bytes / t_zp / 1e9, 1) if t_zp > 0 else None,
                           "frac": round(zp_bytes / t_zp / 1e9 / peak, 4) if t_zp > 0 else None,
                           "frac_of_nominal": round(zp_bytes / t_zp / 1e9 / NOMINAL_HBM_GBS, 4) if t_zp > 0 else None},
        "roofline_slab": {"kernel": "k_slab_h + k_slab_e (UPML faces, edges, corners, z-UPML rings, wall planes)",
                          "bytes_per_unit": bytes_per_node, "aux_bytes_per_value": 8,
                          "units_per_launch": int(inf["slab_nodes"]), "aux_values": int(inf["slab_aux_values"]),
                          "mean_launch_ms": round(t_sl * 1e3, 5),
                          "achieved": round(sl_bytes / t_sl / 1e9, 1) if t_sl > 0 else None,
                          "frac": round(sl_bytes / t_sl / 1e9 / peak, 4) if t_sl > 0 else None,
                          "frac_of_nominal": round(sl_bytes / t_sl / 1e9 / NOMINAL_HBM_GBS, 4) if t_sl > 0 else None},
        "tuning": {"tile_x": args.tile_x or "default", "tile_y": args.tile_y or "default",
                   "zseg": args.zseg or "default", "depth": depth, "pair_zseg": args.pair_zseg or "default"},
        "gpu_launches": int(args.steps * (singles * (5 if upml_nodes else 4) + pairs * (9 if upml_nodes else 7) + 2)),
        "clocks": clk.summary(),
        "e2e": e2e,
        "device_ms_in_timed_region": round(dev_ms, 3),
    }
    return out


def cpu_baseline(args, sample_steps: int):
    """FP64 oracle on the same full-size workload for a few steps."""
    import oracle
    prob = _workload(args.workload)
    n = os.cpu_count() or 1
    oracle.build()
    t0 = time.perf_counter()
    oracle.run(prob, n_steps=sample_steps, trace=True, dft=False, n_threads=n)
    t1 = time.perf_counter()
    # setup (edge permittivity, grading) is included: it is part of a solve
    v = prob.cells * sample_steps / (t1 - t0) / 1e9
    return {"value": round(v, 6), "unit": "Gcell-updates/s", "cores": n, "kind": "oracle",
            "sample": f"{sample_steps} leapfrog steps of the full {prob.nx}x{prob.ny}x{prob.nz} grid "
                      f"(FP64, OpenMP {n} threads, setup included)"}


def _plain_solves(probs, precision, tuning=None):
    """Each board solved alone, one after the other (per-board launches)."""
    from paper_1008_2602_gb300 import solver
    t0 = time.perf_counter()
    out = []
    for p in probs:
        s = solver.Solver(p, precision=precision, tuning=tuning)
        s.run()
        out.append(s.traces())
        s.close()
    return time.perf_counter() - t0, out


def batched_record(boards, batch_steps, precision, window, steps, warmup, world, rank, local, plain_boards):
    """64 uneven boards (plane sides 20-120 mm, 1-3 pairs, dx=0.5 mm,
    5000 steps each) in one batch; a step is one full batched solve.  The
    same boards (the first `plain_boards` of them) are then solved one at a
    time with per-board launches, and the traces compared."""
    import numpy as np
    import torch
    from paper_1008_2602_gb300 import solver, tune, workloads as W
    torch.cuda.set_device(local)
    probs = W.batch_boards(seed=4 + 100 * rank, n_boards=boards, n_steps=batch_steps)
    # tuned on the first 8 boards of the batch (same board distribution), cached per grid class
    tuning = tune.tune(probs[:8], precision, steps=16, log=lambda m: print(m, file=sys.stderr))
    cells = sum(p.cells * p.n_steps for p in probs)

    def batched_solve(ps):
        b = solver.Batch(tuning=tuning)
        sols = [solver.Solver(p, precision=precision) for p in ps]
        for s_ in sols:
            b.add(s_)
        done = 0
        while done < len(sols):
            done = b.step(window)
        b.sync()
        return b, sols

    for _ in range(warmup):   # same boards, a few chunks each: plans, graphs and pages warm
        b, sols = batched_solve([p.replace(n_steps=min(p.n_steps, 2 * window)) for p in probs])
        b.close()
        for s_ in sols:
            s_.close()
    if world > 1:
        torch.distributed.barrier()
    times, last = [], None
    with ClockSampler(local) as clk:
        for _ in range(steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            b, sols = batched_solve(probs)
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t0)
            if last is not None:
                for s_ in last[1]:
                    s_.close()
                last[0].close()
            last = (b, sols)
    el = _max_over_ranks(sum(times))
    value = len(probs) * steps * world / el
    # per-board plain launches on the same GPU, same boards, and identity of the results
    n_plain = min(plain_boards, len(probs))
    with ClockSampler(local) as clk_plain:
        plain_t, plain_tr = _plain_solves(probs[:n_plain], precision)
    plain_t = _max_over_ranks(plain_t)
    plain_rate = n_plain * world / plain_t
    diffs = [float(np.abs(last[1][q].traces() - plain_tr[q]).max()) for q in range(n_plain)]
    for s_ in last[1]:
        s_.close()
    last[0].close()
    return {"solves_per_s": round(value, 4), "unit": "solves/s", "boards": len(probs), "steps_per_board": batch_steps,
            "cells_total": int(sum(p.cells for p in probs)), "timed_solves": steps, "wall_s": round(el, 3),
            "gcell_updates_per_s": round(cells * steps * world / el / 1e9, 3), "tuning": tuning,
            "plain": {"solves_per_s": round(plain_rate, 4), "boards": n_plain, "wall_s": round(plain_t, 3),
                      "same_boards": n_plain == len(probs), "clocks": clk_plain.summary()},
            "batched_over_plain": round(value / plain_rate, 3),
            "batched_vs_alone_max_abs_trace_diff": max(diffs), "clocks": clk.summary()}


def served_record(requests, rate, step_scale, cell_scale, precision, window, hbm_budget_gb, world, rank, local,
                  plain_requests):
    """Poisson request stream of multilayer boards, admitted by HBM budget
    into one continuously batched mix (p50/p99 latency, solves/s); the same
    requests (the first `plain_requests`) served one at a time with
    per-board launches, honouring the arrival times."""
    import numpy as np
    import torch
    from paper_1008_2602_gb300 import serve, solver, workloads as W
    torch.cuda.set_device(local)
    # one stream for the whole job; with several ranks the router gives each
    # rank its share (no exchange between ranks)
    reqs = W.request_stream(seed=5, n_requests=requests, rate=rate, step_scale=step_scale, cell_scale=cell_scale)
    if world > 1:
        reqs = [r for r, k in zip(reqs, serve.route(reqs, world)) if k == rank]
    warm = W.request_stream(seed=99, n_requests=4, rate=1000.0, step_scale=0.02, cell_scale=0.05)
    be = serve.CudaBackend(precision=precision)
    serve.Server(be, hbm_budget=int(hbm_budget_gb * 2**30), chunk=window).run(warm)
    be.close()
    if world > 1:
        torch.distributed.barrier()
    be = serve.CudaBackend(precision=precision)
    srv = serve.Server(be, hbm_budget=int(hbm_budget_gb * 2**30), chunk=window)
    with ClockSampler(local) as clk:
        t0 = time.perf_counter()
        res = srv.run(reqs)
        wall = time.perf_counter() - t0
    be.close()
    summ = serve.summarize(res, _max_over_ranks(wall))
    summ["solves_per_s"] = requests / summ["wall_s"]      # the whole stream over the slowest rank
    # the same requests one at a time (per-board plain launches)
    n_plain = min(plain_requests, len(reqs))
    lat = []
    with ClockSampler(local) as clk_plain:
        start = time.perf_counter()
        for r in reqs[:n_plain]:
            now = time.perf_counter() - start
            if now < r.arrival:
                time.sleep(r.arrival - now)
            s_ = solver.Solver(r.problem, precision=precision)
            s_.run()
            s_.spectra()
            s_.close()
            lat.append(time.perf_counter() - start - r.arrival)
        plain_wall = _max_over_ranks(time.perf_counter() - start)
    plain_rate = (n_plain * world if world == 1 else requests * n_plain / max(len(reqs), 1)) / plain_wall
    return {"solves_per_s": round(summ["solves_per_s"], 4), "unit": "solves/s",
            "p50_latency_s": round(summ["p50_latency_s"], 4), "p99_latency_s": round(summ["p99_latency_s"], 4),
            "requests": len(reqs), "rate_req_per_s": rate, "precision": precision, "chunk_steps": window,
            "stream": f"lognormal cells median {2e6 * cell_scale:.3g} (max {40e6 * cell_scale:.3g}), "
                      f"{int(2000 * step_scale)}-{int(20000 * step_scale)} steps, 4-32 probes",
            "wall_s": round(summ["wall_s"], 3), "gcell_updates_per_s": round(summ["gcell_updates_per_s"], 3),
            "plain": {"solves_per_s": round(plain_rate, 4), "requests": n_plain, "same_requests": n_plain == len(reqs),
                      "p50_latency_s": round(float(np.percentile(lat, 50)), 4),
                      "p99_latency_s": round(float(np.percentile(lat, 99)), 4), "clocks": clk_plain.summary()},
            "served_over_plain": round(summ["solves_per_s"] / plain_rate, 3), "clocks": clk.summary()}


def run_batched(args, world, rank, local):
    rec = batched_record(args.boards, args.batch_steps, args.precision, args.window, args.steps, args.warmup, world,
                         rank, local, args.plain_boards)
    return {"metric": METRIC, "value": rec["solves_per_s"], "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(rec["wall_s"] / args.steps * 1e3, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else
            f"{args.precision}-storage/f32-compute", "data": "synthetic (seeded boards, sources, probes)",
            "config": {"workload": f"batched: {args.boards} boards (plane sides 20-120 mm, 1-3 pairs, dx=dy=0.5 mm, "
                                   f"dz=0.2 mm, 6-cell air, 10-cell UPML), {args.batch_steps} steps each; "
                                   "step = one batched solve of all boards",
                       "cells_total": rec["cells_total"], "tuning": rec["tuning"],
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "batched": rec, "gpu_launches": None, "clocks": rec["clocks"], "e2e": None}


def run_served(args, world, rank, local):
    rec = served_record(args.requests, args.rate, args.step_scale, args.cell_scale, args.precision, args.window,
                        args.hbm_budget_gb, world, rank, local, args.plain_requests)
    return {"metric": METRIC, "value": rec["solves_per_s"], "unit": "solves/s", "n_gpus": world,
            "steps": 1, "warmup": 1, "ms_per_step": round(rec["wall_s"] * 1e3, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.precision == "fp32" else f"{args.precision}-storage/f32-compute",
            "data": "synthetic (seeded Poisson stream of boards)",
            "config": {"workload": f"served: {args.requests} requests, Poisson {args.rate} req/s, {rec['stream']}",
                       "chunk_steps": args.window, "hbm_budget_gb": args.hbm_budget_gb,
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "served": rec, "gpu_launches": None, "clocks": rec["clocks"], "e2e": None}


def run_reference(args, world, rank):
    """Reference arm: the FP64 oracle timed as it stands on the host cores."""
    if rank != 0:
        return None
    import oracle
    prob = _workload(args.workload)
    n = os.cpu_count() or 1
    oracle.build()
    per = max(1, args.ref_sample_steps)
    for _ in range(max(1, args.warmup)):   # untimed samples of the same size
        oracle.run(prob, n_steps=per, trace=True, dft=False, n_threads=n)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.run(prob, n_steps=per, trace=True, dft=False, n_threads=n)
        times.append(time.perf_counter() - t0)
    el = sum(times)
    v = prob.cells * per * args.steps / el / 1e9
    sample = (f"each step: {per} leapfrog steps of the full {prob.nx}x{prob.ny}x{prob.nz} grid "
              f"(FP64 oracle, OpenMP {n} threads, setup included)")
    return {"impl": "reference", "metric": METRIC, "value": round(v, 6), "unit": "Gcell-updates/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(el / args.steps * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded board geometry, sources and probes)",
            "config": _describe(prob, args.workload, per, "fp64"),
            "cpu_baseline": {"value": round(v, 6), "unit": "Gcell-updates/s", "cores": n, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(v, 6), "unit": "Gcell-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="multilayer",
                    choices=["small", "realistic", "multilayer", "multilayer_h", "multilayer_q", "batched", "served"])
    ap.add_argument("--boards", type=int, default=64)
    ap.add_argument("--batch-steps", type=int, default=5000)
    ap.add_argument("--plain-boards", type=int, default=64, help="boards also solved one at a time (same set)")
    ap.add_argument("--requests", type=int, default=64)
    ap.add_argument("--rate", type=float, default=20.0)
    ap.add_argument("--step-scale", type=float, default=1.0)
    ap.add_argument("--cell-scale", type=float, default=1.0)
    ap.add_argument("--plain-requests", type=int, default=64, help="requests also served one at a time (same set)")
    ap.add_argument("--hbm-budget-gb", type=float, default=200.0)
    ap.add_argument("--window", type=int, default=200)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp16"])
    ap.add_argument("--tile-x", type=int, default=0, help="fused tile width (62 or 124 columns); 0 = tuned default")
    ap.add_argument("--tile-y", type=int, default=0, help="fused tile height (4 or 8 rows); 0 = tuned default")
    ap.add_argument("--zseg", type=int, default=0, help="fused z-segment length; 0 = tuned default")
    ap.add_argument("--depth", type=int, default=0, help="leapfrog steps per interior pass (1 or 2); 0 = default")
    ap.add_argument("--pair-zseg", type=int, default=0, help="z-segment length of the two-step pass; 0 = default")
    ap.add_argument("--no-batched", action="store_true", help="default run: skip the batched sub-record")
    ap.add_argument("--no-served", action="store_true", help="default run: skip the served sub-records")
    ap.add_argument("--sub-requests", type=int, default=24, help="default run: requests of the served sub-record")
    ap.add_argument("--sub-step-scale", type=float, default=0.25)
    ap.add_argument("--sub-cell-scale", type=float, default=0.25)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-steps", type=int, default=6)
    ap.add_argument("--ref-sample-steps", type=int, default=2)
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3) if args.impl == "ours" else args.warmup

    world, rank, local = _dist()
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl" if args.impl == "ours" else "gloo")
    if args.impl == "reference":
        out = run_reference(args, world, rank)
        if out is not None:
            print(json.dumps(out), flush=True)
        return
    if args.workload in ("batched", "served"):
        out = (run_batched if args.workload == "batched" else run_served)(args, world, rank, local)
        if rank == 0:
            print(json.dumps(out), flush=True)
        if world > 1:
            import torch
            torch.distributed.barrier()
            torch.distributed.destroy_process_group()
        return
    out = run_single(args, world, rank, local)
    # the batched and served halves of the metric, measured in the same run
    # on their own workloads (compact records; --workload batched | served
    # gives the full lines)
    if not args.no_batched:
        out["batched"] = batched_record(args.boards, args.batch_steps, args.precision, args.window, 1, 1, world, rank,
                                        local, args.boards)
    if not args.no_served:
        out["served"] = served_record(args.sub_requests, args.rate, args.sub_step_scale, args.sub_cell_scale,
                                      args.precision, args.window, args.hbm_budget_gb, world, rank, local,
                                      args.sub_requests)
        if args.precision == "fp32":
            out["served_fp16"] = served_record(args.sub_requests, args.rate, args.sub_step_scale, args.sub_cell_scale,
                                               "fp16", args.window, args.hbm_budget_gb, world, rank, local,
                                               args.sub_requests)
    if rank == 0:
        if not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(args, args.cpu_sample_steps)
        else:
            out["cpu_baseline"] = None
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
