#!/usr/bin/env python
"""Benchmark of the GB300 exponential-Krylov solver: frequency responses/s.

One step = the whole hot path for one batch: the responses y_j(T) of eq.
(ode) at the workload's frequencies and their output-plane fields, on seeded
synthetic random-scatterer media.  The default workload restarts in Krylov
dimension with one basis per restart for all 32 frequencies (Fig. alg:rst);
the other workloads run the time-restarted plain method (batched), the
asymptotic splitting, the uneven multi-problem batch and the adjoint.

    python bench.py [--gpus N --steps K --warmup W] [--workload NAME] [--impl reference]

Prints one JSON line (rank 0).  Under torchrun (N > 1) every rank solves
its own replica (independent problems, no data-path collective; weak
scaling); the barrier and max-over-ranks timing use torch.distributed.
"""
import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "freq responses/s at 1e-6 rel err vs per-freq Krylov; A·v+GS HBM GB/s"

# DRAM bytes / algorithmic bytes per launch of the Arnoldi kernels, from ncu
# captures of one launch (single basis, step j = 60): the single sweep at
# 128^3, the default workload itself (3149.6 MB against 3145.7 MB).  None
# where the kernel has changed since its capture (pass A: 32-bit index
# arithmetic; pass B: the compensated update).  Set to None whenever those
# kernels change.
NCU_TRAFFIC_RATIO = {"k_pass_a": None, "k_pass_b": None, "k_sw_pass": 1.001}

WORKLOADS = {
    # 3D Yee 64^3, random eps=2.25 spheres (fill 0.3, r 2-5), 8-cell layer,
    # Ex plane source, FP32 vectors / FP64 projected, m = 64, T = 400
    "3d64_m64_T400": dict(dim=3, n=64, seed=1709, fill=0.3, T=400.0, m=64, nfreq=1,
                          prec="fp32", method="split", rtol=1e-7),
    "3d64_m64_T400_plain": dict(dim=3, n=64, seed=1709, fill=0.3, T=400.0, m=64, nfreq=1,
                                prec="fp32", method="plain", rtol=1e-7),
    # the same medium at 8 / 32 frequencies in [0.8, 1.2] Omega0, advanced in lockstep batches
    "3d64_m64_T400_8f_plain": dict(dim=3, n=64, seed=1709, fill=0.3, T=400.0, m=64, nfreq=8,
                                   prec="fp32", method="plain", rtol=1e-7, batch=8),
    "3d64_m64_T400_32f": dict(dim=3, n=64, seed=1709, fill=0.3, T=400.0, m=64, nfreq=32,
                              prec="fp32", method="plain", rtol=1e-7, batch=32),
    # the same 32 frequencies by restart in Krylov dimension: one basis per
    # restart for all of them (Corollary 2, Fig. alg:rst)
    "3d64_m64_T400_32f_rst": dict(dim=3, n=64, seed=1709, fill=0.3, T=400.0, m=64, nfreq=32,
                                  prec="fp32", method="rstdim", rtol=1e-7, rst_samples=4096,
                                  batch=2),
    "3d96_32f_T400_rst": dict(dim=3, n=96, seed=1713, fill=0.3, T=400.0, m=64, nfreq=32,
                              prec="fp32", method="rstdim", rtol=1e-7, rst_samples=4096,
                              batch=2),
    "3d128_32f_T400_rst": dict(dim=3, n=128, seed=1710, fill=0.3, T=400.0, m=64, nfreq=32,
                               prec="fp32", method="rstdim", rtol=1e-7, rst_samples=4096,
                               batch=2),
    # source splitting (eq. (split2)) on the 64^3 medium, 32 frequencies in lockstep
    "3d64_m64_T400_32f_split2": dict(dim=3, n=64, seed=1709, fill=0.3, T=400.0, m=64, nfreq=32,
                                     prec="fp32", method="split2", rtol=1e-7, batch=32),
    # the neighbouring-frequency difference (eq. (4diff)) against the plain
    # split, on a 2D cavity whose stationary parts converge: 8 frequencies
    # 0.001 Omega0 apart (the paper's step)
    "2d12_m40_T60_8f_split4d": dict(dim=2, n=12, ndisks=2, seed=1708, T=60.0, m=40, nfreq=8, prec="fp64",
                                    method="split4d", rtol=1e-11, batch=8, band=(1.0, 1.007)),
    "2d12_m40_T60_8f_split": dict(dim=2, n=12, ndisks=2, seed=1708, T=60.0, m=40, nfreq=8, prec="fp64",
                                  method="split", rtol=1e-11, batch=8, band=(1.0, 1.007)),
    # config 1 with the paper's perfectly matched layer (auxiliary field P,
    # quadratic sigma up to 3 over the 6-cell layers)
    "2d64_m30_T200_pml": dict(dim=2, n=64, seed=1708, T=200.0, m=30, nfreq=1, prec="fp64",
                              method="plain", rtol=1e-11, pml=True),
    # 2D 64^2, 40 disks, FP64, m = 30, T = 200, plain method
    "2d64_m30_T200": dict(dim=2, n=64, seed=1708, T=200.0, m=30, nfreq=1, prec="fp64",
                          method="plain", rtol=1e-11),
    # 3D 128^3, 32 frequencies in [0.8, 1.2] Omega0 (the multi-frequency batch)
    "3d128_32f_T400": dict(dim=3, n=128, seed=1710, fill=0.3, T=400.0, m=64, nfreq=32,
                           prec="fp32", method="plain", rtol=1e-7, batch=16),
    # uneven batch: 48 instances, sizes U{32..96}^3, 4 frequencies each, concurrent
    "uneven48_4f": dict(kind="uneven", count=48, seed=1711, T=400.0, m=64, nfreq=4, prec="fp32",
                        method="plain", rtol=1e-7, threads=8),
    # the same instances, each by restart in Krylov dimension (one basis per
    # restart for its 4 frequencies)
    "uneven48_4f_rst": dict(kind="uneven", count=48, seed=1711, T=400.0, m=64, nfreq=4, prec="fp32",
                            method="rstdim", rtol=1e-7, threads=8, rst_samples=4096),
    # 48 instances with sizes from {32, 36, ..., 96}^3 (x a multiple of 4), by
    # restart in Krylov dimension: batched (one launch per Arnoldi phase for
    # all instances, autotuned split) and, for comparison, the host-thread
    # driver on the same instances
    "uneven48_4f_rst_batch": dict(kind="uneven", count=48, seed=1711, T=400.0, m=64, nfreq=4, prec="fp32",
                                  method="rstdim", rtol=1e-7, rst_samples=4096, step=4, batched=True),
    "uneven48x4_4f_rst_threads": dict(kind="uneven", count=48, seed=1711, T=400.0, m=64, nfreq=4, prec="fp32",
                                      method="rstdim", rtol=1e-7, threads=8, rst_samples=4096, step=4),
    # adjoint: 3D 96^3, 8 frequencies, gradient of the summed output-plane intensity
    "adjoint3d96_8f": dict(kind="adjoint", dim=3, n=96, seed=1712, fill=0.3, T=400.0, m=64, nfreq=8,
                           prec="fp32", method="plain", rtol=1e-7, checkpoints=128),
}
DEFAULT = "3d128_32f_T400_rst"


def shard_frequencies(nfreq, rank, world, lo=0.8, hi=1.2):
    """This rank's frequencies: every rank gets nfreq of the world * nfreq
    frequencies spread over [lo, hi] * Omega0, interleaved (weak scaling; the
    responses are independent, no data-path collective)."""
    import scenario as S
    allf = S.freq_list(nfreq * world, lo, hi)
    return allf[rank::world]


def scenario_for(w, rank=0, world=1):
    import scenario as S
    if w["dim"] == 2 and w.get("pml"):
        sc = S.config_2d_pml(n=w["n"], seed=w["seed"], T=w["T"], m=w["m"], ndisks=w.get("ndisks", 40))
    elif w["dim"] == 2:
        sc = S.config_2d(n=w["n"], seed=w["seed"], T=w["T"], m=w["m"], ndisks=w.get("ndisks", 40))
    else:
        sc = S.config_3d(n=w["n"], seed=w["seed"], fill=w["fill"], T=w["T"], m=w["m"])
    lo, hi = w.get("band", (0.8, 1.2))
    sc.omegas = shard_frequencies(w["nfreq"], rank, world, lo, hi) if w["nfreq"] > 1 else S.freq_list(1)
    return sc


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self):
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self, dev_index=0):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                if int(parts[0]) != dev_index:
                    continue
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(n_gpus):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
        return rank, world, local, dist
    return 0, 1, 0, None


def barrier_max(dist, value):
    """Max of a host value over ranks (CUDA tensor under NCCL, CPU under gloo)."""
    if dist is None:
        return value
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def config_of(args, w, sc, world=1):
    """The workload description both arms print."""
    return {"workload": args.workload, "grid": list(sc.grid.n), "unknowns": sc.grid.nunk,
            "T": w["T"], "krylov_dim": w["m"], "nfreq": w["nfreq"], "method": w["method"],
            "projected": "f64", "arnoldi": args.arnoldi, "parallelism": f"replicas{world}",
            "l2": "working set (Krylov basis) larger than L2; no flush"}


class OraclePieces:
    """The FP64 oracle, as it stands, on the workload's full grid: the exact
    response y_f(T) by its augmented route (``oracle.exact.y_plain_pieces``,
    scipy expm_multiply), advanced one sub-interval ("piece") of [0, T] per
    call, for two seeded frequencies of the workload in turn.

    A response takes ``pieces`` calls, all of the same length and the same
    work (same matrix, same interval), so responses done = calls / pieces
    exactly; nothing is extrapolated.  The piece length puts ||dt L||_1 near
    10 (eta = ||g||_1 keeps the source column of L at unit 1-norm): one
    Taylor segment of scipy's largest degree and no norm estimation per
    piece.  One call over all of [0, T] would instead run a norm estimation
    and then about the same number of operator products per unit time."""

    def __init__(self, w, sc):
        from oracle import exact, pml, yee
        self.exact = exact
        op = pml.PmlOperator(sc.grid, sc.eps_cell) if getattr(sc.grid, "pml", 0) else yee.Operator(sc.grid, sc.eps_cell)
        t0 = time.perf_counter()
        self.A = op.matrix()
        self.setup_s = time.perf_counter() - t0
        self.g = sc.g
        self.T = w["T"]
        nf = len(sc.omegas)
        rng = np.random.default_rng(1707 + 3)
        self.picks = sorted(int(i) for i in rng.choice(nf, size=min(2, nf), replace=False))
        self.omegas = [float(sc.omegas[i]) for i in self.picks]
        self.eta = float(np.abs(sc.g).sum())
        L = exact.augmented(self.A, sc.g, self.omegas[0], self.eta)
        l1 = float(abs(L).sum(axis=0).max())
        self.pieces = max(1, int(math.ceil(self.T * l1 / 10.0)))
        self.gens = [None] * len(self.omegas)
        self.calls = 0

    def step(self):
        """Advance the next frequency's run by one piece (restarting a run
        that has reached T); returns the elapsed seconds."""
        q = self.calls % len(self.gens)
        self.calls += 1
        t0 = time.perf_counter()
        if self.gens[q] is None:
            self.gens[q] = self.exact.y_plain_pieces(self.A, self.g, self.omegas[q], self.T, self.pieces, self.eta)
        try:
            next(self.gens[q])
        except StopIteration:
            self.gens[q] = self.exact.y_plain_pieces(self.A, self.g, self.omegas[q], self.T, self.pieces, self.eta)
            next(self.gens[q])
        return time.perf_counter() - t0

    def describe(self, calls, secs):
        return (f"oracle exact response (augmented route, scipy expm_multiply, FP64) on the full "
                f"{self.A.shape[0]}-unknown grid, frequencies {self.picks} of the workload: "
                f"{calls} of the {self.pieces} equal pieces of [0, {self.T:g}] a response takes, "
                f"{secs:.1f} s ({secs / max(calls, 1):.2f} s a piece, {self.pieces * secs / max(calls, 1):.0f} s a "
                f"response); operator assembly {self.setup_s:.1f} s not counted")


def cpu_info():
    """Host cores (nproc) and the threads the oracle's sparse products use
    (scipy's CSR product is single-threaded)."""
    return {"nproc": os.cpu_count(), "threads_used": 1}


def run_reference(args, w):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    sc = scenario_for(w)
    orc = OraclePieces(w, sc)
    for _ in range(args.warmup):
        orc.step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        orc.step()
    el = time.perf_counter() - t0
    v = (args.steps / orc.pieces) / el if el > 0 else 0.0
    info = cpu_info()
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "responses/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * el / max(args.steps, 1), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_of(args, w, sc),
            "step": "one piece of one frequency's oracle response (1/%d of a response)" % orc.pieces,
            "cpu_baseline": {"kind": "oracle", "value": v, "unit": "responses/s", "cores": 1,
                             "sample": orc.describe(args.steps, el), **info},
            "e2e": {"value": v, "unit": "responses/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def timed_steps(args, dist, fn, stream):
    """W untimed steps, then K steps between barriers and synchronisations,
    timed by CUDA events on ``stream``; returns (max device ms over ranks,
    wall s, clocks)."""
    import torch
    for _ in range(args.warmup):
        fn()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks()
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        fn()
    ev1.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    if dist:
        dist.barrier()
    clk = clocks.stop(int(os.environ.get("LOCAL_RANK", "0")))
    return barrier_max(dist, ev0.elapsed_time(ev1)), wall, clk


def run_uneven(args, w):
    """Uneven batch: independent instances of different sizes solved
    concurrently by the native multi-problem driver (one stream per instance)."""
    import torch
    import scenario as S
    from paper_1707_00023_gb300 import Context, response_multi

    rank, world, local, dist = dist_setup(args.gpus)
    t0 = time.perf_counter()
    scs = S.config_uneven(count=w["count"], seed=w["seed"] + rank, T=w["T"], m=w["m"], nfreq=w["nfreq"],
                          step=w.get("step", 1))
    t_gen = time.perf_counter() - t0
    dt = torch.float64 if w["prec"] == "fp64" else torch.float32
    ctxs, gs = [], []
    for sc in scs:
        rst = w["method"] == "rstdim"
        ctxs.append(Context(sc.grid, sc.eps_cell, precision=w["prec"], krylov_dim=w["m"], max_freqs=w["nfreq"],
                            batch=2 if rst else w["nfreq"], stream="own", rst_samples=w.get("rst_samples", 0)))
        gs.append(torch.tensor(sc.g, dtype=dt, device="cuda"))
    torch.cuda.synchronize()
    oms = np.stack([sc.omegas for sc in scs])
    planes = np.array([sc.plane for sc in scs])
    main_stream = torch.cuda.current_stream()
    res = {}
    batch = None
    if w.get("batched"):
        from paper_1707_00023_gb300 import Batch
        batch = Batch(ctxs)
        tune = batch.info()

        def step():
            res["out"] = batch.response(gs, oms, w["T"], rtol=w["rtol"], planes=planes)
    else:
        def step():
            res["out"] = response_multi(ctxs, gs, oms, w["T"], rtol=w["rtol"], method=w["method"], planes=planes,
                                        nthreads=w["threads"])

    def launch_count():
        n = sum(c.stats()["kernel_launches"] for c in ctxs)
        return n + (batch.info()["batched_launches"] if batch is not None else 0)

    launches0 = launch_count()
    dev_ms, wall, clk = timed_steps(args, dist, step, main_stream)
    launches = launch_count() - launches0
    roofline = e2e = cpu = None
    if batch is not None:
        # end to end: every instance's source from pinned host memory, the
        # intensities back to the host (the call returns them there)
        hosts = [torch.tensor(sc.g, dtype=dt).pin_memory() for sc in scs]
        torch.cuda.synchronize()
        e0 = time.perf_counter()
        for _ in range(args.steps):
            gd = [h.to("cuda", non_blocking=True) for h in hosts]
            torch.cuda.synchronize()
            batch.response(gd, oms, w["T"], rtol=w["rtol"], planes=planes)
        e_wall = barrier_max(dist, time.perf_counter() - e0)
        e2e = {"value": len(scs) * w["nfreq"] * args.steps * world / e_wall, "unit": "responses/s",
               "h2d_bytes_per_step": int(sum(h.numel() * h.element_size() for h in hosts)),
               "d2h_bytes_per_step": int(3 * 8 * len(scs) * w["nfreq"])}
        # roofline of the batched sweep (an untimed pass with its launches timed by events)
        i0 = batch.info()
        batch.set_timing(True)
        step()
        batch.set_timing(False)
        i1 = batch.info()
        ms = i1["sweep_ms"] - i0["sweep_ms"]
        nl = i1["sweep_timed_launches"] - i0["sweep_timed_launches"]
        by = i1["sweep_bytes"] - i0["sweep_bytes"]
        peak, peak_kind = peaks()
        if ms > 0 and nl > 0:
            ach = by / (ms / 1000.0) / 1e9
            roofline = {"bound": "hbm", "kernel": "k_sw_pass4s_batch", "achieved": round(ach, 1), "peak": peak,
                        "unit": "GB/s", "frac": round(ach / peak, 4), "traffic": None,
                        "algorithmic_bytes_per_launch": round(by / nl), "peak_source": peak_kind,
                        "launches": nl, "avg_launch_us": round(1000 * ms / nl, 2)}
        if rank == 0 and world == 1 and not args.no_cpu_baseline:
            # the oracle on 3 seeded instances: per-response seconds from its pieces, averaged
            rng = np.random.default_rng(1707 + 4)
            picks = sorted(int(i) for i in rng.choice(len(scs), size=3, replace=False))
            secs, parts = [], []
            for i in picks:
                orc = OraclePieces(w, scs[i])
                el = sum(orc.step() for _ in range(2))
                secs.append(orc.pieces * el / 2)
                parts.append(f"instance {i} ({scs[i].grid.n[0]}^3): {el / 2:.2f} s a piece x {orc.pieces} pieces")
            cpu = {"value": 1.0 / float(np.mean(secs)), "unit": "responses/s", "cores": 1, "kind": "oracle",
                   "sample": "oracle exact response (augmented route, scipy expm_multiply, FP64) of one frequency "
                             "on each of 3 seeded instances, 2 equal pieces of [0, T] each, per-response time = "
                             "pieces x piece time, averaged over the instances: " + "; ".join(parts),
                   **cpu_info()}
    # device events on the current stream do not order the instance streams;
    # the wall clock around the synchronised call is the job time here
    job_s = barrier_max(dist, wall)
    responses = len(scs) * w["nfreq"] * args.steps * world
    sizes = [sc.grid.n[0] for sc in scs]
    if rank == 0:
        line = {"metric": METRIC, "value": responses / job_s, "unit": "responses/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * job_s / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": {"workload": args.workload, "method": w["method"], "instances": len(scs),
                           "sizes_min_max": [min(sizes), max(sizes)],
                           "unknowns_total": int(sum(sc.grid.nunk for sc in scs)), "nfreq_each": w["nfreq"],
                           "T": w["T"], "krylov_dim": w["m"],
                           "driver": "batched launches" if batch is not None else f"{w['threads']} host threads",
                           "timing": "wall clock around the synchronised multi-problem call",
                           "media_generation_s": round(t_gen, 1)},
                "gpu_launches": launches, "clocks": clk, "roofline": roofline, "cpu_baseline": cpu,
                "e2e": e2e}
        if batch is not None:
            line["autotune"] = tune
            # batched Arnoldi processes run as replays of their captured graphs
            # (the event-timed pass above launches directly)
            line["graph_replays"] = batch.info()["graph_replays"]
        print(json.dumps(line), flush=True)
    if batch is not None:
        batch.close()
    for c in ctxs:
        c.close()


def run_adjoint(args, w):
    """Gradient of the summed output-plane intensity w.r.t. per-cell eps."""
    import torch
    from paper_1707_00023_gb300 import Context

    rank, world, local, dist = dist_setup(args.gpus)
    sc = scenario_for(w, rank, world)
    dt = torch.float64 if w["prec"] == "fp64" else torch.float32
    stream = torch.cuda.Stream()
    ctx = Context(sc.grid, sc.eps_cell, precision=w["prec"], krylov_dim=w["m"], max_freqs=w["nfreq"],
                  batch=2, stream=stream, max_checkpoints=w["checkpoints"])
    g = torch.tensor(sc.g, dtype=dt, device="cuda")
    torch.cuda.synchronize()
    res = {}

    def step():
        with torch.cuda.stream(stream):
            res["loss"], res["grad"] = ctx.adjoint_response_grad(g, sc.omegas, w["T"], rtol=w["rtol"],
                                                                 plane=sc.plane)

    launches0 = ctx.stats()["kernel_launches"]
    dev_ms, wall, clk = timed_steps(args, dist, step, stream)
    st = ctx.stats()
    launches = st["kernel_launches"] - launches0
    grads = args.steps * world
    # end to end: the source from pinned host memory in, the gradient out to it
    g_host = torch.tensor(sc.g, dtype=dt).pin_memory()
    grad_host = torch.empty(sc.grid.ncell, dtype=torch.float64).pin_memory()
    e0 = time.perf_counter()
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            gd = g_host.to("cuda", non_blocking=True)
            _, gr = ctx.adjoint_response_grad(gd, sc.omegas, w["T"], rtol=w["rtol"], plane=sc.plane)
            grad_host.copy_(gr.reshape(-1), non_blocking=True)
        stream.synchronize()
    e_wall = barrier_max(dist, time.perf_counter() - e0)
    e2e = {"value": grads / e_wall, "unit": "gradients/s",
           "h2d_bytes_per_step": int(g_host.numel() * g_host.element_size()),
           "d2h_bytes_per_step": int(grad_host.numel() * grad_host.element_size() + 8)}
    # roofline of the dominant kernel class (an untimed pass with event timing)
    ctx.set_timing(True)
    step()
    kt = ctx.kernel_times()
    ctx.set_timing(False)
    total_ms = sum(v["ms"] for v in kt.values())
    dom = max(kt, key=lambda k: kt[k]["ms"])
    peak, peak_kind = peaks()
    ach = kt[dom]["bytes"] / (kt[dom]["ms"] / 1000.0) / 1e9 if kt[dom]["ms"] > 0 and kt[dom]["bytes"] > 0 else None
    roofline = {"bound": "hbm", "kernel": {"pass_a": "k_pass_a", "pass_b": "k_pass_b"}.get(dom, dom),
                "achieved": None if ach is None else round(ach, 1), "peak": peak, "unit": "GB/s",
                "frac": None if ach is None else round(ach / peak, 4), "traffic": None, "peak_source": peak_kind,
                "launches": kt[dom]["launches"],
                "avg_launch_us": round(1000 * kt[dom]["ms"] / max(1, kt[dom]["launches"]), 2),
                "share_of_step": round(kt[dom]["ms"] / total_ms, 4) if total_ms else None}
    if rank == 0:
        line = {"metric": "gradients/s of the summed output-plane intensity (8 frequencies) w.r.t. per-cell eps",
                "value": grads / (dev_ms / 1000.0), "unit": "gradients/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": dev_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": args.workload, "grid": list(sc.grid.n), "nfreq": w["nfreq"], "T": w["T"],
                           "krylov_dim": w["m"]},
                "loss": res["loss"], "grad_norm": float(res["grad"].norm()), "clocks": clk,
                "kernel_ms_per_step": {k: round(v["ms"], 3) for k, v in kt.items()},
                "stats": st, "gpu_launches": launches,
                "cpu_baseline": None,
                "cpu_baseline_note": "the oracle's adjoint and its finite differences are dense-matrix or "
                                     "expm_multiply runs that do not finish at 96^3; the gradient is checked against "
                                     "the oracle on small grids and against central differences of the FP64 GPU "
                                     "forward solve at 96^3 in the tests",
                "e2e": e2e, "roofline": roofline}
        print(json.dumps(line), flush=True)
    ctx.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default=DEFAULT, choices=sorted(WORKLOADS))
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--arnoldi", default="default", choices=["default", "twopass", "sweep"],
                    help="Arnoldi form of the timed contexts (descriptor arnoldi_form)")
    args = ap.parse_args()
    w = WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args, w)
    if w.get("kind") == "uneven":
        return run_uneven(args, w)
    if w.get("kind") == "adjoint":
        return run_adjoint(args, w)

    import torch
    from paper_1707_00023_gb300 import Context

    rank, world, local, dist = dist_setup(args.gpus)
    sc = scenario_for(w, rank, world)
    dt = torch.float64 if w["prec"] == "fp64" else torch.float32
    stream = torch.cuda.Stream()
    ctx = Context(sc.grid, sc.eps_cell, precision=w["prec"], krylov_dim=w["m"],
                  max_freqs=w["nfreq"], batch=w.get("batch", 1), stream=stream,
                  rst_samples=w.get("rst_samples", 0), arnoldi=args.arnoldi)
    g_host = torch.tensor(sc.g, dtype=dt).pin_memory()
    g = g_host.to("cuda")
    torch.cuda.synchronize()
    oms = sc.omegas

    def step(gv, want_plane=True):
        with torch.cuda.stream(stream):
            return ctx.response_at_freqs(gv, oms, w["T"], rtol=w["rtol"], method=w["method"],
                                         plane=sc.plane, want_plane=want_plane)

    for _ in range(args.warmup):
        step(g)
    torch.cuda.synchronize()

    # ---- timed region: K steps, inputs resident in HBM ----------------------
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks()
    clocks.start()
    launches0 = ctx.stats()["kernel_launches"]
    steps0 = ctx.stats()["arnoldi_steps"]
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    t0 = time.perf_counter()
    last = None
    for _ in range(args.steps):
        last = step(g)
    ev1.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    if dist:
        dist.barrier()
    clk = clocks.stop(local)
    dev_ms = ev0.elapsed_time(ev1)
    launches = ctx.stats()["kernel_launches"] - launches0
    krylov_steps = ctx.stats()["arnoldi_steps"] - steps0
    dev_ms = barrier_max(dist, dev_ms)
    ms_per_step = dev_ms / args.steps
    responses = w["nfreq"] * args.steps * world
    value = responses / (dev_ms / 1000.0)

    # ---- end to end through host buffers -------------------------------------
    nE, npl = ctx.plane_size(sc.plane)
    host_E = torch.empty((w["nfreq"], nE, npl), dtype=dt).pin_memory()
    torch.cuda.synchronize()
    e0 = time.perf_counter()
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            gd = g_host.to("cuda", non_blocking=True)
            out = step(gd)
            host_E.copy_(out["E_plane"], non_blocking=True)
        stream.synchronize()
    e_wall = barrier_max(dist, time.perf_counter() - e0)
    e2e = {"value": responses / e_wall, "unit": "responses/s",
           "h2d_bytes_per_step": int(g_host.numel() * g_host.element_size()),
           "d2h_bytes_per_step": int(host_E.numel() * host_E.element_size() + 8 * w["nfreq"])}

    # ---- roofline of the dominant kernel (untimed pass with event timing) ------
    ctx.set_timing(True)
    step(g)
    kt = ctx.kernel_times()
    ctx.set_timing(False)
    total_ms = sum(v["ms"] for v in kt.values())
    dom = max(("pass_a", "pass_b", "sweep"), key=lambda k: kt[k]["ms"])
    peak, peak_kind = peaks()
    ach = kt[dom]["bytes"] / (kt[dom]["ms"] / 1000.0) / 1e9 if kt[dom]["ms"] > 0 else 0.0
    arn = ("pass_a", "pass_b", "sweep", "swapply")      # every kernel of the Arnoldi process
    ab_bytes = sum(kt[k]["bytes"] for k in arn)
    ab_ms = sum(kt[k]["ms"] for k in arn)
    ab_gbs = ab_bytes / (ab_ms / 1000.0) / 1e9 if ab_ms > 0 else 0.0
    kname = {"pass_a": "k_pass_a", "pass_b": "k_pass_b", "sweep": "k_sw_pass"}[dom]
    avg_bytes = kt[dom]["bytes"] / max(1, kt[dom]["launches"])
    ratio = NCU_TRAFFIC_RATIO.get(kname)
    roofline = {"bound": "hbm", "kernel": kname, "achieved": round(ach, 1),
                "peak": peak, "unit": "GB/s", "frac": round(ach / peak, 4),
                "traffic": None if ratio is None else round(ratio * avg_bytes),
                "algorithmic_bytes_per_launch": round(avg_bytes),
                "peak_source": peak_kind,
                "launches": kt[dom]["launches"], "avg_launch_us": round(1000 * kt[dom]["ms"] / max(1, kt[dom]["launches"]), 2),
                "share_of_step": round(kt[dom]["ms"] / total_ms, 4) if total_ms else None}

    # ---- accuracy and the one-frequency-at-a-time comparison (untimed) ------
    # (a) every response of the batch against the same responses from the
    #     FP64 path of the same method, and the first and last also against
    #     the FP64 time-restarted plain method (an independent route; both FP64
    #     paths match the FP64 oracle to 1e-9 or better in the parity tests);
    #     (b) the same frequency solved alone, batch 1.
    acc = {}
    pick = sorted({0, w["nfreq"] - 1})
    with torch.cuda.stream(stream):
        full = ctx.response_at_freqs(g, oms, w["T"], rtol=w["rtol"], method=w["method"], plane=sc.plane,
                                     want_full=True)
    stream.synchronize()
    g64 = torch.tensor(sc.g, dtype=torch.float64, device="cuda")

    def rel_errs(got, ref, idx):
        fe, pe = {}, {}
        for q, f in enumerate(idx):
            a = got["Y"][f].double()
            b = ref["Y"][q]
            fe[int(f)] = float(torch.linalg.norm(a - b) / torch.linalg.norm(b))
            pa = got["E_plane"][f].double()
            pb = ref["E_plane"][q]
            pe[int(f)] = float(torch.linalg.norm(pa - pb) / torch.linalg.norm(pb))
        return fe, pe

    if w["method"] == "rstdim":
        ctx64 = Context(sc.grid, sc.eps_cell, precision="fp64", krylov_dim=w["m"], max_freqs=w["nfreq"],
                        batch=2, stream=stream, rst_samples=w.get("rst_samples", 0) * 4)
        with torch.cuda.stream(stream):
            ref_all = ctx64.response_at_freqs(g64, oms, w["T"], rtol=1e-11, method="rstdim", plane=sc.plane,
                                              want_full=True)
        stream.synchronize()
        fe, pe = rel_errs(full, ref_all, list(range(w["nfreq"])))
        acc["rel_l2_field_vs_fp64_same_method"] = fe
        acc["rel_l2_plane_E_vs_fp64_same_method"] = pe
        del ref_all
        ctx64.close()
    ctx64 = Context(sc.grid, sc.eps_cell, precision="fp64", krylov_dim=w["m"], max_freqs=len(pick),
                    batch=len(pick), stream=stream)
    with torch.cuda.stream(stream):
        ref = ctx64.response_at_freqs(g64, oms[pick], w["T"], rtol=1e-11, method="plain", plane=sc.plane,
                                      want_full=True)
    stream.synchronize()
    fe, pe = rel_errs(full, ref, pick)
    acc["rel_l2_field_vs_fp64"] = fe
    acc["rel_l2_plane_E_vs_fp64"] = pe
    allf = list(fe.values()) + list(acc.get("rel_l2_field_vs_fp64_same_method", {}).values())
    allp = list(pe.values()) + list(acc.get("rel_l2_plane_E_vs_fp64_same_method", {}).values())
    acc["max_rel_l2"] = max(allf)
    acc["max_rel_l2_plane_E"] = max(allp)
    acc["frequencies_checked"] = w["nfreq"] if w["method"] == "rstdim" else len(pick)
    ctx64.close()
    single = None
    if w.get("batch", 1) > 1 or w["method"] == "rstdim":
        ctx1 = Context(sc.grid, sc.eps_cell, precision=w["prec"], krylov_dim=w["m"], max_freqs=1,
                       batch=1, stream=stream, rst_samples=w.get("rst_samples", 0), arnoldi=args.arnoldi)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            ctx1.response_at_freqs(g, oms[:1], w["T"], rtol=w["rtol"], method=w["method"], plane=sc.plane)
            e0.record(stream)
            ctx1.response_at_freqs(g, oms[:1], w["T"], rtol=w["rtol"], method=w["method"], plane=sc.plane)
            e1.record(stream)
        stream.synchronize()
        single = 1000.0 / e0.elapsed_time(e1)
        ctx1.close()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        orc = OraclePieces(w, sc)
        nc = 3
        el = sum(orc.step() for _ in range(nc))
        cpu = {"value": (nc / orc.pieces) / el, "unit": "responses/s", "cores": 1, "kind": "oracle",
               "sample": orc.describe(nc, el), **cpu_info()}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "responses/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32" if w["prec"] == "fp32" else "f64", "data": "synthetic",
                "config": config_of(args, w, sc, world),
                "arnoldi_ran": "single sweep" if kt["sweep"]["launches"] else "two-pass",
                "roofline": roofline,
                "arnoldi_hbm_gbs": round(ab_gbs, 1),
                "krylov_steps_per_s": round(krylov_steps * world / (dev_ms / 1000.0), 1),
                "kernel_ms_per_step": {k: round(v["ms"], 3) for k, v in kt.items()},
                "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clk,
                "accuracy": acc,
                "one_at_a_time": None if single is None else {
                    "responses_per_s": single, "batched_speedup": value / single},
                "wall_s": wall,
                "stats": ctx.stats()}
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
