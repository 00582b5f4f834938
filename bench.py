#!/usr/bin/env python
"""Throughput benchmark of the GB300 Allen-Cahn stepper.

One benchmark step is one whole job of the 3D mean-curvature workload:
device-side sphere initial condition on a 512^3 grid (h = 1/512,
dt = 0.1 h^2, eps = 0.003), 2000 explicit Euler steps in FP32 storage and
arithmetic, then the FP64 energy / phase-volume reduction read back to the
host.  Inputs are resident in HBM; two 512 MiB buffers are far larger than
L2, so no flush is needed between steps.

Prints one JSON line (rank 0).  Multi-GPU runs are independent replicas
(one per rank, weak scaling); the only cross-rank traffic is the barrier and
the max-over-ranks of the timed interval.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gcell-updates/s + HBM roofline %; speedup vs plain FP32 at ≤1e-3 rel-L2"
UNIT = "Gcell-updates/s"
FALLBACK_HBM_GBS = 6800.0


# ------------------------------------------------------------ distributed --
def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        backend = os.environ.get("AC_BENCH_BACKEND", "nccl")
        dist.init_process_group(backend=backend)
    return ws, rank, local


def dist_barrier(ws, device=None):
    if ws > 1:
        import torch.distributed as dist
        if dist.get_backend() == "nccl" and device is not None:
            dist.barrier(device_ids=[device.index])
        else:
            dist.barrier()


def dist_max(ws, value: float, device=None) -> float:
    """Maximum of a float over all ranks (the slowest replica sets the time)."""
    if ws == 1:
        return value
    import torch
    import torch.distributed as dist
    dev = device if (device is not None and dist.get_backend() == "nccl") else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ clocks --
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="ac_clocks_", suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sms, maxes, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 8:
                    continue
                try:
                    sms.append(float(parts[0]))
                    maxes.append(float(parts[1]))
                    power.append(float(parts[2]))
                except ValueError:
                    continue
                for name, val in zip(names, parts[4:8]):
                    if val.lower().startswith("active"):
                        reasons.add(name)
        os.unlink(self.path)
        if not sms:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        loaded = [s for s in sms if s >= 0.5 * max(sms)] or sms
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(maxes),
                "reasons": sorted(reasons), "samples": len(sms),
                "power_w_max": max(power) if power else None}


# ------------------------------------------------------------------ peaks ---
def hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


def recorded_traffic(kernel: str, source: str, grid=None):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel source and on this grid (else None)."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            rec = json.load(f).get(kernel)
        with open(os.path.join(ROOT, "paper_2105_09671_gb300", "csrc", source), "rb") as f:
            sha = hashlib.sha256(f.read()).hexdigest()
    except (OSError, ValueError, AttributeError):
        return None
    if not rec or rec.get("source_sha256") != sha:
        return None
    if grid is not None and rec.get("grid") != list(grid):
        return None
    return rec.get("dram_bytes_per_launch")


# -------------------------------------------------------------- workloads --
def workload(name: str):
    from paper_2105_09671_gb300 import workloads as wl
    if name == "sphere512":
        return wl.SPHERE_512, "f32", "stream3d_k<float>", "stream3d.cuh"
    if name == "separation4096":
        return wl.SEPARATION_4096, "f32", "stream2d_k<float>", "stream2d.cuh"
    raise SystemExit(f"unknown workload {name}")


def init_field(sim, w):
    if w.init == "sphere":
        sim.init_sphere(r0=w.r0)
    else:
        sim.init_random(seed=w.seed, amplitude=0.1)


# ------------------------------------------------------------ CPU oracle ---
def oracle_sample(w, target_s: float, max_steps: int = 2000):
    """Time the FP64 oracle on the same grid for a bounded number of steps
    (sized from a 1-step and a 5-step calibration so that the timed sample
    takes about target_s; the per-call cost of allocating the output field
    is separated from the per-step cost)."""
    import numpy as np
    import oracle
    if w.init == "sphere":
        phi0 = oracle.init_sphere(w.shape, w.h, w.r0, w.eps).astype(np.float32).astype(np.float64)
    else:
        phi0 = oracle.init_random(w.shape, seed=w.seed).astype(np.float32).astype(np.float64)
    phi = oracle.step(phi0, w.h, w.eps, w.dt, 1)  # warm-up: threads, first touch
    t0 = time.perf_counter()
    phi = oracle.step(phi, w.h, w.eps, w.dt, 1)
    t1 = time.perf_counter() - t0
    t0 = time.perf_counter()
    phi = oracle.step(phi, w.h, w.eps, w.dt, 5)
    t5 = time.perf_counter() - t0
    per_step = max((t5 - t1) / 4.0, t5 / 20.0, 1e-9)
    steps = int(max(1, min(max_steps, target_s / per_step)))
    t0 = time.perf_counter()
    oracle.step(phi, w.h, w.eps, w.dt, steps)
    dt_s = time.perf_counter() - t0
    return steps, dt_s, oracle.num_threads()


def run_batch(args, ws, rank, local):
    """The batched workload: 512 uneven 2D grids, 2000 steps each, FP32,
    advanced by one persistent launch (graph-replayed) per job; compared
    with the same instances stepped one by one with ac_step."""
    out = measure_batch(args, ws, local)
    if rank == 0:
        print(json.dumps(out), flush=True)


def measure_batch(args, ws, local):
    import numpy as np
    import torch
    import paper_2105_09671_gb300 as ac
    from paper_2105_09671_gb300 import workloads as wl

    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    stream = torch.cuda.Stream(device)
    inst = wl.batch_instances(512, seed=0)
    specs = [((d["n"], d["n"]), d["h"], d["eps"], d["dt"]) for d in inst]
    cells = sum(d["n"] * d["n"] for d in inst)
    steps = inst[0]["steps"]
    b = ac.Batch(specs, dtype="f32", device=device, stream=stream)
    # initial states generated on the device by a Simulation view of each field
    views = []
    for i, d in enumerate(inst):
        v = ac.Simulation((d["n"], d["n"]), d["h"], d["eps"], d["dt"], dtype="f32", device=device,
                          stream=stream)
        views.append(v)

    def init_all():
        for i, d in enumerate(inst):
            v = views[i]
            if d["init"] == "sphere":
                v.init_sphere(r0=d["r0"])
            else:
                v.init_random(seed=d["seed"], amplitude=0.1)
            with torch.cuda.stream(stream):
                b.phi(i).copy_(v.phi)

    # depth: forced with --k, else autotuned on the batch's own fields
    # (untimed; the fields are restored after every trial)
    init_all()
    if args.k:
        b.set_schedule(abs(args.k))
    else:
        b.autotune(64)
    b.set_graph(True)
    n_vec = [steps] * len(inst)
    for _ in range(args.warmup):
        init_all()
        b.step(n_vec)
    torch.cuda.synchronize(device)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    clocks.start()
    dist_barrier(ws, device)
    torch.cuda.synchronize(device)
    total_ms = 0.0
    l0 = b.launch_count()
    for _ in range(args.steps):
        init_all()  # not timed: the initial states
        e0.record(stream)
        b.step(n_vec)
        e1.record(stream)
        torch.cuda.synchronize(device)
        total_ms += e0.elapsed_time(e1)
    launches = b.launch_count() - l0
    clk = clocks.stop()
    assert b.status() == ac.AC_OK
    total_ms = dist_max(ws, total_ms, device)
    value = cells * steps * args.steps * ws / (total_ms / 1e3) / 1e9
    # the same instances stepped one grid at a time with ac_step (default schedule)
    for v in views:
        v.set_graph(False)
    init_all()
    torch.cuda.synchronize(device)
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    for v in views:
        v.step(steps)
    p1.record(stream)
    torch.cuda.synchronize(device)
    plain_ms = p0.elapsed_time(p1)
    peak, peak_kind = hbm_peak()
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "batch512_2d", "instances": len(inst), "cells": cells,
                   "euler_steps_per_instance": steps, "sizes": "uniform {64,96,...,1024}^2",
                   "eps": "uniform [3h, 6h]", "k": b.schedule(), "tile": b.tile(),
                   "k_choice": "forced" if args.k else "autotuned",
                   "graph": True,
                   "l2": "no flush: 2 x %d MiB of fields exceed L2" % (cells * 4 >> 20)},
        "speedup_vs_plain": plain_ms / (total_ms / args.steps),
        "plain_per_instance_ms": plain_ms,
        "roofline": {"bound": "hbm", "achieved": value * 8.0, "peak": peak, "unit": "GB/s",
                     "frac": value * 8.0 / peak, "traffic": None, "peak_kind": peak_kind,
                     "note": "effective: Gcell/s x 8 B per cell-update at k=1"},
        "gpu_launches": launches, "clocks": clk,
    }
    for v in views:
        v.close()
    b.close()
    return out


def measure_grid(w, dtype, jobs, warmup, local):
    """Whole jobs (device initial state + w.steps graph-replayed steps) of
    one workload grid on its default schedule: Gcell-updates/s and the mean
    stencil launch time."""
    import torch
    import paper_2105_09671_gb300 as ac
    device = torch.device("cuda", local)
    stream = torch.cuda.Stream(device)
    sim = ac.Simulation(w.shape, w.h, w.eps, w.dt, dtype=dtype, device=device, stream=stream)
    try:
        sim.set_graph(True)
        for _ in range(warmup):
            init_field(sim, w)
            sim.step(w.steps)
        stream.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ms, launches = 0.0, 0
        for _ in range(jobs):
            init_field(sim, w)
            c0 = sim.launch_count()
            e0.record(stream)
            sim.step(w.steps)
            e1.record(stream)
            stream.synchronize()
            ms += e0.elapsed_time(e1)
            launches += sim.launch_count() - c0
        v, k = sim.schedule()
        es = {"f64": 8, "f32": 4, "f16s": 2}[dtype]
        peak, _ = hbm_peak()
        launch_s = ms / 1e3 / max(1, launches)
        return {"workload": w.name, "grid": list(w.shape), "dtype": dtype, "euler_steps": w.steps,
                "jobs": jobs, "schedule": {"variant": "stream" if v == 2 else "direct", "k": k,
                                           "tile": sim.tile()},
                "value": w.cells * w.steps * jobs / (ms / 1e3) / 1e9, "unit": UNIT,
                "avg_launch_ms": launch_s * 1e3,
                "hbm_frac_per_launch": 2 * es * w.cells / launch_s / 1e9 / peak}
    finally:
        sim.close()


def _learned_cases(args, net, ndim, n, jumps, guard, s, device):
    """Guarded learned advance vs the plain FP32 stepper on an n^ndim grid
    (eps = 4h) from a circle / sphere and from a random state; errors are
    measured against the plain stepper run in FP64 on the GPU (the FP64
    path the parity tests hold to the FP64 oracle within 1e-12)."""
    import numpy as np
    import torch
    import paper_2105_09671_gb300 as ac
    from paper_2105_09671_gb300 import _lib as L

    shape = (n,) * ndim
    h = 1.0 / n
    eps, dt = 4 * h, 0.1 * h * h
    steps = 16 * jumps
    out = {}
    for init in ("circle", "random"):
        def start(sim):
            if init == "circle":
                sim.init_sphere(r0=0.3)
            else:
                sim.init_random(seed=7)
        # the FP64 reference, from the FP32-rounded initial state (every torch
        # operation on the library's stream s, which orders it with the steps)
        ref32 = ac.Simulation(shape, h, eps, dt, dtype="f32", device=device, stream=s)
        start(ref32)
        ref64 = ac.Simulation(shape, h, eps, dt, dtype="f64", device=device, stream=s)
        with torch.cuda.stream(s):
            ref64.phi.copy_(ref32.phi.double())
        ref64.step(steps)
        with torch.cuda.stream(s):
            ref = ref64.phi.clone()
            ref_norm = float(torch.linalg.vector_norm(ref))
        s.synchronize()
        ref32.close()
        ref64.close()
        loose = L.AcGuard(guard.steps_per_jump, guard.energy_rtol, guard.max_abs, guard.residual_tol,
                          guard.spot_rtol * math.sqrt(jumps), guard.spot_samples, guard.spot_size,
                          guard.spot_seed)
        res = {}
        for mode in ("plain", "learned", "learned_loose", "unguarded"):
            sim = ac.Simulation(shape, h, eps, dt, dtype="f32", device=device, stream=s, pitch_x=n)
            times, rep = [], None
            reps = 1 if mode == "unguarded" else args.warmup + args.steps
            for r in range(reps):
                start(sim)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(s)
                if mode == "learned":
                    _, rep = L.ac_learned_advance(sim.ctx, net, jumps, guard, with_report=True)
                elif mode == "learned_loose":
                    _, rep = L.ac_learned_advance(sim.ctx, net, jumps, loose, with_report=True)
                elif mode == "unguarded":
                    _, rep = L.ac_learned_advance(sim.ctx, net, jumps, L.AcGuard(16, 1e30, 1e30, 0.0),
                                                  with_report=True)
                else:
                    sim.step(steps)
                e1.record(s)
                s.synchronize()
                if mode == "unguarded" or r >= args.warmup:
                    times.append(e0.elapsed_time(e1))
            with torch.cuda.stream(s):
                err = float(torch.linalg.vector_norm(sim.phi.double() - ref)) / ref_norm
            s.synchronize()
            res[mode] = (statistics.median(times), rep, err)
            sim.close()
        lr, ll = res["learned"][1], res["learned_loose"][1]
        out[init] = {
            "plain_ms": res["plain"][0], "learned_ms": res["learned"][0],
            "speedup_vs_plain": res["plain"][0] / res["learned"][0],
            "jumps": jumps, "fallbacks": lr["fallbacks"],
            "rejected": {k[9:]: lr[k] for k in lr if k.startswith("rejected_")},
            "max_spot_rel": lr["max_spot_rel"], "max_residual": lr["max_residual"],
            "rel_l2_vs_fp64": {"learned": res["learned"][2], "plain_fp32": res["plain"][2],
                               "unguarded": res["unguarded"][2], "learned_loose": res["learned_loose"][2]},
            "loose_guard": {"spot_rtol": loose.spot_rtol, "ms": res["learned_loose"][0],
                            "fallbacks": ll["fallbacks"],
                            "rejected": {k[9:]: ll[k] for k in ll if k.startswith("rejected_")}},
            "unguarded_ms": res["unguarded"][0],
        }
    return out


def run_learned(args, ws, rank, local):
    """The learned form: train the 2D jump network on plain-stepper
    trajectories of 256^2 grids (eps = 4h; 2000 trajectories by default),
    calibrate its guard on held-out trajectories, then advance 1024^2
    fields 2000 steps (125 guarded jumps) and compare time-to-solution and
    error with the plain stepper; the same for the 3x3x3 network trained on
    64^3 trajectories and evaluated on 128^3."""
    import numpy as np
    import torch
    from paper_2105_09671_gb300 import _lib as L

    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    s = torch.cuda.Stream(device)
    jumps, target = 125, 1e-3

    def train(ndim, n, pool, iterations, seed):
        net = L.ac_net_create(ndim, s.cuda_stream)
        cfg = L.AcTrainConfig(n=n, eps_cells=4.0, pool=pool, trajectory_jumps=jumps, iterations=iterations,
                              steps_per_jump=16, lr=1e-3, lr_final=1e-5, seed=seed)
        t0 = time.perf_counter()
        hist, used = L.ac_net_train(net, cfg)
        secs = time.perf_counter() - t0
        # guard: the per-jump share of the final target for the spot check,
        # the residual threshold calibrated on held-out trajectories
        guard = L.AcGuard(16, 1e-6, 1.001, 0.0, target / jumps, 0, 0, 99)
        cal = L.AcTrainConfig(n=n, eps_cells=4.0, pool=64 if ndim == 2 else 16, trajectory_jumps=jumps,
                              iterations=1, steps_per_jump=16, lr=1e-3, lr_final=1e-5, seed=seed + 1000)
        calib = L.ac_net_calibrate_guard(net, cal, 2.0, guard)
        info = {"n": n, "pool": pool, "iterations": iterations, "trajectories": used, "seconds": secs,
                "loss_first": float(np.median(hist[:50])), "loss_last": float(np.median(hist[-50:])),
                "calibration": calib}
        return net, guard, info

    # 2D: enough iterations for the requested number of trajectories
    pool2 = 32
    iters2 = args.train_iters or int(math.ceil(max(0, args.train_trajectories - pool2) * jumps / pool2))
    net2, guard2, train2 = train(2, 256, pool2, iters2, 1)
    n2 = 1024
    cases2 = _learned_cases(args, net2, 2, n2, jumps, guard2, s, device)
    # tensor-core roofline of the 2D network forward at 1024^2
    x = torch.rand(1, n2, n2, device=device) * 2 - 1
    y = torch.empty_like(x)
    torch.cuda.synchronize(device)
    for _ in range(3):
        L.ac_net_forward(net2, x.data_ptr(), y.data_ptr(), 1, n2, n2, 1, 0.1)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(10):
        L.ac_net_forward(net2, x.data_ptr(), y.data_ptr(), 1, n2, n2, 1, 0.1)
    e1.record(s)
    s.synchronize()
    fwd_ms = e0.elapsed_time(e1) / 10
    flops = n2 * n2 * (4 * 2 * 288 * 32 + 2 * 2 * 9 * 32)
    peak = 1889.1
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peak = float(json.load(f)["bf16_tflops"])
    except (OSError, KeyError, ValueError):
        pass
    achieved = flops / (fwd_ms / 1e3) / 1e12
    guard_cfg = {k: getattr(guard2, k) for k, _ in guard2._fields_}
    L.ac_net_destroy(net2)

    out3 = None
    if not args.no_3d:
        net3, guard3, train3 = train(3, 64, 8, args.train3d_iters, 2)
        cases3 = _learned_cases(args, net3, 3, 128, jumps, guard3, s, device)
        L.ac_net_destroy(net3)
        out3 = {"train": train3, "grid": [128] * 3, "cases": cases3}

    c = cases2["circle"]
    line = {
        "metric": METRIC, "value": n2 * n2 * 16 * jumps / (c["learned_ms"] / 1e3) / 1e9, "unit": UNIT,
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": c["learned_ms"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "config": {"workload": "learned_jump_1024_2d", "grid": [n2, n2], "euler_steps": 16 * jumps,
                   "steps_per_jump": 16, "train": train2, "guard": guard_cfg,
                   "target_rel_l2": target, "error_reference": "plain stepper in FP64 on the GPU"},
        "cases": cases2,
        "cases_3d": out3,
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": None,
                     "kernel": "network forward (4 tcgen05 convs + 2 CUDA-core end layers)",
                     "forward_ms_1024": fwd_ms},
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_slab(args, ws, rank, local):
    """The 512^3 sphere job through the slab decomposition on one GPU: the
    grid split along z into --parts parts with halo planes, each part
    stepped by its own context, halos refreshed by device copies between
    blocks, the whole sequence replayed as one CUDA graph (and, beside it,
    launched one by one); the same job undivided (graph replay) beside it."""
    import torch
    import paper_2105_09671_gb300 as ac
    from paper_2105_09671_gb300.slab import Slab

    w, dtype, _, _ = workload("sphere512")
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    stream = torch.cuda.Stream(device)
    slab = Slab(w.shape, w.h, w.eps, w.dt, parts=args.parts, dtype=dtype, device=device, stream=stream)
    whole = ac.Simulation(w.shape, w.h, w.eps, w.dt, dtype=dtype, device=device, stream=stream)
    whole.set_graph(True)

    def job_slab():
        slab.full.init_sphere(r0=w.r0)
        slab.scatter()
        slab.step(w.steps)
        slab.gather()

    def job_slab_direct():
        slab.set_graph(False)
        job_slab()
        slab.set_graph(True)

    def job_whole():
        whole.init_sphere(r0=w.r0)
        whole.step(w.steps)

    res = {}
    slab.set_graph(True)
    for name, job in (("slab_direct", job_slab_direct), ("slab", job_slab), ("whole", job_whole)):
        for _ in range(args.warmup):
            job()
        torch.cuda.synchronize(device)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            job()
        e1.record(stream)
        torch.cuda.synchronize(device)
        res[name] = e0.elapsed_time(e1) / args.steps
    k0, c0 = slab.launch_count()
    job_slab()
    kernels, copies = slab.launch_count()
    kernels, copies = kernels - k0, copies - c0
    with torch.cuda.stream(stream):
        equal = bool(torch.equal(slab.full.phi, whole.phi))
    torch.cuda.synchronize(device)
    halo = slab.halo
    slab.close()
    whole.close()
    value = w.cells * w.steps / (res["slab"] / 1e3) / 1e9
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": res["slab"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": dtype, "data": "synthetic",
            "config": {"workload": "sphere3d_512_slabs", "parts": args.parts, "halo": halo,
                       "split": "z", "exchange": "device-to-device plane copies on the stream",
                       "graph": True},
            "undivided_ms": res["whole"], "overhead": res["slab"] / res["whole"] - 1.0,
            "slab_launched_one_by_one_ms": res["slab_direct"],
            "bitwise_equal_to_undivided": equal, "kernels_and_copies_per_job": [kernels, copies],
        }), flush=True)


def run_reference(args, ws, rank):
    """The oracle arm: the FP64 C oracle on the host cores, same workload."""
    if rank != 0:
        return
    import oracle
    w, dtype, _, _ = workload(args.workload)
    import numpy as np
    phi0 = (oracle.init_sphere(w.shape, w.h, w.r0, w.eps) if w.init == "sphere"
            else oracle.init_random(w.shape, seed=w.seed)).astype(np.float32).astype(np.float64)
    steps_per = args.ref_steps
    if steps_per <= 0:
        # each call pays a fixed set-up (allocating and filling the two
        # ghost-extended FP64 fields) before its steps: size the steps per
        # benchmark step from a 1-step and a 5-step timing so that a call
        # takes about --ref-seconds and the set-up is a small share of it
        t0 = time.perf_counter()
        oracle.step(phi0, w.h, w.eps, w.dt, 1)
        t1 = time.perf_counter() - t0
        t0 = time.perf_counter()
        oracle.step(phi0, w.h, w.eps, w.dt, 5)
        t5 = time.perf_counter() - t0
        per_step = max((t5 - t1) / 4.0, t5 / 20.0, 1e-9)
        steps_per = int(max(1, min(w.steps, args.ref_seconds / per_step)))
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.step(phi0, w.h, w.eps, w.dt, steps_per)
        dt_s = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt_s)
    total = sum(times)
    value = w.cells * steps_per * len(times) / total / 1e9
    cores = oracle.num_threads()
    sample = (f"{w.name}: {w.cells} cells x {steps_per} Euler step(s) per benchmark step "
              f"(the full job is {w.steps} steps), FP64 oracle, OpenMP")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": w.name, "grid": list(w.shape)},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# ------------------------------------------------------------------ ours ---
def run_ours(args, ws, rank, local):
    import numpy as np
    import torch
    import paper_2105_09671_gb300 as ac

    w, dtype, kname, ksrc = workload(args.workload)
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    stream = torch.cuda.Stream(device)
    sim = ac.Simulation(w.shape, w.h, w.eps, w.dt, dtype=dtype, device=device, stream=stream)
    if args.k:
        sim.set_schedule(ac.AC_VARIANT_STREAM if args.k > 0 else ac.AC_VARIANT_DIRECT, abs(args.k))
    # the 1000 launches of a job are replayed as one CUDA graph (captured in
    # the first warm-up job)
    sim.set_graph(True)
    variant, k = sim.schedule()
    tile = sim.tile()
    kid = f"{kname} k={k} tile={tile}"
    es = {"f64": 8, "f32": 4, "f16s": 2}[dtype]
    field_bytes = w.cells * es

    def job():
        init_field(sim, w)
        sim.step(w.steps)
        return sim.observe()

    for _ in range(args.warmup):
        job()
    torch.cuda.synchronize(device)

    n_ev = args.steps
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(n_ev)]
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    clocks.start()
    dist_barrier(ws, device)
    torch.cuda.synchronize(device)
    l0 = sim.launch_count()
    start.record(stream)
    stencil_launches = 0
    for i in range(n_ev):
        ev[i][0].record(stream)
        init_field(sim, w)
        ev[i][1].record(stream)
        c0 = sim.launch_count()
        sim.step(w.steps)
        stencil_launches += sim.launch_count() - c0
        ev[i][2].record(stream)
        obs = sim.observe()
    end.record(stream)
    torch.cuda.synchronize(device)
    dist_barrier(ws, device)
    launches = sim.launch_count() - l0
    clk = clocks.stop()
    elapsed_ms = start.elapsed_time(end)
    elapsed_ms = dist_max(ws, elapsed_ms, device)
    stencil_ms = sum(ev[i][1].elapsed_time(ev[i][2]) for i in range(n_ev))
    updates = w.cells * w.steps * args.steps * ws
    value = updates / (elapsed_ms / 1e3) / 1e9

    # roofline of the dominant kernel: algorithmic bytes per launch (read phi
    # once and write it once, whatever k) over its live average duration
    avg_launch_s = stencil_ms / 1e3 / max(1, stencil_launches)
    alg_bytes = 2 * field_bytes
    peak, peak_kind = hbm_peak()
    achieved = alg_bytes / avg_launch_s / 1e9
    traffic = recorded_traffic(kid, ksrc, w.shape) if variant == ac.AC_VARIANT_STREAM else None

    # end to end through the public API with host buffers: every job copies
    # its initial state from pinned host memory (H2D), runs the steps and
    # copies the final field back (D2H), all inside the timed region.
    # (1) one job at a time on one stream: copy in, step, copy out.
    host_in = torch.empty(w.shape, dtype=sim.phi.dtype, pin_memory=True)
    host_out = [torch.empty(w.shape, dtype=sim.phi.dtype, pin_memory=True) for _ in range(2)]
    init_field(sim, w)
    with torch.cuda.stream(stream):
        host_in.copy_(sim.phi, non_blocking=True)
    stream.synchronize()
    e2e_steps = max(1, min(args.steps, 3))
    dist_barrier(ws, device)
    torch.cuda.synchronize(device)
    s_s, s_e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ph = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(e2e_steps)]
    s_s.record(stream)
    for i in range(e2e_steps):
        with torch.cuda.stream(stream):
            sim.phi.copy_(host_in, non_blocking=True)
        ph[i][0].record(stream)
        sim.step(w.steps)
        ph[i][1].record(stream)
        with torch.cuda.stream(stream):
            host_out[0].copy_(sim.phi, non_blocking=True)
    s_e.record(stream)
    torch.cuda.synchronize(device)
    single_ms = dist_max(ws, s_s.elapsed_time(s_e), device)
    steps_ms = sum(ph[i][0].elapsed_time(ph[i][1]) for i in range(e2e_steps))
    single_value = w.cells * w.steps * e2e_steps * ws / (single_ms / 1e3) / 1e9
    if not torch.isfinite(host_out[0]).all():
        raise RuntimeError("end-to-end job produced a non-finite field")
    # (2) pipelined: two simulations alternate so that job i+1's H2D and job
    # i's D2H overlap the stepping of the other job (separate copy streams,
    # ordered by events); the two jobs' stepping may overlap on the GPU too.
    sim2 = ac.Simulation(w.shape, w.h, w.eps, w.dt, dtype=dtype, device=device,
                         stream=torch.cuda.Stream(device))
    if args.k:
        sim2.set_schedule(ac.AC_VARIANT_STREAM if args.k > 0 else ac.AC_VARIANT_DIRECT, abs(args.k))
    sim2.set_graph(True)
    sim2.step(w.steps)  # captures its graph outside the timed region
    sim2.stream.synchronize()
    sims = (sim, sim2)
    copy_in, copy_out = torch.cuda.Stream(device), torch.cuda.Stream(device)
    dist_barrier(ws, device)
    torch.cuda.synchronize(device)
    e_s, e_e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e_s.record(copy_in)
    freed = [None, None]
    for i in range(e2e_steps):
        cur = sims[i % 2]
        if freed[i % 2] is not None:
            copy_in.wait_event(freed[i % 2])  # this simulation's previous D2H is done
        with torch.cuda.stream(copy_in):
            cur.phi.copy_(host_in, non_blocking=True)
        loaded = torch.cuda.Event()
        loaded.record(copy_in)
        cur.stream.wait_event(loaded)
        cur.step(w.steps)
        stepped = torch.cuda.Event()
        stepped.record(cur.stream)
        copy_out.wait_event(stepped)
        with torch.cuda.stream(copy_out):
            host_out[i % 2].copy_(cur.phi, non_blocking=True)
        freed[i % 2] = torch.cuda.Event()
        freed[i % 2].record(copy_out)
    e_e.record(copy_out)
    torch.cuda.synchronize(device)
    e2e_ms = dist_max(ws, e_s.elapsed_time(e_e), device)
    e2e_value = w.cells * w.steps * e2e_steps * ws / (e2e_ms / 1e3) / 1e9
    # the last job's result, read back on the host, must be a finite field
    if not torch.isfinite(host_out[(e2e_steps - 1) % 2]).all():
        raise RuntimeError("end-to-end job produced a non-finite field")
    sim2.close()

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": dtype,
        "data": "synthetic",
        "config": {"workload": w.name, "grid": list(w.shape), "euler_steps_per_job": w.steps,
                   "eps": w.eps, "h": w.h, "dt": w.dt, "init": w.init,
                   "schedule": {"variant": "stream" if variant == 2 else "direct", "k": k, "graph": True,
                                "tile": tile},
                   "parallelism": f"replicas x{ws}",
                   "l2": "no flush: two field buffers of %d MiB each exceed L2" % (field_bytes >> 20)},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": kid, "peak_kind": peak_kind,
                     "alg_bytes_per_launch": alg_bytes, "avg_launch_ms": avg_launch_s * 1e3,
                     "effective_frac_k1": value / ws * 2 * es / peak},
        "e2e": {"value": single_value, "unit": UNIT, "h2d_bytes_per_step": field_bytes,
                "d2h_bytes_per_step": field_bytes, "jobs": e2e_steps,
                "ms_per_job": single_ms / e2e_steps, "steps_ms_per_job": steps_ms / e2e_steps,
                "how": "one job at a time on one stream: H2D of the initial field from pinned "
                       "memory, the Euler steps, D2H of the final field"},
        "e2e_pipelined": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": field_bytes,
                          "d2h_bytes_per_step": field_bytes, "jobs": e2e_steps,
                          "how": "two simulations alternate; copies on copy streams overlap the "
                                 "other job's stepping"},
        "gpu_launches": launches,
        "clocks": clk,
        "result": {"energy": obs[0], "phase_volume": obs[1], "nonfinite": obs[2],
                   "radius": ((3 * obs[1]) / (4 * math.pi)) ** (1 / 3) if w.ndim == 3 else math.sqrt(obs[1] / math.pi)},
    }
    if ws == 1 and not args.no_secondary:
        # the other workloads, timed here as well so that their figures come
        # from the same run (each guarded: a failure is reported, not raised)
        from paper_2105_09671_gb300 import workloads as wl
        sec = {}
        for name, fn in (("separation4096_f32", lambda: measure_grid(wl.SEPARATION_4096, "f32", 3, 3, local)),
                         ("sphere512_f16s", lambda: measure_grid(w, "f16s", 3, 3, local) if w.name == "sphere3d_512"
                          else None),
                         ("batch512", lambda: measure_batch(argparse.Namespace(steps=2, warmup=3, k=0), 1, local))):
            try:
                r = fn()
                if r is not None:
                    sec[name] = {k2: r[k2] for k2 in r if k2 not in ("metric", "clocks", "roofline")} \
                        if name == "batch512" else r
            except Exception as e:  # noqa: BLE001 - reported in the JSON line
                sec[name] = {"error": f"{type(e).__name__}: {e}"}
        out["secondary"] = sec
    if ws == 1 and rank == 0 and not args.no_cpu_baseline:
        steps, secs, cores = oracle_sample(w, args.cpu_seconds)
        out["cpu_baseline"] = {
            "value": w.cells * steps / secs / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{w.name}: all {w.cells} cells, {steps} Euler steps of the FP64 oracle "
                      f"(the job runs {w.steps}); {secs:.1f} s"}
        import oracle
        oracle.set_num_threads(1)
        try:
            steps1, secs1, _ = oracle_sample(w, args.cpu_seconds / 4)
        finally:
            oracle.set_num_threads(0)
        out["cpu_baseline"]["single_core"] = {
            "value": w.cells * steps1 / secs1 / 1e9, "unit": UNIT,
            "sample": f"{steps1} Euler steps on one thread; {secs1:.1f} s"}
    sim.close()
    if rank == 0:
        print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="sphere512",
                    choices=["sphere512", "separation4096", "batch512", "learned1024", "slab512"])
    ap.add_argument("--parts", type=int, default=2, help="slab512: parts along z")
    ap.add_argument("--train-iters", type=int, default=0,
                    help="learned workload: Adam steps of the 2D network (0: from --train-trajectories)")
    ap.add_argument("--train-trajectories", type=int, default=2000)
    ap.add_argument("--train3d-iters", type=int, default=1500)
    ap.add_argument("--no-3d", action="store_true", help="learned workload: skip the 3D network")
    ap.add_argument("--k", type=int, default=0,
                    help="force the temporal-block depth (negative: direct kernel, k=1)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-secondary", action="store_true",
                    help="skip the batched / 4096^2 / FP16-storage figures of the default run")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-steps", type=int, default=0,
                    help="oracle steps per benchmark step of --impl reference (0: sized to --ref-seconds)")
    ap.add_argument("--ref-seconds", type=float, default=3.0)
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        # host-only arm: rank 0 runs the oracle, other ranks leave at once
        run_reference(args, int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")))
        return
    ws, rank, local = dist_setup()
    if args.workload == "batch512":
        run_batch(args, ws, rank, local)
    elif args.workload == "learned1024":
        run_learned(args, ws, rank, local)
    elif args.workload == "slab512":
        run_slab(args, ws, rank, local)
    else:
        run_ours(args, ws, rank, local)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
