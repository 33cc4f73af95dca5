#!/usr/bin/env python3
"""Throughput of the immersed-boundary fractional step on GB300.

Metric: cell-steps/s (nx*ny*steps / device time), counted over steps whose
divergence in fluid cells stays below the workload's tolerance.  A bench
step is one full fractional step of the plunging-ellipse workload
(classification, predictor, velocity solves, mass source, pressure solve,
projection, forces) on the 2048x1024 stretched grid (Re 1000, h 0.25, k 2,
dt 1e-3, divergence 1e-8).  Synthetic: the flow starts as the uniform free
stream.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--warmstart learned|plain] [--workload plunge_2048x1024|batch64]

The value is the learned warm start with the mixed path (the U-Net's
prediction added to the previous increment, then FP32 sweeps inside FP64
defect correction to the same tolerance); the mixed path with the plain warm
start and the plain FP64 path are timed on the same steps and reported
beside it.  The U-Net weights come from train_warmstart (trained on
snapshots of seeded runs on the same grid).

--workload batch64 times the batch of 64 cases with uneven grids (512x256 ..
1536x768) advancing together (--cases N: the first N of them).

--impl reference times the FP64 CPU oracle (the slow, plain restatement of
the method) on the host cores with the same metric; under torchrun only rank
0 runs it.  N > 1 runs independent replicas, one per GPU.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FP64_FLOPS_PER_CLK_SM = 4.0   # 2 FP64 FMA per clock per SM on GB300 (sm_103)
FP32_FLOPS_PER_CLK_SM = 256.0  # 128 FP32 FMA per clock per SM
SOR32_BYTES_PER_CELL_LAUNCH = 12  # read e, r; write e (FP32) once per launch
SOR_FLOPS_PER_UPDATE = 12     # 4 products + 3 adds, minus b, times 1/d, relaxation (2)
SOR_BYTES_PER_CELL_HALF = 16  # read phi (8, all cells), read b (4), write phi (4) per half-sweep
# multigrid variant, one FCG iteration per fine cell: smoothing 2 x 12, restriction 9, prolongation 9,
# FCG dot 8 + direction 12 + operator 12 + update 16, coarser levels a third of smoothing + transfers (14)
MG_BYTES_PER_CELL_ITER = 104
# DRAM bytes (read + write) per launch of the FP32 sweep kernel from one ncu capture of the
# unchanged kernel (profiles/k_sor32_rb_*.md), by workload and tile shape (rows, half-sweeps,
# thread rows, form); cold-cache captures
SOR32_TRAFFIC = {
    ("plunge_2048x1024", (80, 16, 16, 7)): 25.221e6,
    ("plunge_4096x2048", (32, 8, 8, 7)): 117.465e6,
    ("plunge_4096x2048", (64, 16, 16, 7)): 115.556e6,
    ("plunge_4096x2048", (80, 16, 16, 7)): 114.906e6,
    ("plunge_2048x1024", (80, 16, 16, 8)): 25.230592e6,
    ("plunge_4096x2048", (80, 16, 16, 8)): 115.323392e6,
    ("plunge_2048x1024", (80, 16, 16, 10)): 25.23136e6,
    ("plunge_4096x2048", (80, 16, 16, 10)): 118.77504e6,
    ("plunge_2048x1024", (80, 16, 16, 9)): 25.23264e6,
    ("plunge_4096x2048", (80, 16, 16, 9)): 115.576576e6,
}
# warp instructions issued per launch of the FP32 sweep kernel (ncu smsp__inst_executed.sum of one
# launch, profiles/k_sor32_rb_*.md), by workload and tile shape: the issue roofline of a kernel that is
# bound by latency and issue, not by DRAM (its working set fits in L2 on 2048x1024)
SOR32_INST = {
    ("plunge_2048x1024", (80, 16, 16, 7)): 15.768846e6,
    ("plunge_4096x2048", (80, 16, 16, 7)): 61.646262e6,
    ("plunge_2048x1024", (80, 16, 16, 8)): 15.773422e6,
    ("plunge_4096x2048", (80, 16, 16, 8)): 61.66415e6,
    ("plunge_2048x1024", (80, 16, 16, 10)): 13.381214e6,
    ("plunge_4096x2048", (80, 16, 16, 10)): 52.308382e6,
    ("plunge_2048x1024", (80, 16, 16, 9)): 13.40867e6,
    ("plunge_4096x2048", (80, 16, 16, 9)): 52.41571e6,
}
WORKLOADS = ("plunge_2048x1024", "plunge_4096x2048", "unet_1024x512", "batch64")
METRIC = "cell-steps/s at div<1e-8: learned warm-start+mixed vs plain FP64, one GB300"


def env_int(k, d):
    try:
        return int(os.environ.get(k, d))
    except ValueError:
        return d


def reduce_over_ranks(x, dist, op, device):
    """x reduced over the ranks of the process group (sum or max; x itself
    with no group).  device: where the reduction tensor lives (cuda for NCCL,
    cpu for gloo)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def replica_throughput(cells_ok, ms, dist=None, device="cuda"):
    """Whole-job throughput of independent replicas (one per rank, weak
    scaling): the cells of every rank's counted steps over the slowest
    rank's time.  Returns (cell-steps/s, total cells, max ms)."""
    cells = reduce_over_ranks(cells_ok, dist, "sum", device)
    t_max = reduce_over_ranks(ms, dist, "max", device)
    return cells / (t_max / 1e3), cells, t_max


def unet_forward_flops(widths, H, W):
    """Algorithmic FLOPs of one U-Net forward pass on an H x W input: 2 * 9 *
    Cin * Cout per output pixel of each 3x3 convolution, with the real input
    (4 features) and output (1) channel counts; encoder convolutions at level
    l (H/2^l x W/2^l), decoder convolutions over the concatenation of the
    upsampled deeper level and the skip, and the output head."""
    w = widths
    px = [(H >> l) * (W >> l) for l in range(4)]
    convs = []
    for l in range(4):
        convs.append((4 if l == 0 else w[l - 1], w[l], px[l]))
        convs.append((w[l], w[l], px[l]))
    for l in (2, 1, 0):
        up = w[3] if l == 2 else w[l + 1]
        convs.append((up + w[l], w[l], px[l]))
        convs.append((w[l], w[l], px[l]))
    convs.append((w[0], 1, px[0]))
    return sum(2 * 9 * ci * co * n for ci, co, n in convs)


def network_roofline(learned, cfg, stream, peaks, peak_src, reps=10, warm=3):
    """The learned warm start's U-Net forward on the coarse grid, timed alone
    with CUDA events on the solver stream, against the measured BF16 tensor
    peak (burst figure: the forward is timed in isolation)."""
    import torch
    H, W = cfg.ny // 2, cfg.nx // 2
    net = learned["net"]
    gen = torch.Generator(device="cpu").manual_seed(5)
    feat = torch.rand((H, W, 4), generator=gen, dtype=torch.float32).to(f"cuda:{torch.cuda.current_device()}")
    out = torch.zeros((H, W), dtype=torch.float32, device=feat.device)
    torch.cuda.synchronize()
    for _ in range(warm):
        net.forward(feat.data_ptr(), H, W, out.data_ptr(), stream.cuda_stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        net.forward(feat.data_ptr(), H, W, out.data_ptr(), stream.cuda_stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    flops = unet_forward_flops(learned["meta"].get("widths", net.widths), H, W)
    achieved = flops / (ms * 1e-3) / 1e12
    peak = peaks.get("bf16_tflops", 1900.0)
    return {"kernel": "U-Net forward (k_conv3x3_tc: BF16 tcgen05.mma, TMEM accumulators, TMA-staged operands; "
                      "pooling, upsampling)", "widths": list(net.widths),
            "input": [H, W], "gflop": flops / 1e9, "ms": ms, "achieved_tflops": achieved,
            "peak_tflops": peak, "frac": achieved / peak,
            "peak_note": f"BF16 dense tensor peak ({peak_src}, burst); the whole forward pass, whose layers have "
                         f"16-128 channels"}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            return json.load(fh), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"bench_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    smax = max(smax, float(f[2]))
                except ValueError:
                    continue
                for n, v in zip(names, f[5:9]):
                    if v.lower() == "active":
                        reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def solver_kwargs(cfg, precision):
    return dict(x0=cfg.x0, x1=cfg.x1, y0=cfg.y0, y1=cfg.y1, nx=cfg.nx, ny=cfg.ny, hmin=cfg.hmin,
                ubox=cfg.ubox, bc=cfg.bc, u_in=cfg.u_in, Re=cfg.Re, dt=cfg.dt, ptol=cfg.ptol,
                htol=cfg.htol, check_p=cfg.check_p, check_h=cfg.check_h, omega_p=cfg.omega(),
                omega_h=cfg.omega_h, precision=precision)


def oracle_sim(cfg, threads):
    """An oracle context for the workload, its pressure relaxation factor
    set by the oracle's own probe of the grid (untimed)."""
    import oracle
    kw = solver_kwargs(cfg, 0)
    kw.pop("precision")
    kw["omega_p"] = oracle.tune_omega(oracle.Sim(**kw, threads=threads))
    return oracle.Sim(**kw, threads=threads), kw["omega_p"]


def host_info():
    """The host's core count and CPU description (nproc, lscpu), for the
    CPU-baseline record."""
    info = {"nproc": os.cpu_count()}
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            k, _, v = line.partition(":")
            if k.strip() in ("Architecture", "Model name", "CPU(s)", "Thread(s) per core", "Core(s) per socket",
                             "Socket(s)", "NUMA node(s)"):
                info[k.strip()] = v.strip()
    except (OSError, subprocess.SubprocessError):
        info["lscpu"] = "unavailable"
    return info


def oracle_sweep_seconds(o, cfg, threads, sweeps=128):
    """Seconds per pressure SOR sweep of the oracle on this grid at the given
    thread count (a fixed number of sweeps on a seeded compatible right-hand
    side, no stopping test)."""
    import numpy as np
    from paper_2402_17337_gb300 import workloads as W
    o._L.or_set_threads(o._h, threads)
    b = W.random_field(o.shape("p"), seed=3)
    b -= b.mean()
    t0 = time.perf_counter()
    o.poisson(b, tol=0.0, check=sweeps, maxs=sweeps)
    return (time.perf_counter() - t0) / sweeps


def cpu_oracle_sample(cfg, state=None, max_seconds=60.0):
    """Times the FP64 oracle on one full step of the workload on all host
    cores, optionally started from a given (u, v, p, phi) state, and
    estimates the same step on one core: the oracle threads only its
    pressure solve, so the one-thread step is the all-core step with its
    sweeps re-timed at the one-thread rate measured on 128 sweeps of the same
    grid."""
    threads = os.cpu_count() or 1
    o, w = oracle_sim(cfg, threads)
    o.set_body(cfg.chord, cfg.tc, cfg.h, cfg.k, cfg.xc, cfg.yc)
    if state is not None:
        for name, arr in state.items():
            o.set(name, arr)
    t0 = time.perf_counter()
    rc, st = o.step(1)
    t = time.perf_counter() - t0
    sw_all = oracle_sweep_seconds(o, cfg, threads)
    sw_one = oracle_sweep_seconds(o, cfg, 1)
    t_one = t + st["sweeps_p"] * (sw_one - sw_all)
    return {"seconds": t, "rc": rc, "sweeps_p": st["sweeps_p"], "threads": threads,
            "div_max": st["div_max"], "omega": w, "seconds_1thread": t_one,
            "sweep_ms_all": 1e3 * sw_all, "sweep_ms_1thread": 1e3 * sw_one, "host": host_info()}


def workload_config(cfg, world):
    """The `config` object of a single-grid workload: the same in both arms."""
    return {"workload": cfg.name, "nx": cfg.nx, "ny": cfg.ny, "global_batch": world,
            "parallelism": f"replicas x{world}",
            "l2": f"state 14 FP64 fields x {cfg.cells * 8 / 1e6:.0f} MB > L2 (129 MB); FP32 sweep "
                  f"arrays {cfg.cells * 16 / 1e6:.0f} MB; no flush"}


def batch_config(cfgs, world):
    """The `config` object of the batch workload: the same in both arms."""
    cells = sum(c.cells for c in cfgs)
    return {"workload": "batch64" if len(cfgs) == 64 else f"batch64[:{len(cfgs)}]", "cases": len(cfgs),
            "cells_per_step": cells, "grids": sorted({f"{c.nx}x{c.ny}" for c in cfgs}),
            "global_batch": len(cfgs) * world, "parallelism": f"replicas x{world}",
            "l2": f"{cells * 16 / 1e6:.0f} MB of FP32 sweep arrays per launch set; no flush"}


def run_reference(args, cfg, config):
    """--impl reference: the oracle on the host cores, same metric; config:
    the timed arm's `config` object (for the batch, one of its cases is the
    bounded sample)."""
    rank = env_int("RANK", 0)
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    threads = os.cpu_count() or 1
    o, w = oracle_sim(cfg, threads)
    o.set_body(cfg.chord, cfg.tc, cfg.h, cfg.k, cfg.xc, cfg.yc)
    o.set("u", cfg.initial_u(o.shape("u")))
    for _ in range(args.warmup):
        rc, _ = o.step(1)
        if rc:
            raise SystemExit(f"oracle failed during warm-up ({rc})")
    times, ok, sweeps = [], 0, []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        rc, st = o.step(1)
        times.append(time.perf_counter() - t0)
        if rc:
            raise SystemExit(f"oracle failed ({rc})")
        ok += st["div_max"] < cfg.div_tol
        sweeps.append(st["sweeps_p"])
    T = sum(times)
    value = cfg.cells * ok / T
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "cell-steps/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * T / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config,
        "details": {"path": "cpu-oracle", "sample_workload": cfg.name,
                    "poisson_sweeps_per_step": statistics.mean(sweeps), "omega_p": w},
        "cpu_baseline": {"value": value, "unit": "cell-steps/s", "cores": threads, "kind": "oracle",
                         "sample": f"{args.warmup} untimed + {args.steps} timed full steps of {cfg.name} "
                                   f"from the uniform free stream, FP64 oracle, {threads} OpenMP threads in the "
                                   f"pressure solve (all host cores)",
                         "host": host_info()},
        "e2e": {"value": value, "unit": "cell-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_batch(args):
    """--workload batch64: the first --cases cases of the 64-case batch
    advancing together; value = sum over cases and timed steps of the cells
    of steps that met the divergence tolerance, over the device time."""
    import numpy as np
    import torch

    import paper_2402_17337_gb300 as ibm
    from paper_2402_17337_gb300 import build as B
    from paper_2402_17337_gb300 import workloads as W

    rank, world, local = env_int("RANK", 0), env_int("WORLD_SIZE", 1), env_int("LOCAL_RANK", 0)
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        B.build()
    if dist:
        dist.barrier()
    B.build()
    cfgs = W.batch64()[:args.cases]
    cells = [c.cells for c in cfgs]

    def barrier():
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()


    omegas = []
    for c in cfgs:  # each case's relaxation factor from the device probe (untimed)
        s = ibm.Solver.from_config(c, precision=1)
        omegas.append(s.tune_omega())
        s.close()
    cfgs = [dataclasses.replace(c, omega_p=w) for c, w in zip(cfgs, omegas)]

    def make():
        ss = []
        for c in cfgs:
            s = ibm.Solver.from_config(c, precision=1)
            s.set("u", c.initial_u(s.shape("u")))
            ss.append(s)
        b = ibm.Batch(ss)
        if args.sor_shape >= 0:
            b.set_sor_shape(args.sor_shape)
        b.set_graphs(args.batch_launch == "graphs")
        return ss, b

    ss, batch = make()
    for _ in range(args.warmup):
        batch.step(1)
    state0 = {n: ss[0].get(n) for n in ("u", "v", "p", "phi")} if rank == 0 else None
    batch.set_profiling(True)
    bstream = torch.cuda.ExternalStream(batch.stream)
    clocks = ClockSampler(local)
    barrier()
    if not args.no_clocks:
        clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.profiler.start()  # marks the timed region for a profiler (no-op otherwise)
    e0.record(bstream)
    stats = [batch.step(1) for _ in range(args.steps)]
    e1.record(bstream)
    barrier()
    torch.cuda.profiler.stop()
    clk = clocks.stop() if not args.no_clocks else None
    prof = batch.profile()
    ok_local = sum(n for st in stats for n, c, x in zip(cells, cfgs, st) if x["div_max"] < c.div_tol)
    value, ok_cells, ms = replica_throughput(ok_local, e0.elapsed_time(e1), dist, "cuda")
    batch.close()
    for s in ss:
        s.close()

    peaks, peak_src = load_peaks()
    roof = None
    if prof["sweep_ms"] > 0:
        nbytes = SOR32_BYTES_PER_CELL_LAUNCH * prof["sweep_cells"]
        achieved = nbytes / (prof["sweep_ms"] / 1e3) / 1e9
        rows, half, _ = prof["sor_shape"]
        roof = {"bound": "hbm", "kernel": f"k_sor32_rb_batch (FP32 red-black SOR over the tiles of every active "
                                          f"case, tile {rows} rows x 128 cells, {half} half-sweeps per launch)",
                "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"],
                "traffic": None, "launch_us": 1e3 * prof["sweep_ms"] / prof["sweep_launches"],
                "shape": list(prof["sor_shape"]) + [prof["sor_form"]], "shape_index": prof["sor_index"],
                "peak_note": f"HBM {peaks['hbm_gbs']} GB/s ({peak_src}); algorithmic bytes {SOR32_BYTES_PER_CELL_LAUNCH}"
                             f" B per covered cell per launch, summed over the timed sweep launches (cases leave "
                             f"the launches as they converge)"}

    e2e = None
    if not args.no_e2e:
        ss2, batch2 = make()
        for _ in range(args.warmup):
            batch2.step(1)
        names = ("u", "v", "p", "phi")
        pinned = [{n: torch.empty(s.shape(n), dtype=torch.float64, pin_memory=True).numpy() for n in names}
                  for s in ss2]
        for s, pn in zip(ss2, pinned):
            for n in names:
                pn[n][...] = s.get(n)
        h2d = sum(a.nbytes for pn in pinned for a in pn.values())
        barrier()
        t0 = time.perf_counter()
        ok2 = 0
        for _ in range(args.steps):
            for s, pn in zip(ss2, pinned):
                for n in names:
                    s.set(n, pn[n])
            st = batch2.step(1)
            for s, pn in zip(ss2, pinned):
                for n in names:
                    s.get(n, out=pn[n])
            ok2 += sum(n for n, c, x in zip(cells, cfgs, st) if x["div_max"] < c.div_tol)
        barrier()
        e2e_value, _, _ = replica_throughput(ok2, 1e3 * (time.perf_counter() - t0), dist, "cuda")
        batch2.close()
        for s in ss2:
            s.close()
        e2e = {"value": e2e_value, "unit": "cell-steps/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": h2d,
               "note": "a second batch over the same steps; per step every case's u, v, p, phi copied in from "
                       "pinned host memory, batch step, copied back; host wall clock"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        r = cpu_oracle_sample(cfgs[0], state0)
        cpu = {"value": cfgs[0].cells / r["seconds"] if r["rc"] == 0 else None, "unit": "cell-steps/s",
               "cores": r["threads"], "kind": "oracle",
               "sample": f"one full step of {cfgs[0].name} ({cfgs[0].nx}x{cfgs[0].ny}) from the GPU run's state at "
                         f"the start of the timed window, {r['sweeps_p']} pressure sweeps at the oracle's own "
                         f"relaxation factor {r['omega']:.6f}, {r['seconds']:.1f} s, FP64 oracle, "
                         f"{r['threads']} OpenMP threads in the pressure solve (all host cores)",
               "one_core": {"value": cfgs[0].cells / r["seconds_1thread"] if r["rc"] == 0 else None,
                            "unit": "cell-steps/s", "cores": 1,
                            "sample": f"the same step with its sweeps at the one-thread rate "
                                      f"({r['sweep_ms_1thread']:.1f} ms per sweep against {r['sweep_ms_all']:.1f} ms)"},
               "host": r["host"]}
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "cell-steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 sweeps, f64 residual/update/norms", "data": "synthetic",
            "config": batch_config(cfgs, world),
            "details": {"path": "mixed, batched, " + ("graph replay" if args.batch_launch == "graphs" else
                                                      "direct programmatic dependent launches"),
                        "warm_start": "previous increment", "sor_us_per_sweep_whole_batch": prof["sor_us_per_sweep"],
                        "poisson_sweeps_per_step_sum": statistics.mean(sum(x["sweeps_p"] for x in st)
                                                                       for st in stats),
                        "div_max": max(x["div_max"] for st in stats for x in st)},
            "gpu_launches": prof["launches"],
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp64", "mixed", "mg"], default="mixed",
                    help="mixed: FP32 SOR sweeps inside FP64 defect correction (the value); fp64: plain FP64; "
                         "mg: the multigrid variant as the timed path")
    ap.add_argument("--no-fp64-compare", action="store_true", help="skip the plain FP64 comparison run")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-clocks", action="store_true", help="no nvidia-smi sampling (for profiler runs)")
    ap.add_argument("--warmstart", choices=["learned", "plain"], default="learned",
                    help="learned: U-Net warm start (the value); plain: previous increment")
    ap.add_argument("--weights", default=None, help="U-Net weights (default: the package's trained weights)")
    ap.add_argument("--workload", choices=WORKLOADS, default=WORKLOADS[0])
    ap.add_argument("--cases", type=int, default=64, help="batch64: number of cases")
    ap.add_argument("--batch-launch", choices=("graphs", "direct"), default="graphs",
                    help="batch sweep pairs replayed from CUDA graphs, or launched directly as programmatic "
                         "dependents")
    ap.add_argument("--sor-shape", type=int, default=-1,
                    help="fixed FP32 sweep tile shape (index into the library's table; -1: autotuner). "
                         "For profiler runs, whose per-launch overhead distorts the autotuner's timings")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        ap.error("--warmup must be >= 3")

    from paper_2402_17337_gb300 import workloads as W
    if args.workload == "batch64":
        if args.impl == "reference":
            return run_reference(args, W.batch64()[0], batch_config(W.batch64()[:args.cases], env_int("WORLD_SIZE", 1)))
        return run_batch(args)
    cfg = getattr(W, args.workload)()
    if args.impl == "reference":
        return run_reference(args, cfg, workload_config(cfg, env_int("WORLD_SIZE", 1)))

    import numpy as np
    import torch

    import paper_2402_17337_gb300 as ibm
    from paper_2402_17337_gb300 import build as B

    rank, world, local = env_int("RANK", 0), env_int("WORLD_SIZE", 1), env_int("LOCAL_RANK", 0)
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        B.build()
    if dist:
        dist.barrier()
    B.build()

    stream = torch.cuda.Stream()

    def barrier():
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()


    # pressure relaxation factor of this grid from the device probe (untimed),
    # used by every timed run below
    probe = ibm.Solver(**solver_kwargs(cfg, 1), stream=stream.cuda_stream)
    omega_default = cfg.omega()
    cfg = dataclasses.replace(cfg, omega_p=probe.tune_omega())
    probe.close()

    learned = None
    if args.warmstart == "learned" and args.precision in ("mixed", "mg"):
        from paper_2402_17337_gb300 import warmstart
        path = args.weights or warmstart.weights_for(cfg.name)
        if not os.path.exists(path):
            path = warmstart.DEFAULT_WEIGHTS
        if not os.path.exists(path):
            raise SystemExit(f"no U-Net weights at {path}: run paper_2402_17337_gb300.train_warmstart "
                             f"or pass --warmstart plain")
        net, cT, meta = warmstart.load(path)
        if meta.get("workload") == cfg.name:
            learned = {"net": net, "cT": cT, "meta": meta}
        else:  # a network is trained for one grid and time step
            print(f"bench: no U-Net weights for {cfg.name} (have {meta.get('workload')}); plain warm start",
                  file=sys.stderr)

    def timed_run(precision, sample_clocks, ws=None):
        """W untimed steps, then K steps timed with CUDA events on the solver's stream."""
        s = ibm.Solver(**solver_kwargs(cfg, precision), stream=stream.cuda_stream)
        s.set_body(cfg.chord, cfg.tc, cfg.h, cfg.k, cfg.xc, cfg.yc)
        s.set("u", cfg.initial_u(s.shape("u")))
        if ws is not None:
            s.set_warmstart(1, ws["net"], ws["cT"])
        if args.sor_shape >= 0 and precision == 1:
            s.set_sor_shape(args.sor_shape)
        for _ in range(args.warmup):
            s.step(1)
        state = {n: s.get(n) for n in ("u", "v", "p", "phi")} if rank == 0 else None
        s.set_profiling(True)
        prof0 = s.profile()
        clocks = ClockSampler(local)
        barrier()
        if sample_clocks:
            clocks.start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.profiler.start()  # marks the timed region for a profiler (no-op otherwise)
        e0.record(stream)
        stats = [s.step(1) for _ in range(args.steps)]
        e1.record(stream)
        barrier()
        torch.cuda.profiler.stop()
        clk = clocks.stop() if sample_clocks else None
        ms_local = e0.elapsed_time(e1)
        prof = s.profile()
        ok_local = sum(1 for st in stats if st["div_max"] < cfg.div_tol)
        value, cells_ok, ms = replica_throughput(cfg.cells * ok_local, ms_local, dist, "cuda")
        ok = cells_ok / cfg.cells
        final = {n: s.get(n) for n in ("u", "v", "p")} if rank == 0 else None
        forces = s.forces() if rank == 0 else None
        s.close()
        return {"value": value, "ms": ms, "stats": stats, "ok": int(ok), "clocks": clk,
                "launches": prof["launches"] - prof0["launches"], "prof": prof, "prof0": prof0, "state": state,
                "final": final, "forces": forces}

    precision = {"fp64": 0, "mixed": 1, "mg": 2}[args.precision]
    main_run = timed_run(precision, not args.no_clocks, learned)
    value, t_max, stats, total_ok = main_run["value"], main_run["ms"], main_run["stats"], main_run["ok"]
    prof, clk, launches, start_state = main_run["prof"], main_run["clocks"], main_run["launches"], main_run["state"]
    fp64_run = timed_run(0, False) if (precision != 0 and not args.no_fp64_compare) else None
    plain_ws_run = timed_run(1, False) if (learned is not None and not args.no_fp64_compare) else None
    mg_run = timed_run(2, False) if (precision != 2 and not args.no_fp64_compare) else None

    # roofline of the dominant kernel
    peaks, peak_src = load_peaks()
    sm_mhz = peaks.get("sm_max_mhz", 2070.0)
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    fp64_peak = n_sm * FP64_FLOPS_PER_CLK_SM * sm_mhz * 1e6 / 1e12  # TFLOP/s
    fp32_peak = n_sm * FP32_FLOPS_PER_CLK_SM * sm_mhz * 1e6 / 1e12
    roof = None
    if prof["sweep_launches"] > 0:
        t_launch = prof["sweep_ms"] / prof["sweep_launches"] / 1e3
        if precision == 2:
            iters = prof["poisson_sweeps"] - main_run["prof0"]["poisson_sweeps"]
            t_iter = prof["sweep_ms"] / max(iters, 1) / 1e3
            achieved = MG_BYTES_PER_CELL_ITER * cfg.cells / t_iter / 1e9
            roof = {"bound": "hbm", "kernel": "multigrid-preconditioned FCG iteration (one V(2,2)-cycle, "
                                              "FP32, graph-replayed)",
                    "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                    "frac": achieved / peaks["hbm_gbs"], "traffic": None, "iter_us": t_iter * 1e6,
                    "peak_note": f"HBM {peaks['hbm_gbs']} GB/s ({peak_src}); algorithmic "
                                 f"{MG_BYTES_PER_CELL_ITER} B per fine cell per iteration; FP32 working set "
                                 f"{cfg.cells * 24 / 1e6:.0f} MB against 129 MB of L2"}
        elif precision == 0:
            flops = SOR_FLOPS_PER_UPDATE * cfg.cells / 2
            achieved = flops / t_launch / 1e12
            roof = {"bound": "alu", "kernel": "k_poisson_half (FP64 red-black SOR half-sweep)",
                    "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s", "frac": achieved / fp64_peak,
                    "traffic": None, "launch_us": t_launch * 1e6,
                    "hbm_gbs": SOR_BYTES_PER_CELL_HALF * cfg.cells / t_launch / 1e9,
                    "peak_note": f"FP64: {n_sm} SMs x 4 flop/clk x {sm_mhz:.0f} MHz (derived)"}
        else:
            nbytes = SOR32_BYTES_PER_CELL_LAUNCH * cfg.cells
            achieved = nbytes / t_launch / 1e9
            rows, half, nyt = prof["sor_shape"]
            sweeps_per_launch = half / 2
            traffic = SOR32_TRAFFIC.get((cfg.name, (rows, half, nyt, prof["sor_form"])))
            inst = SOR32_INST.get((cfg.name, (rows, half, nyt, prof["sor_form"])))
            clk_mhz = (clk or {}).get("sm_mhz") or sm_mhz
            issue = None
            if inst:
                peak_issue = n_sm * 4 * clk_mhz * 1e6  # one warp instruction per clock per SM sub-partition
                issue = {"inst_per_launch": inst, "achieved_inst_per_s": inst / t_launch,
                         "peak_inst_per_s": peak_issue, "frac": inst / t_launch / peak_issue,
                         "note": f"warp instructions of one launch (ncu) over the live launch time, against "
                                 f"{n_sm} SMs x 4 issue slots per clock at {clk_mhz:.0f} MHz (sampled median)"}
            roof = {"bound": "hbm", "kernel": f"k_sor32_rb (FP32 red-black SOR, tile {rows} rows x 128 cells, "
                                              f"{half} half-sweeps per launch, chosen by the autotuner)",
                    "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                    "frac": achieved / peaks["hbm_gbs"], "traffic": traffic, "launch_us": t_launch * 1e6,
                    "shape": [rows, half, nyt, prof["sor_form"]], "shape_index": prof["sor_index"],
                    "fp32_tflops": SOR_FLOPS_PER_UPDATE * cfg.cells * sweeps_per_launch / t_launch / 1e12,
                    "fp32_peak_tflops": fp32_peak, "issue": issue,
                    "peak_note": f"HBM {peaks['hbm_gbs']} GB/s ({peak_src}); algorithmic bytes "
                                 f"{SOR32_BYTES_PER_CELL_LAUNCH} B/cell per launch (e and r read, e written, once "
                                 f"per launch of {half} half-sweeps; the kernel also reads the FP32 reciprocal "
                                 f"diagonal); FP32 working set {cfg.cells * 16 / 1e6:.0f} MB against 129 MB of L2"}

    # ------------------------------------------------------------- end to end
    # A second context runs the same warm-up and the same window of steps
    # through the public API, with the state round-tripped through pinned
    # host memory every step (the data movement of the paper's Sec. 3.4.4).
    e2e = None
    if not args.no_e2e:
        s2 = ibm.Solver(**solver_kwargs(cfg, precision), stream=stream.cuda_stream)
        s2.set_body(cfg.chord, cfg.tc, cfg.h, cfg.k, cfg.xc, cfg.yc)
        s2.set("u", cfg.initial_u(s2.shape("u")))
        if learned is not None:
            s2.set_warmstart(1, learned["net"], learned["cT"])
        for _ in range(args.warmup):
            s2.step(1)
        names = ("u", "v", "p", "phi")
        pinned = {n: torch.empty(s2.shape(n), dtype=torch.float64, pin_memory=True).numpy() for n in names}
        for n in names:
            pinned[n][...] = s2.get(n)
        h2d = sum(a.nbytes for a in pinned.values())
        barrier()
        t0 = time.perf_counter()
        ok_e2e = 0
        for _ in range(args.steps):
            for n in names:
                s2.set(n, pinned[n])
            st = s2.step(1)
            for n in names:
                s2.get(n, out=pinned[n])
            ok_e2e += st["div_max"] < cfg.div_tol
        barrier()
        te = time.perf_counter() - t0
        s2.close()
        e2e_value, _, _ = replica_throughput(cfg.cells * ok_e2e, 1e3 * te, dist, "cuda")
        e2e = {"value": e2e_value, "unit": "cell-steps/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": h2d,
               "note": "same steps as the timed window on a second context; per step u, v, p, phi copied "
                       "in from pinned host memory, step, copied back into pinned host memory; host wall clock"}

    # ------------------------------------------------------------ CPU oracle
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        r = cpu_oracle_sample(cfg, start_state)
        cpu = {"value": cfg.cells / r["seconds"] if r["rc"] == 0 else None, "unit": "cell-steps/s",
               "cores": r["threads"], "kind": "oracle",
               "sample": f"one full step of {cfg.name} started from the GPU run's state at the start of the "
                         f"timed window (AB2 history restarted), {r['sweeps_p']} pressure sweeps at the oracle's "
                         f"own relaxation factor {r['omega']:.6f}, {r['seconds']:.1f} s, FP64 oracle, "
                         f"{r['threads']} OpenMP threads in the pressure solve (all host cores)",
               "one_core": {"value": cfg.cells / r["seconds_1thread"] if r["rc"] == 0 else None,
                            "unit": "cell-steps/s", "cores": 1,
                            "sample": f"the same step with its {r['sweeps_p']} sweeps at the one-thread rate "
                                      f"({r['sweep_ms_1thread']:.1f} ms per sweep against "
                                      f"{r['sweep_ms_all']:.1f} ms on {r['threads']} threads, 128 sweeps each); "
                                      f"the rest of the oracle's step is single-threaded in both"},
               "host": r["host"]}

    if rank == 0:
        sweeps = [st["sweeps_p"] for st in stats]
        def field_errors(run):
            """Per-field relative error (inf-norm) against the plain FP64 run after the same steps."""
            if not run or not fp64_run or run["final"] is None:
                return None
            ref = fp64_run["final"]
            out = {n: float(np.abs(run["final"][n] - ref[n]).max() / np.abs(ref[n]).max()) for n in ref}
            (cl, cd), (cl0, cd0) = run["forces"], fp64_run["forces"]
            out["cl"] = float(np.abs(cl - cl0).max() / np.abs(cl0).max())
            out["cd"] = float(np.abs(cd - cd0).max() / np.abs(cd0).max())
            return out

        fp64 = None
        if fp64_run:
            fp64 = {"value": fp64_run["value"], "ms_per_step": fp64_run["ms"] / args.steps,
                    "poisson_sweeps_per_step": statistics.mean(st["sweeps_p"] for st in fp64_run["stats"]),
                    "speedup_of_value": value / fp64_run["value"]}
        plain_ws = None
        if plain_ws_run:
            plain_ws = {"value": plain_ws_run["value"], "ms_per_step": plain_ws_run["ms"] / args.steps,
                        "error_vs_fp64": field_errors(plain_ws_run),
                        "poisson_sweeps_per_step": statistics.mean(st["sweeps_p"] for st in plain_ws_run["stats"]),
                        "speedup_of_value": value / plain_ws_run["value"]}
        if fp64:
            fp64["error_vs_fp64_of_value"] = field_errors(main_run)
        mg = None
        if mg_run:
            mg = {"value": mg_run["value"], "ms_per_step": mg_run["ms"] / args.steps,
                  "vcycles_per_step": statistics.mean(st["sweeps_p"] for st in mg_run["stats"]),
                  "speedup_of_value": mg_run["value"] / value, "error_vs_fp64": field_errors(mg_run),
                  "note": "variant, not the paper's solver: FP32 geometric-multigrid V(2,2)-cycles (red-black "
                          "Gauss-Seidel smoothing, bilinear prolongation) inside the same FP64 defect correction "
                          "and stopping rule; previous-increment warm start"}
        ws_desc = "previous increment"
        if learned is not None:
            m = learned["meta"]
            kept = prof["ws_kept"] - main_run["prof0"]["ws_kept"]
            applied = prof["ws_applied"] - main_run["prof0"]["ws_applied"]
            ws_desc = (f"learned: U-Net widths {tuple(m.get('widths', ()))} on the 2x coarsened grid, trained on "
                       f"{m.get('samples')} snapshots of {m.get('runs')} seeded runs (h, k, Re drawn), BF16 "
                       f"tensor-core kernels; the learned guess is kept only when its residual is below half the "
                       f"previous increment's: kept in {kept} of {applied} timed steps")
        netroof = network_roofline(learned, cfg, stream, peaks, peak_src) if learned is not None else None
        line = {
            "metric": METRIC, "value": value, "unit": "cell-steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": ("f32 sweeps, f64 residual/update/norms" + (", bf16 U-Net" if learned else ""))
                     if precision >= 1 else "f64",
            "data": "synthetic",
            "config": workload_config(cfg, world),
            "details": {"path": args.precision, "warm_start": ws_desc,
                        "omega_p": cfg.omega_p, "omega_p_grid_formula": omega_default,
                        "mixed_plain_warmstart": plain_ws, "plain_fp64": fp64, "multigrid_variant": mg,
                        "steps_counted": total_ok, "poisson_sweeps_per_step": statistics.mean(sweeps),
                        "helm_sweeps_per_step": statistics.mean(st["sweeps_u"] + st["sweeps_v"] for st in stats),
                        "div_max": max(st["div_max"] for st in stats)},
            "gpu_launches": launches,
            "roofline": roof,
            "network": netroof,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
