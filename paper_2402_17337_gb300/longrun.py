"""Full-length run of a workload on the GPU: the mixed path (FP32 red-black
SOR sweeps inside FP64 defect correction) and the plain FP64 path (the
paper's method, Sec. 2.2) advance side by side for the configuration's whole
step count.  Reported: the largest fluid-cell divergence of any step on each
path, the pressure sweeps per step, and at checkpoints the mixed path's
relative error against the FP64 path, ||a - b||_inf / ||b||_inf for u, v and
p, and for the lift and drag histories max |a - b| / max |b| (the Sec. 4.1
force coefficients).  With --compare-steps the FP64 path stops after that
many steps (the checkpoints fall in that window) and the mixed path runs on
alone.  --workload batch64 advances the 64 cases of uneven grids as one batch
(every part of the step shared across cases) for their step count and
reports the largest divergence of every case over all steps.

    python -m paper_2402_17337_gb300.longrun --workload plunge_2048x1024 [--steps N]
        [--compare-steps M] [--out run.json]
    python -m paper_2402_17337_gb300.longrun --workload batch64 [--steps N]
"""
from __future__ import annotations

import argparse
import json
import sys
import time

import numpy as np

import paper_2402_17337_gb300 as ibm
from paper_2402_17337_gb300 import workloads as W

WORKLOADS = {"plunge_192x128": W.plunge_192x128, "plunge_2048x1024": W.plunge_2048x1024,
             "plunge_4096x2048": W.plunge_4096x2048, "unet_1024x512": W.unet_1024x512}


def rel(a, b):
    d = float(np.abs(b).max())
    return float(np.abs(a - b).max()) / d if d > 0 else float(np.abs(a - b).max())


def run(workload: str, steps: int | None = None, checkpoints: int = 4, compare_steps: int | None = None) -> dict:
    import dataclasses
    cfg = WORKLOADS[workload]()
    n = steps or cfg.steps
    probe = ibm.Solver.from_config(cfg, precision=1)
    cfg = dataclasses.replace(cfg, omega_p=probe.tune_omega())
    probe.close()
    paths = {"mixed": ibm.Solver.from_config(cfg, precision=1), "fp64": ibm.Solver.from_config(cfg, precision=0)}
    for s in paths.values():
        s.set("u", cfg.initial_u(s.shape("u")))
    nc = min(n, compare_steps or n)  # steps of the FP64 path
    marks = sorted({max(1, round(nc * (i + 1) / checkpoints)) for i in range(checkpoints)})
    div = {k: 0.0 for k in paths}
    sweeps = {k: [] for k in paths}
    wall = {k: 0.0 for k in paths}
    report = []
    for t in range(1, n + 1):
        if t == nc + 1:
            paths.pop("fp64").close()
        for k, s in paths.items():
            t0 = time.perf_counter()
            st = s.step(1)  # returns after the step's last host check, so the wall time is the step's
            wall[k] += time.perf_counter() - t0
            div[k] = max(div[k], st["div_max"])
            sweeps[k].append(st["sweeps_p"])
        if t in marks:
            m, f = paths["mixed"], paths["fp64"]
            e = {name: rel(m.get(name), f.get(name)) for name in ("u", "v", "p")}
            (clm, cdm), (clf, cdf) = m.forces(), f.forces()
            e["cl"], e["cd"] = rel(clm, clf), rel(cdm, cdf)
            report.append({"step": t, "error_vs_fp64": e, "cl": float(clm[-1]), "cd": float(cdm[-1])})
            print(f"{workload} step {t}: " + ", ".join(f"{k} {v:.2e}" for k, v in e.items()), file=sys.stderr)
    for s in paths.values():
        s.close()
    steps_run = {"mixed": n, "fp64": nc}
    return {"workload": workload, "steps": n, "steps_run": steps_run, "cells": cfg.cells, "omega_p": cfg.omega_p,
            "div_tol": cfg.div_tol, "div_max": div, "checkpoints": report,
            "poisson_sweeps_per_step": {k: float(np.mean(v)) for k, v in sweeps.items()},
            "wall_s": wall, "cell_steps_per_s_host_wall": {k: cfg.cells * steps_run[k] / wall[k] for k in wall}}


def run_batch(steps: int | None = None, cases: int = 64) -> dict:
    """The batch of cases with uneven grids for its step count: divergence of
    every case in every step (mixed path; no FP64 comparison)."""
    import dataclasses
    cfgs = W.batch64()[:cases]
    n = steps or cfgs[0].steps
    omegas = []
    for c in cfgs:  # each case's relaxation factor from the device probe
        s = ibm.Solver.from_config(c, precision=1)
        omegas.append(s.tune_omega())
        s.close()
    cfgs = [dataclasses.replace(c, omega_p=w) for c, w in zip(cfgs, omegas)]
    ss = []
    for c in cfgs:
        s = ibm.Solver.from_config(c, precision=1)
        s.set("u", c.initial_u(s.shape("u")))
        ss.append(s)
    b = ibm.Batch(ss)
    div = [0.0] * len(cfgs)
    sweeps = 0.0
    t0 = time.perf_counter()
    for t in range(n):
        for i, st in enumerate(b.step(1)):
            div[i] = max(div[i], st["div_max"])
            sweeps += st["sweeps_p"]
    wall = time.perf_counter() - t0
    cells = sum(c.cells for c in cfgs)
    b.close()
    for s in ss:
        s.close()
    return {"workload": "batch64" if cases == 64 else f"batch64[:{cases}]", "steps": n, "cases": len(cfgs),
            "cells_per_step": cells, "div_tol": cfgs[0].div_tol, "div_max_per_case": div,
            "div_max": max(div), "all_below_tol": all(d <= c.div_tol for d, c in zip(div, cfgs)),
            "poisson_sweeps_per_case_step": sweeps / (n * len(cfgs)), "wall_s": wall,
            "cell_steps_per_s_host_wall": cells * n / wall}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + ["batch64"], default="plunge_2048x1024")
    ap.add_argument("--steps", type=int, default=0, help="0: the configuration's step count")
    ap.add_argument("--compare-steps", type=int, default=0, help="FP64 steps (0: all)")
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    if a.workload == "batch64":
        res = run_batch(a.steps or None)
    else:
        res = run(a.workload, a.steps or None, compare_steps=a.compare_steps or None)
    line = json.dumps(res)
    if a.out:
        with open(a.out, "w") as fh:
            fh.write(line + "\n")
    print(line)


if __name__ == "__main__":
    main()
