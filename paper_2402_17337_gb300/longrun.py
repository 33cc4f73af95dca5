"""Full-length run of a workload on the GPU: the mixed path (FP32 red-black
SOR sweeps inside FP64 defect correction) and the plain FP64 path (the
paper's method, Sec. 2.2) advance side by side for the configuration's whole
step count.  Reported: the largest fluid-cell divergence of any step on each
path, the pressure sweeps per step, and at checkpoints the mixed path's
relative error against the FP64 path, ||a - b||_inf / ||b||_inf for u, v and
p, and for the lift and drag histories max |a - b| / max |b| (the Sec. 4.1
force coefficients).

    python -m paper_2402_17337_gb300.longrun --workload plunge_2048x1024 [--steps N] [--out run.json]
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


def run(workload: str, steps: int | None = None, checkpoints: int = 4) -> dict:
    import dataclasses
    cfg = WORKLOADS[workload]()
    n = steps or cfg.steps
    probe = ibm.Solver.from_config(cfg, precision=1)
    cfg = dataclasses.replace(cfg, omega_p=probe.tune_omega())
    probe.close()
    paths = {"mixed": ibm.Solver.from_config(cfg, precision=1), "fp64": ibm.Solver.from_config(cfg, precision=0)}
    for s in paths.values():
        s.set("u", cfg.initial_u(s.shape("u")))
    marks = sorted({max(1, round(n * (i + 1) / checkpoints)) for i in range(checkpoints)})
    div = {k: 0.0 for k in paths}
    sweeps = {k: [] for k in paths}
    wall = {k: 0.0 for k in paths}
    report = []
    for t in range(1, n + 1):
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
    return {"workload": workload, "steps": n, "cells": cfg.cells, "omega_p": cfg.omega_p,
            "div_tol": cfg.div_tol, "div_max": div, "checkpoints": report,
            "poisson_sweeps_per_step": {k: float(np.mean(v)) for k, v in sweeps.items()},
            "wall_s": wall, "cell_steps_per_s_host_wall": {k: cfg.cells * n / wall[k] for k in wall}}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="plunge_2048x1024")
    ap.add_argument("--steps", type=int, default=0, help="0: the configuration's step count")
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    res = run(a.workload, a.steps or None)
    line = json.dumps(res)
    if a.out:
        with open(a.out, "w") as fh:
            fh.write(line + "\n")
    print(line)


if __name__ == "__main__":
    main()
