"""The paper's validation set-up (Sec. 4.1), run on the GPU.

    python -m paper_2402_17337_gb300.validation [--periods 1.5] [--precision 1] [--out result.json]

A plunging elliptic foil (thickness/chord 0.12) at Re 500 with plunge
amplitude h = 0.16 and reduced frequency k = 2 pi, on the paper's domain
[-7.5, 24] x [-12.5, 12.5] with minimum spacing 0.004 and time step 1e-4,
on three meshes of about 0.6, 1.2 and 1.8 million cells (the paper's
M1-M3).  For each mesh: the lift and drag histories over the requested
number of plunge periods (period 2 pi / k = 1), the lift amplitude and the
mean drag over the last full period, and the relative change between
meshes.  The paper compares its histories with a figure of other authors'
data that is not available here; what is reported is the solver's own
mesh convergence and the sign of the mean drag (a foil plunging at k h
near 1 produces thrust, i.e. a negative mean drag).

Reading of the meshes: the paper states one spacing (0.004) for its
validation and names M1-M3 only by their cell counts in its performance
study (Sec. 4.2), so the three meshes here share the uniform region and its
spacing and differ in the stretched far field; their agreement measures
far-field independence, not near-body resolution.  The default solver is
the paper's red-black SOR (FP32 sweeps inside FP64 defect correction,
precision 1); precision 2 is the multigrid variant.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import math
import sys
import time

import numpy as np

import paper_2402_17337_gb300 as ibm
from paper_2402_17337_gb300 import workloads as W

MESHES = {"M1": (1104, 552), "M2": (1552, 776), "M3": (1904, 952)}


# the uniform region (spacing 0.004) covers the body's swept region, x in
# [-0.5, 0.5] and |y| <= h + t/2 = 0.22, with a margin; the paper gives the
# spacing but not the region's extent
UBOX = (-0.6, 1.2, -0.3, 0.3)


def config(nx, ny):
    hmin = 0.004
    return W.FlowConfig(f"validation_{nx}x{ny}", *W.PAPER_DOMAIN, nx, ny, hmin, Re=500.0, dt=1e-4, steps=0,
                        h=0.16, k=2.0 * math.pi, div_tol=1e-8, init="uniform", ubox=UBOX)


def run(cfg, periods, precision):
    probe = ibm.Solver.from_config(cfg, precision=1)
    cfg = dataclasses.replace(cfg, omega_p=probe.tune_omega())
    probe.close()
    s = ibm.Solver.from_config(cfg, precision=precision, max_sweeps=20000 if precision == 2 else 0)
    s.set("u", cfg.initial_u(s.shape("u")))
    period = 2.0 * math.pi / cfg.k
    steps = int(round(periods * period / cfg.dt))
    t0 = time.perf_counter()
    div = 0.0
    chunk = 500
    done = 0
    while done < steps:
        st = s.step(min(chunk, steps - done))
        done = st["n"]
        div = max(div, st["div_max"])
    seconds = time.perf_counter() - t0
    cl, cd = s.forces()
    s.close()
    n_per = int(round(period / cfg.dt))
    last_cl, last_cd = cl[-n_per:], cd[-n_per:]
    return {"nx": cfg.nx, "ny": cfg.ny, "cells": cfg.cells, "steps": steps, "seconds": seconds,
            "cell_steps_per_s": cfg.cells * steps / seconds, "last_step_div_max": div,
            "cl_amplitude": float(0.5 * (last_cl.max() - last_cl.min())), "cl_mean": float(last_cl.mean()),
            "cd_mean": float(last_cd.mean()), "cd_amplitude": float(0.5 * (last_cd.max() - last_cd.min())),
            "omega_p": cfg.omega_p}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--periods", type=float, default=1.5)
    ap.add_argument("--precision", type=int, default=1, help="0 FP64, 1 mixed SOR (default), 2 multigrid variant")
    ap.add_argument("--meshes", nargs="+", default=list(MESHES))
    ap.add_argument("--out", default=None)
    args = ap.parse_args(argv)
    from paper_2402_17337_gb300 import build
    build.build()
    res = {}
    for name in args.meshes:
        nx, ny = MESHES[name]
        res[name] = run(config(nx, ny), args.periods, args.precision)
        print(name, json.dumps(res[name]), flush=True)
    names = [n for n in MESHES if n in res]
    for a, b in zip(names, names[1:]):
        for key in ("cl_amplitude", "cd_mean"):
            res[f"change_{key}_{a}_{b}"] = abs(res[b][key] - res[a][key]) / max(abs(res[b][key]), 1e-300)
    out = {"setup": "Sec. 4.1: Re 500, h 0.16, k 2 pi, t/c 0.12, spacing 0.004, dt 1e-4", "precision": args.precision,
           "periods": args.periods, "meshes": res}
    print(json.dumps(out), flush=True)
    if args.out:
        with open(args.out, "w") as fh:
            json.dump(out, fh, indent=1)
    return 0


if __name__ == "__main__":
    sys.exit(main())
