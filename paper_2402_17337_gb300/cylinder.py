"""Stationary circular cylinder at Re = 100: vortex shedding and its
Strouhal number, a physical check of the whole step.

    python -m paper_2402_17337_gb300.cylinder [--precision 1] [--t-end 150] [--window 50] [--out result.json]

The discrete-forcing method applied to a fixed circle (ellipse of thickness
ratio 1, no plunge) of diameter D = 1 in a uniform stream U = 1, on a
stretched grid over [-10, 30] x [-15, 15] (spacing 0.025, 40 cells per
diameter, inside [-1, 3] x [-1.5, 1.5]).  The flow starts uniform with a
small transverse velocity bump behind the cylinder, which breaks the
top/bottom symmetry so that the wake starts shedding early.  The lift
coefficient oscillates at the shedding frequency f; over the last `window`
time units of the run, f is taken from the up-crossings of C_l through its
mean, and St = f D / U.  Measured values for Re = 100 lie between 0.16 and
0.17; the mean drag coefficient is about 1.3-1.4 and the lift amplitude
about 0.3.
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

CONFIG = W.FlowConfig("cylinder_re100_320x256", -10.0, 30.0, -15.0, 15.0, 320, 256, 0.025, Re=100.0, dt=0.005,
                      steps=0, h=0.0, k=0.0, tc=1.0, ubox=(-1.0, 3.0, -1.5, 1.5), init="uniform")


def perturbation(xf, yf, amplitude=0.2):
    """Transverse velocity bump centred two diameters behind the cylinder,
    on the v nodes (x cell centres, y faces)."""
    xc = 0.5 * (xf[1:] + xf[:-1])
    X, Y = np.meshgrid(xc, yf)
    return amplitude * np.exp(-((X - 2.0) ** 2 + Y ** 2))


def strouhal(cl, dt, window):
    """Shedding frequency from the up-crossings of C_l through its mean over
    the last `window` time units (linear interpolation between steps); also
    the lift amplitude over that window."""
    n = int(round(window / dt))
    c = np.asarray(cl[-n:], dtype=np.float64)
    c = c - c.mean()
    t = dt * np.arange(len(c))
    up = np.nonzero((c[:-1] < 0.0) & (c[1:] >= 0.0))[0]
    times = t[up] + dt * (-c[up]) / (c[up + 1] - c[up])
    amp = 0.5 * (c.max() - c.min())
    if len(times) < 3:
        return float("nan"), amp, len(times)
    return (len(times) - 1) / (times[-1] - times[0]), amp, len(times)


def run(cfg=CONFIG, t_end=150.0, window=50.0, precision=1, log=None):
    s = ibm.Solver.from_config(cfg, precision=precision)
    s.set("u", cfg.initial_u(s.shape("u")))
    xf, yf = s.grid()
    s.set("v", perturbation(xf, yf))
    steps = int(round(t_end / cfg.dt))
    chunk = 1000
    t0 = time.perf_counter()
    done, div, sweeps = 0, 0.0, 0
    while done < steps:
        st = s.step(min(chunk, steps - done))
        done = st["n"]
        div = max(div, st["div_max"])
        sweeps = st["sweeps_p"]
        if log:
            log(f"t = {done * cfg.dt:.1f}: div {st['div_max']:.2e}, last pressure solve {sweeps} sweeps, "
                f"C_l {st['cl']:+.4f}, C_d {st['cd']:.4f}")
    seconds = time.perf_counter() - t0
    cl, cd = s.forces()
    s.close()
    st_num, amp, crossings = strouhal(cl, cfg.dt, window)
    n = int(round(window / cfg.dt))
    return {"workload": cfg.name, "Re": cfg.Re, "dt": cfg.dt, "steps": steps, "precision": precision,
            "seconds": seconds, "strouhal": st_num, "cl_amplitude": float(amp), "cd_mean": float(np.mean(cd[-n:])),
            "up_crossings": crossings, "window": window, "max_step_div": div}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--precision", type=int, default=1, help="0 FP64, 1 mixed, 2 multigrid variant")
    ap.add_argument("--t-end", type=float, default=150.0)
    ap.add_argument("--window", type=float, default=50.0)
    ap.add_argument("--out", default=None)
    args = ap.parse_args(argv)
    from paper_2402_17337_gb300 import build
    build.build()
    probe = ibm.Solver.from_config(CONFIG, precision=1)
    cfg = dataclasses.replace(CONFIG, omega_p=probe.tune_omega())
    probe.close()
    res = run(cfg, args.t_end, args.window, args.precision, log=lambda m: print(m, flush=True))
    print(json.dumps(res), flush=True)
    if args.out:
        with open(args.out, "w") as fh:
            json.dump(res, fh, indent=1)
    return 0


if __name__ == "__main__":
    sys.exit(main())
