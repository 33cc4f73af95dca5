"""The U-Net as preconditioner of the multigrid variant's FCG iteration,
against the V-cycle it would replace.

    python -m paper_2402_17337_gb300.precond_eval [--workload plunge_2048x1024] [--steps 6] [--cap 3000]

The workload runs with precision 2 (FP32 FCG inside the FP64 defect
correction) under four preconditioners: the V(2,2)-cycle; the two-level
cycle whose coarse level is the workload's trained U-Net (the learned warm
start's network, whose target is the coarse change of the pressure increment
per unit residual), with and without pre-smoothing; and the same cycle with
the network's output scaled to nothing, i.e. smoothing alone, which shows
what the network adds.  For each: FCG iterations and host wall time per
step, or, when the iteration cap stops the solve, the residual reached.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import sys
import time

import paper_2402_17337_gb300 as ibm
from paper_2402_17337_gb300 import warmstart
from paper_2402_17337_gb300 import workloads as W


def run(cfg, steps, cap, pc):
    s = ibm.Solver.from_config(cfg, precision=2, max_sweeps=cap)
    s.set("u", cfg.initial_u(s.shape("u")))
    if pc is not None:
        s.set_preconditioner(1, *pc)
    its, ms = [], []
    out = {}
    try:
        for _ in range(steps):
            t0 = time.perf_counter()
            st = s.step(1)  # returns after the step's last norm is read
            ms.append(round(1e3 * (time.perf_counter() - t0), 2))
            its.append(st["sweeps_p"])
        out["div_max"] = st["div_max"]
    except ibm.IbmError as e:
        out["stopped"] = str(e)
    s.close()
    out.update(fcg_iterations=its, ms_per_step=ms)
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--workload", default="plunge_2048x1024")
    ap.add_argument("--weights", default=None, help="network (default: the workload's trained warm-start weights)")
    ap.add_argument("--steps", type=int, default=6)
    ap.add_argument("--cap", type=int, default=3000, help="FCG iterations per solve before it is stopped")
    args = ap.parse_args(argv)
    from paper_2402_17337_gb300 import build
    build.build()
    cfg = getattr(W, args.workload)()
    probe = ibm.Solver.from_config(cfg, precision=1)
    cfg = dataclasses.replace(cfg, omega_p=probe.tune_omega())
    probe.close()
    net, cT, meta = warmstart.load(args.weights or warmstart.weights_for(cfg.name))
    res = {"workload": cfg.name, "network": {"widths": meta.get("widths"), "target_scale": cT}}
    for name, pc in (("v_cycle", None), ("unet_two_level", (net, cT, 1)), ("unet_two_level_no_presmoothing", (net, cT, 0)),
                     ("smoothing_only", (net, 1e-30, 1))):
        res[name] = run(cfg, args.steps, args.cap, pc)
        print(name, json.dumps(res[name]), flush=True)
    net.close()
    print(json.dumps(res), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
