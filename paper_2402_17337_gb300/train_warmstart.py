"""Trains the warm-start U-Net of a workload on snapshots the solver generates.

    python -m paper_2402_17337_gb300.train_warmstart --workload plunge_2048x1024 \
        --runs 4 --steps 60 --epochs 20 --out weights.npz
    python -m paper_2402_17337_gb300.train_warmstart --workload unet_1024x512 \
        --samples 20000 --start 200 --every 1 --steps 700 --epochs 8 --out weights.npz

Training runs use the workload's grid and time step with seeded foil
parameters (h ~ U[0.1, 0.5], k ~ U[1, 4], Re ~ U[100, 1000]) and record one
sample per step from the first step on (features and target of the learned
warm start, as defined by the library).  The U-Net trains with the library's
forward, backward and Adam kernels.  A held-out evaluation on the workload's
own parameters compares pressure sweeps per step with the plain warm start
(previous increment) and the learned one.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import sys
import time

import numpy as np

import paper_2402_17337_gb300 as ibm
from paper_2402_17337_gb300 import workloads as W
from paper_2402_17337_gb300 import warmstart

WIDTHS = (32, 64, 128, 128)


def training_configs(cfg, runs, seed):
    rng = np.random.default_rng(seed)
    out = []
    for r in range(runs):
        h, k, Re = rng.uniform(0.1, 0.5), rng.uniform(1.0, 4.0), rng.uniform(100.0, 1000.0)
        out.append(dataclasses.replace(cfg, name=f"{cfg.name}[train {r}]", h=float(h), k=float(k), Re=float(Re)))
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--workload", default="plunge_2048x1024")
    ap.add_argument("--runs", type=int, default=4)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--epochs", type=int, default=20)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=2402)
    ap.add_argument("--eval-start", type=int, default=3)
    ap.add_argument("--eval-steps", type=int, default=10)
    ap.add_argument("--widths", type=int, nargs=4, default=list(WIDTHS),
                    help="channels of the four levels (multiples of 16)")
    ap.add_argument("--samples", type=int, default=0,
                    help="train on this many snapshots held in device memory, taken every --every steps "
                         "after --start steps of as many seeded runs as it takes (0: one per step of --runs runs)")
    ap.add_argument("--start", type=int, default=200)
    ap.add_argument("--every", type=int, default=1)
    ap.add_argument("--out", required=True)
    args = ap.parse_args(argv)

    from paper_2402_17337_gb300 import build
    build.build()
    cfg = getattr(W, args.workload)()
    t0 = time.perf_counter()
    if args.samples > 0:
        import torch
        Hc, Wc = cfg.ny // 2, cfg.nx // 2
        feats = torch.empty((args.samples, Hc, Wc, 4), dtype=torch.float32, device="cuda")
        targs = torch.empty((args.samples, Hc, Wc), dtype=torch.float32, device="cuda")
        pos, runs = 0, 0
        while pos < args.samples:
            (c,) = training_configs(cfg, runs + 1, args.seed)[runs:]
            pos, sw = warmstart.capture_to_device(c, steps=args.steps, start=args.start, every=args.every,
                                                  feats=feats, targs=targs, pos=pos)
            runs += 1
            print(f"run {runs}: {len(sw)} samples of {c.name} (h={c.h:.3f} k={c.k:.3f} Re={c.Re:.0f}), "
                  f"{pos} in total, {time.perf_counter() - t0:.0f} s", flush=True)
        samples = (feats, targs)
        n_samples, args.runs = pos, runs
    else:
        samples = warmstart.Samples([], [], [])
        for c in training_configs(cfg, args.runs, args.seed):
            s = warmstart.capture(c, steps=args.steps, start=0, every=1)
            samples.feat += s.feat
            samples.target += s.target
            samples.sweeps += s.sweeps
            print(f"captured {len(s.feat)} samples of {c.name} (h={c.h:.3f} k={c.k:.3f} Re={c.Re:.0f}), "
                  f"{time.perf_counter() - t0:.0f} s", flush=True)
        n_samples = len(samples.feat)
    net = ibm.UNet(tuple(args.widths), seed=args.seed)
    t1 = time.perf_counter()
    cT, hist = warmstart.train(net, samples, epochs=args.epochs, lr=args.lr, seed=args.seed,
                               log=lambda m: print(m, flush=True))
    t_train = time.perf_counter() - t1
    res = warmstart.evaluate(cfg, net, cT, steps=args.eval_steps, start=args.eval_start)
    plain, learned = sum(res["plain"]["sweeps"]), sum(res["learned"]["sweeps"])
    meta = {"workload": cfg.name, "widths": list(args.widths), "runs": args.runs, "steps_per_run": args.steps,
            "samples": n_samples, "sample_start": args.start if args.samples else 0,
            "sample_every": args.every if args.samples else 1, "epochs": args.epochs, "lr": args.lr, "seed": args.seed,
            "loss_first_epoch": hist[0], "loss_last_epoch": hist[-1], "train_seconds": t_train,
            "eval": {"steps": [args.eval_start, args.eval_start + args.eval_steps],
                     "plain_sweeps": res["plain"]["sweeps"], "learned_sweeps": res["learned"]["sweeps"],
                     "plain_seconds": res["plain"]["seconds"], "learned_seconds": res["learned"]["seconds"],
                     "sweep_gain": 1.0 - learned / plain}}
    warmstart.save(args.out, net, cT, meta)
    print(json.dumps(meta), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
