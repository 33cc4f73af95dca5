"""Training of the learned warm start (orchestration only).

Every numerical step runs in libibm's kernels: the solver records samples
(ibm_set_warmstart mode 2), the U-Net trains with the library's forward,
backward and Adam kernels (ibm_unet_train_step), and the trained network is
attached to a solver as its warm start (mode 1).  PyTorch only holds the
samples in device memory.

A sample is taken right before a pressure solve: features of the 2x
coarsened grid (initial residual, right-hand side, body-cell fraction,
pressure; each over its infinity norm) and the target, the coarsened change
of the pressure increment over the step in units of the residual's norm.
The model's target scale c_T is the RMS of the training targets, so the
network learns values of order one.
"""
from __future__ import annotations

import dataclasses
import json
import os
import time

import numpy as np

import paper_2402_17337_gb300 as ibm

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_WEIGHTS = os.path.join(HERE, "weights", "unet_plunge_2048x1024.npz")


def weights_for(workload):
    """Path of the package's trained weights for a workload (may not exist):
    weights/unet_<workload>.npz, without doubling a workload name that
    already starts with unet_."""
    stem = workload if workload.startswith("unet_") else f"unet_{workload}"
    return os.path.join(HERE, "weights", f"{stem}.npz")


@dataclasses.dataclass
class Samples:
    feat: list
    target: list
    sweeps: list


def capture(cfg, steps, start, every, precision=1, stream=None):
    """Runs the workload with the plain warm start and records a sample
    every `every` steps after `start`."""
    s = ibm.Solver.from_config(cfg, precision=precision, stream=stream)
    s.set("u", cfg.initial_u(s.shape("u")))
    s.set_warmstart(2, None, 1.0)
    out = Samples([], [], [])
    for n in range(steps):
        st = s.step(1)
        if n >= start and (n - start) % every == 0:
            f, t = s.sample()
            out.feat.append(f)
            out.target.append(t)
            out.sweeps.append(st["sweeps_p"])
    s.close()
    return out


def capture_to_device(cfg, steps, start, every, feats, targs, pos, precision=1, stream=None):
    """As capture, but each sample goes straight into the preallocated device
    tensors feats [N, Hc, Wc, 4] and targs [N, Hc, Wc] from index pos on (no
    host list: a large training set lives in device memory).  Returns the
    next free index and the pressure sweeps of the sampled steps."""
    import torch
    s = ibm.Solver.from_config(cfg, precision=precision, stream=stream)
    s.set("u", cfg.initial_u(s.shape("u")))
    s.set_warmstart(2, None, 1.0)
    sweeps = []
    for n in range(steps):
        if pos >= feats.shape[0]:
            break
        st = s.step(1)
        if n >= start and (n - start) % every == 0:
            f, t = s.sample()
            feats[pos].copy_(torch.from_numpy(f))
            targs[pos].copy_(torch.from_numpy(t))
            sweeps.append(st["sweeps_p"])
            pos += 1
    s.close()
    return pos, sweeps


def target_scale(samples):
    return float(np.sqrt(np.mean([np.mean(t.astype(np.float64) ** 2) for t in samples.target])))


def train(net, samples, epochs, lr=1e-3, cT=None, seed=0, log=None):
    """Adam on the mean squared error, one sample per step, shuffled epochs.
    samples: a Samples of host arrays, or a pair (feats, targs) of device
    tensors [N, Hc, Wc, 4] and [N, Hc, Wc] (capture_to_device)."""
    import torch
    if isinstance(samples, tuple):
        fdev, tdev = samples
        if not cT:
            ss = sum(float(torch.sum(tdev[k:k + 256].double() ** 2)) for k in range(0, tdev.shape[0], 256))
            cT = float(np.sqrt(ss / tdev.numel()))
        tdev.div_(cT)
        feats = [fdev[k] for k in range(fdev.shape[0])]
        targs = [tdev[k] for k in range(tdev.shape[0])]
        Hc, Wc = tdev.shape[1], tdev.shape[2]
    else:
        cT = cT or target_scale(samples)
        feats = [torch.tensor(f, device="cuda") for f in samples.feat]
        targs = [torch.tensor(t / cT, device="cuda") for t in samples.target]
        Hc, Wc = samples.target[0].shape
    torch.cuda.synchronize()
    rng = np.random.default_rng(seed)
    hist = []
    for ep in range(epochs):
        order = rng.permutation(len(feats))
        tot = 0.0
        for k in order:
            tot += net.train_step(feats[k].data_ptr(), targs[k].data_ptr(), Hc, Wc, lr=lr, apply=True)
        hist.append(tot / len(feats))
        if log:
            log(f"epoch {ep}: loss {hist[-1]:.4e}")
    return cT, hist


def evaluate(cfg, net, cT, steps, start, precision=1, stream=None):
    """Sweeps and time per step, plain vs learned warm start, on the same
    steps (start .. start + steps) of the workload."""
    res = {}
    for mode in (0, 1):
        s = ibm.Solver.from_config(cfg, precision=precision, stream=stream)
        s.set("u", cfg.initial_u(s.shape("u")))
        s.set_warmstart(0)
        for _ in range(start):
            s.step(1)
        if mode == 1:
            s.set_warmstart(1, net, cT)
        sw, kept, t0 = [], [], time.perf_counter()
        for _ in range(steps):
            k0 = s.profile()["ws_kept"]
            st = s.step(1)
            sw.append(st["sweeps_p"])
            kept.append(s.profile()["ws_kept"] - k0)
            assert st["div_max"] <= cfg.div_tol * 1.001
        res["learned" if mode else "plain"] = {"sweeps": sw, "kept": kept, "seconds": time.perf_counter() - t0}
        s.close()
    return res


def save(path, net, cT, meta):
    d = os.path.dirname(path)
    if d:
        os.makedirs(d, exist_ok=True)
    np.savez_compressed(path, params=net.params(), widths=np.array(net.widths), cT=cT, meta=json.dumps(meta))


def load(path):
    d = np.load(path)
    net = ibm.UNet(tuple(int(x) for x in d["widths"]), 0)
    net.set_params(d["params"])
    return net, float(d["cT"]), json.loads(str(d["meta"]))
