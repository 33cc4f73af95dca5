"""Learned warm start: the recorded training samples against a recomputation
from the solver's fields, what a trained network gains over the plain warm
start (previous increment) on held-out steps and that a rejected guess costs
no sweeps, and why any warm start saves little on red-black SOR."""
import numpy as np
import pytest

import oracle
from paper_2402_17337_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def small_cfg():
    return W.FlowConfig("plunge_256x128", -7.5, 24.0, -12.5, 12.5, 256, 128, 0.04, Re=500.0, dt=0.01, steps=60,
                        h=0.25, k=2.0, div_tol=1e-8, init="uniform", check_p=8)


def coarse(a):
    return 0.25 * (a[0::2, 0::2] + a[0::2, 1::2] + a[1::2, 0::2] + a[1::2, 1::2])


@pytest.mark.parametrize("precision", [0, 1])
def test_samples_match_recomputation_from_fields(precision):
    import paper_2402_17337_gb300 as ibm
    from paper_2402_17337_gb300 import build
    build.build()
    cfg = small_cfg()
    s = ibm.Solver.from_config(cfg, precision=precision)
    s.set("u", cfg.initial_u(s.shape("u")))
    s.set_warmstart(2, None, 1.0)
    s.step(4)
    phi_n, p_n = s.get("phi"), s.get("p")
    s.step(1)
    b, phi_1 = s.get("b"), s.get("phi")
    body = s.flags(2).astype(np.float64)
    f, t = s.sample()
    o = oracle.Sim(x0=cfg.x0, x1=cfg.x1, y0=cfg.y0, y1=cfg.y1, nx=cfg.nx, ny=cfg.ny, hmin=cfg.hmin,
                   ubox=cfg.ubox, dt=cfg.dt)
    r0 = b - o.lap_p(phi_n)
    feats = [coarse(r0), coarse(b), coarse(body), coarse(p_n)]
    for ch in (0, 1, 3):
        feats[ch] = feats[ch] / np.abs(feats[ch]).max()
    for ch in range(4):
        np.testing.assert_allclose(f[..., ch], feats[ch], rtol=0, atol=1e-5 * max(1.0, np.abs(feats[ch]).max()))
    s0 = np.abs(coarse(r0)).max()
    ref = coarse(phi_1 - phi_n) / s0
    np.testing.assert_allclose(t, ref, rtol=0, atol=1e-5 * np.abs(ref).max())


def test_trained_network_gain_over_plain_warm_start():
    """Trains a small U-Net on samples of steps 5..44 and compares pressure
    sweeps with the plain warm start on steps 45..59 (held out)."""
    import paper_2402_17337_gb300 as ibm
    from paper_2402_17337_gb300 import build, warmstart
    build.build()
    cfg = small_cfg()
    samples = warmstart.capture(cfg, steps=45, start=5, every=1)
    net = ibm.UNet((16, 32, 32, 48), seed=1)
    cT, hist = warmstart.train(net, samples, epochs=30, lr=2e-3)
    # the weight-gradient kernel accumulates with atomics, so loss histories differ from run to
    # run; the property checked is that training reduces the loss clearly
    assert min(hist[-5:]) < 0.75 * hist[0], hist
    res = warmstart.evaluate(cfg, net, cT, steps=15, start=45)
    plain, learned = sum(res["plain"]["sweeps"]), sum(res["learned"]["sweeps"])
    print(f"held-out pressure sweeps: plain {plain}, learned {learned}, gain {1 - learned / plain:+.1%}; "
          f"loss {hist[0]:.3e} -> {hist[-1]:.3e}")
    # the learned start must not cost sweeps on the held-out steps
    assert learned <= 1.02 * plain, res
    # a guess the residual test rejects leaves the plain guess in place: until a
    # guess is kept the two runs take the same iterates and the same sweeps
    first_kept = next((k for k, x in enumerate(res["learned"]["kept"]) if x), len(res["learned"]["kept"]))
    assert res["learned"]["sweeps"][:first_kept] == res["plain"]["sweeps"][:first_kept], res


def test_sweeps_saved_by_a_warm_start_grow_with_the_log_of_its_accuracy():
    """Why a warm start, learned or not, saves little on red-black SOR: near
    the optimal factor every error component decays at about the same rate per
    sweep, so a start within relative error eps of the exact increment (the
    increment a first solve of the same step found, times 1 - eps) saves about
    log(1/eps) / |log rate| sweeps, a number that grows with the logarithm of
    the accuracy.  Measured over three steps of the 256x128 case: the savings
    at eps = 0.5, 0.1, 0.01 increase, and the step from 0.1 to 0.01 saves
    log(10)/log(5) = 1.43 times the step from 0.5 to 0.1 (within 1.0 .. 2.0)."""
    import dataclasses

    import paper_2402_17337_gb300 as ibm
    from paper_2402_17337_gb300 import build
    build.build()
    cfg = dataclasses.replace(small_cfg(), check_p=2)
    s = ibm.Solver.from_config(cfg, precision=0)
    s.set("u", cfg.initial_u(s.shape("u")))
    s.step(20)
    eps = (0.5, 0.1, 0.01)
    saved = {e: [] for e in eps}
    for _ in range(3):
        state = s.save_state()
        phi0 = s.get("phi")
        n0 = s.step(1)["sweeps_p"]
        d = s.get("phi") - phi0
        for e in eps:
            s.load_state(state)
            s.set("phi", phi0 + (1.0 - e) * d)
            saved[e].append(n0 - s.step(1)["sweeps_p"])
        s.load_state(state)
        s.step(1)
    m = {e: float(np.mean(saved[e])) for e in eps}
    print("sweeps saved by a start within eps of the exact increment:", m)
    assert 0 < m[0.5] < m[0.1] < m[0.01], m
    ratio = (m[0.01] - m[0.1]) / (m[0.1] - m[0.5])
    assert 1.0 <= ratio <= 2.0, (m, ratio)
