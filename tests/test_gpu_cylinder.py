"""Stationary circular cylinder at Re = 100 (ellipse of thickness ratio 1,
no plunge): a physical check of the whole step.

The GPU step matches the FP64 oracle step for step on a small stretched
cylinder grid (same pressure sweep counts, fields to 1e-10), and the shedding
run on the 320x256 grid gives a Strouhal number between 0.16 and 0.17, the
range measured for this Reynolds number, with the mean drag coefficient and
the lift amplitude near their measured values (about 1.33-1.40 and 0.3)."""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_2402_17337_gb300 import cylinder

pytestmark = pytest.mark.gpu


def kwargs(cfg):
    return dict(x0=cfg.x0, x1=cfg.x1, y0=cfg.y0, y1=cfg.y1, nx=cfg.nx, ny=cfg.ny, hmin=cfg.hmin,
                ubox=cfg.ubox, bc=cfg.bc, u_in=cfg.u_in, Re=cfg.Re, dt=cfg.dt, ptol=cfg.ptol,
                htol=cfg.htol, check_p=cfg.check_p, check_h=cfg.check_h, omega_p=cfg.omega(),
                omega_h=cfg.omega_h)


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def test_cylinder_steps_match_oracle():
    from paper_2402_17337_gb300 import Solver, build
    build.build()
    cfg = dataclasses.replace(cylinder.CONFIG, name="cylinder_128x96", nx=128, ny=96, hmin=0.08, dt=0.02)
    o = oracle.Sim(**kwargs(cfg))
    g = Solver(**kwargs(cfg))
    xf, yf = o.grid()
    v0 = cylinder.perturbation(xf, yf)
    for s in (o, g):
        s.set_body(cfg.chord, cfg.tc, cfg.h, cfg.k, cfg.xc, cfg.yc)
        s.set("u", cfg.initial_u(s.shape("u")))
        s.set("v", v0)
    for n in range(6):
        rc, so = o.step(1)
        assert rc == 0
        sg = g.step(1)
        assert so["sweeps_p"] == sg["sweeps_p"], (n, so["sweeps_p"], sg["sweeps_p"])
        for f in ("u", "v", "p"):
            assert rel(g.get(f), o.get(f)) <= 1e-10, (n, f)
    clo, cdo = o.forces()
    clg, cdg = g.forces()
    scale = max(np.abs(clo).max(), np.abs(cdo).max())
    assert np.abs(clg - clo).max() <= 1e-8 * scale and np.abs(cdg - cdo).max() <= 1e-8 * scale


def test_cylinder_re100_strouhal_number():
    from paper_2402_17337_gb300 import Solver, build
    build.build()
    probe = Solver.from_config(cylinder.CONFIG, precision=1)
    cfg = dataclasses.replace(cylinder.CONFIG, omega_p=probe.tune_omega())
    probe.close()
    res = cylinder.run(cfg, t_end=100.0, window=40.0, precision=1)
    print(res)
    assert res["max_step_div"] <= cfg.div_tol
    assert res["up_crossings"] >= 5 and res["cl_amplitude"] > 0.2, res  # shedding established
    assert 0.16 <= res["strouhal"] <= 0.17, res
    assert 1.25 <= res["cd_mean"] <= 1.45, res
