"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances: fields within 1e-10 relative (||a - b||_inf / ||b||_inf per field)
and lift/drag within 1e-8 relative to the largest |C| of the history; node
kinds, forcing directions and sweep counts bit-exact.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2402_17337_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FIELD_TOL = 1e-10
FORCE_TOL = 1e-8


def gpu():
    from paper_2402_17337_gb300 import Solver, build
    build.build()
    return Solver


def rel(a, b):
    d = np.abs(a - b).max()
    s = np.abs(b).max()
    return d / s if s > 0 else d


def pair(cfg, **over):
    Solver = gpu()
    kw = dict(x0=cfg.x0, x1=cfg.x1, y0=cfg.y0, y1=cfg.y1, nx=cfg.nx, ny=cfg.ny, hmin=cfg.hmin,
              ubox=cfg.ubox, bc=cfg.bc, u_in=cfg.u_in, Re=cfg.Re, dt=cfg.dt, ptol=cfg.ptol,
              htol=cfg.htol, check_p=cfg.check_p, check_h=cfg.check_h, omega_p=cfg.omega(),
              omega_h=cfg.omega_h)
    kw.update(over)
    o = oracle.Sim(**kw)
    g = Solver(**kw)
    return o, g


def check_state(o, g, names=("u", "v", "p", "phi", "b", "uh", "vh", "Ru", "Rv", "Hu", "Hv", "q"),
                tol=FIELD_TOL):
    for n in names:
        a, b = g.get(n), o.get(n)
        assert rel(a, b) <= tol, (n, rel(a, b))


def check_flags(o, g):
    for grid in (0, 1):
        fo, do, ao = o.flags(grid)
        fg, dg, ag = g.flags(grid)
        assert np.array_equal(fo, fg), grid
        force = fo == 2
        assert np.array_equal(do[force], dg[force]), grid
        np.testing.assert_allclose(ag, ao, rtol=0, atol=1e-15)
    assert np.array_equal(o.flags(2), g.flags(2))


@pytest.mark.parametrize("case", ["plunging_uniform", "plunging_stretched", "stationary_stretched"])
def test_steps_match_oracle_small_grids(case):
    """Small grids, several thread tiles with ragged edges; the last case is
    the degenerate stationary foil (h = 0: no body velocity, fixed forcing
    nodes) in the free stream."""
    import dataclasses
    cfg = {"plunging_uniform": W.small_cases()[0], "plunging_stretched": W.small_cases()[1],
           "stationary_stretched": dataclasses.replace(W.small_cases()[1], h=0.0, k=0.0)}[case]
    o, g = pair(cfg)
    o.set_body(cfg.chord, cfg.tc, cfg.h, cfg.k, cfg.xc, cfg.yc)
    g.set_body(cfg.chord, cfg.tc, cfg.h, cfg.k, cfg.xc, cfg.yc)
    xo, yo = o.grid()
    xg, yg = g.grid()
    np.testing.assert_allclose(xg, xo, rtol=1e-15, atol=1e-15)
    np.testing.assert_allclose(yg, yo, rtol=1e-15, atol=1e-15)
    for n in range(cfg.steps):
        rc, so = o.step(1)
        assert rc == 0
        sg = g.step(1)
        for k in ("sweeps_u", "sweeps_v", "sweeps_p", "n"):
            assert so[k] == sg[k], (n, k, so[k], sg[k])
        check_flags(o, g)
        check_state(o, g)
        assert sg["div_max"] <= cfg.dt * cfg.ptol * (1 + 1e-9)
    clo, cdo = o.forces()
    clg, cdg = g.forces()
    scale = max(np.abs(clo).max(), np.abs(cdo).max())
    assert np.abs(clg - clo).max() <= FORCE_TOL * scale
    assert np.abs(cdg - cdo).max() <= FORCE_TOL * scale


def test_plunging_foil_192x128_100_steps_matches_oracle():
    """The 192x128 plunging-ellipse case (Re 300, h 0.25, k 2, dt 2e-3,
    100 steps, divergence 1e-10) end to end."""
    cfg = W.plunge_192x128()
    o, g = pair(cfg)
    o.set_body(cfg.chord, cfg.tc, cfg.h, cfg.k, cfg.xc, cfg.yc)
    g.set_body(cfg.chord, cfg.tc, cfg.h, cfg.k, cfg.xc, cfg.yc)
    sweeps_o, sweeps_g = [], []
    for n in range(cfg.steps):
        rc, so = o.step(1)
        assert rc == 0
        sg = g.step(1)
        sweeps_o.append(so["sweeps_p"])
        sweeps_g.append(sg["sweeps_p"])
        assert sg["div_max"] < cfg.div_tol
    assert sweeps_o == sweeps_g
    check_state(o, g, names=("u", "v", "p"))
    clo, cdo = o.forces()
    clg, cdg = g.forces()
    for a, b in ((clg, clo), (cdg, cdo)):
        assert np.abs(a - b).max() <= FORCE_TOL * np.abs(b).max()


def test_free_slip_box_taylor_green_matches_oracle():
    h = math.pi / 2
    kw = dict(x0=-h, x1=h, y0=-h, y1=h, nx=40, ny=40, bc=1, Re=100.0, dt=0.02, ptol=1e-11, check_p=4)
    Solver = gpu()
    o = oracle.Sim(**kw)
    g = Solver(**kw)
    xf, yf = o.grid()
    xc, yc = 0.5 * (xf[1:] + xf[:-1]), 0.5 * (yf[1:] + yf[:-1])
    Xu, Yu = np.meshgrid(xf, yc)
    Xv, Yv = np.meshgrid(xc, yf)
    Xp, Yp = np.meshgrid(xc, yc)
    u = -np.cos(Xu) * np.sin(Yu)
    v = np.sin(Xv) * np.cos(Yv)
    p = -0.25 * (np.cos(2 * Xp) + np.cos(2 * Yp))
    u[:, 0] = u[:, -1] = 0
    v[0, :] = v[-1, :] = 0
    for s in (o, g):
        s.set("u", u)
        s.set("v", v)
        s.set("p", p)
    rc, so = o.step(10)
    sg = g.step(10)
    assert rc == 0 and so["sweeps_p"] == sg["sweeps_p"]
    check_state(o, g, names=("u", "v", "p", "phi", "Hu", "Hv"))


def test_uniform_flow_without_body_is_preserved():
    cfg = W.small_cases()[1]
    Solver = gpu()
    g = Solver(x0=cfg.x0, x1=cfg.x1, y0=cfg.y0, y1=cfg.y1, nx=cfg.nx, ny=cfg.ny, hmin=cfg.hmin,
               ubox=cfg.ubox, Re=cfg.Re, dt=cfg.dt, ptol=1e-10)
    g.set("u", np.ones(g.shape("u")))
    st = g.step(4)
    assert np.abs(g.get("u") - 1).max() < 1e-13
    assert np.abs(g.get("v")).max() < 1e-13
    assert st["div_max"] < 1e-12


def test_poisson_solve_entry_point_matches_oracle():
    import torch
    Solver = gpu()
    for (nx, ny, hmin) in ((70, 45, 0.0), (133, 67, 0.09), (45, 160, 0.1)):
        kw = dict(x0=-7.5, x1=24.0, y0=-12.5, y1=12.5, nx=nx, ny=ny, hmin=hmin, ubox=(-1.0, 2.0, -0.8, 0.8),
                  dt=1.0)
        o = oracle.Sim(**kw)
        g = Solver(**kw)
        xf, yf = o.grid()
        V = np.outer(np.diff(yf), np.diff(xf))
        b = W.random_field((ny, nx), seed=nx * 7 + ny)
        b -= np.sum(b * V) / np.sum(V)
        phi0 = W.random_field((ny, nx), seed=5, scale=0.1)
        rc, phio, so, ro = o.poisson(b, phi0=phi0, tol=1e-9, check=8)
        assert rc == 0
        bd = torch.tensor(b, dtype=torch.float64, device="cuda").contiguous()
        pd = torch.tensor(phi0, dtype=torch.float64, device="cuda").contiguous()
        torch.cuda.synchronize()
        rc, sg, rg = g.poisson_solve(bd.data_ptr(), pd.data_ptr(), 1e-9, 8)
        assert rc == 0 and sg == so
        assert rel(pd.cpu().numpy(), phio) <= FIELD_TOL
        assert pd[0, nx - 1].item() == 0.0


def test_nan_rhs_reports_diverged_and_cap_reports_noconv():
    import torch
    Solver = gpu()
    g = Solver(x0=0.0, x1=1.0, y0=0.0, y1=1.0, nx=32, ny=32, dt=1.0)
    b = torch.zeros(32, 32, dtype=torch.float64, device="cuda")
    b[3, 4] = float("nan")
    phi = torch.zeros_like(b)
    torch.cuda.synchronize()
    rc, _, _ = g.poisson_solve(b.data_ptr(), phi.data_ptr(), 1e-8, 1, 10)
    assert rc == -4
    b = torch.tensor(W.random_field((32, 32), 2), device="cuda")
    b -= b.mean()
    torch.cuda.synchronize()
    rc, s, _ = g.poisson_solve(b.data_ptr(), phi.data_ptr(), 1e-14, 1, 3)
    assert rc == -3 and s == 3


@pytest.mark.parametrize("workload,precision", [("plunge_2048x1024", 0), ("plunge_2048x1024", 1),
                                                ("plunge_2048x1024", 2), ("plunge_4096x2048", 1)])
def test_full_size_step_properties(workload, precision):
    """At the full stretched sizes the oracle cannot run a step, so the GPU
    step is checked with the oracle's operators applied to the GPU's own
    fields: the explicit predictor, the velocity-system residuals, the
    right-hand side, the Poisson residual, the projection and the
    classification, at full size, for the plain FP64 path, the mixed path
    (the configuration bench.py times) and the multigrid variant."""
    cfg = getattr(W, workload)()
    Solver = gpu()
    kw = dict(x0=cfg.x0, x1=cfg.x1, y0=cfg.y0, y1=cfg.y1, nx=cfg.nx, ny=cfg.ny, hmin=cfg.hmin,
              ubox=cfg.ubox, Re=cfg.Re, dt=cfg.dt, ptol=cfg.ptol, htol=cfg.htol, check_p=cfg.check_p,
              check_h=cfg.check_h, omega_p=cfg.omega())
    g = Solver(**kw, precision=precision)
    g.set_body(cfg.chord, cfg.tc, cfg.h, cfg.k, cfg.xc, cfg.yc)
    o = oracle.Sim(**kw)
    o.set_body(cfg.chord, cfg.tc, cfg.h, cfg.k, cfg.xc, cfg.yc)
    xo, yo = o.grid()
    xg, yg = g.grid()
    assert np.array_equal(xo, xg) and np.array_equal(yo, yg)
    g.set("u", cfg.initial_u(g.shape("u")))
    g.step(2)  # leave the start behind
    u0, v0, p0 = g.get("u"), g.get("v"), g.get("p")
    Hu0, Hv0 = g.get("Hu"), g.get("Hv")
    st = g.step(1)
    dt, beta = cfg.dt, cfg.dt / (2 * cfg.Re)
    # explicit predictor from the GPU's state at t^n
    Hu, Hv = o.conv(u0, v0)
    gu, gv = o.grad(p0)
    Ru = u0 + dt * (-1.5 * Hu + 0.5 * Hu0 - gu) + beta * o.lap_u(u0)
    Rv = v0 + dt * (-1.5 * Hv + 0.5 * Hv0 - gv) + beta * o.lap_v(v0)
    assert rel(g.get("Hu")[:, 1:-1], Hu[:, 1:-1]) <= FIELD_TOL
    assert rel(g.get("Ru")[:, 1:-1], Ru[:, 1:-1]) <= FIELD_TOL
    assert rel(g.get("Rv")[1:-1, :], Rv[1:-1, :]) <= FIELD_TOL
    # classification at t^{n+1} against the oracle's
    o.classify(3 * dt)
    for grid in (0, 1):
        fo, do, ao = o.flags(grid)
        fg, dg, ag = g.flags(grid)
        assert np.array_equal(fo, fg)
        np.testing.assert_allclose(ag, ao, rtol=0, atol=1e-15)
    assert np.array_equal(o.flags(2), g.flags(2))
    # velocity systems: fluid-row residuals within the tolerance
    uh, vh = g.get("uh"), g.get("vh")
    fu = g.flags(0)[0]
    fv = g.flags(1)[0]
    ru = (Ru - (uh - beta * o.lap_u(uh)))[:, 1:-1][fu[:, 1:-1] == 0]
    rv = (Rv - (vh - beta * o.lap_v(vh)))[1:-1, :][fv[1:-1, :] == 0]
    assert np.abs(ru).max() <= cfg.htol * 1.5 + 1e-15 and np.abs(rv).max() <= cfg.htol * 1.5 + 1e-15
    vb = cfg.k * cfg.h * math.cos(cfg.k * 3 * dt)
    assert np.all(vh[fv == 1] == vb) and np.all(uh[fu == 1] == 0.0)
    # right-hand side and mass source
    D = o.div(uh, vh)
    q = g.get("q")
    body = g.flags(2).astype(bool)
    assert np.all(q[~body] == 0.0)
    np.testing.assert_allclose(g.get("b")[~body], D[~body] / dt, rtol=1e-12, atol=1e-9)
    xf, yf = xg, yg
    V = np.outer(np.diff(yf), np.diff(xf))
    assert abs(np.sum(q * V)) <= 1e-12 * max(1.0, np.abs(D).max())
    # pressure solve and projection
    phi = g.get("phi")
    b = g.get("b")
    assert np.abs(b - o.lap_p(phi)).max() <= cfg.ptol * 1.01
    gu, gv = o.grad(phi)
    u1, v1 = g.get("u"), g.get("v")
    assert rel(u1[:, 1:-1], (uh - dt * gu)[:, 1:-1]) <= FIELD_TOL
    assert rel(v1[1:-1, :], (vh - dt * gv)[1:-1, :]) <= FIELD_TOL
    d1 = o.div(u1, v1)
    assert np.abs(d1[~body]).max() <= cfg.div_tol
    assert abs(np.abs(d1[~body]).max() - st["div_max"]) <= 1e-15 + 1e-9 * st["div_max"]


def test_tallest_grid_step_properties():
    """ny = 8192, the largest the ordered outflow-flux sums accept (256
    chunks of 32 rows), on a tall uniform 64x8192 grid with the foil at the
    centre, mixed path: after a step from the free stream the outflow flux
    equals the inflow flux, the pressure residual (the oracle's operator on
    the GPU's fields) is below the tolerance and the fluid-cell divergence
    below div_tol."""
    import dataclasses
    Solver = gpu()
    cfg = dataclasses.replace(W.plunge_192x128(), name="tall_64x8192", x0=-4.0, x1=4.0, y0=-512.0, y1=512.0,
                              nx=64, ny=8192, dt=2e-3, div_tol=1e-8, init="uniform")
    kw = dict(x0=cfg.x0, x1=cfg.x1, y0=cfg.y0, y1=cfg.y1, nx=cfg.nx, ny=cfg.ny, hmin=cfg.hmin, ubox=cfg.ubox,
              Re=cfg.Re, dt=cfg.dt, ptol=cfg.ptol, htol=cfg.htol, check_p=cfg.check_p, check_h=cfg.check_h,
              omega_p=cfg.omega())
    g = Solver(**kw, precision=1)
    g.set_body(cfg.chord, cfg.tc, cfg.h, cfg.k, cfg.xc, cfg.yc)
    g.set("u", cfg.initial_u(g.shape("u")))
    st = g.step(1)
    xf, yf = g.grid()
    dy = np.diff(yf)
    u = g.get("u")
    q_in, q_out = np.sum(u[:, 0] * dy), np.sum(u[:, -1] * dy)
    assert abs(q_out - q_in) <= 1e-12 * abs(q_in)
    o = oracle.Sim(**kw)
    phi, b = g.get("phi"), g.get("b")
    assert np.abs(b - o.lap_p(phi)).max() <= cfg.ptol * 1.01
    body = g.flags(2).astype(bool)
    d = o.div(u, g.get("v"))
    assert np.abs(d[~body]).max() <= cfg.div_tol and st["div_max"] <= cfg.div_tol
