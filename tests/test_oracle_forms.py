"""The oracle's arithmetic recipe against its textbook form (CPU only).

The oracle computes the scheme (Sec. 2.2 operators and fractional step,
Sec. 2.3 grid, Sec. 3.1 red-black SOR) in one arithmetic recipe that the
GPU path shares: divisions by grid spacings as products with stored
reciprocals, five-point operators as fused multiply-add chains in the order
E, W, N, S, and two-level feedback sums.  The same source compiled with
-DORACLE_PLAIN computes everything in the textbook form: flux differences
divided by the spacings, every product and sum rounded on its own, SOR
updates as (1 - omega) x + omega GS with the Gauss-Seidel value divided by
the diagonal, one-pass sums.  The two forms are the same mathematics, so
they must agree to rounding operator by operator, within the bound the
stopping rule allows for the solves, and within the GPU path's own parity
tolerances over whole steps; and the textbook form must pass the pins the
recipe passes.  A slip common to the recipe's two implementations (oracle
and kernels) would break one of these.
"""
import numpy as np
import pytest

import oracle
import test_oracle_mutants as mutants
from paper_2402_17337_gb300 import workloads as W


def _forms():
    return {"recipe": oracle.build(), "plain": oracle.build_plain()}


def _stretched(nx=97, ny=61):
    return dict(x0=-7.5, x1=24.0, y0=-12.5, y1=12.5, nx=nx, ny=ny, hmin=0.08 * 97 / nx,
                ubox=(-1.0, 2.0, -0.8, 0.8), Re=500.0, dt=5e-3)


def test_operators_agree_to_rounding():
    """Every discrete operator on random fields of a stretched grid: the two
    forms differ by a few roundings of the largest term, i.e. <= 1e-14 of the
    result's maximum (measured: <= 2.2e-16)."""
    out = {}
    for name, path in _forms().items():
        with oracle.use_library(path):
            s = oracle.Sim(**_stretched())
            u = W.random_field(s.shape("u"), 1)
            v = W.random_field(s.shape("v"), 2)
            p = W.random_field(s.shape("p"), 3)
            Hu, Hv = s.conv(u, v)
            gu, gv = s.grad(p)
            out[name] = {"lap_p": s.lap_p(p), "lap_u": s.lap_u(u), "lap_v": s.lap_v(v), "conv_u": Hu,
                         "conv_v": Hv, "grad_u": gu, "grad_v": gv, "div": s.div(u, v)}
    for op, a in out["recipe"].items():
        b = out["plain"][op]
        assert np.abs(a - b).max() <= 1e-14 * np.abs(a).max(), op


def _gauged_inverse_norm(s):
    """||A'^{-1}||_inf of the pressure operator with the gauge cell's row
    replaced by phi_g = 0 (dense, tiny grids).  For a compatible residual r
    (volume-weighted sum zero, which b - L_p phi always is) the gauged
    correction solves A' e = r with r_g set to 0, so ||e|| <= ||A'^{-1}|| ||r||."""
    ny, nx = s.shape("p")
    n = nx * ny
    A = np.zeros((n, n))
    for k in range(n):
        e = np.zeros(n)
        e[k] = 1.0
        A[:, k] = s.lap_p(e.reshape(ny, nx)).ravel()
    g = 0 * nx + (nx - 1)  # cell (nx-1, 0)
    A[g, :] = 0.0
    A[g, g] = 1.0
    return np.abs(np.linalg.inv(A)).sum(axis=1).max()


def test_poisson_solves_agree_within_the_stopping_bound():
    """Both forms solve L_p phi = b (compatible random b, stretched grid) until
    ||b - L_p phi||_inf <= tol and fix the same gauge.  The two solutions then
    differ by at most ||A'^{-1}|| (r_recipe + r_plain)."""
    tol = 1e-9
    sol = {}
    for name, path in _forms().items():
        with oracle.use_library(path):
            s = oracle.Sim(**_stretched(33, 21))
            xf, yf = s.grid()
            V = np.outer(np.diff(yf), np.diff(xf))
            b = W.random_field(s.shape("p"), 4)
            b -= (b * V).sum() / V.sum()
            rc, phi, sweeps, res = s.poisson(b, tol=tol, check=1)
            assert rc == 0 and res <= tol
            sol[name] = (phi, res)
            if name == "recipe":
                bound_norm = _gauged_inverse_norm(s)
    (pa, ra), (pb, rb) = sol["recipe"], sol["plain"]
    assert np.abs(pa - pb).max() <= bound_norm * (ra + rb)


@pytest.mark.parametrize("case", ["plunge_192x128", "plunge_97x61_stretched"])
def test_whole_steps_agree_within_the_parity_tolerances(case):
    """The workloads' own steps (plunging ellipse, Sec. 2.1; 192x128 uniform for
    20 steps and the stretched parity grid for 5): u, v, p within 1e-10 and the
    C_l, C_d histories within 1e-8 relative, the tolerances the GPU path is held
    to against the oracle, so the choice of arithmetic recipe is not what
    decides a parity test.  Sweep counts may differ by a few check intervals
    (the stopping test compares a residual near its rounding floor)."""
    if case == "plunge_192x128":
        c, n = W.plunge_192x128(), 20
    else:
        c = [x for x in W.small_cases() if x.name == case][0]
        n = c.steps
    res = {}
    for name, path in _forms().items():
        with oracle.use_library(path):
            s = oracle.Sim(x0=c.x0, x1=c.x1, y0=c.y0, y1=c.y1, nx=c.nx, ny=c.ny, hmin=c.hmin, ubox=c.ubox,
                           bc=c.bc, Re=c.Re, dt=c.dt, ptol=c.ptol, htol=c.htol, check_p=c.check_p,
                           check_h=c.check_h, omega_p=c.omega(), threads=4)
            s.set_body(c.chord, c.tc, c.h, c.k, c.xc, c.yc)
            s.set("u", c.initial_u(s.shape("u")))
            sweeps = []
            for _ in range(n):
                rc, st = s.step(1)
                assert rc == 0
                sweeps.append(st["sweeps_p"])
            res[name] = ({f: s.get(f) for f in ("u", "v", "p")}, s.forces(), np.array(sweeps))
    (fa, (cla, cda), sa), (fb, (clb, cdb), sb) = res["recipe"], res["plain"]
    for f in ("u", "v", "p"):
        assert np.abs(fa[f] - fb[f]).max() <= 1e-10 * np.abs(fa[f]).max(), f
    assert np.abs(cla - clb).max() <= 1e-8 * np.abs(cla).max()
    assert np.abs(cda - cdb).max() <= 1e-8 * np.abs(cda).max()
    assert np.all(np.abs(sa - sb) <= 0.1 * sa)


def test_textbook_form_passes_the_pins():
    """The pins of every part of the step (the table of planted mistakes in
    test_oracle_mutants names one per part) hold for the textbook form too."""
    with oracle.use_library(oracle.build_plain()):
        for pin, args in mutants.unique_pins():
            pin(*args)
