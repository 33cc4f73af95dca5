"""Multigrid variant of the pressure solve (precision 2: FP32 V-cycles inside
the FP64 defect correction) against the FP64 oracle.

The variant stops at the same FP64 residual tolerance as the oracle's SOR
(the paper's solver), so the solutions agree to the algebraic error of the
two solves, ||L^-1|| times the two residuals, and the fields of whole steps
to the same bound as the SOR mixed path."""
import numpy as np
import pytest

import oracle
from paper_2402_17337_gb300 import workloads as W

pytestmark = pytest.mark.gpu

MIXED_TOL = 1e-6


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def kwargs(cfg):
    return dict(x0=cfg.x0, x1=cfg.x1, y0=cfg.y0, y1=cfg.y1, nx=cfg.nx, ny=cfg.ny, hmin=cfg.hmin,
                ubox=cfg.ubox, bc=cfg.bc, u_in=cfg.u_in, Re=cfg.Re, dt=cfg.dt, ptol=cfg.ptol,
                htol=cfg.htol, check_p=cfg.check_p, check_h=cfg.check_h, omega_p=cfg.omega(),
                omega_h=cfg.omega_h)


@pytest.mark.parametrize("nx,ny,hmin", [(70, 45, 0.0), (261, 133, 0.06), (517, 263, 0.05), (1024, 512, 0.01)])
def test_mg_poisson_solve_matches_oracle(nx, ny, hmin):
    import torch
    from paper_2402_17337_gb300 import Solver, build
    build.build()
    kw = dict(x0=-7.5, x1=24.0, y0=-12.5, y1=12.5, nx=nx, ny=ny, hmin=hmin, ubox=(-1.0, 2.0, -0.8, 0.8), dt=1.0)
    o = oracle.Sim(**kw, threads=8)
    g = Solver(**kw, precision=2)
    xf, yf = o.grid()
    V = np.outer(np.diff(yf), np.diff(xf))
    b = W.random_field((ny, nx), seed=3 * nx + ny)
    b -= np.sum(b * V) / np.sum(V)
    tol = 1e-9 * np.abs(b).max()
    rc, phio, so, ro = o.poisson(b, tol=tol, check=8, maxs=2000000)
    assert rc == 0
    bd = torch.tensor(b, device="cuda")
    pd = torch.zeros_like(bd)
    torch.cuda.synchronize()
    rc, cycles, rg = g.poisson_solve(bd.data_ptr(), pd.data_ptr(), tol, 0, 2000)
    assert rc == 0 and rg <= tol
    print(f"{nx}x{ny}: oracle SOR {so} sweeps, multigrid {cycles} V-cycles")
    # both residuals <= tol: the solutions differ by at most ||L^-1|| * 2 tol
    xc = 0.5 * (xf[1:] + xf[:-1])
    inv_bound = 2.0 * (xf[-1] - xf[0]) ** 2  # ||L^-1||_inf on mean-free data, generous
    d = pd.cpu().numpy() - phio
    d -= d[0, -1]  # both gauges pin cell (nx-1, 0)
    assert np.abs(d).max() <= inv_bound * 2 * tol
    # a V-cycle costs a few fine sweeps; it must replace many more SOR sweeps
    assert cycles <= so / 8, (cycles, so)


@pytest.mark.parametrize("idx", [0, 1])
def test_mg_steps_match_fp64_oracle(idx):
    from paper_2402_17337_gb300 import Solver, build
    build.build()
    cfg = W.small_cases()[idx]
    o = oracle.Sim(**kwargs(cfg))
    g = Solver(**kwargs(cfg), precision=2)
    for s in (o, g):
        s.set_body(cfg.chord, cfg.tc, cfg.h, cfg.k, cfg.xc, cfg.yc)
    for n in range(cfg.steps):
        rc, so = o.step(1)
        assert rc == 0
        sg = g.step(1)
        assert sg["res_p"] <= cfg.ptol and sg["div_max"] <= cfg.div_tol * 1.001
    errs = {n: rel(g.get(n), o.get(n)) for n in ("u", "v", "p")}
    print("multigrid vs fp64 oracle, per-field relative error:", errs)
    assert max(errs.values()) <= MIXED_TOL, errs


def test_unet_two_level_preconditioner_meets_the_same_tolerance():
    """The U-Net as the coarse level of the FCG preconditioner (random
    weights, their output scaled small: whatever the network predicts, the
    FP64 defect correction stops at the same residual), two steps on a
    uniform 128x64 grid against the FP64 oracle, to the bound of the other
    FP32 paths.  Without a coarse hierarchy the iteration count grows with
    the grid, hence the small uniform case; without pre-smoothing (with it,
    the FCG(1) iteration stalled near 1e-5 on this case)."""
    pre_smooth = 0
    import dataclasses
    from paper_2402_17337_gb300 import Solver, UNet, build
    build.build()
    c = dataclasses.replace(W.plunge_192x128(), name="uniform_128x64", x0=-4.0, x1=8.0, y0=-3.0, y1=3.0, nx=128,
                            ny=64, steps=2, div_tol=1e-8)
    o = oracle.Sim(**kwargs(c))
    o.set_body(c.chord, c.tc, c.h, c.k, c.xc, c.yc)
    o.set("u", c.initial_u(o.shape("u")))
    rc, _ = o.step(2)
    assert rc == 0
    net = UNet((16, 16, 32, 32), seed=3)
    g = Solver(**kwargs(c), precision=2, max_sweeps=20000)
    g.set_body(c.chord, c.tc, c.h, c.k, c.xc, c.yc)
    g.set("u", c.initial_u(g.shape("u")))
    g.set_preconditioner(1, net, 1e-4, pre_smooth)
    st = g.step(2)
    assert st["res_p"] <= c.ptol and st["div_max"] <= c.div_tol * 1.001, st
    errs = {n: rel(g.get(n), o.get(n)) for n in ("u", "v", "p")}
    print(f"two-level U-Net preconditioner (pre-smoothing {pre_smooth}): {st['sweeps_p']} FCG iterations, "
          f"errors {errs}")
    assert max(errs.values()) <= MIXED_TOL, errs
    g.close()
    net.close()


def test_unet_preconditioner_with_pre_smoothing_never_returns_a_step_that_misses_the_tolerance():
    """The configuration in which the real use fails: with pre-smoothing the
    two-level cycle is no longer symmetric and the network's coarse correction
    belongs to another residual, and FCG(1) stalls (near 1e-5 on this case
    over two steps; every trained network stalled it on the bench grids).
    Whatever the iteration does, a step either meets the residual and
    divergence tolerances or ends with IBM_E_NOCONV at its iteration cap:
    never fields that miss the tolerance."""
    import dataclasses
    from paper_2402_17337_gb300 import IBM_E_NOCONV, IbmError, Solver, UNet, build
    build.build()
    c = dataclasses.replace(W.plunge_192x128(), name="uniform_128x64", x0=-4.0, x1=8.0, y0=-3.0, y1=3.0, nx=128,
                            ny=64, steps=2, div_tol=1e-8)
    net = UNet((16, 16, 32, 32), seed=3)
    g = Solver(**kwargs(c), precision=2, max_sweeps=1500)
    g.set_body(c.chord, c.tc, c.h, c.k, c.xc, c.yc)
    g.set("u", c.initial_u(g.shape("u")))
    g.set_preconditioner(1, net, 1e-4, 1)
    outcome = []
    for _ in range(c.steps):
        try:
            st = g.step(1)
        except IbmError as e:
            assert e.code == IBM_E_NOCONV, e
            outcome.append("NOCONV")
            break
        assert st["res_p"] <= c.ptol and st["div_max"] <= c.div_tol * 1.001, st
        outcome.append(st["sweeps_p"])
    print("two-level U-Net preconditioner with pre-smoothing:", outcome)
    g.close()
    net.close()


def test_preconditioner_rejects_invalid_use():
    from paper_2402_17337_gb300 import IbmError, Solver, UNet, build
    build.build()
    c = W.batch_small(1)[0]
    net = UNet((16, 16, 32, 32), seed=3)
    for precision, kind, nn, pre in ((1, 1, net, 1), (2, 2, net, 1), (2, 1, None, 1), (2, 1, net, 2)):
        s = Solver(**kwargs(c), precision=precision)
        with pytest.raises(IbmError) as e:
            s.set_preconditioner(kind, nn, 1.0, pre)
        assert e.value.code == -1
        s.close()
    odd = dict(kwargs(W.small_cases()[1]))
    s = Solver(**odd, precision=2)
    with pytest.raises(IbmError):
        s.set_preconditioner(1, net, 1.0, 1)
    s.set_preconditioner(0)  # the V-cycle is always available
    s.close()
    net.close()


def test_mg_full_size_steps_agree_with_sor_mixed_path():
    """Two steps of the 2048x1024 workload: divergence below 1e-8 and the same
    fields, to the solve tolerance, as the SOR mixed path."""
    from paper_2402_17337_gb300 import Solver, build
    build.build()
    cfg = W.plunge_2048x1024()
    runs = {}
    for prec in (1, 2):
        s = Solver.from_config(cfg, precision=prec)
        s.set("u", cfg.initial_u(s.shape("u")))
        st = s.step(2)
        assert st["div_max"] <= cfg.div_tol * 1.001, (prec, st)
        runs[prec] = ({f: s.get(f) for f in ("u", "v")}, st)
        s.close()
    errs = {f: rel(runs[2][0][f], runs[1][0][f]) for f in ("u", "v")}
    print("multigrid vs SOR (mixed):", errs, "V-cycles", runs[2][1]["sweeps_p"], "SOR sweeps", runs[1][1]["sweeps_p"])
    assert max(errs.values()) <= MIXED_TOL
