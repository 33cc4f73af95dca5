"""Batch of cases with uneven grids advancing together (ibm_batch_*).

Every case of a batch is checked against the FP64 oracle stepping that case
alone (same bound as the single-context mixed path: the solves stop at the
same residual tolerance by different iterates), CUDA-graph replay against
direct launches (identical launches, so identical bits), and, at the full
batch sizes, the properties that hold at any size: every case's divergence
below its tolerance and agreement with the same case stepped alone.
"""
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


def solvers(cfgs):
    from paper_2402_17337_gb300 import Solver
    out = []
    for c in cfgs:
        s = Solver.from_config(c, precision=1)
        s.set("u", c.initial_u(s.shape("u")))
        out.append(s)
    return out


def test_batch_cases_match_fp64_oracle():
    from paper_2402_17337_gb300 import Batch, build
    build.build()
    cfgs = W.batch_small(4)
    ss = solvers(cfgs)
    B = Batch(ss)
    steps = cfgs[0].steps
    for n in range(steps):
        st = B.step(1)
        for c, x in zip(cfgs, st):
            assert x["n"] == n + 1
            assert x["res_p"] <= c.ptol and x["div_max"] <= c.div_tol * 1.001, (c.name, x)
    for c, s in zip(cfgs, ss):
        o = oracle.Sim(**kwargs(c))
        o.set_body(c.chord, c.tc, c.h, c.k, c.xc, c.yc)
        o.set("u", c.initial_u(s.shape("u")))
        for _ in range(steps):
            rc, _ = o.step(1)
            assert rc == 0
        errs = {f: rel(s.get(f), o.get(f)) for f in ("u", "v", "p")}
        print(c.name, c.nx, c.ny, "batch vs fp64 oracle:", errs)
        assert max(errs.values()) <= MIXED_TOL, (c.name, errs)
        clo, cdo = o.forces()
        clg, cdg = s.forces()
        assert np.abs(clg - clo).max() <= 1e-4 * np.abs(clo).max(), c.name
        assert np.abs(cdg - cdo).max() <= 1e-4 * np.abs(cdo).max(), c.name
    prof = B.profile()
    assert prof["steps"] == steps and prof["sor_shape"][0] > 0
    B.close()


def test_graph_replay_is_bit_identical_to_direct_launches():
    from paper_2402_17337_gb300 import Batch, build
    build.build()
    cfgs = W.batch_small(5, seed=7)
    runs = []
    for graphs in (True, False):
        ss = solvers(cfgs)
        B = Batch(ss)
        B.set_budgets(False)  # shared rounds: the sweeps graph replay covers
        B.set_graphs(graphs)
        B.set_sor_shape(0)  # the same tile shape in both runs (the autotuner may pick either)
        st = B.step(3)
        runs.append(([s.get("p") for s in ss], [s.get("u") for s in ss], [x["sweeps_p"] for x in st]))
        B.close()
    (p1, u1, s1), (p2, u2, s2) = runs
    assert s1 == s2
    for a, b in zip(p1 + u1, p2 + u2):
        assert np.array_equal(a, b)


def test_sweep_budgets_and_shared_rounds_reach_the_same_tolerance():
    """With sweep budgets (each case its own sweeps per round) and with shared
    rounds the checks fall after different sweeps, so the iterates differ,
    but every case meets the same residual and divergence tolerances and the
    fields agree within the mixed-path bound."""
    from paper_2402_17337_gb300 import Batch, build
    build.build()
    cfgs = W.batch_small(4, seed=11)
    runs = []
    for budgets in (True, False):
        ss = solvers(cfgs)
        B = Batch(ss)
        B.set_budgets(budgets)
        st = B.step(3)
        for c, x in zip(cfgs, st):
            assert x["res_p"] <= c.ptol and x["div_max"] <= c.div_tol * 1.001, (c.name, budgets, x)
        runs.append([{f: s.get(f) for f in ("u", "v", "p")} for s in ss])
        B.close()
    for a, b in zip(*runs):
        for f in ("u", "v", "p"):
            assert rel(a[f], b[f]) <= MIXED_TOL, f


def test_batch_rejects_invalid_cases():
    from paper_2402_17337_gb300 import Batch, IbmError, Solver, build
    build.build()
    c = W.batch_small(1)[0]
    s64 = Solver.from_config(c, precision=0)
    with pytest.raises(IbmError) as e:
        Batch([s64])
    assert e.value.code == -1
    s = Solver.from_config(c, precision=1)
    with pytest.raises(IbmError) as e:
        Batch([s, s])
    assert e.value.code == -1


def test_full_size_batch_cases_agree_with_single_context_runs():
    """Eight cases of the 64-case batch at their full grids (512x256 ..
    1536x768), two steps: divergence below 1e-8 in every case and the same
    fields, to the solve tolerance, as each case stepped alone."""
    from paper_2402_17337_gb300 import Batch, build
    build.build()
    cfgs = W.batch64()[:8]
    ss = solvers(cfgs)
    B = Batch(ss)
    st = B.step(2)
    for c, x in zip(cfgs, st):
        assert x["div_max"] <= c.div_tol * 1.001, (c.name, x)
    for c, s in zip(cfgs, ss):
        (alone,) = solvers([c])
        a = alone.step(2)
        assert a["div_max"] <= c.div_tol * 1.001
        errs = {f: rel(s.get(f), alone.get(f)) for f in ("u", "v")}
        print(c.name, c.nx, c.ny, "batch vs alone:", errs, "sweeps", a["sweeps_p"])
        assert max(errs.values()) <= MIXED_TOL, (c.name, errs)
        alone.close()
    B.close()


def test_fused_batch_step_matches_single_contexts_bit_for_bit_before_the_pressure_solve():
    """A batch step runs classification, boundary values, predictor, velocity
    solves, right-hand side, forces and projection as shared launches over
    all cases.  Up to the pressure solve a case's arithmetic is that of the
    single-context step, so after one step from the same state the
    intermediate velocities and right-hand sides (uh, vh, R_u, R_v), the
    node kinds and the forces (computed from those) are equal bit for bit,
    and so are the velocity sweep counts.  Small cases of the batch recipe
    and two full-size cases with ragged tiles."""
    from paper_2402_17337_gb300 import Batch, build
    build.build()
    cfgs = W.batch_small(4) + W.batch64()[:2]
    ss = solvers(cfgs)
    B = Batch(ss)
    st = B.step(1)
    for c, s, x in zip(cfgs, ss, st):
        (alone,) = solvers([c])
        a = alone.step(1)
        assert (x["sweeps_u"], x["sweeps_v"]) == (a["sweeps_u"], a["sweeps_v"]), c.name
        for f in ("uh", "vh", "Ru", "Rv"):
            assert np.array_equal(s.get(f), alone.get(f)), (c.name, f)
        for grid in (0, 1, 2):
            fa, fb = s.flags(grid), alone.flags(grid)
            for ka, kb in zip(fa if isinstance(fa, tuple) else (fa,), fb if isinstance(fb, tuple) else (fb,)):
                assert np.array_equal(ka, kb), (c.name, grid)
        (cl, cd), (cl0, cd0) = s.forces(), alone.forces()
        assert np.array_equal(cl, cl0) and np.array_equal(cd, cd0), c.name
        assert x["div_max"] <= c.div_tol * 1.001
        alone.close()
    B.close()
