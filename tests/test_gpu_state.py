"""Checkpoint and resume (ibm_state_bytes / ibm_save_state / ibm_load_state).

A context that loads a state saved after n steps and steps on repeats the
saved run's later steps bit for bit (fields, pressure increment, C_l/C_d
histories), for the plain FP64 path and the FP32-in-FP64 path; a state is
refused by a context of another grid or without the same body, and a
truncated or foreign buffer is refused."""
import numpy as np
import pytest

from paper_2402_17337_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def kwargs(cfg):
    return dict(x0=cfg.x0, x1=cfg.x1, y0=cfg.y0, y1=cfg.y1, nx=cfg.nx, ny=cfg.ny, hmin=cfg.hmin,
                ubox=cfg.ubox, bc=cfg.bc, u_in=cfg.u_in, Re=cfg.Re, dt=cfg.dt, ptol=cfg.ptol,
                htol=cfg.htol, check_p=cfg.check_p, check_h=cfg.check_h, omega_p=cfg.omega(),
                omega_h=cfg.omega_h)


@pytest.mark.parametrize("precision", [0, 1])
def test_resume_repeats_the_run_bit_for_bit(precision):
    from paper_2402_17337_gb300 import Solver, build
    build.build()
    cfg = W.small_cases()[1]
    a = Solver.from_config(cfg, precision=precision)
    a.set("u", cfg.initial_u(a.shape("u")))
    a.step(3)
    state = a.save_state()
    sa = a.step(2)
    b = Solver.from_config(cfg, precision=precision)
    b.load_state(state)
    sb = b.step(2)
    assert sa["n"] == sb["n"] == 5
    assert sa["sweeps_p"] == sb["sweeps_p"]
    for f in ("u", "v", "p", "phi"):
        assert np.array_equal(a.get(f), b.get(f)), f
    for x, y in zip(a.forces(), b.forces()):
        assert len(x) == 5 and np.array_equal(x, y)
    a.close()
    b.close()


def test_load_state_refuses_other_grids_bodies_and_buffers():
    from paper_2402_17337_gb300 import IbmError, Solver, build
    build.build()
    cfg = W.small_cases()[1]
    a = Solver.from_config(cfg)
    a.step(1)
    state = a.save_state()
    other = Solver.from_config(W.small_cases()[0])
    no_body = Solver(**kwargs(cfg))
    fresh = Solver.from_config(cfg)
    for target, buf in ((other, state), (no_body, state), (fresh, state[:len(state) // 2]),
                        (fresh, b"\0" * len(state))):
        with pytest.raises(IbmError) as e:
            target.load_state(buf)
        assert e.value.code == -1
    fresh.load_state(state)  # the matching context takes it
    for s in (a, other, no_body, fresh):
        s.close()
