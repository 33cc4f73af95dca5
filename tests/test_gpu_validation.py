"""The paper's validation set-up (Sec. 4.1) on the paper's own solver.

Re 500, thickness/chord 0.12, plunge amplitude h = 0.16, reduced frequency
k = 2 pi, spacing 0.004 near the body and time step 1e-4 on the paper's
domain, mesh M1 (1104 x 552, about 0.6 million cells, Sec. 4.2's smallest
mesh level).  The paper's method is red-black SOR for the pressure; here it
runs as FP32 sweeps inside FP64 defect correction (precision 1) and is
compared with the multigrid variant (precision 2), a different iteration for
the same discrete equations: both stop every step at the same divergence
tolerance (1e-8), so their fields and force histories must agree to a small
multiple of what that tolerance leaves undetermined.  The comparison data of
the paper's figure (other authors' results) is not available, so the lift
and drag histories are pinned by this agreement and by the Re 40 drag and
Re 100 shedding pins of the same step.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

STEPS = 300


def _run(cfg, precision, omega):
    import dataclasses

    import paper_2402_17337_gb300 as ibm
    s = ibm.Solver.from_config(dataclasses.replace(cfg, omega_p=omega), precision=precision,
                               max_sweeps=20000 if precision == 2 else 0)
    s.set("u", cfg.initial_u(s.shape("u")))
    div = 0.0
    for _ in range(STEPS // 50):
        st = s.step(50)
        div = max(div, st["div_max"])
    out = {n: s.get(n) for n in ("u", "v", "p")}
    cl, cd = s.forces()
    s.close()
    return out, cl, cd, div, st


def test_validation_case_on_the_paper_solver_matches_the_multigrid_variant():
    import paper_2402_17337_gb300 as ibm
    from paper_2402_17337_gb300 import build
    from paper_2402_17337_gb300 import validation as V
    build.build()
    cfg = V.config(*V.MESHES["M1"])
    probe = ibm.Solver.from_config(cfg, precision=1)
    omega = probe.tune_omega()
    probe.close()
    f1, cl1, cd1, div1, st1 = _run(cfg, 1, omega)
    f2, cl2, cd2, div2, st2 = _run(cfg, 2, omega)
    assert len(cl1) == len(cl2) == STEPS
    assert div1 <= cfg.div_tol * 1.001 and div2 <= cfg.div_tol * 1.001, (div1, div2)
    # the plunge's added-mass impulse dominates these first 300 steps: the lift
    # is large and both iterations give the same history
    assert np.abs(cl1).max() > 1.0
    for name in ("u", "v", "p"):
        a, b = f1[name], f2[name]
        assert np.abs(a - b).max() <= 1e-6 * np.abs(b).max(), (name, np.abs(a - b).max() / np.abs(b).max())
    assert np.abs(cl1 - cl2).max() <= 1e-6 * np.abs(cl2).max(), np.abs(cl1 - cl2).max() / np.abs(cl2).max()
    assert np.abs(cd1 - cd2).max() <= 1e-6 * np.abs(cd2).max(), np.abs(cd1 - cd2).max() / np.abs(cd2).max()
