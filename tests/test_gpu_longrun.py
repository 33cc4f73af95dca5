"""The full-length run driver (paper_2402_17337_gb300.longrun) on the small
192x128 configuration: both paths keep the divergence below the
configuration's tolerance in every step, and the mixed path (FP32 sweeps in
FP64 defect correction) stays within the mixed-path bound of the FP64 path
at every checkpoint, fields and force histories."""
import pytest

pytestmark = pytest.mark.gpu


def test_longrun_small_configuration():
    from paper_2402_17337_gb300 import build, longrun
    build.build()
    res = longrun.run("plunge_192x128", steps=30, checkpoints=3)
    assert res["steps"] == 30 and len(res["checkpoints"]) == 3
    for path in ("mixed", "fp64"):
        assert res["div_max"][path] <= res["div_tol"] * 1.001, res["div_max"]
        assert res["poisson_sweeps_per_step"][path] > 0
    for cp in res["checkpoints"]:
        for name, err in cp["error_vs_fp64"].items():
            assert err <= 1e-6, (cp["step"], name, err)
