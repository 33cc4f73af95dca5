"""Relaxation factor of the pressure SOR from the observed convergence rate.

The estimator (libibm's host function, the one ibm_tune_omega uses) is
pinned by Young's closed form for the model problem and by brute force: on a
stretched grid the oracle's sweep count at the estimated factor is compared
with the best factor of a fine scan.  The GPU test checks that the device
probe reaches the same factor as the oracle's rate gives.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2402_17337_gb300 import workloads as W


def young_rho(omega, mu):
    """SOR spectral radius for omega below the optimum (Young's relation)."""
    d = (omega * mu) ** 2 - 4.0 * (omega - 1.0)
    return ((omega * mu + math.sqrt(d)) / 2.0) ** 2


def lib_estimator():
    from paper_2402_17337_gb300 import build
    build.build()
    from paper_2402_17337_gb300 import omega_from_rate
    return omega_from_rate


@pytest.mark.parametrize("which", ["library", "oracle"])
@pytest.mark.parametrize("n", [16, 100, 1000])
def test_estimator_inverts_youngs_relation(n, which):
    est = lib_estimator() if which == "library" else oracle.omega_from_rate
    mu = math.cos(math.pi / (n + 1))  # Jacobi radius of the Dirichlet five-point Laplacian, n x n
    w_opt = 2.0 / (1.0 + math.sin(math.pi / (n + 1)))
    for frac in (0.3, 0.6, 0.9):
        w = 1.0 + frac * (w_opt - 1.0)
        got = est(w, young_rho(w, mu))
        assert abs(got - w_opt) <= 1e-9 * max(1.0, 1.0 / (2.0 - w_opt)), (n, frac, got, w_opt)
    # at or above the optimum the rate is omega - 1 and omega is kept
    assert est(1.99, 0.99) == 1.99
    assert est(1.5, 0.0) == 1.5


def oracle_rate(sim, omega, S, seed=5):
    ny, nx = sim.shape("p")
    phi0 = W.random_field((ny, nx), seed)
    zero = np.zeros((ny, nx))
    r = []
    for m in (S // 2, S):
        rc, _, sweeps, res = sim.poisson(zero, phi0=phi0, omega=omega, tol=0.0, check=S // 2, maxs=m)
        assert sweeps == m
        r.append(res)
    return (r[1] / r[0]) ** (1.0 / (S - S // 2))


def sweeps_to(sim, omega, drop=1e-8, seed=9):
    ny, nx = sim.shape("p")
    phi0 = W.random_field((ny, nx), seed)
    zero = np.zeros((ny, nx))
    rc, _, _, r0 = sim.poisson(zero, phi0=phi0, omega=omega, tol=0.0, check=1, maxs=0)
    rc, _, sweeps, _ = sim.poisson(zero, phi0=phi0, omega=omega, tol=drop * r0, check=4, maxs=100000)
    assert rc == 0
    return sweeps


def test_estimated_omega_is_near_the_brute_force_optimum_on_a_stretched_grid():
    est = lib_estimator()
    oracle.build()
    nx, ny = 128, 64
    sim = oracle.Sim(x0=-7.5, x1=24.0, y0=-12.5, y1=12.5, nx=nx, ny=ny, hmin=10.0 / nx,
                     ubox=(-1.0, 2.0, -0.75, 0.75), dt=1.0)
    w0 = 2.0 / (1.0 + math.sin(math.pi / max(nx, ny)))
    w_est = est(w0, oracle_rate(sim, w0, 4 * nx))
    scan = [w0 + (2.0 - w0) * f for f in np.linspace(0.0, 0.8, 33)]
    counts = {w: sweeps_to(sim, w) for w in scan}
    w_best = min(counts, key=counts.get)
    n_est = sweeps_to(sim, w_est)
    w_or = oracle.tune_omega(sim)
    n_or = sweeps_to(sim, w_or)
    print(f"omega0 {w0:.5f} ({counts[w0]} sweeps), library estimate {w_est:.5f} ({n_est}), "
          f"oracle probe {w_or:.5f} ({n_or}), scan best {w_best:.5f} ({counts[w_best]})")
    for w, n in ((w_est, n_est), (w_or, n_or)):
        assert w > w0
        assert n <= 1.1 * counts[w_best] + 8
        assert n < 0.8 * counts[w0]


@pytest.mark.gpu
def test_device_probe_matches_oracle_probe():
    from paper_2402_17337_gb300 import Solver, build
    build.build()
    oracle.build()
    nx, ny = 256, 128
    kw = dict(x0=-7.5, x1=24.0, y0=-12.5, y1=12.5, nx=nx, ny=ny, hmin=10.0 / nx, ubox=(-1.0, 2.0, -0.75, 0.75),
              dt=1.0)
    g = Solver(**kw, precision=1)
    w0 = g.P.omega_p
    w = g.tune_omega()
    sim = oracle.Sim(**kw)
    w_oracle = oracle.tune_omega(sim)
    print(f"omega0 {w0:.6f}, device probe {w:.6f}, oracle-rate estimate {w_oracle:.6f}")
    # both probe the same asymptotic rate (different start vectors): the factors agree to the
    # sensitivity of the estimate, and the device's factor converges as fast as the oracle's
    assert w > w0
    assert abs(w - w_oracle) <= 0.1 * (2.0 - w_oracle)
    assert sweeps_to(sim, w) <= 1.1 * sweeps_to(sim, w_oracle) + 8
