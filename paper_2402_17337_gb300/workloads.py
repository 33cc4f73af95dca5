"""Seeded synthetic workloads: the flow configurations and random test inputs.

This module holds parameter sets and random-number draws only; none of the
method's arithmetic lives here.  Both the CUDA path's tests and the oracle's
tests take their inputs from it.

Configurations (non-dimensional, chord = U_inf = 1).  The 192x128 case starts
from rest; the stretched cases start from the uniform free stream (at
divergence 1e-8 the first pressure increment of a start from rest lies below
the FP64 resolution of the pressure residual on those grids).  The stretched
cases take the paper's ratio of time step to minimum spacing (Sec. 4:
spacing 0.004, time step 1e-4, i.e. dt = 0.025 hmin): the flow round the
thin ellipse's leading edge at the plunge's effective incidence is several
times the free stream, and the explicit convection goes unstable at ratios
near 0.2.
  plunge_192x128   uniform 192x128 on [-4,8]x[-4,4], ellipse t/c 0.12, Re 300,
                   h 0.25, k 2, dt 2e-3, 100 steps, divergence 1e-10 (Poisson residual
                   0.999e-10/dt).
  plunge_2048x1024 stretched 2048x1024 on the paper's domain [-7.5,24]x[-12.5,12.5]
                   (Sec. 2.3), min spacing 0.005, Re 1000, h 0.25, k 2, dt 1.25e-4,
                   divergence 1e-8 (Poisson residual 0.999e-8/dt).
  plunge_4096x2048 stretched 4096x2048, min spacing 0.0025, Re 1000, h 0.4, k 3,
                   dt 6.25e-5, divergence 1e-8.
  batch64          64 cases, numpy default_rng(17337): h~U[0.1,0.5], k~U[1,4],
                   Re~U[100,1000], nx uniform on {512,576,...,1536}, ny = nx/2;
                   min spacing 10/nx (uniform block ~30 % of nx), dt = 0.025 hmin.
  unet_1024x512    1024x512, min spacing 0.01, dt 2.5e-4.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

PAPER_DOMAIN = (-7.5, 24.0, -12.5, 12.5)
DT_PER_HMIN = 0.025  # the paper's time step over its grid spacing (Sec. 4)
UBOX = (-1.0, 2.0, -0.75, 0.75)
DIV_MARGIN = 0.999  # pressure residual tolerance over div_tol / dt


@dataclasses.dataclass
class FlowConfig:
    name: str
    x0: float
    x1: float
    y0: float
    y1: float
    nx: int
    ny: int
    hmin: float            # <= 0: uniform grid
    Re: float
    dt: float
    steps: int
    h: float = 0.25        # plunge amplitude (chords)
    k: float = 2.0         # reduced frequency
    chord: float = 1.0
    tc: float = 0.12       # thickness / chord
    xc: float = 0.0
    yc: float = 0.0
    bc: int = 0
    u_in: float = 1.0
    ubox: tuple = UBOX
    div_tol: float = 1e-8  # divergence left in fluid cells; Poisson residual tol = div_tol/dt
    htol: float = 1e-12    # velocity-system residual tolerance
    check_p: int = 8
    check_h: int = 2
    omega_p: float | None = None
    omega_h: float = 1.0
    init: str = "rest"     # "rest": zero interior flow; "uniform": u = u_in everywhere

    def initial_u(self, shape) -> np.ndarray:
        """Initial u field (canonical layout): zero interior with the inflow
        face at u_in, or the uniform free stream."""
        u = np.zeros(shape)
        if self.init == "uniform":
            u[:] = self.u_in
        elif self.bc == 0:
            u[:, 0] = self.u_in
        return u

    @property
    def ptol(self) -> float:
        # The projection leaves a fluid-cell divergence equal to dt times the
        # pressure residual up to the rounding of the divergence itself; the
        # residual tolerance sits 0.1 % below div_tol / dt so that rounding
        # cannot carry a converged step's divergence over div_tol.
        return DIV_MARGIN * self.div_tol / self.dt

    @property
    def cells(self) -> int:
        return self.nx * self.ny

    def omega(self) -> float:
        if self.omega_p is not None:
            return self.omega_p
        return 2.0 / (1.0 + math.sin(math.pi / max(self.nx, self.ny)))


def plunge_192x128() -> FlowConfig:
    return FlowConfig("plunge_192x128", -4.0, 8.0, -4.0, 4.0, 192, 128, 0.0, Re=300.0, dt=2e-3,
                      steps=100, h=0.25, k=2.0, div_tol=1e-10)


def plunge_2048x1024() -> FlowConfig:
    dt = DT_PER_HMIN * 0.005
    return FlowConfig("plunge_2048x1024", *PAPER_DOMAIN, 2048, 1024, 0.005, Re=1000.0, dt=dt,
                      steps=2000, h=0.25, k=2.0, div_tol=1e-8, init="uniform")


def plunge_4096x2048() -> FlowConfig:
    dt = DT_PER_HMIN * 0.0025
    return FlowConfig("plunge_4096x2048", *PAPER_DOMAIN, 4096, 2048, 0.0025, Re=1000.0, dt=dt,
                      steps=500, h=0.4, k=3.0, div_tol=1e-8, init="uniform")


def batch64(n: int = 64, seed: int = 17337) -> list[FlowConfig]:
    rng = np.random.default_rng(seed)
    out = []
    sizes = np.arange(512, 1536 + 1, 64)
    for c in range(n):
        h = float(rng.uniform(0.1, 0.5))
        k = float(rng.uniform(1.0, 4.0))
        Re = float(rng.uniform(100.0, 1000.0))
        nx = int(rng.choice(sizes))
        ny = nx // 2
        hmin = 10.0 / nx
        dt = DT_PER_HMIN * hmin
        out.append(FlowConfig(f"batch64[{c}]", *PAPER_DOMAIN, nx, ny, hmin, Re=Re, dt=dt, steps=1000,
                              h=h, k=k, div_tol=1e-8, init="uniform"))
    return out


def batch_small(n: int = 4, seed: int = 17337, sizes=(96, 112, 128, 144, 160, 176, 192)) -> list[FlowConfig]:
    """The 64-case batch's recipe at grids the oracle steps in seconds:
    same parameter distributions, nx from `sizes`, ny = nx/2, min spacing
    10/nx, divergence tolerance 1e-10, 5 steps."""
    rng = np.random.default_rng(seed)
    out = []
    for c in range(n):
        h = float(rng.uniform(0.1, 0.5))
        k = float(rng.uniform(1.0, 4.0))
        Re = float(rng.uniform(100.0, 1000.0))
        nx = int(rng.choice(np.asarray(sizes)))
        hmin = 10.0 / nx
        dt = DT_PER_HMIN * hmin
        out.append(FlowConfig(f"batch_small[{c}]", *PAPER_DOMAIN, nx, nx // 2, hmin, Re=Re, dt=dt, steps=5,
                              h=h, k=k, div_tol=1e-10, init="uniform"))
    return out


def unet_1024x512() -> FlowConfig:
    dt = DT_PER_HMIN * 0.01
    return FlowConfig("unet_1024x512", *PAPER_DOMAIN, 1024, 512, 0.01, Re=300.0, dt=dt, steps=1000,
                      div_tol=1e-10, init="uniform")


def small_cases() -> list[FlowConfig]:
    """Small grids for element-wise parity: several tiles and ragged edges."""
    return [
        FlowConfig("plunge_70x45_uniform", -2.0, 5.0, -2.25, 2.25, 70, 45, 0.0, Re=200.0, dt=4e-3,
                   steps=6, h=0.3, k=2.5, div_tol=1e-10, check_p=4),
        FlowConfig("plunge_97x61_stretched", -7.5, 24.0, -12.5, 12.5, 97, 61, 0.08, Re=500.0,
                   dt=5e-3, steps=5, h=0.25, k=2.0, ubox=(-1.0, 2.0, -0.8, 0.8), div_tol=1e-10,
                   check_p=6),
    ]


def random_field(shape, seed: int, scale: float = 1.0) -> np.ndarray:
    """Seeded standard-normal field (float64)."""
    return np.random.default_rng(seed).standard_normal(shape) * scale
