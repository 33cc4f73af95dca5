"""Python access to the FP64 CPU oracle (``ibm_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product path (the
CUDA library and its binding) never imports this package.

The oracle is the plain restatement of the immersed-boundary fractional step
of arXiv 2402.17337 (Sec. 2.1 Eqs. 1-2, Sec. 2.2 Eqs. 3-4, Sec. 2.3, Sec. 3.1):
classification, AB2/CN predictor with red-black SOR, mass source on body cells,
red-black SOR pressure Poisson, projection and force histories.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ibm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


_PLAIN_PATH = os.path.join(_BUILD, "liboracle_plain.so")


def _compile(out_path, force, defines=()):
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(out_path)
            and os.path.getmtime(out_path) >= os.path.getmtime(_SRC)):
        return out_path
    tmp = out_path + f".tmp{os.getpid()}"
    cmd = (["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared", "-Wall"]
           + [f"-D{d}" for d in defines] + ["-o", tmp, _SRC, "-lm"])
    subprocess.run(cmd, check=True)
    os.replace(tmp, out_path)
    return out_path


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no FP contraction, OpenMP)."""
    return _compile(_LIB_PATH, force)


def build_plain(force: bool = False) -> str:
    """Compile the oracle's textbook-arithmetic form (-DORACLE_PLAIN: divisions
    by spacings, no fused multiply-add, flux-form Laplacians, one-pass sums)
    into its own library, for use with `use_library`."""
    return _compile(_PLAIN_PATH, force, ("ORACLE_PLAIN",))


class Params(C.Structure):
    _fields_ = [("x0", C.c_double), ("x1", C.c_double), ("y0", C.c_double), ("y1", C.c_double),
                ("nx", C.c_int), ("ny", C.c_int), ("hmin", C.c_double),
                ("ubox", C.c_double * 4), ("bc", C.c_int), ("u_in", C.c_double),
                ("Re", C.c_double), ("dt", C.c_double), ("ptol", C.c_double), ("prtol", C.c_double),
                ("htol", C.c_double),
                ("check_p", C.c_int), ("check_h", C.c_int), ("max_sweeps", C.c_int),
                ("omega_p", C.c_double), ("omega_h", C.c_double)]


class Stats(C.Structure):
    _fields_ = [("n", C.c_int), ("t", C.c_double), ("sweeps_u", C.c_int), ("sweeps_v", C.c_int),
                ("sweeps_p", C.c_int), ("res_u", C.c_double), ("res_v", C.c_double),
                ("res_p", C.c_double), ("div_max", C.c_double), ("cl", C.c_double),
                ("cd", C.c_double), ("sum_q", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_D = C.POINTER(C.c_double)
_U8 = C.POINTER(C.c_uint8)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _configure(C.CDLL(build()))
    return _lib


def _configure(L):
    """Declares the argument types of the oracle's C entry points on L."""
    L.or_build_axis.argtypes = [C.c_double] * 4 + [C.c_int, C.c_double, _D]
    L.or_create.argtypes = [C.POINTER(Params)]
    L.or_create.restype = C.c_void_p
    L.or_destroy.argtypes = [C.c_void_p]
    L.or_set_threads.argtypes = [C.c_void_p, C.c_int]
    L.or_get_grid.argtypes = [C.c_void_p, _D, _D]
    L.or_set_body.argtypes = [C.c_void_p] + [C.c_double] * 6
    L.or_step.argtypes = [C.c_void_p, C.c_int, C.POINTER(Stats)]
    L.or_get.argtypes = [C.c_void_p, C.c_int, _D]
    L.or_set.argtypes = [C.c_void_p, C.c_int, _D]
    L.or_get_stats.argtypes = [C.c_void_p, C.POINTER(Stats)]
    L.or_forces.argtypes = [C.c_void_p, _D, _D, C.c_int, C.POINTER(C.c_int)]
    L.or_classify.argtypes = [C.c_void_p, C.c_double]
    L.or_get_flags.argtypes = [C.c_void_p, C.c_int, _U8, _U8, _D]
    for name in ("or_lap_p", "or_lap_u", "or_lap_v"):
        getattr(L, name).argtypes = [C.c_void_p, _D, _D]
    L.or_conv.argtypes = [C.c_void_p, _D, _D, _D, _D]
    L.or_grad.argtypes = [C.c_void_p, _D, _D, _D]
    L.or_div.argtypes = [C.c_void_p, _D, _D, _D]
    L.or_poisson.argtypes = [C.c_void_p, _D, _D, C.c_double, C.c_double, C.c_double, C.c_int, C.c_int,
                             C.POINTER(C.c_int), C.POINTER(C.c_double)]
    L.or_helm_solve.argtypes = [C.c_void_p, C.c_int, _D, _D, C.c_double, C.c_double,
                                C.POINTER(C.c_int), C.POINTER(C.c_double)]
    L.or_clear_flags.argtypes = [C.c_void_p]
    return L


def build_variant(name, replacements):
    """Compiles a copy of the oracle with textual replacements (each `old`
    must occur exactly once) into its own library; for tests that plant a
    mistake in the oracle and check that a pin catches it."""
    with open(_SRC) as fh:
        src = fh.read()
    for old, new in replacements:
        if src.count(old) != 1:
            raise ValueError(f"{name}: {old!r} occurs {src.count(old)} times")
        src = src.replace(old, new)
    d = os.path.join(_BUILD, "variants")
    os.makedirs(d, exist_ok=True)
    c_path = os.path.join(d, f"{name}.c")
    so_path = os.path.join(d, f"lib{name}.so")
    with open(c_path, "w") as fh:
        fh.write(src)
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
                    "-o", so_path, c_path, "-lm"], check=True)
    return so_path


class use_library:
    """Context manager: oracle calls made inside go to the library at `path`
    (a variant from build_variant)."""

    def __init__(self, path):
        self.L = _configure(C.CDLL(path))

    def __enter__(self):
        global _lib
        lib()
        with _lock:
            self.saved, _lib = _lib, self.L
        return self.L

    def __exit__(self, *exc):
        global _lib
        with _lock:
            _lib = self.saved
        return False


def _dp(a):
    return a.ctypes.data_as(_D)


def build_axis(a0, a1, b0, b1, n, hmin):
    f = np.zeros(n + 1)
    rc = lib().or_build_axis(a0, a1, b0, b1, n, hmin, _dp(f))
    if rc:
        raise ValueError(f"or_build_axis failed ({rc})")
    return f


FIELDS = {"u": 0, "v": 1, "p": 2, "phi": 3, "b": 4, "uh": 5, "vh": 6, "Ru": 7, "Rv": 8,
          "Hu": 9, "Hv": 10, "q": 11, "D": 12}


class Sim:
    """One oracle simulation (owns the C object)."""

    def __init__(self, *, x0, x1, y0, y1, nx, ny, hmin=0.0, ubox=(-1.0, 2.0, -0.75, 0.75), bc=0,
                 u_in=1.0, Re=100.0, dt=1e-3, ptol=1e-10, prtol=0.0, htol=1e-12, check_p=10, check_h=2,
                 max_sweeps=200000, omega_p=None, omega_h=1.0, threads=1):
        if omega_p is None:
            omega_p = 2.0 / (1.0 + np.sin(np.pi / max(nx, ny)))
        P = Params(x0, x1, y0, y1, nx, ny, hmin, (C.c_double * 4)(*ubox), bc, u_in, Re, dt, ptol,
                   prtol, htol, check_p, check_h, max_sweeps, omega_p, omega_h)
        self.P = P
        self.nx, self.ny = nx, ny
        self._L = lib()
        self._h = self._L.or_create(C.byref(P))
        if not self._h:
            raise ValueError("or_create rejected the parameters")
        self._L.or_set_threads(self._h, threads)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._L.or_destroy(h)
            self._h = None

    # shapes in canonical (row = j) layout
    def shape(self, name):
        nx, ny = self.nx, self.ny
        if name in ("u", "uh", "Ru", "Hu"):
            return (ny, nx + 1)
        if name in ("v", "vh", "Rv", "Hv"):
            return (ny + 1, nx)
        return (ny, nx)

    def grid(self):
        xf = np.zeros(self.nx + 1)
        yf = np.zeros(self.ny + 1)
        self._L.or_get_grid(self._h, _dp(xf), _dp(yf))
        return xf, yf

    def set_body(self, chord=1.0, tc=0.12, h=0.0, k=0.0, xc=0.0, yc=0.0):
        rc = self._L.or_set_body(self._h, chord, tc, h, k, xc, yc)
        if rc:
            raise ValueError("or_set_body failed")

    def step(self, n=1):
        st = Stats()
        rc = self._L.or_step(self._h, n, C.byref(st))
        return rc, st.as_dict()

    def get(self, name):
        out = np.zeros(self.shape(name))
        self._L.or_get(self._h, FIELDS[name], _dp(out))
        return out

    def set(self, name, arr):
        a = np.ascontiguousarray(arr, dtype=np.float64).reshape(self.shape(name))
        rc = self._L.or_set(self._h, FIELDS[name], _dp(a))
        if rc:
            raise ValueError("or_set failed")

    def forces(self):
        n = C.c_int(0)
        self._L.or_forces(self._h, None, None, 0, C.byref(n))
        cl = np.zeros(max(n.value, 1))
        cd = np.zeros(max(n.value, 1))
        self._L.or_forces(self._h, _dp(cl), _dp(cd), n.value, C.byref(n))
        return cl[:n.value], cd[:n.value]

    def classify(self, t):
        if self._L.or_classify(self._h, t):
            raise ValueError("no body")

    def flags(self, grid):
        """grid 0: u nodes, 1: v nodes -> (flags, dir, alpha); 2: cut cells."""
        shp = self.shape("u" if grid == 0 else ("v" if grid == 1 else "p"))
        fl = np.zeros(shp, np.uint8)
        if grid == 2:
            self._L.or_get_flags(self._h, 2, fl.ctypes.data_as(_U8), None, None)
            return fl
        dr = np.zeros(shp, np.uint8)
        al = np.zeros(shp)
        self._L.or_get_flags(self._h, grid, fl.ctypes.data_as(_U8), dr.ctypes.data_as(_U8), _dp(al))
        return fl, dr, al

    # operators
    def lap_p(self, f):
        f = np.ascontiguousarray(f, np.float64)
        out = np.zeros(self.shape("p"))
        self._L.or_lap_p(self._h, _dp(f), _dp(out))
        return out

    def lap_u(self, u):
        u = np.ascontiguousarray(u, np.float64)
        out = np.zeros(self.shape("u"))
        self._L.or_lap_u(self._h, _dp(u), _dp(out))
        return out

    def lap_v(self, v):
        v = np.ascontiguousarray(v, np.float64)
        out = np.zeros(self.shape("v"))
        self._L.or_lap_v(self._h, _dp(v), _dp(out))
        return out

    def conv(self, u, v):
        u = np.ascontiguousarray(u, np.float64)
        v = np.ascontiguousarray(v, np.float64)
        Hu = np.zeros(self.shape("u"))
        Hv = np.zeros(self.shape("v"))
        self._L.or_conv(self._h, _dp(u), _dp(v), _dp(Hu), _dp(Hv))
        return Hu, Hv

    def grad(self, f):
        f = np.ascontiguousarray(f, np.float64)
        gu = np.zeros(self.shape("u"))
        gv = np.zeros(self.shape("v"))
        self._L.or_grad(self._h, _dp(f), _dp(gu), _dp(gv))
        return gu, gv

    def div(self, u, v):
        u = np.ascontiguousarray(u, np.float64)
        v = np.ascontiguousarray(v, np.float64)
        out = np.zeros(self.shape("p"))
        self._L.or_div(self._h, _dp(u), _dp(v), _dp(out))
        return out

    def poisson(self, b, phi0=None, omega=None, tol=1e-10, rtol=0.0, check=10, maxs=200000):
        b = np.ascontiguousarray(b, np.float64)
        phi = np.zeros(self.shape("p")) if phi0 is None else np.array(phi0, np.float64, copy=True)
        if omega is None:
            omega = self.P.omega_p
        s = C.c_int(0)
        r = C.c_double(0)
        rc = self._L.or_poisson(self._h, _dp(b), _dp(phi), omega, tol, rtol, check, maxs, C.byref(s),
                             C.byref(r))
        return rc, phi, s.value, r.value

    def helm_solve(self, grid, R, x0, beta, Ub=0.0):
        """Implicit velocity solve on grid 0 (u) or 1 (v); x0 carries boundary values."""
        R = np.ascontiguousarray(R, np.float64)
        x = np.array(x0, np.float64, copy=True)
        s = C.c_int(0)
        r = C.c_double(0)
        rc = self._L.or_helm_solve(self._h, grid, _dp(x), _dp(R), beta, Ub, C.byref(s), C.byref(r))
        return rc, x, s.value, r.value

    def clear_flags(self):
        self._L.or_clear_flags(self._h)


def omega_from_rate(omega, rho):
    """Optimal SOR relaxation factor from the convergence factor per sweep rho
    observed at omega (Young's relation for consistently ordered matrices,
    omega below the optimum: (rho + omega - 1)^2 = rho omega^2 mu^2 with mu the
    Jacobi spectral radius; optimum 2 / (1 + sqrt(1 - mu^2))).  Returns omega
    when rho <= omega - 1 (at or above the optimum)."""
    if not (0.0 < rho < 1.0) or rho <= omega - 1.0:
        return omega
    mu = (rho + omega - 1.0) / (np.sqrt(rho) * omega)
    if not mu < 1.0:
        return omega
    return float(2.0 / (1.0 + np.sqrt((1.0 - mu) * (1.0 + mu))))


def sor_rate(sim, omega, sweeps, seed=5, chunk=64):
    """Asymptotic convergence factor per sweep of the pressure SOR on the
    homogeneous system from a seeded random start: the residual is taken
    every `chunk` sweeps until it has fallen by 1e-10 or `sweeps` sweeps have
    run, and the factor over the second half of the sweeps run."""
    ny, nx = sim.shape("p")
    phi = np.random.default_rng(seed).standard_normal((ny, nx))
    zero = np.zeros((ny, nx))
    _, _, _, r0 = sim.poisson(zero, phi0=phi, omega=omega, tol=0.0, check=1, maxs=0)
    r = [r0]
    s = 0
    while r[-1] > 1e-10 * r[0] and s + chunk <= sweeps:
        _, phi, _, res = sim.poisson(zero, phi0=phi, omega=omega, tol=0.0, check=chunk, maxs=chunk)
        r.append(res)
        s += chunk
    b = len(r) - 1
    a = b // 2
    if b == a or r[a] <= 0.0 or r[b] <= 0.0:
        return 0.0
    return (r[b] / r[a]) ** (1.0 / (chunk * (b - a)))


def tune_omega(sim, sweeps=0):
    """Relaxation factor of the pressure SOR for the oracle's grid: the rate at
    the current factor through Young's relation, kept if a second probe
    confirms a faster rate (the same procedure as the library's, written
    independently)."""
    ny, nx = sim.shape("p")
    if sweeps <= 0:
        sweeps = min(max(8 * max(nx, ny), 2048), 32768)
    w0 = sim.P.omega_p
    rho0 = sor_rate(sim, w0, sweeps)
    w1 = omega_from_rate(w0, rho0)
    if w1 != w0 and sor_rate(sim, w1, sweeps) < rho0:
        return w1
    return w0
