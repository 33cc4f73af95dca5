"""GB300 (sm_103a) immersed-boundary fractional step of arXiv 2402.17337.

Thin ctypes binding of ``libibm.so`` (C ABI in ``include/ibm.h``): argument
marshalling only, every step of the method runs in the library's CUDA
kernels.  There is no CPU fallback: loading fails loudly when the library
has not been built (``paper_2402_17337_gb300.build.build()``).
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libibm.so")
_lock = threading.Lock()
_lib = None

IBM_OK, IBM_E_INVAL, IBM_E_CUDA, IBM_E_NOCONV, IBM_E_DIVERGED, IBM_E_TIMEOUT = 0, -1, -2, -3, -4, -5
FIELDS = {"u": 0, "v": 1, "p": 2, "phi": 3, "b": 4, "uh": 5, "vh": 6, "Ru": 7, "Rv": 8,
          "Hu": 9, "Hv": 10, "q": 11}


class IbmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libibm error {code}: {msg}")
        self.code = code


class GridParams(C.Structure):
    _fields_ = [("x0", C.c_double), ("x1", C.c_double), ("y0", C.c_double), ("y1", C.c_double),
                ("nx", C.c_int), ("ny", C.c_int), ("hmin", C.c_double), ("ubox", C.c_double * 4),
                ("bc", C.c_int), ("u_in", C.c_double), ("Re", C.c_double), ("dt", C.c_double),
                ("precision", C.c_int), ("poisson_tol", C.c_double), ("poisson_rtol", C.c_double),
                ("helm_tol", C.c_double), ("check_every_p", C.c_int), ("check_every_h", C.c_int),
                ("max_sweeps", C.c_int), ("omega_p", C.c_double), ("omega_h", C.c_double),
                ("cuda_stream", C.c_void_p)]


class StepStats(C.Structure):
    _fields_ = [("n", C.c_int), ("t", C.c_double), ("sweeps_u", C.c_int), ("sweeps_v", C.c_int),
                ("sweeps_p", C.c_int), ("res_u", C.c_double), ("res_v", C.c_double),
                ("res_p", C.c_double), ("div_max", C.c_double), ("cl", C.c_double), ("cd", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Profile(C.Structure):
    _fields_ = [("launches", C.c_longlong), ("sweep_launches", C.c_longlong), ("sweep_ms", C.c_double),
                ("steps", C.c_longlong), ("poisson_sweeps", C.c_longlong), ("helm_sweeps", C.c_longlong),
                ("sor_shape", C.c_int * 3), ("sor_us_per_sweep", C.c_double), ("sweep_cells", C.c_longlong),
                ("sor_form", C.c_int), ("ws_applied", C.c_longlong), ("ws_kept", C.c_longlong),
                ("sor_index", C.c_int)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["sor_shape"] = list(self.sor_shape)
        return d


_D = C.POINTER(C.c_double)
_U8 = C.POINTER(C.c_uint8)
_VP = C.c_void_p


def lib():
    """Loads libibm.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"{LIB_PATH} is missing: run paper_2402_17337_gb300.build.build()")
            L = C.CDLL(LIB_PATH)
            L.ibm_create_grid.argtypes = [C.POINTER(GridParams), C.POINTER(_VP)]
            L.ibm_set_body.argtypes = [_VP] + [C.c_double] * 6
            L.ibm_step.argtypes = [_VP, C.c_int, C.POINTER(StepStats)]
            L.ibm_forces.argtypes = [_VP, _D, _D, C.c_int, C.POINTER(C.c_int)]
            L.ibm_get_field.argtypes = [_VP, C.c_int, _D, C.c_size_t]
            L.ibm_set_field.argtypes = [_VP, C.c_int, _D, C.c_size_t]
            L.ibm_get_flags.argtypes = [_VP, C.c_int, _U8, _U8, _D, C.c_size_t]
            L.ibm_get_grid.argtypes = [_VP, _D, _D]
            L.ibm_poisson_solve.argtypes = [_VP, _VP, _VP, C.c_double, C.c_int, C.c_int,
                                            C.POINTER(C.c_int), C.POINTER(C.c_double)]
            L.ibm_set_profiling.argtypes = [_VP, C.c_int]
            L.ibm_tune.argtypes = [_VP]
            L.ibm_get_profile.argtypes = [_VP, C.POINTER(Profile)]
            L.ibm_unet_create.argtypes = [C.POINTER(C.c_int), C.c_ulonglong, C.POINTER(_VP)]
            L.ibm_unet_destroy.argtypes = [_VP]
            L.ibm_unet_destroy.restype = None
            L.ibm_unet_num_params.argtypes = [_VP]
            L.ibm_unet_num_params.restype = C.c_longlong
            L.ibm_unet_params.argtypes = [_VP, C.POINTER(C.c_float), C.c_longlong, C.c_int]
            L.ibm_unet_grads.argtypes = [_VP, C.POINTER(C.c_float), C.c_longlong]
            L.ibm_unet_forward.argtypes = [_VP, _VP, C.c_int, C.c_int, _VP, _VP]
            L.ibm_unet_train_step.argtypes = [_VP, _VP, _VP, C.c_int, C.c_int, C.c_float, C.c_int,
                                              C.POINTER(C.c_double), _VP]
            L.ibm_set_warmstart.argtypes = [_VP, C.c_int, _VP, C.c_double]
            L.ibm_set_warmstart_base.argtypes = [_VP, C.c_int]
            L.ibm_set_preconditioner.argtypes = [_VP, C.c_int, _VP, C.c_double, C.c_int]
            L.ibm_state_bytes.argtypes = [_VP, C.POINTER(C.c_size_t)]
            L.ibm_save_state.argtypes = [_VP, _VP, C.c_size_t]
            L.ibm_load_state.argtypes = [_VP, _VP, C.c_size_t]
            L.ibm_get_sample.argtypes = [_VP, C.POINTER(C.c_float), C.POINTER(C.c_float), C.POINTER(C.c_int),
                                         C.POINTER(C.c_int)]
            L.ibm_tune_omega.argtypes = [_VP, C.c_int, _D]
            L.ibm_set_sor_shape.argtypes = [_VP, C.c_int]
            L.ibm_sor_num_shapes.argtypes = []
            L.ibm_omega_from_rate.argtypes = [C.c_double, C.c_double]
            L.ibm_omega_from_rate.restype = C.c_double
            L.ibm_batch_create.argtypes = [C.POINTER(_VP), C.c_int, C.POINTER(_VP)]
            L.ibm_batch_step.argtypes = [_VP, C.c_int, C.POINTER(StepStats)]
            L.ibm_batch_set_graphs.argtypes = [_VP, C.c_int]
            L.ibm_batch_set_budgets.argtypes = [_VP, C.c_int]
            L.ibm_batch_set_sor_shape.argtypes = [_VP, C.c_int]
            L.ibm_batch_stream.argtypes = [_VP]
            L.ibm_batch_stream.restype = _VP
            L.ibm_batch_set_profiling.argtypes = [_VP, C.c_int]
            L.ibm_batch_get_profile.argtypes = [_VP, C.POINTER(Profile)]
            L.ibm_batch_destroy.argtypes = [_VP]
            L.ibm_batch_destroy.restype = None
            L.ibm_destroy.argtypes = [_VP]
            L.ibm_destroy.restype = None
            L.ibm_last_error.restype = C.c_char_p
            _lib = L
    return _lib


def _check(rc):
    if rc != IBM_OK:
        raise IbmError(rc, lib().ibm_last_error().decode())
    return rc


def _dp(a):
    return a.ctypes.data_as(_D)


def num_sor_shapes():
    return lib().ibm_sor_num_shapes()


def omega_from_rate(omega, rho):
    """Young's relation: optimal relaxation factor from the rate observed at omega."""
    return lib().ibm_omega_from_rate(omega, rho)


def default_omega(nx, ny):
    return 2.0 / (1.0 + np.sin(np.pi / max(nx, ny)))


class Solver:
    """One simulation context on the GPU (owns the device memory)."""

    def __init__(self, *, x0, x1, y0, y1, nx, ny, hmin=0.0, ubox=(-1.0, 2.0, -0.75, 0.75), bc=0,
                 u_in=1.0, Re=100.0, dt=1e-3, precision=0, ptol=1e-10, prtol=0.0, htol=1e-12,
                 check_p=8, check_h=2, max_sweeps=1000000, omega_p=None, omega_h=1.0, stream=None):
        if omega_p is None:
            omega_p = default_omega(nx, ny)
        P = GridParams(x0, x1, y0, y1, nx, ny, hmin, (C.c_double * 4)(*ubox), bc, u_in, Re, dt,
                       precision, ptol, prtol, htol, check_p, check_h, max_sweeps, omega_p, omega_h,
                       stream)
        self.P = P
        self.nx, self.ny = nx, ny
        h = _VP()
        _check(lib().ibm_create_grid(C.byref(P), C.byref(h)))
        self._h = h

    @classmethod
    def from_config(cls, cfg, **over):
        kw = dict(x0=cfg.x0, x1=cfg.x1, y0=cfg.y0, y1=cfg.y1, nx=cfg.nx, ny=cfg.ny, hmin=cfg.hmin,
                  ubox=cfg.ubox, bc=cfg.bc, u_in=cfg.u_in, Re=cfg.Re, dt=cfg.dt, ptol=cfg.ptol,
                  htol=cfg.htol, check_p=cfg.check_p, check_h=cfg.check_h, omega_p=cfg.omega(),
                  omega_h=cfg.omega_h)
        kw.update(over)
        s = cls(**kw)
        s.set_body(cfg.chord, cfg.tc, cfg.h, cfg.k, cfg.xc, cfg.yc)
        return s

    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            lib().ibm_destroy(h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def shape(self, name):
        nx, ny = self.nx, self.ny
        if name in ("u", "uh", "Ru", "Hu"):
            return (ny, nx + 1)
        if name in ("v", "vh", "Rv", "Hv"):
            return (ny + 1, nx)
        return (ny, nx)

    def set_body(self, chord=1.0, tc=0.12, h=0.0, k=0.0, xc=0.0, yc=0.0):
        _check(lib().ibm_set_body(self._h, chord, tc, h, k, xc, yc))

    def step(self, n=1):
        st = StepStats()
        _check(lib().ibm_step(self._h, n, C.byref(st)))
        return st.as_dict()

    def step_rc(self, n=1):
        """Like step() but returns (rc, stats) instead of raising."""
        st = StepStats()
        rc = lib().ibm_step(self._h, n, C.byref(st))
        return rc, st.as_dict()

    def forces(self):
        n = C.c_int(0)
        _check(lib().ibm_forces(self._h, None, None, 0, C.byref(n)))
        cl = np.zeros(max(n.value, 1))
        cd = np.zeros(max(n.value, 1))
        _check(lib().ibm_forces(self._h, _dp(cl), _dp(cd), n.value, C.byref(n)))
        return cl[:n.value], cd[:n.value]

    def get(self, name, out=None):
        """Field `name` in the compact row-major layout.  out: a C-contiguous
        float64 array of the field's shape to copy into (e.g. pinned memory,
        which the device writes directly); a new array otherwise."""
        if out is None:
            out = np.zeros(self.shape(name))
        elif (out.dtype != np.float64 or out.shape != self.shape(name) or not out.flags["C_CONTIGUOUS"]
              or not out.flags["WRITEABLE"]):
            raise ValueError(f"out must be a writeable C-contiguous float64 array of shape {self.shape(name)}")
        _check(lib().ibm_get_field(self._h, FIELDS[name], _dp(out), out.size))
        return out

    def set(self, name, arr):
        a = np.ascontiguousarray(arr, dtype=np.float64).reshape(self.shape(name))
        _check(lib().ibm_set_field(self._h, FIELDS[name], _dp(a), a.size))

    def flags(self, grid):
        shp = self.shape("u" if grid == 0 else ("v" if grid == 1 else "p"))
        fl = np.zeros(shp, np.uint8)
        dr = np.zeros(shp, np.uint8)
        al = np.zeros(shp)
        _check(lib().ibm_get_flags(self._h, grid, fl.ctypes.data_as(_U8), dr.ctypes.data_as(_U8), _dp(al),
                                   fl.size))
        return (fl, dr, al) if grid < 2 else fl

    def grid(self):
        xf = np.zeros(self.nx + 1)
        yf = np.zeros(self.ny + 1)
        _check(lib().ibm_get_grid(self._h, _dp(xf), _dp(yf)))
        return xf, yf

    def tune(self):
        """Re-runs the autotuner of the FP32 sweep tile (precision 1)."""
        _check(lib().ibm_tune(self._h))
        return self.profile()

    def set_profiling(self, on=True):
        _check(lib().ibm_set_profiling(self._h, 1 if on else 0))

    def profile(self):
        p = Profile()
        _check(lib().ibm_get_profile(self._h, C.byref(p)))
        return p.as_dict()

    def set_sor_shape(self, index):
        """Fixes the FP32 sweep tile shape (index into the library's table; -1: autotune)."""
        _check(lib().ibm_set_sor_shape(self._h, index))

    def tune_omega(self, sweeps=0):
        """Sets the pressure SOR relaxation factor from the observed convergence; returns it."""
        w = C.c_double(0)
        _check(lib().ibm_tune_omega(self._h, sweeps, C.byref(w)))
        self.P.omega_p = w.value
        return w.value

    def set_warmstart(self, mode, net=None, target_scale=1.0):
        """0: previous increment; 1: learned (U-Net net); 2: previous increment + samples."""
        self._ws_net = net  # keep the network alive while the context uses it
        _check(lib().ibm_set_warmstart(self._h, mode, net._h if net is not None else None, target_scale))

    def save_state(self):
        """The context's state (bytes) for load_state: fields, histories, step count."""
        n = C.c_size_t(0)
        _check(lib().ibm_state_bytes(self._h, C.byref(n)))
        buf = np.zeros(n.value, np.uint8)
        _check(lib().ibm_save_state(self._h, buf.ctypes.data, n.value))
        return buf.tobytes()

    def load_state(self, state):
        """Restores a state from save_state (same grid, Re, dt and body)."""
        buf = np.frombuffer(state, np.uint8)
        _check(lib().ibm_load_state(self._h, buf.ctypes.data, buf.size))

    def set_preconditioner(self, kind, net=None, target_scale=1.0, pre_smooth=1):
        """Precision 2: 0 V-cycle; 1 two-level cycle with the U-Net net as coarse level."""
        self._pc_net = net  # keep the network alive while the context uses it
        _check(lib().ibm_set_preconditioner(self._h, kind, net._h if net is not None else None, target_scale,
                                            pre_smooth))

    def set_warmstart_base(self, base):
        """0: previous increment; 1: linear extrapolation 2 phi^n - phi^(n-1)."""
        _check(lib().ibm_set_warmstart_base(self._h, base))

    def sample(self):
        """(features [Hc][Wc][4], target [Hc][Wc]) recorded by the last step (mode 2)."""
        hc, wc = C.c_int(0), C.c_int(0)
        _check(lib().ibm_get_sample(self._h, None, None, C.byref(hc), C.byref(wc)))
        f = np.zeros((hc.value, wc.value, 4), np.float32)
        t = np.zeros((hc.value, wc.value), np.float32)
        _F = C.POINTER(C.c_float)
        _check(lib().ibm_get_sample(self._h, f.ctypes.data_as(_F), t.ctypes.data_as(_F), C.byref(hc), C.byref(wc)))
        return f, t

    def poisson_solve(self, b_ptr, phi_ptr, tol, check_every=8, max_sweeps=0):
        """Standalone pressure solve on device buffers (nx*ny doubles each)."""
        s = C.c_int(0)
        r = C.c_double(0)
        rc = lib().ibm_poisson_solve(self._h, b_ptr, phi_ptr, tol, check_every, max_sweeps, C.byref(s),
                                     C.byref(r))
        return rc, s.value, r.value


class Batch:
    """Many Solver cases (precision 1) advanced together; the pressure solves
    of all cases share every sweep launch.  The solvers are borrowed and
    kept alive by the batch."""

    def __init__(self, solvers):
        self.solvers = list(solvers)
        arr = (_VP * len(self.solvers))(*[s._h for s in self.solvers])
        h = _VP()
        _check(lib().ibm_batch_create(arr, len(self.solvers), C.byref(h)))
        self._h = h

    def step(self, n=1):
        """Advances every case by n steps; returns each case's last-step stats."""
        st = (StepStats * len(self.solvers))()
        _check(lib().ibm_batch_step(self._h, n, st))
        return [x.as_dict() for x in st]

    def set_graphs(self, on=True):
        """CUDA-graph replay of the sweeps when budgets are off."""
        _check(lib().ibm_batch_set_graphs(self._h, 1 if on else 0))

    def set_budgets(self, on=True):
        """Each case its own sweeps per round of the pressure loop (default) or
        the shortest prediction of the round for all (graph-replayable)."""
        _check(lib().ibm_batch_set_budgets(self._h, 1 if on else 0))

    def set_sor_shape(self, index):
        """Fixes the FP32 sweep tile shape of the batch (-1: tune over the batch)."""
        _check(lib().ibm_batch_set_sor_shape(self._h, index))

    @property
    def stream(self):
        """The batch's cudaStream_t (an integer handle)."""
        return lib().ibm_batch_stream(self._h)

    def set_profiling(self, on=True):
        _check(lib().ibm_batch_set_profiling(self._h, 1 if on else 0))

    def profile(self):
        p = Profile()
        _check(lib().ibm_batch_get_profile(self._h, C.byref(p)))
        return p.as_dict()

    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            lib().ibm_batch_destroy(h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class UNet:
    """The warm-start U-Net (device weights; BF16 tensor-core kernels)."""

    def __init__(self, widths=(32, 64, 128, 128), seed=0):
        w = (C.c_int * 4)(*widths)
        h = _VP()
        _check(lib().ibm_unet_create(w, seed, C.byref(h)))
        self._h = h
        self.widths = tuple(widths)
        self.n = lib().ibm_unet_num_params(h)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().ibm_unet_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self):
        a = np.zeros(self.n, np.float32)
        _check(lib().ibm_unet_params(self._h, a.ctypes.data_as(C.POINTER(C.c_float)), self.n, 0))
        return a

    def set_params(self, a):
        a = np.ascontiguousarray(a, np.float32)
        _check(lib().ibm_unet_params(self._h, a.ctypes.data_as(C.POINTER(C.c_float)), self.n, 1))

    def grads(self):
        a = np.zeros(self.n, np.float32)
        _check(lib().ibm_unet_grads(self._h, a.ctypes.data_as(C.POINTER(C.c_float)), self.n))
        return a

    def forward(self, feat_ptr, H, W, out_ptr, stream=None):
        _check(lib().ibm_unet_forward(self._h, feat_ptr, H, W, out_ptr, stream))

    def train_step(self, feat_ptr, target_ptr, H, W, lr=1e-3, apply=True, stream=None):
        loss = C.c_double(0.0)
        _check(lib().ibm_unet_train_step(self._h, feat_ptr, target_ptr, H, W, lr, 1 if apply else 0,
                                         C.byref(loss), stream))
        return loss.value
