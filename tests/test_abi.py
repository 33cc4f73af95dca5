"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/ibm.h declares (no GPU calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(ibm_\w+)\s*\(", src)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    from paper_2402_17337_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    names = declared_functions()
    assert "ibm_step" in names and "ibm_create_grid" in names and "ibm_set_body" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    import paper_2402_17337_gb300 as pkg
    monkeypatch.setattr(pkg, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(pkg, "_lib", None)
    with pytest.raises(ImportError):
        pkg.lib()


def test_product_path_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_2402_17337_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".h", ".cpp", ".cuh")):
                txt = open(os.path.join(dirpath, fn)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, fn
                assert "ibm_oracle" not in txt, fn


def test_create_grid_rejects_invalid_parameters_before_touching_the_device():
    """Parameter validation of ibm_create_grid runs on the host before any
    CUDA call, so it is checked here without a GPU: sizes below 4, ny above
    the 8192 limit of the outflow-flux reduction, an unknown precision,
    non-positive Re or dt, no pressure tolerance, omega outside (0, 2)."""
    import ctypes as C
    from paper_2402_17337_gb300 import build
    build.build()
    import paper_2402_17337_gb300 as ibm
    L = ibm.lib()

    def create(**over):
        kw = dict(x0=-2.0, x1=5.0, y0=-2.0, y1=2.0, nx=70, ny=45, hmin=0.0, ubox=(-1.0, 2.0, -0.75, 0.75), bc=0,
                  u_in=1.0, Re=100.0, dt=1e-3, precision=0, ptol=1e-8, prtol=0.0, htol=1e-12, check_p=8,
                  check_h=2, max_sweeps=1000, omega_p=1.9, omega_h=1.0, stream=None)
        kw.update(over)
        P = ibm.GridParams(kw["x0"], kw["x1"], kw["y0"], kw["y1"], kw["nx"], kw["ny"], kw["hmin"],
                           (C.c_double * 4)(*kw["ubox"]), kw["bc"], kw["u_in"], kw["Re"], kw["dt"], kw["precision"],
                           kw["ptol"], kw["prtol"], kw["htol"], kw["check_p"], kw["check_h"], kw["max_sweeps"],
                           kw["omega_p"], kw["omega_h"], kw["stream"])
        h = C.c_void_p()
        rc = L.ibm_create_grid(C.byref(P), C.byref(h))
        return rc, L.ibm_last_error().decode()

    for over in (dict(nx=3), dict(ny=3), dict(ny=8193), dict(precision=3), dict(precision=-1), dict(Re=0.0),
                 dict(dt=-1.0), dict(ptol=0.0), dict(bc=2), dict(omega_p=2.0), dict(omega_h=2.5)):
        rc, msg = create(**over)
        assert rc == -1 and msg, (over, rc, msg)


def test_entry_points_reject_null_handles_before_touching_the_device():
    """Every entry point checks its handle and pointer arguments first and
    answers IBM_E_INVAL with a message (no CUDA call is made), so this runs
    without a GPU; ibm_destroy and ibm_batch_destroy accept NULL."""
    import ctypes as C
    from paper_2402_17337_gb300 import build
    build.build()
    import paper_2402_17337_gb300 as ibm
    L = ibm.lib()
    n = C.c_int(0)
    size = C.c_size_t(0)
    stats = ibm.StepStats()
    prof = ibm.Profile()
    buf = (C.c_double * 4)()
    calls = {
        "ibm_create_grid": (None, None),
        "ibm_set_body": (None, 1.0, 0.12, 0.25, 2.0, 0.0, 0.0),
        "ibm_step": (None, 1, C.byref(stats)),
        "ibm_forces": (None, None, None, 0, C.byref(n)),
        "ibm_get_field": (None, 0, buf, 4),
        "ibm_set_field": (None, 0, buf, 4),
        "ibm_get_flags": (None, 0, None, None, None, 0),
        "ibm_get_grid": (None, None, None),
        "ibm_set_profiling": (None, 1),
        "ibm_get_profile": (None, C.byref(prof)),
        "ibm_tune": (None,),
        "ibm_tune_omega": (None, 0, None),
        "ibm_set_sor_shape": (None, 0),
        "ibm_set_warmstart": (None, 0, None, 1.0),
        "ibm_set_warmstart_base": (None, 0),
        "ibm_set_preconditioner": (None, 0, None, 1.0, 1),
        "ibm_state_bytes": (None, C.byref(size)),
        "ibm_save_state": (None, None, 0),
        "ibm_load_state": (None, None, 0),
        "ibm_batch_create": (None, 0, None),
        "ibm_batch_step": (None, 1, C.byref(stats)),
        "ibm_batch_set_graphs": (None, 1),
        "ibm_batch_set_budgets": (None, 1),
        "ibm_batch_set_sor_shape": (None, 0),
        "ibm_batch_set_profiling": (None, 1),
        "ibm_batch_get_profile": (None, C.byref(prof)),
        "ibm_unet_create": (None, 0, None),
        "ibm_unet_params": (None, None, 0, 0),
        "ibm_unet_grads": (None, None, 0),
        "ibm_unet_forward": (None, None, 8, 8, None, None),
    }
    for name, args in calls.items():
        rc = getattr(L, name)(*args)
        assert rc == -1, (name, rc)
        assert L.ibm_last_error().decode(), name
    bad = (C.c_int * 4)(16, 24, 32, 32)
    h = C.c_void_p()
    assert L.ibm_unet_create(bad, 0, C.byref(h)) == -1 and not h.value
    assert L.ibm_unet_num_params(None) == 0
    assert L.ibm_batch_stream(None) is None
    L.ibm_destroy(None)
    L.ibm_batch_destroy(None)


def test_noalloc_solve_rejects_non_increasing_faces_before_touching_the_device():
    """ibm_poisson_solve_noalloc checks its face coordinates on the host: a
    repeated or reversed face would give infinite or negative coefficients,
    so it returns IBM_E_INVAL and names the first bad index (dummy device
    pointers: no CUDA call is made before the check)."""
    import ctypes as C

    import numpy as np

    from paper_2402_17337_gb300 import build
    build.build()
    import paper_2402_17337_gb300 as ibm
    fn = ibm.lib().ibm_poisson_solve_noalloc
    D = C.POINTER(C.c_double)
    fn.argtypes = [C.c_int, C.c_int, D, D, C.c_void_p, C.c_void_p, C.c_double, C.c_double, C.c_int, C.c_int,
                   C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_double)]
    fn.restype = C.c_int
    xf = np.linspace(0.0, 1.0, 11)
    yf = np.linspace(0.0, 1.0, 9)
    for axis, k in (("xf", 4), ("yf", 7)):
        x, y = xf.copy(), yf.copy()
        (x if axis == "xf" else y)[k] = (x if axis == "xf" else y)[k - 1]
        rc = fn(10, 8, x.ctypes.data_as(D), y.ctypes.data_as(D), C.c_void_p(16), C.c_void_p(16), 1.5, 1e-8, 8, 10,
                None, None, None)
        assert rc == ibm.IBM_E_INVAL
        assert f"{axis}[{k}]".encode() in ibm.lib().ibm_last_error()
