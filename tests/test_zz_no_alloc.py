"""The allocation-free pressure solve (ibm_poisson_solve_noalloc) against the
context-based one (ibm_poisson_solve).

ibm_poisson_solve_noalloc exists for callers that cannot call cudaMalloc,
such as an application whose device memory belongs to its own allocator or
a pool sized up front: its scratch lives in a static device array of the
library.  This file is collected last, so that a run that stops at the
first failure has already run every other test.  It must pass alone in a
fresh process and after the other tests (the static scratch keeps the last
call's contents, so it is called twice in a row here).
"""
import ctypes as C

import numpy as np
import pytest

from paper_2402_17337_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-10  # relative field tolerance used by the parity tests


def _noalloc():
    import paper_2402_17337_gb300 as ibm
    fn = ibm.lib().ibm_poisson_solve_noalloc
    D = C.POINTER(C.c_double)
    fn.argtypes = [C.c_int, C.c_int, D, D, C.c_void_p, C.c_void_p, C.c_double, C.c_double, C.c_int, C.c_int,
                   C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_double)]
    fn.restype = C.c_int
    return fn


def test_noalloc_solve_matches_context_solve_on_two_calls():
    import torch

    import paper_2402_17337_gb300 as ibm
    from paper_2402_17337_gb300 import build
    build.build()
    fn = _noalloc()
    nx, ny = 133, 67
    # an FP64 (precision 0) context: the allocation-free solve repeats its iterates
    ctx = ibm.Solver(x0=-7.5, x1=24.0, y0=-12.5, y1=12.5, nx=nx, ny=ny, hmin=0.09, ubox=(-1.0, 2.0, -0.8, 0.8),
                     dt=1.0, precision=0)
    xf, yf = ctx.grid()
    V = np.outer(np.diff(yf), np.diff(xf))
    omega = ctx.P.omega_p
    D = C.POINTER(C.c_double)
    for call in range(2):
        b = W.random_field((ny, nx), seed=100 + call)
        b -= np.sum(b * V) / np.sum(V)
        phi0 = W.random_field((ny, nx), seed=200 + call, scale=0.1)
        bd = torch.tensor(b, dtype=torch.float64, device="cuda")
        p_ctx = torch.tensor(phi0, dtype=torch.float64, device="cuda")
        p_na = torch.tensor(phi0, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        rc, s_ctx, r_ctx = ctx.poisson_solve(bd.data_ptr(), p_ctx.data_ptr(), 1e-9, 8)
        assert rc == 0
        s_na, r_na = C.c_int(-1), C.c_double(-1.0)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        rc = fn(nx, ny, xf.ctypes.data_as(D), yf.ctypes.data_as(D), bd.data_ptr(), p_na.data_ptr(), omega, 1e-9,
                8, 0, None, C.byref(s_na), C.byref(r_na))
        assert rc == 0, ibm.lib().ibm_last_error()
        if call == 1:  # after the first call's one-time set-up, a call takes no device memory
            assert torch.cuda.mem_get_info()[0] == free0
        assert s_na.value == s_ctx and r_na.value <= 1e-9
        a, ref = p_na.cpu().numpy(), p_ctx.cpu().numpy()
        assert np.abs(a - ref).max() <= TOL * np.abs(ref).max()
        assert a[0, nx - 1] == 0.0


def test_noalloc_on_a_side_stream():
    """The call on a caller's non-default stream gives the same result."""
    import torch

    import paper_2402_17337_gb300 as ibm
    from paper_2402_17337_gb300 import build
    build.build()
    fn = _noalloc()
    nx, ny = 96, 61
    ctx = ibm.Solver(x0=-7.5, x1=24.0, y0=-12.5, y1=12.5, nx=nx, ny=ny, hmin=0.12, ubox=(-1.0, 2.0, -0.8, 0.8),
                     dt=1.0, precision=0)
    xf, yf = ctx.grid()
    V = np.outer(np.diff(yf), np.diff(xf))
    b = W.random_field((ny, nx), seed=300)
    b -= np.sum(b * V) / np.sum(V)
    D = C.POINTER(C.c_double)
    bd = torch.tensor(b, dtype=torch.float64, device="cuda")
    p_ctx = torch.zeros((ny, nx), dtype=torch.float64, device="cuda")
    p_na = torch.zeros((ny, nx), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    rc, s_ctx, _ = ctx.poisson_solve(bd.data_ptr(), p_ctx.data_ptr(), 1e-9, 8)
    assert rc == 0
    side = torch.cuda.Stream()
    s_na, r_na = C.c_int(-1), C.c_double(-1.0)
    rc = fn(nx, ny, xf.ctypes.data_as(D), yf.ctypes.data_as(D), bd.data_ptr(), p_na.data_ptr(), ctx.P.omega_p,
            1e-9, 8, 0, C.c_void_p(side.cuda_stream), C.byref(s_na), C.byref(r_na))
    assert rc == 0, ibm.lib().ibm_last_error()
    assert s_na.value == s_ctx
    a, ref = p_na.cpu().numpy(), p_ctx.cpu().numpy()
    assert np.abs(a - ref).max() <= TOL * np.abs(ref).max()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import paper_2402_17337_gb300 as ibm
    from paper_2402_17337_gb300 import build
    build.build()
    fn = _noalloc()
    D = C.POINTER(C.c_double)
    xf = np.linspace(0.0, 1.0, 9001)
    yf = np.linspace(0.0, 1.0, 17)
    rc = fn(9000, 16, xf.ctypes.data_as(D), yf.ctypes.data_as(D), None, None, 1.5, 1e-8, 8, 10, None, None, None)
    assert rc == ibm.IBM_E_INVAL
    assert b"8192" in ibm.lib().ibm_last_error()
