"""Pins for the FP64 CPU oracle (no GPU).

Each check ties the oracle to something other than itself: a closed form, an
exact discrete identity, a brute-force recomputation of a definition, or a
dense direct solve.  Paper references: kinematics Eqs. 1-2 (Sec. 2.1);
governing equations Eqs. 3-4 and the fractional-step/SOR scheme (Sec. 2.2);
stretched grid (Sec. 2.3).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2402_17337_gb300 import workloads as W


def box_sim(n, Re=100.0, dt=0.01, **kw):
    h = math.pi / 2
    return oracle.Sim(x0=-h, x1=h, y0=-h, y1=h, nx=n, ny=n, bc=1, Re=Re, dt=dt, **kw)


# ----------------------------------------------------------------- grid (Sec. 2.3)

def test_uniform_axis_exact():
    f = oracle.build_axis(-4.0, 8.0, 0, 0, 192, 0.0)
    assert np.array_equal(f, -4.0 + 0.0625 * np.arange(193))


@pytest.mark.parametrize("n,hmin,a0,a1,b0,b1", [(2048, 0.005, -7.5, 24.0, -1.0, 2.0),
                                                  (1024, 0.005, -12.5, 12.5, -0.75, 0.75),
                                                  (97, 0.08, -7.5, 24.0, -1.0, 2.0)])
def test_stretched_axis_is_uniform_block_plus_geometric_sides(n, hmin, a0, a1, b0, b1):
    f = oracle.build_axis(a0, a1, b0, b1, n, hmin)
    assert f[0] == a0 and f[-1] == a1
    s = np.diff(f)
    assert np.all(s > 0)
    nb = int(round((b1 - b0) / hmin))
    nrest = n - nb
    Ll, Lr = b0 - a0, a1 - (b0 + nb * hmin)
    nl = int(round(nrest * Ll / (Ll + Lr)))
    nr = nrest - nl
    # uniform block of spacing hmin starting at b0
    assert abs(f[nl] - b0) < 1e-12
    np.testing.assert_allclose(s[nl:nl + nb], hmin, rtol=1e-9)
    # geometric progression outward on both sides, first cell hmin*r
    left = s[:nl][::-1]
    right = s[nl + nb:]
    for side in (left, right):
        r = side[1:] / side[:-1]
        assert np.all(r >= 1.0)
        np.testing.assert_allclose(r, r[0], rtol=1e-7)
        np.testing.assert_allclose(side[0], hmin * r[0], rtol=1e-9)


def test_axis_rejects_impossible_stretch():
    with pytest.raises(ValueError):
        oracle.build_axis(0.0, 1.0, 0.2, 0.4, 10, 0.01)  # 20 box cells > 10


# ------------------------------------------------------- operators (Sec. 2.2)

def stretched_small(nx=13, ny=9):
    return oracle.Sim(x0=-2.0, x1=3.0, y0=-1.5, y1=2.0, nx=nx, ny=ny, hmin=0.2,
                      ubox=(-0.6, 0.6, -0.4, 0.4), Re=50.0, dt=1e-2)


def test_pressure_laplacian_identities():
    s = stretched_small()
    xf, yf = s.grid()
    V = np.outer(np.diff(yf), np.diff(xf))
    rng = np.random.default_rng(1)
    phi = rng.standard_normal(s.shape("p"))
    psi = rng.standard_normal(s.shape("p"))
    # constants are in the null space (homogeneous Neumann)
    assert np.array_equal(s.lap_p(np.full(s.shape("p"), 3.25)), np.zeros(s.shape("p")))
    # L_p = D G with G zero on boundary faces
    gu, gv = s.grad(phi)
    np.testing.assert_allclose(s.div(gu, gv), s.lap_p(phi), rtol=0, atol=1e-12 * np.abs(s.lap_p(phi)).max())
    # V-weighted symmetry and negative semi-definiteness
    a = np.sum(V * psi * s.lap_p(phi))
    b = np.sum(V * phi * s.lap_p(psi))
    assert abs(a - b) <= 1e-12 * (abs(a) + abs(b))
    assert np.sum(V * phi * s.lap_p(phi)) < 0


def test_velocity_laplacians_on_a_stretched_grid():
    """Finite-volume diffusion of u and v on a stretched grid (Sec. 2.3):
    exact for a quadratic in the direction normal to the node's faces (the
    three-point difference over the control volume's width gives 2 for x^2
    at u nodes and for y^2 at v nodes), and self-adjoint in the
    volume-weighted inner product over the unknowns (fluxes telescope), with
    the Dirichlet columns of u and rows of v held at zero."""
    s = stretched_small(17, 13)
    xf, yf = s.grid()
    xc, yc = 0.5 * (xf[1:] + xf[:-1]), 0.5 * (yf[1:] + yf[:-1])
    Xu, _ = np.meshgrid(xf, yc)
    _, Yv = np.meshgrid(xc, yf)
    Lu, Lv = s.lap_u(Xu ** 2), s.lap_v(Yv ** 2)
    np.testing.assert_allclose(Lu[:, 1:-1], 2.0, rtol=1e-11)
    np.testing.assert_allclose(Lv[1:-1, 1:], 2.0, rtol=1e-11)  # column 0: the inflow wall's v = 0
    Vu = np.outer(np.diff(yf), np.r_[0.0, np.diff(xc), 0.0])  # CV of u node i: [xc_{i-1}, xc_i]
    Vv = np.outer(np.r_[0.0, np.diff(yc), 0.0], np.diff(xf))
    rng = np.random.default_rng(5)
    for shape, lap, V, interior in ((s.shape("u"), s.lap_u, Vu, (slice(None), slice(1, -1))),
                                    (s.shape("v"), s.lap_v, Vv, (slice(1, -1), slice(None)))):
        phi, psi = np.zeros(shape), np.zeros(shape)
        phi[interior] = rng.standard_normal(phi[interior].shape)
        psi[interior] = rng.standard_normal(psi[interior].shape)
        a = np.sum((V * psi * lap(phi))[interior])
        b = np.sum((V * phi * lap(psi))[interior])
        assert abs(a - b) <= 1e-12 * (abs(a) + abs(b)), (a, b)
        assert np.sum((V * phi * lap(phi))[interior]) < 0


def test_convection_cross_terms_on_a_stretched_grid():
    """The cross fluxes of the convection operator interpolate linearly in
    the coordinate (Sec. 2.3 grid; reading 13): with u = 1 and v = x y the
    u-equation's flux divergence d(uv)/dy is x exactly at interior u nodes,
    and with u = x y and v = 1 the v-equation's d(uv)/dx is y exactly at
    interior v nodes, however uneven the spacing."""
    s = stretched_small(17, 13)
    xf, yf = s.grid()
    xc, yc = 0.5 * (xf[1:] + xf[:-1]), 0.5 * (yf[1:] + yf[:-1])
    Xu, Yu = np.meshgrid(xf, yc)
    Xv, Yv = np.meshgrid(xc, yf)
    Hu, _ = s.conv(np.ones(s.shape("u")), Xv * Yv)
    np.testing.assert_allclose(Hu[1:-1, 1:-1], Xu[1:-1, 1:-1], rtol=1e-11, atol=1e-12)
    _, Hv = s.conv(Xu * Yu, np.ones(s.shape("v")))
    np.testing.assert_allclose(Hv[1:-1, 1:-1], Yv[1:-1, 1:-1], rtol=1e-11, atol=1e-12)


def _mms_error(n, stretched):
    # phi = cos(pi x) cos(pi y) on [0,1]^2 has zero normal derivative on the boundary
    if stretched:
        s = oracle.Sim(x0=0.0, x1=1.0, y0=0.0, y1=1.0, nx=n, ny=n, hmin=0.64 / n,
                       ubox=(0.3, 0.6, 0.35, 0.55), dt=1.0)
    else:
        s = oracle.Sim(x0=0.0, x1=1.0, y0=0.0, y1=1.0, nx=n, ny=n, dt=1.0)
    xf, yf = s.grid()
    xc, yc = 0.5 * (xf[1:] + xf[:-1]), 0.5 * (yf[1:] + yf[:-1])
    X, Y = np.meshgrid(xc, yc)
    V = np.outer(np.diff(yf), np.diff(xf))
    exact = np.cos(np.pi * X) * np.cos(np.pi * Y)
    f = -2 * np.pi ** 2 * exact
    f -= np.sum(f * V) / np.sum(V)  # discrete compatibility
    rc, phi, sweeps, res = s.poisson(f, tol=1e-9, check=20)
    assert rc == 0
    e = phi - exact
    e -= np.sum(e * V) / np.sum(V)
    return np.abs(e).max()


@pytest.mark.parametrize("stretched", [False, True])
def test_poisson_manufactured_second_order(stretched):
    e = [_mms_error(n, stretched) for n in (16, 32, 64)]
    orders = [math.log2(e[i] / e[i + 1]) for i in range(2)]
    assert min(orders) > 1.8, (e, orders)


def _dense(op, shape):
    n = int(np.prod(shape))
    A = np.zeros((n, n))
    for k in range(n):
        x = np.zeros(n)
        x[k] = 1.0
        A[:, k] = op(x.reshape(shape)).ravel()
    return A


@pytest.mark.parametrize("nx,ny,stretched", [(7, 5, False), (11, 8, True)])
def test_poisson_sor_matches_dense_solve(nx, ny, stretched):
    if stretched:
        s = oracle.Sim(x0=-2.0, x1=3.0, y0=-1.5, y1=2.0, nx=nx, ny=ny, hmin=0.3,
                       ubox=(-0.6, 0.6, -0.45, 0.45), dt=1.0)
    else:
        s = oracle.Sim(x0=0.0, x1=1.4, y0=0.0, y1=1.0, nx=nx, ny=ny, dt=1.0)
    xf, yf = s.grid()
    V = np.outer(np.diff(yf), np.diff(xf))
    A = _dense(s.lap_p, (ny, nx))
    b = W.random_field((ny, nx), seed=7)
    b -= np.sum(b * V) / np.sum(V)
    x = np.linalg.lstsq(A, b.ravel(), rcond=None)[0].reshape(ny, nx)
    x -= x[0, nx - 1]  # gauge: cell (nx-1, 0) is zero
    rc, phi, sweeps, res = s.poisson(b, tol=1e-13, check=1)
    assert rc == 0 and res <= 1e-13
    assert phi[0, nx - 1] == 0.0
    np.testing.assert_allclose(phi, x, rtol=0, atol=1e-10 * np.abs(x).max())


def test_poisson_reports_noconv_and_nan():
    s = oracle.Sim(x0=0.0, x1=1.0, y0=0.0, y1=1.0, nx=16, ny=16, dt=1.0)
    b = W.random_field((16, 16), seed=3)
    b -= b.mean()
    rc, *_ = s.poisson(b, tol=1e-14, check=1, maxs=3)
    assert rc == -3
    b[4, 5] = np.nan
    rc, *_ = s.poisson(b, tol=1e-8, check=1, maxs=100)
    assert rc == -4


# -------------------------------------------- TG closed forms on the free-slip box

def tg_fields(s, t=0.0, Re=100.0):
    xf, yf = s.grid()
    xc, yc = 0.5 * (xf[1:] + xf[:-1]), 0.5 * (yf[1:] + yf[:-1])
    g = math.exp(-2 * t / Re)
    Xu, Yu = np.meshgrid(xf, yc)
    Xv, Yv = np.meshgrid(xc, yf)
    Xp, Yp = np.meshgrid(xc, yc)
    u = -np.cos(Xu) * np.sin(Yu) * g
    v = np.sin(Xv) * np.cos(Yv) * g
    p = -0.25 * (np.cos(2 * Xp) + np.cos(2 * Yp)) * g * g
    return (Xu, Yu, u), (Xv, Yv, v), (Xp, Yp, p)


def test_convection_and_diffusion_operators_second_order():
    errs = []
    for n in (16, 32, 64):
        s = box_sim(n)
        (Xu, Yu, u), (Xv, Yv, v), _ = tg_fields(s)
        u[:, 0] = u[:, -1] = 0.0
        v[0, :] = v[-1, :] = 0.0
        Hu, Hv = s.conv(u, v)
        # for Taylor-Green, div(uu) = (u.grad)u = (-sin(2x)/2, -sin(2y)/2); lap u = -2u
        eh = max(np.abs(Hu[:, 1:-1] + 0.5 * np.sin(2 * Xu[:, 1:-1])).max(),
                 np.abs(Hv[1:-1, :] + 0.5 * np.sin(2 * Yv[1:-1, :])).max())
        el = max(np.abs(s.lap_u(u)[:, 1:-1] + 2 * u[:, 1:-1]).max(),
                 np.abs(s.lap_v(v)[1:-1, :] + 2 * v[1:-1, :]).max())
        errs.append((eh, el))
    for k in range(2):
        for i in range(2):
            assert math.log2(errs[i][k] / errs[i + 1][k]) > 1.8, errs


def test_uniform_flow_has_zero_convection_and_is_preserved():
    s = oracle.Sim(x0=-2.0, x1=4.0, y0=-1.5, y1=1.5, nx=48, ny=24, hmin=0.1,
                   ubox=(-0.5, 0.5, -0.5, 0.5), Re=100.0, dt=0.01)
    u = np.ones(s.shape("u"))
    v = np.zeros(s.shape("v"))
    Hu, Hv = s.conv(u, v)
    assert np.abs(Hu).max() == 0.0 and np.abs(Hv).max() == 0.0
    s.set("u", u)
    rc, st = s.step(5)
    assert rc == 0
    assert np.abs(s.get("u") - 1.0).max() < 1e-13
    assert np.abs(s.get("v")).max() < 1e-13
    assert st["div_max"] < 1e-12


def _tg_run(n, Re=100.0, T=0.4):
    dt = 0.25 * (math.pi / n)
    steps = int(round(T / dt))
    dt = T / steps
    s = box_sim(n, Re=Re, dt=dt, ptol=1e-12, check_p=4)
    (_, _, u), (_, _, v), (_, _, p) = tg_fields(s, 0.0, Re)
    s.set("u", u)
    s.set("v", v)
    s.set("p", p)
    rc, st = s.step(steps)
    assert rc == 0
    (_, _, ue), (_, _, ve), _ = tg_fields(s, T, Re)
    return max(np.abs(s.get("u") - ue).max(), np.abs(s.get("v") - ve).max()), st


def test_taylor_green_decay_second_order():
    e16, _ = _tg_run(16)
    e32, _ = _tg_run(32)
    e64, st = _tg_run(64)
    assert math.log2(e16 / e32) > 1.7 and math.log2(e32 / e64) > 1.7, (e16, e32, e64)
    assert st["div_max"] <= st["res_p"] * 1.01 * 0.4 / round(0.4 / (0.25 * math.pi / 64)) + 1e-15


def _two_mode_box_run(n, steps, T=0.5, Re=50.0):
    """Free-slip box from a two-mode stream function, sampled at the cell
    corners so that the initial field is discretely divergence-free."""
    s = box_sim(n, Re=Re, dt=T / steps, ptol=1e-12, check_p=4)
    xf, yf = s.grid()
    h = math.pi / 2
    X, Y = np.meshgrid(xf, yf)
    psi = np.sin(X + h) * np.sin(Y + h) + 0.5 * np.sin(2 * (X + h)) * np.sin(Y + h)
    s.set("u", np.diff(psi, axis=0) / np.diff(yf)[:, None])
    s.set("v", -np.diff(psi, axis=1) / np.diff(xf)[None, :])
    rc, st = s.step(steps)
    assert rc == 0
    return s.get("u"), s.get("v")


def test_time_integration_second_order():
    """AB2 convection with Crank-Nicolson diffusion (Sec. 2.2) is second
    order in time: on a fixed 32x32 grid the change between runs to t = 0.5
    with 10, 20, 40 and 80 steps falls by about 4 per halving of dt (first
    order would give 2).  Two stream-function modes make the convection more
    than a gradient, so the projection cannot absorb its time error, as it
    does for the Taylor-Green vortex alone."""
    runs = [_two_mode_box_run(32, m) for m in (10, 20, 40, 80)]
    d = [max(np.abs(a[0] - b[0]).max(), np.abs(a[1] - b[1]).max()) for a, b in zip(runs, runs[1:])]
    assert d[0] / d[1] > 3.5 and d[1] / d[2] > 3.5, d


# ------------------------------------------------- classification (Sec. 2.2)

def _brute_classify(gx, gy, ilo, ihi, jlo, jhi, xb, yb, a, b):
    X, Y = np.meshgrid(gx, gy)
    inside = ((X - xb) / a) ** 2 + ((Y - yb) / b) ** 2 <= 1.0
    mask = np.zeros_like(inside)
    mask[jlo:jhi + 1, ilo:ihi + 1] = True
    solid = inside & mask
    pad = np.pad(solid, 1)
    nb = pad[1:-1, :-2] | pad[1:-1, 2:] | pad[:-2, 1:-1] | pad[2:, 1:-1]
    forcing = (~solid) & nb & mask
    return solid, forcing


def _wall_distance_bisect(x, y, dx, dy, xb, yb, a, b, span):
    # first crossing of the ellipse boundary along the segment, by bisection
    F = lambda s: ((x + s * dx - xb) / a) ** 2 + ((y + s * dy - yb) / b) ** 2 - 1.0
    lo, hi = 0.0, span
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if F(mid) > 0:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


@pytest.mark.parametrize("t", [0.0, 0.37, 1.3])
def test_classification_matches_brute_force(t):
    c = W.plunge_192x128()
    s = oracle.Sim(x0=c.x0, x1=c.x1, y0=c.y0, y1=c.y1, nx=c.nx, ny=c.ny, Re=c.Re, dt=c.dt)
    s.set_body(c.chord, c.tc, c.h, c.k, c.xc, c.yc)
    s.classify(t)
    yb = c.yc + c.h * math.sin(c.k * t)  # Eq. 1
    a, b = 0.5 * c.chord, 0.5 * c.tc * c.chord
    xf, yf = s.grid()
    xc, yc = 0.5 * (xf[1:] + xf[:-1]), 0.5 * (yf[1:] + yf[:-1])
    nx, ny = c.nx, c.ny
    for grid, gx, gy, rng in ((0, xf, yc, (1, nx - 1, 0, ny - 1)), (1, xc, yf, (0, nx - 1, 1, ny - 1))):
        fl, dr, al = s.flags(grid)
        solid, forcing = _brute_classify(gx, gy, *rng, c.xc, yb, a, b)
        assert np.array_equal(fl == 1, solid)
        assert np.array_equal(fl == 2, forcing)
        assert forcing.sum() > 10
        for j, i in zip(*np.nonzero(forcing)):
            steps = [(-1, 0), (1, 0), (0, -1), (0, 1)]
            dists = []
            for d, (di, dj) in enumerate(steps):
                ii, jj = i + di, j + dj
                if 0 <= jj < len(gy) and 0 <= ii < len(gx) and solid[jj, ii]:
                    span = abs(gx[ii] - gx[i]) + abs(gy[jj] - gy[j])
                    dists.append((_wall_distance_bisect(gx[i], gy[j], di, dj, c.xc, yb, a, b, span), d))
            best = min(dists)
            assert dr[j, i] == best[1] or abs(best[0] - [x for x in dists if x[1] == dr[j, i]][0][0]) < 1e-12
            di, dj = steps[dr[j, i]]
            oi, oj = i - di, j - dj
            opp_ok = (rng[0] <= oi <= rng[1] and rng[2] <= oj <= rng[3]
                      and not solid[oj, oi] and not forcing[oj, oi])
            if not opp_ok:
                assert al[j, i] == 0.0
            else:
                D = abs(gx[oi] - gx[i]) + abs(gy[oj] - gy[j])
                np.testing.assert_allclose(al[j, i], best[0] / (best[0] + D), rtol=1e-9, atol=1e-12)


def test_solid_area_converges_first_order():
    # solid u-node area -> pi a b for the 0.12 ellipse; error O(h)
    errs = []
    for n in (64, 128, 256):
        s = oracle.Sim(x0=-1.0, x1=1.0, y0=-0.5, y1=0.5, nx=n, ny=n // 2, dt=1.0)
        s.set_body(1.0, 0.12, 0.0, 0.0, 0.013, 0.007)
        fl, _, _ = s.flags(0)
        xf, yf = s.grid()
        dxc = np.diff(0.5 * (xf[1:] + xf[:-1]))
        area = np.sum((fl[:, 1:-1] == 1) * np.outer(np.diff(yf), dxc))
        errs.append(abs(area - math.pi * 0.5 * 0.06) / (math.pi * 0.5 * 0.06))
    assert errs[2] < errs[0] / 2.5 and errs[2] < 0.05, errs


def test_solid_nodes_carry_body_velocity_eq2():
    c = W.small_cases()[0]
    s = oracle.Sim(x0=c.x0, x1=c.x1, y0=c.y0, y1=c.y1, nx=c.nx, ny=c.ny, Re=c.Re, dt=c.dt,
                   ptol=1e-8 / c.dt)
    s.set_body(c.chord, 0.3, c.h, c.k, c.xc, c.yc)
    for n in range(1, 4):
        rc, st = s.step(1)
        assert rc == 0
        t = n * c.dt
        fv, _, _ = s.flags(1)
        vh = s.get("vh")
        assert (fv == 1).sum() > 0
        np.testing.assert_array_equal(vh[fv == 1], c.k * c.h * math.cos(c.k * t))  # Eq. 2
        fu, _, _ = s.flags(0)
        assert np.all(s.get("uh")[fu == 1] == 0.0)


# -------------------------------------- implicit velocity solve vs dense solve

@pytest.mark.parametrize("grid", [0, 1])
def test_velocity_sor_matches_dense_solve(grid):
    s = oracle.Sim(x0=-1.0, x1=1.5, y0=-0.6, y1=0.6, nx=25, ny=12, Re=20.0, dt=0.02, htol=1e-14,
                   check_h=1, omega_h=1.2)
    s.set_body(1.0, 0.35, 0.1, 2.0, 0.0, 0.0)
    s.classify(0.3)
    beta = s.P.dt / (2 * s.P.Re)
    Ub = 0.0 if grid == 0 else 0.7
    name = "u" if grid == 0 else "v"
    shp = s.shape(name)
    fl, dr, al = s.flags(grid)
    R = W.random_field(shp, seed=11 + grid)
    x0 = W.random_field(shp, seed=21 + grid, scale=0.1)
    # boundary values (Dirichlet, held fixed by the solve)
    if grid == 0:
        x0[:, 0], x0[:, -1] = 1.0, 0.9
        bmask = np.zeros(shp, bool)
        bmask[:, 0] = bmask[:, -1] = True
    else:
        x0[0, :] = x0[-1, :] = 0.0
        bmask = np.zeros(shp, bool)
        bmask[0, :] = bmask[-1, :] = True
    x0[fl == 1] = Ub
    lap = s.lap_u if grid == 0 else s.lap_v
    n = x0.size
    A = np.eye(n) - beta * _dense(lap, shp)
    rhs = R.ravel().copy()
    steps = [(-1, 0), (1, 0), (0, -1), (0, 1)]
    for k in range(n):
        j, i = divmod(k, shp[1])
        if bmask[j, i] or fl[j, i] == 1:
            A[k, :] = 0.0
            A[k, k] = 1.0
            rhs[k] = x0[j, i]
        elif fl[j, i] == 2:
            A[k, :] = 0.0
            A[k, k] = 1.0
            a = al[j, i]
            di, dj = steps[dr[j, i]]
            if a != 0.0:
                A[k, (j - dj) * shp[1] + (i - di)] = -a
            rhs[k] = (1.0 - a) * Ub
    # the operator rows of fluid nodes next to the boundary already use x0's
    # boundary columns; keep them as unknowns fixed by their identity rows
    ref = np.linalg.solve(A, rhs).reshape(shp)
    rc, x, sweeps, res = s.helm_solve(grid, R, x0, beta, Ub)
    assert rc == 0 and res <= 1e-14
    assert (fl == 2).sum() > 0
    np.testing.assert_allclose(x, ref, rtol=0, atol=1e-12)


# ------------------------------------------------------- whole-step properties

def test_step_divergence_bound_and_zero_net_mass_source_in_body_cells():
    for c in W.small_cases():
        s = oracle.Sim(x0=c.x0, x1=c.x1, y0=c.y0, y1=c.y1, nx=c.nx, ny=c.ny, hmin=c.hmin,
                       ubox=c.ubox, Re=c.Re, dt=c.dt, ptol=1e-9 / c.dt, check_p=c.check_p)
        s.set_body(c.chord, c.tc, c.h, c.k, c.xc, c.yc)
        for _ in range(3):
            rc, st = s.step(1)
            assert rc == 0
            cut = s.flags(2).astype(bool)
            d = s.div(s.get("u"), s.get("v"))
            assert np.abs(d[~cut]).max() == st["div_max"]
            assert st["div_max"] <= c.dt * st["res_p"] * (1 + 1e-3) + 1e-13
            assert st["div_max"] <= 1e-9 * (1 + 1e-3)
            xf, yf = s.grid()
            V = np.outer(np.diff(yf), np.diff(xf))
            q = s.get("q")
            assert np.all(q[~cut] == 0.0)
            assert abs(np.sum(q * V)) < 1e-12 * max(1.0, np.abs(q).max())
            # b = (D uhat - q)/dt and the net source over the domain vanishes
            np.testing.assert_allclose(s.get("b"), (s.get("D") - q) / c.dt, rtol=1e-14, atol=1e-12)


def test_stationary_body_in_quiescent_box_stays_at_rest():
    s = oracle.Sim(x0=-1.0, x1=1.0, y0=-1.0, y1=1.0, nx=40, ny=40, bc=1, Re=100.0, dt=0.01)
    s.set_body(1.0, 0.2, 0.0, 0.0, 0.0, 0.0)
    rc, st = s.step(3)
    assert rc == 0
    for f in ("u", "v", "p"):
        assert np.abs(s.get(f)).max() == 0.0
    cl, cd = s.forces()
    assert np.all(cl == 0.0) and np.all(cd == 0.0)


def test_paper_parameters_fixture():
    """Sec. 2.3 / Sec. 4.1 values kept in tests/golden/paper_parameters.txt."""
    import os
    vals = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", "paper_parameters.txt")) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if line:
                k, v = line.split("=")
                vals[k.strip()] = float(v)
    assert W.PAPER_DOMAIN == (vals["x0"], vals["x1"], vals["y0"], vals["y1"])
    # Eq. 2: peak plunge velocity k*h of the validation case, quoted as ~1.0
    assert abs(vals["k_validation"] * vals["h_validation"] - vals["kh_quoted"]) < 0.01


def test_plunging_circle_feels_added_mass_force():
    """Force formula (Sec. 4.1 lift/drag): a circle of diameter 1 plunging with
    small amplitude in fluid at rest feels the potential-flow added-mass force
    F_y = -rho pi a^2 y'' (a = 0.5), i.e. C_l = 2 pi a^2 k^2 h sin(k t) with
    y = h sin(k t) (Eq. 1).  At D/25 resolution in an 8D box at Re 1000 the
    discrete value sits above the potential one (thick staggered body, box
    blockage, viscous layer); halving the spacing was seen to reduce the excess
    from 27 % to 16 %."""
    h, k, dt = 0.05, 2 * math.pi, 0.01
    s = oracle.Sim(x0=-4, x1=4, y0=-4, y1=4, nx=96, ny=96, hmin=0.04,
                   ubox=(-0.75, 0.75, -0.75, 0.75), bc=1, Re=1000.0, dt=dt, ptol=1e-6 / dt, check_p=8)
    s.set_body(1.0, 1.0, h, k, 0.0, 0.0)
    n = int(round(1.0 / dt))
    rc, st = s.step(n)
    assert rc == 0
    cl, cd = s.forces()
    t = dt * np.arange(1, n + 1)
    m = t > 0.25
    A = np.c_[np.sin(k * t[m]), np.cos(k * t[m])]
    cs, cc = np.linalg.lstsq(A, cl[m], rcond=None)[0]
    pot = 2 * math.pi * 0.25 * k * k * h
    assert 1.05 < cs / pot < 1.4, cs / pot
    assert abs(cc) < 0.2 * cs
    # the circle is symmetric about y = 0: no mean drag beyond noise
    assert abs(np.mean(cd[m])) < 0.1 * pot


def test_steady_cylinder_drag_re40():
    """Drag (Sec. 4.1 histories, C_d = 2 F_x / (rho U^2 c)): steady flow past a
    fixed circular cylinder of diameter 1 at Re 40.  Published steady-state
    values for an unbounded domain: C_d = 1.522 (Dennis & Chang 1970, J. Fluid
    Mech. 42, finite differences) and 1.498 (Fornberg 1980, J. Fluid Mech. 98).
    Here the cylinder sits in a 30 x 24 box with free-slip side walls (blockage
    1/24, which raises the drag by a few per cent) at 16 cells per diameter;
    from the uniform start the drag falls towards its steady value (measured
    1.626 at t = 20, 1.614 at t = 30; 1.607 at 24 cells per diameter).  The pin
    asks for 1.522 within 15 % at t = 20, a drag that is still falling, and no
    lift on the symmetric body."""
    import os
    dt = 0.02
    s = oracle.Sim(x0=-10.0, x1=20.0, y0=-12.0, y1=12.0, nx=128, ny=96, hmin=0.0625,
                   ubox=(-0.75, 1.5, -0.75, 0.75), bc=0, Re=40.0, dt=dt, ptol=1e-6 / dt, check_p=8,
                   threads=min(8, os.cpu_count() or 1))
    s.set_body(1.0, 1.0, 0.0, 0.0, 0.0, 0.0)
    s.set("u", np.ones(s.shape("u")))
    rc, st = s.step(1000)
    assert rc == 0
    cl, cd = s.forces()
    cd_end = cd[-50:].mean()
    assert abs(cd_end - 1.522) <= 0.15 * 1.522, cd_end
    assert cd[-500] > cd[-250] > cd[-1]
    assert np.abs(cl[-500:]).max() < 1e-3
