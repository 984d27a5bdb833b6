"""Pins of the oracle's alternating-order form factor l_a = 2 1/2 (Sec. 4.5:
f = f^(2) at integer points, dF = f^(3) at half-integer points, base index
int(x_p + 1/2)) against what the paper and the mathematics fix.  Each pin takes
a route to the same quantity that the oracle does not: the recursive
form-factor definition by quadrature, the textbook centred B-splines of degree
2 and 3, identities of the interpolation (uniform fields, E = -grad Phi,
B = curl A), the continuity equation and sum rule of the deposit, a
brute-force integration of the quadratic cloud's charge crossing each face
along the six box paths, the six-path closed form, and Gauss's law over a run.
"""
import itertools
import math

import numpy as np
import pytest
from scipy import integrate

import oracle as O
from paper_1101_0809_gb300 import workloads as W

RNG = np.random.default_rng(20110105)
ORDER2 = 5


def quad_spline(r):
    """Centred B-spline of degree 2 (support [-3/2, 3/2])."""
    r = abs(r)
    if r <= 0.5:
        return 0.75 - r * r
    if r <= 1.5:
        return 0.5 * (1.5 - r) ** 2
    return 0.0


def cubic_spline(r):
    """Centred B-spline of degree 3 (support [-2, 2])."""
    r = abs(r)
    if r <= 1.0:
        return 2.0 / 3.0 - r * r + 0.5 * r ** 3
    if r <= 2.0:
        return (2.0 - r) ** 3 / 6.0
    return 0.0


_GL_X, _GL_W = np.polynomial.legendre.leggauss(4)


def piecewise_integral(fn, a, b, knots):
    """Gauss-Legendre on every smooth piece of [a, b] split at ``knots``: exact for
    piecewise polynomials of degree <= 7."""
    if b <= a:
        return 0.0
    pts = sorted({a, b, *[k for k in knots if a < k < b]})
    total = 0.0
    for lo, hi in zip(pts[:-1], pts[1:]):
        mid, half = 0.5 * (lo + hi), 0.5 * (hi - lo)
        total += half * sum(wq * fn(mid + half * xq) for xq, wq in zip(_GL_X, _GL_W))
    return total


QKNOTS = [-1.5, -0.5, 0.5, 1.5]


def quad_cdf(r):
    """Integral of the degree-2 B-spline from -inf to r."""
    return piecewise_integral(quad_spline, -1.5, min(max(r, -1.5), 1.5), QKNOTS)


def interp_alternating5(F, stag, xp, dims):
    """Interpolate grid function F (nz, ny, nx) at xp with the l_a = 2 1/2
    alternating-order form factor from its definition: the weight of a grid
    point is f^(2) = quad_spline at integer points and f^(3) = cubic_spline at
    half-integer points; ``stag`` gives the point's offset (0 or 1/2) per axis."""
    nz, ny, nx = F.shape
    n = (nx, ny, nz)
    rng_ax = []
    for a in range(dims):
        base = math.floor(xp[a])
        fn = quad_spline if stag[a] == 0.0 else cubic_spline
        rng_ax.append([(i, fn(i + stag[a] - xp[a])) for i in range(base - 3, base + 4)])
    if dims == 2:
        rng_ax.append([(0, 1.0)])
    total = 0.0
    for (i, wi), (j, wj), (k, wk) in itertools.product(*rng_ax):
        wgt = wi * wj * wk
        if wgt != 0.0:
            total += wgt * F[k % n[2], j % n[1], i % n[0]]
    return total


def random_positions(g, count, margin=0.0):
    xs = []
    for _ in range(count):
        x = [0.0, 0.0, 0.0]
        for a in range(g.dims):
            x[a] = RNG.integers(0, g.n[a]) + RNG.uniform(margin, 1.0 - margin)
        xs.append(x)
    return xs


GRID3 = O.Grid(3, (8, 7, 9), (1.0, 1.3, 0.8), 0.3, 1.0, ORDER2)
GRID2 = O.Grid(2, (9, 8, 1), (1.0, 1.3, 1.0), 0.3, 1.0, ORDER2)


# --- P1: closed-form values against the recursive definition ----------------------
def _f_recursive(l, r):
    """f^(l)(r) from f^(0) = unit cap and f^(l+1)(r) = int_{r-1/2}^{r+1/2} f^(l) (Sec. 3.1)."""
    if l == 0:
        return 1.0 if abs(r) <= 0.5 else 0.0
    knots = [k * 0.5 for k in range(-2 * l, 2 * l + 1)]
    pts = [p for p in knots if r - 0.5 < p < r + 0.5]
    val, _ = integrate.quad(lambda s: _f_recursive(l - 1, s), r - 0.5, r + 0.5,
                            points=pts or None, epsabs=1e-14, epsrel=1e-14, limit=200)
    return val


@pytest.mark.parametrize("xp", [0.0, 0.13, 0.4999, 0.5, 0.77, 3.999, 12.25, 7.5])
def test_p1_form_factor_matches_recursive_definition(xp):
    i, f, dF = O.form_factor(xp, ORDER2)
    assert i == math.floor(xp + 0.5)            # "int(x_p + 1/2)"
    # f_i = f^(2)(i - x_p) at the integer points i-1, i, i+1
    for a in range(3):
        assert f[a] == pytest.approx(_f_recursive(2, i - 1 + a - xp), abs=1e-12)
    # dF_{c+1/2} = f^(3)(c + 1/2 - x_p) over the cells c = i-2 .. i+1 ...
    for b in range(4):
        cell = i - 2 + b
        assert dF[b] == pytest.approx(_f_recursive(3, cell + 0.5 - xp), abs=1e-12)
        # ... which is the cell integral of f^(2) (Eq. intff) and the cubic B-spline
        integral = piecewise_integral(lambda s: quad_spline(s - xp), cell, cell + 1,
                                      [xp + k for k in QKNOTS])
        assert dF[b] == pytest.approx(integral, abs=1e-13)
        assert dF[b] == pytest.approx(cubic_spline(cell + 0.5 - xp), abs=1e-14)
    # Eq. sum1: both families sum to one
    assert f.sum() == pytest.approx(1.0, abs=1e-15)
    assert dF.sum() == pytest.approx(1.0, abs=1e-15)


def test_p1_derivative_identity():
    """d dF_{c+1/2} / d x_p = -(f_{c+1} - f_c) (Sec. 3.1, property (3)), by
    central differences of the oracle's own closed form."""
    for xp in RNG.uniform(0.05, 9.95, 40):
        if abs((xp + 0.5) - round(xp + 0.5)) < 1e-3:
            continue
        h = 1e-6
        i, f, dF = O.form_factor(xp, ORDER2)
        _, _, dp = O.form_factor(xp + h, ORDER2)
        _, _, dm = O.form_factor(xp - h, ORDER2)
        deriv = (dp - dm) / (2 * h)
        fx = np.concatenate([[0.0], f, [0.0]])     # f at i-2 .. i+2 (zero outside)
        for b in range(4):                        # cell c = i-2+b: f_{c+1} - f_c
            assert deriv[b] == pytest.approx(-(fx[b + 1] - fx[b]), abs=1e-8)


# --- P2: uniform fields are reproduced (Eq. one) ------------------------------------
@pytest.mark.parametrize("g", [GRID3, GRID2], ids=["3d", "2d"])
def test_p2_uniform_field_is_reproduced(g):
    e0, b0 = RNG.normal(size=3), RNG.normal(size=3)
    E = [np.full(g.shape, e0[a]) for a in range(3)]
    B = [np.full(g.shape, b0[a]) for a in range(3)]
    for xp in random_positions(g, 50):
        Ep, Bp = O.gather(g, E, B, xp)
        np.testing.assert_allclose(Ep, e0, rtol=0, atol=1e-14)
        np.testing.assert_allclose(Bp, b0, rtol=0, atol=1e-14)


# --- P3/P4: alpha and beta weights (Eqs. egradphidis, viaA) ---------------------------
E_STAG = [(0.0, 0.5, 0.5), (0.5, 0.0, 0.5), (0.5, 0.5, 0.0)]
B_STAG = [(0.5, 0.0, 0.0), (0.0, 0.5, 0.0), (0.0, 0.0, 0.5)]


def _fd_grad(fn, xp, h=1e-5):
    out = []
    for a in range(3):
        xa, xb = list(xp), list(xp)
        xa[a] += h
        xb[a] -= h
        out.append((fn(xa) - fn(xb)) / (2 * h))
    return np.array(out)


@pytest.mark.parametrize("g", [GRID3, GRID2], ids=["3d", "2d"])
def test_p3_gather_is_minus_grad_of_interpolated_potential(g):
    phi = RNG.normal(size=g.shape)
    d = g.d
    E = [(np.roll(phi, 1, axis=2) - phi) / d[0], (np.roll(phi, 1, axis=1) - phi) / d[1],
         ((np.roll(phi, 1, axis=0) - phi) / d[2]) if g.dims == 3 else np.zeros(g.shape)]
    Bz = [np.zeros(g.shape) for _ in range(3)]
    phi_at = lambda x: interp_alternating5(phi, (0.5, 0.5, 0.5), x, g.dims)
    for xp in random_positions(g, 25, margin=0.05):
        Ep, _ = O.gather(g, E, Bz, xp)
        grad = _fd_grad(phi_at, xp)
        expect = np.array([-grad[a] / d[a] for a in range(3)])
        if g.dims == 2:
            expect[2] = 0.0
        np.testing.assert_allclose(Ep, expect, rtol=0, atol=1e-8)
        for a in range(3):
            assert Ep[a] == pytest.approx(interp_alternating5(E[a], E_STAG[a], xp, g.dims), abs=1e-13)


@pytest.mark.parametrize("g", [GRID3, GRID2], ids=["3d", "2d"])
def test_p4_gathered_B_is_curl_of_interpolated_A(g):
    A = [RNG.normal(size=g.shape) for _ in range(3)]
    d = g.d
    dz = (lambda F: (F - np.roll(F, 1, axis=0)) / d[2]) if g.dims == 3 else (lambda F: np.zeros(g.shape))
    dy = lambda F: (F - np.roll(F, 1, axis=1)) / d[1]
    dx = lambda F: (F - np.roll(F, 1, axis=2)) / d[0]
    B = [dy(A[2]) - dz(A[1]), dz(A[0]) - dx(A[2]), dx(A[1]) - dy(A[0])]
    E0 = [np.zeros(g.shape) for _ in range(3)]
    A_at = [lambda x, a=a: interp_alternating5(A[a], E_STAG[a], x, g.dims) for a in range(3)]
    for xp in random_positions(g, 25, margin=0.05):
        _, Bp = O.gather(g, E0, B, xp)
        gA = [_fd_grad(A_at[a], xp) for a in range(3)]
        curl = np.array([gA[2][1] / d[1] - gA[1][2] / d[2],
                         gA[0][2] / d[2] - gA[2][0] / d[0],
                         gA[1][0] / d[0] - gA[0][1] / d[1]])
        np.testing.assert_allclose(Bp, curl, rtol=0, atol=1e-8)
        for a in range(3):
            assert Bp[a] == pytest.approx(interp_alternating5(B[a], B_STAG[a], xp, g.dims), abs=1e-13)


# --- P5: per-particle continuity equation and the exact sum rule ----------------------
def _grid_cfl(dims, cmax):
    d = (1.0, 1.3, 0.8)
    return O.Grid(dims, (9, 8, 7) if dims == 3 else (9, 8, 1), d, cmax * min(d[:dims]), 1.0, ORDER2)


def _random_move(g):
    x0 = random_positions(g, 1)[0]
    ubc = RNG.normal(size=3)
    ubc *= RNG.uniform(0.0, 0.99) / np.linalg.norm(ubc)
    cN = [g.c * g.dt / g.d[a] for a in range(3)]
    x1 = [x0[a] + ubc[a] * cN[a] for a in range(3)]
    if g.dims == 2:
        x1[2] = x0[2]
    return x0, x1, ubc * g.c


@pytest.mark.parametrize("dims", [3, 2])
def test_p5_continuity_and_sum_rule(dims):
    g = _grid_cfl(dims, 0.9)
    V = g.volume
    for _ in range(150):
        x0, x1, u = _random_move(g)
        J = g.zeros()
        closure = O.deposit(g, x0, x1, u, 1.0, J)
        assert closure < 1e-14
        xw = [x1[a] % g.n[a] if a < dims else x1[a] for a in range(3)]
        r0 = O.rho(g, np.array(x0).reshape(3, 1), 1.0)
        r1 = O.rho(g, np.array(xw).reshape(3, 1), 1.0)
        div = (np.roll(J[0], -1, axis=2) - J[0]) / g.d[0] + (np.roll(J[1], -1, axis=1) - J[1]) / g.d[1]
        if dims == 3:
            div += (np.roll(J[2], -1, axis=0) - J[2]) / g.d[2]
        np.testing.assert_allclose((r0 - r1) / g.dt, div, rtol=0, atol=1e-13)
        for a in range(3):
            assert J[a].sum() * V == pytest.approx(u[a], abs=1e-13)
        assert r1.sum() * V == pytest.approx(1.0, abs=1e-14)
        # the charge cloud covers 4 cells per axis
        assert np.count_nonzero(r1) <= 4 ** dims


# --- P9: the deposit against a brute-force integration of the quadratic cloud ---------
def _xi_bruteforce(g, x0, x1, u):
    """xi on the faces from the definition: the cloud f^(2)(x)f^(2)(y)f^(2)(z)
    moves along each of the six axis-parallel box paths x^n -> x^{n+1}; the
    charge that crosses a face during a leg is the cloud weight of the offsets
    that cross it, integrated exactly on the polynomial pieces.  Averaged over
    the six paths."""
    dims = g.dims
    out = [dict() for _ in range(3)]

    def frac_cell(j, y):
        return piecewise_integral(lambda s: quad_spline(s - y), j, j + 1, [y + k for k in QKNOTS])

    def crossing(i, a, b):
        if b > a:
            return piecewise_integral(quad_spline, i - b, i - a, QKNOTS)
        return -piecewise_integral(quad_spline, i - a, i - b, QKNOTS)

    for order in itertools.permutations(range(3)):
        pos = list(x0)
        for ax in order:
            a, b = pos[ax], x1[ax]
            if ax < dims:
                lo, hi = math.floor(min(a, b)) - 2, math.floor(max(a, b)) + 3
                others = [o for o in range(dims) if o != ax]
                ranges = [range(math.floor(pos[o]) - 2, math.floor(pos[o]) + 3) for o in others]
                for i in range(lo, hi + 1):
                    cr = crossing(i, a, b)
                    if cr == 0.0:
                        continue
                    for cells in itertools.product(*ranges):
                        wgt = cr
                        for o, cidx in zip(others, cells):
                            wgt *= frac_cell(cidx, pos[o])
                        key = [0, 0, 0]
                        key[ax] = i
                        for o, cidx in zip(others, cells):
                            key[o] = cidx
                        key = tuple(key)
                        out[ax][key] = out[ax].get(key, 0.0) + wgt / 6.0 * g.d[ax] / g.dt
            else:
                for i in range(math.floor(pos[0]) - 2, math.floor(pos[0]) + 3):
                    for j in range(math.floor(pos[1]) - 2, math.floor(pos[1]) + 3):
                        wgt = frac_cell(i, pos[0]) * frac_cell(j, pos[1])
                        out[2][(i, j, 0)] = out[2].get((i, j, 0), 0.0) + wgt / 6.0 * u[2]
            pos[ax] = b
    return out


def _to_grid(g, xi_dicts):
    F = g.zeros()
    for a in range(3):
        for (i, j, k), v in xi_dicts[a].items():
            F[a][k % g.shape[0], j % g.n[1], i % g.n[0]] += v
    return F


@pytest.mark.parametrize("dims", [3, 2])
def test_p9_deposit_equals_bruteforce_box_path_flux(dims):
    g = _grid_cfl(dims, 0.9)
    for trial in range(12 if dims == 3 else 30):
        x0, x1, u = _random_move(g)
        J = g.zeros()
        O.deposit(g, x0, x1, u, 1.0, J)
        xi = [J[a] * g.volume for a in range(3)]
        ref = _to_grid(g, _xi_bruteforce(g, x0, x1, u))
        for a in range(3):
            np.testing.assert_allclose(xi[a], ref[a], rtol=0, atol=1e-12,
                                       err_msg=f"component {a}, trial {trial}")


def test_p6_deposit_equals_six_path_closed_form():
    """The six-path form of the current (Eqs. Jx-Jz before Eq. current), with F the
    cumulative integral of the quadratic cloud and dF its cell integrals."""
    g = _grid_cfl(3, 0.9)
    for _ in range(30):
        x0, x1, u = _random_move(g)
        J = g.zeros()
        O.deposit(g, x0, x1, u, 1.0, J)
        ref = g.zeros()
        for ax in range(3):
            o1, o2 = [o for o in range(3) if o != ax]
            for i in range(math.floor(min(x0[ax], x1[ax])) - 3, math.floor(max(x0[ax], x1[ax])) + 4):
                dFi = quad_cdf(i - x1[ax]) - quad_cdf(i - x0[ax])
                if dFi == 0.0:
                    continue
                for j in range(math.floor(min(x0[o1], x1[o1])) - 3, math.floor(max(x0[o1], x1[o1])) + 4):
                    for k in range(math.floor(min(x0[o2], x1[o2])) - 3, math.floor(max(x0[o2], x1[o2])) + 4):
                        a1, a0 = cubic_spline(j + 0.5 - x1[o1]), cubic_spline(j + 0.5 - x0[o1])
                        b1, b0 = cubic_spline(k + 0.5 - x1[o2]), cubic_spline(k + 0.5 - x0[o2])
                        xi = -(1 / 6) * g.d[ax] / g.dt * dFi * (2 * (a1 * b1 + a0 * b0) + a1 * b0 + a0 * b1)
                        idx = [0, 0, 0]
                        idx[ax], idx[o1], idx[o2] = i, j, k
                        ref[ax][idx[2] % g.n[2], idx[1] % g.n[1], idx[0] % g.n[0]] += xi
        for a in range(3):
            np.testing.assert_allclose(J[a] * g.volume, ref[a], rtol=0, atol=1e-12)


# --- P7: full-step Gauss law and charge over a small run ------------------------------
@pytest.mark.parametrize("dims", [2, 3])
def test_p7_gauss_residual_and_charge_conserved(dims):
    if dims == 2:
        wl = W.thermal_plasma("2D l_a 2.5", 2, (16, 16, 1), 8, 0.1, 40, W.SEED_BASE + 21)
    else:
        wl = W.thermal_plasma("3D l_a 2.5", 3, (10, 9, 11), 4, 0.1, 15, W.SEED_BASE + 22, ions=1836.0,
                              dt_courant=0.45)
    g = O.Grid(wl.dims, wl.n, wl.d, wl.dt, wl.c, ORDER2)
    sp = [O.Species(s.q, s.m, s.weight, s.x, s.w) for s in wl.species]
    E, B, J = g.zeros(), g.zeros(), g.zeros()
    d0, _, r0 = O.diagnostics(g, E, B, sp, wl.rho_bg)
    e = wl.species[0]
    scale = 4 * math.pi * abs(e.q * e.weight) * e.x.shape[1] / (np.prod(wl.n[:dims]) * g.volume)
    for _ in range(wl.steps):
        assert O.step(g, E, B, J, sp) < 1e-14
    d, _, r = O.diagnostics(g, E, B, sp, wl.rho_bg)
    assert np.abs(E[0]).max() > 0.0                    # the plasma did move
    assert np.abs(r - r0).max() / scale < 1e-12
    assert abs(d["charge"] - d0["charge"]) < 1e-12


def test_adjoint_is_refused_for_l_a_2_5():
    g = O.Grid(2, (9, 8, 1), (1.0, 1.0, 1.0), 0.3, 1.0, ORDER2)
    with pytest.raises(NotImplementedError):
        O.step_adj(g, g.zeros(), g.zeros(), [], g.zeros(), g.zeros(), [], [])
