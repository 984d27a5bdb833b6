"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

None of these tests re-types an oracle formula: each compares the oracle with a
different route to the same quantity (the recursive form-factor definition by
quadrature, an identity, a closed-form trajectory, a brute-force integration of
a moving cloud, the textbook Yee dispersion relation, numpy's stable sort).
Section and equation names refer to Sokolov, arXiv:1101.0809.
"""
import itertools
import math

import numpy as np
import pytest
from scipy import integrate

import oracle as O
from paper_1101_0809_gb300 import workloads as W

RNG = np.random.default_rng(20110101)


# --- independent textbook pieces used by several pins ----------------------------
def tent(r):
    """Centred B-spline of degree 1 (support [-1, 1])."""
    return max(0.0, 1.0 - abs(r))


def quad_spline(r):
    """Centred B-spline of degree 2 (support [-3/2, 3/2])."""
    r = abs(r)
    if r <= 0.5:
        return 0.75 - r * r
    if r <= 1.5:
        return 0.5 * (1.5 - r) ** 2
    return 0.0


def tent_cdf(r):
    """Integral of the degree-1 B-spline from -inf to r."""
    if r <= -1.0:
        return 0.0
    if r <= 0.0:
        return 0.5 * (1.0 + r) ** 2
    if r <= 1.0:
        return 1.0 - 0.5 * (1.0 - r) ** 2
    return 1.0


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


def interp_alternating(F, stag, xp, dims):
    """Interpolate grid function F (nz, ny, nx) at xp with the alternating-order
    form factor built from its definition (Sec. 4.5): the weight of a grid point
    is f^(1) = tent at integer points and f^(2) = quad_spline at half-integer
    points; ``stag`` gives the point's offset (0 or 1/2) per axis."""
    nz, ny, nx = F.shape
    n = (nx, ny, nz)
    total = 0.0
    rng_ax = []
    for a in range(dims):
        base = math.floor(xp[a])
        idx = range(base - 2, base + 3)
        fn = tent if stag[a] == 0.0 else quad_spline
        rng_ax.append([(i, fn(i + stag[a] - xp[a])) for i in idx])
    if dims == 2:
        rng_ax.append([(0, 1.0)])
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
            cell = RNG.integers(0, g.n[a])
            x[a] = cell + RNG.uniform(margin, 1.0 - margin)
        xs.append(x)
    return xs


GRID3 = O.Grid(3, (6, 5, 7), (1.0, 1.3, 0.8), 0.3, 1.0)
GRID2 = O.Grid(2, (7, 6, 1), (1.0, 1.3, 1.0), 0.3, 1.0)


# --- P1: closed-form l_a = 1 1/2 values against the recursive definition --------
def _f_recursive(l, r):
    """f^(l)(r) from f^(0) = unit cap and f^(l+1)(r) = int_{r-1/2}^{r+1/2} f^(l) (Sec. 3.1)."""
    if l == 0:
        return 1.0 if abs(r) <= 0.5 else 0.0
    knots = [k * 0.5 for k in range(-2 * l, 2 * l + 1)]
    pts = [p for p in knots if r - 0.5 < p < r + 0.5]
    val, _ = integrate.quad(lambda s: _f_recursive(l - 1, s), r - 0.5, r + 0.5,
                            points=pts or None, epsabs=1e-14, epsrel=1e-14, limit=200)
    return val


@pytest.mark.parametrize("xp", [0.0, 0.13, 0.5, 0.77, 3.999, 12.25])
def test_p1_form_factor_matches_recursive_definition(xp):
    i, f, dF = O.form_factor(xp)
    assert i == math.floor(xp)
    # f_i = f^(1)(i - x_p) at the integer points i, i+1
    for a in range(2):
        assert f[a] == pytest.approx(_f_recursive(1, i + a - xp), abs=1e-12)
    # dF_{i+1/2} = f^(2)(i+1/2 - x_p) at i-1/2, i+1/2, i+3/2 ...
    for b in range(3):
        assert dF[b] == pytest.approx(_f_recursive(2, i - 0.5 + b - xp), abs=1e-12)
        # ... which is also the cell integral of f^(1) (Eq. intff)
        cell = i - 1 + b
        integral, _ = integrate.quad(lambda s: tent(s - xp), cell, cell + 1,
                                     points=[xp - 1, xp, xp + 1], epsabs=1e-14)
        assert dF[b] == pytest.approx(integral, abs=1e-12)
    # Eq. sum1: both families sum to one
    assert f.sum() == pytest.approx(1.0, abs=1e-15)
    assert dF.sum() == pytest.approx(1.0, abs=1e-15)


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


# --- P3/P4: alpha weights against the textbook interpolation and the electrostatic
# limit; beta weights against B = curl_p A (Eqs. egradphidis, A, viaA, A2B) ------------
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
    # Eq. egradphidis: E^(x)_{i,j+1/2,k+1/2} = (Phi_{i-1/2} - Phi_{i+1/2})/dx, Phi[i] at i+1/2
    E = [(np.roll(phi, 1, axis=2) - phi) / d[0], (np.roll(phi, 1, axis=1) - phi) / d[1],
         ((np.roll(phi, 1, axis=0) - phi) / d[2]) if g.dims == 3 else np.zeros(g.shape)]
    Bz = [np.zeros(g.shape) for _ in range(3)]
    phi_at = lambda x: interp_alternating(phi, (0.5, 0.5, 0.5), x, g.dims)
    for xp in random_positions(g, 30, margin=0.05):
        Ep, _ = O.gather(g, E, Bz, xp)
        grad = _fd_grad(phi_at, xp)
        expect = np.array([-grad[a] / d[a] for a in range(3)])
        if g.dims == 2:
            expect[2] = 0.0
        np.testing.assert_allclose(Ep, expect, rtol=0, atol=1e-8)
        # and each component equals the textbook alternating-order interpolation
        for a in range(3):
            assert Ep[a] == pytest.approx(interp_alternating(E[a], E_STAG[a], xp, g.dims),
                                          abs=1e-13)


@pytest.mark.parametrize("g", [GRID3, GRID2], ids=["3d", "2d"])
def test_p4_gathered_B_is_curl_of_interpolated_A(g):
    A = [RNG.normal(size=g.shape) for _ in range(3)]
    d = g.d
    if g.dims == 3:
        dz = lambda F: (F - np.roll(F, 1, axis=0)) / d[2]
    else:
        dz = lambda F: np.zeros(g.shape)
    dy = lambda F: (F - np.roll(F, 1, axis=1)) / d[1]
    dx = lambda F: (F - np.roll(F, 1, axis=2)) / d[0]
    # Eq. viaA on the staggered grid (A sits on the E points)
    B = [dy(A[2]) - dz(A[1]), dz(A[0]) - dx(A[2]), dx(A[1]) - dy(A[0])]
    E0 = [np.zeros(g.shape) for _ in range(3)]
    A_at = [lambda x, a=a: interp_alternating(A[a], E_STAG[a], x, g.dims) for a in range(3)]
    for xp in random_positions(g, 30, margin=0.05):
        _, Bp = O.gather(g, E0, B, xp)
        gA = [_fd_grad(A_at[a], xp) for a in range(3)]   # gA[a][b] = d A_a / d x_b
        curl = np.array([gA[2][1] / d[1] - gA[1][2] / d[2],
                         gA[0][2] / d[2] - gA[2][0] / d[0],
                         gA[1][0] / d[0] - gA[0][1] / d[1]])
        np.testing.assert_allclose(Bp, curl, rtol=0, atol=1e-8)
        for a in range(3):
            assert Bp[a] == pytest.approx(interp_alternating(B[a], B_STAG[a], xp, g.dims),
                                          abs=1e-13)


# --- P5: per-particle continuity equation and the exact sum rule ----------------------
def _random_move(g, cmax=0.9):
    x0 = random_positions(g, 1)[0]
    ubc = RNG.normal(size=3)
    ubc *= RNG.uniform(0.0, 0.99) / np.linalg.norm(ubc)      # |u|/c < 1
    cN = [g.c * g.dt / g.d[a] for a in range(3)]
    x1 = [x0[a] + ubc[a] * cN[a] for a in range(3)]
    if g.dims == 2:
        x1[2] = x0[2]
    return x0, x1, ubc * g.c


def _grid_cfl(dims, cmax):
    # Courant numbers up to cmax on every axis
    d = (1.0, 1.3, 0.8)
    return O.Grid(dims, (7, 6, 5) if dims == 3 else (7, 6, 1), d, cmax * min(d[:dims]), 1.0)


@pytest.mark.parametrize("dims", [3, 2])
def test_p5_continuity_and_sum_rule(dims):
    g = _grid_cfl(dims, 0.9)
    V = g.volume
    for _ in range(200):
        x0, x1, u = _random_move(g)
        J = g.zeros()
        closure = O.deposit(g, x0, x1, u, 1.0, J)
        assert closure < 1e-14
        xw = list(x1)
        xw = [xw[a] % g.n[a] if a < dims else xw[a] for a in range(3)]
        r0 = O.rho(g, np.array(x0).reshape(3, 1), 1.0)
        r1 = O.rho(g, np.array(xw).reshape(3, 1), 1.0)
        div = (np.roll(J[0], -1, axis=2) - J[0]) / g.d[0] + (np.roll(J[1], -1, axis=1) - J[1]) / g.d[1]
        if dims == 3:
            div += (np.roll(J[2], -1, axis=0) - J[2]) / g.d[2]
        # Eq. chargelaw: (rho^n - rho^{n+1})/dt = div J
        np.testing.assert_allclose((r0 - r1) / g.dt, div, rtol=0, atol=1e-13)
        # sum over faces of xi = u (Sec. 3.2), with J = (q/V) xi and q = 1
        for a in range(3):
            assert J[a].sum() * V == pytest.approx(u[a], abs=1e-13)
        # total charge of the single particle is one
        assert r1.sum() * V == pytest.approx(1.0, abs=1e-14)


# --- P6 / P9: the deposit against the six-path form and a brute-force integration
# of the cloud's charge crossing each face along the six box paths (Eqs. Jx-Jz) -------
def _xi_bruteforce(g, x0, x1, u):
    """xi on the faces from the definition: the cloud tent(x)tent(y)tent(z) moves
    along each of the six axis-parallel box paths x^n -> x^{n+1}; the charge that
    crosses a face during a leg is the cloud weight of the offsets that cross it,
    integrated exactly on the polynomial pieces.  Averaged over the six paths."""
    dims = g.dims
    out = [dict() for _ in range(3)]

    def frac_cell(j, y):          # cloud fraction in cell [j, j+1] for a cloud at y
        return piecewise_integral(lambda s: tent(s - y), j, j + 1, [y - 1, y, y + 1])

    def crossing(i, a, b):        # net fraction crossing face i on a leg a -> b
        if b > a:
            return piecewise_integral(tent, i - b, i - a, [-1, 0, 1])
        return -piecewise_integral(tent, i - a, i - b, [-1, 0, 1])

    legs = list(range(3))
    orders = list(itertools.permutations(legs))
    for order in orders:
        pos = list(x0)
        for ax in order:
            a, b = pos[ax], x1[ax]
            if ax < dims:
                lo, hi = math.floor(min(a, b)) - 1, math.floor(max(a, b)) + 2
                others = [o for o in range(dims) if o != ax]
                ranges = [range(math.floor(pos[o]) - 1, math.floor(pos[o]) + 2) for o in others]
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
                # 2D: the z leg of the path; summed over all z faces its flux is the
                # z displacement, i.e. u_z dt / dz in normalized units
                for i in range(math.floor(pos[0]) - 1, math.floor(pos[0]) + 2):
                    for j in range(math.floor(pos[1]) - 1, math.floor(pos[1]) + 2):
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
    # crossing 0, 1, 2 or 3 cell faces
    for trial in range(40):
        x0, x1, u = _random_move(g)
        J = g.zeros()
        O.deposit(g, x0, x1, u, 1.0, J)
        xi = [J[a] * g.volume for a in range(3)]
        ref = _to_grid(g, _xi_bruteforce(g, x0, x1, u))
        for a in range(3):
            np.testing.assert_allclose(xi[a], ref[a], rtol=0, atol=1e-12,
                                       err_msg=f"component {a}, trial {trial}")


def test_p6_deposit_equals_six_path_closed_form():
    g = _grid_cfl(3, 0.9)
    for _ in range(60):
        x0, x1, u = _random_move(g)
        J = g.zeros()
        O.deposit(g, x0, x1, u, 1.0, J)
        ref = g.zeros()
        for ax in range(3):
            o1, o2 = [o for o in range(3) if o != ax]
            for i in range(math.floor(min(x0[ax], x1[ax])) - 2, math.floor(max(x0[ax], x1[ax])) + 3):
                dFi = tent_cdf(i - x1[ax]) - tent_cdf(i - x0[ax])
                for j in range(math.floor(min(x0[o1], x1[o1])) - 2, math.floor(max(x0[o1], x1[o1])) + 3):
                    for k in range(math.floor(min(x0[o2], x1[o2])) - 2, math.floor(max(x0[o2], x1[o2])) + 3):
                        a1, a0 = quad_spline(j + 0.5 - x1[o1]), quad_spline(j + 0.5 - x0[o1])
                        b1, b0 = quad_spline(k + 0.5 - x1[o2]), quad_spline(k + 0.5 - x0[o2])
                        xi = -(1 / 6) * g.d[ax] / g.dt * dFi * (2 * (a1 * b1 + a0 * b0) + a1 * b0 + a0 * b1)
                        idx = [0, 0, 0]
                        idx[ax], idx[o1], idx[o2] = i, j, k
                        ref[ax][idx[2] % g.n[2], idx[1] % g.n[1], idx[0] % g.n[0]] += xi
        for a in range(3):
            np.testing.assert_allclose(J[a] * g.volume, ref[a], rtol=0, atol=1e-12)


# --- P8: telescoping of the x-current of a particle moving along x, and the 1D
# self-energy closed form sum (F_i - 1/2)^2/2 = 1/8 + d^2(1-d)^2/4 (Sec. 4.4) ----------
@pytest.mark.parametrize("d_final", [0.0, 0.25, 0.5, 0.7])
def test_p8_telescoped_current_gives_F_and_self_energy(d_final):
    g = O.Grid(3, (16, 5, 5), (1.0, 1.0, 1.0), 0.5, 1.0)
    x0 = [1.5, 2.3, 2.6]
    steps = 12
    xN = 5.0 + d_final
    J = g.zeros()
    acc = np.zeros(g.shape)
    x = list(x0)
    for n in range(steps):
        nxt = [x0[0] + (xN - x0[0]) * (n + 1) / steps, x0[1], x0[2]]
        u = [(nxt[0] - x[0]) * g.d[0] / g.dt, 0.0, 0.0]
        for a in range(3):
            J[a][:] = 0.0
        O.deposit(g, x, nxt, u, 1.0, J)
        acc += J[0] * g.volume * g.dt / g.d[0]
        x = nxt
    # summed over the transverse cells the telescoped flux is -(F_i(x_N) - F_i(x_0))
    flux = acc.sum(axis=(0, 1))
    for i in range(16):
        expect = -(tent_cdf(i - xN) - tent_cdf(i - x0[0]))
        assert flux[i] == pytest.approx(expect, abs=1e-13)
    # F_i(x_0) = 1 for faces i >= 3, so F_i(x_N) = 1 - flux_i there
    J0 = 5
    F = [1.0 - flux[J0], 1.0 - flux[J0 + 1]]
    self_energy = sum((Fi - 0.5) ** 2 / 2 for Fi in F)
    assert self_energy == pytest.approx(1 / 8 + 0.25 * d_final ** 2 * (1 - d_final) ** 2, abs=1e-13)


# --- P10: uniform E, hyperbolic motion ------------------------------------------------
def test_p10_uniform_E_momentum_exact_and_hyperbolic_trajectory():
    c, qm, E0 = 1.0, -1.0, -1.0          # force q E / m = +1 along x
    a = qm * E0
    T = 2.0
    errs = []
    for dt in (0.01, 0.005):
        g = O.Grid(3, (8, 8, 8), (1.0, 1.0, 1.0), dt, c)
        w = np.array([-0.5 * a * dt, 0.0, 0.0])    # w(t) = a t exactly
        x = np.array([0.0, 0.0, 0.0])
        nsteps = int(round(T / dt))
        for n in range(nsteps):
            w = O.boris(w, [E0, 0, 0], [0, 0, 0], qm, dt, c)
            np.testing.assert_allclose(w[0], a * (n + 0.5) * dt, rtol=1e-13)
            x1, _ = O.move(g, w, x)
            x = x1
        t = nsteps * dt
        exact = (c * c / a) * (math.sqrt(1 + (a * t / c) ** 2) - 1) / g.d[0]
        errs.append(abs(x[0] - exact))
    ratio = errs[0] / errs[1]
    assert 3.5 < ratio < 4.5          # second order in dt


# --- P11: uniform B gyration ----------------------------------------------------------
def test_p11_uniform_B_gyration_closed_form():
    c, qm = 1.0, -1.0
    B0 = 10.0                             # omega_Be = |q| B / (m c) = 10 (Sec. 5)
    dt = 0.25 / B0
    g = O.Grid(3, (64, 64, 8), (0.05, 0.05, 0.05), dt, c)
    w = np.array([0.5 * c, 0.0, 0.0])     # w = 0.5 c (Sec. 5)
    x = np.array([32.0, 32.0, 4.0])
    w0 = np.linalg.norm(w)
    gamma = math.sqrt(w0 ** 2 + c * c)
    bmag = abs(0.5 * qm * dt * B0 / gamma)
    theta = 2 * math.atan(bmag)
    pts = [x.copy()]
    prev = w.copy()
    for n in range(60):
        w = O.boris(w, [0, 0, 0], [0, 0, B0], qm, dt, c)
        assert np.linalg.norm(w) == pytest.approx(w0, rel=1e-14)
        ang = math.atan2(prev[0] * w[1] - prev[1] * w[0], prev[0] * w[0] + prev[1] * w[1])
        assert abs(ang) == pytest.approx(theta, rel=1e-12)
        prev = w.copy()
        x, _ = O.move(g, w, x)
        pts.append(x.copy())
    pts = np.array(pts)[:, :2] * g.d[0]
    u = c * w0 / gamma
    R = u * dt / (2 * math.sin(theta / 2))
    # circumcentre of three points, then every point on the circle
    (ax, ay), (bx, by), (cx, cy) = pts[0], pts[7], pts[19]
    dd = 2 * (ax * (by - cy) + bx * (cy - ay) + cx * (ay - by))
    ux = ((ax ** 2 + ay ** 2) * (by - cy) + (bx ** 2 + by ** 2) * (cy - ay) + (cx ** 2 + cy ** 2) * (ay - by)) / dd
    uy = ((ax ** 2 + ay ** 2) * (cx - bx) + (bx ** 2 + by ** 2) * (ax - cx) + (cx ** 2 + cy ** 2) * (bx - ax)) / dd
    radii = np.hypot(pts[:, 0] - ux, pts[:, 1] - uy)
    np.testing.assert_allclose(radii, R, rtol=1e-11)
    # and R equals the Larmor radius times sqrt(1 + b^2) (Boris' known phase error)
    rL = w0 / (abs(qm) * B0)
    assert R == pytest.approx(rL * math.sqrt(1 + bmag ** 2), rel=1e-12)


def test_boris_rotation_angle_takes_gamma_at_the_half_kicked_momentum():
    """With E and B both non-zero, the Appendix's step 2 is a half kick by e, a
    rotation of w~ = w^{n-1/2} + e about B, and a second half kick.  A rotation
    by the vector b (w_n = w~ + w~ x b; w' = w~ + 2 (w_n x b)/(1 + b^2)) is a
    rotation about b by the angle 2 arctan|b| (the Cayley form of a rotation),
    and the Appendix defines |b| with sqrt(w~^2 + c^2), the Lorentz factor of
    the half-kicked momentum.  So the component of w^{n+1/2} - e along B equals
    that of w~, and the angle between their components across B is
    2 arctan(|q dt B / 2m| / sqrt(w~^2 + c^2)), in the sense of -q B.  The
    fields are strong enough that the Lorentz factor of w^{n-1/2} would give an
    angle off by far more than the tolerance."""
    rng = np.random.default_rng(7)
    worst_alt = 0.0
    for _ in range(200):
        c = rng.choice([1.0, 2.0, 20.0])
        qm = rng.choice([-1.0, 1.0 / 1836, 2.0])
        dt = rng.uniform(0.05, 0.5)
        w = rng.normal(size=3) * c
        Ep = rng.normal(size=3) * c / (abs(qm) * dt)      # |e| comparable to |w|
        Bp = rng.normal(size=3) * 3 * c / (abs(qm) * dt)
        w1 = O.boris(w, Ep, Bp, qm, dt, c)
        e = 0.5 * qm * dt * Ep
        wm, wp = w + e, w1 - e
        bh = Bp / np.linalg.norm(Bp)
        scale = np.linalg.norm(wm)
        assert np.dot(wp, bh) == pytest.approx(np.dot(wm, bh), abs=1e-13 * scale)
        pm, pp = wm - np.dot(wm, bh) * bh, wp - np.dot(wp, bh) * bh
        cosang = np.dot(pm, pp)
        sinang = np.dot(np.cross(pm, pp), -np.sign(qm) * bh)
        angle = math.atan2(sinang, cosang)
        half = 0.5 * abs(qm) * dt * np.linalg.norm(Bp)
        want = 2 * math.atan(half / math.sqrt(np.dot(wm, wm) + c * c))
        alt = 2 * math.atan(half / math.sqrt(np.dot(w, w) + c * c))
        assert angle == pytest.approx(want, rel=1e-11, abs=1e-12)
        worst_alt = max(worst_alt, abs(alt - want) / want)
    assert worst_alt > 1e-2      # the test would see the other Lorentz factor


def test_boris_gyration_phase_in_parallel_E_and_B_converges_at_second_order():
    """Uniform E and B both along z: w_z(t) = w_z(0) + (q/m) E t, |w_perp| is
    constant, and w_perp turns at the rate |q| B / (m sqrt(w_perp^2 + w_z(t)^2 + c^2)),
    so the phase turned between t0 and t1 is
    (|q| B / (q E / m)) [asinh(w_z(t1)/s) - asinh(w_z(t0)/s)] with
    s = sqrt(w_perp^2 + c^2) (closed form of the relativistic motion in
    parallel fields).  The push evaluates the rate at the half-kicked momentum
    w~, whose w_z is that of t^n, the centre of the step, so the phase error
    falls as dt^2; a Lorentz factor taken at w^{n-1/2} (time t^{n-1/2}) would
    make it first order."""
    c, qm, B0, E0 = 1.0, -1.0, 2.0, 0.5
    a = qm * E0
    wperp, T = 0.5, 4.0
    s = math.sqrt(wperp ** 2 + c * c)
    errs = []
    for dt in (0.02, 0.01, 0.005):
        nsteps = int(round(T / dt))
        w = np.array([wperp, 0.0, -0.5 * a * dt])          # w^{-1/2}: w_z(t) = a t
        phase = 0.0
        for n in range(nsteps):
            w1 = O.boris(w, [0, 0, E0], [0, 0, B0], qm, dt, c)
            assert w1[2] == pytest.approx(a * (n + 0.5) * dt, rel=1e-13, abs=1e-15)
            assert math.hypot(w1[0], w1[1]) == pytest.approx(wperp, rel=1e-13)
            phase += math.atan2(w[0] * w1[1] - w[1] * w1[0], w[0] * w1[0] + w[1] * w1[1])
            w = w1
        t0, t1 = -0.5 * dt, (nsteps - 0.5) * dt
        turned = (abs(qm) * B0 / a) * (math.asinh(a * t1 / s) - math.asinh(a * t0 / s))
        errs.append(abs(phase - (-np.sign(qm)) * turned))     # charge q < 0 turns counter-clockwise about +B
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5


def test_boris_magnetic_part_preserves_energy_p2():
    for _ in range(100):
        w = RNG.normal(size=3) * 3
        Ep, Bp = RNG.normal(size=3), RNG.normal(size=3) * 5
        qm, dt, c = RNG.choice([-1.0, 1.0 / 1836, 2.0]), 0.3, 2.0
        w1 = O.boris(w, Ep, Bp, qm, dt, c)
        e = 0.5 * qm * dt * Ep
        # Eq. p2: (w^{n+1/2} - e)^2 = (w^{n-1/2} + e)^2
        assert np.dot(w1 - e, w1 - e) == pytest.approx(np.dot(w + e, w + e), rel=1e-13)


# --- P12: Yee in vacuum: discrete plane waves and div B ---------------------------------
def _levi(a, b, t):
    return {(0, 1, 2): 1, (1, 2, 0): 1, (2, 0, 1): 1}.get((a, b, t), -1)


@pytest.mark.parametrize("dims", [3, 2])
def test_p12_yee_plane_waves_obey_discrete_dispersion(dims):
    n = (12, 10, 8) if dims == 3 else (12, 10, 1)
    g = O.Grid(dims, n, (1.0, 1.2, 0.9), 0.35, 1.0)
    for a in range(dims):                         # propagation axis
        for b in range(3):                        # E polarization
            if b == a:
                continue
            t = 3 - a - b
            s = _levi(a, b, t)
            cN = g.c * g.dt / g.d[a]
            k = 2 * math.pi * 2 / n[a]
            om = 2 * math.asin(cN * math.sin(k / 2))   # sin^2(w/2) = c_a^2 sin^2(k/2)
            A = cN * math.sin(k / 2) / math.sin(om / 2)
            idx = np.indices(g.shape)                 # (k, j, i)
            ia = idx[2 - a].astype(float)
            E, B, J = g.zeros(), g.zeros(), g.zeros()
            E[b][:] = np.cos(k * (ia + 0.5))
            B[t][:] = s * A * np.cos(k * ia + om * 0.5)
            for m in range(1, 6):
                O.step(g, E, B, J, [])
                np.testing.assert_allclose(E[b], np.cos(k * (ia + 0.5) - om * m), atol=1e-12)
                np.testing.assert_allclose(B[t], s * A * np.cos(k * ia - om * (m - 0.5)), atol=1e-12)
                for o in range(3):
                    if o not in (b, t):
                        assert np.abs(E[o]).max() < 1e-14 and np.abs(B[o]).max() < 1e-14


def test_p12_div_B_unchanged_by_yee():
    g = O.Grid(3, (8, 7, 6), (1.0, 1.1, 0.9), 0.3, 1.0)
    E = [RNG.normal(size=g.shape) for _ in range(3)]
    B = [RNG.normal(size=g.shape) for _ in range(3)]

    def divB(B):
        # B's divergence lives on the integer nodes: Bx[i] sits at i+1/2, so backward differences
        return ((B[0] - np.roll(B[0], 1, axis=2)) / g.d[0] + (B[1] - np.roll(B[1], 1, axis=1)) / g.d[1]
                + (B[2] - np.roll(B[2], 1, axis=0)) / g.d[2])

    d0 = divB(B)
    for _ in range(5):
        O.yee_half_B(g, E, B)
    np.testing.assert_allclose(divB(B), d0, atol=1e-12)


# --- P7: full-step Gauss law and charge over the small 2D workload ---------------------
def test_p7_gauss_residual_and_charge_conserved_over_50_steps():
    wl = W.c0_small2d()
    g = O.Grid(wl.dims, wl.n, wl.d, wl.dt, wl.c)
    sp = [O.Species(s.q, s.m, s.weight, s.x, s.w) for s in wl.species]
    E, B, J = g.zeros(), g.zeros(), g.zeros()
    d0, _, r0 = O.diagnostics(g, E, B, sp, wl.rho_bg)
    scale = 4 * math.pi * wl.rho_bg               # 4 pi |q_e| n_e
    for n in range(wl.steps):
        closure = O.step(g, E, B, J, sp)
        assert closure < 1e-14
    d, _, r = O.diagnostics(g, E, B, sp, wl.rho_bg)
    assert np.abs(r - r0).max() / scale < 1e-12
    assert abs(d["charge"] - d0["charge"]) < 1e-12
    # the energy integral of Sec. 4.1 stays flat (loose: the paper reports ~1e-5 defects)
    assert abs(d["total"] - d0["total"]) / d0["total"] < 1e-4
    # every particle stays in the box
    for s in sp:
        for a in range(2):
            assert (s.x[a] >= 0).all() and (s.x[a] < wl.n[a]).all()


# --- the stable tile sort -------------------------------------------------------------
def test_sort_is_numpy_stable_argsort():
    g = O.Grid(3, (16, 12, 8), (1.0, 1.0, 1.0), 0.3, 1.0)
    x = np.stack([RNG.uniform(0, g.n[a], 5000) for a in range(3)])
    tile = (4, 5, 3)
    key = O.tile_keys(g, tile, x)
    nt = [math.ceil(g.n[a] / tile[a]) for a in range(3)]
    manual = ((np.floor(x[2]) // tile[2]) * nt[1] + np.floor(x[1]) // tile[1]) * nt[0] + np.floor(x[0]) // tile[0]
    np.testing.assert_array_equal(key, manual.astype(np.int32))
    perm = O.sort_perm(key, nt[0] * nt[1] * nt[2])
    np.testing.assert_array_equal(perm, np.argsort(key, kind="stable"))
