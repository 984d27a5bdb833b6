"""Pins of the oracle's comparison scheme of Eq. wrong1 (order2 = 4): the
"conventional" uniform-order l = 2 interpolation of Sec. 5, in which the
cell-centred form factor weighs the field averaged over the faces of each cell,
with the l_a = 1 1/2 charge and current (Eq. current).  Routes that the oracle
does not take: the face-averaged field interpolated with the textbook
degree-2 B-spline at cell centres, uniform fields, the deposit equal to the
l_a = 1 1/2 one bit for bit, and the paper's energy observation (Sec. 5,
Fig. 2): with this interpolation the energy integral drifts far more than with
the alternating order."""
import itertools
import math

import numpy as np
import pytest

import oracle as O
from paper_1101_0809_gb300 import workloads as W

RNG = np.random.default_rng(20110106)


def quad_spline(r):
    r = abs(r)
    if r <= 0.5:
        return 0.75 - r * r
    if r <= 1.5:
        return 0.5 * (1.5 - r) ** 2
    return 0.0


def interp_cells(F, xp, dims):
    """Interpolate F (nz, ny, nx), located at the cell centres (i+1/2, j+1/2,
    k+1/2), with the degree-2 B-spline."""
    nz, ny, nx = F.shape
    n = (nx, ny, nz)
    ax = []
    for a in range(dims):
        base = math.floor(xp[a])
        ax.append([(i, quad_spline(i + 0.5 - xp[a])) for i in range(base - 2, base + 3)])
    if dims == 2:
        ax.append([(0, 1.0)])
    return sum(wi * wj * wk * F[k % n[2], j % n[1], i % n[0]]
               for (i, wi), (j, wj), (k, wk) in itertools.product(*ax))


def face_average_to_cells(F, axes):
    """Average F over the two points of each listed axis that bound a cell:
    F sits at integer points along those axes and at cell centres along the
    others; the result sits at cell centres along all axes."""
    out = F.copy()
    for a in axes:
        ax = {0: 2, 1: 1, 2: 0}[a]          # numpy axis of x, y, z
        out = 0.5 * (out + np.roll(out, -1, axis=ax))
    return out


GRID3 = O.Grid(3, (8, 7, 9), (1.0, 1.3, 0.8), 0.3, 1.0, 4)
GRID2 = O.Grid(2, (9, 8, 1), (1.0, 1.3, 1.0), 0.3, 1.0, 4)


def positions(g, count):
    return [[RNG.uniform(0, g.n[a]) if a < g.dims else 0.0 for a in range(3)] for _ in range(count)]


@pytest.mark.parametrize("g", [GRID3, GRID2], ids=["3d", "2d"])
def test_gather_is_cell_centred_interpolation_of_face_averaged_fields(g):
    """alpha^(x) = (dF_{i-1/2} + dF_{i+1/2})/2 dF_{j+1/2} dF_{k+1/2} (Eq. wrong1):
    E^x at the particle equals the degree-2 B-spline interpolation, at cell
    centres, of E^x averaged over the two x faces of each cell.  B^x (at
    (i+1/2, j, k)) is averaged over its y and z neighbours; cyclically."""
    E = [RNG.normal(size=g.shape) for _ in range(3)]
    B = [RNG.normal(size=g.shape) for _ in range(3)]
    dims = g.dims
    Ec = [face_average_to_cells(E[a], [a] if a < dims else []) for a in range(3)]
    Bc = [face_average_to_cells(B[a], [o for o in range(dims) if o != a]) for a in range(3)]
    for xp in positions(g, 30):
        Ep, Bp = O.gather(g, E, B, xp)
        for a in range(3):
            assert Ep[a] == pytest.approx(interp_cells(Ec[a], xp, dims), abs=1e-13)
            assert Bp[a] == pytest.approx(interp_cells(Bc[a], xp, dims), abs=1e-13)


@pytest.mark.parametrize("g", [GRID3, GRID2], ids=["3d", "2d"])
def test_uniform_fields_are_reproduced(g):
    e0, b0 = RNG.normal(size=3), RNG.normal(size=3)
    E = [np.full(g.shape, e0[a]) for a in range(3)]
    B = [np.full(g.shape, b0[a]) for a in range(3)]
    for xp in positions(g, 40):
        Ep, Bp = O.gather(g, E, B, xp)
        np.testing.assert_allclose(Ep, e0, rtol=0, atol=1e-14)
        np.testing.assert_allclose(Bp, b0, rtol=0, atol=1e-14)


@pytest.mark.parametrize("dims", [3, 2])
def test_charge_and_current_are_those_of_l_a_1_5(dims):
    g4 = GRID3 if dims == 3 else GRID2
    g3 = O.Grid(g4.dims, g4.n, g4.d, g4.dt, g4.c, 3)
    for _ in range(40):
        x0 = positions(g4, 1)[0]
        u = RNG.normal(size=3) * 0.3
        x1 = [x0[a] + u[a] * g4.c * g4.dt / g4.d[a] if a < dims else x0[a] for a in range(3)]
        J4, J3 = g4.zeros(), g3.zeros()
        O.deposit(g4, x0, x1, u, 1.0, J4)
        O.deposit(g3, x0, x1, u, 1.0, J3)
        for a in range(3):
            np.testing.assert_array_equal(J4[a], J3[a])
        np.testing.assert_array_equal(O.rho(g4, np.array(x0).reshape(3, 1), 1.0),
                                      O.rho(g3, np.array(x0).reshape(3, 1), 1.0))


def energy_defect(order2, steps):
    """Max |W(t) - W(0)| / W(0) of the energy integral (Sec. 4.1) over a small
    3D thermal plasma at the Sec. 5 test ratios (cell = Debye length,
    c dt = dx/2, 2 electrons per cell, immobile neutralising background)."""
    wl = W.thermal_plasma("X1 small", 3, (12, 12, 12), 2, 0.05, steps, W.SEED_BASE + 31)
    g = O.Grid(3, wl.n, wl.d, wl.dt, wl.c, order2)
    sp = [O.Species(s.q, s.m, s.weight, s.x.copy(), s.w.copy()) for s in wl.species]
    E, B, J = g.zeros(), g.zeros(), g.zeros()
    w0 = O.diagnostics(g, E, B, sp, wl.rho_bg)[0]["total"]
    worst = 0.0
    for n in range(steps):
        O.step(g, E, B, J, sp)
        if n % 10 == 9:
            worst = max(worst, abs(O.diagnostics(g, E, B, sp, wl.rho_bg)[0]["total"] - w0) / w0)
    return worst


def test_energy_drifts_far_more_than_with_the_alternating_order():
    """Sec. 5, Fig. 2 (left): with the interpolation of Eq. wrong1 the energy
    defect is about two orders of magnitude above that of l_a = 1 1/2.  Here on
    a 12^3 box with 2 electrons per cell over 120 steps; the bar is a factor 10."""
    d3 = energy_defect(3, 120)
    d4 = energy_defect(4, 120)
    assert d4 > 10 * d3, (d3, d4)
