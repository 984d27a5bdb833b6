"""Pins of the oracle's plane-wave antenna (the one-way source of the
laser-plasma setup; the paper gives no injection).  What the construction
fixes: in vacuum the scattered-field side stays empty (the source is one-way),
the total-field side carries a plane wave of the set amplitude with E and B
related as in a vacuum wave travelling in +x, only the set polarization is
excited, and the source adds no charge (Gauss residual and total charge
unchanged with particles present)."""
import math

import numpy as np
import pytest

import oracle as O

LAMBDA = 20.0
OMEGA = 2 * math.pi / LAMBDA       # c = 1, dx = 1
RAMP = 2 * LAMBDA                  # two periods


def run_vacuum(dims, nx, steps, pol, i0=20, E0=1.5):
    n = (nx, 4, 1) if dims == 2 else (nx, 2, 2)
    g = O.Grid(dims, n, (1.0, 1.0, 1.0), 0.45, 1.0)
    E, B, J = g.zeros(), g.zeros(), g.zeros()
    ant = O.Antenna(pol, i0, E0, OMEGA, RAMP)
    for s in range(steps):
        O.step(g, E, B, J, [], antenna=ant, n=s)
    return g, E, B, ant


@pytest.mark.parametrize("dims,nx,steps", [(2, 240, 300), (3, 160, 250)])
@pytest.mark.parametrize("pol", [1, 2])
def test_antenna_injects_a_one_way_wave_of_the_set_amplitude(dims, nx, steps, pol):
    g, E, B, ant = run_vacuum(dims, nx, steps, pol)
    ea, ba = (1, 2) if pol == 1 else (2, 1)     # driven E and B components
    e = E[ea][0, 0, :]                           # uniform in y and z
    b = B[ba][0, 0, :]
    for z in range(g.shape[0]):
        for y in range(g.shape[1]):
            np.testing.assert_array_equal(E[ea][z, y, :], e)
    # only the set polarization is excited
    for a in range(3):
        if a != ea:
            assert np.abs(E[a]).max() == 0.0
        if a != ba:
            assert np.abs(B[a]).max() == 0.0
    # one-way: the scattered-field side (E nodes x = i + 1/2 < i0 - 1/2) stays empty
    assert np.abs(e[:ant.i0 - 1]).max() <= 0.01 * ant.E0
    assert np.abs(b[:ant.i0]).max() <= 0.01 * ant.E0
    # the total-field side behind the rise carries the set amplitude
    front = ant.i0 + steps * g.dt          # how far light got
    lo, hi = ant.i0 + 5, int(front - RAMP - 10)
    assert hi - lo > 2 * LAMBDA
    assert abs(np.abs(e[lo:hi]).max() / ant.E0 - 1.0) <= 0.02
    assert abs(np.abs(b[lo:hi]).max() / ant.E0 - 1.0) <= 0.02
    # a vacuum wave in +x: B_z = E_y (pol 1), B_y = -E_z (pol 2).  The state holds
    # B^{n-1/2} at the nodes x and E^n at the nodes x + 1/2; the wave seen at
    # (x, t^n - dt/2) is the one at (x + c dt/2, t^n), which lies between the E
    # nodes x - 1/2 and x + 1/2 at fraction 1/2 + c dt/2 from the left
    f = 0.5 + 0.5 * g.c * g.dt / g.d[0]
    e_at_b = (1.0 - f) * e[lo - 1:hi - 1] + f * e[lo:hi]
    sign = 1.0 if pol == 1 else -1.0
    assert np.abs(b[lo:hi] - sign * e_at_b).max() <= 0.05 * ant.E0
    # beyond the light front only the scheme's small dispersive precursor
    assert np.abs(e[int(front) + 3:]).max() <= 1e-3 * ant.E0


def test_antenna_adds_no_charge():
    """With particles crossing the plane region, Gauss's residual and the total
    charge stay constant to rounding: the source is divergence-free."""
    rng = np.random.default_rng(7)
    g = O.Grid(2, (64, 8, 1), (1.0, 1.0, 1.0), 0.45, 1.0)
    count = 64 * 8 * 4
    x = np.zeros((3, count))
    x[0] = rng.uniform(0, 64, count)
    x[1] = rng.uniform(0, 8, count)
    w = rng.normal(0, 0.1, (3, count))
    sp = [O.Species(-1.0, 1.0, 0.01, x, w)]
    E, B, J = g.zeros(), g.zeros(), g.zeros()
    ant = O.Antenna(1, 10, 1.0, OMEGA, RAMP)
    d0, rho0, res0 = O.diagnostics(g, E, B, sp)
    for s in range(60):
        O.step(g, E, B, J, sp, antenna=ant, n=s)
    d1, rho1, res1 = O.diagnostics(g, E, B, sp)
    scale = 4 * math.pi * 0.01 * 4
    assert np.abs(res1 - res0).max() / scale <= 1e-12
    assert d1["charge"] == pytest.approx(d0["charge"], abs=1e-12)
    assert np.abs(E[1]).max() > 0.1      # the wave is there
