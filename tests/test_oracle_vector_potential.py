"""Pins of the oracle's vector-potential formulation (Sec. 4.2: A on the E
points advanced by Eq. dadt, B = curl_h A by Eq. viaA) and of the generalized
momentum m w + q A / c:

- the B that the ordinary step advances stays equal to curl_h A when A is
  advanced alongside by Eq. dadt (the two formulations are one scheme);
- in a field that is constant along z (a 2D run), the z component of a test
  particle's generalized momentum is conserved up to the time discretization:
  its drift over a fixed time falls as dt^2 with the alternating orders, whose
  weights satisfy B(x_p) = curl_p A(x_p) (Eq. A2B), and does not fall with the
  interpolation of Eq. wrong1, whose weights do not.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1101_0809_gb300 import workloads as W

RNG = np.random.default_rng(20110107)


@pytest.mark.parametrize("dims", [2, 3])
def test_step_keeps_B_equal_to_curl_A(dims):
    if dims == 2:
        wl = W.thermal_plasma("2D", 2, (12, 10, 1), 4, 0.2, 25, W.SEED_BASE + 41)
    else:
        wl = W.thermal_plasma("3D", 3, (8, 7, 9), 2, 0.2, 10, W.SEED_BASE + 42, ions=1836.0, dt_courant=0.45)
    g = O.Grid(wl.dims, wl.n, wl.d, wl.dt, wl.c)
    A = [RNG.normal(size=g.shape) for _ in range(3)]
    B = O.curl_A(g, A)
    E, J = g.zeros(), g.zeros()
    sp = [O.Species(s.q, s.m, s.weight, s.x.copy(), s.w.copy()) for s in wl.species]
    for _ in range(wl.steps):
        O.update_A(g, E, A)
        O.step(g, E, B, J, sp)
    assert max(float(np.abs(E[a]).max()) for a in range(3)) > 0.0
    Bc = O.curl_A(g, A)
    scale = max(float(np.abs(Bc[a]).max()) for a in range(3))
    for a in range(3):
        np.testing.assert_allclose(B[a], Bc[a], rtol=0, atol=1e-12 * scale)


def curl_A_matches_B_by_definition():
    """curl_h A written out for one cell, against orc_curl_A (the index
    convention of Eq. viaA)."""
    g = O.Grid(3, (5, 4, 6), (1.0, 1.3, 0.8), 0.3, 1.0)
    A = [RNG.normal(size=g.shape) for _ in range(3)]
    B = O.curl_A(g, A)
    k, j, i = 2, 1, 3
    bx = (A[2][k, j, i] - A[2][k, j - 1, i]) / g.d[1] - (A[1][k, j, i] - A[1][k - 1, j, i]) / g.d[2]
    by = (A[0][k, j, i] - A[0][k - 1, j, i]) / g.d[2] - (A[2][k, j, i] - A[2][k, j, i - 1]) / g.d[0]
    bz = (A[1][k, j, i] - A[1][k, j, i - 1]) / g.d[0] - (A[0][k, j, i] - A[0][k, j - 1, i]) / g.d[1]
    return (B[0][k, j, i], bx), (B[1][k, j, i], by), (B[2][k, j, i], bz)


def test_curl_A_index_convention():
    for got, want in curl_A_matches_B_by_definition():
        assert got == pytest.approx(want, abs=1e-14)


def test_curl_A_is_the_inverse_of_the_B_update():
    """One B half step with E is B -= (c dt / 2) curl_h E; with A = -(c dt / 2) E
    the same change is curl_h A: the operators agree."""
    g = O.Grid(3, (6, 5, 7), (1.0, 1.3, 0.8), 0.3, 1.0)
    E = [RNG.normal(size=g.shape) for _ in range(3)]
    B = g.zeros()
    O.yee_half_B(g, E, B)
    Bc = O.curl_A(g, [-(g.c * g.dt / 2) * e for e in E])
    for a in range(3):
        np.testing.assert_allclose(B[a], Bc[a], rtol=0, atol=1e-13)


def pz_drift(order2, nsub, base_steps=200):
    """Largest change of a test particle's generalized momentum P_z per unit
    weight over a fixed time in the static field A_z = 3 (sin(2 pi x/16) +
    cos(2 pi y/16)) of a 16^2 2D grid, with dt = 0.4 / nsub."""
    n = 16
    g = O.Grid(2, (n, n, 1), (1.0, 1.0, 1.0), 0.4 / nsub, 1.0, order2)
    X, Y = np.meshgrid(np.arange(n) + 0.5, np.arange(n) + 0.5)     # A_z sits at (i+1/2, j+1/2)
    A = g.zeros()
    A[2][0] = 3.0 * (np.sin(2 * math.pi * X / n) + np.cos(2 * math.pi * Y / n))
    B = O.curl_A(g, A)
    E, J = g.zeros(), g.zeros()
    wt = 1e-12        # a test particle: its own field stays below 1e-11 of the applied one
    sp = [O.Species(-1.0, 1.0, wt, np.array([[5.3], [7.1], [0.0]]), np.array([[0.3], [-0.2], [0.4]]))]
    p0 = O.generalized_momentum(g, A, sp) / wt
    worst = 0.0
    for _ in range(base_steps * nsub):
        O.update_A(g, E, A)
        O.step(g, E, B, J, sp)
        worst = max(worst, abs(O.generalized_momentum(g, A, sp)[2] / wt - p0[2]))
    return worst


@pytest.mark.parametrize("order2", [3, 5])
def test_generalized_momentum_is_conserved_to_second_order(order2):
    d = [pz_drift(order2, k) for k in (1, 2, 4)]
    assert 3.0 < d[0] / d[1] < 5.5 and 3.0 < d[1] / d[2] < 5.5, d
    assert d[2] < 5e-3


def test_generalized_momentum_is_not_conserved_with_eq_wrong1():
    d = [pz_drift(4, k) for k in (1, 4)]
    assert d[1] > 0.5 * d[0] and d[1] > 0.1, d
