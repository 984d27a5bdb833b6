"""Pin of the oracle's discrete adjoint (P13): gradients of a field-energy loss
after N steps with respect to the density-perturbation amplitude and the initial
momenta, from the adjoint, against FP64 central finite differences of the
oracle's forward run."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1101_0809_gb300 import workloads as W

N_CELLS, PPC, STEPS, AMP = 32, 16, 20, 0.05
WIN = (12, 20)


def setup(amplitude):
    wl = W.c4_perturbed2d(n=N_CELLS, ppc=PPC, amplitude=amplitude, steps=STEPS)
    g = O.Grid(wl.dims, wl.n, wl.d, wl.dt, wl.c)
    return wl, g


def loss_and_seed(g, E, B):
    """L = V/(8 pi) sum over the window of |E^N|^2 + |B^N|^2 with B^N the half-advanced
    B; returns L and the seeds dL/dE^N, dL/dB^{N-1/2}."""
    Bn = [b.copy() for b in B]
    O.yee_half_B(g, E, Bn)
    mask = np.zeros(g.shape)
    mask[:, WIN[0]:WIN[1], WIN[0]:WIN[1]] = 1.0
    V = g.volume
    L = V / (8 * math.pi) * sum(float((mask * (E[a] ** 2 + Bn[a] ** 2)).sum()) for a in range(3))
    lamB = [V / (4 * math.pi) * mask * Bn[a] for a in range(3)]
    lamE = [V / (4 * math.pi) * mask * E[a] for a in range(3)]
    O.yee_half_B_adj(g, lamB, lamE)
    return L, lamE, lamB


def forward(wl, g, x0, w0, keep=False):
    sp = [O.Species(wl.species[0].q, wl.species[0].m, wl.species[0].weight, x0.copy(), w0.copy())]
    E, B, J = g.zeros(), g.zeros(), g.zeros()
    states = []
    for _ in range(STEPS):
        if keep:
            states.append(([a.copy() for a in E], [a.copy() for a in B], sp[0].x.copy(), sp[0].w.copy()))
        O.step(g, E, B, J, sp)
    return E, B, states


def adjoint(wl, g, x0, w0):
    E, B, states = forward(wl, g, x0, w0, keep=True)
    L, lamE, lamB = loss_and_seed(g, E, B)
    n = x0.shape[1]
    lx = np.zeros((3, n))
    lw = np.zeros((3, n))
    for En, Bn, xn, wn in reversed(states):
        spn = [O.Species(wl.species[0].q, wl.species[0].m, wl.species[0].weight, xn, wn)]
        O.step_adj(g, En, Bn, spn, lamE, lamB, [lx], [lw])
    return L, lx, lw


@pytest.fixture(scope="module")
def base():
    wl, g = setup(AMP)
    wl_u, _ = setup(0.0)
    xu = wl_u.species[0].x.copy()
    k = 2 * math.pi * 2 / N_CELLS
    dxdA = np.zeros_like(xu)
    dxdA[0] = -np.sin(k * xu[0]) / k
    L, lx, lw = adjoint(wl, g, wl.species[0].x.copy(), wl.species[0].w.copy())
    return wl, g, L, lx, lw, dxdA


def fd_loss(wl, g, x0, w0):
    E, B, _ = forward(wl, g, x0, w0)
    return loss_and_seed(g, E, B)[0]


def test_p13_adjoint_gradient_wrt_amplitude_matches_central_fd(base):
    wl, g, L, lx, lw, dxdA = base
    grad = float((lx * dxdA).sum())
    h = 1e-7 * AMP
    wp, _ = setup(AMP + h)
    wm, _ = setup(AMP - h)
    fd = (fd_loss(wp, g, wp.species[0].x, wp.species[0].w) - fd_loss(wm, g, wm.species[0].x, wm.species[0].w)) / (2 * h)
    assert L > 0
    assert grad == pytest.approx(fd, rel=1e-6)


def test_p13_adjoint_gradient_wrt_momenta_matches_central_fd(base):
    wl, g, L, lx, lw, dxdA = base
    rng = np.random.default_rng(13)
    x0, w0 = wl.species[0].x, wl.species[0].w
    scale = float(np.abs(w0).max())
    dirs = [rng.normal(size=w0.shape) for _ in range(3)]
    n = w0.shape[1]
    for k in range(10):
        d = np.zeros_like(w0)
        d[k % 3, rng.integers(n)] = 1.0
        dirs.append(d)
    # Random directions use h = 1e-7 relative.  A single component moves one
    # particle only; its central difference at h = 1e-7 is limited by the
    # rounding noise of the whole run divided by 2h (it converges onto the
    # adjoint value as h grows: 1e-4, 7e-6, 1e-6, 1.6e-7 relative error at
    # h = 1e-8 .. 1e-5), so single components use h = 1e-5 relative.
    # Single components are judged like every other array here, relative to
    # max(|value|, rms of the gradient array): some particles barely touch the
    # window and their gradient sits below the difference quotient's noise floor.
    rms = float(np.sqrt(np.mean(lw ** 2)))
    for j, d in enumerate(dirs):
        rel = 1e-7 if j < 3 else 1e-5
        h = rel * scale / max(np.abs(d).max(), 1e-300)
        fd = (fd_loss(wl, g, x0, w0 + h * d) - fd_loss(wl, g, x0, w0 - h * d)) / (2 * h)
        ad = float((lw * d).sum())
        ref = abs(fd) if j < 3 else max(abs(fd), rms)
        assert abs(ad - fd) <= 1e-6 * ref, (j, ad, fd, rms)


def test_adjoint_of_yee_operators_is_the_transpose():
    """<C v, y> = <v, C^T y> for the B half step and the E step on random fields."""
    g = O.Grid(3, (6, 5, 7), (1.0, 1.3, 0.8), 0.3, 1.0)
    rng = np.random.default_rng(3)
    E = [rng.normal(size=g.shape) for _ in range(3)]
    yB = [rng.normal(size=g.shape) for _ in range(3)]
    zero = g.zeros()
    B = g.zeros()
    O.yee_half_B(g, E, B)            # B = -(1/2) C_B E
    lhs = sum(float((B[a] * yB[a]).sum()) for a in range(3))
    lamE = g.zeros()
    O.yee_half_B_adj(g, yB, lamE)
    rhs = sum(float((E[a] * lamE[a]).sum()) for a in range(3))
    assert lhs == pytest.approx(rhs, rel=1e-12)
