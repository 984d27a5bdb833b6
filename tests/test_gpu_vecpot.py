"""GPU parity of the vector-potential formulation (Sec. 4.2) through the C ABI:
A advanced by Eq. dadt with the E step, B = curl_h A set from it, and the
generalized momentum against the FP64 oracle; B stays the curl of A in FP32;
and the conservation experiment: test particles in a static field constant
along z keep their generalized momentum P_z to second order in dt with the
alternating order, not with the interpolation of Eq. wrong1."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1101_0809_gb300 import workloads as W
from pichelpers import close, make_grid, oracle_grid, oracle_species

pytestmark = pytest.mark.gpu
RNG = np.random.default_rng(20110108)


@pytest.fixture(scope="module")
def P():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1101_0809_gb300 import build as B
    B.build()
    from paper_1101_0809_gb300 import pic
    return pic


def plasma(dims):
    if dims == 2:
        return W.thermal_plasma("2D", 2, (36, 28, 1), 6, 0.2, 12, W.SEED_BASE + 43, tile=(8, 8, 1))
    return W.thermal_plasma("3D", 3, (20, 18, 22), 2, 0.2, 6, W.SEED_BASE + 44, ions=1836.0, tile=(8, 4, 4),
                            dt_courant=0.45)


@pytest.mark.parametrize("dims", [2, 3])
def test_fp64_vector_potential_and_generalized_momentum_match_oracle(P, dims):
    wl = plasma(dims)
    g = oracle_grid(wl)
    A = [RNG.normal(size=g.shape) * 0.3 for _ in range(3)]
    grid = make_grid(P, wl, P.PIC_FP64)
    P.pic_set_vector_potential(grid.h, [a.copy() for a in A], set_B=True)
    B = O.curl_A(g, A)
    E, J = g.zeros(), g.zeros()
    sp = oracle_species(wl)
    close(grid.get_fields()[1][0], B[0], 1e-13, "B from curl A")
    p_gpu0 = P.pic_generalized_momentum(grid.h)
    p_orc0 = O.generalized_momentum(g, A, sp)
    P.pic_step(grid.h, wl.steps)
    for _ in range(wl.steps):
        O.update_A(g, E, A)
        O.step(g, E, B, J, sp)
    gA = [np.empty(g.shape) for _ in range(3)]
    P.pic_get_vector_potential(grid.h, gA)
    gE, gB, gJ = grid.get_fields()
    for a in range(3):
        close(gA[a], A[a], 1e-12, f"A[{a}]")
        close(gB[a], B[a], 1e-12, f"B[{a}]")
    scale = sum(abs(s.m * s.weight) * float(np.abs(s.w).sum()) for s in sp)
    for got, want in ((p_gpu0, p_orc0), (P.pic_generalized_momentum(grid.h), O.generalized_momentum(g, A, sp))):
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-12 * scale)
    grid.close()


def test_fp32_B_stays_curl_of_A(P):
    wl = plasma(3)
    g = oracle_grid(wl)
    grid = make_grid(P, wl, P.PIC_FP32)
    P.pic_set_vector_potential(grid.h, [(RNG.normal(size=g.shape) * 0.3).astype(np.float32) for _ in range(3)])
    P.pic_step(grid.h, 20)
    gA = [np.empty(g.shape, np.float32) for _ in range(3)]
    P.pic_get_vector_potential(grid.h, gA)
    Bc = O.curl_A(g, [a.astype(np.float64) for a in gA])
    gB = grid.get_fields()[1]
    for a in range(3):
        close(gB[a], Bc[a], 2e-5, f"B[{a}] vs curl A")
    grid.close()


def pz_drift(P, order2, nsub, base_steps=120):
    """Largest change of the generalized momentum P_z per unit weight of 4096
    test particles in the static field A_z = 3 (sin(2 pi x/32) + cos(2 pi y/32))
    of a 32^2 grid, over a fixed time, dt = 0.4 / nsub."""
    n = 32
    desc = P.make_desc(2, (n, n, 1), (1.0, 1.0, 1.0), 0.4 / nsub, 1.0, P.PIC_FP64, tile=(8, 8, 1), order2=order2)
    grid = P.Grid(desc)
    X, Y = np.meshgrid(np.arange(n) + 0.5, np.arange(n) + 0.5)
    A = [np.zeros((1, n, n)), np.zeros((1, n, n)),
         (3.0 * (np.sin(2 * math.pi * X / n) + np.cos(2 * math.pi * Y / n))).reshape(1, n, n)]
    P.pic_set_vector_potential(grid.h, A, set_B=True)
    rng = np.random.default_rng(5)
    count = 4096
    x = np.zeros((3, count))
    x[0] = rng.uniform(0, n, count)
    x[1] = rng.uniform(0, n, count)
    w = rng.normal(0, 0.3, (3, count))
    wt = 1e-12
    grid.load(0, -1.0, 1.0, wt, x, w)
    p0 = P.pic_generalized_momentum(grid.h)[2] / wt
    worst = 0.0
    for _ in range(base_steps):
        P.pic_step(grid.h, nsub)
        worst = max(worst, abs(P.pic_generalized_momentum(grid.h)[2] / wt - p0))
    grid.close()
    return worst / count


def test_generalized_momentum_conserved_to_second_order_only_with_the_alternating_order(P):
    d3 = [pz_drift(P, 3, k) for k in (1, 2, 4)]
    assert 3.0 < d3[0] / d3[1] < 5.5 and 3.0 < d3[1] / d3[2] < 5.5, d3
    d4 = [pz_drift(P, 4, k) for k in (1, 4)]
    assert d4[1] > 0.5 * d4[0] and d4[1] > 20 * d3[2], (d3, d4)


def test_calls_check_the_tracking_state(P):
    wl = plasma(2)
    grid = make_grid(P, wl, P.PIC_FP64)
    with pytest.raises(P.PicError) as e:
        P.pic_generalized_momentum(grid.h)
    assert e.value.code == P.PIC_ERR_STATE
    P.pic_set_vector_potential(grid.h, [np.zeros(grid.shape) for _ in range(3)])
    with pytest.raises(P.PicError) as e:
        P.pic_step_persistent(grid.h, 1)
    assert e.value.code == P.PIC_ERR_INVALID_ARG
    P.pic_set_vector_potential(grid.h, None)
    P.pic_step_persistent(grid.h, 1)
    grid.close()
