"""GPU parity of the comparison scheme of Eq. wrong1 (order2 = 4: the
uniform-order l = 2 field interpolation of Sec. 5 with the l_a = 1 1/2 charge
and current) against the FP64 oracle with the same scheme, through the C ABI,
and the paper's energy observation (Sec. 5, Fig. 2) run through the library:
on a small X1 plasma the energy defect of Eq. wrong1 is far above that of the
alternating order."""
import numpy as np
import pytest

import oracle as O
from paper_1101_0809_gb300 import workloads as W
from pichelpers import (FP32_TOL, FP64_TOL, close, compare_particles, fp64_field_tol, make_grid, oracle_grid,
                        oracle_species, positions_from_gpu)

pytestmark = pytest.mark.gpu
ORDER2 = 4


@pytest.fixture(scope="module")
def P():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1101_0809_gb300 import build as B
    B.build()
    from paper_1101_0809_gb300 import pic
    return pic


def small3d(steps=3, vth=0.1, ions=True):
    return W.thermal_plasma("3D small", 3, (20, 18, 22), 4, vth, steps, W.SEED_BASE + 11,
                            ions=1836.0 if ions else None, tile=(8, 4, 4), dt_courant=0.45)


def ragged2d(vth=0.3, steps=20):
    return W.thermal_plasma("2D ragged", 2, (36, 28, 1), 6, vth, steps, W.SEED_BASE + 21,
                            tile=(8, 8, 1), dt_courant=0.5)


def run_oracle(wl, steps):
    g = oracle_grid(wl, ORDER2)
    sp = oracle_species(wl)
    E, B, J = g.zeros(), g.zeros(), g.zeros()
    for _ in range(steps):
        O.step(g, E, B, J, sp)
    return g, sp, E, B, J


def check_state(wl, grid, osp, E, B, J, tol, x_prev=None):
    gE, gB, gJ = grid.get_fields()
    for a in range(3):
        close(gE[a], E[a], tol, f"E[{a}]")
        close(gB[a], B[a], tol, f"B[{a}]")
        close(gJ[a], J[a], tol, f"J[{a}]")
    for s in range(len(wl.species)):
        compare_particles(wl, s, grid, osp, tol, x_prev=None if x_prev is None else x_prev[s])


@pytest.mark.parametrize("which", ["2d", "3d"])
def test_fp64_steps_match_oracle(P, which):
    wl = W.c0_small2d(steps=12) if which == "2d" else small3d(steps=4)
    grid = make_grid(P, wl, P.PIC_FP64, sort_interval=3, order2=ORDER2)
    P.pic_step(grid.h, wl.steps)
    P.pic_sync(grid.h)
    g, osp, E, B, J = run_oracle(wl, wl.steps)
    check_state(wl, grid, osp, E, B, J, fp64_field_tol(wl, osp))
    grid.close()


def test_fp64_particles_past_their_tiles_take_the_global_path(P):
    wl = ragged2d(vth=0.3, steps=16)
    grid = make_grid(P, wl, P.PIC_FP64, halo=0, sort_interval=1000, ppb=512, order2=ORDER2)
    P.pic_step(grid.h, wl.steps)
    g, osp, E, B, J = run_oracle(wl, wl.steps)
    check_state(wl, grid, osp, E, B, J, FP64_TOL)
    grid.close()


def test_split_calls_equal_the_step(P):
    wl = small3d()
    grid = make_grid(P, wl, P.PIC_FP64, order2=ORDER2)
    for _ in range(2):
        P.pic_yee_update(grid.h, P.PIC_B_HALF)
        P.pic_gather_push(grid.h)
        P.pic_deposit_current(grid.h)
        P.pic_yee_update(grid.h, P.PIC_B_HALF)
        P.pic_yee_update(grid.h, P.PIC_E_FULL)
    g, osp, E, B, J = run_oracle(wl, 2)
    check_state(wl, grid, osp, E, B, J, FP64_TOL)
    grid.close()


@pytest.mark.parametrize("which", ["2d", "3d"])
def test_fp32_one_step_from_the_rounded_oracle_state(P, which):
    wl = W.c0_small2d() if which == "2d" else small3d()
    g, osp, E, B, J = run_oracle(wl, 5)
    grid = make_grid(P, wl, P.PIC_FP32, order2=ORDER2)
    grid.set_fields([a.astype(np.float32) for a in E], [a.astype(np.float32) for a in B])
    for s, sp in enumerate(osp):
        grid.load(s, sp.q, sp.m, sp.weight, sp.x, sp.w.astype(np.float32).astype(np.float64))
    for s in range(len(osp)):
        cell, off, w, ident = grid.particles(s)
        order = np.argsort(ident)
        osp[s].x[:] = positions_from_gpu(wl, cell[order], [o[order] for o in off])
        for a in range(3):
            osp[s].w[a][:] = w[a][order]
    E = [a.astype(np.float32).astype(np.float64) for a in E]
    B = [a.astype(np.float32).astype(np.float64) for a in B]
    x_prev = [sp.x.copy() for sp in osp]
    P.pic_step(grid.h, 1)
    P.pic_sync(grid.h)
    O.step(g, E, B, J, osp)
    check_state(wl, grid, osp, E, B, J, FP32_TOL, x_prev=x_prev)
    grid.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_diagnostics_match_oracle_on_the_same_state(P, prec):
    wl = small3d()
    grid = make_grid(P, wl, P.PIC_FP64 if prec == "fp64" else P.PIC_FP32, order2=ORDER2)
    P.pic_step(grid.h, 4)
    d = P.pic_diagnostics(grid.h)
    gE, gB, gJ = grid.get_fields()
    osp = []
    for s, sp in enumerate(wl.species):
        cell, off, w, ident = grid.particles(s)
        osp.append(O.Species(sp.q, sp.m, sp.weight, positions_from_gpu(wl, cell, off), np.array(w, dtype=np.float64)))
    od, rho, res = O.diagnostics(oracle_grid(wl, ORDER2), [np.asarray(a, np.float64) for a in gE],
                                 [np.asarray(a, np.float64) for a in gB], osp, wl.rho_bg)
    tol = 1e-11 if prec == "fp64" else 2e-6
    for k in ("kinetic", "half_step_corr", "total"):
        assert d[k] == pytest.approx(od[k], rel=tol, abs=tol * abs(od["total"])), k
    grid.close()


def test_energy_defect_far_above_the_alternating_order(P):
    """Sec. 5, Fig. 2 (left), on a small X1 plasma (12^3, 2 electrons per cell,
    immovable ions at their positions), 120 FP64 steps through the library."""
    from paper_1101_0809_gb300.energy import energy_run
    wl = W.x1_energy(n=12, steps=120, tile=(4, 4, 4))
    r3 = energy_run(wl, 3, P.PIC_FP64)
    r4 = energy_run(wl, 4, P.PIC_FP64)
    assert r3["max_rel_defect"] < 1e-4
    assert r4["max_rel_defect"] > 10 * r3["max_rel_defect"], (r3["max_rel_defect"], r4["max_rel_defect"])


def test_batch_and_adjoint_calls_refuse_it(P):
    import torch
    wl = W.c0_small2d()
    grid = make_grid(P, wl, P.PIC_FP64, order2=ORDER2)
    with pytest.raises(P.PicError) as e:
        P.pic_step_persistent(grid.h, 1)
    assert e.value.code == P.PIC_ERR_INVALID_ARG
    f = [torch.zeros(grid.shape, dtype=torch.float64, device="cuda") for _ in range(3)]
    p = [torch.zeros(wl.n_particles, dtype=torch.float64, device="cuda") for _ in range(3)]
    with pytest.raises(P.PicError) as e:
        P.pic_adjoint_step(grid.h, f, [t.clone() for t in f], p, [t.clone() for t in p])
    assert e.value.code == P.PIC_ERR_INVALID_ARG
    grid.close()
