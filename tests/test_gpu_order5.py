"""GPU parity of the alternating-order form factor l_a = 2 1/2 (Sec. 4.5;
order2 = 5 in the grid descriptor) against the FP64 oracle with the same
order, through the C ABI: FP64 runs step by step (with sorts between steps,
particles past their tiles' halos, and the split gather/push + deposit
calls), one FP32 step from the oracle state rounded to FP32, Gauss's law over
many FP32 steps, the diagnostics of both precisions, a batch of runs, and the
calls that are built for l_a = 1 1/2 only."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1101_0809_gb300 import workloads as W
from pichelpers import (FP32_TOL, FP64_TOL, close, compare_particles, fp64_field_tol, make_grid, oracle_grid,
                        oracle_species, positions_from_gpu, tile_sort_perm)

pytestmark = pytest.mark.gpu
ORDER2 = 5


@pytest.fixture(scope="module")
def P():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1101_0809_gb300 import build as B
    B.build()
    from paper_1101_0809_gb300 import pic
    return pic


def small3d(steps=3, vth=0.1, ions=True, ppc=4):
    """Tiles of 8x4x4: with l_a = 2 1/2 an FP64 8^3 tile would need more shared
    memory than a block can have (the grid refuses it at creation).  With
    ppc = 16 per species a 4x4x4 tile holds 2048 particles, enough for the FP32
    kernel to take the bias of particles whose base index stayed off at the
    flush (at 4 it takes it off per contribution)."""
    return W.thermal_plasma("3D small", 3, (20, 18, 22), ppc, vth, steps, W.SEED_BASE + 11,
                            ions=1836.0 if ions else None, tile=(8, 4, 4), dt_courant=0.45)


def ragged2d(vth=0.3, steps=20):
    return W.thermal_plasma("2D ragged", 2, (36, 28, 1), 6, vth, steps, W.SEED_BASE + 21,
                            tile=(8, 8, 1), dt_courant=0.5)


def grid5(P, wl, precision, **kw):
    return make_grid(P, wl, precision, order2=ORDER2, **kw)


def run_oracle(wl, steps):
    g = oracle_grid(wl, ORDER2)
    sp = oracle_species(wl)
    E, B, J = g.zeros(), g.zeros(), g.zeros()
    for _ in range(steps):
        assert O.step(g, E, B, J, sp) < 1e-14
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
    grid = grid5(P, wl, P.PIC_FP64, sort_interval=3)
    P.pic_step(grid.h, wl.steps)
    P.pic_sync(grid.h)
    g, osp, E, B, J = run_oracle(wl, wl.steps)
    check_state(wl, grid, osp, E, B, J, fp64_field_tol(wl, osp))
    # the l_a = 2 1/2 result differs from the l_a = 1 1/2 one (the stencil is in use)
    g3 = oracle_grid(wl)
    sp3 = oracle_species(wl)
    E3, B3, J3 = g3.zeros(), g3.zeros(), g3.zeros()
    for _ in range(wl.steps):
        O.step(g3, E3, B3, J3, sp3)
    assert max(float(np.abs(J3[a] - J[a]).max()) for a in range(3)) > 1e-6 * max(
        float(np.abs(J[a]).max()) for a in range(3))
    grid.close()


@pytest.mark.parametrize("halo", [0, 1])
def test_fp64_particles_past_their_tiles_take_the_global_path(P, halo):
    wl = ragged2d(vth=0.3, steps=16)          # fast particles, no sort for 16 steps
    grid = grid5(P, wl, P.PIC_FP64, halo=halo, sort_interval=1000, ppb=512)
    P.pic_step(grid.h, wl.steps)
    g, osp, E, B, J = run_oracle(wl, wl.steps)
    check_state(wl, grid, osp, E, B, J, FP64_TOL)
    grid.close()


def test_fp64_3d_particles_past_their_tiles(P):
    wl = small3d(vth=0.3, steps=8, ions=False)
    grid = grid5(P, wl, P.PIC_FP64, tile=(8, 4, 4), halo=0, sort_interval=1000, ppb=512)
    P.pic_step(grid.h, wl.steps)
    g, osp, E, B, J = run_oracle(wl, wl.steps)
    check_state(wl, grid, osp, E, B, J, fp64_field_tol(wl, osp))
    grid.close()


@pytest.mark.parametrize("which", ["2d", "3d"])
def test_split_calls_equal_the_step(P, which):
    wl = W.c0_small2d() if which == "2d" else small3d()
    grid = grid5(P, wl, P.PIC_FP64)
    for _ in range(2):
        P.pic_yee_update(grid.h, P.PIC_B_HALF)
        P.pic_gather_push(grid.h)
        P.pic_deposit_current(grid.h)
        P.pic_yee_update(grid.h, P.PIC_B_HALF)
        P.pic_yee_update(grid.h, P.PIC_E_FULL)
    g, osp, E, B, J = run_oracle(wl, 2)
    check_state(wl, grid, osp, E, B, J, FP64_TOL)
    grid.close()


@pytest.mark.parametrize("which", ["2d", "3d", "3d-8x8x4", "3d-4x4x4", "3d-4x4x4-dense"])
def test_fp32_one_step_from_the_rounded_oracle_state(P, which):
    wl = W.c0_small2d() if which == "2d" else small3d(ppc=16 if which.endswith("dense") else 4)
    tile = {"3d-8x8x4": (8, 8, 4), "3d-4x4x4": (4, 4, 4), "3d-4x4x4-dense": (4, 4, 4)}.get(which)
    g, osp, E, B, J = run_oracle(wl, 5)
    grid = grid5(P, wl, P.PIC_FP32, tile=tile)
    if which.startswith("3d-4x4x4"):
        assert tuple(P.pic_tile_layout(grid.h)[2]) == (12, 12)    # the fixed-geometry kernel
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


@pytest.mark.parametrize("which", ["2d", "3d-4x4x4", "3d-4x4x4-dense"])
def test_fp32_one_step_with_particles_drifted_into_the_halo(P, which):
    """Six unsorted steps carry particles into the one-cell halo of their tile,
    some past its upper edge with offset >= 1/2, where the base index reaches its
    largest value in the current tile; then one step against the oracle from the
    GPU's own state."""
    wl = ragged2d(vth=0.3) if which == "2d" else small3d(vth=0.3, ppc=16 if which.endswith("dense") else 4)
    tile = (8, 8, 1) if which == "2d" else (4, 4, 4)
    grid = grid5(P, wl, P.PIC_FP32, tile=tile, halo=1, sort_interval=1000)
    P.pic_step(grid.h, 6)
    g = oracle_grid(wl, ORDER2)
    osp = oracle_species(wl)
    E, B, _ = grid.get_fields()
    E = [a.astype(np.float64) for a in E]
    B = [a.astype(np.float64) for a in B]
    J = g.zeros()
    edge = 0
    for s, sp in enumerate(wl.species):
        cell, off, w, ident = grid.particles(s)
        order = np.argsort(ident)
        osp[s].x[:] = positions_from_gpu(wl, cell[order], [o[order] for o in off])
        for a in range(3):
            osp[s].w[a][:] = w[a][order]
        # local coordinate in the tile the particle was sorted into at the load
        for a in range(wl.dims):
            n = wl.n[a]
            t0 = (np.floor(sp.x[a]).astype(np.int64) % n) // tile[a] * tile[a]
            li = (np.floor(osp[s].x[a]).astype(np.int64) - t0) % n
            li[li > n // 2] -= n
            fr = osp[s].x[a] - np.floor(osp[s].x[a])
            edge += int(np.count_nonzero((li == tile[a]) & (fr >= 0.5)))
    assert edge > 0
    x_prev = [sp.x.copy() for sp in osp]
    P.pic_step(grid.h, 1)
    P.pic_sync(grid.h)
    O.step(g, E, B, J, osp)
    check_state(wl, grid, osp, E, B, J, FP32_TOL, x_prev=x_prev)
    grid.close()


@pytest.mark.parametrize("which", ["2d-fp64", "2d-fp32", "3d-fp32"])
def test_banked_sort_is_by_the_bank_of_the_base_index(P, which):
    """After six unsorted steps, pic_sort gives the defined permutation with the
    bank taken at the base index (the cell plus offset >= 1/2 per axis) and the
    current tile one cell wider (h = halo + 1); bit-exact."""
    wl = ragged2d(vth=0.3) if which.startswith("2d") else small3d(vth=0.3)
    tile = (8, 8, 1) if which.startswith("2d") else (4, 4, 4)
    prec = P.PIC_FP64 if which.endswith("fp64") else P.PIC_FP32
    grid = grid5(P, wl, prec, tile=tile, halo=1, sort_interval=1000)
    P.pic_step(grid.h, 6)
    before = [grid.particles(s) for s in range(len(wl.species))]
    P.pic_sort(grid.h)
    pitch = P.pic_tile_layout(grid.h)[2]
    moved = 0
    for s in range(len(wl.species)):
        cell_b, off_b, w_b, id_b = before[s]
        cell_a, off_a, w_a, id_a = grid.particles(s)
        up = [(off_b[a] >= 0.5).astype(np.int64) for a in range(3)]
        perm = tile_sort_perm(wl, cell_b, tile, 2, True, pitch, up)
        np.testing.assert_array_equal(id_a, id_b[perm])
        np.testing.assert_array_equal(cell_a, cell_b[perm])
        for a in range(3):
            np.testing.assert_array_equal(off_a[a], off_b[a][perm])
        moved += int(np.count_nonzero(perm != tile_sort_perm(wl, cell_b, tile, 2, True, pitch)))
    assert moved > 0     # the half-offset flags change the order
    grid.close()


def test_fp32_gauss_residual_over_many_steps(P):
    wl = W.c0_small2d(steps=200)
    grid = grid5(P, wl, P.PIC_FP32)
    P.pic_diagnostics(grid.h)
    P.pic_step(grid.h, wl.steps)
    d = P.pic_diagnostics(grid.h)
    assert d["gauss_resid_max"] / (4 * math.pi * wl.rho_bg) <= 1e-6
    assert d["n_particles"] == wl.n_particles
    grid.close()


@pytest.mark.parametrize("which", ["2d", "3d"])
def test_fp64_diagnostics_match_oracle(P, which):
    wl = W.c0_small2d() if which == "2d" else small3d()
    grid = grid5(P, wl, P.PIC_FP64)
    d0 = P.pic_diagnostics(grid.h)
    P.pic_step(grid.h, 4)
    d = P.pic_diagnostics(grid.h)
    g, osp, E, B, J = run_oracle(wl, 4)
    od, rho, res = O.diagnostics(g, E, B, osp, wl.rho_bg)
    for k in ("kinetic", "field_E", "field_B", "half_step_corr", "total"):
        assert d[k] == pytest.approx(od[k], rel=1e-11, abs=1e-13 * abs(od["total"])), k
    assert d["total_charge"] == pytest.approx(od["charge"], abs=1e-11 * max(1.0, wl.n_particles))
    # Gauss's law is kept against the state at the first call
    assert d["gauss_resid_max"] <= 1e-10 * max(1.0, abs(d0["gauss_resid_max"]) + 4 * math.pi)
    grid.close()


@pytest.mark.parametrize("which", ["2d", "3d"])
def test_fp32_diagnostics_match_oracle_on_the_same_state(P, which):
    wl = W.c0_small2d() if which == "2d" else small3d()
    grid = grid5(P, wl, P.PIC_FP32)
    P.pic_step(grid.h, 4)
    d = P.pic_diagnostics(grid.h)
    gE, gB, gJ = grid.get_fields()
    osp = []
    for s, sp in enumerate(wl.species):
        cell, off, w, ident = grid.particles(s)
        x = positions_from_gpu(wl, cell, off)
        osp.append(O.Species(sp.q, sp.m, sp.weight, x, np.array(w, dtype=np.float64)))
    od, rho, res = O.diagnostics(oracle_grid(wl, ORDER2), [np.asarray(a, np.float64) for a in gE],
                                 [np.asarray(a, np.float64) for a in gB], osp, wl.rho_bg)
    for k in ("field_E", "field_B"):
        assert d[k] == pytest.approx(od[k], rel=1e-12), k
    for k in ("kinetic", "half_step_corr", "total"):
        assert d[k] == pytest.approx(od[k], rel=2e-6, abs=1e-6 * abs(od["total"])), k
    assert d["total_charge"] == pytest.approx(od["charge"], abs=1e-9 * max(1.0, wl.n_particles))
    grid.close()


def test_batch_of_runs_matches_oracle(P):
    runs = [W.c0_small2d(steps=6), ragged2d(vth=0.2, steps=6)]
    descs = [P.make_desc(2, wl.n, wl.d, wl.dt, wl.c, P.PIC_FP64, tile=(8, 8, 1), sort_interval=2,
                         rho_bg=wl.rho_bg, order2=ORDER2) for wl in runs]
    b = P.Batch(descs)
    for r, wl in enumerate(runs):
        sp = wl.species[0]
        b.load_run(r, 0, sp.q, sp.m, sp.weight, sp.x, sp.w)
    P.pic_step(b.h, 6)
    P.pic_sync(b.h)
    for r, wl in enumerate(runs):
        g, osp, E, B, J = run_oracle(wl, 6)
        gE, gB, gJ = b.get_fields_run(r)
        for a in range(3):
            close(gE[a], E[a], FP64_TOL, f"run {r} E[{a}]")
            close(gJ[a], J[a], FP64_TOL, f"run {r} J[{a}]")
    b.close()


def test_calls_built_for_l_a_1_5_refuse_l_a_2_5(P):
    import torch
    wl = W.c0_small2d()
    grid = grid5(P, wl, P.PIC_FP64)
    for call in (lambda: P.pic_step_persistent(grid.h, 1),):
        with pytest.raises(P.PicError) as e:
            call()
        assert e.value.code == P.PIC_ERR_INVALID_ARG
    f = [torch.zeros(grid.shape, dtype=torch.float64, device="cuda") for _ in range(3)]
    p = [torch.zeros(wl.n_particles, dtype=torch.float64, device="cuda") for _ in range(3)]
    with pytest.raises(P.PicError) as e:
        P.pic_adjoint_step(grid.h, f, [t.clone() for t in f], p, [t.clone() for t in p])
    assert e.value.code == P.PIC_ERR_INVALID_ARG
    for bad in (dict(order2=6), dict(order2=5, tile=(8, 8, 8), dims3=True)):
        if bad.pop("dims3", False):
            w3 = small3d()
            desc = P.make_desc(3, w3.n, w3.d, w3.dt, w3.c, P.PIC_FP64, **bad)   # shared memory of the tiles
        else:
            desc = P.make_desc(2, wl.n, wl.d, wl.dt, wl.c, P.PIC_FP64, **bad)
        with pytest.raises(P.PicError) as e:
            P.Grid(desc)
        assert e.value.code == P.PIC_ERR_INVALID_ARG
    grid.close()
