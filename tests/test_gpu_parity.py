"""GPU parity: libpic (through its C ABI) against the FP64 CPU oracle on the same
seeded inputs.  FP64 path: 1e-12; FP32 form: 2e-5 per step from the same
state rounded to FP32; cell indices and sort permutations bit-exact."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1101_0809_gb300 import workloads as W
from pichelpers import (FP32_TOL, FP64_TOL, close, compare_particles, fp64_field_tol, make_grid, oracle_grid,
                        oracle_species, positions_from_gpu, tile_sort_perm)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1101_0809_gb300 import build as B
    B.build()
    from paper_1101_0809_gb300 import pic
    return pic


def small3d(n=(20, 18, 22), ppc=4, steps=3, vth=0.1, ions=True, seed_offset=11):
    """A small 3D3V thermal plasma with mobile ions, ragged against 8^3 tiles."""
    wl = W.thermal_plasma("3D small", 3, n, ppc, vth, steps, W.SEED_BASE + seed_offset,
                          ions=1836.0 if ions else None, tile=(8, 8, 8), dt_courant=0.45)
    return wl


def ragged2d(vth=0.3, steps=20):
    return W.thermal_plasma("2D ragged", 2, (36, 28, 1), 6, vth, steps, W.SEED_BASE + 21,
                            tile=(8, 8, 1), dt_courant=0.5)


def run_oracle(wl, steps):
    g = oracle_grid(wl)
    sp = oracle_species(wl)
    E, B, J = g.zeros(), g.zeros(), g.zeros()
    for _ in range(steps):
        O.step(g, E, B, J, sp)
    return g, sp, E, B, J


# ---------------------------------------------------------------------------- fields
@pytest.mark.parametrize("dims", [2, 3])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_yee_updates_match_oracle(P, dims, prec):
    n = (20, 18, 17) if dims == 3 else (22, 19, 1)
    wl = W.Workload("vacuum", dims, n, (1.0, 1.2, 0.9), 0.3, 1.0, [], 0.0, 1, (8, 8, 8) if dims == 3 else (8, 8, 1))
    precision = P.PIC_FP64 if prec == "fp64" else P.PIC_FP32
    tol = FP64_TOL if prec == "fp64" else FP32_TOL
    grid = make_grid(P, wl, precision)
    rng = np.random.default_rng(5)
    g = oracle_grid(wl)
    E = [rng.normal(size=g.shape) for _ in range(3)]
    B = [rng.normal(size=g.shape) for _ in range(3)]
    if prec == "fp32":
        E = [a.astype(np.float32).astype(np.float64) for a in E]
        B = [a.astype(np.float32).astype(np.float64) for a in B]
    grid.set_fields(E, B)
    P.pic_yee_update(grid.h, P.PIC_B_HALF)
    O.yee_half_B(g, E, B)
    gE, gB, _ = grid.get_fields()
    for a in range(3):
        close(gB[a], B[a], tol, f"B[{a}] after half step")
    P.pic_yee_update(grid.h, P.PIC_E_FULL)
    O.yee_E(g, B, g.zeros(), E)
    gE, gB, _ = grid.get_fields()
    for a in range(3):
        close(gE[a], E[a], tol, f"E[{a}] after full step")
    grid.close()


# ---------------------------------------------------------------------------- load and sort
@pytest.mark.parametrize("which", ["2d", "3d"])
@pytest.mark.parametrize("order", ["banked", "stable"])
def test_load_cells_offsets_and_tile_sort_are_exact(P, which, order):
    wl = W.c0_small2d() if which == "2d" else small3d()
    banked = order == "banked"
    grid = make_grid(P, wl, P.PIC_FP64, sort_order=P.PIC_SORT_BANKED if banked else P.PIC_SORT_STABLE)
    g = oracle_grid(wl)
    for s, sp in enumerate(wl.species):
        cell, off, w, ident = grid.particles(s)
        n = sp.n
        assert sorted(ident.tolist()) == list(range(n))
        # cells and offsets exactly as floor and remainder of the loaded positions
        x = sp.x[:, ident]
        fl = np.floor(x).astype(np.int64)
        want_cell = fl[0] + wl.n[0] * (fl[1] + wl.n[1] * (fl[2] if wl.dims == 3 else 0))
        np.testing.assert_array_equal(cell, want_cell)
        for a in range(wl.dims):
            np.testing.assert_array_equal(off[a], x[a] - fl[a])
            np.testing.assert_array_equal(w[a], sp.w[a][ident])
        # storage order: the tile sort of the load order
        fl0 = np.floor(sp.x).astype(np.int64)
        cells0 = fl0[0] + wl.n[0] * (fl0[1] + wl.n[1] * (fl0[2] if wl.dims == 3 else 0))
        _, _, pitch = P.pic_tile_layout(grid.h)
        np.testing.assert_array_equal(ident, tile_sort_perm(wl, cells0, wl.tile, 1, banked, pitch))
        if not banked:
            keys = O.tile_keys(g, wl.tile, sp.x)
            nt = [math.ceil(wl.n[a] / wl.tile[a]) for a in range(3)]
            perm = O.sort_perm(keys, nt[0] * nt[1] * (nt[2] if wl.dims == 3 else 1))
            np.testing.assert_array_equal(ident, perm)
    grid.close()


@pytest.mark.parametrize("order", ["banked", "stable"])
def test_sort_after_motion_is_the_defined_permutation(P, order):
    wl = ragged2d(vth=0.3)
    banked = order == "banked"
    grid = make_grid(P, wl, P.PIC_FP64, sort_interval=1000,
                     sort_order=P.PIC_SORT_BANKED if banked else P.PIC_SORT_STABLE)
    P.pic_step(grid.h, 6)
    cell_b, off_b, w_b, id_b = grid.particles(0)
    P.pic_sort(grid.h)
    cell_a, off_a, w_a, id_a = grid.particles(0)
    perm = tile_sort_perm(wl, cell_b, wl.tile, 1, banked, P.pic_tile_layout(grid.h)[2])
    if not banked:
        x = positions_from_gpu(wl, cell_b, off_b)
        keys = O.tile_keys(oracle_grid(wl), wl.tile, x)
        nt = [math.ceil(wl.n[a] / wl.tile[a]) for a in range(2)]
        np.testing.assert_array_equal(perm, O.sort_perm(keys, nt[0] * nt[1]))
    np.testing.assert_array_equal(id_a, id_b[perm])
    np.testing.assert_array_equal(cell_a, cell_b[perm])
    for a in range(3):
        np.testing.assert_array_equal(w_a[a], w_b[a][perm])
    grid.close()


# ---------------------------------------------------------------------------- FP64 steps
def _check_state(P, wl, grid, osp, E, B, J, tol, x_prev=None):
    """Fields and particles against the oracle; x_prev (per species, the
    positions both sides started the step from) selects the FP32 rules of
    compare_particles.  Returns the FP32 cell indices that differ next to a face."""
    gE, gB, gJ = grid.get_fields()
    for a in range(3):
        close(gE[a], E[a], tol, f"E[{a}]")
        close(gB[a], B[a], tol, f"B[{a}]")
        close(gJ[a], J[a], tol, f"J[{a}]")
    near = 0
    for s in range(len(wl.species)):
        near += compare_particles(wl, s, grid, osp, tol, x_prev=None if x_prev is None else x_prev[s])
    if x_prev is not None:
        print(f"FP32 cell indices one off next to a face: {near}")
    return near


@pytest.mark.parametrize("which", ["2d", "3d"])
def test_fp64_one_step_matches_oracle(P, which):
    wl = W.c0_small2d() if which == "2d" else small3d()
    grid = make_grid(P, wl, P.PIC_FP64)
    P.pic_step(grid.h, 1)
    P.pic_sync(grid.h)
    g, osp, E, B, J = run_oracle(wl, 1)
    _check_state(P, wl, grid, osp, E, B, J, FP64_TOL)
    grid.close()


def test_fp64_fifty_steps_small2d_match_oracle_and_keep_gauss_law(P):
    wl = W.c0_small2d()
    grid = make_grid(P, wl, P.PIC_FP64)
    d0 = P.pic_diagnostics(grid.h)
    P.pic_step(grid.h, wl.steps)
    d = P.pic_diagnostics(grid.h)
    g, osp, E, B, J = run_oracle(wl, wl.steps)
    _check_state(P, wl, grid, osp, E, B, J, FP64_TOL)
    scale = 4 * math.pi * wl.rho_bg
    assert d["gauss_resid_max"] / scale <= 1e-12
    assert abs(d["total_charge"] - d0["total_charge"]) <= 1e-12 * abs(wl.rho_bg * wl.n_cells)
    grid.close()


def test_fp64_3d_with_sorts_between_steps(P):
    wl = small3d(steps=6)
    grid = make_grid(P, wl, P.PIC_FP64, sort_interval=2)
    P.pic_step(grid.h, wl.steps)
    g, osp, E, B, J = run_oracle(wl, wl.steps)
    _check_state(P, wl, grid, osp, E, B, J, FP64_TOL)
    grid.close()


def past_halo(wl, grid, tile, halo):
    """Particles whose cell lies more than `halo` cells outside the tile of
    their cell at the load (the last sort), along some axis, periodically; and
    how many of those changed cell in the last step (x_prev: the cells before
    it).  Such particles run on the global-memory path."""
    past = 0
    for s, sp in enumerate(wl.species):
        cell, _, _, ident = grid.particles(s)
        c = [cell % wl.n[0], (cell // wl.n[0]) % wl.n[1], cell // (wl.n[0] * wl.n[1])]
        out = np.zeros(cell.size, dtype=bool)
        for a in range(wl.dims):
            c0 = np.floor(sp.x[a][ident]).astype(np.int64) % wl.n[a]
            o = (c0 // tile[a]) * tile[a]
            d = (c[a] - o) % wl.n[a]            # periodic offset from the tile's first cell
            d = np.where(d >= wl.n[a] - halo - tile[a], d - wl.n[a], d)   # the nearer image below the tile
            out |= (d < -halo) | (d >= tile[a] + halo)
        past += int(out.sum())
    return past


@pytest.mark.parametrize("halo", [0, 1, 2])
def test_fp64_particles_far_outside_their_tile_take_the_global_path(P, halo):
    wl = ragged2d(vth=0.3, steps=16)       # fast particles, no sort for 16 steps
    grid = make_grid(P, wl, P.PIC_FP64, halo=halo, sort_interval=1000, ppb=512)
    P.pic_step(grid.h, wl.steps)
    assert past_halo(wl, grid, (8, 8, 1), halo) > 0
    g, osp, E, B, J = run_oracle(wl, wl.steps)
    _check_state(P, wl, grid, osp, E, B, J, FP64_TOL)
    grid.close()


def test_adaptive_sort_policy_sorts_when_particles_drift_and_not_before(P):
    """pic_set_sort_policy: with a long fixed interval and the adaptive
    policy, a fast plasma is re-sorted as its particles leave their tiles' halos
    (and still equals the oracle; the schedule does not change the arithmetic),
    and a plasma at rest is never re-sorted."""
    wl = ragged2d(vth=0.3, steps=40)
    grid = make_grid(P, wl, P.PIC_FP64, halo=1, sort_interval=1000, ppb=512)
    P.pic_set_sort_policy(grid.h, True)
    P.pic_profile(grid.h, True)
    P.pic_step(grid.h, wl.steps)
    prof = P.pic_profile_read(grid.h)
    assert prof["sort"][1] >= 1
    g, osp, E, B, J = run_oracle(wl, wl.steps)
    _check_state(P, wl, grid, osp, E, B, J, FP64_TOL)
    grid.close()
    cold = ragged2d(vth=0.3, steps=8)
    for sp in cold.species:
        sp.w[:] = 0.0
    grid = make_grid(P, cold, P.PIC_FP32, halo=1, sort_interval=1000)
    P.pic_set_sort_policy(grid.h, True)
    P.pic_profile(grid.h, True)
    P.pic_step(grid.h, cold.steps)
    assert P.pic_profile_read(grid.h)["sort"][1] == 0
    grid.close()


@pytest.mark.parametrize("halo", [0, 1])
def test_fp64_3d_particles_far_outside_their_tile_take_the_global_path(P, halo):
    wl = small3d(vth=0.3, steps=8, ions=False)     # fast electrons, no sort for 8 steps
    grid = make_grid(P, wl, P.PIC_FP64, tile=(8, 4, 4), halo=halo, sort_interval=1000, ppb=512)
    P.pic_step(grid.h, wl.steps)
    assert past_halo(wl, grid, (8, 4, 4), halo) > 0
    g, osp, E, B, J = run_oracle(wl, wl.steps)
    tol = fp64_field_tol(wl, osp)
    _check_state(P, wl, grid, osp, E, B, J, tol)
    grid.close()


@pytest.mark.parametrize("which", ["2d", "3d"])
def test_unfused_boundary_calls_equal_the_step(P, which):
    wl = W.c0_small2d() if which == "2d" else small3d()
    grid = make_grid(P, wl, P.PIC_FP64)
    for _ in range(2):
        P.pic_yee_update(grid.h, P.PIC_B_HALF)
        P.pic_gather_push(grid.h)
        P.pic_deposit_current(grid.h)
        P.pic_yee_update(grid.h, P.PIC_B_HALF)
        P.pic_yee_update(grid.h, P.PIC_E_FULL)
    g, osp, E, B, J = run_oracle(wl, 2)
    _check_state(P, wl, grid, osp, E, B, J, FP64_TOL)
    grid.close()


def test_deposit_without_gather_push_is_a_state_error(P):
    wl = W.c0_small2d()
    grid = make_grid(P, wl, P.PIC_FP64)
    with pytest.raises(P.PicError) as e:
        P.pic_deposit_current(grid.h)
    assert e.value.code == P.PIC_ERR_STATE
    grid.close()


# ---------------------------------------------------------------------------- FP32 form
@pytest.mark.parametrize("which", ["2d", "3d"])
def test_fp32_one_step_from_the_rounded_oracle_state(P, which):
    wl = W.c0_small2d() if which == "2d" else small3d()
    # evolve the oracle a few steps so that the fields are not zero
    g, osp, E, B, J = run_oracle(wl, 5)
    grid = make_grid(P, wl, P.PIC_FP32)
    grid.set_fields([a.astype(np.float32) for a in E], [a.astype(np.float32) for a in B])
    for s, sp in enumerate(osp):
        grid.load(s, sp.q, sp.m, sp.weight, sp.x, sp.w.astype(np.float32).astype(np.float64))
    # the oracle restarts from exactly the FP32 state the GPU holds
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
    _check_state(P, wl, grid, osp, E, B, J, FP32_TOL, x_prev=x_prev)
    grid.close()


def test_fp32_gauss_residual_over_many_steps(P):
    wl = W.c0_small2d(steps=200)
    grid = make_grid(P, wl, P.PIC_FP32)
    P.pic_diagnostics(grid.h)
    P.pic_step(grid.h, wl.steps)
    d = P.pic_diagnostics(grid.h)
    assert d["gauss_resid_max"] / (4 * math.pi * wl.rho_bg) <= 1e-6
    grid.close()


# ---------------------------------------------------------------------------- diagnostics
@pytest.mark.parametrize("which", ["2d", "3d"])
def test_diagnostics_match_oracle(P, which):
    wl = W.c0_small2d() if which == "2d" else small3d()
    grid = make_grid(P, wl, P.PIC_FP64)
    P.pic_step(grid.h, 4)
    d = P.pic_diagnostics(grid.h)
    g, osp, E, B, J = run_oracle(wl, 4)
    od, rho, res = O.diagnostics(g, E, B, osp, wl.rho_bg)
    for k in ("kinetic", "field_E", "field_B", "half_step_corr", "total"):
        assert d[k] == pytest.approx(od[k], rel=1e-11, abs=1e-13 * abs(od["total"])), k
    np.testing.assert_allclose(d["momentum"], od["momentum"], rtol=1e-11,
                               atol=1e-12 * np.abs(od["momentum"]).max())
    assert d["total_charge"] == pytest.approx(od["charge"], abs=1e-11 * max(1.0, wl.n_particles))
    assert d["n_particles"] == wl.n_particles
    grid.close()


@pytest.mark.parametrize("which", ["2d", "3d", "3d-8x4x4"])
def test_fp32_diagnostics_match_oracle_on_the_same_state(P, which):
    """The FP32 state's diagnostics (FP32 per-particle terms over the work
    items, FP64 sums) against the oracle's FP64 diagnostics of the very state
    the GPU holds, read back.  The field terms are FP64 on both sides; the
    particle terms carry FP32 rounding per particle."""
    wl = W.c0_small2d() if which == "2d" else small3d()
    tile = (8, 4, 4) if which == "3d-8x4x4" else None
    grid = make_grid(P, wl, P.PIC_FP32, tile=tile)
    P.pic_step(grid.h, 4)
    d = P.pic_diagnostics(grid.h)
    gE, gB, gJ = grid.get_fields()
    osp = []
    for s, sp in enumerate(wl.species):
        cell, off, w, ident = grid.particles(s)
        x = positions_from_gpu(wl, cell, off)
        osp.append(O.Species(sp.q, sp.m, sp.weight, x, np.array(w, dtype=np.float64)))
    od, rho, res = O.diagnostics(oracle_grid(wl), [np.asarray(a, np.float64) for a in gE],
                                 [np.asarray(a, np.float64) for a in gB], osp, wl.rho_bg)
    for k in ("field_E", "field_B"):
        assert d[k] == pytest.approx(od[k], rel=1e-12), k
    for k in ("kinetic", "half_step_corr", "total"):
        assert d[k] == pytest.approx(od[k], rel=2e-6, abs=1e-6 * abs(od["total"])), k
    pabs = sum(float(np.abs(sp.m * sp.weight * sp.w).sum()) for sp in osp)
    np.testing.assert_allclose(d["momentum"], od["momentum"], rtol=0, atol=1e-6 * pabs)
    assert d["total_charge"] == pytest.approx(od["charge"], abs=1e-9 * max(1.0, wl.n_particles))
    assert d["n_particles"] == wl.n_particles
    grid.close()


# ---------------------------------------------------------------------------- edge cases
def test_edge_positions_empty_species_and_reload(P):
    wl = W.c0_small2d()
    grid = make_grid(P, wl, P.PIC_FP64)
    # an empty species next to the electrons
    grid.load(3, 1.0, 1836.0, wl.species[0].weight, np.zeros((3, 0)), np.zeros((3, 0)))
    assert P.pic_num_particles(grid.h, 3) == 0
    # positions on faces, at -tiny, at N - tiny, far outside the box: all wrapped
    x = np.array([[0.0, 1.0, -1e-17, 32 - 1e-14, 64.5, -31.25, 5.0],
                  [0.0, 31.0, 3.5, 0.0, -0.5, 96.0, 7.999999999999999],
                  [0.0] * 7])
    w = np.zeros((3, 7))
    grid.load(1, 1.0, 1.0, 1.0, x, w)
    cell, off, ww, ident = grid.particles(1)
    order = np.argsort(ident)
    xs = positions_from_gpu(wl, cell[order], [o[order] for o in off])
    for a in range(2):
        want = np.mod(x[a], 32.0)
        want[want >= 32.0] = 0.0
        d = xs[a] - want
        d -= 32 * np.round(d / 32)
        assert np.abs(d).max() < 1e-13
        assert (off[a] >= 0).all() and (off[a] < 1).all()
    # reloading species 1 leaves species 0 untouched
    before = grid.particles(0)
    grid.load(1, 1.0, 1.0, 1.0, x[:, :3], w[:, :3])
    after = grid.particles(0)
    for b, a in zip(before, after):
        if isinstance(b, list):
            for u, v in zip(b, a):
                np.testing.assert_array_equal(u, v)
        else:
            np.testing.assert_array_equal(b, a)
    P.pic_step(grid.h, 2)
    P.pic_sync(grid.h)
    grid.close()


def test_nonfinite_momentum_is_reported_not_trapped(P):
    wl = W.c0_small2d()
    grid = make_grid(P, wl, P.PIC_FP64)
    x = np.array([[3.5], [4.5], [0.0]])
    w = np.array([[np.nan], [0.0], [0.0]])
    grid.load(2, -1.0, 1.0, 1.0, x, w)
    P.pic_step(grid.h, 1)
    with pytest.raises(P.PicError) as e:
        P.pic_sync(grid.h)
    assert e.value.code == P.PIC_ERR_NONFINITE
    grid.close()
