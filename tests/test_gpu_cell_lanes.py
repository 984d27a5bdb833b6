"""The cell-lane particle order and the FP32 fused kernel that walks it (3D,
8x4x4 tiles, halo 1, l_a = 1 1/2), against their definitions and the FP64
oracle.

The order is requested explicitly (the default is the banked order).  It is
integer work and is compared bit-exactly with its definition
(pichelpers.tile_sort_perm with cell_lanes): after a load, after motion, and on
a tile whose fullest cell has more particles than the sort's precomputed rank
table.  The kernel is compared with the oracle one step at a time from the
FP32 state the GPU holds: on a freshly sorted plasma, after unsorted steps that
carry particles out of the cell their lane walks (the drift list) and past the
tile's halo (the global path), and on tiles holding more particles than the
fixed-point scale of one work item assumes (the tile's own scale)."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1101_0809_gb300 import workloads as W
from pichelpers import FP32_TOL, close, compare_particles, make_grid, positions_from_gpu, tile_sort_perm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1101_0809_gb300 import build as B
    B.build()
    from paper_1101_0809_gb300 import pic
    return pic, torch


def plasma(vth=0.1, ppc=4, n=(20, 18, 22), seed=61, ions=True):
    return W.thermal_plasma("3D cell lanes", 3, n, ppc, vth, 1, W.SEED_BASE + seed,
                            ions=1836.0 if ions else None, tile=(8, 4, 4), dt_courant=0.45)


def cells_of(wl, x):
    fl = np.floor(x).astype(np.int64)
    return fl[0] + wl.n[0] * (fl[1] + wl.n[1] * fl[2])


def oracle_from_gpu(wl, grid):
    out = []
    for s, sp in enumerate(wl.species):
        cell, off, w, ident = grid.particles(s)
        order = np.argsort(ident)
        x = positions_from_gpu(wl, cell[order], [o[order] for o in off])
        out.append(O.Species(sp.q, sp.m, sp.weight, x, np.array([a[order] for a in w], dtype=np.float64)))
    return out


def one_step_against_oracle(P, wl, grid):
    """One FP32 step of the grid against the oracle started from the GPU's state."""
    osp = oracle_from_gpu(wl, grid)
    E, B, _ = grid.get_fields()
    E = [np.asarray(a, np.float64) for a in E]
    B = [np.asarray(a, np.float64) for a in B]
    g = O.Grid(3, wl.n, wl.d, wl.dt, wl.c)
    J = g.zeros()
    x_prev = [sp.x.copy() for sp in osp]
    P.pic_step(grid.h, 1)
    P.pic_sync(grid.h)
    O.step(g, E, B, J, osp)
    gE, gB, gJ = grid.get_fields()
    for a in range(3):
        close(gE[a], E[a], FP32_TOL, f"E[{a}]")
        close(gB[a], B[a], FP32_TOL, f"B[{a}]")
        close(gJ[a], J[a], FP32_TOL, f"J[{a}]")
    near = 0
    for s in range(len(wl.species)):
        near += compare_particles(wl, s, grid, osp, FP32_TOL, x_prev=x_prev[s])
    print(f"FP32 cell indices one off next to a face: {near}")


def test_the_cell_lane_order_after_a_load(env):
    P, torch = env
    wl = plasma()
    grid = make_grid(P, wl, P.PIC_FP32, sort_order=P.PIC_SORT_CELL_LANES)
    assert tuple(P.pic_tile_layout(grid.h)[2]) == (14, 12)
    _, _, pitch = P.pic_tile_layout(grid.h)
    for s, sp in enumerate(wl.species):
        _, _, _, ident = grid.particles(s)
        np.testing.assert_array_equal(ident, tile_sort_perm(wl, cells_of(wl, sp.x), wl.tile, cell_lanes=True))
    grid.close()
    # the default order is the banked one
    grid = make_grid(P, wl, P.PIC_FP32)
    _, _, _, ident = grid.particles(0)
    np.testing.assert_array_equal(ident, tile_sort_perm(wl, cells_of(wl, wl.species[0].x), wl.tile, 1, True,
                                                        P.pic_tile_layout(grid.h)[2]))
    grid.close()


def test_cell_lane_sort_after_motion_is_the_defined_permutation(env):
    P, torch = env
    wl = plasma(vth=0.3)
    grid = make_grid(P, wl, P.PIC_FP32, sort_interval=1000, sort_order=P.PIC_SORT_CELL_LANES)
    P.pic_step(grid.h, 5)
    before = [grid.particles(s) for s in range(len(wl.species))]
    P.pic_sort(grid.h)
    for s in range(len(wl.species)):
        cell_b, off_b, w_b, id_b = before[s]
        cell_a, off_a, w_a, id_a = grid.particles(s)
        perm = tile_sort_perm(wl, cell_b, wl.tile, cell_lanes=True)
        np.testing.assert_array_equal(id_a, id_b[perm])
        np.testing.assert_array_equal(cell_a, cell_b[perm])
        for a in range(3):
            np.testing.assert_array_equal(off_a[a], off_b[a][perm])
            np.testing.assert_array_equal(w_a[a], w_b[a][perm])
    grid.close()


def test_cell_lane_sort_with_a_cell_beyond_the_rank_table(env):
    """A cell holding 1500 particles (the sort precomputes P(r) for r < 1024 and
    sums the counts beyond), next to a sparse plasma; requested explicitly on an
    FP64 grid, whose fused step keeps the general kernel."""
    P, torch = env
    wl = plasma(ppc=1, ions=False)
    rng = np.random.default_rng(3)
    x = wl.species[0].x
    dense = np.stack([9.0 + rng.random(1500), 5.0 + rng.random(1500), 13.0 + rng.random(1500)])
    wl.species[0].x = np.concatenate([x, dense], axis=1)
    wl.species[0].w = rng.normal(0, 1.0, size=(3, wl.species[0].x.shape[1]))
    grid = make_grid(P, wl, P.PIC_FP64, sort_order=P.PIC_SORT_CELL_LANES)
    _, _, _, ident = grid.particles(0)
    np.testing.assert_array_equal(ident, tile_sort_perm(wl, cells_of(wl, wl.species[0].x), wl.tile,
                                                        cell_lanes=True))
    P.pic_step(grid.h, 1)
    P.pic_sync(grid.h)
    grid.close()


def test_cell_lane_kernel_one_step_after_the_sort(env):
    P, torch = env
    wl = plasma()
    grid = make_grid(P, wl, P.PIC_FP32, sort_order=P.PIC_SORT_CELL_LANES)
    P.pic_step(grid.h, 3)      # fields are not zero any more; the last sort was at the load
    P.pic_sort(grid.h)
    one_step_against_oracle(P, wl, grid)
    grid.close()


@pytest.mark.parametrize("steps", [4, 12])
def test_cell_lane_kernel_with_drifted_particles(env, steps):
    """Unsorted steps of a fast plasma carry particles out of the cell their lane
    walks (the drift list) and, after 12 steps, past the tile's one-cell halo
    (the global-memory path); one step of that state against the oracle."""
    P, torch = env
    wl = plasma(vth=0.3, ions=False)
    grid = make_grid(P, wl, P.PIC_FP32, sort_interval=1000, sort_order=P.PIC_SORT_CELL_LANES)
    P.pic_step(grid.h, steps)
    cell, off, w, ident = grid.particles(0)
    sorted_cells = cells_of(wl, wl.species[0].x)[ident]
    moved = int(np.count_nonzero(cell != sorted_cells))
    assert moved > 0.1 * cell.size
    if steps == 12:
        nx, ny = wl.n[0], wl.n[1]
        def tile_coord(c):
            return [(c % nx) // 8, ((c // nx) % ny) // 4, (c // (nx * ny)) // 4]
        i, j, k = cell % nx, (cell // nx) % ny, cell // (nx * ny)
        ti, tj, tk = tile_coord(sorted_cells)
        def outside(v, t, T, n):
            d = (v - t * T) % n
            return (d >= T + 1) & (d < n - 1)
        past = outside(i, ti, 8, nx) | outside(j, tj, 4, ny) | outside(k, tk, 4, wl.n[2])
        assert past.any()
    one_step_against_oracle(P, wl, grid)
    grid.close()


def test_cell_lane_kernel_on_tiles_fuller_than_one_work_item(env):
    """80 particles per cell and species: a tile holds 10,240 particles of a
    species, more than the 8192 per block the groups' fixed-point scales assume;
    the tile then halves its scale.  One step against the oracle, and Gauss's
    law and the charge over 20 steps."""
    P, torch = env
    wl = W.thermal_plasma("3D dense", 3, (16, 12, 12), 80, 0.1, 1, W.SEED_BASE + 62, ions=1836.0,
                          tile=(8, 4, 4), dt_courant=0.45)
    grid = make_grid(P, wl, P.PIC_FP32, sort_order=P.PIC_SORT_CELL_LANES)
    P.pic_step(grid.h, 2)
    one_step_against_oracle(P, wl, grid)
    d0 = P.pic_diagnostics(grid.h)
    P.pic_step(grid.h, 20)
    d = P.pic_diagnostics(grid.h)
    sp = wl.species[0]
    scale = 4 * math.pi * abs(sp.q) * sp.weight * sp.n / (wl.n_cells * wl.volume)
    assert d["gauss_resid_max"] / scale <= 1e-6
    assert d["total_charge"] == pytest.approx(d0["total_charge"], abs=1e-9 * abs(sp.q) * sp.weight * sp.n)
    grid.close()


def test_cell_lane_snapshot_carries_the_lane_tables(env):
    """A snapshot of a grid in the cell-lane order holds the lane tables, so that
    a restore between sorts steps on like the saved grid: the next step's
    particle state is bit for bit the same (the current J, summed over the
    tiles' borders by float atomics, may differ in its last bit, and through
    the E step so may later steps)."""
    P, torch = env
    wl = plasma(vth=0.3, ions=False)
    grid = make_grid(P, wl, P.PIC_FP32, sort_interval=1000, sort_order=P.PIC_SORT_CELL_LANES)
    P.pic_step(grid.h, 3)
    blob = np.empty(P.pic_state_bytes(grid.h), dtype=np.uint8)
    P.pic_state_save(grid.h, blob)
    P.pic_step(grid.h, 1)
    want = grid.particles(0)
    P.pic_step(grid.h, 3)
    P.pic_state_restore(grid.h, blob)
    P.pic_step(grid.h, 1)
    got = grid.particles(0)
    np.testing.assert_array_equal(got[0], want[0])
    np.testing.assert_array_equal(got[3], want[3])
    for a in range(3):
        np.testing.assert_array_equal(got[1][a], want[1][a])
        np.testing.assert_array_equal(got[2][a], want[2][a])
    grid.close()
