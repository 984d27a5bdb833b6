"""The re-sort: every sort after the first starts from the previous sort's tile
segments and sorts only the particles whose tile changed (the movers).  Its
result must be the defined permutation (stable by tile, then the order inside
the tile), bit for bit, whatever moved: a few particles, most of them, particles
that crossed several tiles, tiles that emptied or filled, tiles past the rank
table, several runs and species in one pool, and a pool restored from a
snapshot.  Integer work: compared exactly with pichelpers.tile_sort_perm."""
import numpy as np
import pytest

from paper_1101_0809_gb300 import workloads as W
from pichelpers import make_grid, positions_from_gpu, tile_sort_perm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1101_0809_gb300 import build as B
    B.build()
    from paper_1101_0809_gb300 import pic
    return pic


def plasma(dims, vth, ppc=6, seed=71, ions=True):
    if dims == 2:
        return W.thermal_plasma("2D re-sort", 2, (36, 28, 1), ppc, vth, 1, W.SEED_BASE + seed,
                                ions=1836.0 if ions else None, tile=(8, 8, 1), dt_courant=0.5)
    return W.thermal_plasma("3D re-sort", 3, (20, 18, 22), ppc, vth, 1, W.SEED_BASE + seed,
                            ions=1836.0 if ions else None, tile=(8, 4, 4), dt_courant=0.45)


def check_sort(P, wl, grid, before, banked, run=None):
    pitch = P.pic_tile_layout(grid.h)[2]
    moved = 0
    for s in range(len(wl.species)):
        cell_b, off_b, w_b, id_b = before[s]
        cell_a, off_a, w_a, id_a = grid.particles(s) if run is None else grid.particles_run(run, s)
        perm = tile_sort_perm(wl, cell_b, wl.tile, 1, banked, pitch)
        np.testing.assert_array_equal(id_a, id_b[perm])
        np.testing.assert_array_equal(cell_a, cell_b[perm])
        for a in range(3):
            np.testing.assert_array_equal(off_a[a], off_b[a][perm])
            np.testing.assert_array_equal(w_a[a], w_b[a][perm])
        moved += int(np.count_nonzero(perm != np.arange(perm.size)))
    return moved


@pytest.mark.parametrize("dims", [2, 3])
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("order", ["banked", "stable"])
@pytest.mark.parametrize("steps", [1, 8, 40])
def test_resort_is_the_defined_permutation(P, dims, prec, order, steps):
    """After 1 step few particles changed tile, after 40 steps of a plasma at
    v_th = 0.3c most did, some by more than a tile; two sorts in a row (the
    second with no movers) are both the defined permutation."""
    wl = plasma(dims, 0.3)
    banked = order == "banked"
    grid = make_grid(P, wl, P.PIC_FP32 if prec == "fp32" else P.PIC_FP64, sort_interval=1000,
                     sort_order=P.PIC_SORT_BANKED if banked else P.PIC_SORT_STABLE)
    P.pic_step(grid.h, steps)
    before = [grid.particles(s) for s in range(len(wl.species))]
    P.pic_sort(grid.h)
    assert check_sort(P, wl, grid, before, banked) > 0
    again = [grid.particles(s) for s in range(len(wl.species))]
    P.pic_sort(grid.h)
    assert check_sort(P, wl, grid, again, banked) == 0     # a sorted pool stays in place
    grid.close()


def test_resort_moves_particles_across_several_tiles(P):
    """Electrons and ions streaming together at u = (2c, -1.5c) (0.74c along x,
    no net current) for 50 steps of 0.5 dx/c: about 18.6 cells along x, so
    particles cross two or three 8-cell tiles and every tile's movers come from
    segments before and after it."""
    wl = plasma(2, 0.05, ions=True)
    e = wl.species[0]
    for sp in wl.species:
        sp.w[0] = np.full(sp.n, 2.0 * wl.c)
        sp.w[1] = np.full(sp.n, -1.5 * wl.c)
    grid = make_grid(P, wl, P.PIC_FP64, sort_interval=1000)
    P.pic_step(grid.h, 50)
    before = [grid.particles(s) for s in range(len(wl.species))]
    cell, _, _, ident = before[0]
    x0 = np.floor(e.x[:, ident]).astype(np.int64)        # cells at the load (the last sort)
    ntx = -(-wl.n[0] // wl.tile[0])
    crossed = (cell % wl.n[0] // wl.tile[0] - x0[0] // wl.tile[0]) % ntx
    assert crossed.max() >= 2
    P.pic_sort(grid.h)
    assert check_sort(P, wl, grid, before, True) > 0
    grid.close()


def test_resort_of_a_tile_beyond_the_rank_table(P):
    """3000 particles in one cell (2D, FP64): after two unsorted steps their
    tile holds bank ranks past the 1024 of the precomputed slot table, and
    movers enter and leave it."""
    wl = plasma(2, 0.2, ppc=2, ions=False)
    sp = wl.species[0]
    rng = np.random.default_rng(5)
    dense = np.zeros((3, 3000))
    dense[0] = 17.0 + rng.random(3000)
    dense[1] = 9.0 + rng.random(3000)
    sp.x = np.concatenate([sp.x, dense], axis=1)
    sp.w = rng.normal(0, 0.2, size=(3, sp.x.shape[1]))
    grid = make_grid(P, wl, P.PIC_FP64, sort_interval=1000)
    P.pic_step(grid.h, 2)
    before = [grid.particles(0)]
    P.pic_sort(grid.h)
    assert check_sort(P, wl, grid, before, True) > 0
    grid.close()


def test_resort_after_a_restore_starts_from_the_saved_segments(P):
    """A snapshot holds the tile segments of its pool: a restore followed by a
    sort gives the defined permutation of the restored state."""
    wl = plasma(3, 0.3)
    grid = make_grid(P, wl, P.PIC_FP32, sort_interval=1000)
    P.pic_step(grid.h, 5)
    blob = np.empty(P.pic_state_bytes(grid.h), dtype=np.uint8)
    P.pic_state_save(grid.h, blob)
    before = [grid.particles(s) for s in range(len(wl.species))]
    P.pic_step(grid.h, 7)
    P.pic_sort(grid.h)
    P.pic_state_restore(grid.h, blob)
    P.pic_sort(grid.h)
    assert check_sort(P, wl, grid, before, True) > 0
    grid.close()


def test_resort_in_a_batch_of_runs(P):
    """Four 2D runs of different sizes, two species each, in one pool: the
    segments of all groups are re-sorted together, each group by its own run's
    tiles."""
    specs = [(32, 32, 5, 0.3), (36, 28, 3, 0.25), (24, 40, 6, 0.35), (16, 16, 8, 0.3)]
    runs = [W.thermal_plasma(f"run{r}", 2, (nx, ny, 1), ppc, vth, 1, W.SEED_BASE + 80 + r, ions=1836.0,
                             tile=(8, 8, 1), dt_courant=0.5) for r, (nx, ny, ppc, vth) in enumerate(specs)]
    descs = [P.make_desc(2, wl.n, wl.d, wl.dt, wl.c, P.PIC_FP32, tile=(8, 8, 1), sort_interval=1000,
                         rho_bg=wl.rho_bg) for wl in runs]
    b = P.Batch(descs)
    for r, wl in enumerate(runs):
        for s, sp in enumerate(wl.species):
            b.load_run(r, s, sp.q, sp.m, sp.weight, sp.x, sp.w)
    P.pic_step(b.h, 9)
    before = [[b.particles_run(r, s) for s in range(2)] for r in range(len(runs))]
    P.pic_sort(b.h)
    moved = 0
    for r, wl in enumerate(runs):
        moved += check_sort(P, wl, b, before[r], True, run=r)
    assert moved > 0
    b.close()


@pytest.mark.parametrize("dims", [2, 3])
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("order", ["banked", "stable"])
def test_sort_inside_a_step_equals_an_explicit_sort(P, dims, prec, order):
    """When pic_step reaches the sort interval, the sort leaves the particle
    arrays where they are and the step's particle kernel reads them through
    the permutation, writing the stepped particles in the new order.  From one
    snapshot, that step equals pic_sort followed by a step (the push of a step
    does not depend on its own current): the ids slot by slot, bit for bit
    (the same order), and positions and momenta to a few units of the last
    place, since the two kernels are separate compilations of the same
    arithmetic and may contract multiply-adds differently."""
    wl = plasma(dims, 0.3)
    banked = order == "banked"
    grid = make_grid(P, wl, P.PIC_FP32 if prec == "fp32" else P.PIC_FP64, sort_interval=4,
                     sort_order=P.PIC_SORT_BANKED if banked else P.PIC_SORT_STABLE)
    P.pic_step(grid.h, 4)            # the next step sorts first
    blob = np.empty(P.pic_state_bytes(grid.h), dtype=np.uint8)
    P.pic_state_save(grid.h, blob)
    before = [grid.particles(s) for s in range(len(wl.species))]
    P.pic_step(grid.h, 1)
    inside = [grid.particles(s) for s in range(len(wl.species))]
    P.pic_state_restore(grid.h, blob)
    P.pic_sort(grid.h)
    check_sort(P, wl, grid, before, banked)
    P.pic_step(grid.h, 1)
    ulp = 2.0 ** -23 if prec == "fp32" else 2.0 ** -52
    for s in range(len(wl.species)):
        got = grid.particles(s)
        np.testing.assert_array_equal(inside[s][3], got[3])
        xa = positions_from_gpu(wl, inside[s][0], inside[s][1])
        xb = positions_from_gpu(wl, got[0], got[1])
        for a in range(dims):
            d = xa[a] - xb[a]
            d -= wl.n[a] * np.round(d / wl.n[a])
            assert np.abs(d).max() <= 8 * ulp, f"species {s} axis {a}: positions differ by {np.abs(d).max()} cells"
            wa = np.asarray(inside[s][2][a], np.float64)
            wb = np.asarray(got[2][a], np.float64)
            scale = np.sqrt(np.mean(wb * wb))
            assert np.all(np.abs(wa - wb) <= 8 * ulp * np.maximum(np.abs(wb), scale)), f"species {s} momentum {a}"
    grid.close()
