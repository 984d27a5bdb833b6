"""The allocation-free tile sort (pic_tile_sort_perm_noalloc) against the
library's own sort.

Callers that cannot allocate device memory (code inside another runtime's
memory budget, or on a path where cudaMalloc would synchronize the device) get
the stable tile permutation from a fixed scratch array.  Here its output must be
bit-identical to the permutation that pic_load_particles / pic_sort apply, on
two calls in a row.  This file is collected last on purpose."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1101_0809_gb300 import workloads as W
from pichelpers import make_grid, oracle_grid

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1101_0809_gb300 import build as B
    B.build()
    from paper_1101_0809_gb300 import pic
    return pic, torch


def _tiles(wl):
    return [math.ceil(wl.n[a] / wl.tile[a]) for a in range(3)] if wl.dims == 3 else \
        [math.ceil(wl.n[0] / wl.tile[0]), math.ceil(wl.n[1] / wl.tile[1]), 1]


def _noalloc(P, torch, wl, cells_host):
    n = cells_host.shape[0]
    cell = torch.from_numpy(cells_host.astype(np.int32)).cuda()
    perm = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    nt = _tiles(wl)
    ts = torch.full((nt[0] * nt[1] * nt[2] + 1,), -1, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    P.pic_tile_sort_perm_noalloc(cell, n, wl.dims, wl.n, wl.tile, perm, ts, stream)
    torch.cuda.synchronize()
    return perm.cpu().numpy(), ts.cpu().numpy()


def _expected_tile_start(wl, cells_sorted):
    g = oracle_grid(wl)
    nx, ny = wl.n[0], wl.n[1]
    x = np.zeros((3, cells_sorted.shape[0]))
    x[0] = cells_sorted % nx + 0.5
    x[1] = (cells_sorted // nx) % ny + 0.5
    x[2] = cells_sorted // (nx * ny) + 0.5 if wl.dims == 3 else 0.0
    keys = O.tile_keys(g, wl.tile, x)
    nt = _tiles(wl)
    return np.searchsorted(keys, np.arange(nt[0] * nt[1] * nt[2] + 1), side="left")


@pytest.mark.parametrize("which", ["2d", "3d"])
def test_noalloc_permutation_equals_the_library_sort_twice_in_a_row(env, which):
    P, torch = env
    if which == "2d":
        wl = W.thermal_plasma("2D ragged", 2, (36, 28, 1), 6, 0.3, 6, W.SEED_BASE + 21, tile=(8, 8, 1))
    else:
        wl = W.thermal_plasma("3D small", 3, (20, 18, 22), 4, 0.3, 6, W.SEED_BASE + 11,
                              tile=(8, 8, 8), dt_courant=0.45)
    # the library sorts inside a tile in bank order by default; the allocation-free
    # entry point computes the stable tile order, which the library also offers
    grid = make_grid(P, wl, P.PIC_FP64, sort_interval=1000, sort_order=P.PIC_SORT_STABLE)
    sp = wl.species[0]
    # call 1: the load order; the library's load sorted the same particles
    fl = np.floor(sp.x).astype(np.int64)
    cells = fl[0] + wl.n[0] * (fl[1] + wl.n[1] * (fl[2] if wl.dims == 3 else 0))
    perm1, ts1 = _noalloc(P, torch, wl, cells)
    _, _, _, ident = grid.particles(0)
    np.testing.assert_array_equal(perm1, ident)
    np.testing.assert_array_equal(ts1, _expected_tile_start(wl, cells[perm1]))
    # call 2 (same scratch, right after): the storage order after 6 unsorted steps
    P.pic_step(grid.h, wl.steps)
    cell_b, _, _, id_b = grid.particles(0)
    perm2, ts2 = _noalloc(P, torch, wl, cell_b.astype(np.int64))
    P.pic_sort(grid.h)
    cell_a, _, _, id_a = grid.particles(0)
    np.testing.assert_array_equal(id_a, id_b[perm2])
    np.testing.assert_array_equal(cell_a, cell_b[perm2])
    np.testing.assert_array_equal(ts2, _expected_tile_start(wl, cell_b[perm2]))
    grid.close()


def test_noalloc_rejects_sizes_beyond_its_scratch(env):
    P, torch = env
    cell = torch.zeros(4, dtype=torch.int32, device="cuda")
    perm = torch.zeros(4, dtype=torch.int32, device="cuda")
    with pytest.raises(P.PicError) as e:
        P.pic_tile_sort_perm_noalloc(cell, P.PIC_NOALLOC_MAX_PARTICLES + 1, 2, (32, 32, 1), (8, 8, 1), perm)
    assert e.value.code == P.PIC_ERR_INVALID_ARG
    bad = torch.tensor([0, 5, 32 * 32], dtype=torch.int32, device="cuda")
    with pytest.raises(P.PicError) as e:
        P.pic_tile_sort_perm_noalloc(bad, 3, 2, (32, 32, 1), (8, 8, 1), perm)
    assert e.value.code == P.PIC_ERR_INVALID_ARG
