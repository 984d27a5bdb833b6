"""The FP32 kernels compiled for fixed tile geometries (3D 8x4x4, 2D 16x16 and
8x8, halo 1; 3D 4x4x4 with halo 2) against the FP64 oracle.  The library picks them whenever a grid's
tile, halo and shared-tile pitches equal theirs; pic_tile_layout shows the
pitches, so each test first checks that its grid has the fixed geometry.  The
oracle starts from exactly the FP32 state the GPU holds (positions and momenta
read back), so the comparison measures the FP32 arithmetic of the steps."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1101_0809_gb300 import workloads as W
from pichelpers import FP32_TOL, close, compare_particles, make_grid, positions_from_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1101_0809_gb300 import build as B
    B.build()
    from paper_1101_0809_gb300 import pic
    return pic, torch


def plasma3d(steps=1):
    """3D3V electrons and ions on a grid ragged against 8x4x4 tiles."""
    return W.thermal_plasma("3D 8x4x4 tiles", 3, (20, 18, 22), 4, 0.1, steps, W.SEED_BASE + 51, ions=1836.0,
                            tile=(8, 4, 4), dt_courant=0.45)


def oracle_from_gpu(wl, particles):
    """Oracle species holding the GPU's FP32 state, in load order."""
    out = []
    for s, sp in enumerate(wl.species):
        cell, off, w, ident = particles(s)
        order = np.argsort(ident)
        x = positions_from_gpu(wl, cell[order], [o[order] for o in off])
        out.append(O.Species(sp.q, sp.m, sp.weight, x, np.array([a[order] for a in w], dtype=np.float64)))
    return out


def test_fp32_3d_fixed_tile_one_step_matches_oracle(env):
    P, torch = env
    wl = plasma3d()
    grid = make_grid(P, wl, P.PIC_FP32)
    assert tuple(P.pic_tile_layout(grid.h)[2]) == (14, 12), "the grid does not have the fixed 8x4x4 geometry"
    osp = oracle_from_gpu(wl, grid.particles)
    g = O.Grid(wl.dims, wl.n, wl.d, wl.dt, wl.c)
    E, B, J = g.zeros(), g.zeros(), g.zeros()
    x_prev = [sp.x.copy() for sp in osp]
    P.pic_step(grid.h, 1)
    P.pic_sync(grid.h)
    O.step(g, E, B, J, osp)
    gE, gB, gJ = grid.get_fields()
    for a in range(3):
        close(gE[a], E[a], FP32_TOL, f"E[{a}]")
        close(gB[a], B[a], FP32_TOL, f"B[{a}]")
        close(gJ[a], J[a], FP32_TOL, f"J[{a}]")
    for s in range(len(wl.species)):
        compare_particles(wl, s, grid, osp, FP32_TOL, x_prev=x_prev[s])
    grid.close()


def test_fp32_3d_fixed_tile_keeps_gauss_law_over_100_steps(env):
    P, torch = env
    wl = plasma3d(steps=100)
    grid = make_grid(P, wl, P.PIC_FP32)
    assert tuple(P.pic_tile_layout(grid.h)[2]) == (14, 12)
    d0 = P.pic_diagnostics(grid.h)
    P.pic_step(grid.h, wl.steps)
    d = P.pic_diagnostics(grid.h)
    # electrons and ions of equal count and opposite charge: the scale is 4 pi |q_e| n_e
    sp = wl.species[0]
    scale = 4 * math.pi * abs(sp.q) * sp.weight * sp.n / (wl.n_cells * wl.volume)
    assert d["gauss_resid_max"] / scale <= 1e-6
    assert d["n_particles"] == wl.n_particles
    assert d["total_charge"] == pytest.approx(d0["total_charge"], abs=1e-9 * abs(sp.q) * sp.weight * sp.n)
    grid.close()


def plasma3d_444(steps, vth):
    """3D3V electrons and ions on a grid ragged against 4x4x4 tiles."""
    return W.thermal_plasma("3D 4x4x4 tiles", 3, (18, 14, 22), 4, vth, steps, W.SEED_BASE + 52, ions=1836.0,
                            tile=(4, 4, 4), dt_courant=0.45)


@pytest.mark.parametrize("steps,vth", [(1, 0.1), (10, 0.3)])
def test_fp32_3d_444_halo2_fixed_tile_matches_oracle(env, steps, vth):
    """The 4x4x4 tile with a two-cell halo (the laser slab's tiles at its long
    sort interval).  Ten unsorted steps of a plasma at v_th = 0.3c carry
    particles past one cell of halo, within two (the tiled path), and past two
    (the global-memory path)."""
    P, torch = env
    wl = plasma3d_444(steps, vth)
    grid = make_grid(P, wl, P.PIC_FP32, halo=2, sort_interval=1000)
    assert tuple(P.pic_tile_layout(grid.h)[2]) == (12, 12), "the grid does not have the fixed 4x4x4 halo-2 geometry"
    osp = oracle_from_gpu(wl, grid.particles)
    g = O.Grid(wl.dims, wl.n, wl.d, wl.dt, wl.c)
    E, B, J = g.zeros(), g.zeros(), g.zeros()
    x_prev = [sp.x.copy() for sp in osp]
    for _ in range(steps):
        x_prev = [sp.x.copy() for sp in osp]
        O.step(g, E, B, J, osp)
    P.pic_step(grid.h, steps)
    P.pic_sync(grid.h)
    tol = steps * FP32_TOL
    gE, gB, gJ = grid.get_fields()
    for a in range(3):
        close(gE[a], E[a], tol, f"E[{a}]")
        close(gB[a], B[a], tol, f"B[{a}]")
        close(gJ[a], J[a], tol, f"J[{a}]")
    if steps == 1:
        for s in range(len(wl.species)):
            compare_particles(wl, s, grid, osp, FP32_TOL, x_prev=x_prev[s])
    else:
        for s, sp in enumerate(wl.species):
            cell, off, w, ident = grid.particles(s)
            order = np.argsort(ident)
            x = positions_from_gpu(wl, cell[order], [o[order] for o in off])
            for a in range(3):
                d = x[a] - osp[s].x[a]
                d -= wl.n[a] * np.round(d / wl.n[a])
                assert np.abs(d).max() <= 1e-4, f"species {s} x[{a}]: {np.abs(d).max()} cells"
                close(w[a][order], osp[s].w[a], tol, f"species {s} w[{a}]")
            # some electrons ran past two cells of halo (the global path) and some past one
            if s == 0:
                c0 = [np.floor(sp.x[a][ident]).astype(np.int64) % wl.n[a] for a in range(3)]
                c = [cell % wl.n[0], (cell // wl.n[0]) % wl.n[1], cell // (wl.n[0] * wl.n[1])]
                far = np.zeros(cell.size, dtype=int)
                for a in range(3):
                    o = (c0[a] // 4) * 4
                    dd = (c[a] - o) % wl.n[a]
                    dd = np.where(dd >= wl.n[a] - 6, dd - wl.n[a], dd)
                    far = np.maximum(far, np.maximum(-dd, dd - 3))   # cells outside the tile
                assert (far > 2).any() and (far == 2).any()
    grid.close()


def ensemble2d():
    specs = [(32, 32, 6, 0.05), (36, 28, 4, 0.3), (48, 40, 10, 0.12), (24, 26, 8, 0.2)]
    runs = []
    for idx, (nx, ny, ppc, vth) in enumerate(specs):
        rng = np.random.Generator(np.random.PCG64(W.SEED_BASE + 500 + idx))
        count = nx * ny * ppc
        x = np.zeros((3, count))
        x[0] = rng.uniform(0, nx, count)
        x[1] = rng.uniform(0, ny, count)
        w = rng.normal(0, vth, (3, count))
        Wt = vth * vth / (4 * math.pi * ppc)
        sp = W.SpeciesInit("electrons", -1.0, 1.0, Wt, x, w)
        runs.append(W.Workload(f"run{idx}", 2, (nx, ny, 1), (1.0, 1.0, 1.0), 0.5, 1.0, [sp], Wt * ppc, 6,
                               (16, 16, 1), 3))
    return runs


@pytest.mark.parametrize("tile,pitch", [(16, (22, 22)), (8, (20, 14))])
@pytest.mark.parametrize("mode", ["step", "persistent", "graph"])
def test_fp32_2d_batch_fixed_tiles_match_oracle(env, tile, pitch, mode):
    P, torch = env
    runs = ensemble2d()
    st = torch.cuda.Stream()
    descs = [P.make_desc(2, wl.n, wl.d, wl.dt, wl.c, P.PIC_FP32, tile=(tile, tile, 1), sort_interval=3,
                         particles_per_block=1024, rho_bg=wl.rho_bg, stream=st.cuda_stream) for wl in runs]
    b = P.Batch(descs)
    for r, wl in enumerate(runs):
        sp = wl.species[0]
        b.load_run(r, 0, sp.q, sp.m, sp.weight, sp.x, sp.w)
    assert tuple(P.pic_tile_layout(b.h)[2]) == pitch
    osps = [oracle_from_gpu(wl, lambda s, r=r: b.particles_run(r, s)) for r, wl in enumerate(runs)]
    # the graph path captures 2K = 6 steps; one replay.  The per-step FP32 bar
    # accumulates over the steps taken.
    steps = 6 if mode == "graph" else 1
    if mode == "step":
        P.pic_step(b.h, steps)
    elif mode == "persistent":
        P.pic_step_persistent(b.h, steps)
    else:
        P.pic_step_graph(b.h, steps)
    P.pic_sync(b.h)
    tol = steps * FP32_TOL
    for r, wl in enumerate(runs):
        g = O.Grid(2, wl.n, wl.d, wl.dt, wl.c)
        E, B, J = g.zeros(), g.zeros(), g.zeros()
        osp = osps[r]
        for _ in range(steps):
            O.step(g, E, B, J, osp)
        gE, gB, gJ = b.get_fields_run(r)
        for a in range(3):
            close(gE[a], E[a], tol, f"run {r} E[{a}]")
            close(gB[a], B[a], tol, f"run {r} B[{a}]")
            close(gJ[a], J[a], tol, f"run {r} J[{a}]")
        cell, off, w, ident = b.particles_run(r, 0)
        order = np.argsort(ident)
        x = positions_from_gpu(wl, cell[order], [o[order] for o in off])
        for a in range(2):
            d = x[a] - osp[0].x[a]
            d -= wl.n[a] * np.round(d / wl.n[a])
            assert np.abs(d).max() <= tol * max(1.0, math.sqrt(np.mean(osp[0].x[a] ** 2))), f"run {r} x[{a}]"
        for a in range(3):
            close(w[a][order], osp[0].w[a], tol, f"run {r} w[{a}]")
    b.close()
