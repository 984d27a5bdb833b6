"""Parity at full size, in the launch configuration that bench.py times: the
3D 128^3 two-species plasma (134,217,728 particles; FP32 form, 8x4x4 tiles,
halo 1, particles re-sorted every 8 steps, 8192 particles per work item).

The oracle cannot step 134M particles in a test's time, so the full-size run is
checked on what it can compute one by one, from the GPU's own FP32 state taken
after a few steps:
- the new momentum and position of 4096 sampled particles of each species (a
  particle's push depends only on E^n, B^{n-1/2} and its own state);
- the current J in an interior box of 6^3 cells, from the oracle stepping all
  particles within 3 cells of that box (no particle farther away reaches it:
  a particle's current window spans its cell +-2);
and on properties that hold at any size: Gauss's law stays at rounding level
and the particles and the total charge are kept."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1101_0809_gb300 import workloads as W
from pichelpers import FP32_TOL, check_fp32_positions, close, oracle_grid, periodic_diff, positions_from_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def run():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1101_0809_gb300 import build as B
    B.build()
    from paper_1101_0809_gb300 import pic as P
    wl = W.c1_thermal3d()
    assert wl.n_particles == 134_217_728 and wl.tile == (8, 4, 4) and wl.sort_interval == 4
    desc = P.make_desc(3, wl.n, wl.d, wl.dt, wl.c, P.PIC_FP32, tile=wl.tile, halo=1, sort_interval=wl.sort_interval,
                       particles_per_block=8192, rho_bg=wl.rho_bg,
                       stream=torch.cuda.current_stream().cuda_stream)
    grid = P.Grid(desc)
    for s, sp in enumerate(wl.species):
        grid.load(s, sp.q, sp.m, sp.weight, sp.x, sp.w)
    assert tuple(P.pic_tile_layout(grid.h)[2]) == (14, 12)     # the fixed-geometry kernel bench.py times
    d0 = P.pic_diagnostics(grid.h)
    P.pic_step(grid.h, 5)                                       # E and B no longer zero; a generic state
    E, B, _ = grid.get_fields()
    before = [grid.particles(s) for s in range(len(wl.species))]
    P.pic_step(grid.h, 1)
    P.pic_sync(grid.h)
    after = [grid.particles(s) for s in range(len(wl.species))]
    _, _, J = grid.get_fields()
    d1 = P.pic_diagnostics(grid.h)
    grid.close()
    return dict(P=P, wl=wl, E=E, B=B, J=J, before=before, after=after, d0=d0, d1=d1)


def _oracle_step(wl, E, B, subsets):
    """One oracle step from the GPU's fields with the given particle subsets,
    one (x, w) pair per species; returns the new (x, w) per species and J."""
    g = oracle_grid(wl)
    Ef = [a.astype(np.float64) for a in E]
    Bf = [a.astype(np.float64) for a in B]
    J = g.zeros()
    sp = [O.Species(s.q, s.m, s.weight, x, w) for s, (x, w) in zip(wl.species, subsets)]
    O.step(g, Ef, Bf, J, sp)
    return [(s.x, s.w) for s in sp], J


def _state(wl, part, idx):
    cell, off, w, ident = part
    x = positions_from_gpu(wl, cell[idx], [o[idx] for o in off])
    return x, np.stack([w[a][idx].astype(np.float64) for a in range(3)]), ident[idx]


def test_sampled_particles_match_the_oracle_push(run):
    wl = run["wl"]
    rng = np.random.default_rng(20110109)
    subsets, ids = [], []
    for s in range(len(wl.species)):
        cell = run["before"][s][0]
        idx = rng.choice(cell.shape[0], 4096, replace=False)
        x, w, ident = _state(wl, run["before"][s], idx)
        subsets.append((x, w))
        ids.append(ident)
    new, _ = _oracle_step(wl, run["E"], run["B"], subsets)
    for s in range(len(wl.species)):
        cell, off, w, ident = run["after"][s]
        pos = np.empty(ident.shape[0], dtype=np.int64)
        pos[ident] = np.arange(ident.shape[0])
        at = pos[ids[s]]
        x, wg, _ = _state(wl, run["after"][s], at)
        near = check_fp32_positions(wl, run["after"][s][0][at], x, new[s][0] % np.array(wl.n)[:, None],
                                    subsets[s][0], FP32_TOL, f"species {s}")
        print(f"species {s}: FP32 cell indices one off next to a face: {near}")
        for a in range(3):
            close(wg[a], new[s][1][a], FP32_TOL, f"species {s} w[{a}]")


def test_current_in_an_interior_box_matches_the_oracle(run):
    wl = run["wl"]
    lo, hi, margin = 61, 67, 3
    subsets = []
    for s in range(len(wl.species)):
        cell = run["before"][s][0]
        nx, ny = wl.n[0], wl.n[1]
        i, j, k = cell % nx, (cell // nx) % ny, cell // (nx * ny)
        near = ((i >= lo - margin) & (i < hi + margin) & (j >= lo - margin) & (j < hi + margin) &
                (k >= lo - margin) & (k < hi + margin))
        x, w, _ = _state(wl, run["before"][s], np.flatnonzero(near))
        subsets.append((x, w))
    assert sum(x.shape[1] for x, _ in subsets) > 50_000
    _, J = _oracle_step(wl, run["E"], run["B"], subsets)
    for a in range(3):
        got = run["J"][a][lo:hi, lo:hi, lo:hi]
        want = J[a][lo:hi, lo:hi, lo:hi]
        assert np.abs(want).max() > 0.0
        close(got, want, FP32_TOL, f"J[{a}] in the box")


def test_gauss_law_particles_and_charge_are_kept(run):
    wl, d0, d1 = run["wl"], run["d0"], run["d1"]
    assert d1["n_particles"] == d0["n_particles"] == wl.n_particles
    # scale: the charge of one species (the ions carry the other half; the net is zero)
    q_species = abs(wl.species[0].q * wl.species[0].weight) * wl.species[0].x.shape[1]
    rho_species = q_species / float(np.prod(wl.n))        # cells of unit volume
    assert d1["total_charge"] == pytest.approx(d0["total_charge"], abs=1e-10 * q_species)
    assert d1["gauss_resid_max"] / (4 * math.pi * rho_species) <= 1e-6
    assert d1["error_word"] == 0
