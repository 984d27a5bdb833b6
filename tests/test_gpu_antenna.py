"""The plane-wave antenna and the laser-plasma slab (test sizes of the 3D
laser-plasma workload) against the FP64 oracle, through the C ABI: FP64 runs
step by step with the antenna's clock, an FP32 step from the rounded oracle
state in the middle of the pulse (the fixed-geometry 8x4x4 kernel), Gauss's law
over many FP32 steps with relativistic electrons, and batches in which one run
has an antenna (multi-kernel, persistent and graph paths)."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1101_0809_gb300 import workloads as W
from pichelpers import (FP32_TOL, FP64_TOL, check_fp32_positions, close, compare_particles, make_grid, oracle_grid,
                        oracle_species, positions_from_gpu)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1101_0809_gb300 import build as B
    B.build()
    from paper_1101_0809_gb300 import pic
    return pic


def slab(which, steps=None):
    """Test sizes of the laser slab, with a quarter-period rise so that the
    pulse reaches the plasma at full strength within a few dozen steps."""
    if which == "2d":
        return W.c2_laser_slab(n=(96, 16, 1), dims=2, slab=(24.0, 32.0, 72.0), tile=(8, 8, 1), steps=steps or 70,
                               ramp_periods=0.25)
    return W.c2_laser_slab(n=(64, 16, 16), dims=3, slab=(16.0, 20.0, 44.0), plane=4, ppc=4, steps=steps or 40,
                           ramp_periods=0.25)


def antenna_of(wl):
    a = wl.antenna
    return O.Antenna(a["pol"], a["plane"], a["amplitude"], a["omega"], a["ramp"])


def set_antenna(P, h, wl, run=0, start=0):
    a = wl.antenna
    P.pic_set_antenna(h, run, a["pol"], a["plane"], a["amplitude"], a["omega"], a["ramp"], start)


def oracle_run(wl, steps, start=0, species=None, fields=None):
    g = oracle_grid(wl)
    sp = species if species is not None else oracle_species(wl)
    E, B, J = fields if fields is not None else (g.zeros(), g.zeros(), g.zeros())
    ant = antenna_of(wl)
    for s in range(start, start + steps):
        O.step(g, E, B, J, sp, antenna=ant, n=s)
    return g, sp, E, B, J


def close_vector(got, want, tol, what):
    """Element-wise comparison of the three components of a vector field on the
    field's scale: |a - b| <= tol * max(|b|, s) with s the RMS over all three
    components.  In the laser runs the longitudinal components are about 1e-9 of
    the transverse ones and carry the oracle's rounding of absolute positions
    (a small displacement of a particle at x ~ 50 keeps only ~1e-10 of its
    digits), so they are judged on the scale of the field they belong to."""
    s = math.sqrt(sum(float(np.mean(np.asarray(w, np.float64) ** 2)) for w in want) / 3.0)
    for a in range(3):
        g = np.asarray(got[a], np.float64)
        w = np.asarray(want[a], np.float64)
        err = np.abs(g - w)
        bad = err > tol * np.maximum(np.abs(w), s) + 1e-300
        assert not bad.any(), (f"{what}[{a}]: {int(bad.sum())}/{w.size} elements off, worst "
                               f"{float((err / np.maximum(np.abs(w), s)).max()):.3e} on the field's scale")


def compare_particles_vector(wl, grid, osp, tol, x_prev=None):
    """Positions per axis (FP64: on the position scale; FP32 with x_prev: in
    cells, with the cell indices, by check_fp32_positions) and momenta on the
    scale of |w| over all three components, for the reason given above."""
    cell, off, w, ident = grid.particles(0)
    order = np.argsort(ident)
    x = positions_from_gpu(wl, cell[order], [o[order] for o in off])
    ref = osp[0]
    if x_prev is None:
        for a in range(wl.dims):
            d = x[a] - ref.x[a]
            d -= wl.n[a] * np.round(d / wl.n[a])
            assert np.abs(d).max() <= tol * max(1.0, math.sqrt(float(np.mean(ref.x[a] ** 2)))), f"x[{a}]"
    else:
        near = check_fp32_positions(wl, cell[order], x, ref.x, x_prev, tol, "electrons")
        print(f"FP32 cell indices one off next to a face: {near}")
    close_vector([wa[order] for wa in w], list(ref.w), tol, "w")


def check_fields(grid, E, B, J, tol):
    gE, gB, gJ = grid.get_fields()
    close_vector(gE, E, tol, "E")
    close_vector(gB, B, tol, "B")
    close_vector(gJ, J, tol, "J")


@pytest.mark.parametrize("which", ["2d", "3d"])
def test_fp64_laser_slab_matches_oracle(P, which):
    wl = slab(which)
    grid = make_grid(P, wl, P.PIC_FP64)
    set_antenna(P, grid.h, wl)
    P.pic_step(grid.h, wl.steps)
    P.pic_sync(grid.h)
    g, osp, E, B, J = oracle_run(wl, wl.steps)
    assert np.abs(B[2]).max() > 0.1 * wl.antenna["amplitude"]      # the pulse is in the box
    check_fields(grid, E, B, J, FP64_TOL)
    compare_particles_vector(wl, grid, osp, FP64_TOL)
    grid.close()


def test_fp32_laser_slab_step_from_rounded_state(P):
    wl = slab("3d")
    start = 32                                   # the pulse front is inside the slab
    g, osp, E, B, J = oracle_run(wl, start)
    grid = make_grid(P, wl, P.PIC_FP32)
    assert tuple(P.pic_tile_layout(grid.h)[2]) == (14, 12)    # fixed-geometry kernel
    grid.set_fields([a.astype(np.float32) for a in E], [a.astype(np.float32) for a in B])
    sp = osp[0]
    grid.load(0, sp.q, sp.m, sp.weight, sp.x, sp.w.astype(np.float32).astype(np.float64))
    cell, off, w, ident = grid.particles(0)
    order = np.argsort(ident)
    sp.x[:] = positions_from_gpu(wl, cell[order], [o[order] for o in off])
    for a in range(3):
        sp.w[a][:] = w[a][order]
    E = [a.astype(np.float32).astype(np.float64) for a in E]
    B = [a.astype(np.float32).astype(np.float64) for a in B]
    set_antenna(P, grid.h, wl, start=start)
    x_prev = sp.x.copy()
    P.pic_step(grid.h, 1)
    P.pic_sync(grid.h)
    oracle_run(wl, 1, start=start, species=osp, fields=(E, B, J))
    assert np.abs(osp[0].w).max() > 0.5                      # relativistic electrons
    check_fields(grid, E, B, J, FP32_TOL)
    compare_particles_vector(wl, grid, osp, FP32_TOL, x_prev=x_prev)
    grid.close()


def test_fp32_laser_slab_keeps_gauss_law(P):
    """Gauss's residual drift over 120 FP32 steps.  Here the laser field is
    about 1600 times 4 pi |q| n dx (an underdense slab), so the rounding of the
    FP32 field updates, not the charge density, sets the scale: each step rounds
    E (of size max|E|) to 2^-24, and the rounding errors of neighbouring cells
    enter div_h E as a random walk.  The drift is judged against
    4 eps32 sqrt(steps) max|E| / dx (eps32 = 2^-24); the scheme's own charge
    conservation is exact, so anything systematic would exceed it."""
    wl = slab("3d", steps=120)
    grid = make_grid(P, wl, P.PIC_FP32)
    set_antenna(P, grid.h, wl)
    d0 = P.pic_diagnostics(grid.h)
    P.pic_step(grid.h, wl.steps)
    d = P.pic_diagnostics(grid.h)
    gE, gB, gJ = grid.get_fields()
    emax = max(float(np.abs(np.asarray(a, np.float64)).max()) for a in gE)
    assert emax > 0.5 * wl.antenna["amplitude"]
    bound = 4 * 2.0 ** -24 * math.sqrt(wl.steps) * emax / wl.d[0]
    assert d["gauss_resid_max"] <= bound
    assert d["n_particles"] == wl.n_particles
    assert d["total_charge"] == pytest.approx(d0["total_charge"], rel=1e-9)
    assert d["kinetic"] > 0.0 and d["field_E"] > 0.0
    grid.close()


@pytest.mark.parametrize("mode", ["step", "persistent", "graph"])
def test_fp64_batch_with_one_antenna(P, mode):
    import torch
    runs = [slab("2d"), W.c2_laser_slab(n=(80, 16, 1), dims=2, slab=(20.0, 30.0, 60.0), tile=(8, 8, 1), steps=70,
                                        seed_offset=12)]
    st = torch.cuda.Stream()
    descs = [P.make_desc(2, wl.n, wl.d, wl.dt, wl.c, P.PIC_FP64, tile=(8, 8, 1), sort_interval=4,
                         rho_bg=0.0, stream=st.cuda_stream) for wl in runs]
    b = P.Batch(descs)
    for r, wl in enumerate(runs):
        sp = wl.species[0]
        b.load_run(r, 0, sp.q, sp.m, sp.weight, sp.x, sp.w)
    set_antenna(P, b.h, runs[0], run=0)          # the second run has none
    steps = 8 * 4 + 9 if mode == "graph" else 41
    if mode == "step":
        P.pic_step(b.h, steps)
    elif mode == "persistent":
        P.pic_step_persistent(b.h, steps)
    else:
        P.pic_step_graph(b.h, steps)
    P.pic_sync(b.h)
    for r, wl in enumerate(runs):
        g = oracle_grid(wl)
        sp = oracle_species(wl)
        E, B, J = g.zeros(), g.zeros(), g.zeros()
        ant = antenna_of(wl) if r == 0 else None
        for s in range(steps):
            O.step(g, E, B, J, sp, antenna=ant, n=s)
        gE, gB, gJ = b.get_fields_run(r)
        close_vector(gE, E, FP64_TOL, f"run {r} E")
        close_vector(gB, B, FP64_TOL, f"run {r} B")
        if r == 1:
            assert np.abs(gB[2]).max() == 0.0 and np.abs(gE[1]).max() == 0.0   # no wave without an antenna
    b.close()


def test_antenna_arguments_are_checked(P):
    wl = slab("2d")
    grid = make_grid(P, wl, P.PIC_FP64)
    for kw in (dict(polarization=3, plane=8), dict(polarization=1, plane=0), dict(polarization=1, plane=96),
               dict(polarization=1, plane=8, ramp=-1.0), dict(polarization=1, plane=8, start=-1)):
        with pytest.raises(P.PicError) as e:
            P.pic_set_antenna(grid.h, 0, **kw)
        assert e.value.code == P.PIC_ERR_INVALID_ARG
    with pytest.raises(P.PicError):
        P.pic_set_antenna(grid.h, 1, 1, 8)
    P.pic_set_antenna(grid.h, 0, 1, 8, 1.0, 0.3, 0.0)
    P.pic_set_antenna(grid.h, 0)                 # removal
    P.pic_step(grid.h, 5)
    gE, gB, gJ = grid.get_fields()
    assert np.abs(gB[2]).max() == 0.0            # cold slab, no wave: nothing moves
    grid.close()
