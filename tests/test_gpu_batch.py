"""Batched form: many independent runs of different sizes in one grid object,
advanced together by pic_step (multi-kernel), pic_step_persistent (one
cooperative launch per step) and pic_step_graph (CUDA graph replay).  Every run
must equal the FP64 oracle run on its own."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1101_0809_gb300 import workloads as W
from pichelpers import FP32_TOL, FP64_TOL, close, fp64_field_tol, positions_from_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1101_0809_gb300 import build as B
    B.build()
    from paper_1101_0809_gb300 import pic
    return pic, torch


def ensemble2d(k=5):
    """Small runs shaped like the batched ensemble: square and ragged grids,
    different ppc and v_th (c = 1, dt = 0.5, dx = Debye length)."""
    specs = [(32, 32, 6, 0.05), (36, 28, 4, 0.3), (48, 40, 10, 0.12), (24, 26, 8, 0.2), (40, 40, 3, 0.01)][:k]
    out = []
    for idx, (nx, ny, ppc, vth) in enumerate(specs):
        rng = np.random.Generator(np.random.PCG64(W.SEED_BASE + 300 + idx))
        count = nx * ny * ppc
        x = np.zeros((3, count))
        x[0] = rng.uniform(0, nx, count)
        x[1] = rng.uniform(0, ny, count)
        w = rng.normal(0, vth, (3, count))
        Wt = vth * vth / (4 * math.pi * ppc)
        sp = W.SpeciesInit("electrons", -1.0, 1.0, Wt, x, w)
        out.append(W.Workload(f"run{idx}", 2, (nx, ny, 1), (1.0, 1.0, 1.0), 0.5, 1.0, [sp], Wt * ppc, 6,
                              (16, 16, 1), 3))
    return out


def make_batch(P, runs, precision, stream=None, sort_interval=3):
    descs = [P.make_desc(wl.dims, wl.n, wl.d, wl.dt, wl.c, precision, tile=(16, 16, 1) if wl.dims == 2 else (8, 8, 8),
                         sort_interval=sort_interval, particles_per_block=1024, rho_bg=wl.rho_bg, stream=stream)
             for wl in runs]
    b = P.Batch(descs)
    for r, wl in enumerate(runs):
        for s, sp in enumerate(wl.species):
            b.load_run(r, s, sp.q, sp.m, sp.weight, sp.x, sp.w)
    return b


def oracle_run(wl, steps):
    g = O.Grid(wl.dims, wl.n, wl.d, wl.dt, wl.c)
    sp = [O.Species(s.q, s.m, s.weight, s.x.copy(), s.w.copy()) for s in wl.species]
    E, B, J = g.zeros(), g.zeros(), g.zeros()
    for _ in range(steps):
        O.step(g, E, B, J, sp)
    return g, sp, E, B, J


def check_run(P, b, r, wl, steps, tol):
    g, sp, E, B, J = oracle_run(wl, steps)
    gE, gB, gJ = b.get_fields_run(r)
    ftol = fp64_field_tol(wl, sp, tol) if tol == FP64_TOL else tol
    for a in range(3):
        close(gE[a], E[a], ftol, f"run {r} E[{a}]")
        close(gB[a], B[a], ftol, f"run {r} B[{a}]")
        close(gJ[a], J[a], ftol, f"run {r} J[{a}]")
    for s in range(len(wl.species)):
        cell, off, w, ident = b.particles_run(r, s)
        order = np.argsort(ident)
        x = positions_from_gpu(wl, cell[order], [o[order] for o in off])
        for a in range(wl.dims):
            d = x[a] - sp[s].x[a]
            d -= wl.n[a] * np.round(d / wl.n[a])
            assert np.abs(d).max() <= tol * max(1.0, math.sqrt(np.mean(sp[s].x[a] ** 2))), f"run {r} x[{a}]"
        for a in range(3):
            close(w[a][order], sp[s].w[a], tol, f"run {r} w[{a}]")


@pytest.mark.parametrize("mode", ["step", "persistent", "graph"])
def test_fp64_batch_runs_equal_their_oracle_runs(env, mode):
    P, torch = env
    runs = ensemble2d()
    st = torch.cuda.Stream()          # graph capture needs a non-default stream
    stream = st.cuda_stream
    b = make_batch(P, runs, P.PIC_FP64, stream=stream, sort_interval=3)
    assert P.pic_num_runs(b.h) == len(runs)
    steps = 9     # the graph path replays one 6-step graph and runs 3 steps uncaptured
    if mode == "step":
        P.pic_step(b.h, steps)
    elif mode == "persistent":
        P.pic_step_persistent(b.h, steps)
    else:
        P.pic_step_graph(b.h, steps)
    P.pic_sync(b.h)
    for r, wl in enumerate(runs):
        check_run(P, b, r, wl, steps, FP64_TOL)
    b.close()


def test_graph_replays_many_times_and_keeps_gauss_law(env):
    P, torch = env
    runs = ensemble2d(3)
    st = torch.cuda.Stream()
    stream = st.cuda_stream
    b = make_batch(P, runs, P.PIC_FP32, stream=stream, sort_interval=2)
    for r in range(len(runs)):
        P.pic_diagnostics_run(b.h, r)
    P.pic_step_graph(b.h, 41)
    P.pic_sync(b.h)
    for r, wl in enumerate(runs):
        d = P.pic_diagnostics_run(b.h, r)
        assert d["gauss_resid_max"] / (4 * math.pi * wl.rho_bg) <= 1e-6
        assert d["n_particles"] == wl.n_particles
    b.close()


def test_fp64_3d_batch_persistent(env):
    P, torch = env
    runs = [W.thermal_plasma("3D a", 3, (20, 18, 22), 2, 0.1, 4, W.SEED_BASE + 40, ions=1836.0,
                             tile=(8, 8, 8), dt_courant=0.45),
            W.thermal_plasma("3D b", 3, (18, 22, 20), 3, 0.2, 4, W.SEED_BASE + 41, tile=(8, 8, 8),
                             dt_courant=0.45)]
    descs = [P.make_desc(3, wl.n, wl.d, wl.dt, wl.c, P.PIC_FP64, tile=(8, 8, 8), sort_interval=2,
                         rho_bg=wl.rho_bg, stream=torch.cuda.current_stream().cuda_stream) for wl in runs]
    b = P.Batch(descs)
    for r, wl in enumerate(runs):
        for s, sp in enumerate(wl.species):
            b.load_run(r, s, sp.q, sp.m, sp.weight, sp.x, sp.w)
    P.pic_step_persistent(b.h, 4)
    P.pic_sync(b.h)
    for r, wl in enumerate(runs):
        check_run(P, b, r, wl, 4, FP64_TOL)
    b.close()


def test_batch_rejects_mixed_dims(env):
    P, torch = env
    d2 = P.make_desc(2, (32, 32, 1), (1.0, 1.0, 1.0), 0.5, 1.0)
    d3 = P.make_desc(3, (20, 20, 20), (1.0, 1.0, 1.0), 0.3, 1.0)
    with pytest.raises(P.PicError) as e:
        P.Batch([d2, d3])
    assert e.value.code == P.PIC_ERR_INVALID_ARG


def test_graph_replay_refuses_the_legacy_default_stream(env):
    P, torch = env
    runs = ensemble2d(1)
    b = make_batch(P, runs, P.PIC_FP32, stream=None)
    with pytest.raises(P.PicError) as e:
        P.pic_step_graph(b.h, 8)
    assert e.value.code == P.PIC_ERR_INVALID_ARG
    b.close()


def test_bulk_load_equals_run_by_run_loads(env):
    P, torch = env
    runs = ensemble2d(4)
    b1 = make_batch(P, runs, P.PIC_FP64)
    descs = [P.make_desc(2, wl.n, wl.d, wl.dt, wl.c, P.PIC_FP64, tile=(16, 16, 1), sort_interval=3,
                         particles_per_block=1024, rho_bg=wl.rho_bg) for wl in runs]
    b2 = P.Batch(descs)
    P.pic_load_particles_runs(b2.h, list(range(len(runs))), 0,
                              [(wl.species[0].q, wl.species[0].m, wl.species[0].weight) for wl in runs],
                              [list(wl.species[0].x) for wl in runs], [list(wl.species[0].w) for wl in runs])
    for r in range(len(runs)):
        for u, v in zip(b1.particles_run(r, 0), b2.particles_run(r, 0)):
            if isinstance(u, list):
                for p, q in zip(u, v):
                    np.testing.assert_array_equal(p, q)
            else:
                np.testing.assert_array_equal(u, v)
    P.pic_step(b1.h, 4)
    P.pic_step(b2.h, 4)
    for r, wl in enumerate(runs):
        E1, B1, J1 = b1.get_fields_run(r)
        E2, B2, J2 = b2.get_fields_run(r)
        for a in range(3):
            close(J2[a], J1[a], FP64_TOL, f"run {r} J[{a}]")
            close(E2[a], E1[a], FP64_TOL, f"run {r} E[{a}]")
    b1.close()
    b2.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_persistent_step_after_a_sort_equals_an_explicit_sort(env, prec):
    """When a persistent step reaches the sort interval, the sort leaves the
    arrays in place and the cooperative launch reads the particles through the
    permutation, writing them in the new order.  From one snapshot that step
    equals pic_sort followed by a persistent step: the ids slot by slot, bit for
    bit, and positions and momenta to a few units of the last place (the two
    launches are separate compilations of the same arithmetic)."""
    P, torch = env
    runs = ensemble2d(4)
    st = torch.cuda.Stream()
    b = make_batch(P, runs, P.PIC_FP32 if prec == "fp32" else P.PIC_FP64, stream=st.cuda_stream, sort_interval=3)
    P.pic_step_persistent(b.h, 3)                 # the next step sorts first
    P.pic_sync(b.h)
    blob = np.empty(P.pic_state_bytes(b.h), dtype=np.uint8)
    P.pic_state_save(b.h, blob)
    P.pic_step_persistent(b.h, 1)
    P.pic_sync(b.h)
    inside = [b.particles_run(r, 0) for r in range(len(runs))]
    P.pic_state_restore(b.h, blob)
    before = [b.particles_run(r, 0)[3] for r in range(len(runs))]
    P.pic_sort(b.h)
    P.pic_step_persistent(b.h, 1)
    P.pic_sync(b.h)
    ulp = 2.0 ** -23 if prec == "fp32" else 2.0 ** -52
    moved = 0
    for r, wl in enumerate(runs):
        got = b.particles_run(r, 0)
        np.testing.assert_array_equal(inside[r][3], got[3])
        xa = positions_from_gpu(wl, inside[r][0], inside[r][1])
        xb = positions_from_gpu(wl, got[0], got[1])
        for a in range(2):
            d = xa[a] - xb[a]
            d -= wl.n[a] * np.round(d / wl.n[a])
            assert np.abs(d).max() <= 8 * ulp, f"run {r} axis {a}: positions differ by {np.abs(d).max()} cells"
        for a in range(3):
            wa = np.asarray(inside[r][2][a], np.float64)
            wb = np.asarray(got[2][a], np.float64)
            scale = np.sqrt(np.mean(wb * wb))
            assert np.all(np.abs(wa - wb) <= 8 * ulp * np.maximum(np.abs(wb), scale)), f"run {r} momentum {a}"
        moved += int(np.count_nonzero(got[3] != before[r]))
    assert moved > 0                               # the sort did reorder particles
    b.close()
