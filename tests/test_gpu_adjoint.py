"""GPU discrete adjoint: one adjoint step against the oracle's hand-derived
adjoint on the same state, the gradient of a window field energy after 20 steps
with respect to the density-perturbation amplitude against the oracle adjoint
and against central finite differences of the GPU forward run, and state
snapshots (checkpoint/restart)."""
import math
import os
import tempfile

import numpy as np
import pytest

import oracle as O
from paper_1101_0809_gb300 import workloads as W
from pichelpers import close, fp64_field_tol, oracle_grid, positions_from_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1101_0809_gb300 import build as B
    B.build()
    from paper_1101_0809_gb300 import pic
    return pic, torch


def _state_after(wl, steps):
    g = oracle_grid(wl)
    sp = [O.Species(s.q, s.m, s.weight, s.x.copy(), s.w.copy()) for s in wl.species]
    E, B, J = g.zeros(), g.zeros(), g.zeros()
    for _ in range(steps):
        O.step(g, E, B, J, sp)
    return g, sp, E, B


@pytest.mark.parametrize("tiled", [True, False])
@pytest.mark.parametrize("which", ["2d", "3d"])
def test_adjoint_step_matches_oracle(env, which, tiled):
    P, torch = env
    if which == "2d":
        wl = W.c4_perturbed2d(n=32, ppc=8, steps=3)
    else:
        wl = W.thermal_plasma("3D small", 3, (20, 18, 22), 2, 0.1, 3, W.SEED_BASE + 11, ions=1836.0,
                              tile=(8, 8, 8), dt_courant=0.45)
    g, sp, E, B = _state_after(wl, 3)
    desc = P.make_desc(wl.dims, wl.n, wl.d, wl.dt, wl.c, P.PIC_FP64, tile=wl.tile, rho_bg=wl.rho_bg)
    grid = P.Grid(desc)
    P.pic_set_adjoint_tiled(grid.h, tiled)
    grid.set_fields(E, B)
    for s, o in enumerate(sp):
        grid.load(s, o.q, o.m, o.weight, o.x, o.w)
    rng = np.random.default_rng(77)
    lamE = [rng.normal(size=g.shape) for _ in range(3)]
    lamB = [rng.normal(size=g.shape) for _ in range(3)]
    lx = [rng.normal(size=(3, o.x.shape[1])) for o in sp]
    lw = [rng.normal(size=(3, o.x.shape[1])) for o in sp]
    if wl.dims == 2:
        for a in lx:
            a[2] = 0.0
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    gE = [dev(a) for a in lamE]
    gB = [dev(a) for a in lamB]
    gx = [dev(np.concatenate([a[c] for a in lx])) for c in range(3)]
    gw = [dev(np.concatenate([a[c] for a in lw])) for c in range(3)]
    torch.cuda.synchronize()
    P.pic_adjoint_step(grid.h, gE, gB, gx, gw)
    torch.cuda.synchronize()
    O.step_adj(g, E, B, sp, lamE, lamB, lx, lw)
    tol = 1e-11
    for a in range(3):
        close(gE[a].cpu().numpy(), lamE[a], tol, f"lamE[{a}]")
        close(gB[a].cpu().numpy(), lamB[a], tol, f"lamB[{a}]")
        close(gw[a].cpu().numpy(), np.concatenate([v[a] for v in lw]), tol, f"lamw[{a}]")
        if a < wl.dims:
            close(gx[a].cpu().numpy(), np.concatenate([v[a] for v in lx]), tol, f"lamx[{a}]")
    grid.close()


@pytest.mark.parametrize("which", ["2d", "3d"])
def test_fp32_tiled_adjoint_fixed_point_tiles_match_oracle(env, which):
    """The FP32 tiled adjoint sums the transposed gather in fixed-point tiles at
    a scale set from the previous launch's largest lambda; the first launch has
    no such scale and scatters into the global arrays.  Both launches, on the
    same FP32 state and adjoint inputs, against the oracle's FP64 adjoint of that
    state (FP32 tolerance), and against each other."""
    P, torch = env
    if which == "2d":
        wl = W.c4_perturbed2d(n=32, ppc=8, steps=3)
        tile = (8, 8, 1)
    else:
        wl = W.thermal_plasma("3D small", 3, (20, 18, 22), 2, 0.1, 3, W.SEED_BASE + 11, ions=1836.0,
                              tile=(8, 4, 4), dt_courant=0.45)
        tile = (8, 4, 4)
    desc = P.make_desc(wl.dims, wl.n, wl.d, wl.dt, wl.c, P.PIC_FP32, tile=tile, rho_bg=wl.rho_bg)
    grid = P.Grid(desc)
    P.pic_set_adjoint_tiled(grid.h, True)
    for s, o in enumerate(wl.species):
        grid.load(s, o.q, o.m, o.weight, o.x, o.w)
    P.pic_step(grid.h, 3)
    P.pic_sync(grid.h)
    g = oracle_grid(wl)
    E, B, _ = grid.get_fields()
    E = [np.asarray(a, np.float64) for a in E]
    B = [np.asarray(a, np.float64) for a in B]
    sp = []
    for s, o in enumerate(wl.species):
        cell, off, w, ident = grid.particles(s)
        order = np.argsort(ident)
        x = positions_from_gpu(wl, cell[order], [a[order] for a in off])
        sp.append(O.Species(o.q, o.m, o.weight, x, np.array([a[order] for a in w], dtype=np.float64)))
    rng = np.random.default_rng(79)
    lamE = [rng.normal(size=g.shape).astype(np.float32).astype(np.float64) for _ in range(3)]
    lamB = [rng.normal(size=g.shape).astype(np.float32).astype(np.float64) for _ in range(3)]
    lx = [rng.normal(size=(3, o.x.shape[1])).astype(np.float32).astype(np.float64) for o in sp]
    lw = [rng.normal(size=(3, o.x.shape[1])).astype(np.float32).astype(np.float64) for o in sp]
    if wl.dims == 2:
        for a in lx:
            a[2] = 0.0
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a).astype(np.float32)).cuda()
    got = []
    for launch in range(2):
        gE = [dev(a) for a in lamE]
        gB = [dev(a) for a in lamB]
        gx = [dev(np.concatenate([a[c] for a in lx])) for c in range(3)]
        gw = [dev(np.concatenate([a[c] for a in lw])) for c in range(3)]
        torch.cuda.synchronize()
        P.pic_adjoint_step(grid.h, gE, gB, gx, gw)
        torch.cuda.synchronize()
        got.append([[t.cpu().numpy().astype(np.float64) for t in v] for v in (gE, gB, gx, gw)])
    O.step_adj(g, E, B, sp, lamE, lamB, lx, lw)
    want = (lamE, lamB, [np.concatenate([v[a] for v in lx]) for a in range(3)],
            [np.concatenate([v[a] for v in lw]) for a in range(3)])
    for launch in range(2):
        for name, gv, wv in zip(("lamE", "lamB", "lamx", "lamw"), got[launch], want):
            for a in range(3):
                if name == "lamx" and a >= wl.dims:
                    continue
                close(gv[a], wv[a], 1e-4, f"launch {launch} {name}[{a}]")
    for name, g0, g1 in zip(("lamE", "lamB", "lamx", "lamw"), got[0], got[1]):
        for a in range(3):
            close(g1[a], g0[a], 2e-5, f"fixed-point tiles vs global scatter {name}[{a}]")
    grid.close()


@pytest.mark.parametrize("which", ["2d", "3d"])
def test_tiled_adjoint_with_particles_past_their_tiles(env, which):
    """Halo 0 and no sort for 4 steps: every particle that left its tile since
    the load takes the global-memory form inside the tiled kernel.  Both forms
    against the oracle's adjoint on the state the GPU reached."""
    P, torch = env
    if which == "2d":
        wl = W.c4_perturbed2d(n=32, ppc=8, steps=4)
        tile = (8, 8, 1)
    else:
        wl = W.thermal_plasma("3D small", 3, (20, 18, 22), 2, 0.1, 4, W.SEED_BASE + 11, ions=1836.0,
                              tile=(8, 8, 8), dt_courant=0.45)
        tile = (8, 8, 8)
    desc = P.make_desc(wl.dims, wl.n, wl.d, wl.dt, wl.c, P.PIC_FP64, tile=tile, halo=0, sort_interval=1000,
                       rho_bg=wl.rho_bg)
    grid = P.Grid(desc)
    for s, o in enumerate(wl.species):
        grid.load(s, o.q, o.m, o.weight, o.x, o.w)
    P.pic_step(grid.h, 4)
    P.pic_sync(grid.h)
    g = oracle_grid(wl)
    E, B, _ = grid.get_fields()
    sp = []
    left = 0
    for s, o in enumerate(wl.species):
        cell, off, w, ident = grid.particles(s)
        order = np.argsort(ident)
        x = positions_from_gpu(wl, cell[order], [a[order] for a in off])
        sp.append(O.Species(o.q, o.m, o.weight, x, np.array([a[order] for a in w])))
        t = [np.floor(x[a] / tile[a]) != np.floor(o.x[a] / tile[a]) for a in range(wl.dims)]
        left += int(np.any(t, axis=0).sum())
    assert left > 20            # particles outside their tiles since the load
    rng = np.random.default_rng(78)
    lamE = [rng.normal(size=g.shape) for _ in range(3)]
    lamB = [rng.normal(size=g.shape) for _ in range(3)]
    lx = [rng.normal(size=(3, o.x.shape[1])) for o in sp]
    lw = [rng.normal(size=(3, o.x.shape[1])) for o in sp]
    if wl.dims == 2:
        for a in lx:
            a[2] = 0.0
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    got = {}
    for tiled in (True, False):
        gE = [dev(a) for a in lamE]
        gB = [dev(a) for a in lamB]
        gx = [dev(np.concatenate([a[c] for a in lx])) for c in range(3)]
        gw = [dev(np.concatenate([a[c] for a in lw])) for c in range(3)]
        torch.cuda.synchronize()
        P.pic_set_adjoint_tiled(grid.h, tiled)
        P.pic_adjoint_step(grid.h, gE, gB, gx, gw)
        torch.cuda.synchronize()
        got[tiled] = [[t.cpu().numpy() for t in v] for v in (gE, gB, gx, gw)]
    O.step_adj(g, E, B, sp, lamE, lamB, lx, lw)
    want = (lamE, lamB, [np.concatenate([v[a] for v in lx]) for a in range(3)],
            [np.concatenate([v[a] for v in lw]) for a in range(3)])
    tol = 1e-11
    for tiled in (True, False):
        for name, gv, wv in zip(("lamE", "lamB", "lamx", "lamw"), got[tiled], want):
            for a in range(3):
                if name == "lamx" and a >= wl.dims:
                    continue
                close(gv[a], wv[a], tol, f"{name}[{a}] tiled={tiled}")
    grid.close()


N_CELLS, PPC, STEPS, AMP, WIN = 32, 16, 20, 0.05, ((12, 20), (12, 20))


def _run(P, torch, precision):
    from paper_1101_0809_gb300.adjoint import DifferentiableRun
    wl = W.c4_perturbed2d(n=N_CELLS, ppc=PPC, amplitude=AMP, steps=STEPS)
    desc = P.make_desc(2, wl.n, wl.d, wl.dt, wl.c, precision, tile=(16, 16, 1), rho_bg=wl.rho_bg)
    sp = wl.species[0]
    return DifferentiableRun(desc, sp.q, sp.m, sp.weight, STEPS, WIN, checkpoint_every=5)


def _xu():
    wl = W.c4_perturbed2d(n=N_CELLS, ppc=PPC, amplitude=0.0, steps=STEPS)
    return wl.species[0].x.copy(), wl.species[0].w.copy()


def _gpu_grad_A(P, torch, precision):
    from paper_1101_0809_gb300.adjoint import WindowEnergyLoss
    run = _run(P, torch, precision)
    xu, w0 = _xu()
    k = 2 * math.pi * 2 / N_CELLS
    A = torch.tensor(AMP, dtype=torch.float64, requires_grad=True)
    xu_t = torch.from_numpy(xu)
    x0 = xu_t.clone()
    x0[0] = torch.remainder(xu_t[0] - (A / k) * torch.sin(k * xu_t[0]), float(N_CELLS))
    L = WindowEnergyLoss.apply(x0, torch.from_numpy(w0), run)
    L.backward()
    return float(L), float(A.grad), run


def _oracle_grad_A():
    import importlib.util
    import sys
    here = os.path.dirname(os.path.abspath(__file__))
    spec = importlib.util.spec_from_file_location("adjpins", os.path.join(here, "test_oracle_adjoint.py"))
    m = importlib.util.module_from_spec(spec)
    sys.modules["adjpins"] = m
    spec.loader.exec_module(m)
    wl, g = m.setup(AMP)
    wl_u, _ = m.setup(0.0)
    k = 2 * math.pi * 2 / N_CELLS
    dxdA = np.zeros_like(wl_u.species[0].x)
    dxdA[0] = -np.sin(k * wl_u.species[0].x[0]) / k
    L, lx, lw = m.adjoint(wl, g, wl.species[0].x.copy(), wl.species[0].w.copy())
    return L, float((lx * dxdA).sum())


def test_fp64_gradient_matches_oracle_adjoint_and_central_fd(env):
    P, torch = env
    L, dLdA, run = _gpu_grad_A(P, torch, P.PIC_FP64)
    Lo, go = _oracle_grad_A()
    assert L == pytest.approx(Lo, rel=1e-10)
    assert dLdA == pytest.approx(go, rel=1e-9)
    # central differences of the GPU forward run itself
    xu, w0 = _xu()
    k = 2 * math.pi * 2 / N_CELLS
    h = 1e-7 * AMP

    def loss(A):
        x0 = xu.copy()
        x0[0] = np.mod(xu[0] - (A / k) * np.sin(k * xu[0]), float(N_CELLS))
        return run.forward(torch.from_numpy(x0), torch.from_numpy(w0))

    fd = (loss(AMP + h) - loss(AMP - h)) / (2 * h)
    assert dLdA == pytest.approx(fd, rel=1e-6)
    run.grid.close()


def test_fp32_gradient_against_fp64(env):
    P, torch = env
    L32, g32, r32 = _gpu_grad_A(P, torch, P.PIC_FP32)
    L64, g64, r64 = _gpu_grad_A(P, torch, P.PIC_FP64)
    assert L32 == pytest.approx(L64, rel=1e-3)
    assert g32 == pytest.approx(g64, rel=1e-2)
    r32.grid.close()
    r64.grid.close()


def test_state_snapshot_restarts_the_same_run(env):
    P, torch = env
    wl = W.c0_small2d(steps=6)
    desc = P.make_desc(2, wl.n, wl.d, wl.dt, wl.c, P.PIC_FP64, tile=wl.tile, rho_bg=wl.rho_bg)
    grid = P.Grid(desc)
    sp = wl.species[0]
    grid.load(0, sp.q, sp.m, sp.weight, sp.x, sp.w)
    P.pic_step(grid.h, 2)
    blob = np.empty(P.pic_state_bytes(grid.h), dtype=np.uint8)
    P.pic_state_save(grid.h, blob)
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "state.bin")
        blob.tofile(path)
        P.pic_step(grid.h, 4)
        E1, B1, J1 = grid.get_fields()
        _, _, w1, id1 = grid.particles(0)
        back = np.fromfile(path, dtype=np.uint8)
    P.pic_state_restore(grid.h, back)
    P.pic_step(grid.h, 4)
    E2, B2, J2 = grid.get_fields()
    _, _, w2, id2 = grid.particles(0)
    for a in range(3):
        close(E2[a], E1[a], 1e-12, f"E[{a}]")
        close(B2[a], B1[a], 1e-12, f"B[{a}]")
        close(w2[a][np.argsort(id2)], w1[a][np.argsort(id1)], 1e-12, f"w[{a}]")
    bad = back.copy()
    bad[0] = ord("X")
    with pytest.raises(P.PicError) as e:
        P.pic_state_restore(grid.h, bad)
    assert e.value.code == P.PIC_ERR_INVALID_ARG
    grid.close()


def test_async_restore_on_two_streams_matches_the_waiting_restore(env):
    """pic_state_restore_async from a pinned host snapshot, two FP32 3D grids on
    two streams taking steps in turn (each upload under the other grid's
    kernels), and from a device snapshot: every step gives the state and
    diagnostics of pic_state_restore + pic_step on one grid."""
    P, torch = env
    wl = W.thermal_plasma("3D", 3, (24, 16, 20), 3, 0.1, 2, W.SEED_BASE + 51, ions=1836.0, tile=(8, 4, 4),
                          dt_courant=0.45)

    def grid_on(stream):
        desc = P.make_desc(3, wl.n, wl.d, wl.dt, wl.c, P.PIC_FP32, tile=wl.tile, rho_bg=wl.rho_bg,
                           stream=stream.cuda_stream)
        g = P.Grid(desc)
        for s, sp in enumerate(wl.species):
            g.load(s, sp.q, sp.m, sp.weight, sp.x, sp.w)
        return g

    s0, s1 = torch.cuda.Stream(), torch.cuda.Stream()
    ga, gb = grid_on(s0), grid_on(s1)
    P.pic_step(ga.h, 3)
    host = torch.empty(P.pic_state_bytes(ga.h), dtype=torch.uint8).pin_memory()
    P.pic_state_save(ga.h, host)
    P.pic_state_restore(ga.h, host)
    P.pic_step(ga.h, 1)
    want_d = P.pic_diagnostics(ga.h)
    E0, B0, J0 = ga.get_fields()
    parts0 = [ga.particles(s) for s in range(len(wl.species))]

    def check(g, d):
        # the particle state is bit-exact; J (global float atomics at the tile
        # borders) and E after it may differ in the last bit
        assert d["total"] == pytest.approx(want_d["total"], rel=1e-9)
        E, B, J = g.get_fields()
        for a in range(3):
            close(E[a], E0[a], 1e-6, f"E[{a}]")
            close(B[a], B0[a], 1e-6, f"B[{a}]")
            close(J[a], J0[a], 1e-6, f"J[{a}]")
        for s in range(len(wl.species)):
            cell, off, w, ident = g.particles(s)
            assert np.array_equal(ident, parts0[s][3]) and np.array_equal(cell, parts0[s][0])
            for a in range(3):
                assert np.array_equal(off[a], parts0[s][1][a]) and np.array_equal(w[a], parts0[s][2][a])

    pair = (ga, gb)
    P.pic_state_restore_async(ga.h, host)
    P.pic_step(ga.h, 1)
    for k in range(4):
        if k + 1 < 4:
            P.pic_state_restore_async(pair[(k + 1) % 2].h, host)
            P.pic_step(pair[(k + 1) % 2].h, 1)
        d = P.pic_diagnostics(pair[k % 2].h)
        assert d["total"] == pytest.approx(want_d["total"], rel=1e-9)
    P.pic_sync(ga.h)
    P.pic_sync(gb.h)
    check(gb, P.pic_diagnostics(gb.h))

    dev = host.to("cuda")
    P.pic_step(ga.h, 2)
    P.pic_state_restore_async(ga.h, dev)
    P.pic_step(ga.h, 1)
    check(ga, P.pic_diagnostics(ga.h))
    bad = host.clone()
    bad[0] = ord("X")
    with pytest.raises(P.PicError) as e:
        P.pic_state_restore_async(gb.h, bad)
    assert e.value.code == P.PIC_ERR_INVALID_ARG
    ga.close()
    gb.close()


def test_batched_segment_calls_match_step_by_step(env):
    """pic_step_saving + pic_adjoint_steps (one host synchronization per
    segment) against pic_state_save / pic_step / pic_state_restore /
    pic_adjoint_step one step at a time, on the same FP64 run with a sort inside
    the segment; and a corrupt snapshot anywhere in the list is refused before
    anything is restored."""
    P, torch = env
    wl = W.c4_perturbed2d(n=32, ppc=8, steps=7)
    desc = P.make_desc(2, wl.n, wl.d, wl.dt, wl.c, P.PIC_FP64, tile=(8, 8, 1), sort_interval=3, rho_bg=wl.rho_bg)
    nbytes = None
    out = []
    for batched in (True, False):
        grid = P.Grid(desc)
        sp = wl.species[0]
        grid.load(0, sp.q, sp.m, sp.weight, sp.x, sp.w)
        P.pic_step(grid.h, 2)
        nbytes = P.pic_state_bytes(grid.h)
        states = [torch.empty(nbytes, dtype=torch.uint8, device="cuda") for _ in range(wl.steps)]
        torch.cuda.synchronize()
        if batched:
            P.pic_step_saving(grid.h, states)
        else:
            for st in states:
                P.pic_state_save(grid.h, st)
                P.pic_step(grid.h, 1)
        P.pic_sync(grid.h)
        E1, B1, _ = grid.get_fields()
        rng = np.random.default_rng(79)
        n = sp.x.shape[1]
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        lam = ([dev(rng.normal(size=grid.shape)) for _ in range(3)], [dev(rng.normal(size=grid.shape)) for _ in range(3)],
               [dev(rng.normal(size=n)) for _ in range(3)], [dev(rng.normal(size=n)) for _ in range(3)])
        torch.cuda.synchronize()
        if batched:
            P.pic_adjoint_steps(grid.h, states, *lam)
        else:
            for st in reversed(states):
                P.pic_state_restore(grid.h, st)
                P.pic_adjoint_step(grid.h, *lam)
        P.pic_sync(grid.h)
        torch.cuda.synchronize()
        out.append((E1, B1, [[t.cpu().numpy() for t in v] for v in lam], grid.particles(0)))
        if batched:
            # a corrupt header in the middle of the list: refused, nothing restored
            bad = [s.clone() for s in states]
            bad[3][0] = ord("X")
            before = grid.particles(0)
            with pytest.raises(P.PicError) as e:
                P.pic_adjoint_steps(grid.h, bad, *lam)
            assert e.value.code == P.PIC_ERR_INVALID_ARG
            after = grid.particles(0)
            for a, b in zip(before, after):
                np.testing.assert_array_equal(np.asarray(a), np.asarray(b))
        grid.close()
    (Ea, Ba, la, pa), (Eb, Bb, lb, pb) = out
    for a in range(3):
        close(Ea[a], Eb[a], 1e-13, f"E[{a}] after the segment")
        close(Ba[a], Bb[a], 1e-13, f"B[{a}] after the segment")
    for name, va, vb in zip(("lamE", "lamB", "lamx", "lamw"), la, lb):
        for a in range(3):
            if name == "lamx" and a == 2:
                continue
            close(va[a], vb[a], 1e-11, f"{name}[{a}]")
    np.testing.assert_array_equal(pa[0], pb[0])     # the grid holds the first snapshot's state
