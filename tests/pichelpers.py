"""Shared helpers of the GPU parity tests: run a workload through libpic and
through the FP64 oracle from the same seeded inputs, and compare them with the
tolerances of the FP64 path (1e-12) and the FP32 form (2e-5, per step).

Tolerance reading: |a - b| <= tol * max(|b|, s) element by element, where s is
the root-mean-square of the oracle array (so that values that cancel to near
zero are judged on the array's scale).
"""
import math

import numpy as np

import oracle as O

FP64_TOL = 1e-12
FP32_TOL = 2e-5


def close(a, b, tol, what=""):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    s = math.sqrt(float(np.mean(b * b))) if b.size else 0.0
    scale = np.maximum(np.abs(b), s)
    err = np.abs(a - b)
    bad = err > tol * scale + 1e-300
    if bad.any():
        k = int(np.argmax(err / (scale + 1e-300)))
        raise AssertionError(f"{what}: {int(bad.sum())}/{b.size} elements off; worst at {k}: "
                             f"got {a.ravel()[k]!r}, want {b.ravel()[k]!r}, rel {err.ravel()[k] / (scale.ravel()[k] + 1e-300):.3e}")


def fp64_field_tol(wl, species, tol=FP64_TOL):
    """FP64 tolerance for J and E.  The oracle keeps absolute positions, so a
    displacement delta carries its rounding ulp(N); currents are proportional to
    displacements.  The bound is therefore max(tol, 4 ulp(N_max) / delta_rms),
    which exceeds 1e-12 only for very slow plasmas (v_th ~ 0.01c)."""
    n_max = float(max(wl.n[:wl.dims]))
    d2, cnt = 0.0, 0
    for sp in species:
        gam = np.sqrt((sp.w ** 2).sum(axis=0) + wl.c ** 2)
        for a in range(wl.dims):
            d = sp.w[a] / gam * (wl.c * wl.dt / wl.d[a])
            d2 += float((d * d).sum())
            cnt += d.size
    delta = math.sqrt(d2 / max(cnt, 1))
    return max(tol, 4 * float(np.spacing(n_max)) / max(delta, 1e-300))


def oracle_grid(wl):
    return O.Grid(wl.dims, wl.n, wl.d, wl.dt, wl.c)


def oracle_species(wl):
    return [O.Species(s.q, s.m, s.weight, s.x.copy(), s.w.copy()) for s in wl.species]


def positions_from_gpu(wl, cell, off):
    """Absolute positions (3, n) from (cell, offset), FP64."""
    nx, ny = wl.n[0], wl.n[1]
    i = cell % nx
    r = cell // nx
    j = r % ny
    k = r // ny
    x = np.zeros((3, cell.shape[0]))
    x[0] = i + off[0].astype(np.float64)
    x[1] = j + off[1].astype(np.float64)
    if wl.dims == 3:
        x[2] = k + off[2].astype(np.float64)
    return x


def periodic_diff(a, b, n):
    d = a - b
    return d - n * np.round(d / n)


def compare_particles(wl, sp_index, grid, osp, tol, check_cells=True):
    cell, off, w, ident = grid.particles(sp_index)
    order = np.argsort(ident)
    x = positions_from_gpu(wl, cell[order], [o[order] for o in off])
    ref = osp[sp_index]
    for a in range(wl.dims):
        d = periodic_diff(x[a], ref.x[a], wl.n[a])
        s = max(math.sqrt(float(np.mean(ref.x[a] ** 2))), 1.0)
        worst = np.abs(d).max() / s if d.size else 0.0
        assert worst <= tol, f"species {sp_index} x[{a}] rel error {worst:.3e} > {tol}"
    if check_cells:
        ci = [cell[order] % wl.n[0], (cell[order] // wl.n[0]) % wl.n[1], cell[order] // (wl.n[0] * wl.n[1])]
        for a in range(wl.dims):
            np.testing.assert_array_equal(ci[a], np.floor(ref.x[a]).astype(np.int64) % wl.n[a],
                                          err_msg=f"cell index axis {a}")
    for a in range(3):
        close(w[a][order], ref.w[a], tol, f"species {sp_index} w[{a}]")


def make_grid(P, wl, precision, stream=None, tile=None, halo=-1, sort_interval=None, ppb=0):
    desc = P.make_desc(wl.dims, wl.n, wl.d, wl.dt, wl.c, precision,
                       tile=tile if tile is not None else wl.tile, halo=halo,
                       sort_interval=sort_interval if sort_interval is not None else wl.sort_interval,
                       particles_per_block=ppb, rho_bg=wl.rho_bg, stream=stream)
    grid = P.Grid(desc)
    for s, sp in enumerate(wl.species):
        grid.load(s, sp.q, sp.m, sp.weight, sp.x, sp.w)
    return grid
