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


def oracle_grid(wl, order2=3):
    return O.Grid(wl.dims, wl.n, wl.d, wl.dt, wl.c, order2)


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


FACE_BAND = 2.0 ** -20    # FP32 cells may differ from the oracle's only this close to a face
OFFSET_ULPS = 4 * 2.0 ** -24   # a few ulps of an FP32 offset in [0, 1), in cells


def check_fp32_positions(wl, cell, x, x_ref, x_prev, tol, what):
    """The FP32 rules for positions and cells, per particle and axis.

    cell: the GPU's linear cell indices; x: the GPU's positions (cell + offset);
    x_ref: the oracle's positions after the step; x_prev: the positions both
    sides started the step from.  Each position is judged in cells:
    |x - x_ref| <= a few FP32 ulps of the offset + tol * |displacement of the
    step|, so that a relative error of the FP32 displacement above tol fails.
    The cell index of every axis equals the oracle's floor(x_ref), except that
    it may differ by one where the oracle's offset lies within 2^-20 of 0 or 1
    (the two sides round the move differently there); those cases are counted
    and the count is returned."""
    cell = np.asarray(cell, dtype=np.int64)
    ci = [cell % wl.n[0], (cell // wl.n[0]) % wl.n[1], cell // (wl.n[0] * wl.n[1])]
    near_face = 0
    for a in range(wl.dims):
        d = periodic_diff(x[a], x_ref[a], wl.n[a])
        disp = periodic_diff(x_ref[a], np.asarray(x_prev[a], dtype=np.float64), wl.n[a])
        bound = OFFSET_ULPS + tol * np.abs(disp)
        bad = np.abs(d) > bound
        if bad.any():
            k = int(np.argmax(np.abs(d) - bound))
            raise AssertionError(f"{what} x[{a}]: {int(bad.sum())}/{d.size} positions off by more than "
                                 f"{OFFSET_ULPS:.1e} cells + {tol} x displacement; worst at {k}: "
                                 f"error {d[k]:.3e} cells, displacement {disp[k]:.3e}")
        want = np.floor(x_ref[a]).astype(np.int64) % wl.n[a]
        diff = periodic_diff(ci[a], want, wl.n[a]).astype(np.int64)
        frac = x_ref[a] - np.floor(x_ref[a])
        at_face = (frac < FACE_BAND) | (frac > 1.0 - FACE_BAND)
        wrong = (diff != 0) & ~((np.abs(diff) == 1) & at_face)
        assert not wrong.any(), (f"{what} cell index axis {a}: {int(wrong.sum())} differ from the oracle's "
                                 f"away from a face (first at {int(np.flatnonzero(wrong)[0])})")
        near_face += int(np.count_nonzero(diff != 0))
    return near_face


def compare_particles(wl, sp_index, grid, osp, tol, x_prev=None):
    """Compare the GPU's particles of one species with the oracle's (load order).

    FP64 path (x_prev None): positions to tol relative to the position scale,
    cells bit-exact, momenta element by element.  FP32 form (x_prev = the
    positions both sides started the step from): positions and cells by
    check_fp32_positions, momenta element by element; returns the number of
    cell indices that differ next to a face."""
    cell, off, w, ident = grid.particles(sp_index)
    order = np.argsort(ident)
    x = positions_from_gpu(wl, cell[order], [o[order] for o in off])
    ref = osp[sp_index]
    near_face = 0
    if x_prev is None:
        for a in range(wl.dims):
            d = periodic_diff(x[a], ref.x[a], wl.n[a])
            s = max(math.sqrt(float(np.mean(ref.x[a] ** 2))), 1.0)
            worst = np.abs(d).max() / s if d.size else 0.0
            assert worst <= tol, f"species {sp_index} x[{a}] rel error {worst:.3e} > {tol}"
        ci = [cell[order] % wl.n[0], (cell[order] // wl.n[0]) % wl.n[1], cell[order] // (wl.n[0] * wl.n[1])]
        for a in range(wl.dims):
            np.testing.assert_array_equal(ci[a], np.floor(ref.x[a]).astype(np.int64) % wl.n[a],
                                          err_msg=f"cell index axis {a}")
    else:
        near_face = check_fp32_positions(wl, cell[order], x, ref.x, x_prev, tol, f"species {sp_index}")
    for a in range(3):
        close(w[a][order], ref.w[a], tol, f"species {sp_index} w[{a}]")
    return near_face


def make_grid(P, wl, precision, stream=None, tile=None, halo=-1, sort_interval=None, ppb=0, sort_order=0,
              order2=3):
    desc = P.make_desc(wl.dims, wl.n, wl.d, wl.dt, wl.c, precision,
                       tile=tile if tile is not None else wl.tile, halo=halo,
                       sort_interval=sort_interval if sort_interval is not None else wl.sort_interval,
                       particles_per_block=ppb, rho_bg=wl.rho_bg, stream=stream, sort_order=sort_order,
                       order2=order2)
    grid = P.Grid(desc)
    for s, sp in enumerate(wl.species):
        grid.load(s, sp.q, sp.m, sp.weight, sp.x, sp.w)
    return grid


def tile_sort_perm(wl, cells, tile, halo=1, banked=True, pitch=None, up=None, cell_lanes=False):
    """The tile sort's permutation written out from its definition (integer work,
    compared bit-exactly): sort by tile key; with ``banked``, inside a tile by
    (r, b) where b is the shared-memory bank of the cell's base address in the
    tile's current stage, base = (i-ox+h+2) + P0*((j-oy+h+2) + P1*(k-oz+h+2)) with
    the grid's tile pitches (pic_tile_layout), and r the particle's rank among
    the tile's particles of bank b in input order.  ``up`` (l_a = 2 1/2): per
    axis the 0/1 flags offset >= 1/2, added to i, j, k in the base (the base
    index of the interpolation), not in the tile key.  With ``cell_lanes``: the
    tile's cells c = (i-ox) + Tx ((j-oy) + Ty (k-oz)) get lanes L(c) by
    descending particle count, ties by c; the particle of rank r among its
    cell's particles (input order) takes slot P(r) + L(c) of the tile, with
    P(r) = sum over the tile's Tx Ty Tz cells of min(count, r).  Returns
    perm[o] = input index at slot o."""
    nx, ny = wl.n[0], wl.n[1]
    cells = np.asarray(cells, dtype=np.int64)
    i, j, k = cells % nx, (cells // nx) % ny, cells // (nx * ny)
    T = tile
    ntx, nty = -(-nx // T[0]), -(-ny // T[1])
    ti, tj, tk = i // T[0], j // T[1], (k // T[2] if wl.dims == 3 else 0 * k)
    key = (tk * nty + tj) * ntx + ti
    if cell_lanes:
        ncell = T[0] * T[1] * (T[2] if wl.dims == 3 else 1)
        c = (i - ti * T[0]) + T[0] * ((j - tj * T[1]) + T[1] * ((k - tk * T[2]) if wl.dims == 3 else 0))
        order = np.argsort(key, kind="stable")
        out = np.empty(cells.size, dtype=np.int64)
        keys_sorted = key[order]
        starts = np.r_[0, np.flatnonzero(np.diff(keys_sorted)) + 1]
        ends = np.r_[starts[1:], keys_sorted.size]
        for s0, e0 in zip(starts, ends):
            members = order[s0:e0]                     # this tile's particles, input order
            cc = c[members]
            count = np.bincount(cc, minlength=ncell)
            lanes = np.lexsort((np.arange(ncell), -count))   # lane -> cell
            lane_of = np.empty(ncell, dtype=np.int64)
            lane_of[lanes] = np.arange(ncell)
            rank = np.empty(cc.size, dtype=np.int64)
            seen = np.zeros(ncell, dtype=np.int64)
            for q, cq in enumerate(cc):
                rank[q] = seen[cq]
                seen[cq] += 1
            P = np.array([np.minimum(count, r).sum() for r in range(int(count.max()) + 1)])
            out[s0 + P[rank] + lane_of[cc]] = members
        return out
    if not banked:
        return np.argsort(key, kind="stable")
    u = [np.zeros_like(i)] * 3 if up is None else [np.asarray(a, dtype=np.int64) for a in up]
    je0, je1 = pitch if pitch is not None else (T[0] + 2 * halo + 4, T[1] + 2 * halo + 4)
    base = (i + u[0] - ti * T[0] + halo + 2) + je0 * (j + u[1] - tj * T[1] + halo + 2)
    if wl.dims == 3:
        base = base + je0 * je1 * (k + u[2] - tk * T[2] + halo + 2)
    b = base % 32
    kb = key * 32 + b
    idx = np.argsort(kb, kind="stable")          # groups (tile, bank), input order inside
    skb = kb[idx]
    start = np.r_[0, np.flatnonzero(np.diff(skb)) + 1]
    grp = np.repeat(start, np.diff(np.r_[start, skb.size]))
    r = np.empty(cells.size, dtype=np.int64)
    r[idx] = np.arange(skb.size) - grp
    return np.lexsort((b, r, key))
