"""Energy-conservation runs of the paper's Sec. 5 tests through the C ABI.

A run loads a workload (the X1 thermal plasma, the X4 two-stream, X5 Langmuir
or X6 gyration setups of workloads.py), optionally a uniform initial B, steps
it with a chosen
interpolation (order2 = 3: the alternating order l_a = 1 1/2; 4: the
uniform-order l = 2 scheme of Eq. wrong1; 5: l_a = 2 1/2), and records the
energy integral of Sec. 4.1 (pic_diagnostics: kinetic energy without rest
mass, E and B field energy at time n, and the half-step term) every `every`
steps.  The field energy of the initial uniform B is left out, as in the
paper's two-stream test.  Everything numerical runs in libpic.
"""
import math
import time

from . import pic as P


def energy_run(wl, order2, precision, every=10, bx=None, stream=None, b0=None):
    """Returns the relative energy defect |W(t) - W(0)| / W(0) (largest and last
    over the sampled steps), the sampled series of (step, defect, kinetic,
    field_E) and the stepping rate in particle-steps/s (diagnostics excluded).
    bx: a uniform initial B_x; b0: a uniform initial B vector (either)."""
    import numpy as np
    desc = P.make_desc(wl.dims, wl.n, wl.d, wl.dt, wl.c, precision, tile=wl.tile, halo=1,
                       sort_interval=wl.sort_interval, rho_bg=wl.rho_bg, stream=stream, order2=order2)
    g = P.Grid(desc)
    eb0 = 0.0
    if bx is not None:
        b0 = (bx, 0.0, 0.0)
    if b0 is not None:
        dtype = np.float64 if precision == P.PIC_FP64 else np.float32
        zero = [np.zeros(g.shape, dtype) for _ in range(3)]
        B = [np.full(g.shape, b0[a], dtype) for a in range(3)]
        g.set_fields(zero, B)
        eb0 = wl.volume / (8.0 * math.pi) * sum(b * b for b in b0) * wl.n_cells
    for s, sp in enumerate(wl.species):
        g.load(s, sp.q, sp.m, sp.weight, sp.x, sp.w)
    w0 = P.pic_diagnostics(g.h)["total"] - eb0
    worst, last, done, t_step = 0.0, 0.0, 0, 0.0
    series = []
    while done < wl.steps:
        k = min(every, wl.steps - done)
        P.pic_sync(g.h)
        t0 = time.perf_counter()
        P.pic_step(g.h, k)
        P.pic_sync(g.h)
        t_step += time.perf_counter() - t0
        done += k
        d = P.pic_diagnostics(g.h)
        last = abs(d["total"] - eb0 - w0) / w0
        worst = max(worst, last)
        series.append((done, last, d["kinetic"], d["field_E"]))
    g.close()
    return {"order2": order2, "max_rel_defect": worst, "final_rel_defect": last, "steps": wl.steps,
            "every": every, "particle_steps_per_s": wl.n_particles * wl.steps / t_step, "series": series}


def oscillation_period(steps, values):
    """Mean spacing (in steps) of the local maxima of a sampled series, each
    located by a parabola through the sample and its two neighbours."""
    peaks = []
    for i in range(1, len(values) - 1):
        a, b, c = values[i - 1], values[i], values[i + 1]
        if b > a and b >= c:
            den = a - 2 * b + c
            shift = 0.5 * (a - c) / den if den != 0 else 0.0
            peaks.append(steps[i] + shift * (steps[i + 1] - steps[i]))
    if len(peaks) < 2:
        return None
    return (peaks[-1] - peaks[0]) / (len(peaks) - 1)


def gyration_run(wl, order2, precision, bz, stream=None):
    """The X6 run: kinetic energy of the two particles at the start and at the
    end, and their distance from the gyration centre (the Larmor radius)
    averaged over the first and the last gyration."""
    import numpy as np
    desc = P.make_desc(wl.dims, wl.n, wl.d, wl.dt, wl.c, precision, tile=wl.tile, halo=1,
                       sort_interval=wl.sort_interval, rho_bg=wl.rho_bg, stream=stream, order2=order2)
    g = P.Grid(desc)
    dtype = np.float64 if precision == P.PIC_FP64 else np.float32
    zero = [np.zeros(g.shape, dtype) for _ in range(3)]
    g.set_fields(zero, [np.zeros(g.shape, dtype), np.zeros(g.shape, dtype), np.full(g.shape, bz, dtype)])
    for s, sp in enumerate(wl.species):
        g.load(s, sp.q, sp.m, sp.weight, sp.x, sp.w)
    eb0 = wl.volume / (8.0 * math.pi) * bz * bz * wl.n_cells
    d0 = P.pic_diagnostics(g.h)
    k0, w0 = d0["kinetic"], d0["total"] - eb0
    # steps per gyration: omega = |q| B / (gamma m c), with |q| = m = 1 here
    sp = wl.species[0]
    gam = math.sqrt(1.0 + float((sp.w[:, 0] ** 2).sum()) / (wl.c * wl.c))
    period = max(2, int(round(2 * math.pi * gam * wl.c / bz / wl.dt)))
    track = []
    for n in range(wl.steps):
        P.pic_step(g.h, 1)
        if n < period or n >= wl.steps - period:
            cell, off, w, ident = g.particles(0)
            nx, ny = wl.n[0], wl.n[1]
            x = cell[0] % nx + float(off[0][0])
            y = (cell[0] // nx) % ny + float(off[1][0])
            track.append((n, x, y))
    d = P.pic_diagnostics(g.h)
    g.close()
    first = np.array([(x, y) for n, x, y in track if n < period])
    last = np.array([(x, y) for n, x, y in track if n >= wl.steps - period])
    r0 = float(np.mean(np.hypot(*(first - first.mean(axis=0)).T)))
    r1 = float(np.mean(np.hypot(*(last - last.mean(axis=0)).T)))
    return {"order2": order2, "kinetic_start": k0, "kinetic_end": d["kinetic"],
            "kinetic_ratio": d["kinetic"] / k0, "larmor_radius_first": r0, "larmor_radius_last": r1,
            "total_rel_defect": abs(d["total"] - eb0 - w0) / w0, "steps": wl.steps, "steps_per_gyration": period}
