"""Energy-conservation runs of the paper's Sec. 5 tests through the C ABI.

A run loads a workload (the X1 thermal plasma or the X4 two-stream setup of
workloads.py), optionally a uniform initial B_x, steps it with a chosen
interpolation (order2 = 3: the alternating order l_a = 1 1/2; 4: the
uniform-order l = 2 scheme of Eq. wrong1; 5: l_a = 2 1/2), and records the
energy integral of Sec. 4.1 (pic_diagnostics: kinetic energy without rest
mass, E and B field energy at time n, and the half-step term) every `every`
steps.  The field energy of the initial uniform B_x is left out, as in the
paper's two-stream test.  Everything numerical runs in libpic.
"""
import math
import time

from . import pic as P


def energy_run(wl, order2, precision, every=10, bx=None, stream=None):
    """Returns the relative energy defect |W(t) - W(0)| / W(0) (largest and last
    over the sampled steps) and the stepping rate in particle-steps/s
    (diagnostics excluded)."""
    import numpy as np
    desc = P.make_desc(wl.dims, wl.n, wl.d, wl.dt, wl.c, precision, tile=wl.tile, halo=1,
                       sort_interval=wl.sort_interval, rho_bg=wl.rho_bg, stream=stream, order2=order2)
    g = P.Grid(desc)
    eb0 = 0.0
    if bx is not None:
        dtype = np.float64 if precision == P.PIC_FP64 else np.float32
        zero = [np.zeros(g.shape, dtype) for _ in range(3)]
        B = [np.full(g.shape, bx, dtype), np.zeros(g.shape, dtype), np.zeros(g.shape, dtype)]
        g.set_fields(zero, B)
        eb0 = wl.volume / (8.0 * math.pi) * bx * bx * wl.n_cells
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
        series.append((done, last))
    g.close()
    return {"order2": order2, "max_rel_defect": worst, "final_rel_defect": last, "steps": wl.steps,
            "every": every, "particle_steps_per_s": wl.n_particles * wl.steps / t_step, "series": series}
