"""Throughput of the charge-conserving PIC step on one GB300 (or N independent
replicas, one per GPU).

Workload: 3D3V periodic 128^3 plasma, electrons and ions (mass ratio 1836), 32
macro-particles per cell each (134,217,728 particles), v_th,e = 0.1c,
dt = 0.45 dx/c, synthetic seeded inputs.  A "step" is one full time step of the
paper's Appendix on every particle: B half step, gather + push + move +
virtual-path deposit, B half step, E full step, and the tile sort every 10
steps.  The headline value is the FP32 form; the FP64 path is timed beside it.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle
on bounded samples of the same workload instead.
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-steps/s and % HBM roofline (fwd, fwd+adjoint) FP32 vs FP64 at 1 GB300"
UNIT = "particle-steps/s"
WORKLOAD = ("3D3V 128^3 periodic, e- and ions (m_i/m_e = 1836), 32+32 per cell, v_th,e = 0.1c, "
            "dt = 0.45 dx/c, FP32 form")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=48, help="timed steps (48: twelve whole sort intervals of 4 steps)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=128, help="cells per axis")
    ap.add_argument("--ppc", type=int, default=32, help="macro-particles per cell per species")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--fp64-steps", type=int, default=5)
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--adj-steps", type=int, default=200)
    ap.add_argument("--batch-runs", type=int, default=256)
    ap.add_argument("--no-laser", action="store_true")
    ap.add_argument("--no-order5", action="store_true", help="skip the l_a = 2 1/2 leg")
    ap.add_argument("--no-energy", action="store_true", help="skip the Sec. 5 energy (X1) leg")
    ap.add_argument("--energy-x4", action="store_true", help="add the 8000-step two-stream run to the energy leg")
    ap.add_argument("--energy-x5-steps", type=int, default=4000, help="steps of the Langmuir run (X5)")
    ap.add_argument("--no-vecpot", action="store_true", help="skip the vector-potential (generalized momentum) leg")
    ap.add_argument("--laser-warmup", type=int, default=480)
    ap.add_argument("--no-gauss", action="store_true", help="skip the 200-step full-size Gauss residual")
    ap.add_argument("--cell-lanes", action="store_true",
                    help="run the main grids in the cell-lane particle order (PIC_SORT_CELL_LANES)")
    ap.add_argument("--sort-interval", type=int, default=0, help="override the main workload's sort interval")
    return ap.parse_args()


from paper_1101_0809_gb300.replicas import max_over_ranks  # noqa: E402  (host arithmetic only)


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


# ----------------------------------------------------------------------------- oracle timing
def time_oracle(n, ppc, target_s=15.0, steps=None, fraction=None):
    """Time the FP64 CPU oracle (single thread) on a random subsample of the
    workload's particles on the full grid; returns (particle-steps/s, sample text)."""
    import oracle as O
    from paper_1101_0809_gb300 import workloads as W

    def run(frac, nsteps):
        wl = W.c1_thermal3d(n=n, ppc=ppc, steps=nsteps, fraction=frac)
        g = O.Grid(wl.dims, wl.n, wl.d, wl.dt, wl.c)
        sp = [O.Species(s.q, s.m, s.weight, s.x, s.w) for s in wl.species]
        E, B, J = g.zeros(), g.zeros(), g.zeros()
        t0 = time.perf_counter()
        for _ in range(nsteps):
            O.step(g, E, B, J, sp)
        dt = time.perf_counter() - t0
        return sum(s.x.shape[1] for s in sp), dt

    if fraction is None:
        probe_frac = 1.0 / 1024
        np_, dt = run(probe_frac, 1)
        per = dt / max(np_, 1)
        fraction = min(1.0, (target_s / 2) / per / (2 * ppc * n ** 3))
        steps = 2
    npart, dt = run(fraction, steps)
    rate = npart * steps / dt
    sample = (f"{npart} of {2 * ppc * n ** 3} particles (random subsample, same weights) on the full "
              f"{n}^3 grid, {steps} full steps, {dt:.1f} s single-threaded")
    return rate, sample, fraction, steps


def time_oracle_small():
    """The oracle single-threaded on the two 2D configurations in full: the 32x32
    correctness run (8,192 electrons, 50 steps) and two steps of the 256x256
    differentiable run (1,048,576 electrons)."""
    import oracle as O
    from paper_1101_0809_gb300 import workloads as W
    out = {}
    for name, wl, nsteps in (("2D 32x32 8 e-/cell, 50 steps", W.c0_small2d(steps=50), 50),
                             ("2D 256x256 16 e-/cell perturbed, 2 steps", W.c4_perturbed2d(steps=2), 2)):
        g = O.Grid(wl.dims, wl.n, wl.d, wl.dt, wl.c)
        sp = [O.Species(s.q, s.m, s.weight, s.x, s.w) for s in wl.species]
        E, B, J = g.zeros(), g.zeros(), g.zeros()
        t0 = time.perf_counter()
        for _ in range(nsteps):
            O.step(g, E, B, J, sp)
        dt = time.perf_counter() - t0
        out[name] = {"value": wl.n_particles * nsteps / dt, "unit": UNIT, "cores": 1, "seconds": dt}
    return out


def _oracle_proc(n, ppc, steps, fraction, barrier, q):
    """One of the concurrent oracle processes of time_oracle_cores."""
    sys.path.insert(0, ROOT)
    import oracle as O
    from paper_1101_0809_gb300 import workloads as W
    wl = W.c1_thermal3d(n=n, ppc=ppc, steps=steps, fraction=fraction)
    g = O.Grid(wl.dims, wl.n, wl.d, wl.dt, wl.c)
    sp = [O.Species(s.q, s.m, s.weight, s.x, s.w) for s in wl.species]
    E, B, J = g.zeros(), g.zeros(), g.zeros()
    barrier.wait()
    t0 = time.perf_counter()
    for _ in range(steps):
        O.step(g, E, B, J, sp)
    q.put((sum(s.x.shape[1] for s in sp), time.perf_counter() - t0))


def time_oracle_cores(n, ppc, steps, fraction):
    """The oracle as it stands, one single-threaded process per host core, all
    started together on the same sample (spawned, before any GPU work); the
    rate is all processes' particle-steps over the slowest one's time."""
    import multiprocessing as mp
    procs = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    ctx = mp.get_context("spawn")
    barrier, q = ctx.Barrier(procs), ctx.Queue()
    ps = [ctx.Process(target=_oracle_proc, args=(n, ppc, steps, fraction, barrier, q)) for _ in range(procs)]
    for p in ps:
        p.start()
    got = [q.get() for _ in ps]
    for p in ps:
        p.join()
    work = sum(k * steps for k, _ in got)
    slowest = max(t for _, t in got)
    sample = (f"{procs} concurrent processes, one per host core, each stepping the oracle single-threaded on "
              f"{got[0][0]} of {2 * ppc * n ** 3} particles (the same random subsample, same weights) on the full "
              f"{n}^3 grid for {steps} full steps; slowest {slowest:.1f} s")
    return work / slowest, sample, procs


def reference_arm(args):
    rank, _, world = dist_env()
    if rank != 0:
        return
    # bounded samples: every step of the K + W run is a small random subsample
    total_s = 0.0
    parts = 0
    frac = 1.0 / 512       # 262,144 particles: the particles, not the grid's field updates, dominate a step
    time_oracle(args.n, args.ppc, steps=max(args.warmup, 1), fraction=frac)      # warm-up steps
    rate1, sample1, _, _ = time_oracle(args.n, args.ppc, steps=args.steps, fraction=frac)
    rate, sample, cores = time_oracle_cores(args.n, args.ppc, args.steps, frac)
    npart = round(frac * 2 * args.ppc * args.n ** 3)
    out = {"impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * npart * cores / rate,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {"workload": WORKLOAD, "sample": sample},
           "cpu_baseline": {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                            "single_core": {"value": rate1, "sample": sample1}},
           "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def wait_first(self, timeout=5.0):
        """Block until nvidia-smi has printed its first sample (it takes a
        fraction of a second to start); the samples before the timed region
        begins are then left out."""
        t0 = time.time()
        while self.proc and not self.lines and time.time() - t0 < timeout:
            time.sleep(0.01)
        self.first = len(self.lines)

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.th.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        timed = self.lines[getattr(self, "first", 0):]
        for ln in timed or self.lines[-1:]:
            f = [v.strip() for v in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- our arm
def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("pic_device.cuh", "pic_particles.cuh", "pic_particles.cu", "pic_particles_fixed.cu"):
        with open(os.path.join(ROOT, "paper_1101_0809_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_per_particle(precision, key):
    """A per-particle figure (DRAM bytes, warp instructions) of the fused
    particle kernel from the committed ncu summary, if it was taken on the
    current kernel source."""
    path = os.path.join(ROOT, "profiles", f"k_particles_fused_3d_{precision}.md")
    if not os.path.exists(path):
        return None
    vals = {}
    for line in open(path):
        if ":" in line and line.startswith("- "):
            k, v = line[2:].split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    if vals.get("source_sha") != kernel_source_hash():
        return None
    try:
        return float(vals[key])
    except (KeyError, ValueError):
        return None


def ncu_traffic_per_particle(precision):
    return ncu_per_particle(precision, "dram_bytes_per_particle")


SORT_ORDER = 0   # PIC_SORT_AUTO; --cell-lanes selects PIC_SORT_CELL_LANES for the main grids


def build_grid(P, wl, precision, stream, sort_interval=None):
    desc = P.make_desc(wl.dims, wl.n, wl.d, wl.dt, wl.c, precision, tile=wl.tile, halo=1,
                       sort_interval=sort_interval or wl.sort_interval, particles_per_block=8192,
                       rho_bg=wl.rho_bg, stream=stream, sort_order=SORT_ORDER)
    grid = P.Grid(desc)
    for s, sp in enumerate(wl.species):
        grid.load(s, sp.q, sp.m, sp.weight, sp.x, sp.w)
    return grid


def timed_steps(P, torch, grid, steps, dist=None, sampler=None):
    st = torch.cuda.current_stream()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = P.pic_kernel_launches(grid.h)
    P.pic_profile(grid.h, True)
    if sampler:
        sampler.start()
        sampler.wait_first()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(steps):
        P.pic_step(grid.h, 1)
    e1.record(st)
    torch.cuda.synchronize()
    clocks = sampler.stop() if sampler else None
    ms = e0.elapsed_time(e1)
    prof = P.pic_profile_read(grid.h)
    P.pic_profile(grid.h, False)
    launches = P.pic_kernel_launches(grid.h) - l0
    if dist is not None:
        ms = max_over_ranks(dist, ms, "cuda")
        dist.barrier()
    return ms, prof, launches, clocks


def batched_arm(P, W, torch, args, dist, hbm_peak):
    """The batched ensemble: independent 2D3V periodic runs with N ~ U{32..256}
    per axis, 4-64 electrons per cell and v_th ~ U[0.01c, 0.3c], FP32, advanced
    together by one cooperative launch per step replayed from CUDA graphs, with
    tile, particles per block and sort interval picked by the autotuner: all
    36 candidates timed on every 8th run, the three fastest again on all runs."""
    from paper_1101_0809_gb300 import autotune as AT
    params = W.c3_ensemble_params(args.batch_runs)
    runs = [W.c3_run(p) for p in params]
    st = torch.cuda.Stream()
    stream = st.cuda_stream

    def build(sub, cand):
        descs = [P.make_desc(2, wl.n, wl.d, wl.dt, wl.c, P.PIC_FP32, tile=(cand["tile"], cand["tile"], 1), halo=1,
                             sort_interval=cand["K"], particles_per_block=cand["ppb"], rho_bg=wl.rho_bg,
                             stream=stream) for wl in sub]
        b = P.Batch(descs)
        P.pic_load_particles_runs(b.h, list(range(len(sub))), 0,
                                  [(wl.species[0].q, wl.species[0].m, wl.species[0].weight) for wl in sub],
                                  [list(wl.species[0].x) for wl in sub], [list(wl.species[0].w) for wl in sub])
        return b

    def timed(b, nsteps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        P.pic_step_graph(b.h, nsteps)
        e1.record(st)
        e1.synchronize()
        return e0.elapsed_time(e1)

    def time_on(sub, c):
        b = build(sub, c)
        try:
            span = 2 * c["K"]
            P.pic_step_graph(b.h, span + c["K"])
            return timed(b, 2 * span) / (2 * span)
        finally:
            b.close()

    def time_candidate(c):
        return time_on(runs[::8], c)

    def time_full(c):
        return time_on(runs, c)

    cands = [dict(tile=t, ppb=p, K=k) for t in (8, 16) for p in (2048, 4096, 8192) for k in (2, 3, 4, 5, 6, 8)]
    key = AT.workload_key("ensemble2d", [(r["n"], r["ppc"], round(r["vth"], 6)) for r in params[::8]])
    best, table, cached = AT.tune(key, torch.cuda.get_device_name(), cands, time_candidate, refine=time_full, top=3)
    b = build(runs, best)
    span = 2 * best["K"]
    P.pic_step_graph(b.h, span + best["K"])        # aligns the sort phase and captures the graph
    P.pic_sync(b.h)
    nsteps = max(span, (args.steps + span - 1) // span * span)
    if dist is not None:
        dist.barrier()
    l0 = P.pic_kernel_launches(b.h)
    ms = timed(b, nsteps)
    launches = P.pic_kernel_launches(b.h) - l0
    P.pic_sync(b.h)
    if dist is not None:
        ms = max_over_ranks(dist, ms, "cuda")
    npart = sum(wl.n_particles for wl in runs)
    ncell = sum(wl.n_cells for wl in runs)
    b.close()
    accuracy = batched_accuracy(P, runs[::8], best, build, 20)
    world = dist.get_world_size() if dist is not None else 1
    # the whole step's algorithmic bytes: the 2D FP32 particle state read and
    # written (24 B each way) and per cell E, B, J through the particle pass and
    # the three field passes (120 B); the sort's share is left out
    alg = npart * 48 + ncell * 120
    ach = alg / (ms / nsteps * 1e-3) / 1e9
    return {"workload": f"{len(runs)} independent 2D3V periodic runs, N ~ U{{32..256}}^2, 4-64 e-/cell, "
                        "v_th ~ U[0.01c, 0.3c], FP32, one cooperative launch per step, CUDA graphs",
            "value": world * npart * nsteps / (ms * 1e-3), "unit": UNIT, "steps": nsteps, "ms_per_step": ms / nsteps,
            "particles": npart, "cells": ncell, "autotuned": best, "autotune_cached": cached,
            "autotune_candidates": len(table), "gpu_launches": launches,
            "autotune_table": [[c, ms, why] for c, ms, why in table],
            "roofline": {"bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s", "frac": ach / hbm_peak,
                         "scope": "whole step (persistent kernel, sorts included in the time)",
                         "alg_bytes_per_step": alg},
            "accuracy_vs_fp64": accuracy}


def main_accuracy(P, wl, stream, g64, steps):
    """The FP32 form against the plain FP64 method on the main workload: a fresh
    FP32 grid takes the `steps` steps that g64 took from the same initial state;
    the largest relative differences of E and J, the rms relative difference of
    the momenta and the largest position difference (cells), particle by
    particle, and both Gauss residuals relative to 4 pi times one species'
    density."""
    g32 = build_grid(P, wl, P.PIC_FP32, stream)
    d0 = P.pic_diagnostics(g32.h)
    P.pic_step(g32.h, steps)
    E32, _, J32 = g32.get_fields()
    E64, _, J64 = g64.get_fields()
    out = {"steps": steps, "E_max_rel": rel_max(E32, E64), "J_max_rel": rel_max(J32, J64)}
    num = den = 0.0
    xmax = 0.0
    for s in range(len(wl.species)):
        c32, o32, w32, i32 = g32.particles(s)
        c64, o64, w64, i64 = g64.particles(s)
        at = np.empty(i64.shape[0], dtype=np.int64)
        at[i64] = np.arange(i64.shape[0])
        k = at[i32]                         # row of each FP32 particle in the FP64 arrays
        for a in range(3):
            d = w32[a].astype(np.float64) - w64[a][k]
            num += float(np.dot(d, d))
            den += float(np.dot(w64[a], w64[a]))
        n3 = wl.n
        for a, (div, mod) in enumerate(((1, n3[0]), (n3[0], n3[1]), (n3[0] * n3[1], n3[2]))):
            x32 = (c32 // div) % mod + o32[a].astype(np.float64)
            x64 = (c64[k] // div) % mod + o64[a][k]
            d = x32 - x64
            d -= mod * np.round(d / mod)
            xmax = max(xmax, float(np.abs(d).max()))
        del c32, o32, w32, i32, c64, o64, w64, i64, at, k
    out["w_rms_rel"] = math.sqrt(num / den) if den > 0 else 0.0
    out["x_max_abs_cells"] = xmax
    rho = abs(wl.species[0].q * wl.species[0].weight) * wl.species[0].x.shape[1] / wl.n_cells
    d32 = P.pic_diagnostics(g32.h)
    out["gauss_rel_fp32"] = d32["gauss_resid_max"] / (4 * math.pi * rho)
    out["energy_rel"] = abs(d32["total"] - P.pic_diagnostics(g64.h)["total"]) / abs(d0["total"])
    g32.close()
    return out


def rel_max(a, b):
    """max |a - b| / max |b| over the arrays of two lists."""
    num = max(float(np.abs(x.astype(np.float64) - y.astype(np.float64)).max()) for x, y in zip(a, b))
    den = max(float(np.abs(y).max()) for y in b)
    return num / den if den > 0 else num


def batched_accuracy(P, sub, cand, build, steps):
    """The batched FP32 form (the persistent kernel) against the plain FP64 method
    (pic_step) on the same runs from the same initial state, after `steps` steps:
    per run the largest relative difference of E and of the total energy, and the
    FP32 Gauss residual; the worst run of each."""
    b32 = build(sub, cand)
    d64 = [P.make_desc(2, wl.n, wl.d, wl.dt, wl.c, P.PIC_FP64, tile=(cand["tile"], cand["tile"], 1), halo=1,
                       sort_interval=cand["K"], rho_bg=wl.rho_bg, stream=b32.desc.cuda_stream) for wl in sub]
    b64 = P.Batch(d64)
    P.pic_load_particles_runs(b64.h, list(range(len(sub))), 0,
                              [(wl.species[0].q, wl.species[0].m, wl.species[0].weight) for wl in sub],
                              [list(wl.species[0].x) for wl in sub], [list(wl.species[0].w) for wl in sub])
    for r in range(len(sub)):       # the residual references are taken at the initial state
        P.pic_diagnostics_run(b32.h, r)
        P.pic_diagnostics_run(b64.h, r)
    P.pic_step_persistent(b32.h, steps)
    P.pic_step(b64.h, steps)
    e_rel, w_rel, gauss = 0.0, 0.0, 0.0
    for r, wl in enumerate(sub):
        E32 = b32.get_fields_run(r)[0]
        E64 = b64.get_fields_run(r)[0]
        e_rel = max(e_rel, rel_max(E32, E64))
        a, c = P.pic_diagnostics_run(b32.h, r), P.pic_diagnostics_run(b64.h, r)
        w_rel = max(w_rel, abs(a["total"] - c["total"]) / abs(c["total"]))
        rho = abs(wl.species[0].q * wl.species[0].weight) * wl.n_particles / wl.n_cells
        gauss = max(gauss, a["gauss_resid_max"] / (4 * math.pi * rho))
    b32.close()
    b64.close()
    return {"runs": len(sub), "steps": steps, "fp32": "pic_step_persistent", "fp64": "pic_step",
            "E_max_rel_worst_run": e_rel, "energy_rel_worst_run": w_rel, "gauss_rel_fp32_worst_run": gauss}


def adjoint_bytes(es):
    """Algorithmic HBM bytes per particle-step of the 2D differentiable run with
    elements of es bytes: the forward step reads and writes the state (cell,
    two offsets, three momenta); the backward pass recomputes each step with a
    snapshot of the state and ids written, restores the snapshot (read, write),
    and the particle adjoint reads the state and reads and writes the adjoints
    of the offsets (two) and the momenta (three).  The grid's share (65,536
    cells against 1,048,576 particles) is left out."""
    state = 4 + 2 * es + 3 * es
    snap = state + 4
    fwd = 2 * state
    bwd = (2 * state + snap) + 2 * snap + (state + 2 * 5 * es)
    return fwd, fwd + bwd


def adjoint_arm(P, W, torch, args, hbm_peak):
    """Differentiable 2D3V run: 256^2 periodic grid, 16 e-/cell, v_th = 0.05c,
    density perturbation A = 0.05 in mode k = 2; loss = field energy in a 32x32
    probe window after `adj_steps` steps; gradient with respect to A and the
    initial momenta by the discrete adjoint with checkpoints every 20 steps.
    Forward and forward+adjoint throughput in FP32 and FP64, and the FP32
    gradient against FP64 central differences of the loss on the GPU."""
    from paper_1101_0809_gb300.adjoint import DifferentiableRun, WindowEnergyLoss
    n, ppc, amp, mode = 256, 16, 0.05, 2
    steps = args.adj_steps
    win = ((112, 144), (112, 144))
    wl0 = W.c4_perturbed2d(n=n, ppc=ppc, amplitude=0.0, mode=mode, steps=steps)
    xu, w0 = wl0.species[0].x.copy(), wl0.species[0].w.copy()
    k = 2 * math.pi * mode / n
    sp = wl0.species[0]

    def x_of(A):
        x = xu.copy()
        x[0] = np.mod(xu[0] - (A / k) * np.sin(k * xu[0]), float(n))
        x[0][x[0] >= n] = 0.0
        return x

    out = {"workload": f"2D3V {n}^2 periodic, {ppc} e-/cell, v_th = 0.05c, perturbation A = {amp} k = {mode}; "
                       f"loss = field energy in a 32x32 window after {steps} steps; checkpoints every 20 steps",
           "particles": wl0.n_particles, "steps": steps}
    for name, prec in (("fp32", P.PIC_FP32), ("fp64", P.PIC_FP64)):
        desc = P.make_desc(2, wl0.n, wl0.d, wl0.dt, wl0.c, prec, tile=(16, 16, 1), rho_bg=wl0.rho_bg)
        # warm-up: a short differentiable run loads every kernel and allocator path once
        warm = DifferentiableRun(desc, sp.q, sp.m, sp.weight, 20, win, checkpoint_every=20)
        Lw = WindowEnergyLoss.apply(torch.from_numpy(x_of(amp)), torch.from_numpy(w0).requires_grad_(), warm)
        Lw.backward()
        torch.cuda.synchronize()
        warm.grid.close()
        run = DifferentiableRun(desc, sp.q, sp.m, sp.weight, steps, win, checkpoint_every=20)
        xu_t = torch.from_numpy(xu)
        passes = []   # the whole pass is short (tens of ms in FP32): the median of three
        for _ in range(3):
            A = torch.tensor(amp, dtype=torch.float64, requires_grad=True)
            x0 = xu_t.clone()
            x0[0] = torch.remainder(xu_t[0] - (A / k) * torch.sin(k * xu_t[0]), float(n))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            L = WindowEnergyLoss.apply(x0, torch.from_numpy(w0), run)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            L.backward()
            torch.cuda.synchronize()
            t2 = time.perf_counter()
            passes.append((t2 - t0, t1 - t0, t2 - t1))
        tot, fwd_s, adj_s = sorted(passes)[1]
        npart = wl0.n_particles
        out[name] = {"fwd": npart * steps / fwd_s, "fwd_adj": npart * steps / tot, "unit": UNIT,
                     "fwd_s": fwd_s, "adj_s": adj_s, "passes": len(passes), "pass_s": [p[0] for p in passes],
                     "loss": float(L.detach()), "dL_dA": float(A.grad.item())}
        bf, bfa = adjoint_bytes(4 if name == "fp32" else 8)
        out[name]["roofline_hbm"] = {
            "scope": "whole pass through the autograd API, host loads included",
            "bytes_per_particle_step": {"fwd": bf, "fwd_adj": bfa},
            "fwd": {"achieved": bf * out[name]["fwd"] / 1e9, "frac": bf * out[name]["fwd"] / 1e9 / hbm_peak},
            "fwd_adj": {"achieved": bfa * out[name]["fwd_adj"] / 1e9,
                        "frac": bfa * out[name]["fwd_adj"] / 1e9 / hbm_peak},
            "unit": "GB/s", "peak": hbm_peak}
        if name == "fp64":
            h = 1e-7 * amp
            lp = run.forward(torch.from_numpy(x_of(amp + h)), torch.from_numpy(w0))
            lm = run.forward(torch.from_numpy(x_of(amp - h)), torch.from_numpy(w0))
            out["fp64_central_fd_dL_dA"] = (lp - lm) / (2 * h)
        run.grid.close()
    out["fp32_device"] = adjoint_device(P, torch, W, wl0, x_of(amp), w0, hbm_peak)
    fd = out["fp64_central_fd_dL_dA"]
    out["fp32_grad_rel_err_vs_fp64_fd"] = abs(out["fp32"]["dL_dA"] - fd) / abs(fd)
    out["fp64_grad_rel_err_vs_fp64_fd"] = abs(out["fp64"]["dL_dA"] - fd) / abs(fd)
    return out


def adjoint_device(P, torch, W, wl0, x0, w0, hbm_peak, nsteps=20):
    """Device-only rates of the FP32 differentiable run's two passes, with CUDA
    events on the grid's stream: the forward step (pic_step) and the adjoint
    step (pic_adjoint_step, with device-resident adjoint arrays), each over
    `nsteps` steps after warm-up.  HBM fractions from the algorithmic bytes of
    the particle kernels (forward: state read and written, 48 B per particle,
    and E, B, J, 36 B per cell; adjoint: state read 24 B, the adjoints of the
    offsets and momenta read and written 40 B, and E, B^n, lamJ, lamE, lamB,
    96 B per cell) over each pass's measured time."""
    st = torch.cuda.Stream()
    desc = P.make_desc(2, wl0.n, wl0.d, wl0.dt, wl0.c, P.PIC_FP32, tile=(16, 16, 1), rho_bg=wl0.rho_bg,
                       stream=st.cuda_stream)
    g = P.Grid(desc)
    sp = wl0.species[0]
    g.load(0, sp.q, sp.m, sp.weight, x0, w0)
    P.pic_step(g.h, 20)            # fields that are not zero
    P.pic_sync(g.h)
    npart, ncell = wl0.n_particles, wl0.n_cells
    gen = torch.Generator(device="cuda").manual_seed(5)
    shape = g.shape
    lamE = [torch.randn(shape, device="cuda", generator=gen) for _ in range(3)]
    lamB = [torch.randn(shape, device="cuda", generator=gen) for _ in range(3)]
    lamx = [torch.randn(npart, device="cuda", generator=gen) for _ in range(3)]
    lamw = [torch.randn(npart, device="cuda", generator=gen) for _ in range(3)]
    torch.cuda.synchronize()

    def timed(fn):
        for _ in range(3):
            fn()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(st):
            e0.record(st)
            for _ in range(nsteps):
                fn()
            e1.record(st)
        e1.synchronize()
        return e0.elapsed_time(e1) / nsteps

    snap = torch.empty(P.pic_state_bytes(g.h), dtype=torch.uint8, device="cuda")
    P.pic_state_save(g.h, snap)
    fwd_ms = timed(lambda: P.pic_step(g.h, 1))
    P.pic_state_restore(g.h, snap)
    adj_ms = timed(lambda: P.pic_adjoint_step(g.h, lamE, lamB, lamx, lamw))
    P.pic_sync(g.h)
    g.close()
    fb, ab = npart * 48 + ncell * 36, npart * 64 + ncell * 96
    fa, aa = fb / (fwd_ms * 1e-3) / 1e9, ab / (adj_ms * 1e-3) / 1e9
    return {"scope": "device only: CUDA events around pic_step and pic_adjoint_step, arrays resident",
            "fwd": npart / (fwd_ms * 1e-3), "adj": npart / (adj_ms * 1e-3),
            "fwd_adj": npart / ((fwd_ms + adj_ms) * 1e-3), "unit": UNIT, "fwd_ms": fwd_ms, "adj_ms": adj_ms,
            "roofline_hbm": {"fwd_frac": fa / hbm_peak, "adj_frac": aa / hbm_peak,
                             "fwd_adj_frac": (fb + ab) / ((fwd_ms + adj_ms) * 1e-3) / 1e9 / hbm_peak,
                             "bytes": {"fwd": fb, "adj": ab}, "peak": hbm_peak, "unit": "GB/s"}}


def laser_arm(P, W, torch, args, hbm_peak):
    """3D relativistic laser-plasma: 512x128x128 periodic box, a0 = 5 plane wave
    of wavelength 20 cells from a one-way antenna plane at x = 8, cold electron
    slab (ramp 128-178, plateau to 384 at 0.01 n_c, 16 per cell), FP32.  Each
    grid runs `laser_warmup` steps with the adaptive tile-sort policy, then 20
    timed steps once the pulse is in the plasma, where the load is most uneven:
    the adaptive policy on 8x4x4 tiles with a one-cell halo, and the
    configuration's fixed sort interval of 10 steps on 4x4x4 tiles with a
    two-cell halo (its fastest tiles: electrons drift farther between sorts,
    and a wider halo keeps more of them on the tiled path)."""
    wl = W.c2_laser_slab()
    sp = wl.species[0]
    a = wl.antenna
    nsteps = 20

    def window(tile, halo, adaptive):
        st = torch.cuda.Stream()
        desc = P.make_desc(3, wl.n, wl.d, wl.dt, wl.c, P.PIC_FP32, tile=tile, halo=halo,
                           sort_interval=wl.sort_interval, particles_per_block=8192, rho_bg=0.0,
                           stream=st.cuda_stream)
        g = P.Grid(desc)
        g.load(0, sp.q, sp.m, sp.weight, sp.x, sp.w)
        P.pic_set_antenna(g.h, 0, a["pol"], a["plane"], a["amplitude"], a["omega"], a["ramp"])
        P.pic_set_sort_policy(g.h, True)
        P.pic_step(g.h, args.laser_warmup)
        P.pic_sync(g.h)
        P.pic_set_sort_policy(g.h, adaptive)
        P.pic_profile(g.h, True)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        P.pic_step(g.h, nsteps)
        e1.record(st)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / nsteps
        prof = P.pic_profile_read(g.h)
        P.pic_profile(g.h, False)
        d = P.pic_diagnostics(g.h)
        g.close()
        pk = prof["particles"][0] / max(prof["particles"][1], 1)
        ach = (wl.n_particles * 56 + wl.n_cells * 36) / (pk * 1e-3) / 1e9
        return {"tile": list(tile), "halo": halo, "value": wl.n_particles / (ms * 1e-3), "ms_per_step": ms,
                "particles_ms": pk, "sorts": prof["sort"][1], "sort_ms": prof["sort"][0] / max(prof["sort"][1], 1),
                "roofline": {"bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
                             "frac": ach / hbm_peak, "alg_bytes_per_launch": wl.n_particles * 56 + wl.n_cells * 36},
                "kinetic": d["kinetic"], "field_E": d["field_E"]}

    adaptive = window((8, 4, 4), 1, True)
    fixed = window((4, 4, 4), 2, False)
    return {"workload": "3D relativistic laser-plasma 512x128x128, a0 = 5, lambda = 20 cells, cold electron slab "
                        "0.01 n_c (ramp 128-178, plateau to 384), 16 per cell, FP32",
            "value": fixed["value"], "unit": UNIT, "particles": wl.n_particles, "cells": wl.n_cells,
            "timed_from_step": args.laser_warmup, "steps": nsteps,
            "fixed_sort_interval_10": fixed, "adaptive_sort": adaptive}


def order5_arm(P, torch, wl, stream, hbm_peak, value_l15, steps):
    """The alternating-order form factor l_a = 2 1/2 (Sec. 4.5) on the main 3D
    workload, FP32, tile 4x4x4 and a sort every 6 steps (its best tile and
    interval: the stencil reaches one cell further, so the staged halos are
    wider).  The particle state read and
    written per step is the same as with l_a = 1 1/2, so the algorithmic bytes
    (and the HBM roofline's numerator) are too."""
    desc = P.make_desc(wl.dims, wl.n, wl.d, wl.dt, wl.c, P.PIC_FP32, tile=(4, 4, 4), halo=1,
                       sort_interval=6, particles_per_block=8192, rho_bg=wl.rho_bg,
                       stream=stream, order2=5)
    g = P.Grid(desc)
    for s, sp in enumerate(wl.species):
        g.load(s, sp.q, sp.m, sp.weight, sp.x, sp.w)
    for _ in range(3):
        P.pic_step(g.h, 1)
    P.pic_sync(g.h)
    ms, prof, launches, _ = timed_steps(P, torch, g, steps)
    npart, ncell = wl.n_particles, wl.n_cells
    pk_ms = prof["particles"][0] / max(prof["particles"][1], 1)
    alg = npart * 56 + ncell * 36
    ach = alg / (pk_ms * 1e-3) / 1e9
    value = npart * steps / (ms * 1e-3)
    g.close()
    return {"workload": "the main 3D workload with l_a = 2 1/2 (order2 = 5), FP32, tile 4x4x4",
            "value": value, "unit": UNIT, "steps": steps, "ms_per_step": ms / steps, "particles_ms": pk_ms,
            "gpu_launches": launches, "ratio_to_l_a_1_5": value / value_l15,
            "roofline": {"bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s", "frac": ach / hbm_peak,
                         "alg_bytes_per_launch": alg}}


def energy_arm(P, args):
    """The energy test of Sec. 5 (X1: 3D 64^3, 2 electrons per cell, v_th = 0.05c,
    immovable ions at the electron positions, 503 steps, FP64) with the
    alternating orders l_a = 1 1/2 and 2 1/2 and the uniform-order l = 2
    interpolation of Eq. wrong1; the largest relative defect of the energy
    integral (sampled every 10 steps) and the stepping rates (FP64 and FP32).
    Also the Langmuir test X5 (1 electron per cell of twice the charge, B_x
    with omega_Be = omega_pe, all electrons streaming at 0.1c: the largest
    defect of the total energy and the period of the field energy) and the
    gyration test X6 (an electron and a positron at w = +-0.5c in B_z with
    omega_Be = 10, 1600 steps: kinetic energy ratio and Larmor radii).  With
    --energy-x4 also the two-stream test (B_x with omega_Be = omega_pe, streams
    +-0.1c, 8000 steps)."""
    from paper_1101_0809_gb300 import workloads as W
    from paper_1101_0809_gb300.energy import energy_run
    wl = W.x1_energy()
    out = {"workload": wl.name + ", 503 steps, FP64", "particles": wl.n_particles, "x1": {}}
    for order2, name in ((3, "l_a_1_5"), (4, "wrong1_l_2"), (5, "l_a_2_5")):
        r64 = energy_run(wl, order2, P.PIC_FP64)
        r32 = energy_run(wl, order2, P.PIC_FP32)
        out["x1"][name] = {"max_rel_defect": r64["max_rel_defect"], "final_rel_defect": r64["final_rel_defect"],
                           "fp64_particle_steps_per_s": r64["particle_steps_per_s"],
                           "fp32_particle_steps_per_s": r32["particle_steps_per_s"],
                           "fp32_max_rel_defect": r32["max_rel_defect"]}
    x1 = out["x1"]
    out["defect_ratio_wrong1_to_l_a_1_5"] = x1["wrong1_l_2"]["max_rel_defect"] / x1["l_a_1_5"]["max_rel_defect"]
    out["speed_ratio_l_a_1_5_to_wrong1_fp32"] = (x1["l_a_1_5"]["fp32_particle_steps_per_s"] /
                                                 x1["wrong1_l_2"]["fp32_particle_steps_per_s"])
    from paper_1101_0809_gb300.energy import gyration_run, oscillation_period
    wl5, bx5 = W.x5_langmuir(steps=args.energy_x5_steps)
    r5 = energy_run(wl5, 3, P.PIC_FP64, every=5, bx=bx5)
    steps5 = [q[0] for q in r5["series"]]
    out["x5"] = {"workload": wl5.name + f", {wl5.steps} steps, FP64, l_a = 1 1/2",
                 "max_rel_defect": r5["max_rel_defect"],
                 "field_energy_period_steps": oscillation_period(steps5, [q[3] for q in r5["series"]]),
                 "expected_period_steps": math.pi * (1.0 + (2.0 / wl5.c) ** 2) ** 0.75 / wl5.dt,
                 "kinetic_range": [min(q[2] for q in r5["series"]), max(q[2] for q in r5["series"])],
                 "field_E_range": [min(q[3] for q in r5["series"]), max(q[3] for q in r5["series"])]}
    wl6, bz6 = W.x6_gyration()
    out["x6"] = {"workload": wl6.name + f", {wl6.steps} steps, FP64, l_a = 1 1/2",
                 **gyration_run(wl6, 3, P.PIC_FP64, bz6)}
    if args.energy_x4:
        wl4, bx = W.x4_two_stream()
        out["x4"] = {"workload": wl4.name + ", 8000 steps, FP64, initial B_x field energy excluded"}
        for order2, name in ((3, "l_a_1_5"), (4, "wrong1_l_2")):
            r = energy_run(wl4, order2, P.PIC_FP64, every=100, bx=bx)
            out["x4"][name] = {"max_rel_defect": r["max_rel_defect"], "final_rel_defect": r["final_rel_defect"],
                               "fp64_particle_steps_per_s": r["particle_steps_per_s"]}
    return out


def vecpot_arm(P):
    """Generalized-momentum conservation (Sec. 4.2) with the vector-potential
    formulation: 262,144 test particles (w ~ N(0, 0.3c), negligible charge) in
    the static field A_z = 3 (sin(2 pi 8 x/256) + cos(2 pi 8 y/256)) of a 2D
    256^2 grid, FP64, over 48 time units (120 x nsub steps of 0.4 / nsub); the largest
    change of the summed P_z per particle, for dt and dt/2, with l_a = 1 1/2
    and with the interpolation of Eq. wrong1."""
    import numpy as np
    n, count, wt = 256, 262144, 1e-12
    X, Y = np.meshgrid(np.arange(n) + 0.5, np.arange(n) + 0.5)
    Az = (3.0 * (np.sin(2 * math.pi * 8 * X / n) + np.cos(2 * math.pi * 8 * Y / n))).reshape(1, n, n)
    rng = np.random.default_rng(9)
    x = np.zeros((3, count))
    x[0] = rng.uniform(0, n, count)
    x[1] = rng.uniform(0, n, count)
    w = rng.normal(0, 0.3, (3, count))
    out = {"workload": "262,144 test particles in a static A_z(x, y) on a 2D 256^2 grid, FP64, 48 time units",
           "unit": "largest |P_z(t) - P_z(0)| per particle and unit weight"}
    for order2, name in ((3, "l_a_1_5"), (4, "wrong1_l_2")):
        drifts = []
        for nsub in (1, 2):
            desc = P.make_desc(2, (n, n, 1), (1.0, 1.0, 1.0), 0.4 / nsub, 1.0, P.PIC_FP64, tile=(16, 16, 1),
                               order2=order2)
            g = P.Grid(desc)
            P.pic_set_vector_potential(g.h, [np.zeros((1, n, n)), np.zeros((1, n, n)), Az], set_B=True)
            g.load(0, -1.0, 1.0, wt, x, w)
            p0 = P.pic_generalized_momentum(g.h)[2] / wt
            worst = 0.0
            for _ in range(120):
                P.pic_step(g.h, nsub)
                worst = max(worst, abs(P.pic_generalized_momentum(g.h)[2] / wt - p0))
            g.close()
            drifts.append(worst / count)
        out[name] = {"drift_dt": drifts[0], "drift_dt_half": drifts[1], "ratio": drifts[0] / drifts[1]}
    return out


def _g(v, digits=4):
    """A number rounded to a few significant digits for the compact summary."""
    if v is None:
        return None
    if isinstance(v, bool) or isinstance(v, int):
        return v
    return float(f"{v:.{digits}g}")


def summary_line(value, ms_step, roof, gauss, fp64, batched, adjoint, laser, order5, energy, vecpot, e2e, cpu):
    """The flat summary that ends the JSON line: every leg's headline figures,
    rounded, so that the end of the line alone carries them.  Rates in
    particle-steps/s; *_frac are fractions of the measured HBM (or FP64 FMA)
    peak; *_rel are relative differences against the FP64 method."""
    s = {"fp32": _g(value), "fp32_ms_step": _g(ms_step), "fp32_kernel_ms": _g(roof["avg_launch_ms"]),
         "fp32_hbm_frac": _g(roof["frac"]), "sort_share": _g(roof["step_share"].get("sort"))}
    if "issue" in roof:
        s["fp32_issue_frac"] = _g(roof["issue"]["frac"])
    if "shared_pipe" in roof:
        s["fp32_shared_pipe_frac"] = _g(roof["shared_pipe"]["frac"])
    if gauss:
        s["gauss_fp32_200_steps_rel"] = _g(gauss["gauss_resid_max_rel"])
    if fp64:
        s["fp64"] = _g(fp64["value"])
        s["fp64_hbm_frac"] = _g(fp64["roofline_hbm"]["frac"])
        if "roofline_fp64" in fp64:
            s["fp64_fma_frac"] = _g(fp64["roofline_fp64"]["frac"])
        s["fp64_fma_peak_per_s"] = _g(fp64["fp64_fma_peak_measured"]["fma_per_s"])
        s["fp32_over_fp64"] = _g(fp64["fp32_speedup"])
        acc = fp64.get("fp32_vs_fp64")
        if acc:
            for k in ("E_max_rel", "J_max_rel", "w_rms_rel", "x_max_abs_cells", "gauss_rel_fp32"):
                s["fp32_vs_fp64_" + k] = _g(acc[k], 3)
    if batched:
        s["batched"] = _g(batched["value"])
        s["batched_hbm_frac"] = _g(batched["roofline"]["frac"])
        s["batched_tile_ppb_K"] = [batched["autotuned"][k] for k in ("tile", "ppb", "K")]
        s["batched_E_rel_worst"] = _g(batched["accuracy_vs_fp64"]["E_max_rel_worst_run"], 3)
    if adjoint:
        s["adj_fp32_fwd_adj"] = _g(adjoint["fp32"]["fwd_adj"])
        s["adj_fp32_fwd_adj_hbm_frac"] = _g(adjoint["fp32"]["roofline_hbm"]["fwd_adj"]["frac"], 3)
        s["adj_fp64_fwd_adj"] = _g(adjoint["fp64"]["fwd_adj"])
        dev = adjoint.get("fp32_device")
        if dev:
            s["adj_dev_fwd_adj"] = _g(dev["fwd_adj"])
            s["adj_dev_adj_hbm_frac"] = _g(dev["roofline_hbm"]["adj_frac"], 3)
            s["adj_dev_fwd_adj_hbm_frac"] = _g(dev["roofline_hbm"]["fwd_adj_frac"], 3)
        s["adj_fp32_grad_rel_vs_fd"] = _g(adjoint["fp32_grad_rel_err_vs_fp64_fd"], 3)
    if laser:
        s["laser_k10"] = _g(laser["fixed_sort_interval_10"]["value"])
        s["laser_k10_hbm_frac"] = _g(laser["fixed_sort_interval_10"]["roofline"]["frac"], 3)
        s["laser_adaptive"] = _g(laser["adaptive_sort"]["value"])
    if order5:
        s["la25"] = _g(order5["value"])
        s["la25_hbm_frac"] = _g(order5["roofline"]["frac"], 3)
    if energy:
        s["x1_defect_la15"] = _g(energy["x1"]["l_a_1_5"]["max_rel_defect"], 3)
        s["x1_defect_wrong1"] = _g(energy["x1"]["wrong1_l_2"]["max_rel_defect"], 3)
        s["x5_period_vs_expected"] = [_g(energy["x5"]["field_energy_period_steps"]),
                                      _g(energy["x5"]["expected_period_steps"])]
    if vecpot:
        s["pz_drift_ratio_la15_wrong1"] = [_g(vecpot["l_a_1_5"]["ratio"], 3), _g(vecpot["wrong1_l_2"]["ratio"], 3)]
    if e2e:
        s["e2e_serial"] = _g(e2e["serial"]["value"])
    if cpu:
        s["cpu_1core"] = _g(cpu["single_core"]["value"])
    return s


def measure_fp64_fma(P, torch):
    """The device's FP64 FMA rate: the pic_measure_fp64_fma kernel (8 blocks of
    256 threads per SM, 8 independent chains per thread), timed with CUDA events
    after a warm-up launch; best of 3."""
    sink = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = torch.cuda.current_stream()
    iters = 20000
    P.pic_measure_fp64_fma(1000, 8, sink, st.cuda_stream)
    best = None
    for _ in range(3):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        n = P.pic_measure_fp64_fma(iters, 8, sink, st.cuda_stream)
        e1.record(st)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        if best is None or ms < best[0]:
            best = (ms, n)
    ms, n = best
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    rate = n / (ms * 1e-3)
    return {"fma_per_s": rate, "flops": 2 * rate, "ms": ms, "fma": n, "sms": sms}


def our_arm(args):
    import torch
    rank, local, world = dist_env()
    dist = None
    if world > 1:
        import torch.distributed as D
        torch.cuda.set_device(local)
        D.init_process_group("nccl")
        dist = D
    else:
        torch.cuda.set_device(0)
    peaks = None
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(peaks_path):
        with open(peaks_path) as f:
            peaks = json.load(f)
    hbm_peak = peaks["hbm_gbs"] if peaks else 6800.0
    peak_note = "measured" if peaks else "fallback"

    # CPU baseline first, before any GPU work in this process
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        rate1, sample1, frac, nst = time_oracle(args.n, args.ppc)
        rate, sample, cores = time_oracle_cores(args.n, args.ppc, nst, frac)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
               "single_core": {"value": rate1, "sample": sample1}, "other_configs": time_oracle_small()}

    from paper_1101_0809_gb300 import build as B
    B.build()
    from paper_1101_0809_gb300 import pic as P
    from paper_1101_0809_gb300 import workloads as W

    global SORT_ORDER
    if args.cell_lanes:
        SORT_ORDER = P.PIC_SORT_CELL_LANES
    wl = W.c1_thermal3d(n=args.n, ppc=args.ppc, steps=args.steps)
    if args.sort_interval > 0:
        wl.sort_interval = args.sort_interval
    npart = wl.n_particles
    ncell = wl.n_cells
    stream = torch.cuda.current_stream().cuda_stream
    sampler = ClockSampler(local)

    # ---- FP32 form, device-resident --------------------------------------------------
    grid = build_grid(P, wl, P.PIC_FP32, stream)
    P.pic_diagnostics(grid.h)          # the residual reference of Gauss's law: the initial state
    for _ in range(args.warmup):
        P.pic_step(grid.h, 1)
    P.pic_sync(grid.h)
    ms, prof, launches, clocks = timed_steps(P, torch, grid, args.steps, dist, sampler)
    P.pic_sync(grid.h)
    # the FP32 charge-conservation residual after the workload's 200 steps at full size
    gauss = None
    if not args.no_gauss:
        done = args.warmup + args.steps
        if done < 200:
            P.pic_step(grid.h, 200 - done)
        dg = P.pic_diagnostics(grid.h)
        rho_e = abs(wl.species[0].q * wl.species[0].weight) * wl.species[0].x.shape[1] / (ncell * wl.volume)
        gauss = {"steps": max(done, 200), "gauss_resid_max_rel": dg["gauss_resid_max"] / (4 * math.pi * rho_e),
                 "gauss_resid_rms_rel": dg["gauss_resid_rms"] / (4 * math.pi * rho_e),
                 "scale": "4 pi |q_e| n_e (one species' density)", "n_particles": dg["n_particles"],
                 "error_word": dg["error_word"]}
    ms_step = ms / args.steps
    value = world * npart * args.steps / (ms * 1e-3)
    pk_ms, pk_n = prof["particles"]
    # algorithmic bytes of the fused kernel: particle SoA read + write (int32 cell,
    # 3 float offsets, 3 float momenta) and the E, B read + J write of the grid
    alg_bytes = npart * 2 * (4 + 12 + 12) + ncell * (6 * 4 + 3 * 4)
    achieved = alg_bytes / (pk_ms / pk_n * 1e-3) / 1e9
    tpp = ncu_traffic_per_particle("fp32")
    roof = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
            "frac": achieved / hbm_peak, "traffic": (tpp * npart) if tpp else None,
            "kernel": "k_particles<3,float,fused>", "peak_source": peak_note,
            "alg_bytes_per_launch": alg_bytes, "avg_launch_ms": pk_ms / pk_n,
            "step_share": {k: v[0] / ms for k, v in prof.items()}}
    # the unit that binds the kernel: instruction issue (warp instructions per
    # particle from the committed ncu summary, 4 per SM per clock at the clock
    # sampled during the timed steps)
    ipp = ncu_per_particle("fp32", "warp_instructions_per_particle")
    sm_mhz = (clocks or {}).get("sm_mhz") or (peaks["sm_max_mhz"] if peaks else 2070.0)
    if ipp:
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        issue_peak = 4.0 * sms * sm_mhz * 1e6
        issue_ach = ipp * npart / (pk_ms / pk_n * 1e-3)
        roof["issue"] = {"achieved": issue_ach, "peak": issue_peak, "unit": "warp instructions/s",
                         "frac": issue_ach / issue_peak, "warp_instructions_per_particle": ipp,
                         "peak_source": f"4 per SM per clock x {sms} SMs x {sm_mhz:.0f} MHz (sampled)"}
    # and the shared-memory data pipe (the gather's loads and the deposit's
    # atomics): shared wavefronts per particle from the same profile, against one
    # wavefront per SM per clock; `ideal` counts them without bank conflicts
    wpp = ncu_per_particle("fp32", "shared_wavefronts_per_particle")
    wpp_ideal = ncu_per_particle("fp32", "shared_wavefronts_ideal_per_particle")
    if wpp:
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        sh_peak = 1.0 * sms * sm_mhz * 1e6
        sh_ach = wpp * npart / (pk_ms / pk_n * 1e-3)
        roof["shared_pipe"] = {"achieved": sh_ach, "peak": sh_peak, "unit": "wavefronts/s", "frac": sh_ach / sh_peak,
                               "wavefronts_per_particle": wpp, "ideal_wavefronts_per_particle": wpp_ideal,
                               "peak_source": f"1 per SM per clock x {sms} SMs x {sm_mhz:.0f} MHz (sampled)"}

    # ---- end to end through the public API with host buffers ---------------------------
    # Each step uploads its whole input state from pinned host memory and reads
    # its diagnostics back.  Headline: the state as the library stores it (a
    # snapshot: cells, ids, offsets, momenta, E, B) through pic_state_restore.
    # Beside it, the initial-condition path: FP64 positions and momenta through
    # pic_load_particles (conversion to cell + offset and a sort from random order).
    e2e = None
    if not args.no_e2e:
        def timed_host(step_fn, nsteps):
            step_fn()
            if dist is not None:
                dist.barrier()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(nsteps):
                step_fn()
            torch.cuda.synchronize()
            el = time.perf_counter() - t0
            if dist is not None:
                el = max_over_ranks(dist, el, "cuda")
            return el

        nbytes = P.pic_state_bytes(grid.h)
        host_state = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
        P.pic_state_save(grid.h, host_state)
        e2e_steps = max(1, min(args.steps, 5))

        def e2e_step():
            P.pic_state_restore(grid.h, host_state)
            P.pic_step(grid.h, 1)
            return P.pic_diagnostics(grid.h)

        el = timed_host(e2e_step, e2e_steps)
        serial = {"value": world * npart * e2e_steps / el, "unit": UNIT, "steps": e2e_steps,
                  "step": "pic_state_restore (pinned host snapshot: cells, ids, offsets, momenta, E, B, tile "
                          "starts) + pic_step + pic_diagnostics, one grid, nothing overlapped"}

        # Pipelined: two grids on two streams take the steps in turn, so the
        # upload of step k+1 (copy engines) runs under the kernels of step k.
        # Every step still uploads its whole state and reads its diagnostics back.
        side = torch.cuda.Stream()
        grid2 = build_grid(P, wl, P.PIC_FP32, side.cuda_stream)
        pair = (grid, grid2)
        pipe_steps = max(2, args.steps)   # as many steps as the device-timed loop: the fill and drain amortize

        def enqueue(k):
            g = pair[k % 2]
            P.pic_state_restore_async(g.h, host_state)
            P.pic_step(g.h, 1)

        def pipelined(nsteps):
            enqueue(0)
            out = []
            for k in range(nsteps):
                if k + 1 < nsteps:
                    enqueue(k + 1)
                out.append(P.pic_diagnostics(pair[k % 2].h))
            return out

        pipelined(2)
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        diags = pipelined(pipe_steps)
        torch.cuda.synchronize()
        el_p = time.perf_counter() - t0
        if dist is not None:
            el_p = max_over_ranks(dist, el_p, "cuda")
        same = all(abs(d["total"] - diags[0]["total"]) <= 1e-9 * abs(diags[0]["total"]) for d in diags)
        e2e = {"value": world * npart * pipe_steps / el_p, "unit": UNIT, "h2d_bytes_per_step": nbytes,
               "d2h_bytes_per_step": 136, "steps": pipe_steps,
               "step": "pic_state_restore_async (pinned host snapshot: cells, ids, offsets, momenta, E, B, tile "
                       "starts) + pic_step + pic_diagnostics, two grids on two streams in turn, the upload of one "
                       "step under the kernels of the previous one",
               "same_result_every_step": bool(same), "serial": serial}
        grid2.close()
        del grid2, pair, host_state

        pinned = []
        for sp in wl.species:
            x = [torch.from_numpy(np.ascontiguousarray(sp.x[a])).pin_memory() for a in range(3)]
            w = [torch.from_numpy(np.ascontiguousarray(sp.w[a])).pin_memory() for a in range(3)]
            pinned.append((sp, x, w))
        fields = [torch.zeros(wl.n[::-1], dtype=torch.float32).pin_memory() for _ in range(6)]
        load_steps = 2

        def load_step():
            P.pic_set_fields(grid.h, fields[:3], fields[3:])
            for s, (sp, x, w) in enumerate(pinned):
                P.pic_load_particles(grid.h, s, sp.q, sp.m, sp.weight, x, w)
            P.pic_step(grid.h, 1)
            return P.pic_diagnostics(grid.h)

        el = timed_host(load_step, load_steps)
        e2e["initial_condition_path"] = {
            "value": world * npart * load_steps / el, "unit": UNIT,
            "h2d_bytes_per_step": npart * 6 * 8 + 6 * ncell * 4, "d2h_bytes_per_step": 136, "steps": load_steps,
            "step": "pic_set_fields + pic_load_particles (pinned host FP64 x, w, one call per species) + pic_step "
                    "+ pic_diagnostics"}
        del pinned, fields
    grid.close()
    del grid

    # ---- FP64 path ----------------------------------------------------------------------
    fp64 = None
    if not args.no_fp64:
        g64 = build_grid(P, wl, P.PIC_FP64, stream)
        for _ in range(min(args.warmup, 2)):
            P.pic_step(g64.h, 1)
        P.pic_sync(g64.h)
        k64 = max(1, min(args.steps, args.fp64_steps))
        ms64, prof64, l64, _ = timed_steps(P, torch, g64, k64, dist, None)
        P.pic_sync(g64.h)
        pk64_ms, pk64_n = prof64["particles"]
        alg64 = npart * 2 * (4 + 24 + 24) + ncell * (6 * 8 + 3 * 8)
        ach64 = alg64 / (pk64_ms / pk64_n * 1e-3) / 1e9
        fp64 = {"value": world * npart * k64 / (ms64 * 1e-3), "unit": UNIT, "steps": k64,
                "ms_per_step": ms64 / k64, "dtype": "f64",
                "roofline_hbm": {"achieved": ach64, "peak": hbm_peak, "unit": "GB/s", "frac": ach64 / hbm_peak},
                "fp32_speedup": (npart * args.steps / (ms * 1e-3)) / (npart * k64 / (ms64 * 1e-3))}
        # the unit that binds the FP64 kernel: the FP64 pipe, 2 instructions (DADD,
        # DMUL or DFMA) per SM per clock; FP64 instructions per particle from the
        # committed ncu summary of the same kernel source
        f64pp = ncu_per_particle("fp64", "fp64_instr_per_particle")
        fma_rate = measure_fp64_fma(P, torch)
        fp64["fp64_fma_peak_measured"] = fma_rate
        if f64pp:
            alu_ach = f64pp * npart / (pk64_ms / pk64_n * 1e-3)
            fp64["roofline_fp64"] = {"bound": "alu", "achieved": alu_ach, "peak": fma_rate["fma_per_s"],
                                     "unit": "FP64 instructions/s", "frac": alu_ach / fma_rate["fma_per_s"],
                                     "fp64_instructions_per_particle": f64pp,
                                     "peak_source": "measured: the FP64 FMA rate of pic_measure_fp64_fma"}
        if rank == 0:
            fp64["fp32_vs_fp64"] = main_accuracy(P, wl, stream, g64, min(args.warmup, 2) + k64)
        g64.close()

    batched = None
    if not args.no_batch:
        batched = batched_arm(P, W, torch, args, dist, hbm_peak)
    adjoint = None
    if not args.no_adjoint and rank == 0:
        adjoint = adjoint_arm(P, W, torch, args, hbm_peak)
    laser = None
    if not args.no_laser:
        laser = laser_arm(P, W, torch, args, hbm_peak)
    energy = None
    if not args.no_energy and rank == 0:
        energy = energy_arm(P, args)
    vecpot = None
    if not args.no_vecpot and rank == 0:
        vecpot = vecpot_arm(P)
    order5 = None
    if not args.no_order5:
        order5 = order5_arm(P, torch, wl, stream, hbm_peak, value / world, min(args.steps, 10))

    if rank == 0:
        detail = {"roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gauss_200": gauss, "fp64": fp64,
                  "batched": batched, "adjoint": adjoint, "laser": laser, "l_a_2_5": order5, "energy": energy,
                  "vector_potential": vecpot}
        # every leg in full on stderr; stdout carries the one compact line
        print(json.dumps({"detail": detail}), file=sys.stderr, flush=True)
        roof_line = {k: roof[k] for k in ("bound", "achieved", "peak", "unit", "frac", "traffic", "kernel",
                                          "peak_source", "alg_bytes_per_launch", "avg_launch_ms")}
        cpu_line = None if cpu is None else {k: cpu[k] for k in ("value", "unit", "cores", "kind", "sample")}
        e2e_line = None if e2e is None else {k: e2e[k] for k in ("value", "unit", "h2d_bytes_per_step",
                                                                 "d2h_bytes_per_step", "steps")}
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": "f32", "data": "synthetic",
               "config": {"workload": WORKLOAD, "model": "ChCPIC step, FP32 form",
                          "global_batch": world * npart, "particles_per_gpu": npart, "cells": ncell,
                          "tile": list(wl.tile), "sort_interval": wl.sort_interval,
                          "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                          "l2": "inputs larger than L2 (3.76 GB of particle SoA); no flush"},
               "roofline": roof_line, "cpu_baseline": cpu_line, "e2e": e2e_line, "gpu_launches": launches,
               "clocks": clocks,
               "summary": summary_line(value, ms_step, roof, gauss, fp64, batched, adjoint, laser, order5, energy,
                                       vecpot, e2e, cpu)}
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        reference_arm(args)
    else:
        our_arm(args)


if __name__ == "__main__":
    main()
