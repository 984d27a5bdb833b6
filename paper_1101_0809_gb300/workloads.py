"""Seeded synthetic plasmas shaped like the paper's workloads.

This module holds no arithmetic of the method: it only draws positions and
momenta and fixes the run parameters (grid, time step, speed of light, species
charges, masses and macro weights).  Both the CUDA library's tests/benchmark and
the CPU oracle are fed from it.

Normalization (Gaussian units, Sec. 5 of the paper): the cell is one Debye
length, dx = v_th/omega_pe with omega_pe = 1, so c = v_th/(v_th/c).  One electron
has q = -1, m = 1; the macro weight W makes 4 pi n q^2/m = omega_pe^2 = 1 with
n = W*ppc/V, i.e. W = V/(4 pi ppc).  Momenta are w-space Maxwellians: every
component of w = gamma*v is drawn from N(0, v_th^2).  Positions are uniform.
Random streams are numpy PCG64 seeded with SEED_BASE + config index.
"""
from dataclasses import dataclass, field
import math

import numpy as np

SEED_BASE = 1101080900


@dataclass
class SpeciesInit:
    name: str
    q: float            # physical charge per particle
    m: float            # physical mass per particle
    weight: float       # physical particles per macro-particle
    x: np.ndarray       # (3, n) float64 absolute normalized positions in [0, N)
    w: np.ndarray       # (3, n) float64 momentum-to-mass ratio at t = -1/2

    @property
    def n(self):
        return self.x.shape[1]


@dataclass
class Workload:
    name: str
    dims: int
    n: tuple            # (nx, ny, nz); nz == 1 for dims == 2
    d: tuple            # (dx, dy, dz)
    dt: float
    c: float
    species: list = field(default_factory=list)
    rho_bg: float = 0.0  # uniform immobile background charge density
    steps: int = 1
    tile: tuple = (8, 8, 8)
    sort_interval: int = 10
    antenna: dict = None   # plane-wave antenna: pol, plane, amplitude, omega, ramp

    @property
    def n_particles(self):
        return sum(s.n for s in self.species)

    @property
    def n_cells(self):
        return self.n[0] * self.n[1] * (self.n[2] if self.dims == 3 else 1)

    @property
    def volume(self):
        return self.d[0] * self.d[1] * (self.d[2] if self.dims == 3 else 1.0)


def _uniform_positions(rng, dims, n_cells_axes, count):
    x = np.zeros((3, count))
    for a in range(dims):
        x[a] = rng.uniform(0.0, float(n_cells_axes[a]), size=count)
        # uniform() is half-open; guard the float edge so that x < N holds
        x[a][x[a] >= n_cells_axes[a]] = 0.0
    return x


def thermal_plasma(name, dims, n, ppc, vth_over_c, steps, seed, ions=None, tile=None,
                   sort_interval=10, dt_courant=0.5, fraction=1.0):
    """A periodic thermal electron plasma with dx = lambda_De, omega_pe = 1.

    ``ions`` None gives a uniform immobile neutralising background; a mass ratio
    gives a mobile ion species with the same ppc and v_th,i = v_th,e/sqrt(ratio).
    ``fraction`` < 1 keeps a random subset of the particles (same weight), used
    only for bounded CPU samples of a large workload.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    nn = (n[0], n[1], n[2] if dims == 3 else 1)
    vth = 1.0                       # dx = v_th/omega_pe = 1
    c = vth / vth_over_c
    dt = dt_courant / c             # dt = dt_courant * dx / c
    V = 1.0
    cells = nn[0] * nn[1] * nn[2]
    W = V / (4.0 * math.pi * ppc)
    count = int(round(cells * ppc * fraction))
    species = []
    xe = _uniform_positions(rng, dims, nn, count)
    we = rng.normal(0.0, vth, size=(3, count))
    species.append(SpeciesInit("electrons", -1.0, 1.0, W, xe, we))
    rho_bg = 0.0
    if ions is None:
        rho_bg = W * ppc / V        # uniform background of charge +e per electron
    else:
        xi = _uniform_positions(rng, dims, nn, count)
        wi = rng.normal(0.0, vth / math.sqrt(ions), size=(3, count))
        species.append(SpeciesInit("ions", 1.0, float(ions), W, xi, wi))
    if tile is None:
        tile = (8, 8, 8) if dims == 3 else (16, 16, 1)
    return Workload(name, dims, nn, (1.0, 1.0, 1.0), dt, c, species, rho_bg, steps,
                    tuple(tile), sort_interval)


def c0_small2d(steps=50):
    """2D3V periodic 32x32, 8 e-/cell, v_th = 0.05c, dt = 0.5 dx/c, uniform ion background."""
    return thermal_plasma("2D3V 32x32 8ppc vth=0.05c", 2, (32, 32, 1), 8, 0.05, steps,
                          SEED_BASE + 0, tile=(8, 8, 1))


def c1_thermal3d(n=128, ppc=32, steps=200, fraction=1.0, tile=(8, 4, 4), sort_interval=4):
    """3D3V periodic n^3, electrons and ions (mass ratio 1836) ppc each, v_th,e = 0.1c,
    dt = 0.45 dx/c.  At n = 128, ppc = 32 this is 134,217,728 particles.  The
    particles are re-sorted every 4 steps: electrons move 0.045 cells per step
    on average (0.2 in the tail), so over longer intervals more of them collide
    on shared-memory banks or drift past the one-cell halo of their tile and
    take the slower global-memory path, while shorter ones spend more on sorts."""
    return thermal_plasma(f"3D3V {n}^3 e+i {ppc}ppc each vth=0.1c", 3, (n, n, n), ppc, 0.1,
                          steps, SEED_BASE + 1, ions=1836.0, tile=tile,
                          sort_interval=sort_interval, dt_courant=0.45, fraction=fraction)


def c2_laser_slab(n=(512, 128, 128), ppc=16, a0=5.0, wavelength=20.0, steps=1000, dims=3,
                  slab=(128.0, 178.0, 384.0), plane=8, tile=(8, 4, 4), sort_interval=10, dt_courant=0.45,
                  seed_offset=2, ramp_periods=2.0):
    """3D relativistic laser-plasma.  Periodic box, c = 1, dx = 1, dt = 0.45;
    a linearly polarized (E_y) plane wave of wavelength 20 cells and a0 = 5
    (E_0 = a0 m omega c / e = a0 omega) from a one-way antenna plane at x = 8
    with a sin^2 rise over two periods; cold electrons in a slab, density
    rising linearly over x in [128, 178), plateau at 0.01 n_c (n_c = m omega^2 /
    (4 pi e^2)) up to x = 384, vacuum elsewhere.  16 candidates per cell, one
    at x kept with probability n(x)/n_plateau, so all weights are equal.  The
    immobile ions enter only rho and are left out: Gauss's residual is tracked
    against its initial value.  ``dims`` = 2 gives the same slab in 2D (test
    sizes; they also take a shorter rise, ``ramp_periods``)."""
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + seed_offset))
    nn = (n[0], n[1], n[2] if dims == 3 else 1)
    c = 1.0
    dt = dt_courant / c
    omega = 2.0 * math.pi * c / wavelength
    n_c = omega * omega / (4.0 * math.pi)
    V = 1.0
    W = 0.01 * n_c * V / ppc
    x0, x1, x2 = slab
    i_lo, i_hi = int(math.floor(x0)), int(math.ceil(x2))
    ncand = (i_hi - i_lo) * nn[1] * nn[2] * ppc
    x = np.zeros((3, ncand))
    x[0] = rng.uniform(float(i_lo), float(i_hi), size=ncand)
    x[1] = rng.uniform(0.0, float(nn[1]), size=ncand)
    if dims == 3:
        x[2] = rng.uniform(0.0, float(nn[2]), size=ncand)
    keep_p = np.clip((x[0] - x0) / (x1 - x0), 0.0, 1.0)
    keep_p[x[0] >= x2] = 0.0
    keep = rng.uniform(0.0, 1.0, size=ncand) < keep_p
    x = np.ascontiguousarray(x[:, keep])
    for a in range(dims):
        x[a][x[a] >= nn[a]] = 0.0
    w = np.zeros_like(x)
    sp = SpeciesInit("electrons", -1.0, 1.0, W, x, w)
    ant = {"pol": 1, "plane": plane, "amplitude": a0 * omega * c, "omega": omega,
           "ramp": ramp_periods * wavelength / c}
    name = f"{dims}D laser slab {n[0]}x{n[1]}" + (f"x{n[2]}" if dims == 3 else "") + f" a0={a0}"
    return Workload(name, dims, nn, (1.0, 1.0, 1.0), dt, c, [sp], 0.0, steps,
                    tuple(tile) if dims == 3 else (tile[0], tile[1], 1), sort_interval, ant)


def c4_perturbed2d(n=256, ppc=16, amplitude=0.05, mode=2, steps=200, seed_offset=4):
    """2D3V periodic n^2, 16 e-/cell, v_th = 0.05c, density perturbation
    n = n0 (1 + A cos(k x)) loaded as x_p = x_u - (A/k) sin(k x_u), k = 2 pi mode / L_x."""
    wl = thermal_plasma(f"2D3V {n}x{n} {ppc}ppc perturbed A={amplitude} k={mode}", 2,
                        (n, n, 1), ppc, 0.05, steps, SEED_BASE + seed_offset, tile=(16, 16, 1))
    xe = wl.species[0].x
    k = 2.0 * math.pi * mode / n
    xe[0] = np.mod(xe[0] - (amplitude / k) * np.sin(k * xe[0]), float(n))
    xe[0][xe[0] >= n] = 0.0
    return wl


def c3_ensemble_params(nruns=256, seed=SEED_BASE + 3):
    """Per-run parameters of the batched 2D3V ensemble: square grids N ~ U{32..256},
    ppc ~ U{4..64}, v_th ~ U[0.01c, 0.3c]; c = 1, dx = 1, dt = 0.5 (reading c-9:
    omega_pe = v_th/c so that dx = lambda_De in every run)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for r in range(nruns):
        N = int(rng.integers(32, 257))
        ppc = int(rng.integers(4, 65))
        vth = float(rng.uniform(0.01, 0.3))
        out.append({"n": N, "ppc": ppc, "vth": vth, "seed": int(rng.integers(0, 2**31))})
    return out


def c3_run(params):
    """One run of the batched ensemble (c = 1, dx = 1, dt = 0.5, omega_pe = v_th)."""
    rng = np.random.Generator(np.random.PCG64(params["seed"]))
    N, ppc, vth = params["n"], params["ppc"], params["vth"]
    c, dt, V = 1.0, 0.5, 1.0
    wpe = vth                       # dx = v_th/omega_pe = 1
    W = wpe * wpe * V / (4.0 * math.pi * ppc)
    count = N * N * ppc
    x = _uniform_positions(rng, 2, (N, N, 1), count)
    w = rng.normal(0.0, vth, size=(3, count))
    sp = SpeciesInit("electrons", -1.0, 1.0, W, x, w)
    return Workload(f"2D3V {N}x{N} {ppc}ppc vth={vth:.3f}c", 2, (N, N, 1), (1.0, 1.0, 1.0), dt, c,
                    [sp], W * ppc / V, 500, (16, 16, 1), 10)


# Ions that do not move: a species of charge +e whose mass makes q dt/(2m) about
# 1e-32 of the electrons', so that over any run here they stay put to about
# 1e-30 cells and carry no kinetic energy (the paper's immovable ions).
IMMOVABLE_MASS = 1.0e30


def x1_energy(n=64, ppc=2, steps=503, seed_offset=6, tile=(8, 4, 4)):
    """The energy test of Sec. 5: 3D n^3 periodic, ppc electrons per cell,
    v_th = 0.05c, dx = lambda_De (omega_pe = 1), omega_pe dt = 0.025, 503 steps
    (about two plasma periods); the same number of immovable ions at the
    electrons' initial positions, so that the field is zero at t = 0."""
    wl = thermal_plasma(f"X1 {n}^3 {ppc}ppc vth=0.05c, immovable ions at the electron positions", 3,
                        (n, n, n), ppc, 0.05, steps, SEED_BASE + seed_offset, tile=tile)
    e = wl.species[0]
    wl.species.append(SpeciesInit("immovable ions", 1.0, IMMOVABLE_MASS, e.weight, e.x.copy(), np.zeros_like(e.w)))
    wl.rho_bg = 0.0
    return wl


def x4_two_stream(n=64, ppc=2, steps=8000, seed_offset=7, tile=(8, 4, 4)):
    """The two-stream test of Sec. 5: X1's plasma with a uniform B_x such that
    the electron cyclotron frequency equals omega_pe (B_x = m c / |q| = c), and
    a directed momentum +2 v_th (= 0.1c in w = gamma v) along x added to half of
    the electrons and -2 v_th to the other half.  Returns the workload and B_x;
    the energy integral excludes the field energy of the initial B_x."""
    wl = x1_energy(n, ppc, steps, seed_offset, tile)
    wl.name = f"X4 two-stream {n}^3 {ppc}ppc, B_x with omega_Be = omega_pe, streams +-0.1c"
    e = wl.species[0]
    half = e.n // 2
    e.w[0][:half] += 2.0
    e.w[0][half:] -= 2.0
    return wl, wl.c


def x5_langmuir(n=64, steps=4000, seed_offset=8, tile=(8, 4, 4)):
    """The Langmuir test of Sec. 5 (Fig. 3, left): X4's setup with one electron
    per cell of twice the charge (still omega_pe = 1), B_x with
    omega_Be = omega_pe, and the directed momentum +2 v_th (0.1c) added to every
    electron, so that the electrons oscillate as a whole against the immovable
    ions.  Returns the workload and B_x."""
    wl = x1_energy(n, 1, steps, seed_offset, tile)
    wl.name = f"X5 Langmuir {n}^3 1ppc (charge x2), B_x with omega_Be = omega_pe, stream +0.1c"
    wl.species[0].w[0] += 2.0
    return wl, wl.c


def x6_gyration(n=64, steps=1600, tile=(8, 4, 4)):
    """The gyration test of Sec. 5 (Fig. 3, right): an electron and a positron at
    the centre of an n^3 box with opposite momenta w = +-0.5c along x, in a
    uniform B_z with omega_Be = 10 (B_z = 10 m c / |q|), so that
    omega_Be dt = 0.25; the charge is that of X5's particles.  Returns the
    workload and B_z."""
    vth = 1.0
    c = vth / 0.05
    dt = 0.5 / c
    V = 1.0
    W = V / (4.0 * math.pi)        # X5's macro charge: one particle per cell gives omega_pe = 1
    x = np.full((3, 1), n / 2.0 + 0.25)
    e = SpeciesInit("electron", -1.0, 1.0, W, x.copy(), np.array([[0.5 * c], [0.0], [0.0]]))
    p = SpeciesInit("positron", 1.0, 1.0, W, x.copy(), np.array([[-0.5 * c], [0.0], [0.0]]))
    wl = Workload(f"X6 gyration in B_z with omega_Be = 10, w = +-0.5c, {n}^3 box", 3, (n, n, n), (1.0, 1.0, 1.0),
                  dt, c, [e, p], 0.0, steps, tuple(tile), 10)
    return wl, 10.0 * c
