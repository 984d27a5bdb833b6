"""FP64 CPU oracle for the ChCPIC step (arXiv:1101.0809) -- TEST INFRASTRUCTURE ONLY.

Python marshalling around ``chcpic_oracle.c``.  Only the test suite, the smoke
check and the benchmark's CPU-baseline leg may import this package.  It never
imports the CUDA library, and the CUDA library never imports it.

Array conventions: fields are float64 arrays of shape (nz, ny, nx), x fastest
(nz == 1 for 2D); particle positions and momenta are float64 arrays of shape
(3, n).  Positions are absolute normalized coordinates in [0, N).
"""
import ctypes as C
from dataclasses import dataclass

import numpy as np

from .build import build_oracle

_lib = None


class _Grid(C.Structure):
    _fields_ = [("dims", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double),
                ("dt", C.c_double), ("c", C.c_double), ("order2", C.c_int)]


class _Antenna(C.Structure):
    _fields_ = [("pol", C.c_int), ("i0", C.c_int), ("E0", C.c_double), ("omega", C.c_double),
                ("ramp", C.c_double)]


class _Species(C.Structure):
    _fields_ = [("q", C.c_double), ("m", C.c_double), ("weight", C.c_double),
                ("n", C.c_longlong), ("x", C.POINTER(C.c_double) * 3),
                ("w", C.POINTER(C.c_double) * 3)]


class _Diag(C.Structure):
    _fields_ = [("kinetic", C.c_double), ("field_E", C.c_double), ("field_B", C.c_double),
                ("half_step_corr", C.c_double), ("total", C.c_double),
                ("momentum", C.c_double * 3), ("charge", C.c_double)]


_P = C.POINTER(C.c_double)
_PP = _P * 3


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build_oracle())
        _lib.orc_deposit.restype = C.c_double
        _lib.orc_step.restype = C.c_double
        _lib.orc_step_antenna.restype = C.c_double
        _lib.orc_push_deposit.restype = C.c_double
        _lib.orc_sort_perm.restype = C.c_int
    return _lib


@dataclass
class Grid:
    """Grid geometry in the paper's normalized form (Sec. 2)."""
    dims: int
    n: tuple          # (nx, ny, nz); nz == 1 for dims == 2
    d: tuple = (1.0, 1.0, 1.0)
    dt: float = 0.5
    c: float = 1.0
    order2: int = 3   # 3: l_a = 1 1/2; 5: l_a = 2 1/2; 4: the uniform l = 2 comparison scheme (Eq. wrong1)

    def cstruct(self):
        nz = self.n[2] if self.dims == 3 else 1
        return _Grid(self.dims, self.n[0], self.n[1], nz, self.d[0], self.d[1], self.d[2],
                     self.dt, self.c, self.order2)

    @property
    def shape(self):
        return (self.n[2] if self.dims == 3 else 1, self.n[1], self.n[0])

    @property
    def volume(self):
        return self.d[0] * self.d[1] * (self.d[2] if self.dims == 3 else 1.0)

    def zeros(self):
        return [np.zeros(self.shape) for _ in range(3)]


@dataclass
class Species:
    """One particle species: physical q, m, macro weight, x and w as (3, n) float64."""
    q: float
    m: float
    weight: float
    x: np.ndarray
    w: np.ndarray

    def __post_init__(self):
        self.x = np.ascontiguousarray(self.x, dtype=np.float64)
        self.w = np.ascontiguousarray(self.w, dtype=np.float64)

    def copy(self):
        return Species(self.q, self.m, self.weight, self.x.copy(), self.w.copy())


def _ptr(a):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_P)


def _fields(F):
    for a in F:
        assert a.dtype == np.float64 and a.flags.c_contiguous
    return _PP(*[_ptr(a) for a in F])


def _species_array(species):
    arr = (_Species * len(species))()
    for s, sp in enumerate(species):
        arr[s].q, arr[s].m, arr[s].weight = sp.q, sp.m, sp.weight
        arr[s].n = sp.x.shape[1]
        for a in range(3):
            arr[s].x[a] = _ptr(sp.x[a]) if sp.x[a].flags.c_contiguous else None
            arr[s].w[a] = _ptr(sp.w[a])
    return arr


def form_factor(xp, order2=3):
    """Closed-form alternating-order values at one position (Sec. 4.5):
    (i, f, dF) with f[2], dF[3] for l_a = 1 1/2 (order2 = 3) and f[3], dF[4]
    for l_a = 2 1/2 (order2 = 5)."""
    i = C.c_longlong()
    if order2 == 5:
        f = (C.c_double * 3)()
        dF = (C.c_double * 4)()
        lib().orc_form_factor5(C.c_double(xp), C.byref(i), f, dF)
    else:
        f = (C.c_double * 2)()
        dF = (C.c_double * 3)()
        lib().orc_form_factor(C.c_double(xp), C.byref(i), f, dF)
    return i.value, np.array(f[:]), np.array(dF[:])


def gather(g: Grid, E, B, xp):
    """E(x_p), B(x_p) by the alpha/beta weights (Eqs. alphax, betax)."""
    Ep = (C.c_double * 3)()
    Bp = (C.c_double * 3)()
    x = (C.c_double * 3)(*[float(v) for v in xp])
    lib().orc_gather(C.byref(g.cstruct()), _fields(E), _fields(B), x, Ep, Bp)
    return np.array(Ep[:]), np.array(Bp[:])


def boris(w, Ep, Bp, qm, dt, c):
    """One momentum push of the Appendix; returns the new w."""
    wa = (C.c_double * 3)(*[float(v) for v in w])
    lib().orc_boris(wa, (C.c_double * 3)(*Ep), (C.c_double * 3)(*Bp),
                    C.c_double(qm), C.c_double(dt), C.c_double(c))
    return np.array(wa[:])


def move(g: Grid, w, x0):
    """u^{n+1/2} and the unwrapped x^{n+1} (Eq. coordscheme)."""
    x1 = (C.c_double * 3)()
    u = (C.c_double * 3)()
    lib().orc_move(C.byref(g.cstruct()), (C.c_double * 3)(*w), (C.c_double * 3)(*x0), x1, u)
    return np.array(x1[:]), np.array(u[:])


def deposit(g: Grid, x0, x1, u, qp, J):
    """Add one particle's virtual-path current (Eq. current) into J; returns the closure."""
    return lib().orc_deposit(C.byref(g.cstruct()), (C.c_double * 3)(*x0), (C.c_double * 3)(*x1),
                             (C.c_double * 3)(*u), C.c_double(qp), _fields(J))


def rho(g: Grid, x, qp, out=None):
    """Charge density of particles at x (3, n) with macro charge qp (Eq. rho)."""
    out = np.zeros(g.shape) if out is None else out
    x = np.ascontiguousarray(x, dtype=np.float64)
    lib().orc_rho(C.byref(g.cstruct()), C.c_longlong(x.shape[1]), _fields(list(x)),
                  C.c_double(qp), _ptr(out))
    return out


def yee_half_B(g: Grid, E, B):
    lib().orc_yee_half_B(C.byref(g.cstruct()), _fields(E), _fields(B))


def yee_E(g: Grid, B, J, E):
    lib().orc_yee_E(C.byref(g.cstruct()), _fields(B), _fields(J), _fields(E))


def push_deposit(g: Grid, E, B, J, sp: Species):
    """Particle part of one step for one species, in place; returns the worst closure."""
    arr = _species_array([sp])
    return lib().orc_push_deposit(C.byref(g.cstruct()), _fields(E), _fields(B), _fields(J),
                                  C.byref(arr[0]))


@dataclass
class Antenna:
    """Plane-wave antenna (one-way source on the plane x = i0): pol 1 = E_y/B_z,
    pol 2 = E_z/B_y; amplitude E0, angular frequency omega, sin^2 rise time ramp."""
    pol: int
    i0: int
    E0: float
    omega: float
    ramp: float = 0.0


def step(g: Grid, E, B, J, species, antenna: Antenna = None, n: int = 0):
    """One full time step of the Appendix, in place; returns the worst closure.
    With an antenna, n is the step's index on the antenna's clock."""
    arr = _species_array(species)
    if antenna is None:
        return lib().orc_step(C.byref(g.cstruct()), _fields(E), _fields(B), _fields(J),
                              C.c_int(len(species)), arr)
    a = _Antenna(antenna.pol, antenna.i0, antenna.E0, antenna.omega, antenna.ramp)
    return lib().orc_step_antenna(C.byref(g.cstruct()), C.byref(a), C.c_longlong(n), _fields(E), _fields(B),
                                  _fields(J), C.c_int(len(species)), arr)


def diagnostics(g: Grid, E, Bh, species, rho_bg=0.0):
    """FP64 diagnostics at time level n; returns (dict, rho, resid)."""
    arr = _species_array(species)
    r = np.zeros(g.shape)
    res = np.zeros(g.shape)
    d = _Diag()
    lib().orc_diagnostics(C.byref(g.cstruct()), _fields(E), _fields(Bh), C.c_int(len(species)),
                          arr, C.c_double(rho_bg), _ptr(r), _ptr(res), C.byref(d))
    out = {k: getattr(d, k) for k in ("kinetic", "field_E", "field_B", "half_step_corr",
                                       "total", "charge")}
    out["momentum"] = np.array(d.momentum[:])
    return out, r, res


def tile_keys(g: Grid, tile, x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    key = np.zeros(x.shape[1], dtype=np.int32)
    lib().orc_tile_keys(C.byref(g.cstruct()), (C.c_int * 3)(*tile), C.c_longlong(x.shape[1]),
                        _fields(list(x)), key.ctypes.data_as(C.POINTER(C.c_int)))
    return key


def sort_perm(key, nkeys):
    key = np.ascontiguousarray(key, dtype=np.int32)
    perm = np.zeros(key.shape[0], dtype=np.int64)
    rc = lib().orc_sort_perm(C.c_longlong(key.shape[0]), key.ctypes.data_as(C.POINTER(C.c_int)),
                             C.c_int(nkeys), perm.ctypes.data_as(C.POINTER(C.c_longlong)))
    if rc != 0:
        raise ValueError(f"orc_sort_perm failed ({rc})")
    return perm


def update_A(g: Grid, E, A):
    """A^{n+1/2} = A^{n-1/2} - c dt E^n (Eq. dadt), in place; call with E^n before step()."""
    lib().orc_update_A(C.byref(g.cstruct()), _fields(E), _fields(A))


def curl_A(g: Grid, A):
    """B = curl_h A on the staggered grid (Eq. viaA)."""
    B = g.zeros()
    lib().orc_curl_A(C.byref(g.cstruct()), _fields(A), _fields(B))
    return B


def generalized_momentum(g: Grid, A, species):
    """sum_p m_p w_p + (q_p/c) A(x_p - (dt/2) u_p), A at the E points (Sec. 4.2)."""
    arr = _species_array(species)
    P = (C.c_double * 3)()
    lib().orc_generalized_momentum(C.byref(g.cstruct()), _fields(A), C.c_int(len(species)), arr, P)
    return np.array(P[:])


def yee_half_B_adj(g: Grid, lamB, lamE):
    """lamE += (-(1/2) C_B)^T lamB (transpose of the B half step)."""
    lib().orc_yee_half_B_adj(C.byref(g.cstruct()), _fields(lamB), _fields(lamE))


def step_adj(g: Grid, E, Bh, species, lamE, lamB, lam_x, lam_w):
    """One step of the discrete adjoint at level n (state E^n, B^{n-1/2}, species
    at n).  lamE, lamB (fields) and lam_x, lam_w (one (3, n) float64 array per
    species) hold dL/d(state n+1) on entry and dL/d(state n) on return.
    Written for l_a = 1 1/2 only."""
    if g.order2 in (4, 5):
        raise NotImplementedError("the oracle's adjoint is written for l_a = 1 1/2")
    arr = _species_array(species)
    LX = (_P * len(species))(*[_ptr(a) for a in lam_x])
    LW = (_P * len(species))(*[_ptr(a) for a in lam_w])
    for a in list(lam_x) + list(lam_w):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    lib().orc_step_adj(C.byref(g.cstruct()), _fields(E), _fields(Bh), C.c_int(len(species)), arr,
                       _fields(lamE), _fields(lamB), LX, LW)

