"""ctypes front end of the plain FP64 CPU oracle (``pic_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``; never by the product package.

The oracle's leapfrog state is (E^n, B^{n-1/2}, x^n, u^{n-1/2}), the paper's
Eq. (1) / Eq. (7) scheme with the time-centred B formed by averaging.
Arrays are float64, C-contiguous, shaped (n3, n2, n1) in 3D and (n2, n1) in 2D
(x1 fastest).  Positions are physical (normalised to 1/k_n), periodic.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pic_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

_dp = C.POINTER(C.c_double)


_LIB_OMP = os.path.join(_HERE, "liboracle_omp.so")


def build(force: bool = False, openmp: bool = False) -> str:
    """Compile ``liboracle.so`` with gcc (no FMA contraction, portable flags);
    openmp: the same source with OpenMP (``liboracle_omp.so``), used only as the
    multi-core CPU baseline (its current sums run in another order)."""
    out = _LIB_OMP if openmp else _LIB
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
        tmp = out + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                               "-std=c11", "-D_DEFAULT_SOURCE"] + (["-fopenmp"] if openmp else [])
                              + ["-o", tmp, _SRC, "-lm"])
        os.replace(tmp, out)
    return out


class _Grid(C.Structure):
    _fields_ = [("ndim", C.c_int), ("n1", C.c_int), ("n2", C.c_int), ("n3", C.c_int),
                ("dx1", C.c_double), ("dx2", C.c_double), ("dx3", C.c_double),
                ("dt", C.c_double), ("M", C.c_int), ("cE", _dp), ("cB", _dp)]


class _Fields(C.Structure):
    _fields_ = [(n, _dp) for n in ("e1", "e2", "e3", "b1", "b2", "b3", "j1", "j2", "j3")]


_lib = None
_libs = {}


def use_openmp(on: bool):
    """Route the calls below to the OpenMP build (CPU baseline timing) or back."""
    global _lib
    key = bool(on)
    if key not in _libs:
        _libs[key] = _setup(C.CDLL(build(openmp=key)))
    _lib = _libs[key]


def lib():
    global _lib
    if _lib is None:
        use_openmp(False)
    return _lib


def _setup(L):
    """Declare the C signatures on a loaded oracle library."""
    G, F = C.POINTER(_Grid), C.POINTER(_Fields)
    L.orc_faraday.argtypes = [G, F, C.c_double]
    L.orc_ampere.argtypes = [G, F, C.c_double]
    L.orc_kspace.argtypes = [C.c_int, _dp, C.c_double, C.c_double]
    L.orc_kspace.restype = C.c_double
    L.orc_correct_j1.argtypes = [G, _dp]
    L.orc_correct_j1.restype = C.c_int
    L.orc_div_e.argtypes = [G, F, _dp]
    L.orc_div_yee.argtypes = [G, _dp, _dp, _dp, _dp]
    L.orc_gather.argtypes = [G] + [_dp] * 6 + [_dp, _dp]
    L.orc_boris.argtypes = [C.c_double, C.c_double, _dp, _dp]
    L.orc_hc.argtypes = [C.c_double, C.c_double, _dp, _dp]
    L.orc_analytic.argtypes = [C.c_double, C.c_double, _dp, _dp]
    L.orc_analytic.restype = C.c_int
    L.orc_deposit.argtypes = [G, F, C.c_double, _dp, _dp, C.c_double]
    L.orc_deposit.restype = C.c_int
    L.orc_rho.argtypes = [G, C.c_int64, _dp, _dp, _dp, _dp, _dp]
    L.orc_step.argtypes = [G, F, C.c_int64] + [_dp] * 7 + [C.c_double, C.c_int]
    L.orc_step.restype = C.c_int
    L.orc_step_gain.argtypes = [G, F, C.c_int64] + [_dp] * 7 + [C.c_double, C.c_int, _dp, _dp]
    L.orc_step_gain.restype = C.c_int
    L.orc_bbar.argtypes = [G, F, _dp, _dp, _dp]
    L.orc_laser_profile.argtypes = [G] + [C.c_double] * 5 + [_dp, _dp]
    L.orc_laser_load.argtypes = [G, F] + [C.c_double] * 8
    L.orc_gather_centred.argtypes = [G, F, _dp, _dp]
    L.orc_point_update.argtypes = [G, F, C.c_int, C.c_int, C.c_int, _dp]
    return L


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


class Grid:
    """Grid, time step and x1 stencil coefficients (C^E, C^B of App. B)."""

    def __init__(self, n, dx, dt, cE, cB):
        n = tuple(int(v) for v in n)
        self.ndim = len(n)
        assert self.ndim in (2, 3)
        self.n = n
        self.dx = tuple(float(v) for v in dx)
        self.dt = float(dt)
        self.cE = np.ascontiguousarray(cE, dtype=np.float64)
        self.cB = np.ascontiguousarray(cB, dtype=np.float64)
        assert self.cE.shape == self.cB.shape and self.cE.ndim == 1
        self.M = self.cE.size
        n3 = n[2] if self.ndim == 3 else 1
        dx3 = self.dx[2] if self.ndim == 3 else 1.0
        self._g = _Grid(self.ndim, n[0], n[1], n3, self.dx[0], self.dx[1], dx3, self.dt,
                        self.M, _p(self.cE), _p(self.cB))

    @property
    def shape(self):
        return tuple(reversed(self.n))

    @property
    def length(self):
        return tuple(a * b for a, b in zip(self.n, self.dx))

    def zeros(self):
        return np.zeros(self.shape, dtype=np.float64)

    def ref(self):
        return C.byref(self._g)


class Fields:
    """E, B, J arrays of the oracle.  ``b*`` holds B^{n-1/2}."""

    NAMES = ("e1", "e2", "e3", "b1", "b2", "b3", "j1", "j2", "j3")

    def __init__(self, grid: Grid):
        self.grid = grid
        for nm in self.NAMES:
            setattr(self, nm, grid.zeros())
        self._sync()

    def _sync(self):
        self._f = _Fields(*[_p(getattr(self, nm)) for nm in self.NAMES])

    def ref(self):
        self._sync()
        return C.byref(self._f)

    def copy(self):
        o = Fields(self.grid)
        for nm in self.NAMES:
            getattr(o, nm)[...] = getattr(self, nm)
        return o


class Particles:
    """SoA particle arrays: positions x (ndim arrays), momenta u = gamma*beta
    (3 arrays), deposit weight w (0 for a test particle), charge/mass qm."""

    def __init__(self, x, u, w, qm=-1.0):
        self.x = [np.ascontiguousarray(v, dtype=np.float64).copy() for v in x]
        self.u = [np.ascontiguousarray(v, dtype=np.float64).copy() for v in u]
        self.w = np.ascontiguousarray(w, dtype=np.float64).copy()
        self.qm = float(qm)

    @property
    def n(self):
        return self.w.size

    def copy(self):
        return Particles(self.x, self.u, self.w, self.qm)


def faraday(grid: Grid, F: Fields, h: float):
    lib().orc_faraday(grid.ref(), F.ref(), h)


def ampere(grid: Grid, F: Fields, h: float):
    lib().orc_ampere(grid.ref(), F.ref(), h)


def kspace(c, k1, dx1):
    c = np.ascontiguousarray(c, dtype=np.float64)
    return lib().orc_kspace(c.size, _p(c), float(k1), float(dx1))


def correct_j1(grid: Grid, j1: np.ndarray) -> int:
    return lib().orc_correct_j1(grid.ref(), _p(j1))


def div_e(grid: Grid, F: Fields) -> np.ndarray:
    out = grid.zeros()
    lib().orc_div_e(grid.ref(), F.ref(), _p(out))
    return out


def div_yee(grid: Grid, f1, f2, f3) -> np.ndarray:
    out = grid.zeros()
    lib().orc_div_yee(grid.ref(), _p(f1), _p(f2), _p(f3), _p(out))
    return out


def gather(grid: Grid, e, b, xp) -> np.ndarray:
    """Interpolate (E1,E2,E3,B1,B2,B3) at one position xp (ndim values)."""
    x = np.zeros(3)
    x[: grid.ndim] = xp
    out = np.zeros(6)
    lib().orc_gather(grid.ref(), *[_p(a) for a in (*e, *b)], _p(x), _p(out))
    return out


def boris(qm, dt, EB, u) -> np.ndarray:
    u = np.array(u, dtype=np.float64)
    EB = np.ascontiguousarray(EB, dtype=np.float64)
    lib().orc_boris(float(qm), float(dt), _p(EB), _p(u))
    return u


def hc(qm, dt, EB, u) -> np.ndarray:
    """Higuera-Cary push of u over dt (pic_oracle.c orc_hc)."""
    u = np.array(u, dtype=np.float64)
    EB = np.ascontiguousarray(EB, dtype=np.float64)
    lib().orc_hc(float(qm), float(dt), _p(EB), _p(u))
    return u


def analytic(qm, dt, EB, u):
    """Returns (u_new, iterations); iterations < 0 means no convergence."""
    u = np.array(u, dtype=np.float64)
    EB = np.ascontiguousarray(EB, dtype=np.float64)
    it = lib().orc_analytic(float(qm), float(dt), _p(EB), _p(u))
    return u, it


def deposit(grid: Grid, F: Fields, w, xo, xn, v3) -> int:
    a = np.zeros(3); a[: grid.ndim] = xo
    b = np.zeros(3); b[: grid.ndim] = xn
    return lib().orc_deposit(grid.ref(), F.ref(), float(w), _p(a), _p(b), float(v3))


def rho(grid: Grid, P: Particles) -> np.ndarray:
    out = grid.zeros()
    x3 = P.x[2] if grid.ndim == 3 else P.x[0]
    lib().orc_rho(grid.ref(), P.n, _p(P.x[0]), _p(P.x[1]), _p(x3), _p(P.w), _p(out))
    return out


PUSHERS = {"boris": 0, "analytic": 1, "hc": 2}


def step(grid: Grid, F: Fields, P: Particles | None, pusher: str = "boris", nsteps: int = 1):
    """Advance the oracle state by ``nsteps`` full steps (Sec. 2-3 scheme)."""
    if P is None:
        P = Particles([np.zeros(0)] * grid.ndim, [np.zeros(0)] * 3, np.zeros(0))
    x3 = P.x[2] if grid.ndim == 3 else P.x[0]
    for _ in range(nsteps):
        st = lib().orc_step(grid.ref(), F.ref(), P.n, _p(P.x[0]), _p(P.x[1]), _p(x3),
                            _p(P.u[0]), _p(P.u[1]), _p(P.u[2]), _p(P.w), P.qm,
                            PUSHERS[pusher])
        if st != 0:
            raise RuntimeError("oracle step failed with status %d" % st)
    return F, P


def step_gain(grid: Grid, F: Fields, P: Particles, wl, wd, pusher: str = "boris", nsteps: int = 1):
    """As step, also accumulating each particle's energy-gain integrals of
    Sec. 4.2 into wl (W_LWFA, longitudinal field) and wd (W_DLA, transverse)."""
    x3 = P.x[2] if grid.ndim == 3 else P.x[0]
    for _ in range(nsteps):
        st = lib().orc_step_gain(grid.ref(), F.ref(), P.n, _p(P.x[0]), _p(P.x[1]), _p(x3),
                                 _p(P.u[0]), _p(P.u[1]), _p(P.u[2]), _p(P.w), P.qm,
                                 PUSHERS[pusher], _p(wl), _p(wd))
        if st != 0:
            raise RuntimeError("oracle step failed with status %d" % st)
    return F, P


def bbar(grid: Grid, F: Fields):
    """Time-centred B^n = (B^{n-1/2} + B^{n+1/2})/2 of the current state."""
    out = [grid.zeros() for _ in range(3)]
    lib().orc_bbar(grid.ref(), F.ref(), *[_p(a) for a in out])
    return out


def laser_profile(grid: Grid, a0, k0, phase, Lenv, x_front):
    e = np.zeros(grid.n[0]); b = np.zeros(grid.n[0])
    lib().orc_laser_profile(grid.ref(), a0, k0, phase, Lenv, x_front, _p(e), _p(b))
    return e, b


def laser_load(grid: Grid, F: Fields, a0, k0=1.0, phase=0.0, Lenv=20 * np.pi, x_front=0.0,
               w0=0.0, x2c=None, x3c=None):
    """E2^0 and B3^{-1/2} of a forward-moving, x2-polarised pulse (E1=E3=B1=B2=0)."""
    L = grid.length
    x2c = L[1] / 2 if x2c is None else x2c
    x3c = (L[2] / 2 if grid.ndim == 3 else 0.0) if x3c is None else x3c
    lib().orc_laser_load(grid.ref(), F.ref(), a0, k0, phase, Lenv, x_front, w0, x2c, x3c)


def gather_centred(grid: Grid, F: Fields, xp) -> np.ndarray:
    """Gather E^n and the time-centred B^n at xp, forming B^n only at the nodes used."""
    x = np.zeros(3)
    x[: grid.ndim] = xp
    out = np.zeros(6)
    lib().orc_gather_centred(grid.ref(), F.ref(), _p(x), _p(out))
    return out


def point_update(grid: Grid, F: Fields, i, j, k=0) -> np.ndarray:
    """E^{n+1} and B^{n+1/2} at cell (i, j, k) for J = 0, evaluated locally."""
    out = np.zeros(6)
    lib().orc_point_update(grid.ref(), F.ref(), int(i), int(j), int(k), _p(out))
    return out
