"""Thin Python binding of libpic (``include/pic.h``): argument marshalling only.

Every step of the PIC path runs in the CUDA library; this module converts numpy
arrays (host) or CUDA torch tensors (device) into pointers and sizes.  Importing
it loads ``libpic.so``; a missing library raises immediately -- there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpic.so")

PIC_OK, PIC_ERR_ARG, PIC_ERR_CFL, PIC_ERR_OOM = 0, -1, -2, -3
PIC_ERR_CUDA, PIC_ERR_DEVICE_CHECK, PIC_ERR_TIMEOUT, PIC_ERR_STATE = -4, -5, -6, -7
PIC_FP64, PIC_MIXED, PIC_COMPENSATED = 0, 1, 2
PIC_SHAPE_QUADRATIC, PIC_BOUNDARY_PERIODIC = 2, 1   # pic_grid.shape / .boundary (0: the same)
PIC_BORIS, PIC_ANALYTIC, PIC_HC = 0, 1, 2
PUSHERS = {"boris": PIC_BORIS, "analytic": PIC_ANALYTIC, "hc": PIC_HC}
PIC_E1, PIC_E2, PIC_E3, PIC_B1, PIC_B2, PIC_B3 = range(6)
PIC_J1, PIC_J2, PIC_J3, PIC_BBAR1, PIC_BBAR2, PIC_BBAR3 = range(6, 12)
PIC_MAX_M = 32
PIC_NOALLOC_MAX_N1 = 65536
COMPONENTS = {"e1": 0, "e2": 1, "e3": 2, "b1": 3, "b2": 4, "b3": 5, "j1": 6, "j2": 7, "j3": 8,
              "bbar1": 9, "bbar2": 10, "bbar3": 11}


class PicError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("libpic status %d: %s" % (status, msg))
        self.status = status


class pic_grid(C.Structure):
    _fields_ = [("ndim", C.c_int), ("n", C.c_int * 3), ("dx", C.c_double * 3),
                ("precision", C.c_int), ("pusher", C.c_int), ("shape", C.c_int),
                ("boundary", C.c_int)]


class pic_coeffs(C.Structure):
    _fields_ = [("M", C.c_int), ("cE", C.POINTER(C.c_double)), ("cB", C.POINTER(C.c_double))]


class pic_laser(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("a0", "k0", "phase", "L_env", "x_front", "w0", "x2c", "x3c")]


class pic_info(C.Structure):
    _fields_ = [("sort_interval", C.c_int), ("tile", C.c_int * 3), ("guard", C.c_int * 3),
                ("n_particles", C.c_int64), ("steps_done", C.c_int64),
                ("last_stragglers", C.c_int64), ("correction_active", C.c_int),
                ("cfl_lhs", C.c_double), ("cfl_sufficient_dt", C.c_double),
                ("kernels_per_step", C.c_int)]


class pic_timing(C.Structure):
    _fields_ = [("ms_rebin", C.c_double), ("ms_particles", C.c_double),
                ("ms_stragglers", C.c_double), ("ms_correction", C.c_double),
                ("ms_fields", C.c_double), ("launches", C.c_int64), ("steps", C.c_int64)]


class pic_batch_desc(C.Structure):
    _fields_ = [("nruns", C.c_int), ("n1", C.POINTER(C.c_int)), ("n2", C.POINTER(C.c_int)),
                ("dx", C.c_double * 2), ("precision", C.c_int), ("pusher", C.c_int)]


class pic_batch_info(C.Structure):
    _fields_ = [("tile", C.c_int * 2), ("grid_blocks", C.c_int), ("blocks_per_sm", C.c_int),
                ("work_items", C.c_int), ("graph", C.c_int), ("total_cells", C.c_int64),
                ("max_steps", C.c_int64), ("cell_steps", C.c_int64), ("particle_steps", C.c_int64),
                ("last_run_ms", C.c_double), ("has_current", C.c_int),
                ("correction_active", C.c_int)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libpic.so not built: run `python -m paper_2004_03754_gb300.build` "
                          "(needs nvcc); there is no CPU fallback")
    L = C.CDLL(LIB_PATH)
    vp, dp = C.c_void_p, C.POINTER(C.c_double)  # noqa: F841
    sig = {
        "pic_init": ([C.POINTER(pic_grid), C.c_double, C.POINTER(pic_coeffs), vp, C.POINTER(vp)], C.c_int),
        "pic_load_laser": ([vp, C.POINTER(pic_laser)], C.c_int),
        "pic_load_field": ([vp, C.c_int, vp, C.c_int], C.c_int),
        "pic_load_particles": ([vp, C.c_int64, vp, vp, vp, C.c_double, C.c_int], C.c_int),
        "pic_step": ([vp, C.c_int64], C.c_int),
        "pic_read_field": ([vp, C.c_int, vp, C.c_int], C.c_int),
        "pic_read_particles": ([vp, vp, vp, vp, C.c_int], C.c_int),
        "pic_sync": ([vp], C.c_int),
        "pic_state_size": ([vp, C.POINTER(C.c_size_t)], C.c_int),
        "pic_laser_profile": ([C.c_int, C.c_double, C.c_double, C.POINTER(pic_coeffs),
                               C.POINTER(pic_laser), vp, vp], C.c_int),
        "pic_correction_taps": ([C.c_int, C.c_double, C.c_int, vp, vp, C.POINTER(C.c_int),
                                 C.POINTER(C.c_int)], C.c_int),
        "pic_save_state": ([vp, vp, C.c_size_t], C.c_int),
        "pic_load_state": ([vp, vp, C.c_size_t], C.c_int),
        "pic_get_info": ([vp, C.POINTER(pic_info)], C.c_int),
        "pic_set_sort_interval": ([vp, C.c_int], C.c_int),
        "pic_set_field_tile": ([vp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int], C.c_int),
        "pic_set_field_strip": ([vp, C.c_int, C.c_int, C.c_int, C.c_int], C.c_int),
        "pic_set_correction_path": ([vp, C.c_int], C.c_int),
        "pic_set_timing": ([vp, C.c_int], C.c_int),
        "pic_set_energy_gain": ([vp, C.c_int], C.c_int),
        "pic_analytic_push_vjp": ([C.c_double, C.c_double, vp, vp, vp, vp, vp, vp], C.c_int),
        "pic_set_moving_window": ([vp, C.c_int64], C.c_int),
        "pic_set_spectral": ([vp, C.c_int, vp, vp, C.c_double], C.c_int),
        "pic_get_window": ([vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64)], C.c_int),
        "pic_read_energy_gain": ([vp, vp, vp], C.c_int),
        "pic_get_timing": ([vp, C.POINTER(pic_timing)], C.c_int),
        "pic_laser_fields_noalloc": ([C.POINTER(pic_grid), C.c_double, C.POINTER(pic_coeffs),
                                      C.POINTER(pic_laser), vp, vp, vp], C.c_int),
        "pic_batch_init": ([C.POINTER(pic_batch_desc), C.c_double, C.POINTER(pic_coeffs), vp,
                            C.POINTER(vp)], C.c_int),
        "pic_batch_load_laser": ([vp, C.POINTER(pic_laser)], C.c_int),
        "pic_batch_load_particles": ([vp, C.POINTER(C.c_int64), vp, vp, vp, C.c_double], C.c_int),
        "pic_batch_set_steps": ([vp, C.POINTER(C.c_int64)], C.c_int),
        "pic_batch_autotune": ([vp, C.c_int], C.c_int),
        "pic_batch_set_strip": ([vp, C.c_int, C.c_int, C.c_int, C.c_int], C.c_int),
        "pic_batch_run": ([vp], C.c_int),
        "pic_batch_read_particles": ([vp, vp, vp, vp], C.c_int),
        "pic_batch_read_field": ([vp, C.c_int, C.c_int, vp], C.c_int),
        "pic_batch_get_info": ([vp, C.POINTER(pic_batch_info)], C.c_int),
        "pic_batch_set_barrier": ([vp, C.c_double, C.c_int], C.c_int),
        "pic_batch_last_error": ([vp], C.c_char_p),
        "pic_batch_destroy": ([vp], C.c_int),
        "pic_adjoint_laser_energy": ([vp, C.POINTER(pic_laser), C.c_int64, vp, vp, C.c_int64, C.c_int,
                                      dp, dp, dp], C.c_int),
        "pic_adjoint_laser_energy_w": ([vp, C.POINTER(pic_laser), C.c_int64, vp, vp, vp, C.c_int64,
                                        C.c_int, dp, dp, dp], C.c_int),
        "pic_adjoint_dispersion": ([vp, vp, vp, vp, C.c_int64, C.c_int, dp, dp, dp], C.c_int),
        "pic_last_error": ([vp], C.c_char_p),
        "pic_destroy": ([vp], C.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    return L


lib = _load()


def _check(ctx, st):
    if st != PIC_OK:
        msg = lib.pic_last_error(ctx)
        raise PicError(st, msg.decode() if msg else "")


def _ptr(a):
    """(pointer, on_device) for a numpy array or a CUDA torch tensor (float64, contiguous)."""
    if a is None:
        return None, 0
    if isinstance(a, np.ndarray):
        assert a.dtype == np.float64 and a.flags.c_contiguous, "need contiguous float64"
        return a.ctypes.data, 0
    # torch tensor
    assert a.is_contiguous() and str(a.dtype) == "torch.float64", "need contiguous float64"
    return a.data_ptr(), 1 if a.is_cuda else 0


# ---- C-ABI names ----------------------------------------------------------

def pic_init(grid: pic_grid, dt: float, cE, cB, stream=None):
    cE = np.ascontiguousarray(cE, dtype=np.float64)
    cB = np.ascontiguousarray(cB, dtype=np.float64)
    co = pic_coeffs(cE.size, cE.ctypes.data_as(C.POINTER(C.c_double)),
                    cB.ctypes.data_as(C.POINTER(C.c_double)))
    out = C.c_void_p()
    st = lib.pic_init(C.byref(grid), float(dt), C.byref(co), C.c_void_p(stream or 0), C.byref(out))
    _check(None, st)
    return out


def pic_load_laser(ctx, laser: pic_laser):
    _check(ctx, lib.pic_load_laser(ctx, C.byref(laser)))


def pic_load_field(ctx, comp: int, buf):
    p, dev = _ptr(buf)
    _check(ctx, lib.pic_load_field(ctx, comp, C.c_void_p(p), dev))


def pic_load_particles(ctx, n: int, x, u, w, qm: float):
    px, dx = _ptr(x)
    pu, _ = _ptr(u)
    pw, _ = _ptr(w)
    _check(ctx, lib.pic_load_particles(ctx, int(n), C.c_void_p(px), C.c_void_p(pu), C.c_void_p(pw),
                                       float(qm), dx))


def pic_step(ctx, nsteps: int):
    _check(ctx, lib.pic_step(ctx, int(nsteps)))


def pic_read_field(ctx, comp: int, buf):
    p, dev = _ptr(buf)
    _check(ctx, lib.pic_read_field(ctx, comp, C.c_void_p(p), dev))


def pic_read_particles(ctx, x, u, w):
    px, dev = _ptr(x)
    pu, _ = _ptr(u)
    pw, _ = _ptr(w)
    _check(ctx, lib.pic_read_particles(ctx, C.c_void_p(px), C.c_void_p(pu), C.c_void_p(pw), dev))


def pic_set_spectral(ctx, kE1, kB1, slope0: float = 1.0):
    """Spectral x1 field path with [k]_E1, [k]_B1 at the n1/2 + 1 non-negative x1
    wavenumbers; kE1 = None returns to the stencils."""
    if kE1 is None:
        _check(ctx, lib.pic_set_spectral(ctx, 0, None, None, 1.0))
        return
    kE1 = np.ascontiguousarray(kE1, dtype=np.float64)
    kB1 = np.ascontiguousarray(kB1, dtype=np.float64)
    _check(ctx, lib.pic_set_spectral(ctx, kE1.size, kE1.ctypes.data, kB1.ctypes.data, float(slope0)))


def pic_set_moving_window(ctx, start_step: int):
    _check(ctx, lib.pic_set_moving_window(ctx, int(start_step)))


def pic_get_window(ctx):
    """(origin, shifts) of the moving window."""
    o, s = C.c_int64(0), C.c_int64(0)
    _check(ctx, lib.pic_get_window(ctx, C.byref(o), C.byref(s)))
    return o.value, s.value


def pic_analytic_push_vjp(qm: float, dt: float, eb, u, lam):
    """Host-only analytic push and its VJP: (u_out, d_eb, d_u)."""
    eb = np.ascontiguousarray(eb, dtype=np.float64)
    u = np.ascontiguousarray(u, dtype=np.float64)
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    uo, deb, du = np.empty(3), np.empty(6), np.empty(3)
    st = lib.pic_analytic_push_vjp(float(qm), float(dt), eb.ctypes.data, u.ctypes.data,
                                   lam.ctypes.data, uo.ctypes.data, deb.ctypes.data, du.ctypes.data)
    if st != PIC_OK:
        raise PicError(st, "pic_analytic_push_vjp: bad arguments or no convergence")
    return uo, deb, du


def pic_set_energy_gain(ctx, on: bool):
    _check(ctx, lib.pic_set_energy_gain(ctx, 1 if on else 0))


def pic_read_energy_gain(ctx, n: int):
    """(W_LWFA, W_DLA) per particle in load order (Sec. 4.2)."""
    wl, wd = np.empty(int(n)), np.empty(int(n))
    _check(ctx, lib.pic_read_energy_gain(ctx, wl.ctypes.data, wd.ctypes.data))
    return wl, wd


def pic_laser_profile(n1: int, dx1: float, dt: float, cE, cB, laser: "pic_laser"):
    """Host-only x1 profiles (E2^0 at integer nodes, B3^{-1/2} at half nodes) of
    the laser load; returns (e2, b3)."""
    cE = np.ascontiguousarray(cE, dtype=np.float64)
    cB = np.ascontiguousarray(cB, dtype=np.float64)
    co = pic_coeffs(cE.size, cE.ctypes.data_as(C.POINTER(C.c_double)),
                    cB.ctypes.data_as(C.POINTER(C.c_double)))
    e2, b3 = np.empty(int(n1)), np.empty(int(n1))
    st = lib.pic_laser_profile(int(n1), float(dx1), float(dt), C.byref(co), C.byref(laser),
                               e2.ctypes.data, b3.ctypes.data)
    if st != PIC_OK:
        raise PicError(st, "pic_laser_profile: bad arguments")
    return e2, b3


def pic_correction_taps(n1: int, dx1: float, cB):
    """Taps of the x1 current correction on a periodic row of n1 cells (host
    only): returns (taps, lo) with J1'_i = sum_q taps[q] J1_{(i+lo+q) mod n1}."""
    cB = np.ascontiguousarray(cB, dtype=np.float64)
    taps = np.empty(max(int(n1), 1))
    lo, cnt = C.c_int(0), C.c_int(0)
    st = lib.pic_correction_taps(int(n1), float(dx1), cB.size, cB.ctypes.data, taps.ctypes.data,
                                 C.byref(lo), C.byref(cnt))
    if st != PIC_OK:
        raise PicError(st, "pic_correction_taps: bad arguments or singular [k]_B1")
    return taps[:cnt.value].copy(), lo.value


def pic_state_size(ctx) -> int:
    n = C.c_size_t(0)
    _check(ctx, lib.pic_state_size(ctx, C.byref(n)))
    return int(n.value)


def pic_save_state(ctx) -> np.ndarray:
    buf = np.empty(pic_state_size(ctx), dtype=np.uint8)
    _check(ctx, lib.pic_save_state(ctx, buf.ctypes.data, buf.nbytes))
    return buf


def pic_load_state(ctx, buf):
    buf = np.ascontiguousarray(buf, dtype=np.uint8)
    _check(ctx, lib.pic_load_state(ctx, buf.ctypes.data, buf.nbytes))


def pic_sync(ctx):
    _check(ctx, lib.pic_sync(ctx))


def pic_get_info(ctx) -> pic_info:
    info = pic_info()
    _check(ctx, lib.pic_get_info(ctx, C.byref(info)))
    return info


def pic_set_sort_interval(ctx, k: int):
    _check(ctx, lib.pic_set_sort_interval(ctx, int(k)))


def pic_set_field_tile(ctx, t1: int, t2: int, t3: int = 1, threads: int = 256, staging: int = 0):
    _check(ctx, lib.pic_set_field_tile(ctx, int(t1), int(t2), int(t3), int(threads), int(staging)))


def pic_set_field_strip(ctx, width: int, rows: int, warps: int = 4, stages: int = 4):
    _check(ctx, lib.pic_set_field_strip(ctx, int(width), int(rows), int(warps), int(stages)))


def pic_set_correction_path(ctx, path: int):
    _check(ctx, lib.pic_set_correction_path(ctx, int(path)))


def pic_set_timing(ctx, enable: bool):
    _check(ctx, lib.pic_set_timing(ctx, 1 if enable else 0))


def pic_get_timing(ctx) -> pic_timing:
    t = pic_timing()
    _check(ctx, lib.pic_get_timing(ctx, C.byref(t)))
    return t


def pic_laser_fields_noalloc(grid: pic_grid, dt: float, cE, cB, laser: pic_laser, e2, b3,
                             stream=None) -> int:
    """Allocation-free laser load into caller-owned FP64 device arrays e2, b3
    (CUDA tensors); returns the pic_status (0 = ok) instead of raising."""
    cE = np.ascontiguousarray(cE, dtype=np.float64)
    cB = np.ascontiguousarray(cB, dtype=np.float64)
    co = pic_coeffs(cE.size, cE.ctypes.data_as(C.POINTER(C.c_double)),
                    cB.ctypes.data_as(C.POINTER(C.c_double)))
    pe, _ = _ptr(e2)
    pb, _ = _ptr(b3)
    return lib.pic_laser_fields_noalloc(C.byref(grid), float(dt), C.byref(co), C.byref(laser),
                                        C.c_void_p(pe), C.c_void_p(pb), C.c_void_p(stream or 0))


def pic_adjoint_laser_energy(ctx, laser: pic_laser, x, u, nsteps: int, checkpoint_every: int = 100):
    """(J, dJ/da0, dJ/dphase) for J = mean(gamma - 1) of the test particles after nsteps.
    x: (ndim*n,) and u: (3*n,) host float64."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    u = np.ascontiguousarray(u, dtype=np.float64)
    n = u.size // 3
    J, ga, gp = C.c_double(), C.c_double(), C.c_double()
    _check(ctx, lib.pic_adjoint_laser_energy(ctx, C.byref(laser), n, C.c_void_p(x.ctypes.data),
                                             C.c_void_p(u.ctypes.data), int(nsteps),
                                             int(checkpoint_every), C.byref(J), C.byref(ga),
                                             C.byref(gp)))
    return J.value, ga.value, gp.value


def pic_adjoint_laser_energy_w(ctx, laser: pic_laser, x, u, w, nsteps: int,
                               checkpoint_every: int = 100):
    """(J, dJ/da0, dJ/dphase) for J = mean(gamma - 1) after nsteps of particles with weights w
    (those of non-zero weight deposit current).  x: (ndim*n,), u: (3*n,), w: (n,) host float64."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    u = np.ascontiguousarray(u, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    n = w.size
    if u.size != 3 * n:
        raise ValueError("u must hold 3*n values")
    J, ga, gp = C.c_double(), C.c_double(), C.c_double()
    _check(ctx, lib.pic_adjoint_laser_energy_w(ctx, C.byref(laser), n, C.c_void_p(x.ctypes.data),
                                               C.c_void_p(u.ctypes.data), C.c_void_p(w.ctypes.data),
                                               int(nsteps), int(checkpoint_every), C.byref(J),
                                               C.byref(ga), C.byref(gp)))
    return J.value, ga.value, gp.value


def pic_adjoint_dispersion(ctx, e2_0, b3_0, target, nsteps: int, M: int, checkpoint_every: int = 100):
    """(J, dJ/dC^E, dJ/dC^B) for J = 1/2 |E2^N - target|^2 (host float64 arrays)."""
    a = [np.ascontiguousarray(v, dtype=np.float64) for v in (e2_0, b3_0, target)]
    J = C.c_double()
    gE, gB = np.zeros(M), np.zeros(M)
    _check(ctx, lib.pic_adjoint_dispersion(ctx, *[C.c_void_p(v.ctypes.data) for v in a], int(nsteps),
                                           int(checkpoint_every), C.byref(J),
                                           gE.ctypes.data_as(C.POINTER(C.c_double)),
                                           gB.ctypes.data_as(C.POINTER(C.c_double))))
    return J.value, gE, gB


def pic_last_error(ctx=None) -> str:
    m = lib.pic_last_error(ctx)
    return m.decode() if m else ""


def pic_destroy(ctx):
    _check(None, lib.pic_destroy(ctx))


# ---- convenience wrapper --------------------------------------------------

class Simulation:
    """One libpic context.  n, dx: per-axis cells and sizes (2 or 3 entries)."""

    def __init__(self, n, dx, dt, cE, cB, precision="fp64", pusher="boris", stream=None):
        n = tuple(int(v) for v in n)
        self.ndim = len(n)
        g = pic_grid()
        g.ndim = self.ndim
        for d in range(3):
            g.n[d] = n[d] if d < self.ndim else 1
            g.dx[d] = float(dx[d]) if d < self.ndim else 1.0
        g.precision = {"fp64": PIC_FP64, "mixed": PIC_MIXED, "compensated": PIC_COMPENSATED}[precision]
        g.pusher = PUSHERS[pusher]
        self.n, self.dx, self.dt = n, tuple(float(v) for v in dx), float(dt)
        self.ctx = pic_init(g, dt, cE, cB, stream)
        self.np = 0
        self._window = False

    @property
    def shape(self):
        return tuple(reversed(self.n))

    def close(self):
        if self.ctx:
            pic_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load_laser(self, a0, k0=1.0, phase=0.0, L_env=20 * np.pi, x_front=0.0, w0=0.0,
                   x2c=None, x3c=None):
        L = [a * b for a, b in zip(self.n, self.dx)]
        las = pic_laser(a0, k0, phase, L_env, x_front, w0,
                        L[1] / 2 if x2c is None else x2c,
                        (L[2] / 2 if self.ndim == 3 else 0.0) if x3c is None else x3c)
        pic_load_laser(self.ctx, las)

    def load_field(self, name, arr):
        pic_load_field(self.ctx, COMPONENTS[name], np.ascontiguousarray(arr, dtype=np.float64)
                       if isinstance(arr, np.ndarray) else arr)

    def read_field(self, name, out=None):
        if out is None:
            out = np.empty(self.shape, dtype=np.float64)
        pic_read_field(self.ctx, COMPONENTS[name], out)
        return out

    def load_particles(self, x, u, w, qm=-1.0):
        """x: list of ndim arrays, u: list of 3 arrays, w: array (host numpy)."""
        w = np.ascontiguousarray(w, dtype=np.float64)
        n = w.size
        X = np.ascontiguousarray(np.concatenate([np.asarray(v, np.float64) for v in x]) if n else np.zeros(0))
        U = np.ascontiguousarray(np.concatenate([np.asarray(v, np.float64) for v in u]) if n else np.zeros(0))
        pic_load_particles(self.ctx, n, X, U, w, qm)
        self.np = n

    def read_particles(self):
        n = self.np
        X = np.empty(self.ndim * n)
        U = np.empty(3 * n)
        W = np.empty(n)
        if n:
            pic_read_particles(self.ctx, X, U, W)
        return [X[d * n:(d + 1) * n] for d in range(self.ndim)], [U[c * n:(c + 1) * n] for c in range(3)], W

    def step(self, nsteps=1):
        pic_step(self.ctx, nsteps)
        if self._window:   # a moving window removes particles
            self.np = int(pic_get_info(self.ctx).n_particles)

    def set_spectral(self, kE1, kB1, slope0=1.0):
        """Spectral x1 derivatives with the given k-space operators (FP64)."""
        pic_set_spectral(self.ctx, kE1, kB1, slope0)

    def set_moving_window(self, start_step=0):
        """Move a window along x1 at c from start_step on (negative: off)."""
        pic_set_moving_window(self.ctx, start_step)
        self._window = start_step >= 0

    def window(self):
        return pic_get_window(self.ctx)

    def enable_energy_gain(self, on=True):
        """Keep the per-particle energy-gain integrals W_LWFA, W_DLA (Sec. 4.2)."""
        pic_set_energy_gain(self.ctx, on)

    def read_energy_gain(self):
        if not self.np:
            return np.zeros(0), np.zeros(0)
        return pic_read_energy_gain(self.ctx, self.np)

    def set_field_tile(self, t1, t2, t3=1, threads=256, staging=0):
        """Field-kernel tile (x1 fastest) and CTA size; staging 1 forces plain loads."""
        pic_set_field_tile(self.ctx, t1, t2, t3, threads, staging)

    def set_field_strip(self, width, rows, warps=4, stages=4):
        """2D row streaming per warp: strip width, rows per item, warps per CTA, ring depth."""
        pic_set_field_strip(self.ctx, width, rows, warps, stages)

    def set_correction_path(self, path: int):
        """x1 current-correction form: 0 auto, 1 rows in place, 2 segments, 3 global."""
        pic_set_correction_path(self.ctx, path)

    def save_state(self) -> np.ndarray:
        """Checkpoint (fields, particles, step count) as a host byte array."""
        return pic_save_state(self.ctx)

    def load_state(self, buf):
        """Resume from a checkpoint saved by a Simulation of the same configuration."""
        pic_load_state(self.ctx, buf)
        self.np = int(pic_get_info(self.ctx).n_particles)

    def sync(self):
        pic_sync(self.ctx)

    def info(self):
        return pic_get_info(self.ctx)


# ---- ensembles ------------------------------------------------------------

def _bcheck(b, st):
    if st != PIC_OK:
        m = lib.pic_batch_last_error(b) if b else b""
        raise PicError(st, m.decode() if m else "")


def pic_batch_init(desc: pic_batch_desc, dt: float, cE, cB, stream=None):
    cE = np.ascontiguousarray(cE, dtype=np.float64)
    cB = np.ascontiguousarray(cB, dtype=np.float64)
    co = pic_coeffs(cE.size, cE.ctypes.data_as(C.POINTER(C.c_double)),
                    cB.ctypes.data_as(C.POINTER(C.c_double)))
    out = C.c_void_p()
    _bcheck(None, lib.pic_batch_init(C.byref(desc), float(dt), C.byref(co), C.c_void_p(stream or 0),
                                     C.byref(out)))
    return out


def pic_batch_load_laser(b, lasers):
    arr = (pic_laser * len(lasers))(*lasers)
    _bcheck(b, lib.pic_batch_load_laser(b, arr))


def pic_batch_load_particles(b, counts, x, u, w, qm):
    cnt = np.ascontiguousarray(counts, dtype=np.int64)
    _bcheck(b, lib.pic_batch_load_particles(b, cnt.ctypes.data_as(C.POINTER(C.c_int64)),
                                            C.c_void_p(_ptr(x)[0]), C.c_void_p(_ptr(u)[0]),
                                            C.c_void_p(_ptr(w)[0]), float(qm)))


def pic_batch_set_steps(b, nsteps):
    ns = np.ascontiguousarray(nsteps, dtype=np.int64)
    _bcheck(b, lib.pic_batch_set_steps(b, ns.ctypes.data_as(C.POINTER(C.c_int64))))


def pic_batch_autotune(b, trial_steps):
    _bcheck(b, lib.pic_batch_autotune(b, int(trial_steps)))


def pic_batch_set_strip(b, width, rows, stages, warps):
    _bcheck(b, lib.pic_batch_set_strip(b, int(width), int(rows), int(stages), int(warps)))


def pic_batch_run(b):
    _bcheck(b, lib.pic_batch_run(b))


def pic_batch_read_particles(b, x, u, w):
    _bcheck(b, lib.pic_batch_read_particles(b, C.c_void_p(_ptr(x)[0]), C.c_void_p(_ptr(u)[0]),
                                            C.c_void_p(_ptr(w)[0])))


def pic_batch_read_field(b, run, comp, buf):
    _bcheck(b, lib.pic_batch_read_field(b, int(run), int(comp), C.c_void_p(_ptr(buf)[0])))


def pic_batch_get_info(b) -> pic_batch_info:
    info = pic_batch_info()
    _bcheck(b, lib.pic_batch_get_info(b, C.byref(info)))
    return info


def pic_batch_set_barrier(b, timeout_s, impossible=False):
    _bcheck(b, lib.pic_batch_set_barrier(b, float(timeout_s), 1 if impossible else 0))


def pic_batch_destroy(b):
    _bcheck(None, lib.pic_batch_destroy(b))


class Ensemble:
    """Independent 2D runs advanced by one persistent kernel (libpic ensembles)."""

    def __init__(self, n1, n2, dx, dt, cE, cB, precision="mixed", pusher="analytic", stream=None):
        self.n1 = np.ascontiguousarray(n1, dtype=np.int32)
        self.n2 = np.ascontiguousarray(n2, dtype=np.int32)
        d = pic_batch_desc()
        d.nruns = self.n1.size
        d.n1 = self.n1.ctypes.data_as(C.POINTER(C.c_int))
        d.n2 = self.n2.ctypes.data_as(C.POINTER(C.c_int))
        d.dx[0], d.dx[1] = float(dx[0]), float(dx[1])
        d.precision = {"fp64": PIC_FP64, "mixed": PIC_MIXED, "compensated": PIC_COMPENSATED}[precision]
        d.pusher = PUSHERS[pusher]
        self.dx, self.dt = tuple(dx), float(dt)
        self.b = pic_batch_init(d, dt, cE, cB, stream)
        self.counts = np.zeros(self.n1.size, dtype=np.int64)

    @property
    def nruns(self):
        return int(self.n1.size)

    def close(self):
        if self.b:
            pic_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load_lasers(self, lasers):
        pic_batch_load_laser(self.b, lasers)

    def load_particles(self, counts, x, u, w, qm=-1.0):
        """counts per run; x: [x1, x2] concatenated over runs; u: [u1, u2, u3]; w."""
        self.counts = np.ascontiguousarray(counts, dtype=np.int64)
        X = np.ascontiguousarray(np.concatenate([np.asarray(v, np.float64) for v in x]))
        U = np.ascontiguousarray(np.concatenate([np.asarray(v, np.float64) for v in u]))
        pic_batch_load_particles(self.b, self.counts, X, U, np.ascontiguousarray(w, np.float64), qm)

    def set_steps(self, nsteps):
        pic_batch_set_steps(self.b, nsteps)

    def autotune(self, trial_steps=8):
        pic_batch_autotune(self.b, trial_steps)

    def set_strip(self, width, rows, stages, warps):
        """Field strip shape of the persistent kernel (see pic_batch_set_strip)."""
        pic_batch_set_strip(self.b, width, rows, stages, warps)

    def run(self):
        pic_batch_run(self.b)

    def read_particles(self):
        n = int(self.counts.sum())
        X, U, W = np.empty(2 * n), np.empty(3 * n), np.empty(n)
        if n:
            pic_batch_read_particles(self.b, X, U, W)
        return [X[:n], X[n:]], [U[:n], U[n:2 * n], U[2 * n:]], W

    def read_field(self, run, name):
        out = np.empty((int(self.n2[run]), int(self.n1[run])))
        pic_batch_read_field(self.b, run, COMPONENTS[name], out)
        return out

    def info(self):
        return pic_batch_get_info(self.b)
