"""Closed forms the paper derives, used to pin the oracle.

TEST INFRASTRUCTURE ONLY (imported by tests and the benchmark's CPU leg).
Plain numpy, FP64; each function cites the passage it restates.
"""
from __future__ import annotations

import math

import numpy as np


def k_yee(k, dx):
    """Yee operator sin(k dx/2)/(dx/2) (Sec. 2.1, below Eq. (6))."""
    return np.sin(np.asarray(k) * dx / 2.0) / (dx / 2.0)


def k_stencil(c, k, dx):
    """[k] = sum_j C_j sin((2j-1) k dx/2)/(dx/2)  (Eq. (6), App. B Eq. (B.3))."""
    k = np.asarray(k, dtype=np.float64)
    out = np.zeros_like(k)
    for j, cj in enumerate(np.asarray(c, dtype=np.float64), start=1):
        out = out + cj * np.sin((2 * j - 1) * k * dx / 2.0)
    return out / (dx / 2.0)


def omega_t(omega, dt):
    """Leapfrog time operator [omega]_t = sin(omega dt/2)/(dt/2) (Sec. 2.1)."""
    return np.sin(np.asarray(omega) * dt / 2.0) / (dt / 2.0)


def k1t(k, dt):
    """[k]_{1,t} = sin(k dt/2)/(dt/2), the Xu operator (Sec. 3.1, Eq. (15))."""
    return np.sin(np.asarray(k) * dt / 2.0) / (dt / 2.0)


def omega_disc(kE, kB, dt):
    """omega of the vacuum dispersion relation Eq. (4): [omega]_t^2 = [k]_B1 [k]_E1."""
    return (2.0 / dt) * np.arcsin((dt / 2.0) * np.sqrt(np.asarray(kE) * np.asarray(kB)))


def bspline2(x):
    """Quadratic B-spline shape S (App. A, Table 1): 3/4 - x^2 for |x| <= 1/2,
    (3/2 - |x|)^2 / 2 for 1/2 <= |x| <= 3/2, zero beyond."""
    a = np.abs(np.asarray(x, dtype=np.float64))
    return np.where(a <= 0.5, 0.75 - a * a, np.where(a <= 1.5, 0.5 * (1.5 - a) ** 2, 0.0))


def lattice_shape_response(k, dx, offsets):
    """Grid-to-grid response of a uniform particle lattice to a field mode e^{ikx}
    gathered and deposited with the same shape S: the particles sit at the
    fractional cell offsets `offsets` in every cell, and the mode comes back
    multiplied by r(k) = mean_p |G(d_p)|^2, G(d) = sum_m S(m - d) e^{ik(m - d)dx}
    (exact for the lattice; r -> S~(k)^2 for a continuum of particles)."""
    m = np.arange(-3, 5)
    r = 0.0
    for d in np.asarray(offsets, dtype=np.float64):
        G = np.sum(bspline2(m - d) * np.exp(1j * k * (m - d) * dx))
        r += abs(G) ** 2
    return r / len(offsets)


def cold_plasma_omega(kE, kB, wp2, r, dt):
    """Numerical frequency of the transverse electromagnetic mode in a cold
    plasma with immobile ions (App. C, eps_33 = 0 with k along x1):
    [omega]_t^2 = [k]_E1 [k]_B1 + wp^2 s.  Here s is taken with its sum over the
    time aliases mu in closed form, sum_mu (-1)^mu [omega]_t/(omega + mu omega_g)
    = 1 (partial fractions of pi/sin), and the spatial aliases folded into the
    lattice response r, so s = r; the continuous limit is omega^2 = k^2 + wp^2."""
    return (2.0 / dt) * np.arcsin((dt / 2.0) * np.sqrt(np.asarray(kE) * np.asarray(kB) + wp2 * r))


def vphi(kE, kB, k1, dt):
    """Phase velocity along x1, Eq. (5)."""
    return omega_disc(kE, kB, dt) / np.asarray(k1)


def vphi_oblique(k0, theta, dt, dx2, eta):
    """Phase velocity at incidence angle theta, Eq. (16).  eta = 1 for the proposed
    operators of Eq. (15), eta = dx1/dt for Yee."""
    a = np.sin(eta * k0 * dt * np.cos(theta) / 2.0) / (eta * dt / 2.0)
    b = np.sin(k0 * dx2 * np.sin(theta) / 2.0) / (dx2 / 2.0)
    return (2.0 / (k0 * dt)) * np.arcsin((dt / 2.0) * np.sqrt(a * a + b * b))


def F_factor(kE, kB, dt):
    """Cancellation factor F = sqrt([k]_E1/[k]_B1) cos(omega dt/2), Eq. (10), with omega
    from the discrete dispersion relation (Sec. 3.1, Fig. 2(c))."""
    om = omega_disc(kE, kB, dt)
    return np.sqrt(np.asarray(kE) / np.asarray(kB)) * np.cos(om * dt / 2.0)


def kappa(kE1, kB1, kE2, kB2, theta, dt):
    """Oblique-incidence force factor kappa, Eq. (19) and the text after it."""
    s = kE1 * kB1 + kE2 * kB2
    om = (2.0 / dt) * np.arcsin((dt / 2.0) * np.sqrt(s))
    return (kE1 * np.cos(theta) + kE2 * np.sin(theta)) / np.sqrt(s) * np.cos(om * dt / 2.0)


def standard_coeffs(M: int) -> np.ndarray:
    """Coefficients of the standard staggered 2M-th order first derivative, the
    M = p/2 case of App. B (the constraint matrix alone fixes them).  Closed form
    C_j = (-1)^{j+1} ((2M-1)!!)^2 / ((2j-1)^2 (M-j)! (M+j-1)! 4^{M-1})."""
    df = 1
    for q in range(1, 2 * M, 2):
        df *= q
    out = []
    for j in range(1, M + 1):
        num = (-1) ** (j + 1) * df * df
        den = (2 * j - 1) ** 2 * math.factorial(M - j) * math.factorial(M + j - 1) * 4 ** (M - 1)
        out.append(num / den)
    return np.array(out)


def constraint_matrix(p: int, M: int) -> np.ndarray:
    """M_ij = (2j-1)^{2i-1}/(2i-1)!, i = 1..p/2, j = 1..M (App. B)."""
    return np.array([[(2 * j - 1) ** (2 * i - 1) / math.factorial(2 * i - 1)
                      for j in range(1, M + 1)] for i in range(1, p // 2 + 1)], dtype=np.float64)


def target_ops(kn, r, kind="proposed"):
    """Targets normalised to k_g1 = 2 pi/dx1 (App. B), r = dt/dx1, kn in [0, 1/2].
    proposed (Eq. (15)): T_E = tan(pi kn r)/(pi r), T_B = sin(2 pi kn r)/(2 pi r).
    xu (Sec. 3.1): T_E = T_B = sin(pi kn r)/(pi r).
    yee_tstagger (Sec. 4.1 solver 3): Yee dispersion with the time-stagger
    correction, T_E = T_Y/c, T_B = T_Y c, T_Y = sin(pi kn)/pi,
    c = cos(omega dt/2) = sqrt(1 - r^2 sin^2(pi kn))."""
    kn = np.asarray(kn, dtype=np.float64)
    if kind == "proposed":
        return np.tan(np.pi * kn * r) / (np.pi * r), np.sin(2 * np.pi * kn * r) / (2 * np.pi * r)
    if kind == "xu":
        t = np.sin(np.pi * kn * r) / (np.pi * r)
        return t, t
    if kind == "yee_tstagger":
        ty = np.sin(np.pi * kn) / np.pi
        c = np.sqrt(1.0 - (r * np.sin(np.pi * kn)) ** 2)
        return ty / c, ty * c
    raise ValueError(kind)


def cfl_lhs(cE, cB, dx, dt, nk=20001):
    """max over k of the left side of the CFL inequality Eq. (21):
    (dt/2)^2 [ (sum C^B s_1j)(sum C^E s_1j) + sum_{i>=2} s_{x_i,1}^2 ].
    The Yee terms reach (2/dx_i)^2 at the grid Nyquist.  Also returns the minimum
    of the x1 product (negative means imaginary omega for that mode)."""
    k = np.linspace(0.0, np.pi / dx[0], nk)
    prod = k_stencil(cB, k, dx[0]) * k_stencil(cE, k, dx[0])
    yee = sum((2.0 / d) ** 2 for d in dx[1:])
    return (dt / 2.0) ** 2 * (prod.max() + yee), prod.min()


def cfl_sufficient(cE, cB, dx):
    """Sufficient time-step bound Eq. (22)."""
    s = np.abs(cB).sum() * np.abs(cE).sum() / dx[0] ** 2 + sum(1.0 / d ** 2 for d in dx[1:])
    return 1.0 / math.sqrt(s)


def supergauss(kn, wk1=0.3, n=10):
    """Weight w(k1) = exp(-ln 2 (2 k1/w_k1)^n), App. B Eq. (B.10)."""
    return np.exp(-math.log(2.0) * (2.0 * np.asarray(kn) / wk1) ** n)


def laser_a(phi, a0, k0=1.0, phase=0.0, Lenv=20 * np.pi):
    """Vector potential of the sin^2 pulse used for the laser load."""
    phi = np.asarray(phi, dtype=np.float64)
    inside = (phi > 0) & (phi < Lenv)
    return np.where(inside, a0 * np.sin(np.pi * phi / Lenv) ** 2 * np.sin(k0 * phi + phase), 0.0)


def plane_wave_electron(phi, a0, k0=1.0, phase=0.0, Lenv=20 * np.pi):
    """Electron initially at rest in a plane wave a(phi), phi = x_front - x1 + t
    (Sec. 4.1, the canonical-momentum relation after Eq. (26)): u2 = a,
    u1 = a^2/2, gamma = 1 + a^2/2, hence gamma - u1 = 1.
    Returns (u1, u2, gamma) at phase phi."""
    a = laser_a(phi, a0, k0, phase, Lenv)
    return 0.5 * a * a, a, 1.0 + 0.5 * a * a


def plane_wave_drift(a0, k0=1.0, phase=0.0, Lenv=20 * np.pi, nq=200001):
    """Net displacement of an electron at rest after the whole pulse passed:
    dx1 = int a^2/2 dphi, dx2 = int a dphi (dx/dphi = u since dphi/dt = 1/gamma),
    by composite Simpson on nq points."""
    phi = np.linspace(0.0, Lenv, nq)
    a = laser_a(phi, a0, k0, phase, Lenv)
    h = phi[1] - phi[0]

    def simpson(y):
        return h / 3.0 * (y[0] + y[-1] + 4 * y[1:-1:2].sum() + 2 * y[2:-1:2].sum())

    return simpson(0.5 * a * a), simpson(a)
