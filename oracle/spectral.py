"""Spectral (FFT) field step with prescribed x1 operators, 2D and 3D.

TEST INFRASTRUCTURE ONLY (imported by tests).  Plain numpy, FP64.

The paper designs the solver through its k-space operators: [k]_E1 in Faraday's
law and [k]_B1 in Ampere's law (Sec. 3.1, Eqs. (11)-(15)), which can be used
directly in an FFT-based solver at any time step (Sec. 1, Sec. 3.1) before the
finite-difference stencils of App. B approximate them.  This module applies the
leapfrog step of Eq. (1) with the derivatives taken in Fourier space.

On a periodic staggered grid every stencil is diagonal in Fourier space.  Arrays
are stored at their own staggered positions (index i <-> x = (i + s) dx, s = 0
or 1/2, as in the finite-difference oracle: E1 (i+1/2,j,k), E2 (i,j+1/2,k),
E3 (i,j,k+1/2), B1 (i,j+1/2,k+1/2), B2 (i+1/2,j,k+1/2), B3 (i+1/2,j+1/2,k), J
with E; in 2D the x3 offsets drop out), so a
derivative from integer to half-integer positions multiplies the DFT by
i [k] e^{+i k dx/2}, and one from half-integer to integer positions by
i [k] e^{-i k dx/2} (App. B Eq. (B.3) for the symbol of a stencil).  The x2 and
x3 operators are Yee's.  With the symbols of the fitted stencils the step is the
finite-difference step; with the target operators it has no x1 dispersion error
and a unit transverse-force factor.  The current J1 is used as given (a caller
applying the x1 correction of Sec. 3.3 passes the corrected J1).
"""
from __future__ import annotations

import numpy as np

from . import closed_forms as cf


def x1_wavenumbers(n1, dx1):
    """k of the DFT bins along x1 (numpy order; the Nyquist bin of an even n1
    carries k = -pi/dx1, equivalent for the odd symbols used here)."""
    return 2.0 * np.pi * np.fft.fftfreq(n1, d=dx1)


def stencil_symbol(c, n1, dx1):
    """[k] = sum_j C_j sin((2j-1) k dx/2)/(dx/2) at the DFT bins (App. B Eq. (B.3))."""
    return cf.k_stencil(c, x1_wavenumbers(n1, dx1), dx1)


def target_symbols(kind, n1, dx1, dt):
    """The target operators ([k]_E1, [k]_B1) of `kind` ("proposed", Eq. (15); "xu";
    "yee_tstagger") at the DFT bins: k_g T(|k|/k_g) with the sign of k."""
    kn = np.fft.fftfreq(n1)              # k / k_g, k_g = 2 pi/dx1
    tE, tB = cf.target_ops(np.abs(kn), dt / dx1, kind)
    kg = 2.0 * np.pi / dx1
    return np.sign(kn) * kg * tE, np.sign(kn) * kg * tB


class SpectralSolver:
    """Leapfrog field step of Eq. (1) on a periodic grid, (n2, n1) in 2D or
    (n3, n2, n1) in 3D, with x1 operators kE1 (Faraday) and kB1 (Ampere) given
    at the x1 DFT bins and Yee operators along x2 and x3."""

    def __init__(self, n, dx, dt, kE1, kB1, slope0=1.0):
        self.ndim = len(n)
        self.dt = float(dt)
        self.dx = tuple(dx)
        self.kB1 = np.asarray(kB1, dtype=np.float64)
        self.slope0 = float(slope0)   # d[k]_B1/dk at k = 0
        axes = list(range(self.ndim))[::-1]          # array axis of x1, x2, (x3)

        def along(vec, d):
            s = [1] * self.ndim
            s[axes[d]] = vec.size
            return vec.reshape(s)

        self.dE, self.dB = [], []
        for d in range(self.ndim):
            k = 2.0 * np.pi * np.fft.fftfreq(n[d], d=dx[d])
            if d == 0:
                kE, kB = np.asarray(kE1, dtype=np.float64), np.asarray(kB1, dtype=np.float64)
            else:
                kE = kB = np.sin(k * dx[d] / 2.0) / (dx[d] / 2.0)
            # integer -> half-integer (Faraday side), half-integer -> integer (Ampere side)
            self.dE.append(along(1j * kE * np.exp(0.5j * k * dx[d]), d))
            self.dB.append(along(1j * kB * np.exp(-0.5j * k * dx[d]), d))
        if self.ndim == 2:
            z = np.zeros((1, 1))
            self.dE.append(z)
            self.dB.append(z)

    def correct_j1(self, j1):
        """x1 current correction of Sec. 3.3 done as the paper states it, with an
        FFT along x1 only: J1 <- ([k]_Yee / [k]_B1) J1 per x1 Fourier mode, with
        the k = 0 mode unchanged when [k]_B1 has slope 1 there (the target
        operators; a stencil's slope is sum_j (2j-1) C^B_j and is divided out)."""
        n1 = j1.shape[-1]
        k = x1_wavenumbers(n1, self.dx[0])
        kY = cf.k_yee(k, self.dx[0])
        ratio = np.ones(n1)
        nz = k != 0
        ratio[nz] = kY[nz] / self.kB1[nz]
        ratio[~nz] = 1.0 / self.slope0
        return np.fft.ifft(np.fft.fft(j1, axis=-1) * ratio, axis=-1).real

    def div_b(self, F):
        """Divergence of E at the integer nodes with the Ampere-side operators
        (the form Gauss's law takes with this solver, Sec. 3.3)."""
        fft, ifft = np.fft.fftn, np.fft.ifftn
        d1B, d2B, d3B = self.dB
        return ifft(d1B * fft(F.e1) + d2B * fft(F.e2) + d3B * fft(F.e3)).real

    def step(self, F, J=None):
        """Advance F (attributes e1..e3 = E^n, b1..b3 = B^{n-1/2}, arrays of the
        grid's shape) to E^{n+1}, B^{n+1/2} in place; J = (J1, J2, J3) at the E
        positions, or None for no current.  In 2D every d/dx3 is zero."""
        fft, ifft = np.fft.fftn, np.fft.ifftn
        dt = self.dt
        d1E, d2E, d3E = self.dE
        d1B, d2B, d3B = self.dB
        e1, e2, e3 = fft(F.e1), fft(F.e2), fft(F.e3)
        b1, b2, b3 = fft(F.b1), fft(F.b2), fft(F.b3)
        # Faraday: B^{n+1/2} = B^{n-1/2} - dt curl_E E^n
        b1 = b1 - dt * (d2E * e3 - d3E * e2)
        b2 = b2 - dt * (d3E * e1 - d1E * e3)
        b3 = b3 - dt * (d1E * e2 - d2E * e1)
        # Ampere: E^{n+1} = E^n + dt (curl_B B^{n+1/2} - J)
        e1 = e1 + dt * (d2B * b3 - d3B * b2)
        e2 = e2 + dt * (d3B * b1 - d1B * b3)
        e3 = e3 + dt * (d1B * b2 - d2B * b1)
        if J is not None:
            e1 = e1 - dt * fft(J[0])
            e2 = e2 - dt * fft(J[1])
            e3 = e3 - dt * fft(J[2])
        for nm, a in (("e1", e1), ("e2", e2), ("e3", e3), ("b1", b1), ("b2", b2), ("b3", b3)):
            getattr(F, nm)[...] = ifft(a).real

