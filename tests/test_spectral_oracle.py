"""Spectral (FFT) field step of the oracle (oracle/spectral.py), CPU.

Pinned to (1) the finite-difference oracle step, which it must reproduce to FFT
rounding when given the stencils' own symbols (App. B Eq. (B.3)), with and
without current; (2) the dispersion the target operators fix (Sec. 3.1,
Eq. (15)): a standing mode along x1 oscillates at omega = k exactly up to the
Nyquist mode, which the fitted stencils reach only inside their band."""
import math

import numpy as np
import pytest

from oracle import oracle as orc
from oracle import spectral as sp
from oracle.gen_tables import load as load_table
from paper_2004_03754_gb300 import coeffs, inputs

DX1, DX2, DT = inputs.DX1, inputs.DX2, inputs.DT
NAMES6 = ("e1", "e2", "e3", "b1", "b2", "b3")


def cases():
    return [("proposed r=1/2", load_table(16, 0.5, 0.3), DT),
            ("proposed r=1/4", load_table(16, 0.25, 0.3), 0.25 * DX1),
            ("xu r=1/4", coeffs.load("xu", 16, 0.25, 0.3), 0.25 * DX1),
            ("yee", (np.array([1.0]), np.array([1.0])), DT),
            ("random M=5", inputs.random_coeffs(5, seed=1), 0.3 * DX1)]


def worst(A, B):
    return max(np.abs(getattr(A, nm) - getattr(B, nm)).max() / np.abs(getattr(B, nm)).max()
               for nm in NAMES6)


@pytest.mark.parametrize("n", [(48, 20), (49, 21), (24, 10, 8), (25, 9, 7)])
@pytest.mark.parametrize("name,cc,dt", cases())
def test_stencil_symbols_reproduce_the_fd_step(name, cc, dt, n):
    cE, cB = cc
    dx = (DX1, DX2, DX2)[:len(n)]
    if len(n) == 3:
        dt = 0.8 * dt                     # inside the 3D CFL bound of every set
    g = orc.Grid(n, dx, dt, cE, cB)
    F = orc.Fields(g)
    for nm, a in zip(NAMES6, inputs.random_fields(g.shape, amp=0.5, seed=3)[:6]):
        getattr(F, nm)[...] = a
    S = F.copy()
    orc.step(g, F, None, nsteps=3)
    sol = sp.SpectralSolver(n, dx, dt, sp.stencil_symbol(cE, n[0], DX1),
                            sp.stencil_symbol(cB, n[0], DX1))
    for _ in range(3):
        sol.step(S)
    assert worst(S, F) < 1e-13, name


@pytest.mark.parametrize("name,cc,dt", cases()[:2])
def test_stencil_symbols_with_current(name, cc, dt):
    # the finite-difference oracle deposits (and, for C^B != e_1, corrects) J;
    # given that J, the spectral step lands on the same fields
    cE, cB = cc
    n = (40, 16)
    g = orc.Grid(n, (DX1, DX2), dt, cE, cB)
    F = orc.Fields(g)
    for nm, a in zip(NAMES6, inputs.random_fields(g.shape, amp=0.5, seed=7)[:6]):
        getattr(F, nm)[...] = a
    P = inputs.random_particles(n, (DX1, DX2), 2000, umax=2.0, seed=8)
    Po = orc.Particles(P.x, P.u, P.w)
    S = F.copy()
    orc.step(g, F, Po)
    assert np.abs(F.j1).max() > 0
    sol = sp.SpectralSolver(n, (DX1, DX2), dt, sp.stencil_symbol(cE, n[0], DX1),
                            sp.stencil_symbol(cB, n[0], DX1))
    sol.step(S, (F.j1, F.j2, F.j3))
    assert worst(S, F) < 1e-13, name


def standing_mode_omega(kE1, kB1, n1, m, dt, nsteps=240):
    """omega of the standing mode E2 = cos(k x1) (B = 0 at t = -dt/2) from the
    exact recurrence y_{n+1} + y_{n-1} = 2 cos(omega dt) y_n of its projection."""
    n = (n1, 2)

    class St:
        pass

    F = St()
    x1 = np.arange(n1) * DX1
    k = 2 * np.pi * m / (n1 * DX1)
    for nm in NAMES6:
        setattr(F, nm, np.zeros((2, n1)))
    F.e2[...] = np.cos(k * x1)
    sol = sp.SpectralSolver(n, (DX1, DX2), dt, kE1, kB1)
    basis = np.cos(k * x1)
    y = [float((F.e2 * basis).sum())]
    for _ in range(nsteps):
        sol.step(F)
        y.append(float((F.e2 * basis).sum()))
    y = np.array(y)
    c = (y[1:-1] * (y[2:] + y[:-2])).sum() / (2 * (y[1:-1] ** 2).sum())
    return k, math.acos(c) / dt


@pytest.mark.parametrize("r", [0.5, 0.25])
def test_target_operators_are_luminal_to_nyquist(r):
    n1, dt = 32, r * DX1
    kE1, kB1 = sp.target_symbols("proposed", n1, DX1, dt)
    cE, cB = load_table(16, r, 0.3)
    sE, sB = sp.stencil_symbol(cE, n1, DX1), sp.stencil_symbol(cB, n1, DX1)
    for m in (1, 4, 9, 12, 15, 16):
        k, om = standing_mode_omega(kE1, kB1, n1, m, dt)
        assert abs(om / k - 1) < 1e-12, m
        _, om_fit = standing_mode_omega(sE, sB, n1, m, dt)
        kn = m / n1
        if kn < 0.3:                       # inside the fitted band: the stencils are luminal too
            assert abs(om_fit / k - 1) < 1e-6, m
        elif kn > 0.4:                     # beyond it only the k-space operators are
            assert abs(om_fit / k - 1) > 1e-4, m
    # Yee for contrast: a visible phase error already at 4 modes per box
    k, om = standing_mode_omega(sp.stencil_symbol([1.0], n1, DX1), sp.stencil_symbol([1.0], n1, DX1),
                                n1, 4, DT)
    assert abs(om / k - 1) > 1e-3


@pytest.mark.parametrize("kind,r", [("proposed", 0.5), ("proposed", 0.25), ("yee_tstagger", 0.25)])
def test_fourier_current_correction_keeps_gauss(kind, r):
    # Sec. 3.3: with [k]_B1 != [k]_Yee, the Esirkepov current (continuity with the
    # Yee divergence, Eq. (24)) corrected in x1-Fourier space keeps the change of
    # div_B E - rho at round-off through the spectral step; uncorrected it does not.
    n, dt = (32, 8), r * DX1
    g = orc.Grid(n, (DX1, DX2), dt, np.array([1.0]), np.array([1.0]))
    kE1, kB1 = sp.target_symbols(kind, n[0], DX1, dt)
    rng = np.random.Generator(np.random.PCG64(31))
    npart = 60
    L = np.array([n[0] * DX1, n[1] * DX2])
    xo = rng.uniform(0, 1, (npart, 2)) * L
    xn = xo + rng.uniform(-0.9, 0.9, (npart, 2)) * np.array([DX1, DX2])
    xn = np.mod(xn, L)
    w = rng.uniform(-1, 1, npart)
    v3 = rng.uniform(-0.5, 0.5, npart)
    FJ = orc.Fields(g)
    for q in range(npart):
        d = xn[q] - xo[q]
        d -= L * np.round(d / L)                      # the move, not the wrapped difference
        orc.deposit(g, FJ, w[q], xo[q], xo[q] + d, v3[q])
    rho0 = orc.rho(g, orc.Particles([xo[:, 0], xo[:, 1]], [np.zeros(npart)] * 3, w))
    rho1 = orc.rho(g, orc.Particles([xn[:, 0], xn[:, 1]], [np.zeros(npart)] * 3, w))
    scale = np.abs(rho0).max()
    # the deposit's own continuity with the Yee divergence (Eq. (24))
    assert np.abs(rho1 - rho0 + dt * orc.div_yee(g, FJ.j1, FJ.j2, FJ.j3)).max() < 1e-13 * scale

    def gauss_change(correct):
        sol = sp.SpectralSolver(n, (DX1, DX2), dt, kE1, kB1)
        F = orc.Fields(g)
        for nm, a in zip(NAMES6, inputs.random_fields(g.shape, amp=0.5, seed=13)[:6]):
            getattr(F, nm)[...] = a
        G0 = sol.div_b(F) - rho0
        j1 = sol.correct_j1(FJ.j1) if correct else FJ.j1
        sol.step(F, (j1, FJ.j2, FJ.j3))
        return np.abs(sol.div_b(F) - rho1 - G0).max()

    assert gauss_change(True) < 1e-12 * scale
    kY = np.sin(sp.x1_wavenumbers(n[0], DX1) * DX1 / 2) / (DX1 / 2)
    if kind == "proposed" and r == 0.5:
        # at dt = dx1/2 the target [k]_B1 = sin(k dt)/dt is Yee's operator: nothing to correct
        assert np.abs(kB1 - kY).max() < 1e-12 * np.abs(kY).max()
        assert gauss_change(False) < 1e-12 * scale
    else:
        assert gauss_change(False) > 1e-6 * scale
