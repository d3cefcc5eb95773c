"""The spectral x1 field path (pic_set_spectral) on the GPU against the oracle.

With the symbols of the App. B stencils, [k] = sum_j C_j sin((2j-1) k dx1/2)/(dx1/2)
(App. B Eq. (B.3)), the spectral path applies exactly the finite-difference
operators, so the whole PIC step (gather with the time-centred B, push, deposit,
x1 current correction, fields) must equal the finite-difference oracle: 1e-12
(FP64), 2D and 3D, dt/dx1 = 1/4 (correction active).  With the target operators
of Eq. (15) the field step must equal the oracle's spectral step
(oracle/spectral.py) and carry every x1 mode at the speed of light.
"""
import numpy as np
import pytest

from oracle import closed_forms as cf
from oracle import oracle as orc
from oracle import spectral as sp
from oracle.gen_tables import load as load_table
from paper_2004_03754_gb300 import inputs

pytestmark = pytest.mark.gpu

DX1, DX2 = inputs.DX1, inputs.DX2
NAMES6 = ("e1", "e2", "e3", "b1", "b2", "b3")


@pytest.fixture(scope="module")
def pic():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2004_03754_gb300 import pic as P
    return P


def _half(sym, n1):
    return np.ascontiguousarray(np.abs(sym[: n1 // 2 + 1]) * np.sign(np.arange(n1 // 2 + 1)))


@pytest.mark.parametrize("ndim", [2, 3])
def test_spectral_path_with_stencil_symbols_equals_fd_oracle(pic, ndim):
    r = 0.25
    cE, cB = load_table(16, r, 0.3)
    dt = r * DX1
    n = (96, 24) if ndim == 2 else (64, 10, 8)
    dx = (DX1, DX2, DX2)[:ndim]
    g = orc.Grid(n, dx, dt, cE, cB)
    F = orc.Fields(g)
    sim = pic.Simulation(n, dx, dt, cE, cB, precision="fp64", pusher="boris")
    for nm, a in zip(NAMES6, inputs.random_fields(g.shape, amp=0.5, seed=61)[:6]):
        getattr(F, nm)[...] = a
        sim.load_field(nm, a)
    k = 2 * np.pi * np.arange(n[0] // 2 + 1) / (n[0] * DX1)
    kE, kB = cf.k_stencil(cE, k, DX1), cf.k_stencil(cB, k, DX1)
    slope = float(np.dot(2 * np.arange(1, cB.size + 1) - 1, cB))
    sim.set_spectral(kE, kB, slope)
    P = inputs.random_particles(n, dx, 2500 if ndim == 2 else 800, umax=1.5, seed=62)
    sim.load_particles(P.x, P.u, P.w)
    Po = orc.Particles(P.x, P.u, P.w)
    orc.step(g, F, Po, nsteps=5)
    sim.step(5)
    for nm in NAMES6:
        ref = getattr(F, nm)
        assert np.abs(sim.read_field(nm) - ref).max() <= 1e-12 * np.abs(ref).max(), nm
    x, u, _ = sim.read_particles()
    for c in range(3):
        assert np.abs(u[c] - Po.u[c]).max() <= 1e-12 * np.abs(Po.u[c]).max()
    for d in range(ndim):
        L = g.length[d]
        assert np.abs((x[d] - Po.x[d] + L / 2) % L - L / 2).max() <= 1e-12 * L
    # back to the stencils: the state continues on the finite-difference path
    sim.set_spectral(None, None)
    sim.step(1)
    orc.step(g, F, Po)
    assert np.abs(sim.read_field("e2") - F.e2).max() <= 1e-12 * np.abs(F.e2).max()
    sim.close()


def test_spectral_path_with_target_operators_equals_spectral_oracle(pic):
    r = 0.25
    dt = r * DX1
    n = (128, 16)
    cE, cB = load_table(16, r, 0.3)          # only for the context; the symbols replace them
    sim = pic.Simulation(n, (DX1, DX2), dt, cE, cB, precision="fp64", pusher="boris")
    kE, kB = sp.target_symbols("proposed", n[0], DX1, dt)
    S = sp.SpectralSolver(n, (DX1, DX2), dt, kE, kB)
    g = orc.Grid(n, (DX1, DX2), dt, cE, cB)
    F = orc.Fields(g)
    for nm, a in zip(NAMES6, inputs.random_fields(g.shape, amp=0.5, seed=63)[:6]):
        getattr(F, nm)[...] = a
        sim.load_field(nm, a)
    sim.set_spectral(_half(kE, n[0]), _half(kB, n[0]), 1.0)
    for _ in range(6):
        S.step(F)
    sim.step(6)
    for nm in NAMES6:
        ref = getattr(F, nm)
        assert np.abs(sim.read_field(nm) - ref).max() <= 1e-12 * np.abs(ref).max(), nm
    sim.close()


def test_spectral_path_is_luminal_up_to_nyquist(pic):
    # a standing x1 mode oscillates at exactly omega = k with the target operators
    # of Eq. (15), up to the highest modes of the grid (the 16-coefficient stencils
    # do so only inside their fitted band)
    r = 0.25
    dt = r * DX1
    n = (64, 2)
    cE, cB = load_table(16, r, 0.3)
    kE, kB = sp.target_symbols("proposed", n[0], DX1, dt)
    for m in (4, 20, 30):
        kx = 2 * np.pi * m / (n[0] * DX1)
        sim = pic.Simulation(n, (DX1, DX2), dt, cE, cB, precision="fp64", pusher="boris")
        sim.set_spectral(_half(kE, n[0]), _half(kB, n[0]), 1.0)
        x = np.arange(n[0]) * DX1
        # the discrete standing mode with omega = k: E2(x, 0) = cos(k x) and, from
        # B3^{1/2} = -B3^{-1/2} and Faraday's update with [k]_E1 = (2/dt) tan(k dt/2),
        # B3(x + dx1/2, -dt/2) = -tan(k dt/2) sin(k (x + dx1/2))
        e2 = np.tile(np.cos(kx * x), (n[1], 1))
        b3 = np.tile(-np.tan(kx * dt / 2) * np.sin(kx * (x + DX1 / 2)), (n[1], 1))
        sim.load_field("e2", e2)
        sim.load_field("b3", b3)
        steps = 200
        sim.step(steps)
        want = np.cos(kx * steps * dt) * e2
        got = sim.read_field("e2")
        assert np.abs(got - want).max() <= 1e-10, m
        sim.close()
