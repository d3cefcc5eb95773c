"""Moving window along x1 (Sec. 4.1 boundary) on the GPU path against the
oracle's window (oracle/moving_window.py): same cleared columns, same particles
removed, fields and surviving particles equal to 1e-12 (FP64)."""
import numpy as np
import pytest

from oracle import moving_window as mw
from oracle import oracle as orc
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


@pytest.mark.parametrize("r,start,ndim", [(0.5, 0, 2), (0.25, 3, 2), (0.5, 2, 3)])
def test_moving_window_matches_oracle(pic, r, start, ndim):
    cE, cB = load_table(16, r, 0.3)
    dt = r * DX1
    n = (96, 20) if ndim == 2 else (48, 8, 6)
    dx = (DX1, DX2, DX2)[:ndim]
    g = orc.Grid(n, dx, dt, cE, cB)
    F = orc.Fields(g)
    sim = pic.Simulation(n, dx, dt, cE, cB, precision="fp64", pusher="boris")
    for nm, a in zip(NAMES6, inputs.random_fields(g.shape, amp=0.5, seed=51)[:6]):
        getattr(F, nm)[...] = a
        sim.load_field(nm, a)
    P = inputs.random_particles(n, dx, 1500 if ndim == 2 else 600, umax=1.0, seed=52)
    sim.load_particles(P.x, P.u, P.w)
    Po = orc.Particles(P.x, P.u, P.w)
    sim.set_moving_window(start)
    W = mw.MovingWindow(g, start_step=start)
    nsteps = 22
    for _ in range(nsteps):
        orc.step(g, F, Po)
        Po = W.after_step(F, Po)
    sim.step(nsteps)
    origin, shifts = sim.window()
    assert shifts == W.shifts > 0 and origin == W.origin
    for nm in NAMES6:
        ref = getattr(F, nm)
        assert np.abs(sim.read_field(nm) - ref).max() <= 1e-12 * np.abs(ref).max(), nm
    x, u, w = sim.read_particles()
    assert 0 < Po.n < P.n and len(w) == Po.n
    assert np.array_equal(w, Po.w)
    for c in range(3):
        assert np.abs(u[c] - Po.u[c]).max() <= 1e-12 * np.abs(Po.u[c]).max()
    for d in range(ndim):
        L = g.length[d]
        dxp = (x[d] - Po.x[d] + L / 2) % L - L / 2
        assert np.abs(dxp).max() <= 1e-12 * L
    # the cleared columns hold only what the later steps put there: with the
    # window off the state simply continues
    sim.set_moving_window(-1)
    sim.step(2)
    orc.step(g, F, Po, nsteps=2)
    assert np.abs(sim.read_field("e2") - F.e2).max() <= 1e-12 * np.abs(F.e2).max()
    sim.close()
