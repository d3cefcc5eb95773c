"""Energy-gain integrals of Sec. 4.2 (W_LWFA from E1, W_DLA from E_perp) kept per
particle by the GPU particle kernels, against the oracle's step (FP64, 1e-12),
through the C ABI; with re-binning every other step so that the sums travel
with their particles, and with the mixed form's stated error."""
import numpy as np
import pytest

from oracle import oracle as orc
from oracle.gen_tables import load as load_table
from paper_2004_03754_gb300 import inputs

pytestmark = pytest.mark.gpu

DX1, DX2, DT = inputs.DX1, inputs.DX2, inputs.DT
NAMES6 = ("e1", "e2", "e3", "b1", "b2", "b3")


@pytest.fixture(scope="module")
def pic():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2004_03754_gb300 import pic as P
    return P


@pytest.mark.parametrize("case", ["2d_boris", "2d_hc_deposit", "3d_analytic", "2d_mixed"])
def test_energy_gain_integrals_match_oracle(pic, case):
    ndim = 3 if case.startswith("3d") else 2
    n = (40, 12, 9) if ndim == 3 else (150, 40)
    dx = (DX1, DX2, DX2)[:ndim]
    pusher = {"2d_boris": "boris", "2d_hc_deposit": "hc", "3d_analytic": "analytic",
              "2d_mixed": "boris"}[case]
    precision = "mixed" if case == "2d_mixed" else "fp64"
    cE, cB = load_table(16, 0.5, 0.3)
    g = orc.Grid(n, dx, DT, cE, cB)
    sim = pic.Simulation(n, dx, DT, cE, cB, precision=precision, pusher=pusher)
    F = orc.Fields(g)
    for nm, a in zip(NAMES6, inputs.random_fields(g.shape, amp=0.7, seed=41)[:6]):
        getattr(F, nm)[...] = a
        sim.load_field(nm, a)
    P = inputs.random_particles(n, dx, 3000 if ndim == 2 else 800, umax=2.0, seed=42)
    if case != "2d_hc_deposit":
        P.w[:] = 0.0
    sim.enable_energy_gain(True)
    sim.load_particles(P.x, P.u, P.w)
    pic.pic_set_sort_interval(sim.ctx, 2)
    Po = orc.Particles(P.x, P.u, P.w)
    wl, wd = np.zeros(Po.n), np.zeros(Po.n)
    g0 = np.sqrt(1 + sum(c ** 2 for c in Po.u))
    orc.step_gain(g, F, Po, wl, wd, pusher=pusher, nsteps=7)
    sim.step(7)
    gl, gd = sim.read_energy_gain()
    scale = max(np.abs(wl).max(), np.abs(wd).max())
    assert scale > 1e-2
    tol = 1e-5 if precision == "mixed" else 1e-12
    assert np.abs(gl - wl).max() <= tol * scale
    assert np.abs(gd - wd).max() <= tol * scale
    if pusher == "boris":
        # Boris: the two integrals add up to each particle's energy change
        _, u, _ = sim.read_particles()
        g1 = np.sqrt(1 + u[0] ** 2 + u[1] ** 2 + u[2] ** 2)
        assert np.abs(gl + gd - (g1 - g0)).max() <= (1e-12 if precision == "fp64" else 1e-5) * g1.max()
    # a new load restarts them at zero; turning them off refuses the read
    sim.load_particles(P.x, P.u, P.w)
    gl, gd = sim.read_energy_gain()
    assert not gl.any() and not gd.any()
    sim.enable_energy_gain(False)
    with pytest.raises(pic.PicError):
        pic.pic_read_energy_gain(sim.ctx, P.n)
    sim.close()
