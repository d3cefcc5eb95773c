"""The compensated reduced-precision form (PIC_COMPENSATED: E and B as FP32
pairs with error-free FP32 arithmetic, FP64 push and positions, FP32 current)
against the FP64 oracle, through the C ABI.

Bars: with no current, fields and particles within 1e-12 of the oracle (the
pairs carry 48 bits); with depositing particles the FP32 current's error is
stated (as in the mixed form).  The single-electron energy, the quantity the
plain FP32 fields cannot hold beyond a0 ~ 10 (an electron co-moving with the
laser feels E2 - beta1 B3 ~ E/(2 gamma^2), Sec. 1, Sec. 4.1), stays within 1e-4
of the oracle up to a0 = 1e4, in single runs and in ensembles.
"""
import math

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


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("case", ["2d", "2d_quarter", "3d"])
def test_compensated_fields_and_test_particles_match_oracle(pic, case):
    if case == "3d":
        n, dx, table = (40, 12, 9), (DX1, DX2, DX2), (16, 0.5, 0.3)
    elif case == "2d_quarter":
        n, dx, table = (131, 22), (DX1, DX2), (16, 0.25, 0.3)   # C^B != e1
    else:
        n, dx, table = (203, 37), (DX1, DX2), (16, 0.5, 0.3)
    cE, cB = load_table(*table)
    dt = table[1] * DX1
    g = orc.Grid(n, dx, dt, cE, cB)
    sim = pic.Simulation(n, dx, dt, cE, cB, precision="compensated", pusher="boris")
    F = orc.Fields(g)
    for nm, a in zip(NAMES6, inputs.random_fields(g.shape, amp=0.5, seed=11)[:6]):
        getattr(F, nm)[...] = a
        sim.load_field(nm, a)
    P = inputs.random_particles(n, dx, 600, umax=2.0, seed=12)
    P.w[:] = 0.0                                   # test particles: no current
    sim.load_particles(P.x, P.u, P.w)
    Po = orc.Particles(P.x, P.u, P.w)
    orc.step(g, F, Po, nsteps=4)
    sim.step(4)
    sim.sync()
    for nm in NAMES6:
        assert rel(sim.read_field(nm), getattr(F, nm)) <= 1e-12, nm
    x, u, _ = sim.read_particles()
    for c in range(3):
        assert rel(u[c], Po.u[c]) <= 1e-12, c
    for d in range(len(n)):
        L = g.length[d]
        dxp = (x[d] - Po.x[d] + L / 2) % L - L / 2
        assert np.abs(dxp).max() <= 1e-12 * L
    sim.close()


def test_compensated_with_current_states_its_error(pic):
    # depositing particles: the current is accumulated in FP32 (as in the mixed
    # form); fields and momenta then carry that error, the fields themselves 48 bits
    cE, cB = load_table(16, 0.5, 0.3)
    n = (128, 32)
    g = orc.Grid(n, (DX1, DX2), DT, cE, cB)
    sim = pic.Simulation(n, (DX1, DX2), DT, cE, cB, precision="compensated", pusher="boris")
    F = orc.Fields(g)
    for nm, a in zip(NAMES6, inputs.random_fields(g.shape, amp=1.0, seed=5)[:6]):
        getattr(F, nm)[...] = a
        sim.load_field(nm, a)
    P = inputs.random_particles(n, (DX1, DX2), 4000, umax=2.0, seed=5)
    sim.load_particles(P.x, P.u, P.w)
    Po = orc.Particles(P.x, P.u, P.w)
    orc.step(g, F, Po, nsteps=5)
    sim.step(5)
    sim.sync()
    errf = max(rel(sim.read_field(nm), getattr(F, nm)) for nm in NAMES6)
    _, u, _ = sim.read_particles()
    erru = max(rel(u[c], Po.u[c]) for c in range(3))
    assert errf < 1e-6, errf
    assert erru < 1e-6, erru


def _plane_wave_electron(a0, n1):
    """The ensemble recipe for one run: plane sin^2 pulse of min(10 wavelengths,
    n1/2 cells), electron at rest 16 cells ahead of its front."""
    Lc = min(320, n1 // 2)
    laser = dict(a0=a0, L_env=Lc * DX1, x_front=(Lc + 4) * DX1)
    xe = [np.array([(Lc + 20) * DX1]), np.array([0.5 * DX2])]
    return laser, xe


@pytest.mark.parametrize("a0", [1e3, 1e4])
def test_single_electron_energy_within_1e4_at_high_a0(pic, a0):
    # analytic pusher (the only one of the three that follows a0 >= 1e3, Sec. 4.1)
    cE, cB = load_table(16, 0.5, 0.3)
    n, nsteps, chunk = (512, 2), 2000, 250
    laser, xe = _plane_wave_electron(a0, n[0])
    g = orc.Grid(n, (DX1, DX2), DT, cE, cB)
    F = orc.Fields(g)
    orc.laser_load(g, F, a0=a0, Lenv=laser["L_env"], x_front=laser["x_front"])
    Po = orc.Particles(xe, [np.zeros(1)] * 3, np.zeros(1))
    sims = {}
    for prec in ("compensated", "mixed"):
        s = pic.Simulation(n, (DX1, DX2), DT, cE, cB, precision=prec, pusher="analytic")
        s.load_laser(**laser)
        s.load_particles(xe, [np.zeros(1)] * 3, np.zeros(1))
        sims[prec] = s
    worst = {"compensated": 0.0, "mixed": 0.0}
    peak = 0.0
    for _ in range(nsteps // chunk):
        orc.step(g, F, Po, pusher="analytic", nsteps=chunk)
        kin = math.sqrt(1 + sum(float(Po.u[c][0]) ** 2 for c in range(3))) - 1
        peak = max(peak, kin)
        for prec, s in sims.items():
            s.step(chunk)
            _, u, _ = s.read_particles()
            k = math.sqrt(1 + sum(float(u[c][0]) ** 2 for c in range(3))) - 1
            worst[prec] = max(worst[prec], abs(k - kin) / kin)
    assert peak > 10.0                      # the electron is relativistic by then
    assert worst["compensated"] <= 1e-4, worst
    for s in sims.values():
        s.close()


def test_ensemble_compensated_matches_oracle_and_holds_energy(pic):
    # an ensemble of vacuum plane-wave runs, a0 from 10 to 1e4 (log-spaced), 16
    # test electrons each: per-run fields and momenta against the oracle, and the
    # electrons' energy within 1e-4 of the oracle's
    import torch
    cE, cB = load_table(16, 0.5, 0.3)
    a0s = [10.0, 100.0, 1000.0, 10000.0]
    sizes = [(512, 64), (384, 16), (640, 24), (512, 8)]
    nsteps = 1200
    stream = torch.cuda.Stream()
    ens = pic.Ensemble([s[0] for s in sizes], [s[1] for s in sizes], (DX1, DX2), DT, cE, cB,
                       precision="compensated", pusher="analytic", stream=stream.cuda_stream)
    lasers, xs = [], ([], [])
    for (n1, n2), a0 in zip(sizes, a0s):
        Lc = min(320, n1 // 2)
        xf = (Lc + 4) * DX1
        lasers.append(pic.pic_laser(a0, 1.0, 0.0, Lc * DX1, xf, 0.0, n2 * DX2 / 2, 0.0))
        for i in range(16):
            xs[0].append(xf + (16 + 2 * i) * DX1)
            xs[1].append((i + 0.5) * n2 * DX2 / 16)
    ens.load_lasers(lasers)
    npart = 16 * len(sizes)
    ens.load_particles([16] * len(sizes), [np.array(xs[0]), np.array(xs[1])],
                       [np.zeros(npart)] * 3, np.zeros(npart))
    ens.set_steps([nsteps] * len(sizes))
    ens.run()
    _, u, _ = ens.read_particles()
    for r, ((n1, n2), a0) in enumerate(zip(sizes, a0s)):
        las = lasers[r]
        g = orc.Grid((n1, n2), (DX1, DX2), DT, cE, cB)
        F = orc.Fields(g)
        orc.laser_load(g, F, a0=las.a0, Lenv=las.L_env, x_front=las.x_front, x2c=las.x2c)
        sl = slice(16 * r, 16 * r + 16)
        Po = orc.Particles([np.array(xs[0][sl]), np.array(xs[1][sl])], [np.zeros(16)] * 3,
                           np.zeros(16))
        orc.step(g, F, Po, pusher="analytic", nsteps=nsteps)
        for nm in ("e2", "b3"):
            assert rel(ens.read_field(r, nm), getattr(F, nm)) <= 1e-11, (r, nm)
        kin_o = np.sqrt(1 + Po.u[0] ** 2 + Po.u[1] ** 2 + Po.u[2] ** 2) - 1
        kin_g = np.sqrt(1 + u[0][sl] ** 2 + u[1][sl] ** 2 + u[2][sl] ** 2) - 1
        assert np.abs(kin_g - kin_o).max() <= 1e-4 * kin_o.max(), (r, a0)
    ens.close()
