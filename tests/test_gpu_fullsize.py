"""Parity at the benchmark's full size and launch configuration: 2D 4096 x 1024,
Gaussian laser a0 = 4 entering the 8-ppc plasma (29,368,320 electrons),
customised M = 16 solver, Boris pusher -- exactly what bench.py times.

The oracle cannot run 29 million particles in seconds, so it checks
  * a seeded sample of particles one by one (gather from the oracle's own
    fields and time-centred B, push, move),
  * every cell of the vacuum region whose update involves no current
    (an oracle field step with J = 0 is exact there),
  * and, everywhere, a property that holds at any size: the per-step change of
    Gauss's law d_B . E + rho (Eq. (26)), with rho from the GPU's positions.
"""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2004_03754_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def workload():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import bench
    n, dx, P = bench.workload_arrays()
    lk = bench.laser_kwargs(n, dx)
    from oracle.gen_tables import load as load_table
    cE, cB = load_table(16, 0.5, 0.3)
    g = orc.Grid(n, dx, inputs.DT, cE, cB)
    F0 = orc.Fields(g)
    orc.laser_load(g, F0, a0=lk["a0"], k0=lk["k0"], phase=lk["phase"], Lenv=lk["L_env"],
                   x_front=lk["x_front"], w0=lk["w0"], x2c=lk["x2c"])
    bb = orc.bbar(g, F0)
    Fv = F0.copy()
    orc.step(g, Fv, None)      # field-only oracle step (J = 0)
    return dict(n=n, dx=dx, P=P, lk=lk, cE=cE, cB=cB, g=g, F0=F0, bb=bb, Fv=Fv)


def _sample_push(W, idx):
    g, F0, bb, P = W["g"], W["F0"], W["bb"], W["P"]
    L = g.length
    xs, us = [], []
    for p in idx:
        xp = [P.x[0][p], P.x[1][p]]
        eb = orc.gather(g, (F0.e1, F0.e2, F0.e3), bb, xp)
        u = orc.boris(-1.0, g.dt, eb, [P.u[0][p], P.u[1][p], P.u[2][p]])
        gam = np.sqrt(1 + u @ u)
        xn = [(xp[d] + g.dt * u[d] / gam) % L[d] for d in range(2)]
        xs.append(xn)
        us.append(u)
    return np.array(xs), np.array(us)


@pytest.mark.parametrize("precision,tol_u,tol_f", [("fp64", 1e-12, 1e-12), ("mixed", 2e-6, 2e-6)])
def test_full_size_one_step(workload, precision, tol_u, tol_f):
    from paper_2004_03754_gb300 import pic as Pm
    W = workload
    n, dx, P, g = W["n"], W["dx"], W["P"], W["g"]
    sim = Pm.Simulation(n, dx, inputs.DT, W["cE"], W["cB"], precision=precision, pusher="boris")
    sim.load_laser(**W["lk"])
    sim.load_particles(P.x, P.u, P.w, P.qm)
    # the field state the GPU starts from is the oracle's laser load
    for nm in ("e2", "b3"):
        ref = getattr(W["F0"], nm)
        assert np.abs(sim.read_field(nm) - ref).max() <= tol_f * np.abs(ref).max()
    sim.step(1)
    sim.sync()
    info = sim.info()
    assert info.last_stragglers == 0
    x, u, _ = sim.read_particles()
    # sampled particles, one by one
    rng = inputs.rng(7)
    idx = np.sort(rng.choice(P.n, 3000, replace=False))
    xo, uo = _sample_push(W, idx)
    umax = max(np.abs(uo).max(), 1e-300)
    assert np.abs(np.stack([u[c][idx] for c in range(3)], 1) - uo).max() <= tol_u * umax
    for d in range(2):
        L = g.length[d]
        dxp = (x[d][idx] - xo[:, d] + L / 2) % L - L / 2
        assert np.abs(dxp).max() <= max(tol_u, 1e-13) * L
    # vacuum cells far from every particle: exact against the J = 0 oracle step
    i_lo, i_hi = 3840 + 40, 4096 - 40
    for nm in ("e1", "e2", "e3", "b1", "b2", "b3"):
        got = sim.read_field(nm)[:, i_lo:i_hi]
        ref = getattr(W["Fv"], nm)[:, i_lo:i_hi]
        scale = max(np.abs(getattr(W["Fv"], nm)).max(), 1e-300)
        assert np.abs(got - ref).max() <= tol_f * scale, nm
    # Gauss's law change everywhere (rho from the GPU's own particle positions)
    if precision == "fp64":
        F1 = orc.Fields(g)
        for nm in ("e1", "e2", "e3", "b1", "b2", "b3"):
            getattr(F1, nm)[...] = sim.read_field(nm)
        P1 = orc.Particles(x, u, P.w)
        P0 = orc.Particles(P.x, P.u, P.w)
        G0 = orc.div_e(g, W["F0"]) - orc.rho(g, P0)
        G1 = orc.div_e(g, F1) - orc.rho(g, P1)
        scale = np.abs(orc.rho(g, P0)).max()
        assert np.abs(G1 - G0).max() <= 1e-12 * scale
    sim.close()


# ---------------------------------------------------------------------------
# 3D, 1024 x 256 x 256 cells, 2 electrons per cell in x1 in [255, 896) cells
# (84,017,152 electrons), Gaussian laser w0 = 30, a0 = 10, customised solver,
# analytic pusher (the 3D workload of `bench.py --workload c3`)
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def workload3d():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import bench
    n, dx, P = bench.c3_workload_arrays()
    # the bench's pulse starts behind the plasma; for a one-step check the same
    # pulse is placed 245 cells into it, so that the sampled electrons feel it
    lk = dict(bench.c3_laser_kwargs(n, dx), x_front=500 * dx[0])
    from oracle.gen_tables import load as load_table
    cE, cB = load_table(16, 0.5, 0.3)
    g = orc.Grid(n, dx, inputs.DT, cE, cB)
    F0 = orc.Fields(g)
    orc.laser_load(g, F0, a0=lk["a0"], k0=lk["k0"], phase=lk["phase"], Lenv=lk["L_env"],
                   x_front=lk["x_front"], w0=lk["w0"], x2c=lk["x2c"], x3c=lk["x3c"])
    return dict(n=n, dx=dx, P=P, lk=lk, cE=cE, cB=cB, g=g, F0=F0)


@pytest.mark.parametrize("precision,tol", [("mixed", 2e-6), ("fp64", 1e-12)])
def test_full_size_3d_one_step(workload3d, precision, tol):
    from paper_2004_03754_gb300 import pic as Pm
    W = workload3d
    n, dx, P, g, F0 = W["n"], W["dx"], W["P"], W["g"], W["F0"]
    sim = Pm.Simulation(n, dx, inputs.DT, W["cE"], W["cB"], precision=precision, pusher="analytic")
    sim.load_laser(**W["lk"])
    sim.load_particles(P.x, P.u, P.w, P.qm)
    sim.step(1)
    sim.sync()
    assert sim.info().last_stragglers == 0
    x, u, _ = sim.read_particles()
    rng = inputs.rng(9)
    # particles: recompute one by one a sample of the electrons inside the pulse
    # near its axis: gather with the time-centred B formed locally, analytic push, move
    c2, c3 = n[1] * dx[1] / 2, n[2] * dx[2] / 2
    inside = np.nonzero((P.x[0] > 300 * dx[0]) & (P.x[0] < 480 * dx[0]) &
                        (np.abs(P.x[1] - c2) < 20) & (np.abs(P.x[2] - c3) < 20))[0]
    idx = np.sort(rng.choice(inside, 600, replace=False))
    L = g.length
    ref_u, ref_x = [], []
    for p in idx:
        xp = [P.x[d][p] for d in range(3)]
        eb = orc.gather_centred(g, F0, xp)
        uu, it = orc.analytic(-1.0, g.dt, eb, [P.u[c][p] for c in range(3)])
        assert it > 0
        gam = np.sqrt(1 + uu @ uu)
        ref_u.append(uu)
        ref_x.append([(xp[d] + g.dt * uu[d] / gam) % L[d] for d in range(3)])
    ref_u, ref_x = np.array(ref_u), np.array(ref_x)
    assert np.abs(ref_u).max() > 0.1           # the sample does feel the laser
    got_u = np.stack([u[c][idx] for c in range(3)], 1)
    assert np.abs(got_u - ref_u).max() <= tol * np.abs(ref_u).max()
    for d in range(3):
        dxp = (x[d][idx] - ref_x[:, d] + L[d] / 2) % L[d] - L[d] / 2
        assert np.abs(dxp).max() <= max(tol, 1e-13) * L[d]
    # fields: vacuum cells inside the pulse body (x1 in [185, 215) cells: farther
    # from the plasma than the stencil and shape reach) recomputed with J = 0
    cells = [(int(i), int(j), int(k)) for i, j, k in zip(rng.integers(185, 215, 300),
                                                        rng.integers(0, n[1], 300),
                                                        rng.integers(0, n[2], 300))]
    got = {nm: sim.read_field(nm) for nm in ("e1", "e2", "e3", "b1", "b2", "b3")}
    scale = max(np.abs(F0.e2).max(), 1e-300)
    for (i, j, k) in cells:
        ref = orc.point_update(g, F0, i, j, k)
        for c, nm in enumerate(("e1", "e2", "e3", "b1", "b2", "b3")):
            assert abs(got[nm][k, j, i] - ref[c]) <= tol * scale, (nm, i, j, k)
    sim.close()
