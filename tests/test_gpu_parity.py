"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Bar (FP64 path): max |gpu - oracle| <= 1e-12 * max |oracle| per field
component and per particle coordinate.  Reduced precision (FP32 fields, FP64
pusher) states its error against the same oracle.
"""
import math

import numpy as np
import pytest

from oracle import oracle as orc
from oracle.gen_tables import load as load_table
from paper_2004_03754_gb300 import inputs

pytestmark = pytest.mark.gpu

DX1, DX2, DT = inputs.DX1, inputs.DX2, inputs.DT
TOL64 = 1e-12
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


def make_pair(pic, n, cE, cB, dt=DT, precision="fp64", pusher="boris", dx=None):
    dx = dx or (DX1, DX2, DX2)[: len(n)]
    g = orc.Grid(n, dx, dt, cE, cB)
    sim = pic.Simulation(n, dx, dt, cE, cB, precision=precision, pusher=pusher)
    return g, sim


def load_same_fields(g, sim, seed=5, amp=0.5):
    F = orc.Fields(g)
    fs = inputs.random_fields(g.shape, amp=amp, seed=seed)
    for nm, a in zip(NAMES6, fs[:6]):
        getattr(F, nm)[...] = a
        sim.load_field(nm, a)
    return F


def load_same_particles(g, sim, P, qm=-1.0):
    sim.load_particles(P.x, P.u, P.w, qm)
    return orc.Particles(P.x, P.u, P.w, qm)


def compare_fields(g, F, sim, tol, names=NAMES6):
    worst = 0.0
    for nm in names:
        r = rel(sim.read_field(nm), getattr(F, nm))
        worst = max(worst, r)
        assert r <= tol, "%s: rel err %.3e > %.1e" % (nm, r, tol)
    return worst


def compare_particles(g, Po, sim, tol):
    x, u, w = sim.read_particles()
    worst = 0.0
    for d in range(g.ndim):
        L = g.length[d]
        dxp = (x[d] - Po.x[d] + L / 2) % L - L / 2
        r = float(np.abs(dxp).max() / max(np.abs(Po.x[d]).max(), 1e-300))
        worst = max(worst, r)
        assert r <= tol, "x%d: rel err %.3e" % (d + 1, r)
    for c in range(3):
        r = rel(u[c], Po.u[c])
        worst = max(worst, r)
        assert r <= tol, "u%d: rel err %.3e" % (c + 1, r)
    assert np.array_equal(w, Po.w)
    return worst


# --------------------------------------------------------------------------
# Fields only
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n,table", [
    ((200, 37), "random5"),            # ragged against the 128x8 field tile
    ((256, 64), (16, 0.5, 0.3)),
    ((96, 24), (16, 0.25, 0.3)),
    ((40, 13, 11), "random5"),         # 3D, ragged
    ((64, 16, 8), (16, 0.5, 0.3)),
    ((7, 3), "yee"),                   # grid smaller than the stencil reach
])
def test_field_step_parity(pic, n, table):
    if table == "random5":
        cE, cB = inputs.random_coeffs(5, seed=1)
    elif table == "yee":
        cE = cB = np.array([1.0])
    else:
        cE, cB = load_table(*table)
    dt = DT if table != (16, 0.25, 0.3) else 0.25 * DX1
    g, sim = make_pair(pic, n, cE, cB, dt=dt)
    F = load_same_fields(g, sim)
    for _ in range(4):
        orc.step(g, F, None)
    sim.step(4)
    compare_fields(g, F, sim, TOL64)
    # the time-centred B of the state
    bb = orc.bbar(g, F)
    for c in range(3):
        assert rel(sim.read_field("bbar%d" % (c + 1)), bb[c]) <= TOL64


@pytest.mark.parametrize("n,tile,strip,precision,table", [
    ((1000, 37), (64, 8, 1), None, "fp64", "m16"),         # default row strips, ragged x1/x2 edges
    ((1000, 37), (128, 4, 1), None, "mixed", "m16"),
    ((1000, 37), (128, 4, 1), (64, 5, 2, 2), "mixed", "m16"),   # shallow ring, short items
    ((1000, 37), (128, 4, 1), (224, 0, 3, 3), "mixed", "m16"),
    ((1001, 37), (128, 4, 1), None, "mixed", "m16"),       # row pitch not a multiple of 16 bytes
    ((1002, 21), (64, 4, 1), (32, 3, 4, 8), "fp64", "m16"),  # FP64 rows aligned, FP32 would not be
    ((400, 12, 10), (64, 4, 4), None, "mixed", "m16"),     # 3D: double-buffered tiles
    ((400, 12, 10), (32, 4, 2), None, "fp64", "m16"),
    # 3D plane groups (a CTA of P warps on P consecutive x3 planes): a last group of
    # fewer planes, ragged strips, deeper rings, P above n3 (planes wrap)
    ((400, 12, 10), (64, 4, 4), (128, 0, 4, 2), "mixed", "m16"),
    ((400, 12, 10), (64, 4, 4), (64, 3, 3, 3), "mixed", "m16"),
    ((400, 12, 10), (32, 4, 2), (32, 5, 2, 2), "fp64", "m16"),
    ((256, 8, 3), (64, 4, 1), (64, 0, 8, 2), "mixed", "m16"),
    ((200, 8, 6), (32, 4, 2), (64, 0, 3, 2), "compensated", "m16"),
    ((240, 9, 7), (32, 4, 2), (32, 4, 2, 2), "fp64", "random5"),
    # 3D one warp per plane (warps = 1)
    ((400, 12, 10), (64, 4, 4), (128, 0, 1, 2), "mixed", "m16"),
    ((400, 12, 10), (32, 4, 2), (64, 3, 1, 2), "fp64", "m16"),
    ((600, 20), (96, 8, 1), None, "fp64", "random5"),      # M = 5 on the 8-tap unrolled kernel
    ((600, 20), (96, 8, 1), (96, 7, 2, 2), "fp64", "yee"),
    ((160, 9), (32, 8, 1), (96, 5, 1, 4), "mixed", "m16"),  # strip wider than the last piece
])
def test_field_staging_modes(pic, n, tile, strip, precision, table):
    """Streamed (bulk-copy) and plain-load staging give bit-identical fields; FP64 meets the oracle."""
    if table == "random5":
        cE, cB = inputs.random_coeffs(5, seed=3)
    elif table == "yee":
        cE = cB = np.array([1.0])
    else:
        cE, cB = load_table(16, 0.5, 0.3)
    out = []
    for staging in (0, 1):
        g, sim = make_pair(pic, n, cE, cB, precision=precision)
        sim.set_field_tile(*tile, staging=staging)
        if strip is not None:
            sim.set_field_strip(*strip)
        F = load_same_fields(g, sim, seed=11)
        sim.step(3)
        out.append([sim.read_field(nm) for nm in NAMES6])
    for a, b in zip(*out):
        assert np.array_equal(a, b)
    if precision == "fp64":
        for _ in range(3):
            orc.step(g, F, None)
        compare_fields(g, F, sim, TOL64)


def test_field_shape_arguments_are_checked(pic):
    cE, cB = load_table(16, 0.5, 0.3)
    g, sim = make_pair(pic, (256, 16), cE, cB, precision="mixed")
    with pytest.raises(pic.PicError):
        sim.set_field_tile(30, 8)                 # not a multiple of 16 bytes of FP32
    with pytest.raises(pic.PicError):
        sim.set_field_tile(64, 8, threads=96)
    with pytest.raises(pic.PicError):
        sim.set_field_strip(1024, 0, 16, 8)       # ring does not fit in shared memory
    with pytest.raises(pic.PicError):
        sim.set_field_strip(96, -1, 2, 2)
    g3, sim3 = make_pair(pic, (256, 8, 4), cE, cB, precision="mixed")
    with pytest.raises(pic.PicError):
        sim3.set_field_strip(32, 0, 9, 2)         # 3D plane groups take at most 8 planes
    sim3.set_field_strip(32, 0, 8, 2)
    sim3.step(1)
    sim.set_field_strip(96, 4, 2, 2)              # valid shapes still step
    sim.step(1)


def test_laser_load_parity(pic):
    cE, cB = load_table(16, 0.5, 0.3)
    for n, w0 in (((512, 16), 3.0), ((300, 8), 0.0), ((128, 8, 6), 2.0)):
        g, sim = make_pair(pic, n, cE, cB)
        F = orc.Fields(g)
        kw = dict(a0=2.0, phase=0.3, Lenv=6 * np.pi, x_front=0.8 * g.length[0], w0=w0)
        orc.laser_load(g, F, **kw)
        sim.load_laser(a0=kw["a0"], phase=kw["phase"], L_env=kw["Lenv"], x_front=kw["x_front"], w0=w0)
        compare_fields(g, F, sim, TOL64)


# --------------------------------------------------------------------------
# Full step with particles (FP64)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("case", ["boris2d", "analytic2d", "corr2d", "boris3d", "analytic3d",
                                  "hc2d", "hc3d"])
def test_particle_step_parity(pic, case):
    ndim = 3 if case.endswith("3d") else 2
    pusher = ("analytic" if case.startswith("analytic") else
              "hc" if case.startswith("hc") else "boris")
    if case == "corr2d":
        cE, cB = load_table(16, 0.25, 0.3)
        dt = 0.25 * DX1
    else:
        cE, cB = load_table(16, 0.5, 0.3)
        dt = DT
    n = (96, 40) if ndim == 2 else (24, 12, 10)
    g, sim = make_pair(pic, n, cE, cB, dt=dt, pusher=pusher)
    F = load_same_fields(g, sim, amp=2.0)
    dx = (DX1, DX2, DX2)[:ndim]
    P = inputs.random_particles(n, dx, 3000 if ndim == 2 else 2000, umax=4.0, seed=21)
    P.w[:10] = 0.0  # a few test particles (pushed, not deposited)
    Po = load_same_particles(g, sim, P)
    for _ in range(6):
        orc.step(g, F, Po, pusher=pusher)
    sim.step(6)
    sim.sync()
    compare_fields(g, F, sim, TOL64)
    compare_particles(g, Po, sim, TOL64)


@pytest.mark.parametrize("n", [(2100, 3), (1001, 2, 2)])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_current_correction_long_rows(pic, precision, n):
    """x1 current correction (Sec. 3.3) on rows spanning several 1024-cell
    segments with a ragged last one (and a 3D grid whose rows are not a multiple
    of 16 bytes), against the oracle's exact per-row DFT; particles fill every
    row with current.  The three correction forms agree bit for bit on the same
    deposited current."""
    cE, cB = load_table(16, 0.25, 0.3)
    dx = (DX1, DX2, DX2)[:len(n)]
    g, _ = make_pair(pic, n, cE, cB, dt=0.25 * DX1, precision=precision)
    F = load_same_fields(g, _, amp=1.0)
    P = inputs.random_particles(n, dx, 6000, umax=3.0, seed=33)
    Po = load_same_particles(g, _, P)
    _.close()
    for _i in range(3):
        orc.step(g, F, Po)
    got = {}
    for path in (0, 1, 2, 3):
        g2, sim = make_pair(pic, n, cE, cB, dt=0.25 * DX1, precision=precision)
        assert sim.info().correction_active == 1
        sim.set_correction_path(path)
        load_same_fields(g2, sim, amp=1.0)
        load_same_particles(g2, sim, P)
        sim.step(3)
        sim.sync()
        if precision == "fp64":
            compare_fields(g, F, sim, TOL64)
            compare_particles(g, Po, sim, TOL64)
        else:
            errf = max(rel(sim.read_field(nm), getattr(F, nm)) for nm in NAMES6)
            assert errf < 5e-6, errf
        sim.close()
    # Bit-identity of the forms needs the same J1 going in: atomically deposited
    # sums of several particles per cell differ in their last bits from run to
    # run, so here particles sit 10 cells apart in x1 (one deposit per J cell).
    xs = [np.arange(5.3, n[0] - 5, 10.0) * DX1]
    xs += [np.full(len(xs[0]), 0.6 * d) for d in dx[1:]]
    us = [np.full(len(xs[0]), v) for v in (0.7, -0.4, 0.3)]
    for path in (0, 1, 2, 3):
        g2, sim = make_pair(pic, n, cE, cB, dt=0.25 * DX1, precision=precision)
        sim.set_correction_path(path)
        load_same_fields(g2, sim, amp=1.0)
        sim.load_particles(xs, us, np.ones(len(xs[0])), -1.0)
        sim.step(3)
        got[path] = [sim.read_field(nm) for nm in NAMES6 + ("j1",)]
        sim.close()
    assert np.abs(got[0][-1]).max() > 0
    for path in (1, 2, 3):
        for a, b in zip(got[0], got[path]):
            assert np.array_equal(a, b), path


def test_straggler_path_parity(pic):
    # rebinning disabled: particles drift out of their tile windows and take
    # the global-memory path; results must not change
    cE, cB = load_table(16, 0.5, 0.3)
    n = (64, 32)
    g, sim = make_pair(pic, n, cE, cB)
    F = load_same_fields(g, sim, amp=1.0)
    P = inputs.random_particles(n, (DX1, DX2), 1500, umax=20.0, seed=3)
    Po = load_same_particles(g, sim, P)
    from paper_2004_03754_gb300 import pic as Pm
    Pm.pic_set_sort_interval(sim.ctx, 1 << 30)
    strag = 0
    for _ in range(12):
        orc.step(g, F, Po)
        sim.step(1)
        strag += sim.info().last_stragglers
    assert strag > 0
    compare_fields(g, F, sim, TOL64)
    compare_particles(g, Po, sim, TOL64)


def test_edge_cases(pic):
    cE, cB = load_table(16, 0.5, 0.3)
    # empty particle set
    g, sim = make_pair(pic, (32, 8), cE, cB)
    sim.load_particles([np.zeros(0)] * 2, [np.zeros(0)] * 3, np.zeros(0))
    F = load_same_fields(g, sim)
    orc.step(g, F, None, nsteps=2)
    sim.step(2)
    compare_fields(g, F, sim, TOL64)
    # one particle on a grid smaller than a particle tile, starting at x = 0
    g, sim = make_pair(pic, (8, 4), cE, cB)
    F = load_same_fields(g, sim, seed=9)
    P = inputs.ParticleSet([np.array([0.0]), np.array([3.9 * DX2])], [np.array([0.9]), np.array([-0.5]), np.array([0.2])],
                           np.array([-0.3]))
    Po = load_same_particles(g, sim, P)
    for _ in range(5):
        orc.step(g, F, Po)
    sim.step(5)
    compare_fields(g, F, sim, TOL64)
    compare_particles(g, Po, sim, TOL64)
    # zero steps is a no-op
    sim.step(0)
    # invalid arguments are rejected, not crashed on
    from paper_2004_03754_gb300 import pic as Pm
    with pytest.raises(Pm.PicError):
        sim.load_particles([np.array([-1.0]), np.array([0.0])], [np.zeros(1)] * 3, np.zeros(1))
    with pytest.raises(Pm.PicError):
        Pm.pic_read_field(sim.ctx, 42, np.zeros(g.shape))


# --------------------------------------------------------------------------
# Reduced precision: FP32 fields / FP64 pusher against the FP64 oracle
# --------------------------------------------------------------------------

@pytest.mark.parametrize("pusher", ["boris", "hc"])
def test_mixed_precision_error_is_stated(pic, pusher):
    cE, cB = load_table(16, 0.5, 0.3)
    n = (128, 32)
    g, sim = make_pair(pic, n, cE, cB, precision="mixed", pusher=pusher)
    F = load_same_fields(g, sim, amp=1.0)
    P = inputs.random_particles(n, (DX1, DX2), 4000, umax=2.0, seed=5)
    Po = load_same_particles(g, sim, P)
    for _ in range(5):
        orc.step(g, F, Po, pusher=pusher)
    sim.step(5)
    sim.sync()
    errf = max(rel(sim.read_field(nm), getattr(F, nm)) for nm in NAMES6)
    x, u, _ = sim.read_particles()
    erru = max(rel(u[c], Po.u[c]) for c in range(3))
    # FP32 storage of fields: ~1e-7 relative per value, a few steps of growth
    assert errf < 5e-6, errf
    assert erru < 5e-6, erru


def test_single_electron_energy_mixed_vs_fp64(pic):
    # Precision bar for the reduced form: single-electron energy
    # within 1e-4 relative of the FP64 oracle (plane wave, electron at rest).
    cE, cB = load_table(16, 0.5, 0.3)
    n = (256, 4)
    res = {}
    for prec in ("mixed", "fp64"):
        g, sim = make_pair(pic, n, cE, cB, precision=prec)
        sim.load_laser(a0=3.0, L_env=6 * np.pi, x_front=80 * DX1)
        sim.load_particles([np.array([84 * DX1]), np.array([0.5 * DX2])], [np.zeros(1)] * 3, np.zeros(1))
        sim.step(150)
        _, u, _ = sim.read_particles()
        res[prec] = math.sqrt(1 + sum(float(c[0]) ** 2 for c in u)) - 1
    g = orc.Grid(n, (DX1, DX2), DT, cE, cB)
    F = orc.Fields(g)
    orc.laser_load(g, F, a0=3.0, Lenv=6 * np.pi, x_front=80 * DX1)
    Po = orc.Particles([np.array([84 * DX1]), np.array([0.5 * DX2])], [np.zeros(1)] * 3, np.zeros(1))
    orc.step(g, F, Po, nsteps=150)
    ref = math.sqrt(1 + sum(float(c[0]) ** 2 for c in Po.u)) - 1
    assert ref > 0.5
    assert abs(res["fp64"] - ref) <= 1e-12 * ref
    assert abs(res["mixed"] - ref) <= 1e-4 * ref
