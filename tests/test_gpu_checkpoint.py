"""Checkpoint / resume (pic_save_state, pic_load_state).

A run saved after k steps and resumed in a fresh context continues exactly as
the uninterrupted run: bit for bit when no particle deposits (the only
non-associative step, the atomic current deposit, is then absent), and to the
FP64 oracle at 1e-12 with depositing particles and the x1 current correction.
States from another configuration, truncated or foreign buffers are refused.
"""
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


def _sim(P, n, cE, cB, dt, precision="fp64"):
    # re-binning every step: each particle then takes the tiled path at every step
    # in the saved and in the resumed run alike (their binning histories differ)
    dx = (DX1, DX2, DX2)[:len(n)]
    sim = P.Simulation(n, dx, dt, cE, cB, precision=precision, pusher="boris")
    P.pic_set_sort_interval(sim.ctx, 1)
    return sim


def _load(sim, n, seed, depositing, npart=3000):
    dx = (DX1, DX2, DX2)[:len(n)]
    fs = inputs.random_fields(tuple(n[::-1]), amp=0.5, seed=seed)
    for nm, a in zip(NAMES6, fs[:6]):
        sim.load_field(nm, a)
    ps = inputs.random_particles(n, dx, npart, umax=2.0, seed=seed + 1)
    if not depositing:
        ps.w[:] = 0.0
    sim.load_particles(ps.x, ps.u, ps.w, -1.0)
    return fs, ps


def _state(sim):
    x, u, w = sim.read_particles()
    return [sim.read_field(nm) for nm in NAMES6] + list(x) + list(u) + [w]


@pytest.mark.parametrize("n,precision", [((96, 40), "fp64"), ((24, 12, 10), "fp64"),
                                         ((130, 33), "mixed")])
def test_resume_is_bit_identical_without_deposit(pic, n, precision):
    cE, cB = load_table(16, 0.5, 0.3)
    a = _sim(pic, n, cE, cB, DT, precision)
    _load(a, n, 11, depositing=False)
    a.step(7)
    saved = a.save_state()
    assert saved.nbytes == pic.pic_state_size(a.ctx)
    a.step(5)
    ref = _state(a)
    assert a.info().steps_done == 12
    b = _sim(pic, n, cE, cB, DT, precision)
    b.load_state(saved)
    assert b.info().steps_done == 7
    b.step(5)
    got = _state(b)
    for r, g in zip(ref, got):
        assert np.array_equal(r, g)
    # a state saved again right after loading is the same bytes
    c = _sim(pic, n, cE, cB, DT, precision)
    c.load_state(saved)
    assert np.array_equal(c.save_state(), saved)
    for s in (a, b, c):
        s.close()


def test_resume_with_deposit_and_correction_matches_oracle(pic):
    # dt/dx1 = 1/4 tables: C^B != e_1, so the x1 current correction runs
    cE, cB = load_table(16, 0.25, 0.3)
    n, dt = (96, 24), 0.25 * DX1
    a = _sim(pic, n, cE, cB, dt)
    fs, ps = _load(a, n, 21, depositing=True)
    a.step(6)
    saved = a.save_state()
    a.close()
    b = _sim(pic, n, cE, cB, dt)
    b.load_state(saved)
    b.step(4)
    b.sync()
    g = orc.Grid(n, (DX1, DX2), dt, cE, cB)
    F = orc.Fields(g)
    for nm, arr in zip(NAMES6, fs[:6]):
        getattr(F, nm)[...] = arr
    Po = orc.Particles(ps.x, ps.u, ps.w, -1.0)
    orc.step(g, F, Po, nsteps=10)
    for nm in NAMES6:
        ref = getattr(F, nm)
        assert np.abs(b.read_field(nm) - ref).max() <= 1e-12 * np.abs(ref).max(), nm
    x, u, _ = b.read_particles()
    for c in range(3):
        assert np.abs(u[c] - Po.u[c]).max() <= 1e-12 * np.abs(Po.u[c]).max()
    for d in range(2):
        L = g.length[d]
        assert np.abs((x[d] - Po.x[d] + L / 2) % L - L / 2).max() <= 1e-12 * L
    b.close()


def test_foreign_or_damaged_states_are_refused(pic):
    cE, cB = load_table(16, 0.5, 0.3)
    n = (64, 16)
    a = _sim(pic, n, cE, cB, DT)
    _load(a, n, 3, depositing=True, npart=500)
    a.step(2)
    saved = a.save_state()
    b = _sim(pic, n, cE, cB, 0.9 * DT)           # another time step
    with pytest.raises(pic.PicError):
        b.load_state(saved)
    c = _sim(pic, (64, 17), cE, cB, DT)           # another grid
    with pytest.raises(pic.PicError):
        c.load_state(saved)
    d = _sim(pic, n, cE, cB, DT, "mixed")         # another precision
    with pytest.raises(pic.PicError):
        d.load_state(saved)
    e = _sim(pic, n, cE, cB, DT)
    with pytest.raises(pic.PicError):
        e.load_state(saved[: saved.nbytes - 8])   # truncated
    bad = saved.copy()
    bad[0] ^= 0xFF                                # not a state
    with pytest.raises(pic.PicError):
        e.load_state(bad)
    e.load_state(saved)                           # the context is still usable
    e.step(1)
    e.sync()
    for s in (a, b, c, d, e):
        s.close()
