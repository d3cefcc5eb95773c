"""Ensembles (persistent kernel over many independent runs) against the oracle.

Each run of the ensemble is an independent PIC simulation; the oracle runs
them one by one.  FP64 ensembles must match to 1e-12; the reduced form (FP32
fields, FP64 analytic pusher) states its error.
"""
import math

import numpy as np
import pytest

from oracle import oracle as orc
from oracle.gen_tables import load as load_table
from paper_2004_03754_gb300 import inputs

pytestmark = pytest.mark.gpu

DX1, DX2, DT = inputs.DX1, inputs.DX2, inputs.DT


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2004_03754_gb300 import pic
    return pic


def _setup(P, sizes, precision, pusher, depositing, seed=3, table=(16, 0.5, 0.3), dt=DT):
    cE, cB = load_table(*table)
    n1 = [s[0] for s in sizes]
    n2 = [s[1] for s in sizes]
    import torch
    stream = torch.cuda.Stream()   # a real stream, so the run goes through a CUDA graph
    ens = P.Ensemble(n1, n2, (DX1, DX2), dt, cE, cB, precision=precision, pusher=pusher,
                     stream=stream.cuda_stream)
    ens._stream = stream
    lasers, parts = [], []
    g = inputs.rng(seed)
    for r, (a, b) in enumerate(sizes):
        L = min(6 * np.pi, 0.5 * a * DX1)
        lasers.append(P.pic_laser(float(2.0 + r), 1.0, 0.2 * r, L, L + 4 * DX1,
                                  3.0 if r % 2 else 0.0, b * DX2 / 2, 0.0))
        npart = 40 + 10 * r
        ps = inputs.random_particles((a, b), (DX1, DX2), npart, umax=1.5, seed=seed + r)
        if not depositing:
            ps.w[:] = 0.0
        parts.append(ps)
    ens.load_lasers(lasers)
    counts = [p.n for p in parts]
    x = [np.concatenate([p.x[d] for p in parts]) for d in range(2)]
    u = [np.concatenate([p.u[c] for p in parts]) for c in range(3)]
    w = np.concatenate([p.w for p in parts])
    ens.load_particles(counts, x, u, w)
    return ens, lasers, parts, cE, cB


def _oracle_run(size, las, ps, cE, cB, nsteps, pusher, dt=DT):
    g = orc.Grid(size, (DX1, DX2), dt, cE, cB)
    F = orc.Fields(g)
    orc.laser_load(g, F, a0=las.a0, k0=las.k0, phase=las.phase, Lenv=las.L_env,
                   x_front=las.x_front, w0=las.w0, x2c=las.x2c)
    Po = orc.Particles(ps.x, ps.u, ps.w)
    orc.step(g, F, Po, pusher=pusher, nsteps=nsteps)
    return g, F, Po


@pytest.mark.parametrize("depositing", [False, True])
def test_ensemble_fp64_matches_oracle(P, depositing):
    # widths that are and are not 16-byte multiples, several strips with a ragged
    # last one, and a run narrower than the rows' ghost columns (element copies)
    sizes = [(96, 16), (131, 20), (64, 9), (200, 12), (448, 10), (251, 7), (24, 6)]
    ens, lasers, parts, cE, cB = _setup(P, sizes, "fp64", "boris", depositing)
    nsteps = [7, 3, 0, 11, 5, 9, 4]
    ens.set_steps(nsteps)
    ens.run()
    info = ens.info()
    assert info.has_current == (1 if depositing else 0)
    assert info.graph == 1
    x, u, _ = ens.read_particles()
    off = 0
    for r, size in enumerate(sizes):
        g, F, Po = _oracle_run(size, lasers[r], parts[r], cE, cB, nsteps[r], "boris")
        for nm in ("e1", "e2", "e3", "b1", "b2", "b3"):
            ref = getattr(F, nm)
            got = ens.read_field(r, nm)
            assert np.abs(got - ref).max() <= 1e-12 * max(np.abs(ref).max(), 1e-300), (r, nm)
        n = parts[r].n
        for c in range(3):
            ref = Po.u[c]
            assert np.abs(u[c][off:off + n] - ref).max() <= 1e-12 * max(np.abs(ref).max(), 1e-300)
        for d in range(2):
            L = g.length[d]
            dxp = (x[d][off:off + n] - Po.x[d] + L / 2) % L - L / 2
            assert np.abs(dxp).max() <= 1e-12 * L
        off += n
    # a second run continues from the state (parities carried per run)
    ens.set_steps([2] * len(sizes))
    ens.run()
    g, F, Po = _oracle_run(sizes[1], lasers[1], parts[1], cE, cB, nsteps[1] + 2, "boris")
    ref = F.e2
    assert np.abs(ens.read_field(1, "e2") - ref).max() <= 1e-12 * np.abs(ref).max()
    ens.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_ensemble_current_correction_matches_oracle(P, precision):
    # Delta t/Delta x1 = 1/4 tables: C^B != e_1, so every step corrects each run's
    # deposited J1 along x1 (Sec. 3.3) with the taps of its own n1: runs shorter
    # than the tap set (full circulant) and than the ghost width, ragged rows,
    # and runs longer than one 1024-cell segment
    sizes = [(24, 6), (50, 5), (131, 9), (200, 7), (1100, 4), (64, 3)]
    dt = 0.25 * DX1
    ens, lasers, parts, cE, cB = _setup(P, sizes, precision, "boris", True,
                                        table=(16, 0.25, 0.3), dt=dt)
    nsteps = [5, 3, 6, 0, 4, 7]
    ens.set_steps(nsteps)
    ens.run()
    info = ens.info()
    assert info.has_current == 1 and info.correction_active == 1
    x, u, _ = ens.read_particles()
    tol = 1e-12 if precision == "fp64" else 2e-5
    off = 0
    for r, size in enumerate(sizes):
        g, F, Po = _oracle_run(size, lasers[r], parts[r], cE, cB, nsteps[r], "boris", dt=dt)
        names = ("e1", "e2", "e3", "b1", "b2", "b3")
        # FP32 storage errors scale with the run's largest field (the laser)
        scale = max(np.abs(getattr(F, nm)).max() for nm in names)
        for nm in names:
            ref = getattr(F, nm)
            got = ens.read_field(r, nm)
            ref_scale = np.abs(ref).max() if precision == "fp64" else scale
            assert np.abs(got - ref).max() <= tol * max(ref_scale, 1e-300), (r, nm)
        n = parts[r].n
        for c in range(3):
            ref = Po.u[c]
            assert np.abs(u[c][off:off + n] - ref).max() <= tol * max(np.abs(ref).max(), 1e-300)
        off += n
    ens.close()


def test_ensemble_mixed_analytic_error_is_stated(P):
    sizes = [(128, 8), (161, 12), (803, 8)]
    ens, lasers, parts, cE, cB = _setup(P, sizes, "mixed", "analytic", False)
    ens.set_steps([20, 20, 20])
    ens.run()
    x, u, _ = ens.read_particles()
    off = 0
    for r, size in enumerate(sizes):
        g, F, Po = _oracle_run(size, lasers[r], parts[r], cE, cB, 20, "analytic")
        n = parts[r].n
        for c in range(3):
            ref = Po.u[c]
            assert np.abs(u[c][off:off + n] - ref).max() <= 1e-5 * max(np.abs(ref).max(), 1.0)
        off += n
    ens.close()


def test_ensemble_barrier_timeout_returns_error(P):
    sizes = [(64, 8), (96, 8)]
    ens, *_ = _setup(P, sizes, "mixed", "boris", False)
    ens.set_steps([3, 3])
    # every barrier waits for one CTA more than the launch has: each bounded
    # wait runs out and the run reports a timeout instead of hanging
    P.pic_batch_set_barrier(ens.b, 0.2, impossible=True)
    with pytest.raises(P.PicError) as e:
        ens.run()
    assert e.value.status == P.PIC_ERR_TIMEOUT
    # the context stays usable
    P.pic_batch_set_barrier(ens.b, 5.0, impossible=False)
    ens.run()
    assert np.isfinite(ens.read_field(0, "e2")).all()
    ens.close()


def test_ensemble_autotune_keeps_results(P):
    sizes = [(300, 20), (512, 16), (257, 9)]
    res = []
    for tune in (False, True):
        ens, lasers, parts, cE, cB = _setup(P, sizes, "fp64", "boris", True, seed=11)
        if tune:
            # autotune advances and then clears the state: reload afterwards
            ens.autotune(3)
            ens.load_lasers(lasers)
            counts = [p.n for p in parts]
            ens.load_particles(counts, [np.concatenate([p.x[d] for p in parts]) for d in range(2)],
                               [np.concatenate([p.u[c] for p in parts]) for c in range(3)],
                               np.concatenate([p.w for p in parts]))
        ens.set_steps([5, 4, 6])
        ens.run()
        res.append([ens.read_field(r, "e2") for r in range(3)])
        tile = tuple(ens.info().tile)
        ens.close()
    for a, b in zip(*res):
        assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()
    assert tile in ((96, 32), (160, 32), (224, 32), (160, 16))   # FP64 strip candidates
