"""One step of the product's particle update (csrc/particle_core.cuh: gather of
E^n and the time-centred B^n with the quadratic spline (App. A), Boris / HC /
analytic push, FP64 move, Esirkepov deposit (Sec. 3.3)) compiled by nvcc and
run on the host, against the oracle's step: positions, momenta and the
deposited current.  CPU only (no device); the GPU parity tests check the same
code on the device."""
import os
import shutil
import struct
import subprocess

import numpy as np
import pytest

from oracle import oracle as orc
from oracle.gen_tables import load as load_table
from paper_2004_03754_gb300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_2004_03754_gb300", "csrc")
DX1, DX2, DT = inputs.DX1, inputs.DX2, inputs.DT
PUSHERS = {"boris": 0, "analytic": 1, "hc": 2}


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc"
                                    if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("no nvcc")
    exe = str(tmp_path_factory.mktemp("pch") / "particle_check_host")
    subprocess.check_call([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-std=c++17",
                           "--expt-relaxed-constexpr", "-diag-suppress", "128", "-I", CSRC,
                           "-I", os.path.join(ROOT, "include"), "-o", exe,
                           os.path.join(HERE, "native", "particle_check_host.cu")])
    return exe


def _check(harness, tmp_path, n, pusher, precision, seed, form=0):
    cE, cB = load_table(16, 0.5, 0.3)                  # C^B = e_1: J as deposited
    nd = len(n)
    dx = (DX1, DX2, DX2)[:nd]
    g = orc.Grid(n, dx, DT, cE, cB)
    F = orc.Fields(g)
    for nm, a in zip(("e1", "e2", "e3", "b1", "b2", "b3"),
                     inputs.random_fields(g.shape, amp=1.0, seed=seed)[:6]):
        getattr(F, nm)[...] = a
    P = inputs.random_particles(n, dx, 3000, umax=4.0, seed=seed + 1)
    if form == 0:                                      # time-centred B^n of this state
        bb = orc.bbar(g, F)
        fields = [F.e1, F.e2, F.e3, bb[0], bb[1], bb[2]]
    else:                                              # B^{n-1/2}: the product forms B^n
        fields = [F.e1, F.e2, F.e3, F.b1.copy(), F.b2.copy(), F.b3.copy()]
    Po = orc.Particles(P.x, P.u, P.w, -1.0)
    Fo = F.copy()
    orc.step(g, Fo, Po, pusher=pusher)

    n3 = n[2] if nd == 3 else 1
    fin, fout = tmp_path / "in.bin", tmp_path / "out.bin"
    with open(fin, "wb") as f:
        f.write(struct.pack("<6i", n[0], n[1], n3, PUSHERS[pusher], 1 if precision == "fp32" else 0,
                            form))
        f.write(struct.pack("<5d", DX1, DX2, DX2 if nd == 3 else 1.0, DT, -1.0))
        if form:
            f.write(struct.pack("<i", cE.size))
            f.write(np.asarray(cE, dtype="<f8").tobytes())
        for a in fields:
            f.write(np.ascontiguousarray(a, dtype="<f8").tobytes())
        f.write(struct.pack("<q", P.n))
        for a in (*P.x, P.u[0], P.u[1], P.u[2], P.w):
            f.write(np.ascontiguousarray(a, dtype="<f8").tobytes())
    subprocess.check_call([harness, str(fin), str(fout)])
    out = np.fromfile(fout, dtype="<f8")
    np_, nc = P.n, int(np.prod(n))
    x = out[:nd * np_].reshape(nd, np_)
    u = out[nd * np_:(nd + 3) * np_].reshape(3, np_)
    J = out[(nd + 3) * np_:(nd + 3) * np_ + 3 * nc].reshape((3,) + g.shape)
    assert out[-1] == 0.0                              # no error latched

    tol = 1e-12 if precision == "fp64" else 2e-6       # FP32 fields, gather and deposit
    for c in range(3):
        assert np.abs(u[c] - Po.u[c]).max() <= tol * np.abs(Po.u[c]).max(), c
    for d in range(nd):
        L = g.length[d]
        assert np.abs((x[d] - Po.x[d] + L / 2) % L - L / 2).max() <= max(tol, 1e-12) * L
    for c, ref in enumerate((Fo.j1, Fo.j2, Fo.j3)):
        assert np.abs(J[c] - ref).max() <= tol * np.abs(ref).max(), c


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("pusher", ["boris", "analytic", "hc"])
def test_particle_update_equals_the_oracle_step_2d(harness, tmp_path, pusher, precision):
    _check(harness, tmp_path, (40, 12), pusher, precision, 23)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("pusher", ["boris", "analytic"])
def test_particle_update_equals_the_oracle_step_3d(harness, tmp_path, pusher, precision):
    _check(harness, tmp_path, (20, 10, 8), pusher, precision, 41)


@pytest.mark.parametrize("n", [(40, 12), (20, 10, 8)])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_time_centred_b_formed_on_the_fly(harness, tmp_path, n, precision):
    # the straggler and ensemble paths form B^n = B^{n-1/2} - (dt/2) d_E x E^n
    # while gathering (Eq. (7)); the oracle averages B^{n-1/2} and B^{n+1/2}
    _check(harness, tmp_path, n, "boris", precision, 57, form=1)
