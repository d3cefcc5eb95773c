"""The product's momentum pushers (csrc/pushers.cuh) compiled for the host and
compared with the oracle's pushers, CPU: Boris (Sec. 1), Higuera-Cary (Sec. 1,
Sec. 4.1) and the analytic constant-field push (Sec. 1, Sec. 4.1), on weak,
strong and null (plane-wave) fields.  The GPU parity tests check the same code
on the device; this keeps every commit checked without one."""
import os
import shutil
import struct
import subprocess

import numpy as np
import pytest

from oracle import oracle as orc

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_2004_03754_gb300", "csrc")
KINDS = {0: orc.boris, 2: orc.hc}


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path_factory.mktemp("push") / "push_check_host")
    subprocess.check_call([cxx, "-O2", "-std=c++17", "-Wno-unknown-pragmas", "-I", CSRC,
                           "-I", os.path.join(ROOT, "include"), "-o", exe,
                           os.path.join(HERE, "native", "push_check_host.cpp")])
    return exe


def _cases():
    rng = np.random.Generator(np.random.PCG64(17))
    out = []
    for scale in (0.3, 3.0, 30.0):
        for _ in range(20):
            out.append((rng.uniform(-scale, scale, 6), rng.uniform(-8, 8, 3)))
    for E in (0.5, 5.0, 50.0):
        out.append((np.array([0.0, E, 0.0, 0.0, 0.0, E]), np.array([20.0, 1.0, -0.5])))
        out.append((np.array([0.0, E, 0.0, 0.0, 0.0, E]), np.zeros(3)))
    return out


@pytest.mark.parametrize("kind", [0, 1, 2], ids=["boris", "analytic", "hc"])
def test_product_pushers_equal_the_oracle(harness, tmp_path, kind):
    qm, dt = -1.0, 0.0981747704
    cases = _cases()
    fin, fout = tmp_path / "in.bin", tmp_path / "out.bin"
    with open(fin, "wb") as f:
        f.write(struct.pack("<i", len(cases)))
        for eb, u in cases:
            f.write(struct.pack("<i", kind))
            f.write(np.concatenate([[qm, dt], eb, u]).astype("<f8").tobytes())
    subprocess.check_call([harness, str(fin), str(fout)])
    got = np.fromfile(fout, dtype="<f8").reshape(len(cases), 4)
    for (eb, u), g in zip(cases, got):
        if kind == 1:
            ref, it = orc.analytic(qm, dt, eb, u)
            assert it > 0 and g[3] > 0
        else:
            ref = KINDS[kind](qm, dt, eb, u)
        scale = max(np.abs(ref).max(), 1.0)
        assert np.abs(g[:3] - ref).max() <= 1e-13 * scale, (kind, eb, u, g[:3], ref)
