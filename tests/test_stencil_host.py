"""The field kernels' register-blocked x1 stencils (csrc/field_tile.cuh
x1_stencil, App. B Eqs. (B.1)-(B.2)) compiled by nvcc and run on the host over
every output of a periodic row, against the derivative the oracle's Faraday and
Ampere updates apply (CPU, no device): checks the window offsets and lengths of
every unrolled form (M up to 8, 16, 32; FP64, FP32 and compensated FP32
pairs)."""
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


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc"
                                    if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("no nvcc")
    exe = str(tmp_path_factory.mktemp("sch") / "stencil_check_host")
    subprocess.check_call([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-std=c++17",
                           "--expt-relaxed-constexpr", "-diag-suppress", "128", "-I", CSRC,
                           "-I", os.path.join(ROOT, "include"), "-o", exe,
                           os.path.join(HERE, "native", "stencil_check_host.cu")])
    return exe


def _coeffs(M):
    if M == 16:
        return load_table(16, 0.5, 0.3)
    return inputs.random_coeffs(M, seed=M)


@pytest.mark.parametrize("precision", ["fp64", "fp32", "compensated"])
@pytest.mark.parametrize("faraday", [True, False], ids=["dE", "dB"])
@pytest.mark.parametrize("M", [5, 16, 32])
def test_x1_stencils_equal_the_oracle_operators(harness, tmp_path, M, faraday, precision):
    cE, cB = _coeffs(M)
    n1 = 101                                             # ragged against every V
    g = orc.Grid((n1, 2), (DX1, DX2), DT, cE, cB)
    row = inputs.rng(M + 7).uniform(-1, 1, n1)
    F = orc.Fields(g)
    if faraday:                                          # B3 -= h d^E E2 (E2 uniform in x2)
        F.e2[...] = row
        orc.faraday(g, F, 1.0)
        ref = -F.b3[0]
        k = cE / DX1
    else:                                                # E2 += h (-d^B B3)
        F.b3[...] = row
        orc.ampere(g, F, 1.0)
        ref = -F.e2[0]
        k = cB / DX1
    fin, fout = tmp_path / "in.bin", tmp_path / "out.bin"
    with open(fin, "wb") as f:
        f.write(struct.pack("<4i", n1, M, 1 if faraday else 0,
                            {"fp64": 0, "fp32": 1, "compensated": 2}[precision]))
        f.write(row.astype("<f8").tobytes())
        f.write(np.asarray(k, dtype="<f8").tobytes())
    subprocess.check_call([harness, str(fin), str(fout)])
    got = np.fromfile(fout, dtype="<f8")
    # compensated: inputs rounded to 48 bits, ~2^-46 per tap
    tol = {"fp64": 1e-13, "fp32": 2e-6, "compensated": 2e-13}[precision]
    assert np.abs(got - ref).max() <= tol * np.abs(ref).max()
