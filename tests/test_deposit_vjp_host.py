"""Reverse mode of the Esirkepov deposit (Sec. 3.3, Eq. (24)) used by the adjoint
of depositing particles (csrc/deposit_vjp.cuh: the product's deposit template on
dual numbers), compiled by nvcc and run on the host, against central
differences of the ORACLE's deposit: for random adjoint grids lambda and random
sub-cell moves, d/d(x^n, x^{n+1}, v3) of sum_c <lambda_c, J_c>.  CPU only."""
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
    exe = str(tmp_path_factory.mktemp("dvjp") / "deposit_vjp_check_host")
    subprocess.check_call([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-std=c++17",
                           "--expt-relaxed-constexpr", "-I", CSRC, "-I", os.path.join(ROOT, "include"),
                           "-o", exe, os.path.join(HERE, "native", "deposit_vjp_check_host.cu")])
    return exe


def _oracle_objective(g, lam, w, xo, xn, v3):
    """sum_c <lambda_c, J_c> of one particle's deposit, by the oracle."""
    F = orc.Fields(g)
    assert orc.deposit(g, F, w, xo, xn, v3) == 0
    return float(np.sum(lam[0] * F.j1) + np.sum(lam[1] * F.j2) + np.sum(lam[2] * F.j3))


def test_deposit_vjp_matches_oracle_central_differences(harness, tmp_path):
    n = (16, 12)
    cE, cB = load_table(16, 0.5, 0.3)
    g = orc.Grid(n, (DX1, DX2), DT, cE, cB)
    r = inputs.rng(29)
    lam = [r.standard_normal(g.shape) for _ in range(3)]
    m = 120
    r0 = np.stack([r.uniform(0, n[0], m), r.uniform(0, n[1], m)], 1)
    r0[:8, 0] = [0.01, 0.49, 0.5, 0.51, 15.99, 3.0, 7.25, 0.75]   # node / half-node / seam cases
    dl = r.uniform(-0.9, 0.9, (m, 2))
    dl[:4, 0] = [0.0, -0.6, 0.6, 0.02]
    w = r.uniform(0.5, 2.0, m)
    v3 = r.uniform(-0.9, 0.9, m)
    fin, fout = tmp_path / "in.bin", tmp_path / "out.bin"
    with open(fin, "wb") as f:
        f.write(struct.pack("<2i", *n))
        f.write(struct.pack("<3d", DX1, DX2, DT))
        for a in lam:
            f.write(np.ascontiguousarray(a, dtype="<f8").tobytes())
        f.write(struct.pack("<q", m))
        f.write(np.ascontiguousarray(np.column_stack([r0, dl, w, v3]), dtype="<f8").tobytes())
    subprocess.check_call([harness, str(fin), str(fout)])
    got = np.fromfile(fout, dtype="<f8").reshape(m, 5)

    dx = np.array([DX1, DX2])
    h = 1e-7   # cells
    scale = 0.0
    errs = []
    for q in range(m):
        xo = r0[q] * dx
        xn = (r0[q] + dl[q]) * dx
        L = lambda a, b, v=v3[q]: _oracle_objective(g, lam, w[q], a, b, v)
        d_xo, d_xn = np.zeros(2), np.zeros(2)
        for d in range(2):
            e = np.zeros(2)
            e[d] = h * dx[d]
            d_xo[d] = (L(xo + e, xn) - L(xo - e, xn)) / (2 * h * dx[d])
            d_xn[d] = (L(xo, xn + e) - L(xo, xn - e)) / (2 * h * dx[d])
        # J is linear in v3: one difference is exact up to rounding
        d_v3 = (L(xo, xn, v3[q] + 0.5) - L(xo, xn, v3[q] - 0.5))
        # r0 moves both ends (delta held), delta moves the end only; j3f = w v3
        want = np.array([dx[0] * (d_xo[0] + d_xn[0]), dx[1] * (d_xo[1] + d_xn[1]),
                         dx[0] * d_xn[0], dx[1] * d_xn[1], d_v3 / w[q]])
        scale = max(scale, float(np.max(np.abs(want))))
        errs.append(np.abs(got[q] - want))
    errs = np.array(errs)
    assert scale > 1.0
    # central differences at 1e-7 cells: rounding ~1e-9 of the scale, and at most h times
    # the jump of the B-spline's second derivative where a node sits inside [-h, h]
    assert errs.max() <= 1e-7 * scale, (errs.max(), scale, np.unravel_index(errs.argmax(), errs.shape))
