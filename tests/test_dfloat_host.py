"""The compensated FP32-pair arithmetic of the reduced-precision field path
(csrc/dfloat.cuh, used by PIC_COMPENSATED) compiled for the host and checked
against FP64, which represents every FP32 sum and product exactly (CPU, no
device).  Dekker's and Knuth's error-free transformations must be exact; sums
and products of pairs must carry about 48 significant bits; results stay
normalised (|lo| <= half an ulp of hi)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_2004_03754_gb300", "csrc")


@pytest.fixture(scope="module")
def report(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path_factory.mktemp("dfl") / "dfloat_check_host")
    subprocess.check_call([cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-I", CSRC, "-o", exe,
                           os.path.join(HERE, "native", "dfloat_check_host.cpp")])
    out = subprocess.check_output([exe]).decode()
    return {k: float(v) for k, v in (l.split() for l in out.strip().splitlines())}


def test_error_free_transformations_are_exact(report):
    assert report["two_sum_exact"] == 0.0
    assert report["two_prod_exact"] == 0.0


def test_pair_arithmetic_keeps_48_bits(report):
    assert report["ctor"] <= 2.0 ** -48
    assert report["add"] <= 2.0 ** -46
    assert report["sub"] <= 2.0 ** -46
    assert report["mul"] <= 2.0 ** -45
    # and far more than single precision
    assert report["mul"] < 1e-12


def test_results_are_normalised(report):
    assert report["norm"] <= 1.0
