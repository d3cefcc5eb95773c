"""The particle kernels' integer-pipe FP32 <-> FP64 conversions and cell
floor/fraction split (csrc/fpbits.cuh) compiled for the host and checked
against the compiler's IEEE conversions on their operand domains (CPU; the GPU
build is checked the same way by test_gpu_conversions.py)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2004_03754_gb300", "csrc")


def test_integer_conversions_match_ieee_on_the_host(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path / "conv_check_host")
    subprocess.check_call([cxx, "-O2", "-std=c++17", "-I", CSRC, "-o", exe,
                           os.path.join(HERE, "native", "conv_check_host.cpp")])
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    print(r.stdout)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "widen 0  narrow_pos 0  widen_pos 0  floor_split 0  narrow_signed 0" in r.stdout
