"""The integer-pipe FP32 <-> FP64 conversions of the particle kernels (widening of
the gathered fields, narrowing and widening of the Newton seeds, the exact cell
floor/fraction split) give the hardware conversion's bits on their operand
domains.  The check program is built with nvcc and run on the GPU."""
import os
import shutil
import subprocess

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2004_03754_gb300", "csrc")


def test_integer_conversions_match_hardware(tmp_path):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    exe = str(tmp_path / "conv_check")
    subprocess.check_call([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                           "-I", CSRC, "-o", exe, os.path.join(HERE, "native", "conv_check.cu")])
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    print(r.stdout)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "mismatches: widen 0  narrow_pos/widen_pos 0  floor_split 0" in r.stdout
