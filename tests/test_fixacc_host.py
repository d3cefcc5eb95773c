"""Fixed-point current window of the 2D particle kernel (csrc/particle_core.cuh:
fix_scales, fix_encode), compiled by nvcc and run on the host, checked in exact
arithmetic: the per-tile scales keep both int32 sums from overflowing for any
n contributions bounded by `bound`, each contribution is encoded as
v S = ih + il/L + e with |e| <= 1/(2L), and a sum of many contributions of
mixed sign and size decodes to the exact sum within n/(2SL) plus the FP32
rounding of the result.  CPU only."""
import math
import os
import shutil
import struct
import subprocess
from fractions import Fraction

import numpy as np
import pytest

from paper_2004_03754_gb300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_2004_03754_gb300", "csrc")
I31 = 2 ** 31


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc"
                                    if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("no nvcc")
    exe = str(tmp_path_factory.mktemp("fix") / "fixacc_check_host")
    subprocess.check_call([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-std=c++17",
                           "--expt-relaxed-constexpr", "-I", CSRC, "-I", os.path.join(ROOT, "include"),
                           "-o", exe, os.path.join(HERE, "native", "fixacc_check_host.cu")])
    return exe


def _run(harness, tmp_path, pairs, vals, pairs64=(), vals64=()):
    fin, fout = tmp_path / "in.bin", tmp_path / "out.bin"
    with open(fin, "wb") as f:
        f.write(struct.pack("<q", len(pairs)))
        for n, b in pairs:
            f.write(struct.pack("<qf", n, b))
        f.write(struct.pack("<q", len(vals)))
        f.write(np.asarray(vals, dtype="<f4").reshape(-1).tobytes())
        f.write(struct.pack("<q", len(pairs64)))
        for n, b in pairs64:
            f.write(struct.pack("<qd", n, b))
        f.write(struct.pack("<q", len(vals64)))
        for v, e, l in vals64:
            f.write(struct.pack("<dii", v, e, l))
    subprocess.check_call([harness, str(fin), str(fout)])
    raw = open(fout, "rb").read()
    o = 0
    sl = np.frombuffer(raw[o:o + 8 * len(pairs)], dtype="<f4").reshape(-1, 2)
    o += 8 * len(pairs)
    enc = np.frombuffer(raw[o:o + 8 * len(vals)], dtype="<i4").reshape(-1, 2)
    o += 8 * len(vals)
    if not pairs64 and not vals64:
        return sl.astype(np.float64), enc.astype(np.int64)
    el = np.frombuffer(raw[o:o + 8 * len(pairs64)], dtype="<i4").reshape(-1, 2)
    o += 8 * len(pairs64)
    abc = np.frombuffer(raw[o:o + 12 * len(vals64)], dtype="<i4").reshape(-1, 3)
    return el.astype(np.int64), abc.astype(np.int64)


def test_scales_cannot_overflow_and_are_tight(harness, tmp_path):
    r = inputs.rng(5)
    pairs = [(1, 1.0), (4096, 2.5e-3), (4096, 0.5), (65536, 1e-4), (1 << 20, 3e-6), (7, 1e3),
             (300000, 2.0), (2, 1e-30)]
    pairs += [(int(r.integers(1, 1 << 22)), float(10 ** r.uniform(-8, 3))) for _ in range(200)]
    pairs = [(n, float(np.float32(b))) for n, b in pairs]
    sl, _ = _run(harness, tmp_path, pairs, [])
    for (n, b), (S, L) in zip(pairs, sl):
        assert S == 2.0 ** round(math.log2(S)) and L == 2.0 ** round(math.log2(L))
        assert n * (b * S + 0.5) < I31, (n, b, S)          # hi sum
        assert b * S <= 2 ** 21                             # rounding trick's range
        assert n * (L / 2 + 0.5) < I31 and L <= 2 ** 21      # lo sum
        # tight within the factor-2 margin: doubling S would leave the margin (S is
        # capped at 2^100, far above any current's resolution need)
        assert S == 2.0 ** 100 or 2 * S > min(2 ** 30 / (n * b), 2 ** 21 / b) * (1 - 1e-6), (n, b, S)


def test_encoding_is_exact_to_half_a_lo_unit(harness, tmp_path):
    r = inputs.rng(6)
    vals = []
    for _ in range(4000):
        S = float(2.0 ** r.integers(-10, 40))
        L = float(2.0 ** r.integers(0, 22))
        bound = 2 ** 21 / S
        v = float(np.float32(r.choice([-1, 1]) * bound * 10 ** r.uniform(-9, 0)))
        vals.append((v, S, L))
    vals += [(0.0, 1024.0, 65536.0), (-0.0, 8.0, 2.0), (2.0 ** 21, 1.0, 65536.0), (-(2.0 ** 21), 1.0, 65536.0),
             (0.5, 1.0, 1.0), (1.5, 1.0, 65536.0), (-2.5, 1.0, 65536.0), (float(np.float32(1e-30)), 2.0 ** 40, 65536.0)]
    _, enc = _run(harness, tmp_path, [], vals)
    for (v, S, L), (ih, il) in zip(vals, enc):
        err = Fraction(v) * Fraction(S) - ih - Fraction(int(il)) / Fraction(L)
        assert abs(err) <= Fraction(1, 2) / Fraction(L), (v, S, L, ih, il)
        assert abs(ih) <= abs(v) * S + 0.5 and abs(il) <= L / 2


def test_sums_decode_to_the_exact_sum(harness, tmp_path):
    """4096 contributions of one tile (random sign, sizes over nine decades) into one
    node: the int32 sums stay in range and decode to the exact sum within
    n/(2SL) + the FP32 rounding of the decoded value, independent of the order."""
    r = inputs.rng(7)
    n, bound = 4096, float(np.float32(3.1e-3))
    sl, _ = _run(harness, tmp_path, [(n, bound)], [])
    S, L = sl[0]
    v = (r.choice([-1.0, 1.0], n) * bound * 10 ** r.uniform(-9, 0, n)).astype(np.float32)
    _, enc = _run(harness, tmp_path, [], [(float(x), S, L) for x in v])
    hi, lo = int(enc[:, 0].sum()), int(enc[:, 1].sum())
    assert abs(hi) < I31 and abs(lo) < I31
    exact = math.fsum(float(x) for x in v)
    dec = float(np.float32(np.float32(lo) * np.float32(1 / (S * L)) + np.float32(np.float32(hi) / np.float32(S))))
    tol = n / (2 * S * L) + 2 * abs(exact) * 2.0 ** -24 + 1e-45
    assert abs(dec - exact) <= tol, (dec, exact, tol)
    # the FP32 running sum for comparison: the fixed-point sum is not worse
    acc = np.float32(0)
    for x in v:
        acc = np.float32(acc + x)
    assert abs(dec - exact) <= max(abs(float(acc) - exact), tol)


def test_fp64_limbs_cannot_overflow_and_encode_exactly(harness, tmp_path):
    """FP64 window (fix64_scales, fix64_encode): for any n contributions with |v| <= bound
    the three int32 limb sums stay in range, and each v is encoded as
    v S L^2 = a L^2 + b L + c + e with 0 <= b, c < L and |e| <= 1/2 (exact arithmetic)."""
    r = inputs.rng(8)
    pairs = [(1, 1.0), (4096, 6.25e-4), (4096, 2.0 ** -11), (65536, 1e-4), (1 << 20, 3e-6),
             (7, 1e3), (2, 1e-300)]
    pairs += [(int(r.integers(1, 1 << 22)), float(10 ** r.uniform(-12, 3))) for _ in range(200)]
    el, _ = _run(harness, tmp_path, [], [], pairs64=pairs)
    vals = []
    for (n, b), (eS, l) in zip(pairs, el):
        S, L = Fraction(2) ** int(eS), 2 ** int(l)
        assert Fraction(b) * S < 2 ** 20 and n * Fraction(b) * S < 2 ** 30, (n, b, eS)
        assert n * L < I31 and 0 <= l <= 21
        # tight: one more power of two in S would break a limit (eS capped at 1000)
        assert eS == 1000 or Fraction(b) * S * 2 >= 2 ** 19 or n * Fraction(b) * S * 2 >= 2 ** 29 / 2
        for _ in range(20):
            v = float(r.choice([-1, 1]) * b * 10 ** r.uniform(-16, 0))
            vals.append((v, int(eS), int(l), n, b))
        vals.append((b, int(eS), int(l), n, b))
        vals.append((-b, int(eS), int(l), n, b))
        vals.append((0.0, int(eS), int(l), n, b))
    _, abc = _run(harness, tmp_path, [], [], vals64=[(v, e, l) for v, e, l, _, _ in vals])
    for (v, eS, l, n, b), (a, bb, c) in zip(vals, abc):
        S, L = Fraction(2) ** eS, 2 ** l
        Y = a * L * L + bb * L + c
        assert 0 <= bb < L and 0 <= c < L
        assert abs(Fraction(v) * S * L * L - Y) <= Fraction(1, 2), (v, eS, l, a, bb, c)
        # limb sums of n such contributions stay inside int32
        assert n * (abs(a) + 1) < I31 and n * L < I31
