"""Taps of the x1 current correction built by the library's host code
(pic_correction_taps, the form pic_step applies) against the oracle's exact
per-row DFT correction (Sec. 3.3, Eq. (23)): CPU only, no device."""
import numpy as np
import pytest

from oracle import oracle as orc
from oracle.gen_tables import load as load_table
from paper_2004_03754_gb300 import coeffs, inputs

DX1, DX2 = inputs.DX1, inputs.DX2


@pytest.fixture(scope="module")
def P():
    from paper_2004_03754_gb300 import build
    build.build()
    from paper_2004_03754_gb300 import pic
    return pic


def apply_taps(taps, lo, rows):
    n1 = rows.shape[-1]
    out = np.zeros_like(rows)
    for q, t in enumerate(taps):
        out += t * np.roll(rows, -(lo + q), axis=-1)   # J1_{i+lo+q}
    return out


def oracle_corrected(cE, cB, rows):
    n2, n1 = rows.shape
    g = orc.Grid((n1, n2), (DX1, DX2), 0.25 * DX1, cE, cB)
    j = rows.copy()
    orc.correct_j1(g, j)
    return j


def tables():
    out = [("proposed", load_table(16, 0.25, 0.3)),
           ("random5", inputs.random_coeffs(5, seed=4))]
    for kind in ("xu", "yee_tstagger"):
        out.append((kind, coeffs.load(kind, 16, 0.25, 0.3)))
    return out


@pytest.mark.parametrize("n1", [7, 24, 61, 96, 257, 1000])
@pytest.mark.parametrize("name,cc", tables())
def test_taps_match_exact_dft_correction(P, name, cc, n1):
    cE, cB = cc
    taps, lo = P.pic_correction_taps(n1, DX1, cB)
    assert len(taps) <= n1 and lo <= 0
    rows = inputs.rng(n1).uniform(-1, 1, (3, n1))
    ref = oracle_corrected(cE, cB, rows)
    got = apply_taps(taps, lo, rows)
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max(), name


def test_taps_are_short_at_the_bench_row_length(P):
    # the symbol is smooth: at n1 = 4096 the 16-coefficient dt/dx1 = 1/4 set
    # keeps 57 taps (m = -28..28), not n1
    cE, cB = load_table(16, 0.25, 0.3)
    taps, lo = P.pic_correction_taps(4096, DX1, cB)
    assert (len(taps), lo) == (57, -28)
    # even symbol: symmetric taps, up to the rounding floor of the DFT sum
    assert np.allclose(taps, taps[::-1], rtol=0, atol=1e-16)
    rows = inputs.rng(9).uniform(-1, 1, (1, 4096))
    ref = oracle_corrected(cE, cB, rows)
    assert np.abs(apply_taps(taps, lo, rows) - ref).max() <= 1e-13


def test_identity_and_errors(P):
    taps, lo = P.pic_correction_taps(128, DX1, [1.0])
    assert list(taps) == [1.0] and lo == 0
    with pytest.raises(P.PicError):
        P.pic_correction_taps(0, DX1, [1.0])
    with pytest.raises(P.PicError):
        P.pic_correction_taps(64, DX1, [0.0])          # [k]_B1 = 0 at every mode
    with pytest.raises(P.PicError):
        P.pic_correction_taps(64, -DX1, [1.0])
