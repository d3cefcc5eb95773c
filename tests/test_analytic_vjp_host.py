"""The adjoint's derivative of the analytic push (csrc/analytic_vjp.cuh: the push
in a form smooth at null fields, differentiated by forward-mode dual numbers
with the proper time through the implicit function theorem), run on the host
through the C ABI (no device), against the oracle: the push itself against the
oracle's C analytic pusher, and the vector-Jacobian product against the
complex-step derivative of oracle/analytic_ref.py (Sec. 1, Sec. 4.1)."""
import numpy as np
import pytest

from oracle import analytic_ref as ar
from oracle import oracle as orc
from paper_2004_03754_gb300 import inputs


@pytest.fixture(scope="module")
def P():
    from paper_2004_03754_gb300 import build
    build.build()
    from paper_2004_03754_gb300 import pic
    return pic


def _cases():
    r = np.random.Generator(np.random.PCG64(71))
    out = []
    for scale in (0.05, 1.0, 30.0):                 # weak, moderate, strong (X + Y >= 2)
        for _ in range(6):
            out.append((r.normal(size=6) * scale, r.normal(size=3) * 2.0))
    # null fields (plane waves: E perp B, |E| = |B|), the case the smooth form is for
    for a in (0.3, 5.0, 100.0):
        out.append((np.array([0.0, a, 0.0, 0.0, 0.0, a]), np.array([0.5, 0.2, 0.0])))
        out.append((np.array([0.0, a, 0.0, 0.0, 0.0, a]), np.zeros(3)))
    return out


@pytest.mark.parametrize("k", range(24))
def test_analytic_vjp_matches_complex_step(P, k):
    eb, u = _cases()[k]
    dt, qm = inputs.DT, -1.0
    lam = np.array([0.7, -1.3, 0.4])
    uo, deb, du = P.pic_analytic_push_vjp(qm, dt, eb, u, lam)
    ref_u, it = orc.analytic(qm, dt, eb, u)
    assert np.abs(uo - ref_u).max() <= 1e-12 * max(1.0, np.abs(ref_u).max())
    d_eb, d_u = ar.vjp(qm, dt, eb, u, lam)
    scale = max(np.abs(d_eb).max(), np.abs(d_u).max(), 1e-300)
    assert np.abs(deb - d_eb).max() <= 1e-9 * scale, (deb, d_eb)
    assert np.abs(du - d_u).max() <= 1e-9 * scale, (du, d_u)
