"""The smooth form of the analytic pusher (oracle/analytic_ref.py) and its VJP,
CPU.  The forward equals the oracle's C analytic push (which switches between
the series and the closed forms of h, f, k, g) on weak, strong and null fields;
the complex-step VJP equals central differences of the C push, also at null
fields (plane waves), where the (lE, lB) form of the coefficients is not
differentiable.  This is the reference the analytic pusher's adjoint is held to."""
import numpy as np
import pytest

from oracle import analytic_ref as ar
from oracle import oracle as orc

DT = 0.0981747704


def _cases():
    rng = np.random.Generator(np.random.PCG64(5))
    out = []
    for scale in (0.5, 3.0, 30.0):               # (X + Y) from ~1e-3 to ~10: both C branches
        for _ in range(6):
            out.append((rng.uniform(-scale, scale, 6), rng.uniform(-5, 5, 3)))
    for E in (0.3, 2.5, 40.0):                    # null fields: plane waves along x1
        out.append((np.array([0.0, E, 0.0, 0.0, 0.0, E]), np.array([3.0, -1.0, 0.5])))
    out.append((np.array([1.0, -2.0, 0.5, 0, 0, 0]), np.array([0.2, 0.1, -0.3])))    # pure E
    out.append((np.array([0, 0, 0, 1.5, 0.2, -2.0]), np.array([0.2, 4.0, -0.3])))    # pure B
    return out


def test_smooth_form_equals_the_c_pusher():
    for eb, u in _cases():
        ref, it = orc.analytic(-1.0, DT, eb, u)
        assert it > 0
        got = ar.push(-1.0, DT, eb, u)
        assert np.abs(got - ref).max() <= 1e-13 * max(np.abs(ref).max(), 1.0), (eb, u)


@pytest.mark.parametrize("k", range(0, 24, 3))
def test_vjp_equals_central_differences(k):
    eb, u = _cases()[k]
    lam = np.array([0.7, -0.4, 0.25])
    d_eb, d_u = ar.vjp(-1.0, DT, eb, u, lam)
    h = 1e-6 * max(1.0, np.abs(eb).max())

    def J(e, v):
        return lam @ orc.analytic(-1.0, DT, e, v)[0]

    fd_eb = np.array([(J(eb + h * np.eye(6)[i], u) - J(eb - h * np.eye(6)[i], u)) / (2 * h)
                      for i in range(6)])
    hu = 1e-6
    fd_u = np.array([(J(eb, u + hu * np.eye(3)[i]) - J(eb, u - hu * np.eye(3)[i])) / (2 * hu)
                     for i in range(3)])
    assert np.abs(d_eb - fd_eb).max() <= 1e-6 * max(np.abs(fd_eb).max(), 1e-3)
    assert np.abs(d_u - fd_u).max() <= 1e-6 * max(np.abs(fd_u).max(), 1e-3)
