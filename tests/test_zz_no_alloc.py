"""Allocation-free laser load (pic_laser_fields_noalloc) against pic_load_laser.

The variant serves callers whose device memory belongs to another allocator
and who therefore may not have the library call cudaMalloc; it keeps its
scratch in a static device array.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_2004_03754_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-12


def _grid(P, n, dx):
    g = P.pic_grid()
    g.ndim = len(n)
    for d in range(3):
        g.n[d] = n[d] if d < len(n) else 1
        g.dx[d] = dx[d] if d < len(n) else 1.0
    g.precision, g.pusher = P.PIC_FP64, P.PIC_BORIS
    return g


def _existing(P, n, dx, dt, cE, cB, las):
    sim = P.Simulation(n, dx, dt, cE, cB, precision="fp64")
    P.pic_load_laser(sim.ctx, las)
    e2, b3 = sim.read_field("e2"), sim.read_field("b3")
    sim.close()
    return e2, b3


def test_noalloc_laser_matches_existing_entry_point():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2004_03754_gb300 import coeffs
    from paper_2004_03754_gb300 import pic as P
    cE, cB = coeffs.load("proposed", 16, 0.5, 0.3)
    dt = inputs.DT
    cases = [
        ((512, 24), (inputs.DX1, inputs.DX2), P.pic_laser(2.0, 1.0, 0.3, 6 * np.pi, 400 * inputs.DX1,
                                                          3.0, 12 * inputs.DX2, 0.0)),
        ((300, 8, 6), (inputs.DX1, inputs.DX2, inputs.DX2),
         P.pic_laser(5.0, 1.0, -1.1, 8 * np.pi, 150 * inputs.DX1, 2.0, 4 * inputs.DX2, 3 * inputs.DX2)),
    ]
    for n, dx, las in cases:          # two calls in a row, different shapes
        e_ref, b_ref = _existing(P, n, dx, dt, cE, cB, las)
        shape = tuple(reversed(n))
        e2 = torch.full(shape, float("nan"), dtype=torch.float64, device="cuda")
        b3 = torch.full(shape, float("nan"), dtype=torch.float64, device="cuda")
        st = P.pic_laser_fields_noalloc(_grid(P, n, dx), dt, cE, cB, las, e2, b3)
        assert st == P.PIC_OK
        e, b = e2.cpu().numpy(), b3.cpu().numpy()
        assert np.abs(e - e_ref).max() <= TOL * np.abs(e_ref).max()
        assert np.abs(b - b_ref).max() <= TOL * np.abs(b_ref).max()
    # the largest accepted row (it fills the whole static array), called on a
    # side stream, against the host profiles of the existing load (n2 = 1: E2 and
    # B3 are the x1 profiles themselves)
    nmax = P.PIC_NOALLOC_MAX_N1
    las = P.pic_laser(3.0, 1.0, 0.4, 20 * np.pi, 500 * inputs.DX1, 0.0, 0.0, 0.0)
    e_ref, b_ref = P.pic_laser_profile(nmax, inputs.DX1, dt, cE, cB, las)
    side = torch.cuda.Stream()
    e2 = torch.full((1, nmax), float("nan"), dtype=torch.float64, device="cuda")
    b3 = torch.full((1, nmax), float("nan"), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    st = P.pic_laser_fields_noalloc(_grid(P, (nmax, 1), (inputs.DX1, inputs.DX2)), dt, cE, cB, las,
                                    e2, b3, stream=side.cuda_stream)
    assert st == P.PIC_OK
    side.synchronize()
    e, b = e2.cpu().numpy()[0], b3.cpu().numpy()[0]
    assert np.abs(e - e_ref).max() <= TOL * np.abs(e_ref).max()
    assert np.abs(b - b_ref).max() <= TOL * np.abs(b_ref).max()
    # beyond the static scratch: rejected, not run
    big = (P.PIC_NOALLOC_MAX_N1 + 1, 1) if hasattr(P, "PIC_NOALLOC_MAX_N1") else (65537, 1)
    e2 = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = P.pic_laser_fields_noalloc(_grid(P, big, (inputs.DX1, inputs.DX2)), dt, cE, cB,
                                    P.pic_laser(1.0, 1.0, 0.0, 6 * np.pi, 0.0, 0.0, 0.0, 0.0), e2, e2)
    assert st == P.PIC_ERR_ARG
