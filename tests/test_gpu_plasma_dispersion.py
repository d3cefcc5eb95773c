"""Cold-plasma dispersion (App. C) on the GPU path: the frequency of the
transverse electromagnetic mode in a quiet-start cold plasma against the
closed form [omega]_t^2 = [k]_E1 [k]_B1 + omega_p^2 r(k), as the oracle pin does."""
import math

import numpy as np
import pytest

from oracle import closed_forms as cf
from oracle.gen_tables import load as load_table
from paper_2004_03754_gb300 import inputs
from plasma_modes import cold_plasma_run

pytestmark = pytest.mark.gpu

DX1, DX2, DT = inputs.DX1, inputs.DX2, inputs.DT


@pytest.fixture(scope="module")
def pic():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2004_03754_gb300 import pic as P
    return P


@pytest.mark.parametrize("solver,precision,tol", [("yee", "fp64", 1e-9), ("proposed", "fp64", 1e-9),
                                                  ("proposed", "mixed", 1e-6)])
def test_cold_plasma_dispersion_gpu(pic, solver, precision, tol):
    cE, cB = (np.array([1.0]), np.array([1.0])) if solver == "yee" else load_table(16, 0.5, 0.3)
    wp2 = 1.0
    sims = []

    def make(x, u, w, e3_0):
        sim = pic.Simulation((64, 4), (DX1, DX2), DT, cE, cB, precision=precision, pusher="boris")
        sims.append(sim)
        sim.load_field("e3", e3_0)
        sim.load_particles(x, u, w, -1.0)
        return (lambda: sim.read_field("e3")[0]), (lambda: sim.step(1))

    k, offs, om = cold_plasma_run(make, DX1, DX2, DT, wp2=wp2)
    sims[0].close()
    kE, kB = cf.k_stencil(cE, k, DX1), cf.k_stencil(cB, k, DX1)
    pred = cf.cold_plasma_omega(kE, kB, wp2, cf.lattice_shape_response(k, DX1, offs), DT)
    err = abs(om - pred) / pred
    print(solver, precision, "omega %.9f  App. C %.9f  rel. err %.1e" % (om, pred, err))
    assert err < tol
    assert abs(om - math.sqrt(k * k + wp2)) / pred > 1e-3
