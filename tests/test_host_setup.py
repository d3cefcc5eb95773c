"""Host-side setup logic of the library, CPU only (no device): the laser load's
x1 profiles against the oracle's laser load (Eq. (8) eigenmode partner), and the
argument and CFL checks of the ensemble entry point (Eq. (21)), which run before
any CUDA call."""
import numpy as np
import pytest

from oracle import oracle as orc
from oracle.gen_tables import load as load_table
from paper_2004_03754_gb300 import inputs

DX1, DX2, DT = inputs.DX1, inputs.DX2, inputs.DT


@pytest.fixture(scope="module")
def P():
    from paper_2004_03754_gb300 import build
    build.build()
    from paper_2004_03754_gb300 import pic
    return pic


@pytest.mark.parametrize("n1", [64, 101, 16384])     # 16384: the FFT path of long rows
@pytest.mark.parametrize("table,dt", [((16, 0.5, 0.3), DT), ((16, 0.25, 0.3), 0.25 * DX1),
                                      ("yee", DT)])
def test_laser_profile_matches_oracle_load(P, table, dt, n1):
    if n1 > 1000 and table != (16, 0.25, 0.3):
        pytest.skip("one coefficient set suffices for the long row")
    cE, cB = (np.array([1.0]), np.array([1.0])) if table == "yee" else load_table(*table)
    a0, k0, phase, Lenv, xf = 3.0, 1.0, 0.4, 0.4 * n1 * DX1, 0.7 * n1 * DX1
    g = orc.Grid((n1, 1 if n1 > 1000 else 4), (DX1, DX2), dt, cE, cB)
    F = orc.Fields(g)
    orc.laser_load(g, F, a0=a0, k0=k0, phase=phase, Lenv=Lenv, x_front=xf, w0=0.0)
    las = P.pic_laser(a0, k0, phase, Lenv, xf, 0.0, 0.0, 0.0)
    e2, b3 = P.pic_laser_profile(n1, DX1, dt, cE, cB, las)
    assert np.abs(e2 - F.e2[0]).max() <= 1e-12 * np.abs(F.e2).max()
    assert np.abs(b3 - F.b3[0]).max() <= 1e-12 * np.abs(F.b3).max()


def test_laser_profile_rejects_bad_arguments(P):
    cE, cB = load_table(16, 0.5, 0.3)
    good = P.pic_laser(1.0, 1.0, 0.0, 10.0, 20.0, 0.0, 0.0, 0.0)
    P.pic_laser_profile(128, DX1, DT, cE, cB, good)
    for las in (P.pic_laser(1.0, 1.0, 0.0, 128 * DX1 + 1.0, 20.0, 0.0, 0.0, 0.0),   # longer than the box
                P.pic_laser(1.0, 0.0, 0.0, 10.0, 20.0, 0.0, 0.0, 0.0),              # k0 = 0
                P.pic_laser(float("nan"), 1.0, 0.0, 10.0, 20.0, 0.0, 0.0, 0.0)):    # a0 not finite
        with pytest.raises(P.PicError):
            P.pic_laser_profile(128, DX1, DT, cE, cB, las)
    with pytest.raises(P.PicError):
        P.pic_laser_profile(0, DX1, DT, cE, cB, good)
    with pytest.raises(P.PicError):
        P.pic_laser_profile(128, DX1, -DT, cE, cB, good)


def test_ensemble_checks_cfl_and_arguments_on_the_host(P):
    cE, cB = load_table(16, 0.5, 0.3)
    n1, n2 = [128, 300], [16, 40]
    # above the exact CFL bound of the customised stencil for every run's grid
    with pytest.raises(P.PicError) as e:
        P.Ensemble(n1, n2, (DX1, DX2), 1.2 * DX1, cE, cB, precision="fp64", pusher="boris")
    assert e.value.status == P.PIC_ERR_CFL
    with pytest.raises(P.PicError) as e:
        P.Ensemble(n1, n2, (DX1, -DX2), DT, cE, cB, precision="fp64", pusher="boris")
    assert e.value.status == P.PIC_ERR_ARG
    with pytest.raises(P.PicError) as e:
        P.Ensemble([128, 0], n2, (DX1, DX2), DT, cE, cB, precision="fp64", pusher="boris")
    assert e.value.status == P.PIC_ERR_ARG
