"""The C ABI library loads and exports what include/pic.h declares (no GPU needed);
argument validation and the CFL check of Eq. (21) run before any device call."""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pic.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pic_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2004_03754_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("pic_init", "pic_load_laser", "pic_load_particles", "pic_step",
                 "pic_read_field", "pic_read_particles", "pic_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.check_output(["nm", "-D", "--defined-only", libpath]).decode()
    exported = set(l.split()[-1] for l in out.splitlines() if l.strip())
    for name in declared_functions():
        assert name in exported, name
    lib = C.CDLL(libpath)
    for name in declared_functions():
        getattr(lib, name)


def test_init_validates_arguments_and_cfl(libpath):
    from paper_2004_03754_gb300 import pic as P
    from oracle.gen_tables import load as load_table
    cE, cB = load_table(16, 0.5, 0.3)
    dx1 = 2 * np.pi / 32
    g = P.pic_grid()
    g.ndim = 2
    g.n[0], g.n[1], g.n[2] = 64, 16, 1
    g.dx[0], g.dx[1], g.dx[2] = dx1, 4 * dx1, 1.0
    g.precision, g.pusher = P.PIC_FP64, P.PIC_BORIS
    # dt well above the exact CFL bound of the customised stencil
    with pytest.raises(P.PicError) as e:
        P.pic_init(g, 1.2 * dx1, cE, cB)
    assert e.value.status == P.PIC_ERR_CFL
    assert "CFL" in P.pic_last_error(None)
    # Yee at the 1D Courant limit dt = dx1 with a 2nd axis: violated
    with pytest.raises(P.PicError) as e:
        P.pic_init(g, dx1, [1.0], [1.0])
    assert e.value.status == P.PIC_ERR_CFL
    # bad arguments
    g.ndim = 4
    with pytest.raises(P.PicError) as e:
        P.pic_init(g, 0.5 * dx1, cE, cB)
    assert e.value.status == P.PIC_ERR_ARG
    g.ndim = 2
    with pytest.raises(P.PicError) as e:
        P.pic_init(g, -1.0, cE, cB)
    assert e.value.status == P.PIC_ERR_ARG
    with pytest.raises(P.PicError) as e:
        P.pic_init(g, 0.5 * dx1, np.ones(40), np.ones(40))
    assert e.value.status == P.PIC_ERR_ARG
    # only the quadratic shape and periodic boundaries are built: others are refused
    for field, bad in (("shape", 1), ("shape", 3), ("boundary", 2), ("boundary", -1)):
        setattr(g, field, bad)
        with pytest.raises(P.PicError) as e:
            P.pic_init(g, 0.5 * dx1, cE, cB)
        assert e.value.status == P.PIC_ERR_ARG
        assert field in P.pic_last_error(None)
        setattr(g, field, 0)
