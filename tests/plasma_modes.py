"""Cold-plasma mode measurement shared by the oracle pin and the GPU test
(App. C): a standing transverse wave in a quiet-start cold electron plasma."""
import math

import numpy as np


def cold_plasma_run(make, DX1, DX2, DT, n1=64, n2=4, mode=4, ppc=4, wp2=1.0, nsteps=1200, amp=1e-6):
    """Standing E3 wave cos(k x1) at rest in a uniform cold electron plasma of
    density wp2 (= omega_p^2 with q/m = -1); returns the frequency measured from
    the projection y_n of E3 onto the mode, which for a single linear mode obeys
    y_{n+1} + y_{n-1} = 2 cos(omega dt) y_n exactly (least squares over the run).
    `make(x, u, w, e3_0)` builds the state (E3 = e3_0, other fields zero) and
    returns (e3_reader, stepper)."""
    k = 2 * np.pi * mode / (n1 * DX1)
    offs = (np.arange(ppc) + 0.5) / ppc
    i = np.repeat(np.arange(n1), ppc)
    x1 = (i + np.tile(offs, n1)) * DX1
    x1 = np.tile(x1, n2)
    x2 = np.repeat((np.arange(n2) + 0.5) * DX2, n1 * ppc)
    npart = x1.size
    w = np.full(npart, -wp2 / ppc)
    u = [np.zeros(npart)] * 3
    e3_0 = amp * np.tile(np.cos(k * np.arange(n1) * DX1), (n2, 1))
    read_e3, advance = make([x1, x2], u, w, e3_0)
    basis = np.cos(k * np.arange(n1) * DX1)
    y = np.empty(nsteps + 1)
    y[0] = (read_e3() * basis).sum()
    for s in range(nsteps):
        advance()
        y[s + 1] = (read_e3() * basis).sum()
    c = (y[1:-1] * (y[2:] + y[:-2])).sum() / (2 * (y[1:-1] ** 2).sum())
    return k, offs, math.acos(c) / DT
