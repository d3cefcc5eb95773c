"""Write the oracle's stencil-coefficient tables (App. B fits) to ``oracle/data``.

TEST INFRASTRUCTURE ONLY.  Calls nothing outside ``oracle/``.  Run from the
repository root:  python -m oracle.gen_tables

Each table is one text file: a header of '#' lines stating the fit
parameters, then M lines "C^E_j C^B_j" in %.17e.  Entries whose magnitude is
below 1e-24 are written as 0: the fit runs at 60 digits with a condition
number up to ~1e34, so nothing below that floor is significant.  At
r = dt/dx1 = 1/2 this makes C^B exactly e_1, which the mathematics fixes:
the Ampere target sin(2 pi k r)/(2 pi r) is then the Yee operator itself.
"""
import os

import numpy as np

from oracle import fit

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data")

TABLES = [
    # (M, r, w_k1, kind)
    (16, 0.5, 0.3, "proposed"),
    (8, 0.5, 0.4, "proposed"),
    (16, 0.25, 0.3, "proposed"),
    (16, 0.125, 0.3, "proposed"),
    (16, 0.5, 0.3, "xu"),
    (16, 0.25, 0.3, "xu"),             # the Sec. 4.1 single-particle set-up
    (16, 0.25, 0.3, "yee_tstagger"),
]


def name(M, r, wk1, kind):
    return "coeffs_%s_M%d_r%g_w%g.txt" % (kind, M, r, wk1)


def main():
    os.makedirs(HERE, exist_ok=True)
    for M, r, wk1, kind in TABLES:
        cE, cB = fit.fit(M, r, wk1, kind=kind)
        for c in (cE, cB):
            c[np.abs(c) < 1e-24] = 0.0
        path = os.path.join(HERE, name(M, r, wk1, kind))
        with open(path, "w") as f:
            f.write("# App. B constrained least-squares stencil fit (oracle/fit.py)\n")
            f.write("# kind=%s M=%d r=dt/dx1=%r w_k1=%r n=10 p=2 nq=768 dps=60\n" % (kind, M, r, wk1))
            f.write("# columns: C^E_j C^B_j, j = 1..M\n")
            for a, b in zip(cE, cB):
                f.write("%.17e %.17e\n" % (a, b))
        print("wrote", path)


def load(M, r, wk1, kind="proposed"):
    d = np.loadtxt(os.path.join(HERE, name(M, r, wk1, kind)), ndmin=2)
    return d[:, 0].copy(), d[:, 1].copy()


if __name__ == "__main__":
    main()
