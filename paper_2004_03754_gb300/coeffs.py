"""x1 stencil coefficients of the customised solver (App. B) for pic_init.

``load()`` reads a shipped table (``data/``); ``fit()`` recomputes one.  The
fit minimises F = int_0^{1/2} w(k) ([k~](k) - [k](k))^2 dk (k normalised to
k_g1 = 2 pi/dx1, super-Gaussian w of Eq. (B.10)) subject to the accuracy
constraint M C = e_1 of App. B.  It is solved here by the null-space method:
C = C_p + N z with M N = 0, then z from a weighted linear least-squares
problem solved by QR, so the normal equations (whose condition number reaches
~1e34 at M = 16) are never formed.  The arithmetic runs in mpmath at ``dps``
digits; mpmath is needed only to fit, not to load.

Targets (Eq. (15), normalised, r = dt/dx1):
  proposed: [k]_E1 = tan(pi k r)/(pi r),  [k]_B1 = sin(2 pi k r)/(2 pi r)
  xu:       [k]_E1 = [k]_B1 = sin(pi k r)/(pi r)
  yee_tstagger: Yee dispersion with the time-stagger correction (Sec. 4.1),
            [k]_E1 = [k]_Y/c, [k]_B1 = [k]_Y c, [k]_Y = sin(pi k)/pi,
            c = cos(omega dt/2) = sqrt(1 - r^2 sin^2(pi k))
  yee:      C^E = C^B = (1)
"""
from __future__ import annotations

import math
import os

import numpy as np

DATA = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data")


def table_name(kind, M, r, wk1):
    return "stencil_%s_M%d_r%g_w%g.txt" % (kind, M, r, wk1)


def load(kind="proposed", M=16, r=0.5, wk1=0.3):
    """(C^E, C^B) float64 arrays from a shipped table; kind 'yee' needs no table."""
    if kind == "yee":
        return np.array([1.0]), np.array([1.0])
    d = np.loadtxt(os.path.join(DATA, table_name(kind, M, r, wk1)), ndmin=2)
    return d[:, 0].copy(), d[:, 1].copy()


def fit(M, r, wk1=0.3, n=10, p=2, kind="proposed", degree=9, dps=50):
    """Return (C^E, C^B).  degree: mpmath Gauss-Legendre degree (3*2^(degree-1) nodes)."""
    import mpmath as mp
    from mpmath.calculus.quadrature import GaussLegendre

    with mp.workdps(dps):
        half = mp.mpf(1) / 2
        # nodes on [-1, 1] mapped to [0, 1/2]
        nodes = GaussLegendre(mp.mp).calc_nodes(degree, mp.mp.prec)
        ks = [(x + 1) * half * half for x, _ in nodes]
        qw = [w * half * half for _, w in nodes]
        ln2 = mp.log(2)
        rr, wk = mp.mpf(r), mp.mpf(wk1)
        P = p // 2
        # accuracy constraint rows M_ij = (2j-1)^(2i-1)/(2i-1)!
        Mc = mp.matrix(P, M)
        for i in range(P):
            for j in range(M):
                Mc[i, j] = mp.mpf(2 * j + 1) ** (2 * i + 1) / math.factorial(2 * i + 1)
        # particular solution (minimum norm) and null-space basis from the QR of Mc^T
        Q, R = mp.qr(Mc.T, mode="full")
        Rt = mp.matrix(P, P)
        for i in range(P):
            for j in range(P):
                Rt[i, j] = R[j, i]
        y = mp.lu_solve(Rt, mp.matrix([1] + [0] * (P - 1)))
        Cp = Q[:, 0:P] * y
        N = Q[:, P:M]
        # weighted design matrix rows sqrt(w_q) * sin((2j-1) pi k_q)/pi
        rows = []
        sq = []
        for k, w in zip(ks, qw):
            wt = w * mp.e ** (-ln2 * (2 * k / wk) ** n)
            s = mp.sqrt(wt)
            sq.append(s)
            rows.append([s * mp.sin((2 * j + 1) * mp.pi * k) / mp.pi for j in range(M)])
        A = mp.matrix(rows)
        AN = A * N
        Qa, Ra = mp.qr(AN, mode="skinny")
        out = []
        for which in (0, 1):
            tgt = []
            for k, s in zip(ks, sq):
                if kind == "proposed":
                    t = (mp.tan(mp.pi * k * rr) / (mp.pi * rr), mp.sin(2 * mp.pi * k * rr) / (2 * mp.pi * rr))[which]
                elif kind == "xu":
                    t = mp.sin(mp.pi * k * rr) / (mp.pi * rr)
                elif kind == "yee_tstagger":
                    ty = mp.sin(mp.pi * k) / mp.pi
                    cc = mp.sqrt(1 - (rr * mp.sin(mp.pi * k)) ** 2)
                    t = (ty / cc, ty * cc)[which]
                else:
                    raise ValueError(kind)
                tgt.append(s * t)
            b = mp.matrix(tgt) - A * Cp
            z = mp.lu_solve(Ra, Qa.T * b)   # R z = Q^T b (upper triangular)
            C = Cp + N * z
            out.append(np.array([float(C[j]) for j in range(M)]))
        return out[0], out[1]


def write_table(kind, M, r, wk1, path=None):
    cE, cB = fit(M, r, wk1, kind=kind)
    for c in (cE, cB):
        c[np.abs(c) < 1e-24] = 0.0   # below the fit's working accuracy
    path = path or os.path.join(DATA, table_name(kind, M, r, wk1))
    with open(path, "w") as f:
        f.write("# customised x1 stencil (App. B), null-space QR fit at 50 digits\n")
        f.write("# kind=%s M=%d r=dt/dx1=%r w_k1=%r n=10 p=2\n" % (kind, M, r, wk1))
        for a, b in zip(cE, cB):
            f.write("%.17e %.17e\n" % (a, b))
    return path


if __name__ == "__main__":
    for spec in (("proposed", 16, 0.5, 0.3), ("proposed", 8, 0.5, 0.4), ("proposed", 16, 0.25, 0.3),
                 ("proposed", 16, 0.125, 0.3), ("xu", 16, 0.5, 0.3), ("xu", 16, 0.25, 0.3),
                 ("yee_tstagger", 16, 0.25, 0.3)):
        print(write_table(*spec))
