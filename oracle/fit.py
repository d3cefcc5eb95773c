"""Stencil-coefficient customisation of App. B, written plainly in extended precision.

TEST INFRASTRUCTURE ONLY.

Minimise F = int_0^{1/2} w(k) ( [k~] - [k] )^2 dk  subject to  M C = e_1 by
solving the Lagrange (KKT) system of App. B Eq. (B.7),

    [[A, M^T], [M, 0]] (C; lambda) = (b; e_1),
    A_ij = (2/pi^2) int w sin((2i-1) pi k) sin((2j-1) pi k) dk,
    b_i  = (2/pi)   int w sin((2i-1) pi k) [k](k) dk,

with k normalised to k_g1 and the super-Gaussian weight of Eq. (B.10).  The
integrals use Gauss-Legendre quadrature on [0, 1/2]; the system is
ill-conditioned (its condition number reaches ~1e34 for M = 16), so it is
formed and solved with mpmath at ``dps`` decimal digits.
"""
from __future__ import annotations

import math

import mpmath as mp
import numpy as np


def _targets(k, r, kind):
    pi = mp.pi
    if kind == "proposed":   # Eq. (15), normalised
        return mp.tan(pi * k * r) / (pi * r), mp.sin(2 * pi * k * r) / (2 * pi * r)
    if kind == "xu":         # [k]_{1,t} in both laws
        t = mp.sin(pi * k * r) / (pi * r)
        return t, t
    if kind == "yee_tstagger":
        # Yee dispersion kept, [omega]_t = [k]_Yee, with the time-stagger
        # correction of the general solution (Sec. 3.1, Sec. 4.1 solver 3):
        # [k]_E1 = [k]_Yee / cos(omega dt/2), [k]_B1 = [k]_Yee cos(omega dt/2),
        # sin(omega dt/2) = (dt/2) [k]_Yee = r sin(pi k)
        ty = mp.sin(pi * k) / pi
        c = mp.sqrt(1 - (r * mp.sin(pi * k)) ** 2)
        return ty / c, ty * c
    raise ValueError(kind)


def fit(M: int, r: float, wk1: float = 0.3, n: int = 10, p: int = 2, kind: str = "proposed",
        nq: int = 768, dps: int = 60):
    """Return (C^E, C^B) as float64 arrays of length M.

    r = dt/dx1.  p = order of accuracy (p/2 constraint rows).  nq quadrature nodes."""
    with mp.workdps(dps):
        xs, ws = np.polynomial.legendre.leggauss(nq)
        half = mp.mpf(1) / 2
        nodes = [(mp.mpf(float(x)) + 1) * half * half for x in xs]       # map to [0, 1/2]
        weights = [mp.mpf(float(w)) * half * half for w in ws]
        ln2 = mp.log(2)
        r_m = mp.mpf(r)
        wk = mp.mpf(wk1)
        wts, sins, tE, tB = [], [], [], []
        for k, qw in zip(nodes, weights):
            wts.append(qw * mp.e ** (-ln2 * (2 * k / wk) ** n))
            sins.append([mp.sin((2 * i - 1) * mp.pi * k) for i in range(1, M + 1)])
            a, b = _targets(k, r_m, kind)
            tE.append(a)
            tB.append(b)
        P = p // 2
        N = M + P
        A = mp.matrix(N, N)
        for i in range(M):
            for j in range(i, M):
                s = mp.fsum(wts[q] * sins[q][i] * sins[q][j] for q in range(nq))
                A[i, j] = A[j, i] = 2 * s / mp.pi ** 2
        for i in range(P):
            for j in range(M):
                v = mp.mpf(2 * j + 1) ** (2 * i + 1) / math.factorial(2 * i + 1)
                A[M + i, j] = v
                A[j, M + i] = v
        out = []
        for tgt in (tE, tB):
            rhs = mp.matrix(N, 1)
            for i in range(M):
                rhs[i] = 2 * mp.fsum(wts[q] * sins[q][i] * tgt[q] for q in range(nq)) / mp.pi
            rhs[M] = 1
            sol = mp.lu_solve(A, rhs)
            out.append(np.array([float(sol[j]) for j in range(M)]))
        return out[0], out[1]


def kkt_residual(cE, cB, M, r, wk1=0.3, n=10, p=2, kind="proposed", nq=768, dps=60):
    """Projected gradient of F at (C^E, C^B) onto the constraint's null space,
    relative to the gradient's scale: zero at the constrained optimum."""
    with mp.workdps(dps):
        xs, ws = np.polynomial.legendre.leggauss(nq)
        half = mp.mpf(1) / 2
        res = []
        Mrow = np.array([[float((2 * j - 1) ** (2 * i - 1)) / math.factorial(2 * i - 1)
                          for j in range(1, M + 1)] for i in range(1, p // 2 + 1)])
        # orthonormal basis of null(Mrow) in float64 is enough for a residual check
        _, _, vt = np.linalg.svd(Mrow)
        Nb = vt[p // 2:].T
        for c, which in ((cE, 0), (cB, 1)):
            grad = [mp.mpf(0)] * M
            scale = mp.mpf(0)
            for x, wq in zip(xs, ws):
                k = (mp.mpf(float(x)) + 1) * half * half
                qw = mp.mpf(float(wq)) * half * half * mp.e ** (-mp.log(2) * (2 * k / wk1) ** n)
                s = [mp.sin((2 * i - 1) * mp.pi * k) for i in range(1, M + 1)]
                approx = mp.fsum(mp.mpf(float(c[j])) * s[j] for j in range(M)) / mp.pi
                t = _targets(k, mp.mpf(r), kind)[which]
                for i in range(M):
                    grad[i] += 2 * qw * (approx - t) * s[i] / mp.pi
                    scale += qw * abs(t * s[i]) / mp.pi
            g = np.array([float(v) for v in grad])
            res.append(float(np.linalg.norm(Nb.T @ g)) / float(scale))
        return res
