"""The analytic pusher (constant E, B over the step; Sec. 1, Sec. 4.1) in a form
that is smooth in all its inputs, and its vector-Jacobian product.

TEST INFRASTRUCTURE ONLY (imported by tests).  Plain numpy, FP64 / complex128.

The exact step is U(tau) = exp(L tau) U0 for the four-velocity U = (gamma, u),
L U = (e.u, gamma e + u x b), e = qm E, b = qm B, with the proper time tau fixed
by the lab time t(tau) = dt.  L satisfies L^4 = s1 L^2 + s2 with s1 = e.e - b.b
and s2 = (e.b)^2, so exp(L tau) = c0 + c1 L + c2 L^2 + c3 L^3.  Written with the
invariant-pair roots X = lE^2 tau^2, Y = lB^2 tau^2 (as the oracle's C pusher
does) the coefficients involve lE, lB, which are not differentiable where the
field is null (e.b = 0, |e| = |b|: every plane wave).  They are, however,
symmetric functions of z1 = X and z2 = -Y, the roots of z^2 - S1 z - S2 = 0 with
S1 = s1 tau^2, S2 = s2 tau^4, because k(Y) = h(-Y) and g(Y) = f(-Y) for the
series h(z) = sum z^n/(2n+2)!, f(z) = sum z^n/(2n+3)!.  With the divided
differences P_n = (z1^n - z2^n)/(z1 - z2) (P_0 = 0, P_1 = 1,
P_{n+1} = S1 P_n + S2 P_{n-1}):
  c0 = 1 + S2 sum h_n P_n,          c1 = tau (1 + S2 sum f_n P_n),
  c2 = tau^2 sum h_n P_{n+1},       c3 = tau^3 sum f_n P_{n+1},
and for the lab time t(tau) = c1 U0 + d1 (LU)_0 + c3 (L^2 U)_0 + d3 (L^3 U)_0,
  d1 = tau^2 (h_0 + S2 sum_{n>=1} h_n P_{n-1}),   d3 = tau^4 sum h_n P_n.
All are polynomials in (e, b, tau) summed to convergence, so the push is smooth,
and its derivatives can be taken by the complex-step method (exact to rounding
for an analytic function, no subtraction): d f/d x = Im f(x + i eps)/eps.
"""
from __future__ import annotations

import math

import numpy as np

NTERMS = 40
_H = np.array([1.0 / math.factorial(2 * n + 2) for n in range(NTERMS + 1)])
_F = np.array([1.0 / math.factorial(2 * n + 3) for n in range(NTERMS + 1)])


def _apply(e, b, U):
    """L U for U = (gamma, u1, u2, u3)."""
    g, u = U[0], U[1:]
    return np.concatenate([[e @ u], g * e + np.cross(u, b)])


def _coeffs(s1, s2, tau):
    S1, S2 = s1 * tau * tau, s2 * tau ** 4
    P = [0.0 * S1, 1.0 + 0.0 * S1]
    for _ in range(NTERMS + 1):
        P.append(S1 * P[-1] + S2 * P[-2])
    Dh = sum(_H[n] * P[n] for n in range(NTERMS))
    Df = sum(_F[n] * P[n] for n in range(NTERMS))
    c0 = 1.0 + S2 * Dh
    c1 = tau * (1.0 + S2 * Df)
    c2 = tau ** 2 * sum(_H[n] * P[n + 1] for n in range(NTERMS))
    c3 = tau ** 3 * sum(_F[n] * P[n + 1] for n in range(NTERMS))
    d1 = tau ** 2 * (_H[0] + S2 * sum(_H[n] * P[n - 1] for n in range(1, NTERMS)))
    d3 = tau ** 4 * Dh
    return c0, c1, c2, c3, d1, d3


def push(qm, dt, eb, u, iters=40):
    """u^{n+1/2} of the analytic push (works for real and complex inputs)."""
    eb = np.asarray(eb)
    u = np.asarray(u)
    e, b = qm * eb[:3], qm * eb[3:]
    g0 = np.sqrt(1.0 + u @ u)
    U = np.concatenate([[g0], u])
    LU = _apply(e, b, U)
    L2U = _apply(e, b, LU)
    L3U = _apply(e, b, L2U)
    s1, s2 = e @ e - b @ b, (e @ b) ** 2
    tau = dt / g0
    for _ in range(iters):        # Newton on t(tau) = dt; fixed count (converged long before)
        c0, c1, c2, c3, d1, d3 = _coeffs(s1, s2, tau)
        gam = c0 * U[0] + c1 * LU[0] + c2 * L2U[0] + c3 * L3U[0]
        t = c1 * U[0] + d1 * LU[0] + c3 * L2U[0] + d3 * L3U[0]
        tau = tau - (t - dt) / gam
    c0, c1, c2, c3, _, _ = _coeffs(s1, s2, tau)
    return c0 * U[1:] + c1 * LU[1:] + c2 * L2U[1:] + c3 * L3U[1:]


def vjp(qm, dt, eb, u, lam, eps=1e-30):
    """Gradient of lam . push(eb, u) with respect to (E1..E3, B1..B3) and
    (u1..u3), by the complex step.  Returns (d_eb[6], d_u[3])."""
    eb = np.asarray(eb, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    lam = np.asarray(lam, dtype=np.float64)
    d_eb, d_u = np.zeros(6), np.zeros(3)
    for i in range(6):
        z = eb.astype(np.complex128)
        z[i] += 1j * eps
        d_eb[i] = (lam @ push(qm, dt, z, u.astype(np.complex128))).imag / eps
    for i in range(3):
        z = u.astype(np.complex128)
        z[i] += 1j * eps
        d_u[i] = (lam @ push(qm, dt, eb.astype(np.complex128), z)).imag / eps
    return d_eb, d_u
