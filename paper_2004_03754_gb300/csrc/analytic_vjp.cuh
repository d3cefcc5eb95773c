// analytic_vjp.cuh -- derivatives of the analytic push (constant E, B over the
// step; Sec. 1, Sec. 4.1) for the adjoint: the Jacobian of u^{n+1/2} with
// respect to (u^{n-1/2}, E, B), by forward-mode dual numbers through a form of
// the push that is smooth in every input.
//
// The push is U(tau) = exp(L tau) U0 for U = (gamma, u), L U = (e.u, gamma e + u x b),
// e = qm E, b = qm B, with tau fixed by the lab time t(tau) = dt.  L^4 = s1 L^2 + s2
// (s1 = e.e - b.b, s2 = (e.b)^2), so exp(L tau) = c0 + c1 L + c2 L^2 + c3 L^3.  In
// terms of the roots X, -Y of z^2 - S1 z - S2 (S1 = s1 tau^2, S2 = s2 tau^4) the
// coefficients are symmetric functions of the roots: with P_0 = 0, P_1 = 1,
// P_{n+1} = S1 P_n + S2 P_{n-1} and h_n = 1/(2n+2)!, f_n = 1/(2n+3)!,
//   c0 = 1 + S2 sum h_n P_n,   c1 = tau (1 + S2 sum f_n P_n),
//   c2 = tau^2 sum h_n P_{n+1},   c3 = tau^3 sum f_n P_{n+1},
//   t  = c1 U0 + d1 (LU)0 + c3 (L^2U)0 + d3 (L^3U)0,
//   d1 = tau^2 (h_0 + S2 sum_{n>=1} h_n P_{n-1}),   d3 = tau^4 sum h_n P_n,
// polynomials in (e, b, tau): smooth also where the field is null (every plane
// wave), where the (lambda_E, lambda_B) form of the forward kernel is not.  For
// X + Y >= 2 the closed forms h(X) = (cosh sqrt X - 1)/X, ... are used with X, Y
// from the roots, which are then distinct and differentiable.  The proper time
// enters through the implicit function theorem: dtau = -(dt/dp) dp / gamma(tau).
// Compiles for host and device (the host copy is what the CPU tests check
// against a complex-step differentiation of the same push).
#pragma once
#include <math.h>

#include <type_traits>

#include "fpbits.cuh"   // PIC_HD

namespace pic {

// value and N directional derivatives
template <int N>
struct Dual {
  double v;
  double d[N];
};

template <int N>
PIC_HD Dual<N> dconst(double v) {
  Dual<N> r;
  r.v = v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = 0.0;
  return r;
}
template <int N>
PIC_HD Dual<N> operator+(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r;
  r.v = a.v + b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] + b.d[i];
  return r;
}
template <int N>
PIC_HD Dual<N> operator-(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r;
  r.v = a.v - b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] - b.d[i];
  return r;
}
template <int N>
PIC_HD Dual<N> operator*(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r;
  r.v = a.v * b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
  return r;
}
template <int N>
PIC_HD Dual<N> operator*(double s, const Dual<N>& a) {
  Dual<N> r;
  r.v = s * a.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = s * a.d[i];
  return r;
}
template <int N>
PIC_HD Dual<N> operator+(double s, const Dual<N>& a) {
  Dual<N> r = a;
  r.v += s;
  return r;
}
template <int N>
PIC_HD Dual<N> operator/(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r;
  const double ib = 1.0 / b.v;
  r.v = a.v * ib;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = (a.d[i] - r.v * b.d[i]) * ib;
  return r;
}
// f(a) with f(a.v) = fv and f'(a.v) = fp
template <int N>
PIC_HD Dual<N> dchain(const Dual<N>& a, double fv, double fp) {
  Dual<N> r;
  r.v = fv;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = fp * a.d[i];
  return r;
}
template <int N>
PIC_HD Dual<N> dsqrt(const Dual<N>& a) {
  const double s = sqrt(a.v);
  return dchain(a, s, 0.5 / s);
}

// the same operations on plain doubles, so one template serves value and dual
PIC_HD double sval(double x) { return x; }
template <int N>
PIC_HD double sval(const Dual<N>& x) { return x.v; }
template <class S>
PIC_HD S sconst(double v) {
  if constexpr (std::is_same<S, double>::value) return v;
  else return dconst<sizeof(S::d) / sizeof(double)>(v);
}
PIC_HD double ssqrt(double x) { return sqrt(x); }
template <int N>
PIC_HD Dual<N> ssqrt(const Dual<N>& x) { return dsqrt(x); }
PIC_HD double scosh(double x) { return cosh(x); }
PIC_HD double ssinh(double x) { return sinh(x); }
PIC_HD double scos(double x) { return cos(x); }
PIC_HD double ssin(double x) { return sin(x); }
template <int N>
PIC_HD Dual<N> scosh(const Dual<N>& x) { return dchain(x, cosh(x.v), sinh(x.v)); }
template <int N>
PIC_HD Dual<N> ssinh(const Dual<N>& x) { return dchain(x, sinh(x.v), cosh(x.v)); }
template <int N>
PIC_HD Dual<N> scos(const Dual<N>& x) { return dchain(x, cos(x.v), -sin(x.v)); }
template <int N>
PIC_HD Dual<N> ssin(const Dual<N>& x) { return dchain(x, sin(x.v), cos(x.v)); }

// 1/m! for the series (exact small reciprocals multiplied, folded per call site)
PIC_HD double inv_fact(int m) {
  double f = 1.0;
  for (int k = 2; k <= m; ++k) f /= (double)k;
  return f;
}

// sum_{n>=0} z^n/(2n+A)!, |z| < 1 (A = 2: h, A = 3: f)
template <int A, class S>
PIC_HD S an_series1(const S& z) {
  S s = sconst<S>(0.0), zn = sconst<S>(1.0);
  double c = inv_fact(A);
  for (int n = 0; n < 24; ++n) {
    s = s + c * zn;
    zn = zn * z;
    c /= (double)((2 * n + A + 1) * (2 * n + A + 2));
  }
  return s;
}

// c0, c1, c2, c3, d1, d3 of the step at proper time tau (see the file header)
template <class S>
PIC_HD void an_smooth_coeffs(const S& s1, const S& s2, const S& tau, S c[6]) {
  const S t2 = tau * tau;
  const S S1 = s1 * t2, S2 = s2 * (t2 * t2);
  const double xy = sqrt(sval(S1) * sval(S1) + 4.0 * sval(S2));   // X + Y
  S Dh, Df, Hh1, Ff1, Hm1 = sconst<S>(0.0);
  if (xy < 2.0) {
    S Pm = sconst<S>(0.0), P = sconst<S>(0.0), Pn = sconst<S>(1.0);   // P_{n-1}, P_n, P_{n+1}
    Dh = Df = Hh1 = Ff1 = Hm1 = sconst<S>(0.0);
    double h = 0.5, f = 1.0 / 6.0;   // 1/(2n+2)!, 1/(2n+3)!
    for (int n = 0; n < 40; ++n) {
      Dh = Dh + h * P;
      Df = Df + f * P;
      Hh1 = Hh1 + h * Pn;
      Ff1 = Ff1 + f * Pn;
      if (n >= 1) Hm1 = Hm1 + h * Pm;
      if (h * (fabs(sval(P)) + fabs(sval(Pn)) + fabs(sval(Pm))) < 1e-19 && n > 2) break;
      Pm = P;
      P = Pn;
      Pn = S1 * P + S2 * Pm;
      h /= (double)((2 * n + 3) * (2 * n + 4));
      f /= (double)((2 * n + 4) * (2 * n + 5));
    }
  } else {
    const S root = ssqrt(S1 * S1 + 4.0 * S2);
    const S X = 0.5 * (S1 + root), Y = 0.5 * (root - S1);
    S hX, fX, kY, gY;
    if (sval(X) < 1.0) {
      hX = an_series1<2>(X);
      fX = an_series1<3>(X);
    } else {
      const S x = ssqrt(X);
      hX = (scosh(x) - sconst<S>(1.0)) / X;
      fX = (ssinh(x) - x) / (X * x);
    }
    if (sval(Y) < 1.0) {
      kY = an_series1<2>(-1.0 * Y);
      gY = an_series1<3>(-1.0 * Y);
    } else {
      const S y = ssqrt(Y);
      kY = (sconst<S>(1.0) - scos(y)) / Y;
      gY = (y - ssin(y)) / (Y * y);
    }
    Dh = (hX - kY) / root;
    Df = (fX - gY) / root;
    Hh1 = hX - Y * Dh;
    Ff1 = fX - Y * Df;
  }
  c[0] = 1.0 + S2 * Dh;
  c[1] = tau * (1.0 + S2 * Df);
  c[2] = t2 * Hh1;
  c[3] = t2 * tau * Ff1;
  // d1 = tau^2 (h - X Dhk) = tau^2 (Hh1 - S1 Dh) in the closed form (X - Y = S1)
  c[4] = xy < 2.0 ? t2 * (0.5 + S2 * Hm1) : t2 * (Hh1 - S1 * Dh);
  c[5] = (t2 * t2) * Dh;
}

template <class S>
struct AnSmooth {
  S U[4], LU[4], L2U[4], L3U[4];
  S s1, s2;
};

template <class S>
PIC_HD void an_smooth_apply(const S e[3], const S b[3], const S V[4], S o[4]) {
  o[0] = e[0] * V[1] + e[1] * V[2] + e[2] * V[3];
  o[1] = V[0] * e[0] + (V[2] * b[2] - V[3] * b[1]);
  o[2] = V[0] * e[1] + (V[3] * b[0] - V[1] * b[2]);
  o[3] = V[0] * e[2] + (V[1] * b[1] - V[2] * b[0]);
}

template <class S>
PIC_HD void an_smooth_setup(double qm, const S eb[6], const S u[3], AnSmooth<S>& a) {
  S e[3], b[3];
  for (int m = 0; m < 3; ++m) {
    e[m] = qm * eb[m];
    b[m] = qm * eb[3 + m];
  }
  a.U[0] = ssqrt(1.0 + (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]));
  for (int m = 0; m < 3; ++m) a.U[m + 1] = u[m];
  an_smooth_apply(e, b, a.U, a.LU);
  an_smooth_apply(e, b, a.LU, a.L2U);
  an_smooth_apply(e, b, a.L2U, a.L3U);
  a.s1 = (e[0] * e[0] + e[1] * e[1] + e[2] * e[2]) - (b[0] * b[0] + b[1] * b[1] + b[2] * b[2]);
  const S eb_ = e[0] * b[0] + e[1] * b[1] + e[2] * b[2];
  a.s2 = eb_ * eb_;
}

// gamma, lab time and u at proper time tau
template <class S>
PIC_HD void an_smooth_eval(const AnSmooth<S>& a, const S& tau, S* gam, S* tl, S uo[3]) {
  S c[6];
  an_smooth_coeffs(a.s1, a.s2, tau, c);
  *gam = c[0] * a.U[0] + c[1] * a.LU[0] + c[2] * a.L2U[0] + c[3] * a.L3U[0];
  *tl = c[1] * a.U[0] + c[4] * a.LU[0] + c[3] * a.L2U[0] + c[5] * a.L3U[0];
  for (int m = 0; m < 3; ++m)
    uo[m] = c[0] * a.U[m + 1] + c[1] * a.LU[m + 1] + c[2] * a.L2U[m + 1] + c[3] * a.L3U[m + 1];
}

// The analytic push in the smooth form with its Jacobian: uo = u^{n+1/2} and
// jac[m][k] = d uo_m / d p_k for p = (u1, u2, u3, E1, E2, E3, B1, B2, B3).
// Returns false if the proper-time iteration did not converge.
PIC_HD bool analytic_push_jacobian(double qm, double dt, const double eb[6], const double u[3],
                                   double uo[3], double jac[3][9]) {
  // proper time on values: bracketed Newton on t(tau) = dt (t(tau) >= tau)
  AnSmooth<double> av;
  an_smooth_setup<double>(qm, eb, u, av);
  double lo = 0.0, hi = dt, tau = dt / av.U[0], gam, tl, w[3];
  bool ok = false;
  for (int it = 0; it < 80; ++it) {
    an_smooth_eval<double>(av, tau, &gam, &tl, w);
    if (tl > dt) hi = tau;
    else lo = tau;
    double nt = tau - (tl - dt) / gam;
    if (!(nt > lo && nt < hi)) nt = 0.5 * (lo + hi);
    const double step = fabs(nt - tau);
    tau = nt;
    if (step <= 4.0 * 2.220446049250313e-16 * tau) {
      ok = true;
      break;
    }
  }
  // dual pass 1: dt/dp at fixed tau; dual pass 2: u(tau(p)) with
  // dtau/dp = -(dt/dp) / gamma (implicit function theorem)
  Dual<9> ud[3], ebd[6];
  for (int m = 0; m < 3; ++m) {
    ud[m] = dconst<9>(u[m]);
    ud[m].d[m] = 1.0;
  }
  for (int c = 0; c < 6; ++c) {
    ebd[c] = dconst<9>(eb[c]);
    ebd[c].d[3 + c] = 1.0;
  }
  AnSmooth<Dual<9>> ad;
  an_smooth_setup<Dual<9>>(qm, ebd, ud, ad);
  Dual<9> g9, t9, u9[3];
  Dual<9> tau9 = dconst<9>(tau);
  an_smooth_eval(ad, tau9, &g9, &t9, u9);
  for (int k = 0; k < 9; ++k) tau9.d[k] = -t9.d[k] / g9.v;
  an_smooth_eval(ad, tau9, &g9, &t9, u9);
  for (int m = 0; m < 3; ++m) {
    uo[m] = u9[m].v;
    for (int k = 0; k < 9; ++k) jac[m][k] = u9[m].d[k];
  }
  return ok;
}

}  // namespace pic
