// pushers.cuh -- particle momentum advance u^{n-1/2} -> u^{n+1/2}, FP64.
//
// Both pushers take the fields at the particle (E^n and the time-centred B^n,
// Eq. (7)) and q/m; u = gamma*beta.  FP64 throughout: at a0 ~ 1e4 the electron
// reaches gamma ~ 1e7-1e8 and the transverse force E2 - beta1 B3 is a difference
// of nearly equal terms (Sec. 1), which single precision cannot resolve.
#pragma once
#include <math.h>

#include "fpbits.cuh"

#ifdef __CUDACC__
#define PIC_HDI __host__ __device__ inline
#else
#define PIC_HDI inline
#endif

namespace pic {

// Single-precision seeds of the Newton iterations below: the hardware estimate
// on the device; on the host (where the tests run these pushers against the
// oracle) the correctly rounded value, which the Newton steps refine alike.
PIC_HD float seed_rsqrt(float v) {
#ifdef __CUDA_ARCH__
  return rsqrtf(v);
#else
  return 1.0f / sqrtf(v);
#endif
}
PIC_HD float seed_rcp(float v) {
#ifdef __CUDA_ARCH__
  return __frcp_rn(v);
#else
  return 1.0f / v;
#endif
}

// 1/sqrt(x) and 1/x for x >= 1 in FP64 by Newton-Raphson iteration from the
// single-precision hardware estimate: each step squares the relative error
// (2^-22 -> 2^-44 -> 2^-88), so two steps (NR = 2, the FP64 path) reach double
// rounding.  With FP32 fields (NR = 1) one step leaves a relative error near
// 1e-13, six orders below the rounding of the fields the push consumes.  This
// keeps the FP64 pipe -- 1/64 of the FP32 rate on this GPU -- for the arithmetic
// the push needs rather than for a general IEEE divide or square root.
// Each step is y <- y + (y/2)(1 - x y^2); in the first, y/2 is the FP32 seed
// halved (exact) and widened on the integer pipe, so that step costs three
// FP64 operations.
template <int NR = 2>
PIC_HD double rsqrt_nr(double x) {
  const float s = seed_rsqrt(narrow_pos(x));
  double y = widen_pos(s);
  y = fma(widen_pos(0.5f * s), fma(-x * y, y, 1.0), y);
#pragma unroll
  for (int k = 1; k < NR; ++k) y = fma(0.5 * y, fma(-x * y, y, 1.0), y);
  return y;
}
template <int NR = 2>
PIC_HD double rcp_nr(double x) {
  double y = widen_pos(seed_rcp(narrow_pos(x)));
#pragma unroll
  for (int k = 0; k < NR; ++k) y = fma(y, fma(-x, y, 1.0), y);
  return y;
}

// 2/x for x >= 1: with one step the doubling rides on the seed (2 s is exact),
// two FP64 operations in all.
template <int NR = 2>
PIC_HD double twice_rcp_nr(double x) {
  if constexpr (NR == 1) {
    const float s = seed_rcp(narrow_pos(x));
    const double y2 = widen_pos(2.0f * s);
    return fma(y2, fma(-x, widen_pos(s), 1.0), y2);
  } else {
    return 2.0 * rcp_nr<NR>(x);
  }
}

// Relativistic Boris pusher (Sec. 1): half electric kick, rotation about B
// with the half-kicked gamma, second half kick.
template <int NR = 2>
PIC_HD void boris_push(double qm, double dt, const double eb[6], double u[3]) {
  const double h = 0.5 * qm * dt;
  double ux = u[0] + h * eb[0], uy = u[1] + h * eb[1], uz = u[2] + h * eb[2];
  const double hig = h * rsqrt_nr<NR>(1.0 + ux * ux + uy * uy + uz * uz);
  const double tx = hig * eb[3], ty = hig * eb[4], tz = hig * eb[5];
  const double f = twice_rcp_nr<NR>(1.0 + tx * tx + ty * ty + tz * tz);
  // u' = u- + u- x t and u+ = u- + u' x s, each component as two fused
  // multiply-adds
  const double px = fma(-uz, ty, fma(uy, tz, ux));
  const double py = fma(-ux, tz, fma(uz, tx, uy));
  const double pz = fma(-uy, tx, fma(ux, ty, uz));
  const double sx = f * tx, sy = f * ty, sz = f * tz;
  ux = fma(-pz, sy, fma(py, sz, ux));
  uy = fma(-px, sz, fma(pz, sx, uy));
  uz = fma(-py, sx, fma(px, sy, uz));
  u[0] = ux + h * eb[0];
  u[1] = uy + h * eb[1];
  u[2] = uz + h * eb[2];
}

// Higuera-Cary pusher (Sec. 1, Sec. 4.1; Higuera & Cary 2017): the rotation
// about B uses the Lorentz factor gbar of the mean proper velocity of the
// rotation, the positive root of gbar^4 - sigma gbar^2 - (|beta|^2 + u*^2) = 0
// with beta = (qm dt/2) B, sigma = gamma-^2 - |beta|^2, u* = u-.beta.  This keeps
// the relativistic E x B drift exact.
template <int NR = 2>
PIC_HD void hc_push(double qm, double dt, const double eb[6], double u[3]) {
  const double h = 0.5 * qm * dt;
  const double ux = u[0] + h * eb[0], uy = u[1] + h * eb[1], uz = u[2] + h * eb[2];
  const double bx = h * eb[3], by = h * eb[4], bz = h * eb[5];
  const double gm2 = 1.0 + ux * ux + uy * uy + uz * uz;
  const double b2 = bx * bx + by * by + bz * bz;
  const double us = ux * bx + uy * by + uz * bz;
  const double sigma = gm2 - b2;
  const double gbar2 = 0.5 * (sigma + sqrt(sigma * sigma + 4.0 * (b2 + us * us)));
  const double ig = rsqrt_nr<NR>(gbar2);
  const double tx = bx * ig, ty = by * ig, tz = bz * ig;
  const double ut = ux * tx + uy * ty + uz * tz;
  const double s = rcp_nr<NR>(1.0 + tx * tx + ty * ty + tz * tz);
  const double wx = s * (ux + ut * tx + (uy * tz - uz * ty));
  const double wy = s * (uy + ut * ty + (uz * tx - ux * tz));
  const double wz = s * (uz + ut * tz + (ux * ty - uy * tx));
  u[0] = wx + (wy * tz - wz * ty) + h * eb[0];
  u[1] = wy + (wz * tx - wx * tz) + h * eb[1];
  u[2] = wz + (wx * ty - wy * tx) + h * eb[2];
}

// ---------------------------------------------------------------------------
// Analytic pusher for E, B constant over the step (Sec. 1, Sec. 4.1): the
// four-velocity U = (gamma, u) obeys dU/dtau = L U with
//   L U = (e.u, gamma e + u x b),  e = qm E, b = qm B.
// L^4 = (lE^2 - lB^2) L^2 + lE^2 lB^2 with lE^2 - lB^2 = e^2 - b^2, lE lB = |e.b|,
// so exp(L tau) = c0 + c1 L + c2 L^2 + c3 L^3.  With X = (lE tau)^2, Y = (lB tau)^2
// and the entire functions
//   h(X) = (cosh x - 1)/X,  f(X) = (sinh x - x)/(X x),
//   k(Y) = (1 - cos y)/Y,   g(Y) = (y - sin y)/(Y y),
//   Dhk = (h - k)/(X + Y),  Dfg = (f - g)/(X + Y),
// the coefficients are c0 = 1 + XY Dhk, c1 = tau (1 + XY Dfg),
// c2 = tau^2 (h - Y Dhk), c3 = tau^3 (f - Y Dfg), and the lab time is
// t(tau) = [c1 U + tau^2 (h - X Dhk) LU + c3 L^2U + tau^4 Dhk L^3U]_0.
// Every form is finite as X, Y -> 0 (null fields, the plane-wave case).
// The proper time with t(tau) = dt is found by bracketed Newton (dt/dtau = gamma).
// ---------------------------------------------------------------------------

// sum_{n>=0} z^n / (2n + A)! for A = 2, 3: fully unrolled, so the reciprocal
// factorial ratios fold to compile-time constants (no FP64 division at run time).
template <int A>
PIC_HD double series_even(double z) {
  double s = 0.0, t = (A == 2) ? 0.5 : 1.0 / 6.0;
#pragma unroll
  for (int n = 0; n < 16; ++n) {
    s += t;
    t *= z * (1.0 / (double)((2 * n + A + 1) * (2 * n + A + 2)));
  }
  return s;
}

PIC_HD double an_h(double X) {
  if (X < 1.0) return series_even<2>(X);
  const double x = sqrt(X);
  return (cosh(x) - 1.0) / X;
}
PIC_HD double an_k(double Y) {
  if (Y < 1.0) return series_even<2>(-Y);
  const double y = sqrt(Y);
  return (1.0 - cos(y)) / Y;
}
PIC_HD double an_f(double X) {
  if (X < 1.0) return series_even<3>(X);
  const double x = sqrt(X);
  return (sinh(x) - x) / (X * x);
}
PIC_HD double an_g(double Y) {
  if (Y < 1.0) return series_even<3>(-Y);
  const double y = sqrt(Y);
  return (y - sin(y)) / (Y * y);
}

// sum_{n>=1} [(X^n - (-Y)^n)/(X+Y)] / (2n+A)!,  with the recurrence
// P_n = (X^n - (-Y)^n)/(X+Y):  P_1 = 1,  P_{n+1} = X P_n + (-Y)^n.
template <int A>
PIC_HD double an_divided(double X, double Y) {
  double c = (A == 2) ? 1.0 / 24.0 : 1.0 / 120.0;   // 1/(2+A)!
  double P = 1.0, mY = -Y, s = 0.0;
#pragma unroll
  for (int n = 1; n <= 18; ++n) {
    s += P * c;
    P = X * P + mY;
    mY *= -Y;
    c *= 1.0 / (double)((2 * n + A + 1) * (2 * n + A + 2));
  }
  return s;
}

struct AnState {
  double lE2, lB2;
  double U[4], LU[4], L2U[4], L3U[4];
};

PIC_HD void an_apply(const double e[3], const double b[3], const double V[4],
                                         double o[4]) {
  o[0] = e[0] * V[1] + e[1] * V[2] + e[2] * V[3];
  o[1] = V[0] * e[0] + (V[2] * b[2] - V[3] * b[1]);
  o[2] = V[0] * e[1] + (V[3] * b[0] - V[1] * b[2]);
  o[3] = V[0] * e[2] + (V[1] * b[1] - V[2] * b[0]);
}

// h(X), f(X), Dhk(X,Y), Dfg(X,Y) in one pass.  For X + Y < 2 all four are power
// series summed together, with as many terms as keep the neglected ones below
// 2^-60 of the leading ones (a handful in the weak-field steps that dominate);
// otherwise the closed forms.
struct AnFuncs {
  double h, f, Dhk, Dfg;
};

// 1/(2n+2)! and 1/(2n+3)!, n = 0..20, as products of exact small reciprocals
// folded at compile time (the series loop below stops early, so it indexes a
// table instead of forming each coefficient by an FP64 division)
struct AnCoef {
  double c2[21], c3[21];
};
constexpr AnCoef an_coef_table() {
  AnCoef t{};
  double f = 1.0;  // 1/m!
  for (int m = 1; m <= 43; ++m) {
    f /= (double)m;
    if (m >= 2 && m % 2 == 0 && (m - 2) / 2 <= 20) t.c2[(m - 2) / 2] = f;
    if (m >= 3 && m % 2 == 1 && (m - 3) / 2 <= 20) t.c3[(m - 3) / 2] = f;
  }
  return t;
}
#ifdef __CUDACC__
__constant__ constexpr AnCoef kAnCoef = an_coef_table();
#endif
constexpr AnCoef kAnCoefHost = an_coef_table();

// Terms needed by the series of an_funcs: the sums stop once a term falls below
// 2^-60 of the leading ones.  With M = max(X, Y), term n of every series is at
// most B_n(M) = (M^n + n M^(n-1)) / (2n+2)! (X^n <= M^n and |P_n| <= n M^(n-1)),
// increasing in M; kAnTerms.m[K] is the largest M (found by bisection at compile
// time, rounded down to FP32 with a 1e-6 margin) for which B_(K-1)(M) < 2^-60,
// so K terms (n = 0 .. K-1) are enough for every M <= m[K].
struct AnTerms {
  float m[22];
};
constexpr double an_bound(int n, double M) {
  double p = 1.0, c = 0.5;   // M^(n-1) (1 for n = 0 and 1), 1/(2n+2)!
  for (int k = 1; k < n; ++k) p *= M;
  for (int k = 1; k <= n; ++k) c /= (double)((2 * k + 1) * (2 * k + 2));
  return (n == 0 ? 1.0 : p * M + n * p) * c;
}
constexpr AnTerms an_terms_table() {
  AnTerms t{};
  for (int K = 0; K < 22; ++K) {
    if (K < 1) {
      t.m[K] = -1.0f;
      continue;
    }
    double lo = 0.0, hi = 2.0;
    if (an_bound(K - 1, 0.0) >= 8.7e-19) {
      t.m[K] = -1.0f;   // not enough terms even for M = 0
      continue;
    }
    for (int it = 0; it < 80; ++it) {
      const double mid = 0.5 * (lo + hi);
      if (an_bound(K - 1, mid) < 8.7e-19) lo = mid; else hi = mid;
    }
    t.m[K] = (float)(lo * (1.0 - 1e-6));
  }
  return t;
}
#ifdef __CUDACC__
__constant__ constexpr AnTerms kAnTerms = an_terms_table();
#endif
constexpr AnTerms kAnTermsHost = an_terms_table();

PIC_HD AnFuncs an_funcs(double X, double Y) {
  AnFuncs r;
  if (X + Y < 2.0) {
    // K terms n = 0 .. K-1 of h = sum c2[n] X^n and f = sum c3[n] X^n, and of
    // their divided differences between X and -Y, Dhk = sum c2[n] P_n and
    // Dfg = sum c3[n] P_n (P_n = (X^n - (-Y)^n)/(X + Y)), by a double Horner
    // scheme from the highest term: r <- r X + c[n] gives the series at X and
    // q <- q (-Y) + r its divided difference (two FMAs per term and series).
    const float Mf = narrow_signed(fmax(X, Y));   // FP32 copy on the integer pipe
    int K = 1;
#ifdef __CUDA_ARCH__
    while (K < 21 && !(Mf <= kAnTerms.m[K])) ++K;
#else
    while (K < 21 && !(Mf <= kAnTermsHost.m[K])) ++K;
#endif
    const double mY = -Y;
#ifdef __CUDA_ARCH__
    double rh = kAnCoef.c2[K - 1], rf = kAnCoef.c3[K - 1];
#else
    double rh = kAnCoefHost.c2[K - 1], rf = kAnCoefHost.c3[K - 1];
#endif
    double qh = 0.0, qf = 0.0;
#pragma unroll 1
    for (int n = K - 2; n >= 0; --n) {
#ifdef __CUDA_ARCH__
      const double c2 = kAnCoef.c2[n], c3 = kAnCoef.c3[n];
#else
      const double c2 = kAnCoefHost.c2[n], c3 = kAnCoefHost.c3[n];
#endif
      qh = fma(qh, mY, rh);
      qf = fma(qf, mY, rf);
      rh = fma(rh, X, c2);
      rf = fma(rf, X, c3);
    }
    r.h = rh;
    r.f = rf;
    r.Dhk = qh;
    r.Dfg = qf;
  } else {
    r.h = an_h(X);
    r.f = an_f(X);
    r.Dhk = (r.h - an_k(Y)) / (X + Y);
    r.Dfg = (r.f - an_g(Y)) / (X + Y);
  }
  return r;
}

// gamma(tau) and t(tau); c[0..3] receive the coefficients of exp(L tau) from
// which an_momentum forms the spatial part of U(tau)
PIC_HD void an_eval(const AnState& a, double tau, double* gam, double* tl, double c[4]) {
  const double t2 = tau * tau;
  const double X = a.lE2 * t2, Y = a.lB2 * t2;
  const AnFuncs F = an_funcs(X, Y);
  const double c0 = 1.0 + X * Y * F.Dhk;
  const double c1 = tau * (1.0 + X * Y * F.Dfg);
  const double c2 = t2 * (F.h - Y * F.Dhk);
  const double c3 = t2 * tau * (F.f - Y * F.Dfg);
  const double d1 = t2 * (F.h - X * F.Dhk);
  const double d3 = t2 * t2 * F.Dhk;
  *gam = c0 * a.U[0] + c1 * a.LU[0] + c2 * a.L2U[0] + c3 * a.L3U[0];
  *tl = c1 * a.U[0] + d1 * a.LU[0] + c3 * a.L2U[0] + d3 * a.L3U[0];
  c[0] = c0;
  c[1] = c1;
  c[2] = c2;
  c[3] = c3;
}
PIC_HD void an_momentum(const AnState& a, const double c[4], double* uo) {
#pragma unroll
  for (int m = 0; m < 3; ++m)
    uo[m] = c[0] * a.U[m + 1] + c[1] * a.LU[m + 1] + c[2] * a.L2U[m + 1] + c[3] * a.L3U[m + 1];
}

// Returns the number of evaluations (> 0), or -1 if the proper-time iteration
// did not converge within its bound (u is then left unchanged).
PIC_HDI int analytic_push(double qm, double dt, const double eb[6], double u[3]) {
  AnState a;
  const double e[3] = {qm * eb[0], qm * eb[1], qm * eb[2]};
  const double b[3] = {qm * eb[3], qm * eb[4], qm * eb[5]};
  const double ee = e[0] * e[0] + e[1] * e[1] + e[2] * e[2];
  const double bb = b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
  const double ebd = e[0] * b[0] + e[1] * b[1] + e[2] * b[2];
  const double I1 = ee - bb;
  const double root = sqrt(I1 * I1 + 4.0 * ebd * ebd);
  if (I1 >= 0.0) {
    a.lE2 = 0.5 * (I1 + root);
    a.lB2 = a.lE2 > 0.0 ? ebd * ebd / a.lE2 : 0.0;
  } else {
    a.lB2 = 0.5 * (root - I1);
    a.lE2 = a.lB2 > 0.0 ? ebd * ebd / a.lB2 : 0.0;
  }
  // gamma0 = x / sqrt(x) from the Newton 1/sqrt (x >= 1), which also gives dt/gamma0
  const double x0 = 1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  const double ig0 = rsqrt_nr(x0);
  const double g0 = x0 * ig0;
  a.U[0] = g0; a.U[1] = u[0]; a.U[2] = u[1]; a.U[3] = u[2];
  an_apply(e, b, a.U, a.LU);
  an_apply(e, b, a.LU, a.L2U);
  an_apply(e, b, a.L2U, a.L3U);
  // t(tau) >= tau (gamma >= 1): the root lies in (0, dt].  Start Newton at
  // dt/gamma0, keeping a bracket [lo, hi] (t increasing) for bisection fallback.
  // (A start from the root of the expansion of t(tau) in tau saves evaluations
  // when the fields are moderate but costs more than it saves on the plasma
  // workloads, where most electrons see fields too weak for it to matter.)
  double lo = 0.0, hi = dt, tau = dt * ig0, gam, tl, cf[4];
  const double eps4 = 4.0 * 2.220446049250313e-16;
  int it = 1;
  for (; it <= 64; ++it) {
    an_eval(a, tau, &gam, &tl, cf);
    const double r = tl - dt;
    // gam >= 1; one Newton step of 1/gam suffices: its 1e-13 relative error only
    // scales the (then tiny) correction, the state is taken at the evaluated tau
    double tn = tau - r * rcp_nr<1>(gam);
    // converged: the Newton step is below rounding of tau (tested before the
    // bracket, whose strict bounds would turn a step that rounds to nothing,
    // or a zero residual, into a bisection step away from the root)
    if (fabs(tn - tau) <= eps4 * fabs(tau)) break;
    if (r > 0.0) hi = tau; else lo = tau;
    if (!(tn > lo && tn < hi)) tn = 0.5 * (lo + hi);
    if (hi - lo <= eps4 * hi) break;
    tau = tn;
  }
  if (it > 64) return -1;
  double uo[3];
  an_momentum(a, cf, uo);   // at the last evaluated tau
  u[0] = uo[0]; u[1] = uo[1]; u[2] = uo[2];
  return it;
}

}  // namespace pic
