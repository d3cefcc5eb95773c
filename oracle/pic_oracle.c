/*
 * pic_oracle.c -- plain, slow, FP64 CPU reference ("the oracle") of the
 * electromagnetic PIC time step of Li, Miller, Xu, Tsung, Decyk, An, Fonseca,
 * Mori, "A new field solver for modeling of relativistic particle-laser
 * interactions using the particle-in-cell algorithm" (arXiv:2004.03754).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call
 * this file; only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark use it.  It shares no code, header or table with the CUDA library.
 *
 * Every function is written as the paper (or the textbook definition it cites)
 * states it: straight loops, periodic index wrapping, no tiling, no fusion.
 * Compile with -O2 -ffp-contract=off so that no FMA contraction changes the
 * rounding between x86-64 and aarch64 hosts.
 *
 * Conventions (App. A, App. B index conventions):
 *   grid nodes X_i = i*dx1 (i = 0..n1-1), periodic in every axis;
 *   arrays are stored x1-fastest: idx = (k*n2 + j)*n1 + i;
 *   staggering  E1(i+1/2,j,k)  E2(i,j+1/2,k)  E3(i,j,k+1/2)
 *               B1(i,j+1/2,k+1/2)  B2(i+1/2,j,k+1/2)  B3(i+1/2,j+1/2,k)
 *   J is co-located with E, rho sits on the nodes (i,j,k).
 *   In 2D (ndim=2, n3=1) every d/dx3 is zero and the x3 staggering drops out.
 *   Normalised units c = m_e = e = 1 (Sec. 2.1).
 *
 * State of the oracle's leapfrog (Eq. (1), Eq. (7)): E^n, B^{n-1/2},
 * particle positions x^n and momenta u^{n-1/2} (u = gamma*beta).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
  int ndim;            /* 2 or 3 */
  int n1, n2, n3;      /* cells; n3 = 1 in 2D */
  double dx1, dx2, dx3;
  double dt;
  int M;               /* number of x1 stencil coefficients */
  const double* cE;    /* C^E_j, j = 1..M (Faraday's law, App. B Eq. (B.1)) */
  const double* cB;    /* C^B_j, j = 1..M (Ampere's law, App. B Eq. (B.2)) */
} orc_grid;

typedef struct {
  double *e1, *e2, *e3, *b1, *b2, *b3, *j1, *j2, *j3;
} orc_fields;

static int wrapi(int i, int n) {
  int r = i % n;
  return r < 0 ? r + n : r;
}

static int64_t at(const orc_grid* g, int i, int j, int k) {
  return ((int64_t)wrapi(k, g->n3) * g->n2 + wrapi(j, g->n2)) * g->n1 + wrapi(i, g->n1);
}

static int64_t ncell(const orc_grid* g) { return (int64_t)g->n1 * g->n2 * g->n3; }

/* ---------------------------------------------------------------------------
 * Spatial operators.
 * ------------------------------------------------------------------------- */

/* Faraday's-law x1 derivative, App. B Eq. (B.1):
 *   d^E f_i = (1/dx1) sum_j C^E_j (f_{i+j} - f_{i-j+1}),  result at i+1/2. */
static double dE1(const orc_grid* g, const double* f, int i, int j, int k) {
  double s = 0.0;
  for (int m = 1; m <= g->M; ++m)
    s += g->cE[m - 1] * (f[at(g, i + m, j, k)] - f[at(g, i - m + 1, j, k)]);
  return s / g->dx1;
}

/* Ampere's-law x1 derivative, App. B Eq. (B.2):
 *   d^B f_i = (1/dx1) sum_j C^B_j (f_{i+j-1} - f_{i-j}),  result at i-1/2 -> i. */
static double dB1(const orc_grid* g, const double* f, int i, int j, int k) {
  double s = 0.0;
  for (int m = 1; m <= g->M; ++m)
    s += g->cB[m - 1] * (f[at(g, i + m - 1, j, k)] - f[at(g, i - m, j, k)]);
  return s / g->dx1;
}

/* Yee differences along x2 / x3 (Sec. 3.1.1: the x2 operators stay Yee).
 * fwd: (f_{j+1} - f_j)/dx, result at j+1/2;  bwd: (f_j - f_{j-1})/dx, at j-1/2. */
static double d2f(const orc_grid* g, const double* f, int i, int j, int k) {
  return (f[at(g, i, j + 1, k)] - f[at(g, i, j, k)]) / g->dx2;
}
static double d2b(const orc_grid* g, const double* f, int i, int j, int k) {
  return (f[at(g, i, j, k)] - f[at(g, i, j - 1, k)]) / g->dx2;
}
static double d3f(const orc_grid* g, const double* f, int i, int j, int k) {
  if (g->ndim < 3) return 0.0;
  return (f[at(g, i, j, k + 1)] - f[at(g, i, j, k)]) / g->dx3;
}
static double d3b(const orc_grid* g, const double* f, int i, int j, int k) {
  if (g->ndim < 3) return 0.0;
  return (f[at(g, i, j, k)] - f[at(g, i, j, k - 1)]) / g->dx3;
}

/* Faraday's law, Eq. (1):  B <- B - h * (d_E x E).
 * Written to a copy first so that every component uses the same old E. */
void orc_faraday(const orc_grid* g, orc_fields* F, double h) {
  int64_t n = ncell(g);
  double* nb1 = malloc(sizeof(double) * n);
  double* nb2 = malloc(sizeof(double) * n);
  double* nb3 = malloc(sizeof(double) * n);
#pragma omp parallel for collapse(2) schedule(static)
  for (int k = 0; k < g->n3; ++k)
    for (int j = 0; j < g->n2; ++j)
      for (int i = 0; i < g->n1; ++i) {
        int64_t c = at(g, i, j, k);
        double curl1 = d2f(g, F->e3, i, j, k) - d3f(g, F->e2, i, j, k);
        double curl2 = d3f(g, F->e1, i, j, k) - dE1(g, F->e3, i, j, k);
        double curl3 = dE1(g, F->e2, i, j, k) - d2f(g, F->e1, i, j, k);
        nb1[c] = F->b1[c] - h * curl1;
        nb2[c] = F->b2[c] - h * curl2;
        nb3[c] = F->b3[c] - h * curl3;
      }
  memcpy(F->b1, nb1, sizeof(double) * n);
  memcpy(F->b2, nb2, sizeof(double) * n);
  memcpy(F->b3, nb3, sizeof(double) * n);
  free(nb1); free(nb2); free(nb3);
}

/* Ampere's law, Eq. (1):  E <- E + h * (d_B x B - J).  J is read from F->j*. */
void orc_ampere(const orc_grid* g, orc_fields* F, double h) {
#pragma omp parallel for collapse(2) schedule(static)
  for (int k = 0; k < g->n3; ++k)
    for (int j = 0; j < g->n2; ++j)
      for (int i = 0; i < g->n1; ++i) {
        int64_t c = at(g, i, j, k);
        double curl1 = d2b(g, F->b3, i, j, k) - d3b(g, F->b2, i, j, k);
        double curl2 = d3b(g, F->b1, i, j, k) - dB1(g, F->b3, i, j, k);
        double curl3 = dB1(g, F->b2, i, j, k) - d2b(g, F->b1, i, j, k);
        F->e1[c] += h * (curl1 - F->j1[c]);
        F->e2[c] += h * (curl2 - F->j2[c]);
        F->e3[c] += h * (curl3 - F->j3[c]);
      }
}

/* k-space forms of the x1 operators, App. B Eq. (B.3) (and Eq. (6) for M=p/2):
 *   [k] = sum_j C_j sin((2j-1) k dx1/2) / (dx1/2). */
double orc_kspace(int M, const double* c, double k1, double dx1) {
  double s = 0.0;
  for (int m = 1; m <= M; ++m) s += c[m - 1] * sin((2 * m - 1) * k1 * dx1 / 2.0);
  return s / (dx1 / 2.0);
}

/* True iff C^B is exactly (1, 0, ..., 0): then [k]_B1 = [k]_Yee and the
 * current correction of Sec. 3.3 is the identity. */
int orc_cb_is_yee(const orc_grid* g) {
  if (g->cB[0] != 1.0) return 0;
  for (int m = 2; m <= g->M; ++m)
    if (g->cB[m - 1] != 0.0) return 0;
  return 1;
}

/* Current correction along x1, Sec. 3.3.  The deposited (Esirkepov) current
 * satisfies the Yee continuity equation, Eq. (24).  Gauss's law with the
 * Ampere operator d^B (Eq. (26)) needs d^B J1^A = d^Yee J1, i.e. in x1-Fourier
 * space  J1^A = ([k]_{1,Yee} / [k]_{B1}) J1  (the reading taken for Eq. (23),
 * whose printed ratio is the reciprocal; the Fourier-continuity derivation that
 * follows it fixes the direction).  Computed with an explicit DFT of every x1 row
 * ("an FFT only along the 1-direction"), written out as the plain O(n1^2) sum. */
int orc_correct_j1(const orc_grid* g, double* j1) {
  if (orc_cb_is_yee(g)) return 0;
  int n = g->n1;
  double* re = malloc(sizeof(double) * n);
  double* im = malloc(sizeof(double) * n);
  double* ratio = malloc(sizeof(double) * n);
  double* row = malloc(sizeof(double) * n);
  double csum = 0.0;
  for (int m = 1; m <= g->M; ++m) csum += (2 * m - 1) * g->cB[m - 1];
  for (int m = 0; m < n; ++m) {
    double k1 = 2.0 * M_PI * m / (n * g->dx1);
    double kyee = sin(k1 * g->dx1 / 2.0) / (g->dx1 / 2.0);
    double kb = orc_kspace(g->M, g->cB, k1, g->dx1);
    ratio[m] = (m == 0) ? 1.0 / csum : kyee / kb;
  }
  for (int k = 0; k < g->n3; ++k)
    for (int j = 0; j < g->n2; ++j) {
      for (int i = 0; i < n; ++i) row[i] = j1[at(g, i, j, k)];
      for (int m = 0; m < n; ++m) {
        double sr = 0.0, si = 0.0;
        for (int i = 0; i < n; ++i) {
          double ph = -2.0 * M_PI * (double)((int64_t)m * i % n) / n;
          sr += row[i] * cos(ph);
          si += row[i] * sin(ph);
        }
        re[m] = sr * ratio[m];
        im[m] = si * ratio[m];
      }
      for (int i = 0; i < n; ++i) {
        double s = 0.0;
        for (int m = 0; m < n; ++m) {
          double ph = 2.0 * M_PI * (double)((int64_t)m * i % n) / n;
          s += re[m] * cos(ph) - im[m] * sin(ph);
        }
        j1[at(g, i, j, k)] = s / n;
      }
    }
  free(re); free(im); free(ratio); free(row);
  return 1;
}

/* Discrete divergence with the Ampere operators, [k]_B . E of Eq. (26),
 * evaluated on the nodes: d^B1 E1 + d^Yee2 E2 + d^Yee3 E3. */
void orc_div_e(const orc_grid* g, const orc_fields* F, double* out) {
  for (int k = 0; k < g->n3; ++k)
    for (int j = 0; j < g->n2; ++j)
      for (int i = 0; i < g->n1; ++i)
        out[at(g, i, j, k)] = dB1(g, F->e1, i, j, k) + d2b(g, F->e2, i, j, k) +
                              d3b(g, F->e3, i, j, k);
}

/* Yee divergence of J (the operator of the continuity equation Eq. (24)). */
void orc_div_yee(const orc_grid* g, const double* f1, const double* f2, const double* f3,
                 double* out) {
  for (int k = 0; k < g->n3; ++k)
    for (int j = 0; j < g->n2; ++j)
      for (int i = 0; i < g->n1; ++i) {
        double d1 = (f1[at(g, i, j, k)] - f1[at(g, i - 1, j, k)]) / g->dx1;
        out[at(g, i, j, k)] = d1 + d2b(g, f2, i, j, k) + d3b(g, f3, i, j, k);
      }
}

/* ---------------------------------------------------------------------------
 * Particle shape: quadratic B-spline (Table 1, "quadratic"), used both to
 * interpolate fields and to deposit charge (momentum-conserving pairing,
 * Sec. 3.1.2).  s is the position in units of the node spacing of the
 * component being interpolated (already shifted by 1/2 for staggered nodes).
 * Nearest node i0 = floor(s + 1/2); weights on nodes i0-1, i0, i0+1.
 * ------------------------------------------------------------------------- */
static double bspline2(double d) {
  double a = fabs(d);
  if (a < 0.5) return 0.75 - a * a;
  if (a < 1.5) return 0.5 * (1.5 - a) * (1.5 - a);
  return 0.0;
}

static void shape3(double s, int* i0, double w[3]) {
  int c = (int)floor(s + 0.5);
  *i0 = c;
  for (int l = 0; l < 3; ++l) w[l] = bspline2(s - (c - 1 + l));
}

/* Field gather, App. A Eq. (A.1): every component is interpolated at its own
 * staggered location with the product of 1D quadratic shapes.  B passed here
 * must be the time-centred B^n (Eq. (7)).  out = {E1,E2,E3,B1,B2,B3}. */
void orc_gather(const orc_grid* g, const double* e1, const double* e2, const double* e3,
                const double* b1, const double* b2, const double* b3, const double* xp,
                double out[6]) {
  const double* comp[6] = {e1, e2, e3, b1, b2, b3};
  /* half-integer offsets of each component along x1, x2, x3 */
  static const double off[6][3] = {{0.5, 0.0, 0.0}, {0.0, 0.5, 0.0}, {0.0, 0.0, 0.5},
                                   {0.0, 0.5, 0.5}, {0.5, 0.0, 0.5}, {0.5, 0.5, 0.0}};
  for (int c = 0; c < 6; ++c) {
    int i0, j0, k0 = 0;
    double w1[3], w2[3], w3[3] = {0.0, 1.0, 0.0};
    shape3(xp[0] / g->dx1 - off[c][0], &i0, w1);
    shape3(xp[1] / g->dx2 - off[c][1], &j0, w2);
    if (g->ndim == 3) shape3(xp[2] / g->dx3 - off[c][2], &k0, w3);
    double s = 0.0;
    for (int c3 = 0; c3 < 3; ++c3) {
      if (w3[c3] == 0.0) continue;
      for (int c2 = 0; c2 < 3; ++c2)
        for (int c1 = 0; c1 < 3; ++c1)
          s += comp[c][at(g, i0 - 1 + c1, j0 - 1 + c2, k0 - 1 + c3)] * w1[c1] * w2[c2] * w3[c3];
    }
    out[c] = s;
  }
}

/* ---------------------------------------------------------------------------
 * Pushers.  u = gamma*beta, qm = charge/mass (-1 for electrons), fields EB
 * = {E1,E2,E3,B1,B2,B3} at time n.  u is advanced from n-1/2 to n+1/2.
 * ------------------------------------------------------------------------- */

/* Relativistic Boris pusher (Sec. 1; Boris 1970, Birdsall & Langdon): half
 * electric impulse, magnetic rotation with gamma of the half-kicked momentum,
 * second half electric impulse. */
void orc_boris(double qm, double dt, const double EB[6], double u[3]) {
  double h = 0.5 * qm * dt;
  double um[3] = {u[0] + h * EB[0], u[1] + h * EB[1], u[2] + h * EB[2]};
  double gm = sqrt(1.0 + um[0] * um[0] + um[1] * um[1] + um[2] * um[2]);
  double t[3] = {h * EB[3] / gm, h * EB[4] / gm, h * EB[5] / gm};
  double t2 = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
  double s[3] = {2.0 * t[0] / (1.0 + t2), 2.0 * t[1] / (1.0 + t2), 2.0 * t[2] / (1.0 + t2)};
  double up[3] = {um[0] + (um[1] * t[2] - um[2] * t[1]), um[1] + (um[2] * t[0] - um[0] * t[2]),
                  um[2] + (um[0] * t[1] - um[1] * t[0])};
  double uq[3] = {um[0] + (up[1] * s[2] - up[2] * s[1]), um[1] + (up[2] * s[0] - up[0] * s[2]),
                  um[2] + (up[0] * s[1] - up[1] * s[0])};
  u[0] = uq[0] + h * EB[0];
  u[1] = uq[1] + h * EB[1];
  u[2] = uq[2] + h * EB[2];
}

/* Higuera-Cary pusher (named in Sec. 1 and used in Sec. 4.1; Higuera & Cary,
 * Phys. Plasmas 24, 052104 (2017)).  Same split as Boris, but the rotation
 * about B uses the Lorentz factor of the mean proper velocity
 * w = (u+ + u-)/2 of the rotation, gbar^2 = 1 + |w|^2.  With
 * beta = (qm dt/2) B, u* = u-.beta and sigma = gm^2 - |beta|^2, the rotation
 * w = u- + w x (beta/gbar) gives |w|^2 = (gbar^2 |u-|^2 + u*^2)/(gbar^2 + |beta|^2),
 * so gbar^2 solves gbar^4 - sigma gbar^2 - (|beta|^2 + u*^2) = 0:
 *   gbar^2 = (sigma + sqrt(sigma^2 + 4 (|beta|^2 + u*^2))) / 2.
 * Then t = beta/gbar, w = (u- + (u-.t) t + u- x t)/(1 + t^2), u+ = w + w x t,
 * and a second half electric impulse. */
void orc_hc(double qm, double dt, const double EB[6], double u[3]) {
  double h = 0.5 * qm * dt;
  double um[3] = {u[0] + h * EB[0], u[1] + h * EB[1], u[2] + h * EB[2]};
  double bt[3] = {h * EB[3], h * EB[4], h * EB[5]};
  double gm2 = 1.0 + um[0] * um[0] + um[1] * um[1] + um[2] * um[2];
  double b2 = bt[0] * bt[0] + bt[1] * bt[1] + bt[2] * bt[2];
  double us = um[0] * bt[0] + um[1] * bt[1] + um[2] * bt[2];
  double sigma = gm2 - b2;
  double gbar = sqrt(0.5 * (sigma + sqrt(sigma * sigma + 4.0 * (b2 + us * us))));
  double t[3] = {bt[0] / gbar, bt[1] / gbar, bt[2] / gbar};
  double t2 = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
  double ut = um[0] * t[0] + um[1] * t[1] + um[2] * t[2];
  double s = 1.0 / (1.0 + t2);
  double w[3] = {s * (um[0] + ut * t[0] + (um[1] * t[2] - um[2] * t[1])),
                 s * (um[1] + ut * t[1] + (um[2] * t[0] - um[0] * t[2])),
                 s * (um[2] + ut * t[2] + (um[0] * t[1] - um[1] * t[0]))};
  double up[3] = {w[0] + (w[1] * t[2] - w[2] * t[1]), w[1] + (w[2] * t[0] - w[0] * t[2]),
                  w[2] + (w[0] * t[1] - w[1] * t[0])};
  u[0] = up[0] + h * EB[0];
  u[1] = up[1] + h * EB[1];
  u[2] = up[2] + h * EB[2];
}

/* Analytic ("exact for constant fields") pusher, Sec. 1 and Sec. 4.1: the
 * paper states what it computes -- the proper-velocity evolution for E, B held
 * constant over the step, mapped from proper to lab time -- and defers the
 * formulas to a separate publication.  Written here from the mathematics:
 *
 *   dU/dtau = L U,  U = (gamma, u),  L = [[0, e^T], [e, -[b]_x]],
 *   e = qm*E, b = qm*B   (du/dtau = gamma e + u x b, dgamma/dtau = e.u).
 *
 * L has eigenvalues +-lE, +-i lB with lE^2 - lB^2 = e^2 - b^2, lE lB = |e.b|,
 * so by Cayley-Hamilton  exp(L tau) = c0 I + c1 L + c2 L^2 + c3 L^3  with
 *   c0 = (lB^2 cosh x + lE^2 cos y)/S,   c1 = (lB^2 sinh x/lE + lE^2 sin y/lB)/S,
 *   c2 = (cosh x - cos y)/S,             c3 = (sinh x/lE - sin y/lB)/S,
 * x = lE tau, y = lB tau, S = lE^2 + lB^2; the lab time elapsed is
 * t(tau) = [int_0^tau exp(L s) ds U]_0 (time component).  The proper time tau*
 * with t(tau*) = dt is found by safeguarded Newton (t' = gamma > 0).  The
 * formulas are evaluated in the forms below, which stay finite for null
 * fields (S -> 0, the plane-wave case) where exp(L tau) = I + L tau + L^2 tau^2/2.
 */

/* h(x) = (cosh x - 1)/x^2,  f(x) = (sinh x - x)/x^3,
 * k(y) = (1 - cos y)/y^2,   g(y) = (y - sin y)/y^3,  X = x^2, Y = y^2. */
static double fn_h(double X) {
  if (X < 1.0) {
    double s = 0.0, t = 0.5;
    for (int n = 0; n < 16; ++n) { s += t; t *= X / ((2 * n + 3) * (2 * n + 4)); }
    return s;
  }
  double x = sqrt(X);
  return (cosh(x) - 1.0) / X;
}
static double fn_k(double Y) {
  if (Y < 1.0) {
    double s = 0.0, t = 0.5;
    for (int n = 0; n < 16; ++n) { s += t; t *= -Y / ((2 * n + 3) * (2 * n + 4)); }
    return s;
  }
  double y = sqrt(Y);
  return (1.0 - cos(y)) / Y;
}
static double fn_f(double X) {
  if (X < 1.0) {
    double s = 0.0, t = 1.0 / 6.0;
    for (int n = 0; n < 16; ++n) { s += t; t *= X / ((2 * n + 4) * (2 * n + 5)); }
    return s;
  }
  double x = sqrt(X);
  return (sinh(x) - x) / (X * x);
}
static double fn_g(double Y) {
  if (Y < 1.0) {
    double s = 0.0, t = 1.0 / 6.0;
    for (int n = 0; n < 16; ++n) { s += t; t *= -Y / ((2 * n + 4) * (2 * n + 5)); }
    return s;
  }
  double y = sqrt(Y);
  return (y - sin(y)) / (Y * y);
}
/* D_hk = (h(x) - k(y)) / (X + Y),  D_fg = (f(x) - g(y)) / (X + Y).
 * For small X+Y the power series of h - k and f - g are divided term by term:
 * (X^n - (-Y)^n)/(X + Y) = sum_{m=0}^{n-1} X^m (-Y)^{n-1-m}. */
static double series_div(double X, double Y, int shift) {
  /* sum_{n>=1} [(X^n - (-Y)^n)/(X+Y)] / (2n+shift)! */
  double s = 0.0, fact = 1.0;
  for (int q = 2; q <= shift; ++q) fact *= q; /* shift! */
  for (int n = 1; n <= 18; ++n) {
    fact *= (2 * n + shift - 1) * (2 * n + shift);
    double geo = 0.0, xm = 1.0;
    for (int m = 0; m < n; ++m) {
      geo += xm * pow(-Y, n - 1 - m);
      xm *= X;
    }
    s += geo / fact;
  }
  return s;
}
static double fn_Dhk(double X, double Y) {
  if (X + Y < 2.0) return series_div(X, Y, 2);
  return (fn_h(X) - fn_k(Y)) / (X + Y);
}
static double fn_Dfg(double X, double Y) {
  if (X + Y < 2.0) return series_div(X, Y, 3);
  return (fn_f(X) - fn_g(Y)) / (X + Y);
}

/* Apply L to a four-vector V = (v0, v). */
static void applyL(const double e[3], const double b[3], const double V[4], double out[4]) {
  out[0] = e[0] * V[1] + e[1] * V[2] + e[2] * V[3];
  out[1] = V[0] * e[0] + (V[2] * b[2] - V[3] * b[1]);
  out[2] = V[0] * e[1] + (V[3] * b[0] - V[1] * b[2]);
  out[3] = V[0] * e[2] + (V[1] * b[1] - V[2] * b[0]);
}

typedef struct {
  double lE2, lB2;
  double U[4], LU[4], L2U[4], L3U[4];
} an_ctx;

/* exp(L tau) U and t(tau) for the current invariants. */
static void an_eval(const an_ctx* a, double tau, double Uout[4], double* tlab) {
  double X = a->lE2 * tau * tau, Y = a->lB2 * tau * tau;
  double Dhk = fn_Dhk(X, Y), Dfg = fn_Dfg(X, Y);
  double h = fn_h(X), f = fn_f(X);
  double t2 = tau * tau, t3 = t2 * tau, t4 = t2 * t2;
  double c0 = 1.0 + X * Y * Dhk;
  double c1 = tau * (1.0 + X * Y * Dfg);
  double c2 = t2 * (h - Y * Dhk);
  double c3 = t3 * (f - Y * Dfg);
  for (int m = 0; m < 4; ++m)
    Uout[m] = c0 * a->U[m] + c1 * a->LU[m] + c2 * a->L2U[m] + c3 * a->L3U[m];
  /* integral coefficients: d0 = c1, d1 = tau^2 (h - X D_hk), d2 = c3, d3 = tau^4 D_hk */
  double d1 = t2 * (h - X * Dhk);
  double d3 = t4 * Dhk;
  *tlab = c1 * a->U[0] + d1 * a->LU[0] + c3 * a->L2U[0] + d3 * a->L3U[0];
}

/* Returns the number of Newton/bisection iterations used, or -1 if the
 * iteration did not converge (u is then left unchanged). */
int orc_analytic(double qm, double dt, const double EB[6], double u[3]) {
  an_ctx a;
  double e[3] = {qm * EB[0], qm * EB[1], qm * EB[2]};
  double b[3] = {qm * EB[3], qm * EB[4], qm * EB[5]};
  double e2 = e[0] * e[0] + e[1] * e[1] + e[2] * e[2];
  double b2 = b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
  double eb = e[0] * b[0] + e[1] * b[1] + e[2] * b[2];
  double I1 = e2 - b2;
  double root = sqrt(I1 * I1 + 4.0 * eb * eb);
  /* larger root computed directly, the smaller from lE2 * lB2 = (e.b)^2 */
  if (I1 >= 0.0) {
    a.lE2 = 0.5 * (I1 + root);
    a.lB2 = a.lE2 > 0.0 ? eb * eb / a.lE2 : 0.0;
  } else {
    a.lB2 = 0.5 * (-I1 + root);
    a.lE2 = a.lB2 > 0.0 ? eb * eb / a.lB2 : 0.0;
  }
  double gam = sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
  a.U[0] = gam; a.U[1] = u[0]; a.U[2] = u[1]; a.U[3] = u[2];
  applyL(e, b, a.U, a.LU);
  applyL(e, b, a.LU, a.L2U);
  applyL(e, b, a.L2U, a.L3U);

  /* Newton on t(tau) = dt from tau0 = dt/gamma, bracketed: t is increasing,
   * t(0) = 0, and t(tau) >= ... so tau* lies in (0, hi] once t(hi) >= dt. */
  double lo = 0.0, hi = dt / gam, tau, Ut[4], tl;
  for (int it = 0; it < 200; ++it) {
    an_eval(&a, hi, Ut, &tl);
    if (tl >= dt) break;
    lo = hi;
    hi *= 2.0;
  }
  tau = dt / gam;
  if (tau < lo || tau > hi) tau = 0.5 * (lo + hi);
  int it;
  for (it = 1; it <= 60; ++it) {
    an_eval(&a, tau, Ut, &tl);
    double r = tl - dt;
    if (r > 0.0) hi = tau; else lo = tau;
    double step = r / Ut[0];
    double tn = tau - step;
    if (!(tn > lo && tn < hi)) tn = 0.5 * (lo + hi);
    double dtau = fabs(tn - tau);
    tau = tn;
    if (dtau <= 4.0 * 2.220446049250313e-16 * fabs(tau) ||
        hi - lo <= 4.0 * 2.220446049250313e-16 * hi)
      break;
  }
  if (it > 60) return -1;
  an_eval(&a, tau, Ut, &tl);
  u[0] = Ut[1];
  u[1] = Ut[2];
  u[2] = Ut[3];
  return it;
}

/* ---------------------------------------------------------------------------
 * Esirkepov charge-conserving deposit (Sec. 3.3; Esirkepov 2001) for the
 * quadratic shape.  Current of one particle of weight w (charge density it
 * carries when its shape sums to one) moving from xo to xn during dt, v3 is
 * the out-of-plane velocity used in 2D3V.  The densities W are the textbook
 * decomposition of S(xn) - S(xo); J1 is the running sum along x1, J2 along
 * x2 (and J3 along x3 in 3D), so that rho^{n+1} - rho^n + dt div_Yee J = 0.
 * Adds into F->j1, j2, j3.
 * ------------------------------------------------------------------------- */
static void esirkepov_1d(double so, double sn, int* base, double S0[5], double dS[5]) {
  int io, in;
  double wo[3], wn[3];
  shape3(so, &io, wo);
  shape3(sn, &in, wn);
  *base = io - 2;
  for (int l = 0; l < 5; ++l) S0[l] = 0.0, dS[l] = 0.0;
  for (int l = 0; l < 3; ++l) S0[l + 1] = wo[l];
  double S1[5] = {0, 0, 0, 0, 0};
  int sh = in - io; /* -1, 0 or +1 because a particle moves less than a cell */
  for (int l = 0; l < 3; ++l) S1[l + 1 + sh] = wn[l];
  for (int l = 0; l < 5; ++l) dS[l] = S1[l] - S0[l];
}

int orc_deposit(const orc_grid* g, orc_fields* F, double w, const double xo[3],
                const double xn[3], double v3) {
  double S0a[5], dSa[5], S0b[5], dSb[5], S0c[5] = {0, 0, 1, 0, 0}, dSc[5] = {0, 0, 0, 0, 0};
  int ba, bb, bc = -2;
  double so1 = xo[0] / g->dx1, sn1 = xn[0] / g->dx1;
  double so2 = xo[1] / g->dx2, sn2 = xn[1] / g->dx2;
  if (fabs(sn1 - so1) >= 1.0 || fabs(sn2 - so2) >= 1.0) return -1;
  esirkepov_1d(so1, sn1, &ba, S0a, dSa);
  esirkepov_1d(so2, sn2, &bb, S0b, dSb);
  if (g->ndim == 3) {
    double so3 = xo[2] / g->dx3, sn3 = xn[2] / g->dx3;
    if (fabs(sn3 - so3) >= 1.0) return -1;
    esirkepov_1d(so3, sn3, &bc, S0c, dSc);
  }
  double c1 = -w * g->dx1 / g->dt, c2 = -w * g->dx2 / g->dt, c3 = -w * g->dx3 / g->dt;
  if (g->ndim == 2) {
    /* 2D3V: W1, W2 as in Esirkepov's 2D form, W3 = time-averaged shape */
    for (int b = 0; b < 5; ++b) {
      double run = 0.0;
      for (int a = 0; a < 5; ++a) {
        double W1 = dSa[a] * (S0b[b] + 0.5 * dSb[b]);
        run += c1 * W1;
        if (run != 0.0) F->j1[at(g, ba + a, bb + b, 0)] += run;
      }
    }
    for (int a = 0; a < 5; ++a) {
      double run = 0.0;
      for (int b = 0; b < 5; ++b) {
        double W2 = dSb[b] * (S0a[a] + 0.5 * dSa[a]);
        run += c2 * W2;
        if (run != 0.0) F->j2[at(g, ba + a, bb + b, 0)] += run;
      }
    }
    for (int b = 0; b < 5; ++b)
      for (int a = 0; a < 5; ++a) {
        double W3 = S0a[a] * S0b[b] + 0.5 * dSa[a] * S0b[b] + 0.5 * S0a[a] * dSb[b] +
                    dSa[a] * dSb[b] / 3.0;
        if (W3 != 0.0) F->j3[at(g, ba + a, bb + b, 0)] += w * v3 * W3;
      }
    return 0;
  }
  /* 3D */
  for (int c = 0; c < 5; ++c)
    for (int b = 0; b < 5; ++b) {
      double run = 0.0;
      for (int a = 0; a < 5; ++a) {
        double W1 = dSa[a] * (S0b[b] * S0c[c] + 0.5 * dSb[b] * S0c[c] + 0.5 * S0b[b] * dSc[c] +
                              dSb[b] * dSc[c] / 3.0);
        run += c1 * W1;
        if (run != 0.0) F->j1[at(g, ba + a, bb + b, bc + c)] += run;
      }
    }
  for (int c = 0; c < 5; ++c)
    for (int a = 0; a < 5; ++a) {
      double run = 0.0;
      for (int b = 0; b < 5; ++b) {
        double W2 = dSb[b] * (S0a[a] * S0c[c] + 0.5 * dSa[a] * S0c[c] + 0.5 * S0a[a] * dSc[c] +
                              dSa[a] * dSc[c] / 3.0);
        run += c2 * W2;
        if (run != 0.0) F->j2[at(g, ba + a, bb + b, bc + c)] += run;
      }
    }
  for (int b = 0; b < 5; ++b)
    for (int a = 0; a < 5; ++a) {
      double run = 0.0;
      for (int c = 0; c < 5; ++c) {
        double W3 = dSc[c] * (S0a[a] * S0b[b] + 0.5 * dSa[a] * S0b[b] + 0.5 * S0a[a] * dSb[b] +
                              dSa[a] * dSb[b] / 3.0);
        run += c3 * W3;
        if (run != 0.0) F->j3[at(g, ba + a, bb + b, bc + c)] += run;
      }
    }
  return 0;
}

/* Charge density on the nodes from the quadratic shape. */
void orc_rho(const orc_grid* g, int64_t np, const double* x1, const double* x2,
             const double* x3, const double* w, double* rho) {
  memset(rho, 0, sizeof(double) * ncell(g));
  for (int64_t p = 0; p < np; ++p) {
    int i0, j0, k0 = 0;
    double w1[3], w2[3], w3[3] = {0.0, 1.0, 0.0};
    shape3(x1[p] / g->dx1, &i0, w1);
    shape3(x2[p] / g->dx2, &j0, w2);
    if (g->ndim == 3) shape3(x3[p] / g->dx3, &k0, w3);
    for (int c = 0; c < 3; ++c)
      for (int b = 0; b < 3; ++b)
        for (int a = 0; a < 3; ++a)
          rho[at(g, i0 - 1 + a, j0 - 1 + b, k0 - 1 + c)] += w[p] * w1[a] * w2[b] * w3[c];
  }
}

/* ---------------------------------------------------------------------------
 * Full time step (Sec. 2, Sec. 3.3):
 *   1. B^{n+1/2} = B^{n-1/2} - dt d_E x E^n                 (Eq. (1))
 *   2. Bbar^n = (B^{n-1/2} + B^{n+1/2}) / 2                  (Eq. (7))
 *   3. per particle: gather E^n, Bbar^n at x^n; push u^{n-1/2} -> u^{n+1/2};
 *      x^{n+1} = x^n + dt u^{n+1/2}/gamma^{n+1/2};  Esirkepov J^{n+1/2}
 *      (weight 0 = test particle: pushed, not deposited); periodic wrap
 *   4. J1 <- ([k]_Yee/[k]_B1) J1  (Sec. 3.3; identity when C^B = e_1)
 *   5. E^{n+1} = E^n + dt (d_B x B^{n+1/2} - J)             (Eq. (1))
 * pusher: 0 = Boris, 1 = analytic, 2 = Higuera-Cary.  On return the state is
 * (E^{n+1}, B^{n+1/2}, x^{n+1}, u^{n+1/2}).  Returns 0, or -1 when a particle
 * moved a full cell or more in one step (outside the scheme's validity), or
 * -2 when the analytic pusher failed to converge.
 * ------------------------------------------------------------------------- */
/* Gather, push, move and deposit (into J's current arrays) of particle p, with
 * the energy-gain sums when wl / wd are given.  Returns 0, -1 (moved a cell or
 * more) or -2 (analytic pusher did not converge). */
static int particle_update(const orc_grid* g, const orc_fields* F, orc_fields* J,
                           const double* bb1, const double* bb2, const double* bb3, int64_t p,
                           double* x1, double* x2, double* x3, double* u1, double* u2, double* u3,
                           const double* w, double qm, int pusher, double* wl, double* wd,
                           const double L[3]) {
  int status = 0;
  double xo[3] = {x1[p], x2[p], g->ndim == 3 ? x3[p] : 0.0};
  double EB[6], u[3] = {u1[p], u2[p], u3[p]};
  const double um[3] = {u1[p], u2[p], u3[p]};
  orc_gather(g, F->e1, F->e2, F->e3, bb1, bb2, bb3, xo, EB);
  if (pusher == 1) {
    if (orc_analytic(qm, g->dt, EB, u) < 0) status = -2;
  } else if (pusher == 2) {
    orc_hc(qm, g->dt, EB, u);
  } else {
    orc_boris(qm, g->dt, EB, u);
  }
  double gam = sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
  if (wl || wd) {
    const double gm = sqrt(1.0 + um[0] * um[0] + um[1] * um[1] + um[2] * um[2]);
    double vb[3];
    for (int d = 0; d < 3; ++d) vb[d] = (um[d] + u[d]) / (gm + gam);
    if (wl) wl[p] += qm * g->dt * EB[0] * vb[0];
    if (wd) wd[p] += qm * g->dt * (EB[1] * vb[1] + EB[2] * vb[2]);
  }
  double xn[3] = {xo[0] + g->dt * u[0] / gam, xo[1] + g->dt * u[1] / gam,
                  g->ndim == 3 ? xo[2] + g->dt * u[2] / gam : 0.0};
  if (w[p] != 0.0)
    if (orc_deposit(g, J, w[p], xo, xn, u[2] / gam) < 0) status = -1;
  u1[p] = u[0]; u2[p] = u[1]; u3[p] = u[2];
  x1[p] = xn[0] - L[0] * floor(xn[0] / L[0]);
  x2[p] = xn[1] - L[1] * floor(xn[1] / L[1]);
  if (g->ndim == 3) x3[p] = xn[2] - L[2] * floor(xn[2] / L[2]);
  /* a wrapped value can round to L itself; map it to 0 */
  if (x1[p] >= L[0]) x1[p] = 0.0;
  if (x2[p] >= L[1]) x2[p] = 0.0;
  if (g->ndim == 3 && x3[p] >= L[2]) x3[p] = 0.0;
  return status;
}

int orc_step_gain(const orc_grid* g, orc_fields* F, int64_t np, double* x1, double* x2,
                  double* x3, double* u1, double* u2, double* u3, const double* w, double qm,
                  int pusher, double* wl, double* wd);

int orc_step(const orc_grid* g, orc_fields* F, int64_t np, double* x1, double* x2, double* x3,
             double* u1, double* u2, double* u3, const double* w, double qm, int pusher) {
  return orc_step_gain(g, F, np, x1, x2, x3, u1, u2, u3, w, qm, pusher, NULL, NULL);
}

/* The same step, also adding each particle's work of this step into the
 * energy-gain integrals of Sec. 4.2 when wl / wd are given (NULL: not kept):
 *   W_LWFA += (q/m) dt E1 vbar1,   W_DLA += (q/m) dt (E2 vbar2 + E3 vbar3),
 * i.e. -int v1 E1 dt and -int v_perp . E_perp dt for electrons (q/m = -1), with E
 * the field the push used (E^n at x^n) and the velocity of the step taken as
 * vbar = (u^{n-1/2} + u^{n+1/2}) / (gamma^{n-1/2} + gamma^{n+1/2}). */
int orc_step_gain(const orc_grid* g, orc_fields* F, int64_t np, double* x1, double* x2,
                  double* x3, double* u1, double* u2, double* u3, const double* w, double qm,
                  int pusher, double* wl, double* wd) {
  int64_t n = ncell(g);
  double* bo1 = malloc(sizeof(double) * n);
  double* bo2 = malloc(sizeof(double) * n);
  double* bo3 = malloc(sizeof(double) * n);
  double* bb1 = malloc(sizeof(double) * n);
  double* bb2 = malloc(sizeof(double) * n);
  double* bb3 = malloc(sizeof(double) * n);
  memcpy(bo1, F->b1, sizeof(double) * n);
  memcpy(bo2, F->b2, sizeof(double) * n);
  memcpy(bo3, F->b3, sizeof(double) * n);
  orc_faraday(g, F, g->dt);
  for (int64_t c = 0; c < n; ++c) {
    bb1[c] = 0.5 * (bo1[c] + F->b1[c]);
    bb2[c] = 0.5 * (bo2[c] + F->b2[c]);
    bb3[c] = 0.5 * (bo3[c] + F->b3[c]);
  }
  memset(F->j1, 0, sizeof(double) * n);
  memset(F->j2, 0, sizeof(double) * n);
  memset(F->j3, 0, sizeof(double) * n);
  int status = 0;
  const double L[3] = {g->n1 * g->dx1, g->n2 * g->dx2, g->n3 * g->dx3};
#ifdef _OPENMP
  /* baseline build only (-fopenmp): particles split statically over threads,
   * each depositing into its own current arrays, summed in thread order */
  const int nt = omp_get_max_threads();
  if (nt > 1 && np > 0) {
    double* jp = calloc((size_t)nt * 3 * (size_t)n, sizeof(double));
    int* st = calloc((size_t)nt, sizeof(int));
#pragma omp parallel num_threads(nt)
    {
      const int t = omp_get_thread_num();
      orc_fields J = *F;
      J.j1 = jp + (size_t)t * 3 * n;
      J.j2 = J.j1 + n;
      J.j3 = J.j2 + n;
#pragma omp for schedule(static)
      for (int64_t p = 0; p < np; ++p) {
        const int s1 = particle_update(g, F, &J, bb1, bb2, bb3, p, x1, x2, x3, u1, u2, u3, w, qm,
                                       pusher, wl, wd, L);
        if (s1 < st[t]) st[t] = s1;
      }
    }
    for (int t = 0; t < nt; ++t) {
      const double* a = jp + (size_t)t * 3 * n;
      for (int64_t c = 0; c < n; ++c) {
        F->j1[c] += a[c];
        F->j2[c] += a[n + c];
        F->j3[c] += a[2 * n + c];
      }
      if (st[t] < status) status = st[t];
    }
    free(jp);
    free(st);
  } else
#endif
  for (int64_t p = 0; p < np; ++p) {
    const int s1 = particle_update(g, F, F, bb1, bb2, bb3, p, x1, x2, x3, u1, u2, u3, w, qm, pusher,
                                   wl, wd, L);
    if (s1 < status) status = s1;
  }
  orc_correct_j1(g, F->j1);
  orc_ampere(g, F, g->dt);
  free(bo1); free(bo2); free(bo3); free(bb1); free(bb2); free(bb3);
  return status;
}

/* Time-centred B^n = B^{n-1/2} - (dt/2) d_E x E^n, i.e. the average of
 * Eq. (7), for reading out the state.  Writes into bb1..bb3. */
void orc_bbar(const orc_grid* g, const orc_fields* F, double* bb1, double* bb2, double* bb3) {
  int64_t n = ncell(g);
  orc_fields H = *F;
  H.b1 = bb1; H.b2 = bb2; H.b3 = bb3;
  memcpy(bb1, F->b1, sizeof(double) * n);
  memcpy(bb2, F->b2, sizeof(double) * n);
  memcpy(bb3, F->b3, sizeof(double) * n);
  orc_faraday(g, &H, g->dt); /* B^{n+1/2} */
  for (int64_t c = 0; c < n; ++c) {
    bb1[c] = 0.5 * (F->b1[c] + bb1[c]);
    bb2[c] = 0.5 * (F->b2[c] + bb2[c]);
    bb3[c] = 0.5 * (F->b3[c] + bb3[c]);
  }
}

/* ---------------------------------------------------------------------------
 * Laser load (setup).  Linearly polarised along x2, moving in +x1, defined by
 * its vector potential a(phi) = a0 sin^2(pi phi/L) sin(k0 phi + phase) for
 * 0 < phi < L, phi = x_front - x1 (+ t), a0 = eE/(m omega0 c) (Sec. 1).
 * E2 = -da/dt.  Transverse factor exp(-(x2 - x2c)^2/w0^2) (and x3 in 3D),
 * none when w0 <= 0 (plane wave).  B3^{-1/2} is the discrete forward
 * eigenmode partner of E2^0 per x1-Fourier mode, Eq. (8):
 *   B3~ = ([k]_E1/[omega]_t) E2~ e^{i k dx1/2} e^{i omega dt/2},
 * omega from the discrete dispersion relation Eq. (4) with omega k1 > 0.  The
 * Nyquist mode of B3 is set to zero.  E1, E3, B1, B2 are zero.  The transform
 * is the plain O(n1^2) DFT of the 1D profile (the profile is separable).
 * ------------------------------------------------------------------------- */
static double laser_dadphi(double phi, double a0, double k0, double phase, double Lenv) {
  if (phi <= 0.0 || phi >= Lenv) return 0.0;
  double s = sin(M_PI * phi / Lenv), c = cos(M_PI * phi / Lenv);
  return a0 * (2.0 * s * c * (M_PI / Lenv) * sin(k0 * phi + phase) +
               s * s * k0 * cos(k0 * phi + phase));
}

void orc_laser_profile(const orc_grid* g, double a0, double k0, double phase, double Lenv,
                       double x_front, double* e_prof, double* b_prof) {
  int n = g->n1;
  double L = n * g->dx1;
  for (int i = 0; i < n; ++i) {
    double x = i * g->dx1;
    /* the pulse may wrap around the periodic box: use the image in (x_front - L, x_front] */
    double phi = x_front - x;
    phi -= L * floor(phi / L);
    e_prof[i] = -laser_dadphi(phi, a0, k0, phase, Lenv); /* E2 = -da/dt = -a'(phi) */
  }
  double* re = calloc(n, sizeof(double));
  double* im = calloc(n, sizeof(double));
  for (int m = 0; m < n; ++m) {
    for (int i = 0; i < n; ++i) {
      double ph = -2.0 * M_PI * (double)((int64_t)m * i % n) / n;
      re[m] += e_prof[i] * cos(ph);
      im[m] += e_prof[i] * sin(ph);
    }
  }
  for (int m = 0; m < n; ++m) {
    int ms = (m <= n / 2) ? m : m - n;
    double k1 = 2.0 * M_PI * ms / L;
    double ratio, ph;
    if (ms == 0) {
      ratio = 1.0;
      ph = 0.0;
    } else if (2 * m == n) {
      ratio = 0.0;
      ph = 0.0;
    } else {
      double kE = orc_kspace(g->M, g->cE, k1, g->dx1);
      double kB = orc_kspace(g->M, g->cB, k1, g->dx1);
      double prod = kE * kB;
      double arg = prod > 0.0 ? 0.5 * g->dt * sqrt(prod) : 0.0;
      if (arg > 1.0) arg = 1.0;
      double om = (2.0 / g->dt) * asin(arg) * (k1 > 0 ? 1.0 : -1.0);
      double omt = sin(om * g->dt / 2.0) / (g->dt / 2.0);
      ratio = omt != 0.0 ? kE / omt : 0.0;
      ph = k1 * g->dx1 / 2.0 + om * g->dt / 2.0;
    }
    double r2 = ratio * (re[m] * cos(ph) - im[m] * sin(ph));
    double i2 = ratio * (re[m] * sin(ph) + im[m] * cos(ph));
    re[m] = r2;
    im[m] = i2;
  }
  for (int i = 0; i < n; ++i) {
    double s = 0.0;
    for (int m = 0; m < n; ++m) {
      double ph = 2.0 * M_PI * (double)((int64_t)m * i % n) / n;
      s += re[m] * cos(ph) - im[m] * sin(ph);
    }
    b_prof[i] = s / n;
  }
  free(re);
  free(im);
}

static double gauss_t(double x, double c, double w0) {
  if (w0 <= 0.0) return 1.0;
  double d = (x - c) / w0;
  return exp(-d * d);
}

void orc_laser_load(const orc_grid* g, orc_fields* F, double a0, double k0, double phase,
                    double Lenv, double x_front, double w0, double x2c, double x3c) {
  int64_t n = ncell(g);
  double* ep = malloc(sizeof(double) * g->n1);
  double* bp = malloc(sizeof(double) * g->n1);
  orc_laser_profile(g, a0, k0, phase, Lenv, x_front, ep, bp);
  memset(F->e1, 0, sizeof(double) * n);
  memset(F->e2, 0, sizeof(double) * n);
  memset(F->e3, 0, sizeof(double) * n);
  memset(F->b1, 0, sizeof(double) * n);
  memset(F->b2, 0, sizeof(double) * n);
  memset(F->b3, 0, sizeof(double) * n);
  for (int k = 0; k < g->n3; ++k)
    for (int j = 0; j < g->n2; ++j) {
      /* E2 and B3 both sit at x2 = (j+1/2) dx2, x3 = k dx3 */
      double tr = gauss_t((j + 0.5) * g->dx2, x2c, w0);
      if (g->ndim == 3) tr *= gauss_t(k * g->dx3, x3c, w0);
      for (int i = 0; i < g->n1; ++i) {
        F->e2[at(g, i, j, k)] = ep[i] * tr;
        F->b3[at(g, i, j, k)] = bp[i] * tr;
      }
    }
  free(ep);
  free(bp);
}

/* ---------------------------------------------------------------------------
 * Local forms for very large grids (same definitions, evaluated only where
 * needed).
 * ------------------------------------------------------------------------- */

/* Time-centred B^n at one staggered node (i,j,k) of component c (0..2):
 * B^{n-1/2} - (dt/2) (d_E x E^n)_c, the average of Eq. (7). */
static double bbar_node(const orc_grid* g, const orc_fields* F, int c, int i, int j, int k) {
  double curl;
  if (c == 0) curl = d2f(g, F->e3, i, j, k) - d3f(g, F->e2, i, j, k);
  else if (c == 1) curl = d3f(g, F->e1, i, j, k) - dE1(g, F->e3, i, j, k);
  else curl = dE1(g, F->e2, i, j, k) - d2f(g, F->e1, i, j, k);
  const double* b = c == 0 ? F->b1 : (c == 1 ? F->b2 : F->b3);
  return b[at(g, i, j, k)] - 0.5 * g->dt * curl;
}

/* Gather of E^n and the time-centred B^n at xp (App. A), with B^n formed at the
 * 27 nodes each component needs instead of on the whole grid. */
void orc_gather_centred(const orc_grid* g, const orc_fields* F, const double* xp, double out[6]) {
  static const double off[6][3] = {{0.5, 0.0, 0.0}, {0.0, 0.5, 0.0}, {0.0, 0.0, 0.5},
                                   {0.0, 0.5, 0.5}, {0.5, 0.0, 0.5}, {0.5, 0.5, 0.0}};
  const double* E[3] = {F->e1, F->e2, F->e3};
  for (int c = 0; c < 6; ++c) {
    int i0, j0, k0 = 0;
    double w1[3], w2[3], w3[3] = {0.0, 1.0, 0.0};
    shape3(xp[0] / g->dx1 - off[c][0], &i0, w1);
    shape3(xp[1] / g->dx2 - off[c][1], &j0, w2);
    if (g->ndim == 3) shape3(xp[2] / g->dx3 - off[c][2], &k0, w3);
    double s = 0.0;
    for (int c3 = 0; c3 < 3; ++c3) {
      if (w3[c3] == 0.0) continue;
      for (int c2 = 0; c2 < 3; ++c2)
        for (int c1 = 0; c1 < 3; ++c1) {
          const int i = i0 - 1 + c1, j = j0 - 1 + c2, k = k0 - 1 + c3;
          const double v = c < 3 ? E[c][at(g, i, j, k)] : bbar_node(g, F, c - 3, i, j, k);
          s += v * w1[c1] * w2[c2] * w3[c3];
        }
    }
    out[c] = s;
  }
}

/* B^{n+1/2} at node (i,j,k): Faraday, Eq. (1). */
static void bhalf_node(const orc_grid* g, const orc_fields* F, int i, int j, int k, double b[3]) {
  b[0] = F->b1[at(g, i, j, k)] - g->dt * (d2f(g, F->e3, i, j, k) - d3f(g, F->e2, i, j, k));
  b[1] = F->b2[at(g, i, j, k)] - g->dt * (d3f(g, F->e1, i, j, k) - dE1(g, F->e3, i, j, k));
  b[2] = F->b3[at(g, i, j, k)] - g->dt * (dE1(g, F->e2, i, j, k) - d2f(g, F->e1, i, j, k));
}

/* One field step (Faraday then Ampere, Eq. (1)) at a single cell with J = 0:
 * out = {E1,E2,E3}^{n+1} and {B1,B2,B3}^{n+1/2} at (i,j,k).  Exact wherever the
 * current vanishes. */
void orc_point_update(const orc_grid* g, const orc_fields* F, int i, int j, int k, double out[6]) {
  double bc[3];
  bhalf_node(g, F, i, j, k, bc);
  /* d^B along x1 of B2, B3 at (i,j,k) needs B^{n+1/2} at i+m-1 and i-m */
  double dB3 = 0.0, dB2 = 0.0;
  for (int m = 1; m <= g->M; ++m) {
    double bp[3], bm[3];
    bhalf_node(g, F, i + m - 1, j, k, bp);
    bhalf_node(g, F, i - m, j, k, bm);
    dB3 += g->cB[m - 1] * (bp[2] - bm[2]);
    dB2 += g->cB[m - 1] * (bp[1] - bm[1]);
  }
  dB3 /= g->dx1;
  dB2 /= g->dx1;
  double bj[3], bk[3] = {0, 0, 0};
  bhalf_node(g, F, i, j - 1, k, bj);
  if (g->ndim == 3) bhalf_node(g, F, i, j, k - 1, bk);
  const double d2B3 = (bc[2] - bj[2]) / g->dx2, d2B1 = (bc[0] - bj[0]) / g->dx2;
  const double d3B2 = g->ndim == 3 ? (bc[1] - bk[1]) / g->dx3 : 0.0;
  const double d3B1 = g->ndim == 3 ? (bc[0] - bk[0]) / g->dx3 : 0.0;
  const int64_t q = at(g, i, j, k);
  out[0] = F->e1[q] + g->dt * (d2B3 - d3B2);
  out[1] = F->e2[q] + g->dt * (d3B1 - dB3);
  out[2] = F->e3[q] + g->dt * (dB2 - d2B1);
  out[3] = bc[0];
  out[4] = bc[1];
  out[5] = bc[2];
}
