// laser_host.h -- host-side x1 profiles of the laser load (setup, not timed).
//
// E2^0 on the integer x1 nodes: E2 = -da/dt = -a'(phi), a(phi) = a0 sin^2(pi phi/L)
// sin(k0 phi + phase) on 0 < phi < L, phi = x_front - x1.  B3^{-1/2} on the
// half nodes is its discrete forward eigenmode partner per x1-Fourier mode,
// Eq. (8): B3~ = ([k]_E1/[omega]_t) E2~ e^{i k dx1/2} e^{i omega dt/2}, omega from
// Eq. (4); the Nyquist mode of B3 is zero.  Plain O(n1^2) DFT with a twiddle
// table; radix-2 FFT for power-of-two rows of 16384 cells or more.
#pragma once
#include <math.h>
#include <stdint.h>

#include <vector>

#include "pic.h"

namespace pic {

inline double host_kspace(int M, const double* c, double k, double dx) {
  double s = 0;
  for (int j = 1; j <= M; ++j) s += c[j - 1] * sin((2 * j - 1) * k * dx / 2.0);
  return s / (dx / 2.0);
}

// In-place complex DFT of length n, a power of two (iterative radix-2
// Cooley-Tukey): x_k <- sum_j x_j e^{sgn 2 pi i j k / n}; cs, sn hold cos and sin
// of 2 pi q / n, q < n.  Rows of other lengths take the plain O(n^2) sums.
inline void fft_pow2(int n, double* re, double* im, int sgn, const double* cs, const double* sn) {
  for (int i = 1, j = 0; i < n; ++i) {   // bit-reversal permutation
    int bit = n >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) {
      const double tr = re[i], ti = im[i];
      re[i] = re[j]; im[i] = im[j];
      re[j] = tr; im[j] = ti;
    }
  }
  for (int len = 2; len <= n; len <<= 1) {
    const int half = len >> 1, step = n / len;
    for (int s0 = 0; s0 < n; s0 += len)
      for (int k = 0; k < half; ++k) {
        const double wr = cs[k * step], wi = sgn * sn[k * step];
        const int a = s0 + k, b = a + half;
        const double xr = re[b] * wr - im[b] * wi, xi = re[b] * wi + im[b] * wr;
        re[b] = re[a] - xr;
        im[b] = im[a] - xi;
        re[a] += xr;
        im[a] += xi;
      }
  }
}

constexpr int kFftMinRow = 16384;

inline void laser_profiles(int n, double dx, double dt, int M, const double* cE, const double* cB,
                           const pic_laser& L, double* ep, double* bp) {
  const double Lbox = n * dx;
  std::vector<double> re(n), im(n), cs(n), sn(n);
  for (int i = 0; i < n; ++i) {
    double phi = L.x_front - i * dx;
    phi -= Lbox * floor(phi / Lbox);
    double v = 0;
    if (phi > 0 && phi < L.L_env) {
      const double s = sin(M_PI * phi / L.L_env), co = cos(M_PI * phi / L.L_env);
      v = L.a0 * (2 * s * co * (M_PI / L.L_env) * sin(L.k0 * phi + L.phase) +
                  s * s * L.k0 * cos(L.k0 * phi + L.phase));
    }
    ep[i] = -v;
    cs[i] = cos(2.0 * M_PI * i / n);
    sn[i] = sin(2.0 * M_PI * i / n);
  }
  // spectrum of the E2 profile: fa + i fb = sum_i ep_i e^{-2 pi i m i / n}
  std::vector<double> fa(n), fb(n);
  // the FFT only where the plain sums get slow (long rows, e.g. the largest
  // allocation-free load); shorter rows keep the plain sums' rounding
  const bool pow2 = (n & (n - 1)) == 0 && n >= kFftMinRow;
  if (pow2) {
    for (int i = 0; i < n; ++i) fa[i] = ep[i], fb[i] = 0.0;
    fft_pow2(n, fa.data(), fb.data(), -1, cs.data(), sn.data());
  } else {
    for (int m = 0; m < n; ++m) {
      double a = 0, b = 0;
      for (int i = 0; i < n; ++i) {
        const int64_t r = (int64_t)m * i % n;
        a += ep[i] * cs[r];
        b -= ep[i] * sn[r];
      }
      fa[m] = a;
      fb[m] = b;
    }
  }
  for (int m = 0; m < n; ++m) {
    const double a = fa[m], b = fb[m];
    const int ms = m <= n / 2 ? m : m - n;
    const double k = 2.0 * M_PI * ms / Lbox;
    double ratio = 0, ph = 0;
    if (ms == 0) {
      ratio = 1.0;
    } else if (2 * m != n) {
      const double kE = host_kspace(M, cE, k, dx), kB = host_kspace(M, cB, k, dx);
      const double prod = kE * kB;
      double arg = prod > 0 ? 0.5 * dt * sqrt(prod) : 0.0;
      if (arg > 1) arg = 1;
      const double om = (2.0 / dt) * asin(arg) * (k > 0 ? 1.0 : -1.0);
      const double wt = sin(om * dt / 2) / (dt / 2);
      ratio = wt != 0 ? kE / wt : 0.0;
      ph = k * dx / 2 + om * dt / 2;
    }
    re[m] = ratio * (a * cos(ph) - b * sin(ph));
    im[m] = ratio * (a * sin(ph) + b * cos(ph));
  }
  if (pow2) {
    fft_pow2(n, re.data(), im.data(), +1, cs.data(), sn.data());
    for (int i = 0; i < n; ++i) bp[i] = re[i] / n;
    return;
  }
  for (int i = 0; i < n; ++i) {
    double s = 0;
    for (int m = 0; m < n; ++m) {
      const int64_t r = (int64_t)m * i % n;
      s += re[m] * cs[r] - im[m] * sn[r];
    }
    bp[i] = s / n;
  }
}

}  // namespace pic
