// correction_host.h -- taps of the x1 current correction (Sec. 3.3, Eq. (23)),
// built on the host once per row length (setup, not timed).
//
// The deposited current satisfies the Yee continuity equation; Gauss's law under
// the Ampere operator d^B needs the x1 current J1' with [k]_B1 J1' = [k]_Yee J1
// per x1-Fourier mode.  On a periodic row of n cells that is a circulant map with
// symbol ratio(k) = [k]_Yee/[k]_B1 (k = 0: the limit 1/sum_j (2j-1) C^B_j), i.e.
// the periodic convolution J1'_i = sum_m g_m J1_{i+m} with g = inverse DFT of the
// ratio.  The ratio is smooth, so the taps decay geometrically down to the
// rounding floor of the DFT sum (~1e-17 max|ratio|); taps below 1e-15 max|ratio|
// are dropped, which moves J1' by ~1e-15 relative.
#pragma once
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "laser_host.h"

namespace pic {

// On success taps[q] = g_{lo+q}, q < taps.size().  False when [k]_B1 vanishes at
// a grid mode (the map is singular).
inline bool inv_circulant_taps(int n, double dx, int M, const double* cB,
                               std::vector<double>& taps, int& lo) {
  double csum = 0;
  for (int j = 1; j <= M; ++j) csum += (2 * j - 1) * cB[j - 1];
  std::vector<double> ratio(n), cosv(n);
  double rmax = 0;
  for (int m = 0; m < n; ++m) {
    const double k = 2.0 * M_PI * m / (n * dx);
    if (m == 0) {
      ratio[m] = 1.0 / csum;
    } else {
      const double kb = host_kspace(M, cB, k, dx);
      if (!(fabs(kb) > 1e-300)) return false;
      ratio[m] = (sin(k * dx / 2.0) / (dx / 2.0)) / kb;
    }
    rmax = std::max(rmax, fabs(ratio[m]));
    cosv[m] = cos(2.0 * M_PI * m / n);
  }
  std::vector<double> gt(n);
  for (int i = 0; i < n; ++i) {
    double s = 0;
    for (int m = 0; m < n; ++m) s += ratio[m] * cosv[(int64_t)m * i % n];
    gt[i] = s / n;
  }
  int L = 0;
  const double thr = 1e-15 * rmax;
  for (int i = 1; i <= n / 2; ++i)
    if (fabs(gt[i]) > thr) L = i;
  taps.clear();
  if (2 * L + 1 < n) {
    lo = -L;
    for (int m = -L; m <= L; ++m) taps.push_back(gt[(m + n) % n]);
  } else {
    lo = -((n - 1) / 2);
    for (int m = lo; m < lo + n; ++m) taps.push_back(gt[((m % n) + n) % n]);
  }
  return true;
}

}  // namespace pic
