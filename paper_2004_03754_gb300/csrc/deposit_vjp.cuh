// deposit_vjp.cuh -- reverse mode of the Esirkepov deposit (Sec. 3.3, Eq. (24))
// for the adjoint of depositing particles.
//
// The deposit template of particle_core.cuh (esir_axis + deposit) is run on
// forward-mode dual numbers whose tangents are the particle's start position
// in cells r0, its move in cells delta and (2D) the out-of-plane factor
// w v3.  Every current contribution it adds is dotted with the current's
// adjoint lambda_J at that node, so one pass gives
//   d/d(r0, delta, w v3) of sum_c <lambda_J[c], J_c>
// for the particle: the exact derivative of the same arithmetic the forward
// deposit performs (the quadratic B-spline shapes are C1 in the positions, so
// the node bookkeeping of esir_axis does not break differentiability).
#pragma once
#include <math.h>

#include "common.cuh"
#include "particle_core.cuh"

namespace pic {

// Dual number with N tangents, constructible from int and double so that the
// deposit templates' literals ((T)0.5, (T)h0, T run = 0) work unchanged.
// Comparisons and floor act on the value; floor is a hidden friend so that it
// does not hide ::floor for plain doubles in namespace pic.
template <int N>
struct DualT {
  double v;
  double d[N];
  PIC_HD DualT() : v(0.0) {
#pragma unroll
    for (int i = 0; i < N; ++i) d[i] = 0.0;
  }
  PIC_HD DualT(double x) : v(x) {
#pragma unroll
    for (int i = 0; i < N; ++i) d[i] = 0.0;
  }
  PIC_HD DualT(int x) : v((double)x) {
#pragma unroll
    for (int i = 0; i < N; ++i) d[i] = 0.0;
  }
  friend PIC_HD DualT operator+(const DualT& a, const DualT& b) {
    DualT r(a.v + b.v);
#pragma unroll
    for (int i = 0; i < N; ++i) r.d[i] = a.d[i] + b.d[i];
    return r;
  }
  friend PIC_HD DualT operator-(const DualT& a, const DualT& b) {
    DualT r(a.v - b.v);
#pragma unroll
    for (int i = 0; i < N; ++i) r.d[i] = a.d[i] - b.d[i];
    return r;
  }
  friend PIC_HD DualT operator*(const DualT& a, const DualT& b) {
    DualT r(a.v * b.v);
#pragma unroll
    for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
    return r;
  }
  PIC_HD DualT& operator+=(const DualT& b) {
    v += b.v;
#pragma unroll
    for (int i = 0; i < N; ++i) d[i] += b.d[i];
    return *this;
  }
  friend PIC_HD bool operator>=(const DualT& a, const DualT& b) { return a.v >= b.v; }
  friend PIC_HD bool operator<(const DualT& a, const DualT& b) { return a.v < b.v; }
  friend PIC_HD double floor(const DualT& a) { return ::floor(a.v); }
};

// The deposit's accumulator for the reverse pass: each contribution v added at
// node (l1, l2, l3) of component c adds lambda_J[c](node) * dv into g.
template <int N>
struct AdjointDot {
  const double* lam;   // adjoint of one current component, periodic n1 x n2 x n3 grid
  int n1, n2, n3;
  double* g;           // N tangent sums
  PIC_HD void add(int l1, int l2, int l3, const DualT<N>& v) const {
    const double L =
        lam[((int64_t)wrap_index(l3, n3) * n2 + wrap_index(l2, n2)) * n1 + wrap_index(l1, n1)];
#pragma unroll
    for (int k = 0; k < N; ++k) g[k] += L * v.d[k];
  }
};

// Gradient of sum_c <lam[c], J_c> over the deposit of one particle that starts
// at r0 (cells, global) and moves by delta (cells), with running-sum factors
// cf[d] = -w dx_d/dt and (2D) out-of-plane factor j3f = w v3: returns
// g_r0[d], g_delta[d] and (2D) g_j3f.  lam: the three adjoint component arrays.
template <int NDIM>
PIC_HD void deposit_vjp(const double* const* lam, int n1, int n2, int n3, const double* r0,
                        const double* delta, const double* cf, double j3f, double* g_r0,
                        double* g_delta, double* g_j3f) {
  constexpr int N = 2 * NDIM + 1;
  using D = DualT<N>;
  int li[3] = {0, 0, 0};
  D f[3], dl[3], cfd[3];
#pragma unroll
  for (int d = 0; d < NDIM; ++d) {
    const double fl = ::floor(r0[d]);
    li[d] = (int)fl;
    f[d] = D(r0[d] - fl);
    f[d].d[d] = 1.0;
    dl[d] = D(delta[d]);
    dl[d].d[NDIM + d] = 1.0;
    cfd[d] = D(cf[d]);
  }
  D j3(j3f);
  j3.d[2 * NDIM] = 1.0;
  double gs[N];
#pragma unroll
  for (int k = 0; k < N; ++k) gs[k] = 0.0;
  const AdjointDot<N> acc[3] = {{lam[0], n1, n2, n3, gs}, {lam[1], n1, n2, n3, gs},
                                {lam[2], n1, n2, n3, gs}};
  deposit<D, NDIM>(acc, li, f, dl, cfd, j3);
#pragma unroll
  for (int d = 0; d < NDIM; ++d) {
    g_r0[d] = gs[d];
    g_delta[d] = gs[NDIM + d];
  }
  *g_j3f = gs[2 * NDIM];
}

}  // namespace pic
