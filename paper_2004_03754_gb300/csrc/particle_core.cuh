// particle_core.cuh -- per-particle device code shared by the tiled particle
// kernel, the straggler kernel and the persistent ensemble kernel:
//   gather (App. A, quadratic B-spline at each component's staggered node)
//   -> push (Boris or analytic, FP64) -> x^{n+1} = x^n + dt u/gamma (FP64)
//   -> Esirkepov deposit (Sec. 3.3).
// Field access goes through "views" (shared-memory window or global memory with
// periodic wrap) and current accumulation through "accumulators".
#pragma once
#include <math.h>

#include "common.cuh"
#include "field_tile.cuh"
#include "pushers.cuh"

namespace pic {

// Precision of the current deposit for field type T: the field type itself,
// except compensated fields (dfl), whose current is accumulated in FP32 (the
// reduced form's accuracy for plasma currents; test particles deposit nothing).
template <typename T>
struct DepositOf {
  using type = T;
};
template <>
struct DepositOf<dfl> {
  using type = float;
};

// p += v for the current arrays: hardware atomics for float/double; for a
// compensated array an atomic compare-and-swap of the (hi, lo) pair carrying the
// compensated sum (lock-free: a failed swap means another thread's add landed).
template <typename T, typename V>
__device__ __forceinline__ void atomic_acc(T* p, V v) {
  if constexpr (is_dfl<T>::value) {
    unsigned long long* a = reinterpret_cast<unsigned long long*>(p);
    unsigned long long old = *reinterpret_cast<volatile unsigned long long*>(a), seen;
    do {
      seen = old;
      const dfl cur(__uint_as_float((unsigned)(seen & 0xffffffffull)),
                    __uint_as_float((unsigned)(seen >> 32)));
      const dfl nw = cur + dfl(v);
      const unsigned long long bits =
          (unsigned long long)__float_as_uint(nw.hi) | ((unsigned long long)__float_as_uint(nw.lo) << 32);
      old = atomicCAS(a, seen, bits);
    } while (old != seen);
  } else {
    atomicAdd(p, v);
  }
}

// An FP64 value in the shape/deposit precision D: for FP32 the branch-free
// integer-pipe narrowing (the FP64 pipe carries the push, not conversions)
template <typename D>
PIC_HD D to_prec(double x) {
  return (D)x;
}
template <>
PIC_HD float to_prec<float>(double x) {
  return narrow_signed(x);
}

template <typename T>
struct SmemView {
  const T* p;
  int s2, s3, off1;
  __device__ __forceinline__ T at(int l1, int l2, int l3) const {
    return p[l1 + off1 + l2 * s2 + l3 * s3];
  }
};

template <typename T, bool CG = false>
struct GlobView {
  const T* p;
  int n1, n2, n3;
  int ld;  // row pitch (values), >= n1
  __device__ __forceinline__ T at(int l1, int l2, int l3) const {
    return gload<CG>(p + ((int64_t)wrap_index(l3, n3) * n2 + wrap_index(l2, n2)) * ld +
                     wrap_index(l1, n1));
  }
};

// time-centred B read straight from global memory (straggler path)
template <typename T, int NDIM, bool CG = false>
struct BbarView {
  const T* e[3];
  const T* b;
  int comp;
  int n1, n2, n3;
  const StencilArgs<T>* s;
  int pitch;  // row pitch (values), >= n1
  __host__ __device__ __forceinline__ T ld(const T* a, int l1, int l2, int l3) const {
    return gload<CG>(a + ((int64_t)wrap_index(l3, n3) * n2 + wrap_index(l2, n2)) * pitch +
                     wrap_index(l1, n1));
  }
  __host__ __device__ __forceinline__ T at(int l1, int l2, int l3) const {
    T c = 0;
    auto dE1 = [&](const T* a) {
      T acc = 0;
      for (int m = 1; m <= s->M; ++m) acc += s->kE[m - 1] * (ld(a, l1 + m, l2, l3) - ld(a, l1 - m + 1, l2, l3));
      return acc;
    };
    if (comp == 0) {
      c = s->y2 * (ld(e[2], l1, l2 + 1, l3) - ld(e[2], l1, l2, l3));
      if (NDIM == 3) c -= s->y3 * (ld(e[1], l1, l2, l3 + 1) - ld(e[1], l1, l2, l3));
    } else if (comp == 1) {
      c = -dE1(e[2]);
      if (NDIM == 3) c += s->y3 * (ld(e[0], l1, l2, l3 + 1) - ld(e[0], l1, l2, l3));
    } else {
      c = dE1(e[1]) - s->y2 * (ld(e[0], l1, l2 + 1, l3) - ld(e[0], l1, l2, l3));
    }
    return ld(b, l1, l2, l3) - (T)0.5 * c;
  }
};

// Shared-memory current window in fixed point.  On this GPU an FP32 atomic add
// to shared memory runs as a compare-and-swap loop (about ten instructions and
// a round trip per add) while an int32 add is one instruction, so the 2D window
// keeps each component as two int32 sums: a contribution v adds round(v S) to
// hi and the remainder v S - round(v S) (|.| <= 1/2, exact in FP32) times L,
// rounded, to lo.  The value is hi/S + lo/(S L).  S and L are powers of two set
// per tile by fix_scales so that neither sum can overflow; the resolution
// 1/(S L) is far below the FP32 rounding of the value itself, and the sums do
// not depend on the order of the adds.
// v S = ih + il / L + e, |e| <= 1/(2L), for |v S| <= 2^21 and L <= 2^21.
PIC_HD void fix_encode(float v, float S, float L, int& ih, int& il) {
  constexpr float M = 12582912.0f;   // 1.5 * 2^23: x + M rounds x to an integer for |x| < 2^22
  const float m1 = fmaf(v, S, M);
  const float r = fmaf(v, S, -(m1 - M));   // the remainder v S - round(v S), exact
  const float m2 = fmaf(r, L, M);
  ih = (int)(f32_bits(m1) - 0x4B400000u);
  il = (int)(f32_bits(m2) - 0x4B400000u);
}
PIC_HD float fix_decode(int hi, int lo, float invS, float invSL) {
  return fmaf((float)lo, invSL, (float)hi * invS);
}

struct FixAcc {
  int* hi;
  int* lo;
  int s2, s3;
  float S, L;
  __device__ __forceinline__ void add(int l1, int l2, int l3, float v) const {
    const int q = l1 + l2 * s2 + l3 * s3;
    int ih, il;
    fix_encode(v, S, L, ih, il);
    atomicAdd(&hi[q], ih);
    atomicAdd(&lo[q], il);
  }
};

// Scales of FixAcc for a tile of n particles whose contributions are bounded by
// bound in magnitude (each particle adds at most once per node and component):
// S = 2^e with n (bound S + 1/2) < 2^31 and bound S <= 2^21 (the rounding
// trick's range), L = 2^l <= 2^21 with n (L/2 + 1/2) < 2^31.  FP32 arithmetic
// with a factor-2 margin on both limits (one rounding cannot cross them).
PIC_HD void fix_scales(int64_t n, float bound, float& S, float& L) {
  int e = 21;
  if (bound > 0.0f) {
    const float lim = fminf(1073741824.0f / ((float)n * bound), 2097152.0f / bound);
    e = ilogbf(lim);   // floor(log2(lim))
  }
  S = ldexpf(1.0f, e < -100 ? -100 : (e > 100 ? 100 : e));
  int l = 21, cap = 29;
  for (int64_t m = n; m > 1; m >>= 1) --cap;   // cap = 29 - floor(log2 n)
  if (l > cap) l = cap < 0 ? 0 : cap;
  L = ldexpf(1.0f, l);
}

// FP64 form of the fixed-point window: three int32 limbs per node, a + b/L +
// c/L^2 in units of 1/S (S = 2^eS, L = 2^l), each contribution encoded by
// integer operations on its IEEE bits (no FP64 arithmetic: on this GPU FP64
// shared-memory atomic adds are compare-and-swap loops around an FP64 add, on
// the pipe the push needs).  Y = round(|v| S L^2) (half away from zero, with
// the sign of v) splits as Y = a L^2 + b L + c with 0 <= b, c < L.
// fix64_scales: eS, l for a tile of n particles with |v| <= bound: bound S <
// 2^20 and n bound S < 2^30 (so |Y| < 2^62 and n |a| < 2^31), l = min(21,
// 29 - ceil(log2 n)) (n L < 2^31): no limb sum can overflow.  The resolution
// 1/(S L^2) is at most 2^-51 bound for n = 4096.
PIC_HD void fix64_scales(int64_t n, double bound, int& eS, int& l) {
  int cl2n = 0;
  while (((int64_t)1 << cl2n) < n) ++cl2n;   // ceil(log2 n)
  const uint64_t bb = f64_bits(bound) & 0x7fffffffffffffffull;
  const int eb = bb < (1ull << 52) ? -1022 : (int)(bb >> 52) - 1023;   // floor(log2 bound)
  const int e1 = 19 - eb, e2 = 29 - eb - cl2n;
  eS = e1 < e2 ? e1 : e2;
  if (eS > 1000) eS = 1000;
  l = 29 - cl2n;
  if (l > 21) l = 21;
  if (l < 0) l = 0;
}
PIC_HD void fix64_encode(double v, int eS, int l, int& a, int& b, int& c) {
  const uint64_t bits = f64_bits(v);
  const int ex = (int)((bits >> 52) & 0x7ffu);
  int64_t y = 0;
  {
    // |v| = m 2^(e - 1075) with the implicit bit for normal numbers (e = ex), without
    // it for subnormals and zero (e = 1)
    const int64_t m = (int64_t)((bits & 0xfffffffffffffull) | (ex != 0 ? 0x10000000000000ull : 0ull));
    const int sh = (ex != 0 ? ex : 1) - 1075 + eS + 2 * l;   // |v| S L^2 = m 2^sh
    if (sh >= 0) y = m << (sh > 9 ? 9 : sh);   // sh <= 9 for normal |v| <= bound
    else if (sh > -64) y = (m + ((int64_t)1 << (-sh - 1))) >> (-sh);
    if (bits >> 63) y = -y;
  }
  const int64_t mask = ((int64_t)1 << l) - 1;
  c = (int)(y & mask);
  b = (int)((y >> l) & mask);
  a = (int)(y >> (2 * l));
}
// sums of the three limbs back to the value
PIC_HD double fix64_decode(int a, int b, int c, double invS, double invSL, double invSL2) {
  return fma((double)c, invSL2, fma((double)b, invSL, (double)a * invS));
}

struct FixAcc64 {
  int* a;
  int* b;
  int* c;
  int s2, s3;
  int eS, l;
  __device__ __forceinline__ void add(int l1, int l2, int l3, double v) const {
    const int q = l1 + l2 * s2 + l3 * s3;
    int ia, ib, ic;
    fix64_encode(v, eS, l, ia, ib, ic);
    atomicAdd(&a[q], ia);
    atomicAdd(&b[q], ib);
    atomicAdd(&c[q], ic);
  }
};

template <typename T>
struct GlobAcc {
  T* p;
  int n1, n2, n3;
  int ld;  // row pitch (values), >= n1
  __device__ __forceinline__ void add(int l1, int l2, int l3, typename DepositOf<T>::type v) const {
    atomic_acc(&p[((int64_t)wrap_index(l3, n3) * n2 + wrap_index(l2, n2)) * ld + wrap_index(l1, n1)],
               v);
  }
};

// Quadratic B-spline weights around the nearest node, d in [-1/2, 1/2).
template <typename T>
PIC_HD void bspline3(T d, T w[3]) {
  const T a = (T)0.5 - d, b = (T)0.5 + d;
  w[0] = (T)0.5 * a * a;
  w[1] = (T)0.75 - d * d;
  w[2] = (T)0.5 * b * b;
}

// Per-axis interpolation data for a window-local position r (cell units):
// integer-node set (E1 along x2, ...) and half-node set (E1 along x1, ...).
template <typename T>
struct Axis {
  int bn, bh;    // first node of the 3-point stencils
  T wn[3], wh[3];
};

// Position along one axis as integer node li plus fraction f in [0, 1).
template <typename T>
PIC_HD void axis_weights(int li, T f, Axis<T>& a) {
  if (f < (T)0.5) {
    a.bn = li - 1;
    bspline3<T>(f, a.wn);
  } else {
    a.bn = li;
    bspline3<T>(f - (T)1, a.wn);
  }
  a.bh = li - 1;
  bspline3<T>(f - (T)0.5, a.wh);
}

// Gather (App. A): component c sampled at its own staggered node.
// half[c][d] = 1 when component c sits at a half-integer node along axis d.
template <typename T, int NDIM, class VE, class VB>
PIC_HD void gather(const VE* ve, const VB* vb, const Axis<T>* ax, double eb[6]) {
  constexpr int half[6][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {0, 1, 1}, {1, 0, 1}, {1, 1, 0}};
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    const int b1 = half[c][0] ? ax[0].bh : ax[0].bn;
    const int b2 = half[c][1] ? ax[1].bh : ax[1].bn;
    const T* w1 = half[c][0] ? ax[0].wh : ax[0].wn;
    const T* w2 = half[c][1] ? ax[1].wh : ax[1].wn;
    T acc = 0;
    if (NDIM == 3) {
      const int b3 = half[c][2] ? ax[2].bh : ax[2].bn;
      const T* w3 = half[c][2] ? ax[2].wh : ax[2].wn;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        T acc2 = 0;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          T acc1 = 0;
#pragma unroll
          for (int i = 0; i < 3; ++i)
            acc1 += w1[i] * (c < 3 ? ve[c].at(b1 + i, b2 + j, b3 + k) : vb[c - 3].at(b1 + i, b2 + j, b3 + k));
          acc2 += w2[j] * acc1;
        }
        acc += w3[k] * acc2;
      }
    } else {
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        T acc1 = 0;
#pragma unroll
        for (int i = 0; i < 3; ++i)
          acc1 += w1[i] * (c < 3 ? ve[c].at(b1 + i, b2 + j, 0) : vb[c - 3].at(b1 + i, b2 + j, 0));
        acc += w2[j] * acc1;
      }
    }
    if constexpr (is_dfl<T>::value) eb[c] = widen(acc.hi) + widen(acc.lo);
    else if constexpr (sizeof(T) == 4) eb[c] = widen(acc);
    else eb[c] = acc;
  }
}

// Esirkepov shape data on a 4-node window starting at base = min(i_old, i_new) - 1;
// the particle moves from li + f to li + f + delta (|delta| < 1).  na = number of
// nodes the move touches (3 if it stays on the same nearest node, else 4).
template <typename T>
PIC_HD void esir_axis(int li, T f, T delta, int& base, int& na, T S0[4],
                                          T dS[4]) {
  const int h0 = f >= (T)0.5 ? 1 : 0;
  const T t1 = f + delta;
  const int k1 = (int)floor(t1 + (T)0.5);
  const int i0 = li + h0, i1 = li + k1;
  base = (i0 < i1 ? i0 : i1) - 1;
  na = (i0 == i1) ? 3 : 4;
  T w0[3], w1[3];
  bspline3<T>(f - (T)h0, w0);
  bspline3<T>(t1 - (T)k1, w1);
  const bool s0 = i0 > base + 1, s1 = i1 > base + 1;   // shape starts at node 1 (else 0)
  T S1[4];
  S0[0] = s0 ? (T)0 : w0[0];
  S0[1] = s0 ? w0[0] : w0[1];
  S0[2] = s0 ? w0[1] : w0[2];
  S0[3] = s0 ? w0[2] : (T)0;
  S1[0] = s1 ? (T)0 : w1[0];
  S1[1] = s1 ? w1[0] : w1[1];
  S1[2] = s1 ? w1[1] : w1[2];
  S1[3] = s1 ? w1[2] : (T)0;
#pragma unroll
  for (int l = 0; l < 4; ++l) dS[l] = S1[l] - S0[l];
}

// Esirkepov deposit (Sec. 3.3) of one particle moving r0 -> r1 (cell units).
// cf[d] = -w dx_d/dt (running-sum factor), j3f = w v3 (2D out-of-plane current).
template <typename T, int NDIM, class ACC>
PIC_HD void deposit(const ACC* acc, const int* li, const T* f, const T* delta,
                                        const T* cf, T j3f) {
  int b[3], na[3];
  T S0[3][4], dS[3][4];
#pragma unroll
  for (int d = 0; d < NDIM; ++d) esir_axis<T>(li[d], f[d], delta[d], b[d], na[d], S0[d], dS[d]);
  const T third = (T)(1.0 / 3.0);
  // Entries outside a move's na-node footprint are zero: the running sums end
  // at node na-2 and rows/columns >= na carry no shape.
  if constexpr (NDIM == 2) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (j >= na[1]) break;
      const T f2 = S0[1][j] + (T)0.5 * dS[1][j];
      T run = 0;
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        if (i >= na[0] - 1) break;
        run += cf[0] * dS[0][i] * f2;
        acc[0].add(b[0] + i, b[1] + j, 0, run);
      }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if (i >= na[0]) break;
      const T f1 = S0[0][i] + (T)0.5 * dS[0][i];
      T run = 0;
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        if (j >= na[1] - 1) break;
        run += cf[1] * dS[1][j] * f1;
        acc[1].add(b[0] + i, b[1] + j, 0, run);
      }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (j >= na[1]) break;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        if (i >= na[0]) break;
        const T W3 = S0[0][i] * S0[1][j] + (T)0.5 * dS[0][i] * S0[1][j] +
                     (T)0.5 * S0[0][i] * dS[1][j] + third * dS[0][i] * dS[1][j];
        acc[2].add(b[0] + i, b[1] + j, 0, j3f * W3);
      }
    }
  } else {
    // 3D: W_d = dS_d * (S0_a S0_b + dS_a S0_b/2 + S0_a dS_b/2 + dS_a dS_b/3)
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int a = (d + 1) % 3, c = (d + 2) % 3;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (q >= na[c]) break;
#pragma unroll
        for (int p = 0; p < 4; ++p) {
          if (p >= na[a]) break;
          const T pre = S0[a][p] * S0[c][q] + (T)0.5 * dS[a][p] * S0[c][q] +
                        (T)0.5 * S0[a][p] * dS[c][q] + third * dS[a][p] * dS[c][q];
          T run = 0;
#pragma unroll
          for (int m = 0; m < 3; ++m) {
            if (m >= na[d] - 1) break;
            run += cf[d] * dS[d][m] * pre;
            int l[3];
            l[d] = b[d] + m;
            l[a] = b[a] + p;
            l[c] = b[c] + q;
            acc[d].add(l[0], l[1], l[2], run);
          }
        }
      }
    }
  }
}

PIC_HD void latch(unsigned* err, unsigned bit) {
#ifdef __CUDA_ARCH__
  atomicOr(err, bit);
#else
  *err |= bit;
#endif
}

// Push + move of one particle at window-local node li + fraction f per axis.
// PUSH: PIC_BORIS, PIC_ANALYTIC or PIC_HC fixed at compile time, or -1 to follow a.pusher.
// GAIN: also add the step's work into the energy-gain integrals p.wl, p.wd
// (Sec. 4.2): W_LWFA += (q/m) dt E1 vbar1, W_DLA += (q/m) dt E_perp . vbar_perp with
// vbar = (u^{n-1/2} + u^{n+1/2}) / (gamma^{n-1/2} + gamma^{n+1/2}), the velocity for
// which the two add up to the Boris push's energy change exactly.
template <typename T, int NDIM, int PUSH = -1, bool GAIN = false, class VE, class VB, class ACC>
PIC_HD void advance_particle(const VE* ve, const VB* vb, const ACC* acc,
                                                 const PartPtrs& p, int64_t q, const int* li,
                                                 const T* f, const int* gcell, const GridArgs& g,
                                                 const PartArgs& a, unsigned* err) {
  // Newton steps of the FP64 reciprocals: one from the FP32 seed suffices next to
  // FP32 fields; FP64 and compensated fields take two (FP64 accuracy)
  constexpr int NR = std::is_same<T, float>::value ? 1 : 2;
  using D = typename DepositOf<T>::type;
  Axis<T> ax[3];
#pragma unroll
  for (int d = 0; d < NDIM; ++d) axis_weights<T>(li[d], f[d], ax[d]);
  double eb[6];
  gather<T, NDIM>(ve, vb, ax, eb);
  double u[3] = {p.u[0][q], p.u[1][q], p.u[2][q]};
  const double um[3] = {u[0], u[1], u[2]};
  if (PUSH == PIC_ANALYTIC || (PUSH < 0 && a.pusher == PIC_ANALYTIC)) {
    if (analytic_push(a.qm, g.dt, eb, u) < 0) {
      latch(err, ERRBIT_ANALYTIC);
      return;
    }
  } else if (PUSH == PIC_HC || (PUSH < 0 && a.pusher == PIC_HC)) {
    hc_push<NR>(a.qm, g.dt, eb, u);
  } else {
    boris_push<NR>(a.qm, g.dt, eb, u);
  }
  const double gp2 = 1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  const double ig = rsqrt_nr<NR>(gp2);
  const double dtig = g.dt * ig;
  if constexpr (GAIN) {
    const double gm2 = 1.0 + um[0] * um[0] + um[1] * um[1] + um[2] * um[2];
    const double gsum = gm2 * rsqrt_nr<NR>(gm2) + gp2 * ig;   // gamma^{n-1/2} + gamma^{n+1/2}
    const double f = a.qm * g.dt * rcp_nr<NR>(gsum);
    p.wl[q] += f * eb[0] * (um[0] + u[0]);
    p.wd[q] += f * (eb[1] * (um[1] + u[1]) + eb[2] * (um[2] + u[2]));
  }
  // FP32 fields: the move in cells is formed from the narrowed factors, and the
  // FP64 position takes the move as one fused multiply-add per axis.  FP64 and
  // compensated fields: the FP64 move dx, its cells and the position from it.
  constexpr bool F32 = std::is_same<T, float>::value;
  double dx[3];   // the move, FP64 (FP64 and compensated fields)
  T delta[3];     // the move in cells, in the field precision (shape weights)
  bool moved_ok = true;
#pragma unroll
  for (int d = 0; d < NDIM; ++d) {
    if constexpr (F32) {
      delta[d] = to_prec<float>(dtig) * to_prec<float>(u[d]) * to_prec<float>(g.inv_dx[d]);
    } else {
      dx[d] = dtig * u[d];
      if constexpr (is_dfl<T>::value) delta[d] = T(dx[d] * g.inv_dx[d]);
      else delta[d] = dx[d] * g.inv_dx[d];
    }
    moved_ok = moved_ok && (fabs(delta[d]) < (T)1);   // false for NaN as well
  }
  if (!moved_ok) {
    latch(err, isfinite(dtig) ? ERRBIT_MOVE : ERRBIT_NONFINITE);
    return;
  }
  const double w = p.w[q];
  if (f64_bits(w) != 0) {   // weight 0 (a test particle) deposits nothing
    D cf[3], fd[3], dd[3];
    const D wt = to_prec<D>(w);
#pragma unroll
    for (int d = 0; d < NDIM; ++d) {
      cf[d] = -wt * to_prec<D>(g.dx_dt[d]);
      fd[d] = (D)f[d];
      dd[d] = (D)delta[d];
    }
    // w v3 = w u3 / gamma; in FP32 as the product of the narrowed factors
    D v3;
    if constexpr (std::is_same<D, float>::value) v3 = to_prec<D>(u[2]) * to_prec<D>(ig);
    else v3 = to_prec<D>(u[2] * ig);
    deposit<D, NDIM>(acc, li, fd, dd, cf, wt * v3);
  }
  // FP64 position accumulation.  A move is shorter than one cell; the cell the
  // particle lands in, estimated from the fraction and the move, flags the rare
  // steps that cross the box edge, which take the exact periodic wrap.
#pragma unroll
  for (int d = 0; d < NDIM; ++d) {
    double x;
    if constexpr (F32) x = fma(dtig, u[d], p.x[d][q]);
    else x = p.x[d][q] + dx[d];
    const int land = gcell[d] + (int)floorf((float)f[d] + (float)delta[d]);
    if (land <= 0 || land >= g.n[d] - 1) {
      if (x < 0.0) x += g.len[d];
      else if (x >= g.len[d]) x -= g.len[d];
      if (x >= g.len[d]) x = 0.0;
    }
    p.x[d][q] = x;
  }
  p.u[0][q] = u[0];
  p.u[1][q] = u[1];
  p.u[2][q] = u[2];
}


}  // namespace pic
