// dfloat.cuh -- compensated single precision: a value held as an unevaluated
// sum hi + lo of two FP32 numbers (|lo| <= ulp(hi)/2 after normalisation), 48
// significant bits, with arithmetic built from FP32 error-free transformations:
//   TwoSum (Knuth): s = fl(a + b) and the exact error e = a + b - s;
//   FastTwoSum (Dekker, for |a| >= |b|);
//   TwoProd with one fused multiply-add: p = fl(a b), e = fma(a, b, -p) exactly.
// Dekker 1971; the "double-single" arithmetic of GPU mixed-precision codes.
// Every operation runs on the FP32 pipe, which on GB300 issues 64 times the FP64
// rate, so the field update keeps close to FP64 accuracy (~2^-48 relative per
// operation) at FP32 arithmetic cost and FP64 storage (8 bytes per value).
//
// Why the fields need it (Sec. 1, Sec. 4.1): an electron co-moving with the
// laser feels E2 - beta1 B3, which cancels to ~E/(2 gamma^2); FP32 rounding of E2
// and B3 (6e-8 relative) is amplified by gamma^2 and breaks the single-electron
// energy beyond a0 ~ 10, while 2^-48 does not up to a0 = 1e4.
//
// Compiles for host and device (host tests run the same arithmetic).  The
// error-free transformations need every rounded product to be rounded on its
// own: a product that feeds TwoSum is formed by mul_rn (never contracted into
// a fused multiply-add with the sum), and the exact product errors use fmaf
// explicitly.  The arithmetic is declared as
// friends of the type (found by argument-dependent lookup only), so that the
// float and double math functions (fabs, fma) stay visible in this namespace.
#pragma once
#include <math.h>

#include <type_traits>

#include "fpbits.cuh"   // PIC_HD

namespace pic {

// fl(a b), never fused with a following addition
PIC_HD float mul_rn(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fmul_rn(a, b);
#else
  return a * b;
#endif
}

struct dfl {
  float hi, lo;
  dfl() = default;
  PIC_HD constexpr dfl(float h, float l) : hi(h), lo(l) {}
  // integer and double constants (T acc = 0, (T)0.5); the double constructor
  // rounds to the nearest pair (exact for constants, folded at compile time)
  template <typename I, typename = typename std::enable_if<std::is_same<I, int>::value>::type>
  PIC_HD constexpr dfl(I v) : hi((float)v), lo((float)((double)v - (double)(float)v)) {}
  PIC_HD constexpr explicit dfl(double v) : hi((float)v), lo((float)(v - (double)(float)v)) {}
  PIC_HD constexpr explicit dfl(float v) : hi(v), lo(0.0f) {}
  PIC_HD explicit operator double() const { return (double)hi + (double)lo; }
  PIC_HD explicit operator float() const { return hi + lo; }

  PIC_HD static dfl two_sum(float a, float b) {
    const float s = a + b;
    const float v = s - a;
    const float e = (a - (s - v)) + (b - v);
    return dfl(s, e);
  }
  PIC_HD static dfl fast_two_sum(float a, float b) {
    const float s = a + b;
    const float e = b - (s - a);
    return dfl(s, e);
  }

  // a + b: TwoSum of the high parts, low parts added, renormalised.  The error
  // is at most a few units of 2^-48 (|a| + |b|).
  friend PIC_HD dfl operator+(dfl a, dfl b) {
    dfl s = two_sum(a.hi, b.hi);
    s.lo += a.lo + b.lo;
    return fast_two_sum(s.hi, s.lo);
  }
  friend PIC_HD dfl operator-(dfl a) { return dfl(-a.hi, -a.lo); }
  friend PIC_HD dfl operator-(dfl a, dfl b) { return a + dfl(-b.hi, -b.lo); }
  // a b: exact product of the high parts plus the two cross terms (the lo*lo
  // term is below 2^-48 of the result), renormalised.
  friend PIC_HD dfl operator*(dfl a, dfl b) {
    const float p = mul_rn(a.hi, b.hi);
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return fast_two_sum(p, e);
  }
  friend PIC_HD dfl& operator+=(dfl& a, dfl b) { return a = a + b; }
  friend PIC_HD dfl& operator-=(dfl& a, dfl b) { return a = a - b; }
  friend PIC_HD dfl& operator*=(dfl& a, dfl b) { return a = a * b; }
  friend PIC_HD bool operator==(dfl a, dfl b) { return a.hi == b.hi && a.lo == b.lo; }
  friend PIC_HD bool operator!=(dfl a, dfl b) { return !(a == b); }
  // ordering of normalised pairs: by hi, ties by lo
  friend PIC_HD bool operator<(dfl a, dfl b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
  friend PIC_HD bool operator>(dfl a, dfl b) { return b < a; }
  friend PIC_HD bool operator<=(dfl a, dfl b) { return !(b < a); }
  friend PIC_HD bool operator>=(dfl a, dfl b) { return !(a < b); }
  friend PIC_HD dfl fabs(dfl a) {
    return (a.hi < 0.0f || (a.hi == 0.0f && a.lo < 0.0f)) ? dfl(-a.hi, -a.lo) : a;
  }
  friend PIC_HD dfl fma(dfl a, dfl b, dfl c) { return a * b + c; }
};

PIC_HD dfl two_sum(float a, float b) { return dfl::two_sum(a, b); }
PIC_HD dfl fast_two_sum(float a, float b) { return dfl::fast_two_sum(a, b); }

// largest integer <= a, as a float (|a| < 2^24)
PIC_HD float floor_df(dfl a) {
  const float f = floorf(a.hi);
  return (f == a.hi && a.lo < 0.0f) ? f - 1.0f : f;
}

template <typename T>
struct is_dfl {
  static constexpr bool value = false;
};
template <>
struct is_dfl<dfl> {
  static constexpr bool value = true;
};

}  // namespace pic
