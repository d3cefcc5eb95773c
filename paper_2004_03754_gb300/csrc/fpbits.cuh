// fpbits.cuh -- FP32 <-> FP64 conversions and the cell floor/fraction split on
// the integer pipe, for the particle kernels.
//
// On this GPU a conversion to or from FP64 is an FP64-pipe instruction (16 SM
// cycles per warp, like a DFMA): measured on the 2D particle kernel, 22 of the 77
// FP64-pipe instructions of a push were conversions.  These forms work on the
// IEEE 754 binary32 / binary64 bit patterns and are branch-free (a predicated
// hardware fallback would still issue on the FP64 pipe), so each is written for
// the operands its call sites can produce.  Each gives the hardware
// conversion's bits on its domain.  The functions also compile for the host
// (portable bit casts), where the tests check them against the compiler's own
// conversions; on the device they use the CUDA bit-cast intrinsics.
#pragma once
#include <stdint.h>
#include <string.h>

#ifdef __CUDACC__
#define PIC_HD __host__ __device__ __forceinline__
#else
#define PIC_HD inline
#endif

namespace pic {

PIC_HD uint64_t f64_bits(double x) {
#ifdef __CUDA_ARCH__
  return (uint64_t)__double_as_longlong(x);
#else
  uint64_t b;
  memcpy(&b, &x, 8);
  return b;
#endif
}
PIC_HD double f64_from_bits(uint64_t b) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)b);
#else
  double x;
  memcpy(&x, &b, 8);
  return x;
#endif
}
PIC_HD double f64_from_hilo(uint32_t hi, uint32_t lo) {
#ifdef __CUDA_ARCH__
  return __hiloint2double((int)hi, (int)lo);
#else
  return f64_from_bits(((uint64_t)hi << 32) | lo);
#endif
}
PIC_HD uint32_t f32_bits(float f) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(f);
#else
  uint32_t b;
  memcpy(&b, &f, 4);
  return b;
#endif
}
PIC_HD float f32_from_bits(uint32_t b) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(b);
#else
  float f;
  memcpy(&f, &b, 4);
  return f;
#endif
}
PIC_HD int clz32(uint32_t v) {  // leading zeros; v != 0
#ifdef __CUDA_ARCH__
  return __clz((int)v);
#else
  return __builtin_clz(v);
#endif
}

// Round-to-nearest-even FP64 -> FP32 for x in [2^-126, 2^128) (positive, result
// normal or, past the largest float, infinity): drop 29 mantissa bits with
// rounding, rebias the exponent 1023 -> 127.  Non-finite x gives a finite or
// negative value, so a Newton step seeded from it stays non-finite.
PIC_HD float narrow_pos(double x) {
  const uint64_t b = f64_bits(x);
  const uint64_t r = b + 0x0fffffffull + ((b >> 29) & 1ull);
  return f32_from_bits((uint32_t)(r >> 29) - (896u << 23));
}

// Round-to-nearest-even FP64 -> FP32 for any sign and |x| in [2^-126, 2^128)
// (as narrow_pos on the magnitude, the sign bit carried over); zero and
// magnitudes below 2^-126 give a zero of the same sign.  For the particle
// kernels' moves, fractions, weights and current factors: none of them needs
// FP32 subnormals (they would change a shape weight by < 1e-38).
PIC_HD float narrow_signed(double x) {
  const uint64_t b = f64_bits(x);
  const uint64_t mag = b & 0x7fffffffffffffffull;
  const uint32_t sign = (uint32_t)(b >> 32) & 0x80000000u;
  const uint64_t r = mag + 0x0fffffffull + ((mag >> 29) & 1ull);
  const uint32_t m = (uint32_t)(r >> 29) - (896u << 23);
  return f32_from_bits(sign | (mag < (897ull << 52) ? 0u : m));
}

// Exact FP32 -> FP64 for a positive normal float (rebias 127 -> 1023).
PIC_HD double widen_pos(float f) {
  const uint32_t b = f32_bits(f);
  return f64_from_hilo((b >> 3) + 0x38000000u, b << 29);
}

// Exact FP32 -> FP64 for every float: normal, zero, subnormal (normalised by
// its leading-zero count), infinity and NaN (returned quiet).
PIC_HD double widen(float f) {
  const uint32_t b = f32_bits(f);
  const uint32_t mag = b & 0x7fffffffu, sign = b & 0x80000000u;
  uint32_t hi, lo;
  if (mag >= 0x00800000u && mag < 0x7f800000u) {
    hi = sign | ((mag >> 3) + 0x38000000u);
    lo = b << 29;
  } else if (mag == 0u) {
    hi = sign;
    lo = 0u;
  } else if (mag >= 0x7f800000u) {
    hi = sign | 0x7ff00000u | ((mag & 0x7fffffu) >> 3) | (mag > 0x7f800000u ? 0x80000u : 0u);
    lo = mag << 29;
  } else {
    const int s = clz32(mag) - 8;               // shift bringing the leading one to bit 23
    const uint32_t m = (mag << s) & 0x7fffffu;
    hi = sign | ((uint32_t)(897 - s) << 20) | (m >> 3);
    lo = m << 29;
  }
  return f64_from_hilo(hi, lo);
}

// floor(c) and c - floor(c) for a cell coordinate c in [0, 2^31), both exact,
// by masking the fraction bits of c (no FP64 floor or conversion).  Positions
// stay in [0, L) (checked on load, wrapped every step, never written after a
// non-finite move), so c = x / dx is always in that range.
PIC_HD int floor_split(double c, double& frac) {
  const int64_t b = (int64_t)f64_bits(c);
  const int e = (int)(b >> 52) - 1023;       // unbiased exponent (c < 1: e < 0)
  const int sh = 52 - (e < 0 ? 0 : (e > 52 ? 52 : e));  // fraction bits of the mantissa
  const int64_t ip = e < 0 ? 0ll : (b & (int64_t)(~0ull << sh));
  frac = c - f64_from_bits((uint64_t)ip);
  const int64_t m = (b & 0x000fffffffffffffll) | 0x0010000000000000ll;
  return e < 0 ? 0 : (int)(m >> sh);
}

// floor(c) for c in [0, 2^31) by the mantissa shift alone (integer pipe)
PIC_HD int floor_pos(double c) {
  const int64_t b = (int64_t)f64_bits(c);
  const int e = (int)(b >> 52) - 1023;
  if (e < 0) return 0;
  const int64_t m = (b & 0x000fffffffffffffll) | 0x0010000000000000ll;
  return (int)(m >> (52 - (e > 52 ? 52 : e)));
}

}  // namespace pic
