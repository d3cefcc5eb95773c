// The integer-pipe conversions of fpbits.cuh compiled for the host, against the
// compiler's own IEEE conversions and floor(), on each form's stated domain, over
// random and edge bit patterns.  Prints the mismatch counts; exit status 0 iff
// there are none.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <random>

#include "fpbits.cuh"

static uint64_t dbits(double x) {
  uint64_t b;
  std::memcpy(&b, &x, 8);
  return b;
}
static uint32_t fbits(float x) {
  uint32_t b;
  std::memcpy(&b, &x, 4);
  return b;
}

int main() {
  const int n = 1 << 22;
  std::mt19937_64 rng(11);
  long bad_widen = 0, bad_narrow = 0, bad_wpos = 0, bad_split = 0, bad_signed = 0;
  const uint32_t fe[] = {0u, 0x80000000u, 0x00800000u, 0x80800000u, 0x007fffffu, 0x00000001u,
                         0x7f7fffffu, 0xff7fffffu, 0x7f800000u, 0xff800000u, 0x7fc00000u,
                         0x7f800001u, 0x3f800000u};
  for (int i = 0; i < n; ++i) {
    // widen: every float class
    uint32_t fb = (uint32_t)rng();
    if (i < 13) fb = fe[i];
    float f;
    std::memcpy(&f, &fb, 4);
    const double a = pic::widen(f), h = (double)f;
    if (!(dbits(a) == dbits(h) || (a != a && h != h))) ++bad_widen;
    // narrow_pos: positive doubles in [2^-126, 2^128), near both ends and at ties
    const uint64_t r = rng();
    uint64_t db;
    switch (i % 4) {
      case 0: db = (r & 0x000fffffffffffffull) | ((uint64_t)(897 + (r >> 52) % 254) << 52); break;
      case 1: db = (r & 0x000fffffffffffffull) | ((uint64_t)(897 + (r >> 53) % 6) << 52); break;
      case 2: db = (r & 0x000fffffffffffffull) | ((uint64_t)(1144 + (r >> 53) % 7) << 52); break;
      default: db = 0x3ff0000010000000ull | (r & 0x000fffffe0000000ull); break;   // ties
    }
    double x;
    std::memcpy(&x, &db, 8);
    const float nb = pic::narrow_pos(x), nh = (float)x;
    if (fbits(nb) != fbits(nh)) ++bad_narrow;
    // narrow_signed: either sign on the same magnitudes, and zeros
    {
      const double xs = (i & 1) ? -x : x;
      const float sb = pic::narrow_signed(xs), sh = (float)xs;
      if (fbits(sb) != fbits(sh)) ++bad_signed;
      if (i < 2) {
        const double z = i ? -0.0 : 0.0;
        if (fbits(pic::narrow_signed(z)) != fbits((float)z)) ++bad_signed;
      }
    }
    // widen_pos: positive normal floats
    if (nh >= 0x1.0p-126f && nh < 0x1.0p127f && dbits(pic::widen_pos(nh)) != dbits((double)nh))
      ++bad_wpos;
    // floor_split: cell coordinates in [0, 2^31)
    double c = (double)(r % 5000) + (double)(rng() >> 11) * 0x1.0p-53;
    if (i % 7 == 0) c = (double)(rng() >> 11) * 0x1.0p-53 * 1e-3;
    if (i % 11 == 0) c = (double)(r % 5000);
    if (i % 13 == 0) c = (double)(r % 2147483647ull) + 0.25;
    double fr;
    const int k = pic::floor_split(c, fr);
    const double fl = std::floor(c);
    if (k != (int)fl || dbits(fr) != dbits(c - fl)) ++bad_split;
  }
  std::printf("mismatches: widen %ld  narrow_pos %ld  widen_pos %ld  floor_split %ld  "
              "narrow_signed %ld  (of %d each)\n",
              bad_widen, bad_narrow, bad_wpos, bad_split, bad_signed, n);
  return (bad_widen | bad_narrow | bad_wpos | bad_split | bad_signed) ? 1 : 0;
}
