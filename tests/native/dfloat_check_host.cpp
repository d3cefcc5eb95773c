// The compensated (FP32-pair) arithmetic of the field kernels (csrc/dfloat.cuh)
// run on the host against FP64, which holds every FP32 sum and product exactly:
// prints, for random operands, the largest violation of each property as
// "name value" lines (0 where the property is exact).
#include <cmath>
#include <cstdio>
#include <random>

#include "dfloat.cuh"

using pic::dfl;

static double ulp_half(float h) {
  if (h == 0.0f) return 0.0;
  int e;
  std::frexp((double)h, &e);
  return std::ldexp(1.0, e - 25);   // half an ulp of a float with exponent e
}

int main() {
  std::mt19937_64 g(20040375);
  std::uniform_real_distribution<double> u(-1.0, 1.0);
  std::uniform_int_distribution<int> ex(-20, 20);
  auto rnd = [&]() { return std::ldexp(u(g), ex(g)); };
  double two_sum_exact = 0, two_prod_exact = 0, ctor = 0, add = 0, sub = 0, mul = 0, norm = 0;
  for (int it = 0; it < 2000000; ++it) {
    const float a = (float)rnd(), b = (float)rnd();
    const dfl s = pic::two_sum(a, b);
    two_sum_exact = std::fmax(two_sum_exact, std::fabs(((double)s.hi + (double)s.lo) - ((double)a + (double)b)));
    const float p = pic::mul_rn(a, b);
    const float pe = std::fmaf(a, b, -p);
    two_prod_exact = std::fmax(two_prod_exact, std::fabs(((double)p + (double)pe) - (double)a * (double)b));
    const double X = rnd(), Y = rnd();
    const dfl x(X), y(Y);
    ctor = std::fmax(ctor, std::fabs((double)x - X) / std::fabs(X));
    const double xs = (double)x, ys = (double)y;
    const dfl z = x + y, d = x - y, m = x * y;
    add = std::fmax(add, std::fabs((double)z - (xs + ys)) / (std::fabs(xs) + std::fabs(ys)));
    sub = std::fmax(sub, std::fabs((double)d - (xs - ys)) / (std::fabs(xs) + std::fabs(ys)));
    mul = std::fmax(mul, std::fabs((double)m - xs * ys) / std::fabs(xs * ys));
    for (const dfl* r : {&z, &d, &m})
      if (std::fabs((double)r->lo) > ulp_half(r->hi)) norm = std::fmax(norm, std::fabs((double)r->lo) / ulp_half(r->hi));
  }
  std::printf("two_sum_exact %.17g\ntwo_prod_exact %.17g\nctor %.17g\nadd %.17g\nsub %.17g\nmul %.17g\nnorm %.17g\n",
              two_sum_exact, two_prod_exact, ctor, add, sub, mul, norm);
  return 0;
}
