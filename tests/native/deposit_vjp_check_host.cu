// The reverse-mode deposit of the adjoint (deposit_vjp.cuh: the Esirkepov
// deposit of particle_core.cuh on dual numbers, each contribution dotted with
// the current's adjoint), run on the host.  Compiled by nvcc, run without a GPU.
//
// Input (argv[1], little-endian): int32 n1, n2; FP64 dx1, dx2, dt; FP64 lambda_1,
// lambda_2, lambda_3 (n1*n2 each, x1 fastest); int64 np; per particle FP64 r0_1,
// r0_2 (start in cells), delta_1, delta_2 (move in cells), w, v3.
// Output (argv[2]): per particle FP64 d/dr0_1, d/dr0_2, d/ddelta_1, d/ddelta_2,
// d/d(w v3) of sum_c <lambda_c, J_c>.
#include <cstdint>
#include <cstdio>
#include <vector>

#include "deposit_vjp.cuh"

using namespace pic;

int main(int argc, char** argv) {
  if (argc != 3) return 2;
  FILE* f = fopen(argv[1], "rb");
  if (!f) return 3;
  int32_t n[2];
  double dx[2], dt;
  if (fread(n, 4, 2, f) != 2 || fread(dx, 8, 2, f) != 2 || fread(&dt, 8, 1, f) != 1) return 4;
  const size_t nc = (size_t)n[0] * n[1];
  std::vector<double> lam(3 * nc);
  if (fread(lam.data(), 8, 3 * nc, f) != 3 * nc) return 4;
  int64_t np = 0;
  if (fread(&np, 8, 1, f) != 1) return 4;
  std::vector<double> in(6 * (size_t)np);
  if (fread(in.data(), 8, in.size(), f) != in.size()) return 4;
  fclose(f);
  const double* lp[3] = {lam.data(), lam.data() + nc, lam.data() + 2 * nc};
  std::vector<double> out(5 * (size_t)np);
  for (int64_t q = 0; q < np; ++q) {
    const double* a = &in[6 * q];
    const double r0[2] = {a[0], a[1]}, del[2] = {a[2], a[3]};
    const double w = a[4], v3 = a[5];
    const double cf[2] = {-w * dx[0] / dt, -w * dx[1] / dt};
    double gr[2], gd[2], gj;
    deposit_vjp<2>(lp, n[0], n[1], 1, r0, del, cf, w * v3, gr, gd, &gj);
    double* o = &out[5 * q];
    o[0] = gr[0];
    o[1] = gr[1];
    o[2] = gd[0];
    o[3] = gd[1];
    o[4] = gj;
  }
  FILE* g = fopen(argv[2], "wb");
  if (!g) return 5;
  fwrite(out.data(), 8, out.size(), g);
  fclose(g);
  return 0;
}
