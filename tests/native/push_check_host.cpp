// The product's momentum pushers (pushers.cuh: Boris, Higuera-Cary, analytic)
// compiled for the host.  Reads cases from argv[1] -- int32 count, then per case
// int32 pusher (0 Boris, 1 analytic, 2 Higuera-Cary), qm, dt, E1..E3, B1..B3,
// u1..u3 as FP64 -- and writes per case u1..u3 after the push and the analytic
// pusher's iteration count (as FP64) to argv[2].
#include <cstdint>
#include <cstdio>
#include <vector>

#include "pushers.cuh"

int main(int argc, char** argv) {
  if (argc != 3) return 2;
  FILE* in = std::fopen(argv[1], "rb");
  if (!in) return 2;
  int32_t n = 0;
  if (std::fread(&n, 4, 1, in) != 1 || n < 0) return 2;
  std::vector<double> out;
  for (int32_t c = 0; c < n; ++c) {
    int32_t kind = 0;
    double v[11];
    if (std::fread(&kind, 4, 1, in) != 1 || std::fread(v, 8, 11, in) != 11) return 2;
    const double qm = v[0], dt = v[1];
    const double* eb = v + 2;
    double u[3] = {v[8], v[9], v[10]};
    double it = 0;
    if (kind == 0) pic::boris_push<2>(qm, dt, eb, u);
    else if (kind == 2) pic::hc_push<2>(qm, dt, eb, u);
    else it = pic::analytic_push(qm, dt, eb, u);
    out.insert(out.end(), {u[0], u[1], u[2], it});
  }
  std::fclose(in);
  FILE* o = std::fopen(argv[2], "wb");
  if (!o) return 2;
  std::fwrite(out.data(), 8, out.size(), o);
  std::fclose(o);
  return 0;
}
