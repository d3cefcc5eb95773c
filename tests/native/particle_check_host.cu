// One step of the product's particle update (particle_core.cuh: quadratic-spline
// gather of E^n and the time-centred B^n, push, FP64 move, Esirkepov deposit),
// run on the host through plain periodic-array views the way the straggler
// kernel runs it through global memory.  Compiled by nvcc, run without a GPU.
//
// Input (argv[1], little-endian): int32 n1, n2, pusher (0 Boris, 1 analytic,
// 2 Higuera-Cary), fp32 (0: FP64 fields, 1: FP32 fields); FP64 dx1, dx2, dt, qm;
// FP64 E1 E2 E3 Bbar1 Bbar2 Bbar3 (n1*n2 each, x1 fastest); int64 np; FP64
// x1, x2, u1, u2, u3, w (np each).
// Output (argv[2]): FP64 x1, x2, u1, u2, u3 (np each), J1 J2 J3 (n1*n2 each),
// then the latched error word as FP64.
#include <cstdint>
#include <cstdio>
#include <vector>

#include "particle_core.cuh"

using namespace pic;

template <typename T>
struct HostView {
  const T* p;
  int n1, n2;
  __host__ __device__ T at(int l1, int l2, int) const {
    return p[(int64_t)wrap_index(l2, n2) * n1 + wrap_index(l1, n1)];
  }
};

template <typename T>
struct HostAcc {
  T* p;
  int n1, n2;
  __host__ __device__ void add(int l1, int l2, int, T v) const {
    p[(int64_t)wrap_index(l2, n2) * n1 + wrap_index(l1, n1)] += v;
  }
};

template <typename T>
static int run(FILE* in, FILE* out, int n1, int n2, int pusher, double dx1, double dx2, double dt,
               double qm) {
  const int64_t nc = (int64_t)n1 * n2;
  std::vector<double> f64(6 * nc);
  if (std::fread(f64.data(), 8, f64.size(), in) != f64.size()) return 2;
  std::vector<T> f(f64.begin(), f64.end());
  int64_t np = 0;
  if (std::fread(&np, 8, 1, in) != 1 || np < 0) return 2;
  std::vector<double> pd(6 * np);
  if (std::fread(pd.data(), 8, pd.size(), in) != pd.size()) return 2;
  std::vector<T> J(3 * nc, (T)0);
  PartPtrs p{};
  for (int d = 0; d < 2; ++d) p.x[d] = pd.data() + d * np;
  p.x[2] = pd.data();
  for (int c = 0; c < 3; ++c) p.u[c] = pd.data() + (2 + c) * np;
  p.w = pd.data() + 5 * np;
  GridArgs g{};
  g.ndim = 2;
  g.n[0] = n1; g.n[1] = n2; g.n[2] = 1;
  g.dx[0] = dx1; g.dx[1] = dx2; g.dx[2] = 1.0;
  for (int d = 0; d < 3; ++d) {
    g.inv_dx[d] = 1.0 / g.dx[d];
    g.len[d] = g.n[d] * g.dx[d];
    g.dx_dt[d] = g.dx[d] / dt;
  }
  g.dt = dt;
  g.ncell = nc;
  PartArgs a{qm, pusher, np};
  HostView<T> ve[3], vb[3];
  HostAcc<T> acc[3];
  for (int c = 0; c < 3; ++c) {
    ve[c] = HostView<T>{f.data() + c * nc, n1, n2};
    vb[c] = HostView<T>{f.data() + (3 + c) * nc, n1, n2};
    acc[c] = HostAcc<T>{J.data() + c * nc, n1, n2};
  }
  unsigned err = 0;
  for (int64_t q = 0; q < np; ++q) {
    int li[3] = {0, 0, 0};
    T fr[3] = {0, 0, 0};
    for (int d = 0; d < 2; ++d) {
      double frac;
      li[d] = floor_split(p.x[d][q] * g.inv_dx[d], frac);
      fr[d] = (T)frac;
    }
    advance_particle<T, 2>(ve, vb, acc, p, q, li, fr, li, g, a, &err);
  }
  std::vector<double> o(pd.begin(), pd.begin() + 5 * np);
  o.insert(o.end(), J.begin(), J.end());
  o.push_back((double)err);
  std::fwrite(o.data(), 8, o.size(), out);
  return 0;
}

int main(int argc, char** argv) {
  if (argc != 3) return 2;
  FILE* in = std::fopen(argv[1], "rb");
  FILE* out = std::fopen(argv[2], "wb");
  if (!in || !out) return 2;
  int32_t hdr[4];
  double par[4];
  if (std::fread(hdr, 4, 4, in) != 4 || std::fread(par, 8, 4, in) != 4) return 2;
  const int rc = hdr[3] ? run<float>(in, out, hdr[0], hdr[1], hdr[2], par[0], par[1], par[2], par[3])
                        : run<double>(in, out, hdr[0], hdr[1], hdr[2], par[0], par[1], par[2], par[3]);
  std::fclose(in);
  std::fclose(out);
  return rc;
}
