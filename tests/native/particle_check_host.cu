// One step of the product's particle update (particle_core.cuh: quadratic-spline
// gather of E^n and the time-centred B^n, push, FP64 move, Esirkepov deposit),
// run on the host through plain periodic-array views the way the straggler
// kernel runs it through global memory.  Compiled by nvcc, run without a GPU.
//
// Input (argv[1], little-endian): int32 n1, n2, n3 (1 in 2D), pusher (0 Boris,
// 1 analytic, 2 Higuera-Cary), fp32 (0: FP64 fields, 1: FP32 fields), form (0:
// the time-centred B given; 1: B^{n-1/2} given, the time-centred B formed on the
// fly by BbarView as the straggler and ensemble paths do); FP64 dx1, dx2, dx3,
// dt, qm; with form 1: int32 M, FP64 C^E_1..C^E_M; FP64 E1 E2 E3 and the three B
// components (n1*n2*n3 each, x1 fastest); int64 np; FP64 x1, x2, x3 (3D only),
// u1, u2, u3, w (np each).
// Output (argv[2]): FP64 x1..x_ndim, u1, u2, u3 (np each), J1 J2 J3 (ncell
// each), then the latched error word as FP64.
#include <cstdint>
#include <cstdio>
#include <type_traits>
#include <vector>

#include "particle_core.cuh"

using namespace pic;

template <typename T>
struct HostView {
  const T* p;
  int n1, n2, n3;
  __host__ __device__ T at(int l1, int l2, int l3) const {
    return p[((int64_t)wrap_index(l3, n3) * n2 + wrap_index(l2, n2)) * n1 + wrap_index(l1, n1)];
  }
};

template <typename T>
struct HostAcc {
  T* p;
  int n1, n2, n3;
  __host__ __device__ void add(int l1, int l2, int l3, T v) const {
    p[((int64_t)wrap_index(l3, n3) * n2 + wrap_index(l2, n2)) * n1 + wrap_index(l1, n1)] += v;
  }
};

template <typename T, int NDIM, class VB>
static int run_views(FILE* in, FILE* out, const int* n, int pusher, const double* dx, double dt,
                     double qm, const std::vector<double>& cE) {
  const int64_t nc = (int64_t)n[0] * n[1] * n[2];
  std::vector<double> f64(6 * nc);
  if (std::fread(f64.data(), 8, f64.size(), in) != f64.size()) return 2;
  std::vector<T> f(f64.begin(), f64.end());
  int64_t np = 0;
  if (std::fread(&np, 8, 1, in) != 1 || np < 0) return 2;
  std::vector<double> pd((NDIM + 4) * np);
  if (std::fread(pd.data(), 8, pd.size(), in) != pd.size()) return 2;
  std::vector<T> J(3 * nc, (T)0);
  PartPtrs p{};
  for (int d = 0; d < 3; ++d) p.x[d] = pd.data() + (d < NDIM ? d : 0) * np;
  for (int c = 0; c < 3; ++c) p.u[c] = pd.data() + (NDIM + c) * np;
  p.w = pd.data() + (NDIM + 3) * np;
  GridArgs g{};
  g.ndim = NDIM;
  for (int d = 0; d < 3; ++d) {
    g.n[d] = n[d];
    g.dx[d] = dx[d];
    g.inv_dx[d] = 1.0 / g.dx[d];
    g.len[d] = g.n[d] * g.dx[d];
    g.dx_dt[d] = g.dx[d] / dt;
  }
  g.dt = dt;
  g.ncell = nc;
  PartArgs a{qm, pusher, np};
  HostView<T> ve[3];
  VB vb[3];
  HostAcc<T> acc[3];
  StencilArgs<T> sa{};
  sa.M = (int)cE.size();
  for (size_t j = 0; j < cE.size(); ++j) sa.kE[j] = (T)(dt * cE[j] / dx[0]);
  sa.y2 = (T)(dt / dx[1]);
  sa.y3 = (T)(NDIM == 3 ? dt / dx[2] : 0.0);
  for (int c = 0; c < 3; ++c) {
    ve[c] = HostView<T>{f.data() + c * nc, n[0], n[1], n[2]};
    if constexpr (std::is_same_v<VB, HostView<T>>) {
      vb[c] = VB{f.data() + (3 + c) * nc, n[0], n[1], n[2]};
    } else {
      vb[c] = VB{{f.data(), f.data() + nc, f.data() + 2 * nc}, f.data() + (3 + c) * nc, c,
                 n[0], n[1], n[2], &sa, n[0]};
    }
    acc[c] = HostAcc<T>{J.data() + c * nc, n[0], n[1], n[2]};
  }
  unsigned err = 0;
  for (int64_t q = 0; q < np; ++q) {
    int li[3] = {0, 0, 0};
    T fr[3] = {0, 0, 0};
    for (int d = 0; d < NDIM; ++d) {
      double frac;
      li[d] = floor_split(p.x[d][q] * g.inv_dx[d], frac);
      fr[d] = (T)frac;
    }
    advance_particle<T, NDIM>(ve, vb, acc, p, q, li, fr, li, g, a, &err);
  }
  std::vector<double> o(pd.begin(), pd.begin() + (NDIM + 3) * np);
  o.insert(o.end(), J.begin(), J.end());
  o.push_back((double)err);
  std::fwrite(o.data(), 8, o.size(), out);
  return 0;
}

template <typename T, int NDIM>
static int run(FILE* in, FILE* out, const int* n, int pusher, int form, const double* dx,
               double dt, double qm, const std::vector<double>& cE) {
  if (form)
    return run_views<T, NDIM, BbarView<T, NDIM>>(in, out, n, pusher, dx, dt, qm, cE);
  return run_views<T, NDIM, HostView<T>>(in, out, n, pusher, dx, dt, qm, cE);
}

int main(int argc, char** argv) {
  if (argc != 3) return 2;
  FILE* in = std::fopen(argv[1], "rb");
  FILE* out = std::fopen(argv[2], "wb");
  if (!in || !out) return 2;
  int32_t hdr[6];
  double par[5];
  if (std::fread(hdr, 4, 6, in) != 6 || std::fread(par, 8, 5, in) != 5) return 2;
  std::vector<double> cE;
  if (hdr[5]) {
    int32_t M = 0;
    if (std::fread(&M, 4, 1, in) != 1 || M < 1 || M > PIC_MAX_M) return 2;
    cE.resize(M);
    if (std::fread(cE.data(), 8, M, in) != (size_t)M) return 2;
  }
  const int n[3] = {hdr[0], hdr[1], hdr[2]};
  const bool three = hdr[2] > 1;
  int rc;
  if (hdr[4])
    rc = three ? run<float, 3>(in, out, n, hdr[3], hdr[5], par, par[3], par[4], cE)
               : run<float, 2>(in, out, n, hdr[3], hdr[5], par, par[3], par[4], cE);
  else
    rc = three ? run<double, 3>(in, out, n, hdr[3], hdr[5], par, par[3], par[4], cE)
               : run<double, 2>(in, out, n, hdr[3], hdr[5], par, par[3], par[4], cE);
  std::fclose(in);
  std::fclose(out);
  return rc;
}
