// The register-blocked x1 stencils of the field kernels (field_tile.cuh
// x1_stencil: Faraday's d^E and Ampere's d^B with M taps, V outputs per call
// from a window of L values starting D columns before the first output),
// run on the host over every output of a periodic row.  Compiled by nvcc, run
// without a GPU.
//
// Input (argv[1]): int32 n, M, A (1: d^E, 0: d^B), type (0: double, 1: float,
// 2: compensated FP32 pair);
// FP64 row[n], k[M] (the x1 coefficients divided by dx1).
// Output (argv[2]): FP64 out[n], out[i] = the derivative the kernel forms at
// window position i (d^E at i + 1/2 from values at integer nodes, d^B at i from
// values at half nodes).
#include <cstdint>
#include <cstdio>
#include <vector>

#include "field_tile.cuh"

using namespace pic;

template <typename T, int MT, int A>
static void run(const std::vector<double>& row, const std::vector<double>& k, std::vector<double>& out) {
  constexpr int V = VecOf<T>::V;
  constexpr Reach RC(MT, V);
  constexpr int D = A ? RC.DE : RC.DB;
  constexpr int L = A ? RC.LE : RC.LB;
  const int n = (int)row.size();
  T kk[MT] = {};
  for (size_t m = 0; m < k.size() && m < (size_t)MT; ++m) kk[m] = (T)k[m];
  alignas(16) T win[L];
  for (int i0 = 0; i0 < n; i0 += V) {
    for (int t = 0; t < L; ++t) win[t] = (T)row[wrap_index(i0 - D + t, n)];
    T o[V];
    x1_stencil<T, V, MT, D, L, A>(o, win, kk);
    for (int v = 0; v < V && i0 + v < n; ++v) out[i0 + v] = (double)o[v];
  }
}

template <typename T, int A>
static void dispatch(int M, const std::vector<double>& row, const std::vector<double>& k,
                     std::vector<double>& out) {
  if (M <= 8) run<T, 8, A>(row, k, out);
  else if (M <= 16) run<T, 16, A>(row, k, out);
  else run<T, 32, A>(row, k, out);
}

int main(int argc, char** argv) {
  if (argc != 3) return 2;
  FILE* in = std::fopen(argv[1], "rb");
  if (!in) return 2;
  int32_t h[4];
  if (std::fread(h, 4, 4, in) != 4 || h[0] < 1 || h[1] < 1 || h[1] > 32) return 2;
  std::vector<double> row(h[0]), k(h[1]), out(h[0]);
  if (std::fread(row.data(), 8, row.size(), in) != row.size() ||
      std::fread(k.data(), 8, k.size(), in) != k.size())
    return 2;
  std::fclose(in);
  if (h[3] == 2) {
    if (h[2]) dispatch<dfl, 1>(h[1], row, k, out);
    else dispatch<dfl, 0>(h[1], row, k, out);
  } else if (h[3] == 1) {
    if (h[2]) dispatch<float, 1>(h[1], row, k, out);
    else dispatch<float, 0>(h[1], row, k, out);
  } else {
    if (h[2]) dispatch<double, 1>(h[1], row, k, out);
    else dispatch<double, 0>(h[1], row, k, out);
  }
  FILE* o = std::fopen(argv[2], "wb");
  if (!o) return 2;
  std::fwrite(out.data(), 8, out.size(), o);
  std::fclose(o);
  return 0;
}
