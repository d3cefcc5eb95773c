// Integer-pipe FP32 <-> FP64 helpers of the particle kernels (pushers.cuh)
// against the hardware conversions, on their stated operand domains, over random
// and edge bit patterns.  Every thread touches only its own index < n of the
// input arrays.  Exit status 0 iff no mismatch.
#include <cstdio>
#include <cstdint>
#include <vector>
#include <random>
#include <cuda_runtime.h>
#include "pushers.cuh"

__global__ void check_widen(const uint32_t* in, int n, unsigned long long* bad) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float f = __uint_as_float(in[i]);
  double a = pic::widen(f), b = (double)f;
  bool same = (__double_as_longlong(a) == __double_as_longlong(b)) || (a != a && b != b);
  if (!same) atomicAdd(bad, 1ull);
}
__global__ void check_narrow_pos(const uint64_t* in, int n, unsigned long long* bad) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double x = fabs(__longlong_as_double((long long)in[i]));
  if (!(x >= 0x1.0p-126 && x < 0x1.0p128)) return;
  float a = pic::narrow_pos(x), b = (float)x;
  float y = rsqrtf(b);
  if (y >= 0x1.0p-126f && y < 0x1.0p127f &&
      __double_as_longlong(pic::widen_pos(y)) != __double_as_longlong((double)y))
    atomicAdd(bad, 1ull);
  bool same = (__float_as_uint(a) == __float_as_uint(b)) || (a != a && b != b);
  if (!same) atomicAdd(bad, 1ull);
}
__global__ void check_split(const uint64_t* in, int n, unsigned long long* bad) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double c = fabs(__longlong_as_double((long long)in[i]));
  if (!(c < 2.0e9)) return;
  double fr;
  int k = pic::floor_split(c, fr);
  double fl = floor(c);
  if (k != (int)fl || __double_as_longlong(fr) != __double_as_longlong(c - fl)) atomicAdd(bad, 1ull);
}

int main() {
  const int n = 1 << 22;
  std::mt19937_64 rng(7);
  std::vector<uint32_t> f(n);
  std::vector<uint64_t> d(n), s(n);
  for (int i = 0; i < n; ++i) f[i] = (uint32_t)rng();
  // edges: zeros, smallest/largest normals, subnormals, inf, nan
  uint32_t fe[] = {0u, 0x80000000u, 0x00800000u, 0x80800000u, 0x007fffffu, 0x00000001u,
                   0x7f7fffffu, 0xff7fffffu, 0x7f800000u, 0xff800000u, 0x7fc00000u, 0x3f800000u};
  for (int i = 0; i < 12; ++i) f[i] = fe[i];
  for (int i = 0; i < n; ++i) {
    uint64_t r = rng();
    switch (i % 4) {
      case 0: d[i] = r; break;                                         // any pattern
      case 1: d[i] = (r & 0x800fffffffffffffull) | ((uint64_t)(880 + (r >> 53) % 40) << 52); break;  // near 2^-126
      case 2: d[i] = (r & 0x800fffffffffffffull) | ((uint64_t)(1140 + (r >> 53) % 12) << 52); break; // near 2^128
      default: d[i] = (r & 0x800000001fffffffull) | 0x3ff0000010000000ull | (r & 0x000fffffe0000000ull); break;  // ties
    }
    double c = (double)(r % 5000) + (double)(rng() >> 11) * 0x1.0p-53;
    if (i % 7 == 0) c = (double)(rng() >> 11) * 0x1.0p-53 * 1e-3;
    if (i % 11 == 0) c = (double)(r % 5000);
    s[i] = *(uint64_t*)&c;
  }
  uint64_t de[] = {0ull, 0x8000000000000000ull, 0x3810000000000000ull, 0x380fffffffffffffull,
                   0x47efffffe0000000ull, 0x47effffff0000000ull, 0x47efffffffffffffull,
                   0x47f0000000000000ull, 0x7ff0000000000000ull, 0x7ff8000000000000ull,
                   0x3ff0000010000000ull, 0x3ff0000030000000ull};
  for (int i = 0; i < 12; ++i) d[i] = de[i];
  uint32_t* df; uint64_t *dd, *ds; unsigned long long* bad;
  cudaMalloc(&df, 4ull * n); cudaMalloc(&dd, 8ull * n); cudaMalloc(&ds, 8ull * n);
  cudaMalloc(&bad, 3 * sizeof(unsigned long long));
  cudaMemset(bad, 0, 3 * sizeof(unsigned long long));
  cudaMemcpy(df, f.data(), 4ull * n, cudaMemcpyHostToDevice);
  cudaMemcpy(dd, d.data(), 8ull * n, cudaMemcpyHostToDevice);
  cudaMemcpy(ds, s.data(), 8ull * n, cudaMemcpyHostToDevice);
  int blocks = (n + 255) / 256;
  check_widen<<<blocks, 256>>>(df, n, bad);
  check_narrow_pos<<<blocks, 256>>>(dd, n, bad + 1);
  check_split<<<blocks, 256>>>(ds, n, bad + 2);
  unsigned long long h[3];
  cudaError_t e = cudaMemcpy(h, bad, sizeof h, cudaMemcpyDeviceToHost);
  printf("status %s  mismatches: widen %llu  narrow_pos/widen_pos %llu  floor_split %llu  (of %d each)\n",
         cudaGetErrorString(e), h[0], h[1], h[2], n);
  return (e == cudaSuccess && h[0] == 0 && h[1] == 0 && h[2] == 0) ? 0 : 1;
}
