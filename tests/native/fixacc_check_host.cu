// The fixed-point current window's scale choice and encoding (particle_core.cuh:
// fix_scales, fix_encode), compiled by nvcc and run on the host.
//
// Input (argv[1], little-endian): int64 np; np pairs (int64 n, FP32 bound);
// int64 nv; nv triples (FP32 v, FP32 S, FP32 L); then the FP64 form
// (fix64_scales, fix64_encode): int64 mp; mp pairs (int64 n, FP64 bound); int64
// mv; mv triples (FP64 v, int32 eS, int32 l).
// Output (argv[2]): np pairs (FP32 S, FP32 L), nv pairs (int32 ih, int32 il),
// mp pairs (int32 eS, int32 l), mv triples (int32 a, int32 b, int32 c).
#include <cstdint>
#include <cstdio>
#include <vector>

#include "particle_core.cuh"

using namespace pic;

int main(int argc, char** argv) {
  if (argc != 3) return 2;
  FILE* f = fopen(argv[1], "rb");
  if (!f) return 3;
  int64_t np = 0, nv = 0;
  if (fread(&np, 8, 1, f) != 1) return 4;
  std::vector<int64_t> n(np);
  std::vector<float> bound(np);
  for (int64_t i = 0; i < np; ++i)
    if (fread(&n[i], 8, 1, f) != 1 || fread(&bound[i], 4, 1, f) != 1) return 4;
  if (fread(&nv, 8, 1, f) != 1) return 4;
  std::vector<float> in(3 * (size_t)nv);
  if (fread(in.data(), 4, in.size(), f) != in.size()) return 4;
  int64_t mp = 0, mv = 0;
  if (fread(&mp, 8, 1, f) != 1) return 4;
  std::vector<int64_t> n64(mp);
  std::vector<double> b64(mp);
  for (int64_t i = 0; i < mp; ++i)
    if (fread(&n64[i], 8, 1, f) != 1 || fread(&b64[i], 8, 1, f) != 1) return 4;
  if (fread(&mv, 8, 1, f) != 1) return 4;
  std::vector<double> v64(mv);
  std::vector<int32_t> el(2 * (size_t)mv);
  for (int64_t i = 0; i < mv; ++i)
    if (fread(&v64[i], 8, 1, f) != 1 || fread(&el[2 * i], 4, 2, f) != 2) return 4;
  fclose(f);
  FILE* g = fopen(argv[2], "wb");
  if (!g) return 5;
  for (int64_t i = 0; i < np; ++i) {
    float S, L;
    fix_scales(n[i], bound[i], S, L);
    fwrite(&S, 4, 1, g);
    fwrite(&L, 4, 1, g);
  }
  for (int64_t i = 0; i < nv; ++i) {
    int32_t o[2];
    fix_encode(in[3 * i], in[3 * i + 1], in[3 * i + 2], o[0], o[1]);
    fwrite(o, 4, 2, g);
  }
  for (int64_t i = 0; i < mp; ++i) {
    int32_t o[2];
    fix64_scales(n64[i], b64[i], o[0], o[1]);
    fwrite(o, 4, 2, g);
  }
  for (int64_t i = 0; i < mv; ++i) {
    int32_t o[3];
    fix64_encode(v64[i], el[2 * i], el[2 * i + 1], o[0], o[1], o[2]);
    fwrite(o, 4, 3, g);
  }
  fclose(g);
  return 0;
}
