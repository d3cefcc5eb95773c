// Shared-memory layout and row chunking of the 3D plane-group field kernel
// (march_layout.cuh: Planes3, planes3_cta_elems, balanced_rows; field_tile.cuh:
// Reach), compiled by nvcc and run on the host.
//
// stdin, one request per line:
//   L V MT SW P NS   -> "L WE WB DE LE DB LB stage warp cta" then one line per
//                       staged row "E pe c off" / "B pb c off"
//   R n2 cols slots  -> "R r"
#include <cstdint>
#include <cstdio>

#include "field_tile.cuh"
#include "march_layout.cuh"

using namespace pic;

template <int V, int MT>
static void layout(int SW, int P, int NS) {
  constexpr Reach RC(MT, V);
  const int WE = RC.WE(SW, V), WB = RC.WB(SW, V);
  const Planes3 L{P, WE, WB, SW};
  std::printf("L %d %d %d %d %d %d %lld %d %lld\n", WE, WB, RC.DE, RC.LE, RC.DB, RC.LB,
              (long long)planes3_stage_elems(P, SW, WE, WB), L.warp_elems(),
              (long long)planes3_cta_elems(P, SW, WE, WB, NS));
  for (int pe = 0; pe <= P + 1; ++pe)
    for (int c = 0; c < (pe == P + 1 ? 2 : 3); ++c) std::printf("E %d %d %d\n", pe, c, L.er(pe, c));
  for (int pb = 0; pb <= P; ++pb)
    for (int c = 0; c < (pb == 0 ? 2 : 3); ++c) std::printf("B %d %d %d\n", pb, c, L.br(pb, c));
}

template <int V>
static bool by_mt(int MT, int SW, int P, int NS) {
  switch (MT) {
    case 8: layout<V, 8>(SW, P, NS); return true;
    case 16: layout<V, 16>(SW, P, NS); return true;
    case 32: layout<V, 32>(SW, P, NS); return true;
    default: return false;
  }
}

int main() {
  char kind;
  while (std::scanf(" %c", &kind) == 1) {
    if (kind == 'L') {
      int V, MT, SW, P, NS;
      if (std::scanf("%d %d %d %d %d", &V, &MT, &SW, &P, &NS) != 5) return 2;
      const bool ok = V == 4 ? by_mt<4>(MT, SW, P, NS) : (V == 2 ? by_mt<2>(MT, SW, P, NS) : false);
      if (!ok) return 3;
    } else if (kind == 'R') {
      int n2;
      long long cols, slots;
      if (std::scanf("%d %lld %lld", &n2, &cols, &slots) != 3) return 2;
      std::printf("R %d\n", balanced_rows(n2, cols, slots));
    } else {
      return 4;
    }
  }
  return 0;
}
