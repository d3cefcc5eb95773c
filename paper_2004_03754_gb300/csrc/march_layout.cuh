// march_layout.cuh -- shared-memory layout and work split of the 3D plane-group
// field kernel (field_planes3_kernel): host and device, no CUDA calls, so that
// the launcher, the argument checks and a host test use the same arithmetic.
#pragma once
#include <stdint.h>

#include <algorithm>

#ifdef __CUDACC__
#define PIC_LAYOUT_HD __host__ __device__
#else
#define PIC_LAYOUT_HD
#endif

namespace pic {

// 3D rows of a group of consecutive x3 planes k0 .. k0+P-1 streamed along x2 by
// a CTA of P warps, warp w on plane k0+w.  The group's rows are staged once for
// all its planes, and the Faraday result of plane k feeds Ampere's x3
// difference at plane k+1 through shared memory; only the B1, B2 of plane k0-1
// are recomputed, their columns spread over the warps.
// Stage layout (row t): E1 E2 E3 rows of planes k0-1+pe, pe = 0 .. P (offset
// er(pe, c)) and E1 E2 of plane k0+P (pe = P+1), WE values from column
// i0-DB-DE; B1 B2 of plane k0-1 (pb = 0) and B1 B2 B3 of planes k0-1+pb, pb =
// 1 .. P (offset br(pb, c)), WB values from column i0-DB.  A group with fewer
// than P planes (the last one when P does not divide n3) uses the first of
// these rows.  J is read from global memory into registers (it is used once).
// Per warp, after the NS stages: B^{n+1/2} row t of its plane ([3][WB]) and B1,
// B3 of row t-1 over the strip ([2][SW]); then B1 B2 of plane k0-1, row t
// ([2][WB]).
struct Planes3 {
  int P, WE, WB, SW;
  PIC_LAYOUT_HD int er(int pe, int c) const { return (3 * pe + c) * WE; }
  PIC_LAYOUT_HD int br(int pb, int c) const {
    return (3 * P + 5) * WE + (pb == 0 ? c : 3 * pb - 1 + c) * WB;
  }
  PIC_LAYOUT_HD int stage_elems() const { return (3 * P + 5) * WE + (3 * P + 2) * WB; }
  PIC_LAYOUT_HD int warp_elems() const { return 3 * WB + 2 * SW; }
};

// Shared-memory elements of the plane-group kernel (strip width sw, E / B region
// widths we / wb): one stage, and a CTA's ring of ns stages with the warps'
// B^{n+1/2} rows and the plane-k0-1 B1, B2.
inline int64_t planes3_stage_elems(int P, int sw, int we, int wb) {
  return Planes3{P, we, wb, sw}.stage_elems();
}
inline int64_t planes3_cta_elems(int P, int sw, int we, int wb, int ns) {
  const Planes3 L{P, we, wb, sw};
  return (int64_t)ns * L.stage_elems() + (int64_t)P * L.warp_elems() + 2 * wb;
}

// Rows per item for `cols` item columns on `slots` resident CTAs: the chunking of
// n2 rows that minimises rounds x (rows + 2 staged halo rows).
inline int balanced_rows(int n2, int64_t cols, int64_t slots) {
  int best_r = n2;
  int64_t best = -1;
  for (int chunks = 1; chunks <= std::min(n2, 256); ++chunks) {
    const int r = (n2 + chunks - 1) / chunks;
    const int64_t items = cols * ((n2 + r - 1) / r);
    const int64_t cost = (items + slots - 1) / slots * (r + 2);
    if (best < 0 || cost < best) {
      best = cost;
      best_r = r;
    }
  }
  return best_r;
}

}  // namespace pic
